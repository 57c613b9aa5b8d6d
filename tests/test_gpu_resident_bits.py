"""Resident sweeps of small bit-sliced lattices (k_resident_bits,
k_resident_fused): many sweeps per launch with the lattice in shared
memory.  Every case is compared bit for bit with the oracle and with the
same lattice swept launch by launch (ianus_set_resident off).

Cases span L = 2 to 16 in 3D and up to 64 in 2D (the sizes that fit in a
block's shared memory), one and two replicas, one and several
temperatures, ragged sample counts, both algorithms, measurement cadences
that split the sweeps into blocks of different lengths, runs longer than
one launch (4096 sweeps), and fused serving pools of small jobs.
"""

import numpy as np
import pytest

from oracle import HEATBATH, METROPOLIS, Oracle

pytestmark = pytest.mark.gpu

SEED = 0x0704357300000000 + 900


def _lattice(ianus, dim, L, S, R, K, resident, seed):
    lat = ianus.Lattice(dim=dim, L=L, n_samples=S, n_replicas=R, n_temps=K, seed=seed, layout="bits64")
    lat.set_resident(resident)
    return lat


def _series(lat):
    return [np.asarray(x) for x in lat.series() if x is not None]


@pytest.mark.parametrize("dim,L,S,R,K", [(3, 2, 67, 2, 1), (3, 4, 64, 1, 1), (3, 6, 70, 2, 1), (3, 8, 130, 2, 1),
                                         (3, 12, 64, 1, 1), (3, 16, 100, 2, 1), (3, 16, 64, 1, 1),
                                         (2, 2, 5, 1, 1), (2, 10, 65, 2, 1), (2, 32, 64, 2, 1), (2, 64, 30, 1, 1),
                                         (3, 8, 64, 2, 3), (2, 16, 70, 1, 2)])
def test_resident_bits_equals_oracle_and_eager(ianus, dim, L, S, R, K):
    beta = [0.7 + 0.23 * k for k in range(K)]
    steps = [(HEATBATH, beta, 7, 7), (METROPOLIS, beta, 9, 3), (HEATBATH, beta, 5, 0)]
    res = _lattice(ianus, dim, L, S, R, K, 2, SEED)  # resident wherever it fits
    eag = _lattice(ianus, dim, L, S, R, K, 0, SEED)
    orc = Oracle(dim=dim, L=L, sample_ids=list(range(S)), n_replicas=R, n_temps=K, seed=SEED)
    for algo, b, n, every in steps:
        res.sweep(algo, b, n, measure_every=every)
        eag.sweep(algo, b, n, measure_every=every)
        orc.sweep(algo, b, n, measure_every=every, nthreads=8)
    sp = res.spins()
    assert np.array_equal(sp, orc.spins())
    assert np.array_equal(sp, eag.spins())
    sw, E, M, Q = res.series()
    swo, Eo, Mo, Qo = orc.series()
    assert np.array_equal(sw, swo) and np.array_equal(E, Eo) and np.array_equal(M, Mo)
    if R >= 2:
        assert np.array_equal(Q, Qo)
    for a, b in zip(_series(res), _series(eag)):
        assert np.array_equal(a, b)
    assert res.sweeps == eag.sweeps == 21


def test_resident_bits_longer_than_one_launch(ianus):
    """5000 sweeps without a measurement: two launches (4096 + 904)."""
    res = _lattice(ianus, 2, 4, 64, 2, 1, 2, SEED + 1)
    res.sweep(HEATBATH, 0.8, 5000)
    orc = Oracle(dim=2, L=4, sample_ids=list(range(64)), n_replicas=2, seed=SEED + 1)
    orc.sweep(HEATBATH, 0.8, 5000, nthreads=8)
    assert np.array_equal(res.spins(), orc.spins())
    E, M, Q = res.measure()
    Eo, Mo, Qo = orc.measure()
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo) and np.array_equal(Q, Qo)


def test_resident_bits_is_the_kernel_that_runs(ianus):
    """Under the automatic variant and the default resident mode, a 3D L=8
    lattice of one replica sweeps with the resident kernel (one launch for
    the block of sweeps), an L=32 one does not."""
    prof = pytest.importorskip("torch.profiler")
    import torch

    small = _lattice(ianus, 3, 8, 64, 1, 1, 1, SEED + 2)
    large = _lattice(ianus, 3, 32, 64, 2, 1, 1, SEED + 2)
    small.sweep(HEATBATH, 1.0, 2)
    large.sweep(HEATBATH, 1.0, 2)
    torch.cuda.synchronize()
    with prof.profile(activities=[prof.ProfilerActivity.CUDA]) as p:
        small.sweep(HEATBATH, 1.0, 40)
        torch.cuda.synchronize()
    names = [e.name for e in p.events() if e.device_type == torch.autograd.DeviceType.CUDA]
    if not names:
        pytest.skip("the profiler records no CUDA kernels here")
    assert sum("k_resident_bits" in n for n in names) == 1, names
    with prof.profile(activities=[prof.ProfilerActivity.CUDA]) as p:
        large.sweep(HEATBATH, 1.0, 4)
        torch.cuda.synchronize()
    names = [e.name for e in p.events() if e.device_type == torch.autograd.DeviceType.CUDA]
    assert not any("k_resident" in n for n in names), names


@pytest.mark.parametrize("dim,L", [(3, 8), (2, 16), (3, 4), (2, 64)])
def test_resident_pool_equals_eager_pool_and_oracle(ianus, dim, L):
    """Jobs in the lanes of a pool lattice, swept resident and launch by
    launch: identical lanes and segment counters, and each job's lanes equal
    the oracle's run of that job."""
    jobs = [  # (seed, [(group, lane0, n)], algo, beta, sweeps)
        (SEED + 11, [(0, 0, 5)], METROPOLIS, 0.9, 40),
        (SEED + 12, [(0, 5, 27)], HEATBATH, 1.3, 25),
        (SEED + 13, [(1, 3, 60)], HEATBATH, 0.4, 61),
        (SEED + 14, [(1, 63, 1)], METROPOLIS, 2.2, 7),
    ]
    pools = []
    for resident in (2, 0):
        pool = ianus.Lattice(dim=dim, L=L, n_samples=2 * 64, n_replicas=1, seed=1, layout="bits64",
                             series_capacity=1)
        pool.set_resident(resident)
        for seed, where, algo, beta, sweeps in jobs[:2]:
            for k, (g, l0, n) in enumerate(where):
                pool.segment_load(g, l0, n, seed, algo, beta, sweeps, job_group=k)
        pool.sweep_segments(11)
        for seed, where, algo, beta, sweeps in jobs[2:]:
            for k, (g, l0, n) in enumerate(where):
                pool.segment_load(g, l0, n, seed, algo, beta, sweeps, job_group=k)
        pool.sweep_segments(100)
        pools.append(pool)
    assert np.array_equal(pools[0].spins(), pools[1].spins())
    for seed, where, algo, beta, sweeps in jobs:
        for g, l0, n in where:
            assert pools[0].segment_state(g, l0) == pools[1].segment_state(g, l0)
            assert pools[0].segment_state(g, l0)[0] == sweeps
    sp = pools[0].spins()[:, 0]
    for seed, where, algo, beta, sweeps in jobs:
        n = sum(k for _, _, k in where)
        orc = Oracle(dim=dim, L=L, sample_ids=list(range(n)), n_replicas=1, seed=seed)
        orc.sweep(algo, beta, sweeps, nthreads=8)
        idx = np.concatenate([np.arange(64 * g + l0, 64 * g + l0 + k) for g, l0, k in where])
        assert np.array_equal(sp[idx], orc.spins()[:, 0]), seed
