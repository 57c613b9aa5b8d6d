"""Fused serving: several jobs in the 64-bit lanes of one pool lattice, each
with its own temperature, algorithm, sweep count and random stream.

The bar is bit-exact, against two independent references: the job run on
its own lattice through the ordinary path, and the CPU oracle run of the
job's samples.  Jobs are loaded at different times (so their sweep counters
differ from the pool's), at ragged lane offsets, across two groups, with
more than 64 samples (two segments), and lanes are released and reused.
"""

import numpy as np
import pytest

from oracle import Oracle
from paper_0704_3573_gb300 import serve

pytestmark = pytest.mark.gpu

SEED = 0x0704357300000C00


def _alone(ianus, dim, L, n, seed, algo, beta, sweeps):
    lat = ianus.Lattice(dim=dim, L=L, n_samples=n, n_replicas=1, seed=seed, layout="bits64", series_capacity=1)
    lat.sweep(algo, beta, sweeps)
    sp = lat.spins()[:, 0]
    E, M, _ = lat.measure(overlap=False)
    return sp, E[:, 0, 0], M[:, 0, 0]


def _lanes(pool, where, n):
    """Spins [n, N] and E, M [n] of a segment list [(group, lane0, n_k)]."""
    sp = pool.spins()[:, 0]
    E, M, _ = pool.measure(overlap=False)
    idx = np.concatenate([np.arange(64 * g + l0, 64 * g + l0 + k) for g, l0, k in where])
    assert len(idx) == n
    return sp[idx], E[idx, 0, 0], M[idx, 0, 0]


@pytest.mark.parametrize("dim,L", [(3, 8), (2, 16), (3, 6)])
def test_jobs_in_a_pool_equal_their_own_lattices(ianus, dim, L):
    from paper_0704_3573_gb300 import HEATBATH, METROPOLIS

    pool = ianus.Lattice(dim=dim, L=L, n_samples=3 * 64, n_replicas=1, seed=1, layout="bits64", series_capacity=1)
    # (seed, segments [(group, lane0, n)], algo, beta, sweeps); the 100-sample
    # job takes a full group and 36 lanes of another
    jobs = [
        (SEED + 1, [(0, 0, 5)], METROPOLIS, 0.9, 40),
        (SEED + 2, [(0, 5, 27)], HEATBATH, 1.3, 25),
        (SEED + 3, [(0, 40, 24)], HEATBATH, 0.4, 60),
        (SEED + 4, [(1, 0, 64), (2, 3, 36)], METROPOLIS, 1.7, 33),
        (SEED + 5, [(2, 50, 1)], HEATBATH, 2.5, 57),
    ]
    for seed, where, algo, beta, sweeps in jobs[:3]:
        for k, (g, l0, n) in enumerate(where):
            pool.segment_load(g, l0, n, seed, algo, beta, sweeps, job_group=k)
    pool.sweep_segments(17)  # the later jobs start with different counters
    for seed, where, algo, beta, sweeps in jobs[3:]:
        for k, (g, l0, n) in enumerate(where):
            pool.segment_load(g, l0, n, seed, algo, beta, sweeps, job_group=k)
    pool.sweep_segments(70)  # beyond every request: each job stops at its own count
    for seed, where, algo, beta, sweeps in jobs:
        n = sum(k for _, _, k in where)
        assert pool.segment_state(where[0][0], where[0][1]) == (sweeps, sweeps)
        sp, E, M = _lanes(pool, where, n)
        sa, Ea, Ma = _alone(ianus, dim, L, n, seed, algo, beta, sweeps)
        assert np.array_equal(sp, sa) and np.array_equal(E, Ea) and np.array_equal(M, Ma), (seed, where)
        o = Oracle(dim=dim, L=L, sample_ids=list(range(n)), seed=seed)
        o.sweep(algo, beta, sweeps)
        assert np.array_equal(sp, o.spins()[:, 0]), seed
        Eo, Mo, _ = o.measure()
        assert np.array_equal(E, Eo[:, 0, 0]) and np.array_equal(M, Mo[:, 0, 0])


def test_release_reuse_graphs_and_errors(ianus):
    from paper_0704_3573_gb300 import HEATBATH, METROPOLIS

    def run(graphs):
        pool = ianus.Lattice(dim=3, L=4, n_samples=64, seed=2, layout="bits64", series_capacity=1)
        pool.set_graphs(graphs)
        pool.segment_load(0, 0, 10, SEED + 7, HEATBATH, 1.0, 100)
        pool.segment_load(0, 10, 3, SEED + 8, METROPOLIS, 0.6, 9)
        pool.sweep_segments(9)
        pool.segment_release(0, 10)
        pool.segment_load(0, 10, 20, SEED + 9, METROPOLIS, 1.4, 30)  # reuses the freed lanes
        pool.sweep_segments(30)
        return pool
    a, b = run(True), run(False)
    assert np.array_equal(a.spins(), b.spins())
    sp, E, M = _lanes(a, [(0, 10, 20)], 20)
    sa, Ea, Ma = _alone(ianus, 3, 4, 20, SEED + 9, METROPOLIS, 1.4, 30)
    assert np.array_equal(sp, sa) and np.array_equal(E, Ea)
    sp, _, _ = _lanes(a, [(0, 0, 10)], 10)
    sa, _, _ = _alone(ianus, 3, 4, 10, SEED + 7, HEATBATH, 1.0, 39)
    assert np.array_equal(sp, sa)
    with pytest.raises(ianus.IanusError) as e:
        a.segment_load(0, 5, 10, 1, HEATBATH, 1.0, 10)  # lanes taken
    assert e.value.status == ianus.EINVAL
    with pytest.raises(ianus.IanusError):
        a.sweep(HEATBATH, 1.0, 1)  # a pool is driven by sweep_segments
    with pytest.raises(ianus.IanusError) as e:
        a.get_state()
    assert e.value.status == ianus.EUNSUPPORTED
    two = ianus.Lattice(dim=3, L=4, n_samples=64, n_replicas=2, seed=2, layout="bits64")
    with pytest.raises(ianus.IanusError) as e:
        two.segment_load(0, 0, 4, 1, HEATBATH, 1.0, 10)
    assert e.value.status == ianus.EUNSUPPORTED


@pytest.mark.parametrize("fuse_max_sites", [1 << 16, 100])
def test_fused_server_results_equal_jobs_alone(ianus, fuse_max_sites):
    """Every job of a Poisson stream, fused into pools (and, with a low
    threshold, partly on lattices of its own), equals the job run alone."""
    jobs = serve.job_mix(24, seed=0x0704357300000004, sweep_scale=0.02, min_sweeps=10,
                         L3=(4, 6, 8), L2=(8, 16), max_samples=90)
    jobs = serve.poisson_arrivals(jobs, rate=500.0, seed=3)
    server = serve.FusedServer(mem_budget=64 << 20, groups_per_pool=2, n_streams=3, chunk_sweeps=13,
                               fuse_max_sites=fuse_max_sites, max_solo=4)
    results, stats = server.run(jobs)
    assert stats["jobs"] == len(jobs)
    assert stats["pools"] >= 1
    for r in results:
        E, M = serve.run_alone(r.job)
        assert np.array_equal(r.energy, E), r.job
        assert np.array_equal(r.magnetisation, M), r.job
        assert r.finished >= r.job.arrival
