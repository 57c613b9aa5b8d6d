"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Everything is integer work, so the bar is bit-exact: couplings, initial
states, spins after every sweep, integer energies, magnetisations, overlaps,
PT permutations and acceptance counts.  Sizes span several thread blocks and
ragged tails (odd sample counts crossing the 64-lane and 4-lane packing,
L = 2 where forward and backward neighbours coincide).
"""

import numpy as np
import pytest

import oracle
from oracle import HEATBATH, METROPOLIS, MODEL_ISING, MODEL_POTTS, Oracle

pytestmark = pytest.mark.gpu

SEED = 0x0704357300000000


def _pair(ianus, model="ea", dim=3, L=4, S=1, R=1, K=1, seed=SEED, layout="auto", ferro=False, ids=None):
    variant = 0
    if layout == "bits64-planes":  # bit-sliced kernel with per-lane threshold planes
        layout, variant = "bits64", 1
    elif layout == "bits64-jit":  # kernel specialised at run time for the thresholds
        layout, variant = "bits64", 2
    elif layout == "bits64-queues":  # specialised kernel with per-warp queues
        layout, variant = "bits64", 6
    lat = ianus.Lattice(model=model, dim=dim, L=L, n_samples=S, n_replicas=R, n_temps=K, seed=seed,
                        layout=layout, ferro=ferro, series_capacity=4096)
    if variant:
        lat.set_variant(variant)
    ids = list(range(S)) if ids is None else ids
    orc = Oracle(model=MODEL_ISING if model == "ea" else MODEL_POTTS, dim=dim, L=L, sample_ids=ids,
                 n_replicas=R, n_temps=K, seed=seed, ferro=ferro)
    return lat, orc, ids


@pytest.mark.parametrize("layout", ["i8", "bits64"])
@pytest.mark.parametrize("dim,L,S,R", [(3, 2, 1, 1), (3, 4, 70, 2), (2, 6, 3, 2), (3, 8, 130, 1), (2, 2, 65, 2)])
def test_init_matches_oracle(ianus, layout, dim, L, S, R):
    lat, orc, _ = _pair(ianus, dim=dim, L=L, S=S, R=R, layout=layout)
    assert np.array_equal(lat.couplings(), orc.couplings())
    assert np.array_equal(lat.spins(), orc.spins())


@pytest.mark.parametrize("dim,L,S,R", [(3, 2, 1, 2), (3, 4, 9, 2), (2, 6, 5, 2), (3, 6, 3, 1)])
def test_potts_init_matches_oracle(ianus, dim, L, S, R):
    lat, orc, _ = _pair(ianus, model="potts", dim=dim, L=L, S=S, R=R)
    assert np.array_equal(lat.couplings(), orc.couplings())
    assert np.array_equal(lat.spins(), orc.spins())


CASES = [(3, 2, 1, 1), (3, 4, 3, 2), (2, 4, 65, 1), (3, 6, 70, 2), (2, 8, 2, 2), (3, 8, 1, 1), (2, 2, 5, 2),
         (3, 10, 3, 2), (2, 12, 67, 1)]


@pytest.mark.parametrize("layout", ["i8", "bits64", "bits64-jit", "bits64-queues"])
@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
@pytest.mark.parametrize("dim,L,S,R", CASES)
def test_sweep_bit_exact_every_sweep(ianus, layout, algo, dim, L, S, R):
    lat, orc, _ = _pair(ianus, dim=dim, L=L, S=S, R=R, layout=layout, seed=SEED + 17 * L + S)
    beta = 0.85
    for _ in range(6):
        lat.sweep(algo, beta, 1)
        orc.sweep(algo, beta, 1)
        assert np.array_equal(lat.spins(), orc.spins())
    E, M, Q = lat.measure()
    Eo, Mo, Qo = orc.measure()
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo)
    if R >= 2:
        assert np.array_equal(Q, Qo)


@pytest.mark.parametrize("layout", ["i8", "bits64", "bits64-jit", "bits64-queues"])
def test_series_matches_oracle(ianus, layout):
    lat, orc, _ = _pair(ianus, dim=3, L=6, S=67, R=2, layout=layout)
    lat.sweep(HEATBATH, 1.0, 23, measure_every=5)
    orc.sweep(HEATBATH, 1.0, 23, measure_every=5)
    sw, E, M, Q = lat.series()
    swo, Eo, Mo, Qo = orc.series()
    assert list(sw) == list(swo) == [5, 10, 15, 20]
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo) and np.array_equal(Q, Qo)


@pytest.mark.parametrize("beta", [0.0, 40.0])
def test_extreme_temperatures(ianus, beta):
    """beta = 0 (T_H = 2^31 everywhere, Metropolis always flips) and a
    beta so large that T_M = 0 and T_H reaches 2^32."""
    for layout in ("i8", "bits64", "bits64-jit", "bits64-queues"):
        for algo in (METROPOLIS, HEATBATH):
            lat, orc, _ = _pair(ianus, dim=3, L=4, S=66, R=1, layout=layout)
            lat.sweep(algo, beta, 3)
            orc.sweep(algo, beta, 3)
            assert np.array_equal(lat.spins(), orc.spins()), (layout, algo)


def test_plain_and_bitsliced_agree(ianus):
    """The stream is defined per (sample, slot, site, sweep), not per layout."""
    a = ianus.Lattice(dim=3, L=8, n_samples=40, n_replicas=2, seed=5, layout="i8")
    b = ianus.Lattice(dim=3, L=8, n_samples=40, n_replicas=2, seed=5, layout="bits64")
    for algo in (METROPOLIS, HEATBATH):
        a.sweep(algo, 0.7, 5)
        b.sweep(algo, 0.7, 5)
        assert np.array_equal(a.spins(), b.spins())
        for x, y in zip(a.measure(), b.measure()):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("layout", ["i8", "bits64"])
def test_split_sweeps_and_checkpoint(ianus, layout):
    a = ianus.Lattice(dim=3, L=6, n_samples=5, n_replicas=2, seed=9, layout=layout)
    a.sweep(HEATBATH, 0.9, 7)
    blob = a.get_state()
    a.sweep(HEATBATH, 0.9, 5)
    b = ianus.Lattice(dim=3, L=6, n_samples=5, n_replicas=2, seed=9, layout=layout)
    b.set_state(blob)
    assert b.sweeps == 7
    b.sweep(HEATBATH, 0.9, 2)
    b.sweep(HEATBATH, 0.9, 3)
    assert np.array_equal(a.spins(), b.spins())


@pytest.mark.parametrize("layout", ["i8", "bits64"])
def test_restore_into_a_running_lattice(ianus, layout):
    """A checkpoint restored into the lattice that wrote it, after its
    temperature permutation and captured sweep graphs have moved on, replays
    the same continuation (the per-lane planes follow the restored
    permutation; tables and graphs are kept)."""
    K = 4
    beta = [1.0 / (0.7 + 0.3 * k) for k in range(K)]
    lat = ianus.Lattice(dim=3, L=6, n_samples=67, n_replicas=2, n_temps=K, seed=SEED + 97, layout=layout,
                        series_capacity=64)
    lat.sweep_pt(METROPOLIS, beta, 20, swap_every=5)
    blob = lat.get_state()
    lat.sweep_pt(METROPOLIS, beta, 40, swap_every=8, measure_every=4)
    first = (lat.spins(), lat.pt_state()[0], lat.series(clear=True)[1])
    lat.set_state(blob)
    lat.sweep_pt(METROPOLIS, beta, 40, swap_every=8, measure_every=4)
    again = (lat.spins(), lat.pt_state()[0], lat.series(clear=True)[1])
    for x, y in zip(first, again):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("layout", ["i8", "bits64"])
def test_gauge_invariance_on_gpu(ianus, layout):
    L, dim, S = 6, 3, 3
    N = L ** dim
    a = ianus.Lattice(dim=dim, L=L, n_samples=S, n_replicas=2, seed=21, layout=layout)
    b = ianus.Lattice(dim=dim, L=L, n_samples=S, n_replicas=2, seed=21, layout=layout)
    rng = np.random.default_rng(4)
    eps = rng.choice([-1, 1], size=(S, N)).astype(np.int8)
    J = a.couplings()
    x = np.arange(N) % L
    y = (np.arange(N) // L) % L
    z = np.arange(N) // (L * L)
    fwd = [((x + 1) % L) + L * (y + L * z), x + L * (((y + 1) % L) + L * z), x + L * (y + L * ((z + 1) % L))]
    Jg = J.copy()
    for d in range(dim):
        Jg[:, d, :] = eps * J[:, d, :] * eps[:, fwd[d]]
    b.set_couplings(Jg)
    b.set_spins(a.spins() * eps[:, None, :])
    for algo in (METROPOLIS, HEATBATH):
        a.sweep(algo, 0.8, 4)
        b.sweep(algo, 0.8, 4)
        assert np.array_equal(b.spins(), a.spins() * eps[:, None, :])
        Ea, _, Qa = a.measure()
        Eb, _, Qb = b.measure()
        assert np.array_equal(Ea, Eb) and np.array_equal(Qa, Qb)


@pytest.mark.parametrize("dim,L,S,R", [(3, 2, 1, 2), (3, 4, 9, 2), (2, 6, 6, 2), (3, 8, 5, 1)])
def test_potts_sweep_bit_exact(ianus, dim, L, S, R):
    lat, orc, _ = _pair(ianus, model="potts", dim=dim, L=L, S=S, R=R, seed=SEED + 3)
    for beta in (0.5, 1.25):
        for _ in range(4):
            lat.sweep(HEATBATH, beta, 1)
            orc.sweep(HEATBATH, beta, 1)
            assert np.array_equal(lat.spins(), orc.spins())
    E, M, Q = lat.measure()
    Eo, Mo, Qo = orc.measure()
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo)
    if R >= 2:
        assert np.array_equal(Q, Qo)


@pytest.mark.parametrize("layout", ["i8", "bits64"])
def test_tempering_with_measurements_at_the_swaps(ianus, layout):
    """Series measured at every swap: the swap takes its energies from that
    measurement instead of measuring again; a set_spins between a
    measurement and a swap forces a new one."""
    K = 4
    beta = [1.0 / (0.7 + 0.3 * k) for k in range(K)]
    lat, orc, _ = _pair(ianus, dim=3, L=4, S=67, R=2, K=K, layout=layout, seed=SEED + 98)
    lat.sweep_pt(HEATBATH, beta, 20, swap_every=5, measure_every=5)
    for _ in range(4):
        orc.sweep(HEATBATH, beta, 5, measure_every=5)
        orc.pt_swap(beta)
    assert np.array_equal(lat.spins(), orc.spins())
    assert np.array_equal(lat.pt_state()[0], orc.pt_state()[0])
    _, E, M, Q = lat.series()
    _, Eo, Mo, Qo = orc.series()
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo) and np.array_equal(Q, Qo)
    lat.measure()
    orc.measure()
    fresh = np.random.default_rng(7).choice(np.array([-1, 1], dtype=np.int8), size=lat.spins().shape)
    lat.set_spins(fresh)
    orc.set_spins(fresh)
    lat.pt_swap()
    orc.pt_swap(beta)
    assert np.array_equal(lat.pt_state()[0], orc.pt_state()[0])


@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
@pytest.mark.parametrize("dim,L,S,R,K", [(3, 6, 67, 2, 3), (2, 10, 5, 1, 4), (3, 8, 130, 3, 2), (2, 16, 64, 2, 2)])
def test_per_lane_kernel_compiled_for_the_geometry(ianus, algo, dim, L, S, R, K):
    """The per-lane-plane sweep compiled at run time for the lattice's
    geometry (default) and the precompiled one (variant 1) against the
    oracle, with swaps so that lanes sit at different temperatures; L not a
    power of two, one and three replicas, ragged sample counts."""
    beta = [1.0 / (0.8 + 0.7 * k / (K - 1)) for k in range(K)]
    runs = []
    for variant in (0, 1):
        lat, orc, _ = _pair(ianus, dim=dim, L=L, S=S, R=R, K=K, layout="bits64", seed=SEED + 60 + L)
        lat.set_variant(variant)
        for _ in range(3):
            lat.sweep(algo, beta, 2)
            lat.pt_swap()
        runs.append(lat.spins())
    for _ in range(3):
        orc.sweep(algo, beta, 2)
        orc.pt_swap(beta)
    assert np.array_equal(runs[0], orc.spins()) and np.array_equal(runs[1], orc.spins())


@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
@pytest.mark.parametrize("R,K", [(3, 3), (5, 2), (30, 2), (100, 2)])
def test_many_replicas_with_tempering(ianus, algo, R, K):
    """Per-lane-plane kernel with a run-time replica count: heat-bath words
    queued per warp (up to 97 replicas), beyond that, and for Metropolis,
    each word run to the end in place; swaps give every lane its own
    temperature.  One compiled kernel serves all replica counts, so the
    cases in turn need more and more of its shared memory."""
    beta = [1.0 / (0.8 + 0.6 * k / (K - 1)) for k in range(K)]
    lat, orc, _ = _pair(ianus, dim=3, L=4, S=67, R=R, K=K, layout="bits64", seed=SEED + 50 + R)
    for _ in range(3):
        lat.sweep(algo, beta, 2)
        orc.sweep(algo, beta, 2)
        lat.pt_swap()
        orc.pt_swap(beta)
        assert np.array_equal(lat.spins(), orc.spins())
    sa, acc, _ = lat.pt_state()
    sao, acco, _ = orc.pt_state()
    assert np.array_equal(sa, sao) and np.array_equal(acc, acco)
    E, M, Q = lat.measure()
    Eo, Mo, Qo = orc.measure()
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo) and np.array_equal(Q, Qo)


@pytest.mark.parametrize("layout", ["i8", "bits64"])
@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
def test_parallel_tempering_matches_oracle(ianus, layout, algo):
    K = 5
    beta = [1.0 / (0.7 + 0.9 * k / (K - 1)) for k in range(K)]
    lat, orc, _ = _pair(ianus, dim=3, L=4, S=67, R=2, K=K, layout=layout, seed=SEED + 40)
    for _ in range(6):
        lat.sweep(algo, beta, 3)
        orc.sweep(algo, beta, 3)
        lat.pt_swap()
        orc.pt_swap(beta)
        sa, acc, steps = lat.pt_state()
        sao, acco, stepso = orc.pt_state()
        assert np.array_equal(sa, sao) and np.array_equal(acc, acco) and steps == stepso
        assert np.array_equal(lat.spins(), orc.spins())
    assert acc.sum() > 0
    E, M, Q = lat.measure()
    Eo, Mo, Qo = orc.measure()
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo) and np.array_equal(Q, Qo)


def test_sweep_pt_fused_equals_separate(ianus):
    K = 4
    beta = [1.2, 1.0, 0.8, 0.6]
    a = ianus.Lattice(dim=3, L=4, n_samples=10, n_replicas=2, n_temps=K, seed=3)
    b = ianus.Lattice(dim=3, L=4, n_samples=10, n_replicas=2, n_temps=K, seed=3)
    a.sweep_pt(METROPOLIS, beta, 20, swap_every=5)
    for _ in range(4):
        b.sweep(METROPOLIS, beta, 5)
        b.pt_swap()
    assert np.array_equal(a.spins(), b.spins())
    assert np.array_equal(a.pt_state()[0], b.pt_state()[0])


def test_errors_are_reported_not_raised_in_kernels(ianus):
    lat = ianus.Lattice(dim=3, L=4, n_samples=2)
    with pytest.raises(ianus.IanusError) as e:
        lat.sweep(METROPOLIS, -1.0, 1)
    assert e.value.status == ianus.EINVAL
    with pytest.raises(ianus.IanusError):
        lat.pt_swap()  # one temperature
    p = ianus.Lattice(model="potts", dim=3, L=4, n_samples=2)
    with pytest.raises(ianus.IanusError) as e:
        p.sweep(METROPOLIS, 1.0, 1)
    assert e.value.status == ianus.EUNSUPPORTED
    lat.synchronize()


# ---------------- full-size workloads ----------------

def test_L16_single_sample_metropolis_full_run(ianus):
    """3D EA L=16, one sample, Metropolis T=1.1, 1000 sweeps, E and M after
    every sweep: the whole series bit-exact against the oracle."""
    seed = SEED + 0
    beta = 1.0 / 1.1
    for layout in ("i8", "bits64"):
        lat = ianus.Lattice(dim=3, L=16, n_samples=1, seed=seed, layout=layout, series_capacity=1000)
        lat.sweep(METROPOLIS, beta, 1000, measure_every=1)
        orc = Oracle(dim=3, L=16, sample_ids=[0], seed=seed)
        orc.sweep(METROPOLIS, beta, 1000, measure_every=1)
        sw, E, M, _ = lat.series()
        swo, Eo, Mo, _ = orc.series()
        assert len(sw) == 1000
        assert np.array_equal(sw, swo) and np.array_equal(E, Eo) and np.array_equal(M, Mo)
        assert np.array_equal(lat.spins(), orc.spins())


# The kernel variant and words per block bench.py times on this workload
# (checked against bench.DEFAULT_VARIANT by a CPU test).
BENCH_SHAPE = (24, 0)


@pytest.mark.parametrize("shape", [None, BENCH_SHAPE])
def test_L64_256x2_heatbath_full_size_sampled(ianus, shape):
    """L=64, 256 samples x 2 replicas, heat bath T=1.0 on the GPU, with the
    automatic kernel choice and with the kernel and launch shape bench.py
    times (the lane-queue kernel, variant 24, in its one-wave launch); samples 0, 63, 64, 255 checked
    against the oracle."""
    seed = SEED + 1
    lat = ianus.Lattice(dim=3, L=64, n_samples=256, n_replicas=2, seed=seed, layout="bits64")
    if shape is not None:
        lat.set_variant(shape[0])
        lat.set_block_words(shape[1])
    lat.sweep(HEATBATH, 1.0, 10, measure_every=5)
    ids = [0, 63, 64, 255]
    orc = Oracle(dim=3, L=64, sample_ids=ids, n_replicas=2, seed=seed)
    orc.sweep(HEATBATH, 1.0, 10, measure_every=5, nthreads=8)
    sp = lat.spins()
    assert np.array_equal(sp[ids], orc.spins())
    sw, E, M, Q = lat.series()
    swo, Eo, Mo, Qo = orc.series()
    assert np.array_equal(E[:, ids], Eo) and np.array_equal(Q[:, ids], Qo) and np.array_equal(M[:, ids], Mo)
    # every sample: energy from the series equals the energy of the read-back state
    E_now, _, _ = lat.measure()
    assert np.array_equal(E_now, E[-1])


def test_L32_pt_32_temperatures_full_size_sampled(ianus):
    """L=32, 32 temperatures in [0.7, 1.6], 64 samples x 2 replicas,
    Metropolis with a device PT swap every 10 sweeps; samples 0 and 37."""
    seed = SEED + 2
    K = 32
    beta = [1.0 / (0.7 + 0.9 * k / 31) for k in range(K)]
    lat = ianus.Lattice(dim=3, L=32, n_samples=64, n_replicas=2, n_temps=K, seed=seed, layout="bits64")
    ids = [0, 37]
    orc = Oracle(dim=3, L=32, sample_ids=ids, n_replicas=2, n_temps=K, seed=seed)
    for _ in range(2):
        lat.sweep(METROPOLIS, beta, 10)
        lat.pt_swap()
        orc.sweep(METROPOLIS, beta, 10, nthreads=2)
        orc.pt_swap(beta)
    sa, acc, _ = lat.pt_state()
    sao, acco, _ = orc.pt_state()
    assert np.array_equal(sa[ids], sao) and np.array_equal(acc[ids], acco)
    assert np.array_equal(lat.spins()[ids], orc.spins())
    E, _, _ = lat.measure()
    Eo, _, _ = orc.measure()
    assert np.array_equal(E[ids], Eo)


def test_L32_pt_32_temperatures_sweep_pt_as_benched(ianus):
    """The parallel-tempering workload through ianus_sweep_pt exactly as the
    bench times it (captured sweep graphs, swaps on the device every 10
    sweeps, energies for the swap reused from the measurement pass): L=32,
    32 temperatures, 64 samples x 2 replicas, 30 sweeps; samples 0 and 37
    against the oracle's sweep-then-swap sequence."""
    seed = SEED + 2
    K = 32
    beta = [1.0 / (0.7 + 0.9 * k / 31) for k in range(K)]
    lat = ianus.Lattice(dim=3, L=32, n_samples=64, n_replicas=2, n_temps=K, seed=seed, layout="bits64")
    lat.sweep_pt(METROPOLIS, beta, 30, swap_every=10)
    ids = [0, 37]
    orc = Oracle(dim=3, L=32, sample_ids=ids, n_replicas=2, n_temps=K, seed=seed)
    for _ in range(3):
        orc.sweep(METROPOLIS, beta, 10, nthreads=2)
        orc.pt_swap(beta)
    sa, acc, steps = lat.pt_state()
    sao, acco, stepso = orc.pt_state()
    assert steps == stepso == 3
    assert np.array_equal(sa[ids], sao) and np.array_equal(acc[ids], acco)
    assert np.array_equal(lat.spins()[ids], orc.spins())
    E, _, Q = lat.measure()
    Eo, _, Qo = orc.measure()
    assert np.array_equal(E[ids], Eo) and np.array_equal(Q[ids], Qo)


def test_potts_L32_128x2_full_size_sampled(ianus):
    """Potts q=4, L=32, 128 samples x 2 replicas, heat bath T=0.8."""
    seed = SEED + 3
    lat = ianus.Lattice(model="potts", dim=3, L=32, n_samples=128, n_replicas=2, seed=seed)
    lat.sweep(HEATBATH, 1.0 / 0.8, 10, measure_every=10)
    ids = [0, 127]
    orc = Oracle(model=MODEL_POTTS, dim=3, L=32, sample_ids=ids, n_replicas=2, seed=seed)
    orc.sweep(HEATBATH, 1.0 / 0.8, 10, measure_every=10, nthreads=2)
    assert np.array_equal(lat.spins()[ids], orc.spins())
    _, E, M, Q = lat.series()
    _, Eo, Mo, Qo = orc.series()
    assert np.array_equal(E[:, ids], Eo) and np.array_equal(M[:, ids], Mo) and np.array_equal(Q[:, ids], Qo)


@pytest.mark.parametrize("variant", list(range(1, 28)))
def test_every_variant_and_launch_shape_is_bit_exact(ianus, variant):
    """All kernel variants and several launch shapes give the same
    trajectory (L=16: several blocks per (group, slot), ragged last block;
    shapes of whole warps that leave part of a block idle)."""
    ref = None
    for bw in (0, 256, 768, 96, 480):
        lat = ianus.Lattice(dim=3, L=16, n_samples=100, n_replicas=2, seed=SEED + 77, layout="bits64")
        lat.set_variant(variant)
        lat.set_block_words(bw)
        lat.sweep(HEATBATH, 0.9, 3)
        lat.sweep(METROPOLIS, 1.1, 3)
        sp = lat.spins()
        if ref is None:
            orc = Oracle(dim=3, L=16, sample_ids=list(range(100)), n_replicas=2, seed=SEED + 77)
            orc.sweep(HEATBATH, 0.9, 3, nthreads=8)
            orc.sweep(METROPOLIS, 1.1, 3, nthreads=8)
            ref = orc.spins()
        assert np.array_equal(sp, ref), (variant, bw)


def test_autotuner_does_not_change_the_trajectory(ianus, tmp_path, monkeypatch):
    from paper_0704_3573_gb300 import tune

    monkeypatch.setenv("IANUS_TUNE_CACHE", str(tmp_path / "tune.json"))
    a = ianus.Lattice(dim=3, L=16, n_samples=128, n_replicas=2, seed=SEED + 78, layout="bits64")
    b = ianus.Lattice(dim=3, L=16, n_samples=128, n_replicas=2, seed=SEED + 78, layout="bits64")
    a.sweep(HEATBATH, 1.0, 4)
    b.sweep(HEATBATH, 1.0, 4)
    best = tune.tune(a, HEATBATH, 1.0, sweeps=4, block_words=(0, 512))
    assert best["variant"] in tune.VARIANTS and not best["cached"]
    assert a.sweeps == 4
    a.sweep(HEATBATH, 1.0, 5)
    b.sweep(HEATBATH, 1.0, 5)
    assert np.array_equal(a.spins(), b.spins())
    again = tune.tune(a, HEATBATH, 1.0)
    assert again["cached"] and again["variant"] == best["variant"]


@pytest.mark.parametrize("layout,model", [("i8", "ea"), ("bits64", "ea"), ("bits64-jit", "ea"), ("auto", "potts")])
def test_graph_replay_equals_direct_launches(ianus, layout, model):
    """Sweep blocks replayed from captured graphs (device sweep counter) give
    the same trajectory and series as launching every kernel directly."""
    runs = []
    for graphs in (True, False):
        lat, _, _ = _pair(ianus, model=model, dim=3, L=6, S=70, R=2, layout=layout, seed=SEED + 90)
        lat.set_graphs(graphs)
        algo = HEATBATH
        for n, every in ((7, 0), (69, 6), (3, 0), (64, 0), (130, 0), (12, 4)):
            lat.sweep(algo, 0.95, n, measure_every=every)
        runs.append((lat.spins(), lat.series(), lat.sweeps))
    (s0, ser0, n0), (s1, ser1, n1) = runs
    assert n0 == n1 == 285
    assert np.array_equal(s0, s1)
    for a, b in zip(ser0, ser1):
        assert np.array_equal(a, b)


def test_graphs_with_parallel_tempering(ianus):
    K = 4
    beta = [1.3, 1.1, 0.9, 0.7]
    lat, orc, _ = _pair(ianus, dim=3, L=4, S=66, R=2, K=K, layout="bits64", seed=SEED + 91)
    lat.sweep_pt(METROPOLIS, beta, 40, swap_every=10)
    for _ in range(4):
        orc.sweep(METROPOLIS, beta, 10)
        orc.pt_swap(beta)
    assert np.array_equal(lat.spins(), orc.spins())
    assert np.array_equal(lat.pt_state()[0], orc.pt_state()[0])


@pytest.mark.parametrize("dim,L,S,R,every", [(3, 16, 1, 1, 1), (3, 8, 5, 1, 3), (2, 32, 3, 1, 0), (3, 2, 1, 1, 1),
                                             (3, 32, 2, 1, 7), (3, 6, 2, 1, 1), (2, 12, 1, 1, 2), (3, 8, 3, 2, 0),
                                             (3, 4, 1, 1, 1), (2, 6, 1, 1, 1), (3, 10, 1, 1, 1), (2, 2, 1, 1, 1),
                                             (3, 8, 70, 1, 5)])
def test_resident_mode_equals_oracle_and_eager(ianus, dim, L, S, R, every):
    """Resident modes against the oracle and the launch-per-colour path:
    automatic, every configuration split over a block cluster (slabs along
    the last axis, faces read from the neighbouring block's shared memory;
    L = 2 and one-plane slabs make both faces remote; E and M carried by the
    flips), one block per configuration, and off.  Many sweeps per launch,
    series written in the kernel."""
    runs = []
    for resident in (1, 3, 2, 0):
        lat = ianus.Lattice(dim=dim, L=L, n_samples=S, n_replicas=R, seed=SEED + 95, layout="i8",
                            series_capacity=100)
        lat.set_resident(resident)
        lat.sweep(METROPOLIS, 1.0 / 1.1, 40, measure_every=every)
        lat.sweep(HEATBATH, 0.8, 13, measure_every=every)
        runs.append((lat.spins(), lat.series()))
    orc = Oracle(dim=dim, L=L, sample_ids=list(range(S)), n_replicas=R, seed=SEED + 95)
    orc.sweep(METROPOLIS, 1.0 / 1.1, 40, measure_every=every)
    orc.sweep(HEATBATH, 0.8, 13, measure_every=every)
    for sp, (sw, E, M, _) in runs:
        assert np.array_equal(sp, orc.spins())
        swo, Eo, Mo, _ = orc.series()
        assert np.array_equal(sw, swo) and np.array_equal(E, Eo) and np.array_equal(M, Mo)


def test_resident_mode_values(ianus):
    lat = ianus.Lattice(dim=3, L=4, seed=1, layout="i8")
    for bad in (-1, 4):
        with pytest.raises(ianus.IanusError) as e:
            lat.set_resident(bad)
        assert e.value.status == ianus.EINVAL
