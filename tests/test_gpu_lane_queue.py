"""GPU parity of the lane-queue sweep (variants 22..24): Philox rounds 0 and 1
shared between a site part and a block-uniform part, plane pairs 0..3 for
every word, the still undecided lanes finished from per-warp queues; and of
its persistent form (variants 25, 26), one cooperative launch per block of
sweeps with bounded waits between the blocks of neighbouring rows.  Every
case is compared bit for bit with the oracle (spins and the E, M, Q series).

The cases span several blocks and a ragged last block, 2D and 3D, sides that
are not powers of two, L = 2 (two bonds to one neighbour), partly filled
64-lane words, one and two replicas, both algorithms, and temperatures that
send many lanes to the queue (Metropolis at beta = 40: threshold 0, so a lane
stays undecided while its random bits are 0) or none beyond pair 0
(heat bath at beta = 0: threshold 2^31, decided at plane 0).
"""

import numpy as np
import pytest

from oracle import HEATBATH, METROPOLIS, Oracle

pytestmark = pytest.mark.gpu

SEED = 0x0704357300000000 + 500


def _run(ianus, variant, dim, L, S, R, steps, block_words=0, seed=SEED, graphs=None):
    lat = ianus.Lattice(dim=dim, L=L, n_samples=S, n_replicas=R, seed=seed, layout="bits64")
    lat.set_variant(variant)
    lat.set_block_words(block_words)
    if graphs is not None:
        lat.set_graphs(graphs)
    orc = Oracle(dim=dim, L=L, sample_ids=list(range(S)), n_replicas=R, seed=seed)
    for algo, beta, n, every in steps:
        lat.sweep(algo, beta, n, measure_every=every)
        orc.sweep(algo, beta, n, measure_every=every, nthreads=8)
    assert np.array_equal(lat.spins(), orc.spins())
    sw, E, M, Q = lat.series()
    swo, Eo, Mo, Qo = orc.series()
    assert np.array_equal(sw, swo) and np.array_equal(E, Eo) and np.array_equal(M, Mo)
    if R >= 2:
        assert np.array_equal(Q, Qo)
    return lat


STEPS = [(HEATBATH, 0.9, 4, 2), (METROPOLIS, 1.1, 3, 3)]


@pytest.mark.parametrize("variant", [22, 23, 24, 25, 26, 27])
@pytest.mark.parametrize("dim,L,S,R", [(3, 8, 70, 2), (3, 16, 130, 1), (2, 32, 65, 2), (3, 6, 64, 2),
                                       (2, 10, 3, 1), (3, 2, 67, 2), (2, 2, 1, 1), (3, 12, 100, 2)])
def test_lane_queue_bit_exact(ianus, variant, dim, L, S, R):
    _run(ianus, variant, dim, L, S, R, STEPS)


@pytest.mark.parametrize("block_words", [32, 96, 256, 480])
def test_lane_queue_launch_shapes(ianus, block_words):
    """Explicit launch shapes: many blocks per group, ragged last blocks."""
    _run(ianus, 22, 3, 16, 100, 2, STEPS, block_words=block_words)


@pytest.mark.parametrize("variant", [22, 26])
@pytest.mark.parametrize("algo,beta", [(METROPOLIS, 40.0), (HEATBATH, 0.0), (METROPOLIS, 0.0), (HEATBATH, 40.0),
                                       (HEATBATH, 0.3)])
def test_lane_queue_extreme_temperatures(ianus, variant, algo, beta):
    _run(ianus, variant, 3, 8, 128, 2, [(algo, beta, 5, 1)])


def test_lane_queue_graph_replay(ianus):
    """Captured sweep blocks (sweep counter read from the device) give the
    same trajectory as direct launches and the oracle."""
    a = _run(ianus, 22, 3, 16, 70, 2, [(HEATBATH, 1.0, 40, 10)], graphs=True)
    b = _run(ianus, 22, 3, 16, 70, 2, [(HEATBATH, 1.0, 40, 10)], graphs=False)
    assert np.array_equal(a.spins(), b.spins())


@pytest.mark.parametrize("variant", [22, 25])
def test_lane_queue_L64_256x2_heatbath_full_size_sampled(ianus, variant):
    """The bench lattice (L=64, 256 samples x 2 replicas, heat bath T=1.0)
    with the lane-queue kernel in its default one-wave launch and in its
    persistent form; samples 0, 63, 64 and 255 checked against the oracle,
    and the last series energy of every sample against a fresh measurement of
    the read-back state."""
    seed = SEED + 1
    lat = ianus.Lattice(dim=3, L=64, n_samples=256, n_replicas=2, seed=seed, layout="bits64")
    lat.set_variant(variant)
    lat.set_block_words(0)
    lat.sweep(HEATBATH, 1.0, 20, measure_every=10)
    ids = [0, 63, 64, 255]
    orc = Oracle(dim=3, L=64, sample_ids=ids, n_replicas=2, seed=seed)
    orc.sweep(HEATBATH, 1.0, 20, measure_every=10, nthreads=8)
    assert np.array_equal(lat.spins()[ids], orc.spins())
    sw, E, M, Q = lat.series()
    swo, Eo, Mo, Qo = orc.series()
    assert np.array_equal(E[:, ids], Eo) and np.array_equal(Q[:, ids], Qo) and np.array_equal(M[:, ids], Mo)
    E_now, _, _ = lat.measure()
    assert np.array_equal(E_now, E[-1])


@pytest.mark.parametrize("dim,L,S,R,sweeps", [(3, 16, 200, 2, 25), (2, 64, 64, 1, 30), (3, 10, 70, 2, 12)])
def test_persistent_long_blocks_of_sweeps(ianus, dim, L, S, R, sweeps):
    """Many sweeps in one persistent launch (no measurement in between), on
    lattices where a block's rows reach several other blocks' rows."""
    _run(ianus, 26, dim, L, S, R, [(HEATBATH, 0.8, sweeps, 0), (METROPOLIS, 1.2, sweeps, sweeps)])


def test_persistent_wait_runs_out_and_is_reported(ianus):
    """One block is told to return at once, so the blocks that wait for its
    progress flag time out (20 ms), record ERR_TIMEOUT and return; the next
    synchronisation reports ETIMEOUT, the lattice then refuses work (ESTATE),
    and the device stays usable: a fresh lattice still matches the oracle."""
    lat = ianus.Lattice(dim=3, L=16, n_samples=128, n_replicas=2, seed=SEED + 9, layout="bits64")
    lat.set_variant(26)
    lat.set_persistent_wait(20_000_000, absent_block=1)
    lat.sweep(HEATBATH, 1.0, 4)
    with pytest.raises(ianus.IanusError) as e:
        lat.synchronize()
    assert e.value.status == ianus.ETIMEOUT
    with pytest.raises(ianus.IanusError) as e:
        lat.sweep(HEATBATH, 1.0, 1)
    assert e.value.status == ianus.ESTATE
    _run(ianus, 26, 3, 16, 128, 2, [(HEATBATH, 1.0, 4, 2)], seed=SEED + 9)


def test_persistent_wait_limit_validation(ianus):
    lat = ianus.Lattice(dim=3, L=8, n_samples=64, n_replicas=2, seed=SEED, layout="bits64")
    with pytest.raises(ianus.IanusError):
        lat.set_persistent_wait(0)
    with pytest.raises(ianus.IanusError):
        lat.set_persistent_wait(1000, absent_block=-2)
