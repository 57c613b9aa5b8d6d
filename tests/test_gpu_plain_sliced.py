"""The plain one-byte-per-spin layout swept bit-sliced in shared memory
(k_sweep_i8_sliced, the automatic plain kernel when L is a multiple of
32): tiles of a 64-sample group read as bytes, turned into 64-lane words by
warp bit transposes, updated, and written back as bytes.

Compared bit for bit with the oracle and with the plain word kernel
(variant 2), on 2D and 3D lattices, ragged sample counts (a last group of
1 to 63 samples), one and two replicas, several temperatures, both
algorithms, graph replay, and the bench's plain workload at full size (L=64,
256 samples x 2 replicas, heat bath T=1.0).
"""

import numpy as np
import pytest

from oracle import HEATBATH, METROPOLIS, Oracle

pytestmark = pytest.mark.gpu

SEED = 0x0704357300000000 + 1100


def _plain(ianus, dim, L, S, R, K, variant, seed):
    lat = ianus.Lattice(dim=dim, L=L, n_samples=S, n_replicas=R, n_temps=K, seed=seed, layout="i8")
    lat.set_resident(0)  # the launch-per-colour kernels, not the small-lattice resident sweep
    lat.set_variant(variant)
    return lat


@pytest.mark.parametrize("dim,L,S,R,K", [(3, 32, 64, 1, 1), (3, 32, 70, 2, 1), (3, 32, 130, 1, 2),
                                         (2, 32, 65, 2, 1), (2, 64, 100, 1, 1), (2, 128, 64, 2, 1),
                                         (2, 128, 30, 1, 3), (3, 64, 3, 1, 1)])
def test_sliced_plain_equals_oracle_and_word_kernel(ianus, dim, L, S, R, K):
    beta = [0.6 + 0.3 * k for k in range(K)]
    steps = [(HEATBATH, beta, 3, 3), (METROPOLIS, beta, 4, 2)]
    sl = _plain(ianus, dim, L, S, R, K, 0, SEED)
    wd = _plain(ianus, dim, L, S, R, K, 2, SEED)
    orc = Oracle(dim=dim, L=L, sample_ids=list(range(S)), n_replicas=R, n_temps=K, seed=SEED)
    for algo, b, n, every in steps:
        sl.sweep(algo, b, n, measure_every=every)
        wd.sweep(algo, b, n, measure_every=every)
        orc.sweep(algo, b, n, measure_every=every, nthreads=8)
    sp = sl.spins()
    assert np.array_equal(sp, orc.spins())
    assert np.array_equal(sp, wd.spins())
    sw, E, M, Q = sl.series()
    swo, Eo, Mo, Qo = orc.series()
    assert np.array_equal(sw, swo) and np.array_equal(E, Eo) and np.array_equal(M, Mo)
    if R >= 2:
        assert np.array_equal(Q, Qo)


def test_sliced_plain_graph_replay(ianus):
    runs = []
    for graphs in (True, False):
        lat = _plain(ianus, 3, 32, 70, 2, 1, 0, SEED + 1)
        lat.set_graphs(graphs)
        for n, every in ((7, 0), (69, 6), (64, 0)):
            lat.sweep(HEATBATH, 0.95, n, measure_every=every)
        runs.append((lat.spins(), lat.series()))
    assert np.array_equal(runs[0][0], runs[1][0])
    for a, b in zip(runs[0][1], runs[1][1]):
        if a is not None:
            assert np.array_equal(a, b)


def test_sliced_plain_L64_256x2_heatbath_full_size(ianus):
    """The plain workload bench.py times: samples 0, 63, 64 and 255 against
    the oracle, every sample against the word kernel."""
    seed = SEED + 2
    sl = _plain(ianus, 3, 64, 256, 2, 1, 0, seed)
    wd = _plain(ianus, 3, 64, 256, 2, 1, 2, seed)
    for lat in (sl, wd):
        lat.sweep(HEATBATH, 1.0, 10, measure_every=5)
    ids = [0, 63, 64, 255]
    orc = Oracle(dim=3, L=64, sample_ids=ids, n_replicas=2, seed=seed)
    orc.sweep(HEATBATH, 1.0, 10, measure_every=5, nthreads=8)
    sp = sl.spins()
    assert np.array_equal(sp[ids], orc.spins())
    assert np.array_equal(sp, wd.spins())
    sw, E, M, Q = sl.series()
    swo, Eo, Mo, Qo = orc.series()
    assert np.array_equal(E[:, ids], Eo) and np.array_equal(M[:, ids], Mo) and np.array_equal(Q[:, ids], Qo)
