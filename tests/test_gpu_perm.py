"""GPU parity of the glassy Potts model with permutation couplings (Eq. 3)
through the C ABI against the CPU oracle, in 2, 3 and 4 dimensions.

Integer work throughout, so the bar is bit-exact: permutation codes,
initial states, states after every sweep, energies, state counts and
overlaps.  Sizes span several blocks and ragged tails (sample counts that
are not multiples of the 4 samples of a word; L = 2, where the two bonds
joining a pair of sites carry different permutations).
"""

import itertools

import numpy as np
import pytest

from oracle import HEATBATH, METROPOLIS, MODEL_PERM, Oracle

pytestmark = pytest.mark.gpu

SEED = 0x0704357300000E00
CODES = np.array([p[0] | (p[1] << 2) | (p[2] << 4) | (p[3] << 6) for p in itertools.permutations(range(4))],
                 dtype=np.uint8)


def _pair(ianus, dim=3, L=4, S=1, R=1, K=1, seed=SEED, ferro=False, ids=None):
    lat = ianus.Lattice(model="potts_perm", dim=dim, L=L, n_samples=S, n_replicas=R, n_temps=K, seed=seed,
                        ferro=ferro, series_capacity=4096)
    ids = list(range(S)) if ids is None else ids
    orc = Oracle(model=MODEL_PERM, dim=dim, L=L, sample_ids=ids, n_replicas=R, n_temps=K, seed=seed, ferro=ferro)
    return lat, orc


@pytest.mark.parametrize("dim,L,S,R", [(2, 2, 1, 1), (2, 6, 5, 2), (3, 4, 9, 2), (3, 2, 3, 1), (4, 2, 6, 2),
                                       (4, 4, 7, 1), (3, 8, 70, 1)])
def test_perm_init_matches_oracle(ianus, dim, L, S, R):
    lat, orc = _pair(ianus, dim=dim, L=L, S=S, R=R)
    assert np.array_equal(lat.couplings(), orc.couplings())
    assert np.array_equal(lat.spins(), orc.spins())
    E, M, Q = lat.measure()
    Eo, Mo, Qo = orc.measure()
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo)
    if R >= 2:
        assert np.array_equal(Q, Qo)


CASES = [(2, 2, 1, 1, 1), (2, 8, 6, 2, 1), (3, 2, 5, 2, 1), (3, 4, 9, 2, 1), (3, 6, 3, 1, 2), (4, 2, 5, 2, 1),
         (4, 4, 6, 2, 1), (4, 6, 3, 1, 2), (3, 10, 13, 1, 1)]


@pytest.mark.parametrize("dim,L,S,R,K", CASES)
def test_perm_sweep_bit_exact_every_sweep(ianus, dim, L, S, R, K):
    lat, orc = _pair(ianus, dim=dim, L=L, S=S, R=R, K=K, seed=SEED + 7 * L + S)
    beta = [0.9, 2.4][:K] if dim == 3 else [0.6, 1.405][:K]
    for _ in range(5):
        lat.sweep(HEATBATH, beta, 1)
        orc.sweep(HEATBATH, beta, 1)
        assert np.array_equal(lat.spins(), orc.spins())
    E, M, Q = lat.measure()
    Eo, Mo, Qo = orc.measure()
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo)
    if R >= 2:
        assert np.array_equal(Q, Qo)


@pytest.mark.parametrize("dim", [3, 4])
def test_perm_series_and_graphs(ianus, dim):
    lat, orc = _pair(ianus, dim=dim, L=4, S=11, R=2)
    lat.sweep(HEATBATH, 1.2, 23, measure_every=5)
    orc.sweep(HEATBATH, 1.2, 23, measure_every=5)
    sw, E, M, Q = lat.series()
    swo, Eo, Mo, Qo = orc.series()
    assert list(sw) == list(swo) == [5, 10, 15, 20]
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo) and np.array_equal(Q, Qo)
    eager, _ = _pair(ianus, dim=dim, L=4, S=11, R=2)
    eager.set_graphs(False)
    eager.sweep(HEATBATH, 1.2, 23, measure_every=5)
    assert np.array_equal(eager.spins(), lat.spins())


@pytest.mark.parametrize("beta", [0.0, 80.0])
def test_perm_extreme_temperatures(ianus, beta):
    for dim in (2, 3, 4):
        lat, orc = _pair(ianus, dim=dim, L=4, S=7, R=1)
        lat.sweep(HEATBATH, beta, 3)
        orc.sweep(HEATBATH, beta, 3)
        assert np.array_equal(lat.spins(), orc.spins()), dim


@pytest.mark.parametrize("dim", [2, 3, 4])
def test_perm_set_couplings(ianus, dim):
    """Couplings written through the ABI (random codes, a sample of identity
    bonds) drive the GPU and the oracle alike; non-permutations are refused."""
    L, S = 4, 6
    lat, orc = _pair(ianus, dim=dim, L=L, S=S, R=2)
    rng = np.random.default_rng(11)
    J = CODES[rng.integers(0, 24, size=(S, dim, L ** dim))]
    J[0, :, : L] = CODES[0]
    for obj in (lat, orc):
        obj.set_couplings(J.view(np.int8))
    assert np.array_equal(lat.couplings(), J.view(np.int8))
    for _ in range(3):
        lat.sweep(HEATBATH, 1.0, 1)
        orc.sweep(HEATBATH, 1.0, 1)
        assert np.array_equal(lat.spins(), orc.spins())
    bad = J.copy()
    bad[1, 0, 3] = 0x55  # (1, 1, 1, 1)
    with pytest.raises(ianus.IanusError) as e:
        lat.set_couplings(bad.view(np.int8))
    assert e.value.status == ianus.EINVAL


def test_identity_couplings_equal_the_ferromagnetic_potts_glass(ianus):
    """Identity permutations make Eq. (3) the ferromagnetic Potts model, i.e.
    the J-weighted Potts glass with every J = +1: same streams, same
    trajectory (3D; the J-weighted glass has no 4D form)."""
    a = ianus.Lattice(model="potts_perm", dim=3, L=8, n_samples=9, n_replicas=2, seed=3, ferro=True)
    b = ianus.Lattice(model="potts", dim=3, L=8, n_samples=9, n_replicas=2, seed=3, ferro=True)
    assert np.all(a.couplings().view(np.uint8) == CODES[0])
    for beta in (0.7, 1.5):
        a.sweep(HEATBATH, beta, 4)
        b.sweep(HEATBATH, beta, 4)
        assert np.array_equal(a.spins(), b.spins())
        for u, v in zip(a.measure(), b.measure()):
            assert np.array_equal(u, v)


def test_perm_checkpoint(ianus):
    a, _ = _pair(ianus, dim=4, L=4, S=5, R=2, seed=9)
    a.sweep(HEATBATH, 1.1, 7)
    blob = a.get_state()
    a.sweep(HEATBATH, 1.1, 5)
    b, _ = _pair(ianus, dim=4, L=4, S=5, R=2, seed=9)
    b.set_state(blob)
    assert b.sweeps == 7
    b.sweep(HEATBATH, 1.1, 5)
    assert np.array_equal(a.spins(), b.spins())


def test_perm_errors(ianus):
    lat, _ = _pair(ianus, dim=4, L=2, S=2, K=2)
    with pytest.raises(ianus.IanusError) as e:
        lat.sweep(METROPOLIS, [1.0, 1.2], 1)
    assert e.value.status == ianus.EUNSUPPORTED
    lat.sweep(HEATBATH, [1.0, 1.2], 1)
    with pytest.raises(ianus.IanusError) as e:
        lat.pt_swap()
    assert e.value.status == ianus.EUNSUPPORTED
    with pytest.raises(ianus.IanusError) as e:
        lat.sweep(HEATBATH, [1.0, 90.0], 1)  # 2 D beta > 700
    assert e.value.status == ianus.EINVAL
    with pytest.raises(ianus.IanusError):
        ianus.Lattice(model="potts", dim=4, L=4)  # 4D is the permutation model's only


@pytest.mark.parametrize("dim,L,ids,beta", [(4, 16, [0, 1, 5, 127, 200, 255], 1.405),
                                            (3, 32, [0, 3, 64, 130, 254], 2.4)])
def test_perm_full_size_sampled(ianus, dim, L, ids, beta):
    """The paper's sizes (Sec. 4.2: 4D L=16 at beta=1.405, 3D at beta=2.4 --
    here L=32), 256 samples x 2 replicas: after 10 sweeps a sample of the
    configurations equals the oracle run of exactly those samples, and every
    configuration's E, counts and Q equal the values recomputed from the
    downloaded states and couplings."""
    S, R = 256, 2
    lat = ianus.Lattice(model="potts_perm", dim=dim, L=L, n_samples=S, n_replicas=R, seed=SEED + 99)
    lat.sweep(HEATBATH, beta, 10)
    orc = Oracle(model=MODEL_PERM, dim=dim, L=L, sample_ids=ids, n_replicas=R, seed=SEED + 99)
    orc.sweep(HEATBATH, beta, 10, nthreads=8)
    sp = lat.spins()
    assert np.array_equal(sp[ids], orc.spins())
    E, M, Q = lat.measure()
    Eo, Mo, Qo = orc.measure()
    assert np.array_equal(E[ids], Eo) and np.array_equal(M[ids], Mo) and np.array_equal(Q[ids], Qo)
    # every configuration: counts and overlap from the states; E from Eq. (3)
    assert np.array_equal(M[:, 0], np.stack([(sp == k).sum(axis=2) for k in range(4)], axis=-1))
    assert np.array_equal(Q[:, 0], (sp[:, 0] == sp[:, 1]).sum(axis=1))
    J = lat.couplings().view(np.uint8).astype(np.int64)
    N = L ** dim
    idx = np.arange(N)
    coords = [(idx // L ** d) % L for d in range(dim)]
    Ecalc = np.zeros((S, R), dtype=np.int64)
    for d in range(dim):
        c = [x.copy() for x in coords]
        c[d] = (c[d] + 1) % L
        j = sum(c[e] * L ** e for e in range(dim))
        sj = sp[:, :, j].astype(np.int64)
        target = (J[:, None, d, :] >> (2 * sj)) & 3
        Ecalc -= (target == sp).sum(axis=2)
    assert np.array_equal(E[:, 0], Ecalc)
