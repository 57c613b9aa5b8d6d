"""GPU parity of the field models of Eq. (2): the random-field Ising model
(RFIM: J = +1, h_i = +-|h|) and the diluted antiferromagnet in a field (DAFF:
J = -1, h_i = +|h|, x_i in {0, 1}) through the C ABI against the CPU oracle.

All integer work, so the bar is bit-exact: couplings, field signs,
occupations, initial spins, spins after every sweep, E_J, M, F and Q.  Sizes
span several blocks and ragged tails (sample counts crossing the 64-lane
packing, L = 2 where forward and backward neighbours coincide); |h| covers
zero, non-integer, integer (x = v + w can be 0) and larger than 2D (the
field decides alone).
"""

import numpy as np
import pytest

from oracle import DIS_DAFF, DIS_RFIM, HEATBATH, METROPOLIS, Oracle
from tests import pins

pytestmark = pytest.mark.gpu

SEED = 0x0704357300000F00


def _pair(ianus, disorder, dim=3, L=4, S=1, R=1, K=1, h=0.75, occ=0.7, layout="auto", seed=SEED):
    name = "rfim" if disorder == DIS_RFIM else "daff"
    variant = 0
    if layout == "bits64-jit":  # the field kernel specialised at run time for the tables
        layout, variant = "bits64", 2
    elif layout == "bits64":  # per-lane threshold planes
        variant = 1
    lat = ianus.Lattice(dim=dim, L=L, n_samples=S, n_replicas=R, n_temps=K, seed=seed, layout=layout,
                        disorder=name, field=h, occupation=occ, series_capacity=4096)
    if variant:
        lat.set_variant(variant)
    orc = Oracle(dim=dim, L=L, sample_ids=list(range(S)), n_replicas=R, n_temps=K, seed=seed, disorder=disorder,
                 field=h, occupation=occ)
    return lat, orc


LAYOUTS = [(DIS_RFIM, "i8"), (DIS_RFIM, "bits64"), (DIS_RFIM, "bits64-jit"), (DIS_DAFF, "i8"), (DIS_DAFF, "bits64"),
           (DIS_DAFF, "bits64-jit")]


@pytest.mark.parametrize("disorder,layout", LAYOUTS)
@pytest.mark.parametrize("dim,L,S,R", [(3, 2, 1, 1), (3, 4, 70, 2), (2, 6, 3, 2), (3, 8, 130, 1)])
def test_field_init_matches_oracle(ianus, disorder, layout, dim, L, S, R):
    lat, orc = _pair(ianus, disorder, dim=dim, L=L, S=S, R=R, layout=layout)
    assert np.array_equal(lat.couplings(), orc.couplings())
    hs, x = lat.sites()
    hso, xo = orc.sites()
    assert np.array_equal(hs, hso) and np.array_equal(x, xo)
    assert np.array_equal(lat.spins(), orc.spins())
    E, M, Q = lat.measure()
    Eo, Mo, Qo = orc.measure()
    assert M.shape == (S, 1, R, 2)
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo)
    if R >= 2:
        assert np.array_equal(Q, Qo)


CASES = [(3, 2, 1, 1, 1), (3, 4, 3, 2, 1), (2, 4, 65, 1, 1), (3, 6, 70, 2, 1), (2, 8, 2, 2, 3), (3, 8, 1, 1, 2),
         (2, 2, 5, 2, 1), (3, 10, 67, 2, 1)]


@pytest.mark.parametrize("h", [0.75, 2.0, 0.0])
@pytest.mark.parametrize("disorder,layout", LAYOUTS)
@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
@pytest.mark.parametrize("dim,L,S,R,K", CASES)
def test_field_sweep_bit_exact_every_sweep(ianus, disorder, layout, algo, dim, L, S, R, K, h):
    lat, orc = _pair(ianus, disorder, dim=dim, L=L, S=S, R=R, K=K, h=h, layout=layout, seed=SEED + 13 * L + S)
    beta = [0.45, 0.8, 1.3][:K]
    for _ in range(5):
        lat.sweep(algo, beta, 1)
        orc.sweep(algo, beta, 1)
        assert np.array_equal(lat.spins(), orc.spins())
    E, M, Q = lat.measure()
    Eo, Mo, Qo = orc.measure()
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo)
    if R >= 2:
        assert np.array_equal(Q, Qo)


@pytest.mark.parametrize("disorder,layout", LAYOUTS)
def test_field_series_and_graphs(ianus, disorder, layout):
    """23 sweeps measured every 5 (graph-replayed blocks in between) against
    the oracle, and against the same run with eager launches."""
    lat, orc = _pair(ianus, disorder, dim=3, L=6, S=67, R=2, h=1.25, layout=layout)
    lat.sweep(HEATBATH, 0.9, 23, measure_every=5)
    orc.sweep(HEATBATH, 0.9, 23, measure_every=5)
    sw, E, M, Q = lat.series()
    swo, Eo, Mo, Qo = orc.series()
    assert list(sw) == list(swo) == [5, 10, 15, 20]
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo) and np.array_equal(Q, Qo)
    eager, _ = _pair(ianus, disorder, dim=3, L=6, S=67, R=2, h=1.25, layout=layout)
    eager.set_graphs(False)
    eager.sweep(HEATBATH, 0.9, 23, measure_every=5)
    assert np.array_equal(eager.spins(), lat.spins())


@pytest.mark.parametrize("beta", [0.0, 40.0])
@pytest.mark.parametrize("h", [0.5, 13.0])
def test_field_extreme_temperatures_and_fields(ianus, beta, h):
    """beta = 0, and a beta at which the tables saturate (T = 0 or 2^32);
    |h| = 13 > 2D makes the field decide every site."""
    for disorder, layout in LAYOUTS:
        for algo in (METROPOLIS, HEATBATH):
            lat, orc = _pair(ianus, disorder, dim=3, L=4, S=66, h=h, layout=layout)
            lat.sweep(algo, beta, 3)
            orc.sweep(algo, beta, 3)
            assert np.array_equal(lat.spins(), orc.spins()), (disorder, layout, algo)


@pytest.mark.parametrize("layout", ["i8", "bits64", "bits64-jit"])
@pytest.mark.parametrize("occ", [0.0, 1.0])
def test_daff_occupation_edges(ianus, occ, layout):
    lat, orc = _pair(ianus, DIS_DAFF, dim=3, L=6, S=9, R=2, h=0.5, occ=occ, layout=layout)
    before = lat.spins()
    for algo in (METROPOLIS, HEATBATH):
        lat.sweep(algo, 0.6, 4)
        orc.sweep(algo, 0.6, 4)
    assert np.array_equal(lat.spins(), orc.spins())
    if occ == 0.0:  # nothing to update; every observable vanishes
        assert np.array_equal(lat.spins(), before)
        E, M, Q = lat.measure()
        assert not E.any() and not M.any() and not Q.any()


@pytest.mark.parametrize("disorder,layout", LAYOUTS)
def test_field_set_sites_gauge(ianus, disorder, layout):
    """Gauge-transformed couplings, field signs and spins: GPU against the
    oracle given the same sites, and e s(t) against the untransformed run."""
    L, D, S = 4, 3, 5
    N = L ** D
    eps = np.random.default_rng(3).choice([-1, 1], size=(S, N)).astype(np.int8)
    lat, orc = _pair(ianus, disorder, dim=D, L=L, S=S, R=2, h=1.1, layout=layout)
    ref, _ = _pair(ianus, disorder, dim=D, L=L, S=S, R=2, h=1.1, layout=layout)
    J = lat.couplings()
    Jg = J.copy()
    for s in range(S):
        for i, j, d in pins.bonds(L, D):
            Jg[s, d, i] = eps[s, i] * J[s, d, i] * eps[s, j]
    hs, x = lat.sites()
    for obj in (lat, orc):
        obj.set_couplings(Jg)
        obj.set_sites(hs=hs * eps)
        obj.set_spins(ref.spins() * eps[:, None, :])
    for _ in range(4):
        for obj in (lat, orc, ref):
            obj.sweep(METROPOLIS, 0.7, 1)
        assert np.array_equal(lat.spins(), orc.spins())
        assert np.array_equal(lat.spins(), ref.spins() * eps[:, None, :])
    assert np.array_equal(lat.measure()[0], ref.measure()[0])


def test_rfim_zero_field_equals_ferromagnet(ianus):
    a = ianus.Lattice(dim=3, L=8, n_samples=70, n_replicas=2, seed=4, layout="bits64", disorder="rfim", field=0.0)
    b = ianus.Lattice(dim=3, L=8, n_samples=70, n_replicas=2, seed=4, layout="bits64", ferro=True)
    for algo in (METROPOLIS, HEATBATH):
        a.sweep(algo, 0.3, 6)
        b.sweep(algo, 0.3, 6)
    assert np.array_equal(a.spins(), b.spins())
    Ea, Ma, Qa = a.measure()
    Eb, Mb, Qb = b.measure()
    assert np.array_equal(Ea, Eb) and np.array_equal(Ma[..., 0], Mb) and np.array_equal(Qa, Qb)


def test_rfim_plain_and_bitsliced_agree(ianus):
    a = ianus.Lattice(dim=3, L=8, n_samples=40, n_replicas=2, seed=5, layout="i8", disorder="rfim", field=1.5)
    b = ianus.Lattice(dim=3, L=8, n_samples=40, n_replicas=2, seed=5, layout="bits64", disorder="rfim", field=1.5)
    for algo in (METROPOLIS, HEATBATH):
        a.sweep(algo, 0.7, 5)
        b.sweep(algo, 0.7, 5)
        assert np.array_equal(a.spins(), b.spins())
        for u, v in zip(a.measure(), b.measure()):
            assert np.array_equal(u, v)


@pytest.mark.parametrize("disorder,layout", LAYOUTS)
def test_field_checkpoint(ianus, disorder, layout):
    a, _ = _pair(ianus, disorder, dim=3, L=6, S=5, R=2, layout=layout, seed=9)
    hs, x = a.sites()
    a.set_sites(hs=-hs)  # the blob must carry the sites, not regenerate them
    a.sweep(HEATBATH, 0.9, 7)
    blob = a.get_state()
    a.sweep(HEATBATH, 0.9, 5)
    b, _ = _pair(ianus, disorder, dim=3, L=6, S=5, R=2, layout=layout, seed=9)
    b.set_state(blob)
    assert np.array_equal(b.sites()[0], -hs)
    b.sweep(HEATBATH, 0.9, 5)
    assert np.array_equal(a.spins(), b.spins())
    other, _ = _pair(ianus, disorder, dim=3, L=6, S=5, R=2, layout=layout, seed=9, h=0.5)
    with pytest.raises(ianus.IanusError):  # another |h|: not this lattice's state
        other.set_state(blob)


@pytest.mark.parametrize("disorder", [DIS_RFIM, DIS_DAFF])
def test_field_restore_into_a_running_lattice(ianus, disorder):
    """Two temperatures (per-lane field planes): a checkpoint restored into
    the lattice that wrote it replays the same continuation."""
    lat, _ = _pair(ianus, disorder, dim=3, L=6, S=70, R=2, K=2, layout="bits64", seed=12)
    beta = [0.7, 1.2]
    lat.sweep(HEATBATH, beta, 9)
    blob = lat.get_state()
    lat.sweep(HEATBATH, beta, 13)
    first = lat.spins()
    lat.set_state(blob)
    lat.sweep(HEATBATH, beta, 13)
    assert np.array_equal(lat.spins(), first)


def test_field_errors(ianus):
    lat, _ = _pair(ianus, DIS_RFIM, dim=3, L=4, S=3, K=2)
    lat.sweep(HEATBATH, [0.5, 0.6], 1)
    with pytest.raises(ianus.IanusError) as e:
        lat.pt_swap()
    assert e.value.status == ianus.EUNSUPPORTED
    with pytest.raises(ianus.IanusError) as e:
        lat.set_sites(hs=np.zeros((3, 64), dtype=np.int8))
    assert e.value.status == ianus.EINVAL
    bits, _ = _pair(ianus, DIS_RFIM, dim=3, L=4, S=3, layout="bits64")
    with pytest.raises(ianus.IanusError) as e:
        bits.set_sites(x=np.zeros((3, 64), dtype=np.int8))
    assert e.value.status == ianus.EUNSUPPORTED
    ea = ianus.Lattice(dim=3, L=4, n_samples=2)
    hs, x = ea.sites()
    assert np.all(hs == 1) and np.all(x == 1)
    with pytest.raises(ianus.IanusError):
        ea.set_sites(hs=hs)


def test_rfim_full_size_sampled(ianus):
    """RFIM 3D L = 64, 256 samples x 2 replicas, |h| = 2, heat bath at
    T = 2.5 on the bit-sliced layout: after 20 sweeps a sample of 24
    configurations (ragged lane positions) equals the oracle run of exactly
    those samples, and E_J, M, F, Q of every configuration equal the values
    recomputed from the downloaded spins."""
    L, S, R, h, beta = 64, 256, 2, 2.0, 1 / 2.5
    lat = ianus.Lattice(dim=3, L=L, n_samples=S, n_replicas=R, seed=SEED + 77, layout="bits64", disorder="rfim",
                        field=h)
    lat.sweep(HEATBATH, beta, 20)  # 2^21 site words: the specialised field kernel
    ids = [0, 1, 63, 64, 127, 128, 200, 255, 17, 99, 150, 230]
    orc = Oracle(dim=3, L=L, sample_ids=ids, n_replicas=R, seed=SEED + 77, disorder=DIS_RFIM, field=h)
    orc.sweep(HEATBATH, beta, 20, nthreads=8)
    sp = lat.spins()
    assert np.array_equal(sp[ids], orc.spins())
    E, M, Q = lat.measure()
    Eo, Mo, Qo = orc.measure()
    assert np.array_equal(E[ids], Eo) and np.array_equal(M[ids], Mo) and np.array_equal(Q[ids], Qo)
    hs, _ = lat.sites()
    s = sp.astype(np.int64)
    Ms = s.sum(axis=2)
    Fs = (s * hs[:, None, :]).sum(axis=2)
    assert np.array_equal(M[:, 0, :, 0], Ms) and np.array_equal(M[:, 0, :, 1], Fs)
    assert np.array_equal(Q[:, 0], (s[:, 0] * s[:, 1]).sum(axis=1))


def test_daff_plain_and_bitsliced_agree(ianus):
    kw = dict(dim=3, L=8, n_samples=70, n_replicas=2, seed=6, disorder="daff", field=1.25, occupation=0.65)
    a = ianus.Lattice(layout="i8", **kw)
    b = ianus.Lattice(layout="bits64", **kw)
    assert np.array_equal(a.sites()[1], b.sites()[1])
    for algo in (METROPOLIS, HEATBATH):
        a.sweep(algo, 0.6, 5)
        b.sweep(algo, 0.6, 5)
        assert np.array_equal(a.spins(), b.spins())
        for u, v in zip(a.measure(), b.measure()):
            assert np.array_equal(u, v)


def test_daff_full_size_sampled(ianus):
    """DAFF 3D L=64, 256 samples, occupation 0.7, |h|=1.0, Metropolis T=1.5 on
    the bit-sliced layout (the specialised kernel: 2^20 site words): a sample
    of configurations equals the oracle run of exactly those samples, and
    E_J, M, F of every configuration equal the values recomputed from the
    downloaded spins, sites and couplings."""
    L, S, h, occ, beta = 64, 256, 1.0, 0.7, 1 / 1.5
    lat = ianus.Lattice(dim=3, L=L, n_samples=S, seed=SEED + 78, layout="bits64", disorder="daff", field=h,
                        occupation=occ)
    lat.sweep(METROPOLIS, beta, 12)
    ids = [0, 1, 63, 64, 200, 255, 31]
    orc = Oracle(dim=3, L=L, sample_ids=ids, seed=SEED + 78, disorder=DIS_DAFF, field=h, occupation=occ)
    orc.sweep(METROPOLIS, beta, 12, nthreads=8)
    sp = lat.spins()
    assert np.array_equal(sp[ids], orc.spins())
    E, M, _ = lat.measure(overlap=False)
    Eo, Mo, _ = orc.measure()
    assert np.array_equal(E[ids], Eo) and np.array_equal(M[ids], Mo)
    hs, x = lat.sites()
    s = sp[:, 0].astype(np.int64) * x
    assert np.array_equal(M[:, 0, 0, 0], s.sum(axis=1))
    assert np.array_equal(M[:, 0, 0, 1], (s * hs).sum(axis=1))
    idx = np.arange(L ** 3)
    coords = [(idx // L ** d) % L for d in range(3)]
    EJ = np.zeros(S, dtype=np.int64)
    for d in range(3):
        c = [q.copy() for q in coords]
        c[d] = (c[d] + 1) % L
        j = c[0] + L * (c[1] + L * c[2])
        EJ += (s * s[:, j]).sum(axis=1)  # J = -1: E_J = + sum x x s s
    assert np.array_equal(E[:, 0, 0], EJ)
