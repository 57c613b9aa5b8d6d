"""Pins of the oracle's Ising-like models with fields and dilution (Eq. 2).

The random-field Ising model (RFIM: J = +1, h_i = +-|h|) and the diluted
antiferromagnet in a field (DAFF: J = -1, h_i = +|h|, x_i = 0 or 1) are the
other instances of the Hamiltonian of Eq. (2) that Sec. 2.1 lists.  Each test
checks the oracle against something the mathematics fixes:
* the field-sign and dilution streams against an independent Philox;
* exact enumeration (N = 8): the quantised one-sweep transition matrix has
  the Boltzmann distribution of E = E_J - |h| F as stationary vector on every
  closed class (empty sites are frozen), and the oracle's own chain
  reproduces the enumerated histogram;
* incremental bookkeeping of E_J and F against recomputation;
* symmetries that hold bit for bit: global flip (s, h) -> (-s, -h), gauge
  (J, h, s) -> (e J e, e h, e s), RFIM at h = 0 equals the ferromagnet, the
  fully occupied DAFF at h = 0 equals the ferromagnet under the staggered
  gauge;
* the closed form of the 1D chain in a uniform field (transfer matrix) and of
  independent spins in a field (<h s> = |h| tanh(beta |h|));
* beta -> infinity Metropolis never raises E_J - |h| F.
"""

import math

import numpy as np
import pytest

import oracle
from oracle import DIS_DAFF, DIS_FERRO, DIS_RFIM, HEATBATH, METROPOLIS, Oracle
from tests import pins
from tests.test_oracle_physics import _chi2, _closed_classes, _stationary

SEED = 0x0704357300000F00


def _field_sign_ref(seed, sample, site):
    x = pins.philox4x32_10([site, 0, (7 << 28) | (sample >> 6), 0], pins.key_of(seed))
    return ((x[0] | (x[1] << 32)) >> (sample & 63)) & 1


def _occupation_random_ref(seed, sample, site):
    r = 0
    for p in range(32):
        m = p >> 1
        x = pins.philox4x32_10([site, 0, (8 << 28) | (m << 24) | (sample >> 6), 0], pins.key_of(seed))
        w = (x[2] | (x[3] << 32)) if p & 1 else (x[0] | (x[1] << 32))
        r |= ((w >> (sample & 63)) & 1) << (31 - p)
    return r


def _terms(s, J, hs, x, L, D):
    """(E_J, M, F) of one configuration, written out from Eq. (2)."""
    EJ = 0
    for i, j, d in pins.bonds(L, D):
        EJ -= int(J[d][i]) * int(x[i]) * int(x[j]) * int(s[i]) * int(s[j])
    M = int(sum(int(x[i]) * int(s[i]) for i in range(len(s))))
    F = int(sum(int(hs[i]) * int(x[i]) * int(s[i]) for i in range(len(s))))
    return EJ, M, F


# ---------------- streams ----------------

def test_field_and_dilution_streams_match_independent_philox():
    for s in (0, 1, 63, 64, 200):
        for i in (0, 1, 17, 511, 4096):
            assert oracle.field_sign_bit(SEED, s, i) == _field_sign_ref(SEED, s, i)
            assert oracle.occupation_random(SEED, s, i) == _occupation_random_ref(SEED, s, i)


def test_sites_follow_the_streams():
    L, D, p = 4, 3, 0.6
    ids = [0, 5, 70]
    r = Oracle(dim=D, L=L, sample_ids=ids, seed=SEED, disorder=DIS_RFIM, field=0.7)
    hs, x = r.sites()
    assert np.all(x == 1) and np.all(r.couplings() == 1)
    d = Oracle(dim=D, L=L, sample_ids=ids, seed=SEED, disorder=DIS_DAFF, field=0.7, occupation=p)
    hs_d, x_d = d.sites()
    assert np.all(hs_d == 1) and np.all(d.couplings() == -1)
    T = math.floor(math.ldexp(p, 32))
    for si, s in enumerate(ids):
        for i in range(0, L ** D, 7):
            assert hs[si, i] == (-1 if _field_sign_ref(SEED, s, i) else 1)
            assert x_d[si, i] == (1 if _occupation_random_ref(SEED, s, i) < T else 0)


def test_occupation_fraction_and_edges():
    L, D, p = 8, 3, 0.6
    d = Oracle(dim=D, L=L, sample_ids=list(range(8)), seed=SEED + 1, disorder=DIS_DAFF, field=0.0, occupation=p)
    _, x = d.sites()
    n = x.size
    assert abs(x.mean() - p) < 5 * math.sqrt(p * (1 - p) / n)
    # field signs: a fair coin
    r = Oracle(dim=D, L=L, sample_ids=list(range(8)), seed=SEED + 1, disorder=DIS_RFIM, field=1.0)
    hs, _ = r.sites()
    assert abs(hs.mean()) < 5 / math.sqrt(hs.size)
    assert np.all(Oracle(dim=2, L=4, disorder=DIS_DAFF, occupation=1.0, seed=SEED).sites()[1] == 1)
    assert np.all(Oracle(dim=2, L=4, disorder=DIS_DAFF, occupation=0.0, seed=SEED).sites()[1] == 0)


def test_invalid_field_parameters_rejected():
    with pytest.raises(ValueError):
        Oracle(disorder=DIS_RFIM, field=-1.0)
    with pytest.raises(ValueError):
        Oracle(disorder=DIS_DAFF, occupation=1.5)


# ---------------- bookkeeping and measurements ----------------

@pytest.mark.parametrize("disorder,field,occ,algo,dim,L", [
    (DIS_RFIM, 0.7, 1.0, METROPOLIS, 3, 4), (DIS_RFIM, 1.3, 1.0, HEATBATH, 3, 4), (DIS_RFIM, 2.0, 1.0, HEATBATH, 2, 6),
    (DIS_DAFF, 0.5, 0.7, METROPOLIS, 3, 4), (DIS_DAFF, 1.5, 0.6, HEATBATH, 3, 2), (DIS_DAFF, 0.0, 0.8, HEATBATH, 2, 6)])
def test_field_bookkeeping_and_measurements(disorder, field, occ, algo, dim, L):
    o = Oracle(dim=dim, L=L, sample_ids=[0, 5, 70], n_replicas=2, seed=SEED + 2, disorder=disorder, field=field,
               occupation=occ)
    J = o.couplings()
    hs, x = o.sites()
    for _ in range(5):
        o.sweep(algo, 0.8, 1, measure_every=1)
        assert o.bookkeeping_error() == 0
    sp = o.spins()
    E, M, Q = o.measure()
    assert M.shape == (3, 1, 2, 2)
    for s in range(3):
        for a in range(2):
            EJ, Mv, F = _terms(sp[s, a], J[s], hs[s], x[s], L, dim)
            assert (E[s, 0, a], M[s, 0, a, 0], M[s, 0, a, 1]) == (EJ, Mv, F)
        assert Q[s, 0] == int((x[s].astype(np.int64) * sp[s, 0] * sp[s, 1]).sum())
    sw, Es, Ms, _ = o.series()
    assert Ms.shape == (5, 3, 1, 2, 2) and np.array_equal(Es[-1], E) and np.array_equal(Ms[-1], M)


def test_empty_sites_never_change():
    o = Oracle(dim=3, L=4, sample_ids=[0, 1], n_replicas=2, seed=SEED + 3, disorder=DIS_DAFF, field=0.9,
               occupation=0.5)
    _, x = o.sites()
    before = o.spins()
    o.sweep(HEATBATH, 0.0, 6)  # beta = 0: occupied spins flip half the time
    after = o.spins()
    empty = (x == 0)[:, None, :].repeat(2, axis=1)
    assert np.array_equal(before[empty], after[empty])
    assert (before[~empty] != after[~empty]).mean() > 0.3


# ---------------- exact enumeration ----------------

def _field_sweep_matrix(J, hs, x, h, L, D, algo, beta):
    """Exact one-sweep transition matrix of the quantised rule with fields."""
    N = L ** D
    n = 2 ** N
    states = np.array([[1 - 2 * ((k >> i) & 1) for i in range(N)] for k in range(n)], dtype=np.int64)
    nb = [[] for _ in range(N)]
    for i, j, d in pins.bonds(L, D):
        nb[i].append((j, int(J[d][i])))
        nb[j].append((i, int(J[d][i])))
    P = np.eye(n)
    for c in (0, 1):
        for i in range(N):
            if pins.colour_of(i, L, D) != c or not x[i]:
                continue
            Ki = np.zeros((n, n))
            for k in range(n):
                s = states[k]
                v = int(s[i]) * sum(Jij * int(x[j]) * int(s[j]) for j, Jij in nb[i])
                w = 0.0 if h == 0 else (h if s[i] * hs[i] > 0 else -h)
                xx = v + w
                if algo == METROPOLIS:
                    pf = 1.0 if 2 * xx <= 0 else oracle.table_metropolis_x(beta, xx) / 2.0 ** 32
                else:
                    pf = 1.0 - oracle.table_heatbath_x(beta, xx) / 2.0 ** 32
                Ki[k, k ^ (1 << i)] += pf
                Ki[k, k] += 1.0 - pf
            P = P @ Ki
    E = np.zeros(n)
    for k in range(n):
        EJ, _, F = _terms(states[k], J, hs, x, L, D)
        E[k] = EJ - h * F
    return P, E


def _check_stationary(P, E, beta, p_min):
    tol = max(1e-10, 4.0 * 2.0 ** -32 / p_min)
    boltz = np.exp(-beta * (E - E.min()))
    for cls in _closed_classes(P):
        sub = P[np.ix_(cls, cls)]
        assert np.allclose(sub.sum(axis=1), 1.0)
        pi = _stationary(sub)
        b = boltz[cls] / boltz[cls].sum()
        assert np.max(np.abs(pi - b) / b) < tol


@pytest.mark.parametrize("disorder,h,occ,algo,beta", [
    (DIS_RFIM, 0.5, 1.0, METROPOLIS, 0.35), (DIS_RFIM, 0.5, 1.0, HEATBATH, 0.35),
    (DIS_RFIM, 1.25, 1.0, HEATBATH, 0.8), (DIS_RFIM, 2.0, 1.0, METROPOLIS, 0.6),
    (DIS_DAFF, 0.75, 0.7, METROPOLIS, 0.5), (DIS_DAFF, 0.75, 0.7, HEATBATH, 0.5)])
def test_field_exact_stationary(disorder, h, occ, algo, beta):
    o = Oracle(dim=3, L=2, sample_ids=[3], seed=SEED + 4, disorder=disorder, field=h, occupation=occ)
    J = o.couplings()[0]
    hs, x = o.sites()
    if disorder == DIS_DAFF:
        assert 0 < x.sum() < 8  # some sites empty, some occupied
    else:
        assert 0 < (hs[0] > 0).sum() < 8  # both field signs present
    P, E = _field_sweep_matrix(J, hs[0], x[0], h, 2, 3, algo, beta)
    assert np.allclose(P.sum(axis=1), 1.0)
    xmax = 6 + h
    p_min = min(math.exp(-beta * 2 * xmax), 1.0 / (1.0 + math.exp(2 * beta * xmax)))
    _check_stationary(P, E, beta, p_min)


@pytest.mark.parametrize("disorder,h,occ,algo", [(DIS_RFIM, 0.75, 1.0, METROPOLIS), (DIS_RFIM, 0.75, 1.0, HEATBATH),
                                                (DIS_DAFF, 0.5, 0.75, HEATBATH)])
def test_field_chain_matches_boltzmann_N8(disorder, h, occ, algo):
    """The oracle's own chain (streams, field sign, dilution, decision)
    reproduces the enumerated Boltzmann weights of E_J - |h| F."""
    beta = 0.35
    o = Oracle(dim=3, L=2, sample_ids=[5], seed=SEED + 5, disorder=disorder, field=h, occupation=occ)
    J = o.couplings()[0]
    hs, x = o.sites()
    s0 = o.spins()[0, 0]
    states = np.array([[1 - 2 * ((k >> i) & 1) for i in range(8)] for k in range(256)], dtype=np.int64)
    # the chain lives on the states whose empty sites keep their initial spins
    ok = np.all((states == s0[None, :]) | (x[0][None, :] == 1), axis=1)
    E = np.array([_terms(st, J, hs[0], x[0], 2, 3)[0] - h * _terms(st, J, hs[0], x[0], 2, 3)[2] for st in states])
    p = np.where(ok, np.exp(-beta * (E - E.min())), 0.0)
    p /= p.sum()
    w = 1 << np.arange(8)
    hist = np.zeros(256, dtype=np.int64)
    for _ in range(50000):
        o.sweep(algo, beta, 1)
        hist[int(((1 - o.spins()[0, 0]) // 2 * w).sum())] += 1
    assert hist[~ok].sum() == 0
    chi2, dof = _chi2(hist, p)
    assert chi2 / dof < 1.6, (chi2, dof)


# ---------------- symmetries, bit for bit ----------------

@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
def test_global_flip_symmetry(algo):
    L, D = 4, 3
    a = Oracle(dim=D, L=L, sample_ids=[1, 66], n_replicas=2, seed=SEED + 6, disorder=DIS_RFIM, field=0.9)
    b = Oracle(dim=D, L=L, sample_ids=[1, 66], n_replicas=2, seed=SEED + 6, disorder=DIS_RFIM, field=0.9)
    hs, _ = a.sites()
    b.set_sites(hs=-hs)
    b.set_spins(-a.spins())
    for _ in range(6):
        a.sweep(algo, 0.7, 1)
        b.sweep(algo, 0.7, 1)
        assert np.array_equal(b.spins(), -a.spins())
        Ea, Ma, _ = a.measure()
        Eb, Mb, _ = b.measure()
        assert np.array_equal(Ea, Eb)
        assert np.array_equal(Mb[..., 0], -Ma[..., 0]) and np.array_equal(Mb[..., 1], Ma[..., 1])


@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
@pytest.mark.parametrize("disorder", [DIS_RFIM, DIS_DAFF])
def test_gauge_invariance_with_fields(algo, disorder):
    L, D = 4, 3
    N = L ** D
    eps = np.random.default_rng(5).choice([-1, 1], size=(2, N)).astype(np.int8)
    kw = dict(dim=D, L=L, sample_ids=[2, 9], n_replicas=2, seed=SEED + 7, disorder=disorder, field=1.1,
              occupation=0.7)
    a, b = Oracle(**kw), Oracle(**kw)
    J = a.couplings()
    Jg = J.copy()
    for s in range(2):
        for i, j, d in pins.bonds(L, D):
            Jg[s, d, i] = eps[s, i] * J[s, d, i] * eps[s, j]
    hs, _ = a.sites()
    b.set_couplings(Jg)
    b.set_sites(hs=hs * eps)
    b.set_spins(a.spins() * eps[:, None, :])
    for _ in range(6):
        a.sweep(algo, 0.6, 1)
        b.sweep(algo, 0.6, 1)
        assert np.array_equal(b.spins(), a.spins() * eps[:, None, :])
        Ea, Ma, Qa = a.measure()
        Eb, Mb, Qb = b.measure()
        assert np.array_equal(Ea, Eb) and np.array_equal(Ma[..., 1], Mb[..., 1]) and np.array_equal(Qa, Qb)


@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
def test_rfim_zero_field_is_the_ferromagnet(algo):
    kw = dict(dim=3, L=4, sample_ids=[0, 3], n_replicas=2, seed=SEED + 8)
    a = Oracle(disorder=DIS_RFIM, field=0.0, **kw)
    b = Oracle(disorder=DIS_FERRO, **kw)
    a.sweep(algo, 0.4, 7)
    b.sweep(algo, 0.4, 7)
    assert np.array_equal(a.spins(), b.spins())
    Ea, Ma, Qa = a.measure()
    Eb, Mb, Qb = b.measure()
    assert np.array_equal(Ea, Eb) and np.array_equal(Ma[..., 0], Mb) and np.array_equal(Qa, Qb)


@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
def test_full_daff_zero_field_is_the_staggered_ferromagnet(algo):
    """J = -1 on a bipartite lattice: e_i = (-1)^colour(i) maps it onto J = +1."""
    L, D = 4, 3
    N = L ** D
    eps = np.array([1 - 2 * pins.colour_of(i, L, D) for i in range(N)], dtype=np.int8)
    kw = dict(dim=D, L=L, sample_ids=[0, 3], n_replicas=2, seed=SEED + 9)
    a = Oracle(disorder=DIS_DAFF, field=0.0, occupation=1.0, **kw)
    b = Oracle(disorder=DIS_FERRO, **kw)
    b.set_spins(a.spins() * eps[None, None, :])
    for _ in range(5):
        a.sweep(algo, 0.5, 1)
        b.sweep(algo, 0.5, 1)
        assert np.array_equal(b.spins(), a.spins() * eps[None, None, :])
        assert np.array_equal(a.measure()[0], b.measure()[0])


# ---------------- closed forms ----------------

def _chain_lnZ(beta, J, h, N):
    """ln Z of the periodic 1D Ising chain in a uniform field (transfer matrix)."""
    T = np.array([[math.exp(beta * (J + h)), math.exp(-beta * J)],
                  [math.exp(-beta * J), math.exp(beta * (J - h))]])
    lam = np.linalg.eigvalsh(T)
    return math.log(lam[1] ** N + lam[0] ** N)


@pytest.mark.parametrize("algo,beta,h", [(HEATBATH, 0.5, 0.3), (METROPOLIS, 0.7, 0.6), (HEATBATH, 1.0, 0.25)])
def test_1d_chain_in_uniform_field(algo, beta, h):
    """<sum s_i s_i+1> and <sum s_i> of the 1D chain against the transfer
    matrix: (1/beta) d lnZ / dJ and (1/beta) d lnZ / dh at J = 1."""
    L = 16
    o = Oracle(dim=1, L=L, sample_ids=list(range(8)), seed=SEED + 10, disorder=DIS_RFIM, field=h)
    o.set_sites(hs=np.ones((8, L), dtype=np.int8))  # uniform field h_i = +|h|
    o.sweep(algo, beta, 200, nthreads=4)
    o.clear_series()
    o.sweep(algo, beta, 6000, measure_every=1, nthreads=4)
    _, E, M, _ = o.series()
    eps = 1e-6
    bond = (_chain_lnZ(beta, 1 + eps, h, L) - _chain_lnZ(beta, 1 - eps, h, L)) / (2 * eps * beta)
    mag = (_chain_lnZ(beta, 1, h + eps, L) - _chain_lnZ(beta, 1, h - eps, L)) / (2 * eps * beta)
    e = (-E[:, :, 0, 0]).astype(np.float64).mean(axis=1)
    f = M[:, :, 0, 0, 1].astype(np.float64).mean(axis=1)
    assert np.array_equal(M[..., 0], M[..., 1])  # all field signs +
    for series, exact in ((e, bond), (f, mag)):
        mean, err = pins.batch_mean_error(series, nbatch=20)
        assert abs(mean - exact) < 4 * err + 1e-3, (mean, exact, err)


@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
def test_free_spins_in_random_field(algo):
    """With every J = 0 each spin is alone in its field: <sign(h_i) s_i> =
    tanh(beta |h|), whatever the field signs."""
    L, D, beta, h = 8, 3, 0.6, 0.8
    o = Oracle(dim=D, L=L, sample_ids=[0, 1], seed=SEED + 11, disorder=DIS_RFIM, field=h)
    o.set_couplings(np.zeros((2, D, L ** D), dtype=np.int8))
    o.sweep(algo, beta, 20)
    o.clear_series()
    o.sweep(algo, beta, 400, measure_every=1)
    _, _, M, _ = o.series()
    f = M[:, :, 0, 0, 1].astype(np.float64).ravel() / L ** D
    mean, err = pins.batch_mean_error(f, nbatch=20)
    assert abs(mean - math.tanh(beta * h)) < 4 * err + 1e-3, (mean, math.tanh(beta * h), err)


@pytest.mark.parametrize("disorder", [DIS_RFIM, DIS_DAFF])
def test_zero_temperature_never_raises_energy(disorder):
    h = 1.5
    o = Oracle(dim=3, L=6, sample_ids=[0, 1], seed=SEED + 12, disorder=disorder, field=h, occupation=0.7)
    E0, M0, _ = o.measure()
    o.sweep(METROPOLIS, 50.0, 25, measure_every=1)
    _, E, M, _ = o.series()
    tot = np.concatenate([(E0 - h * M0[..., 1])[None], E - h * M[..., 1]])[:, :, 0, 0]
    assert np.all(np.diff(tot, axis=0) <= 0)
    assert tot[-1].max() < tot[0].max()
