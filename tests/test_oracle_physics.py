"""Physics pins of the oracle's sweep, measurements and parallel tempering.

Each test checks the oracle against something the paper or the mathematics
fixes, not against itself:
* exact enumeration: the quantised one-sweep transition matrix has the
  Boltzmann distribution of Eq. (1) as its stationary vector, and the
  oracle's own long chains reproduce the enumerated Boltzmann histograms;
* incremental energy bookkeeping (sum of the update rule's dE) equals the
  energy recomputed from Eq. (2) after every sweep;
* exact gauge invariance of the EA model, bit for bit;
* the 2D ferromagnet against Onsager's closed-form energy;
* beta = 0 heat bath reduces to "flip iff plane 0 of the stream is 1",
  checked against an independent Philox;
* beta -> infinity Metropolis never raises the energy;
* the q = 2 Potts energy equals (E_Ising - sum J)/2 on the same configuration;
* parallel tempering keeps a permutation, conserves the energy multiset, and
  accepts with frequency T_PT / 2^32.
"""

import math

import numpy as np
import pytest

import oracle
from oracle import HEATBATH, METROPOLIS, MODEL_ISING, MODEL_POTTS, Oracle
from tests import pins

SEED = 0x0704357300000000


# ---------------- bookkeeping ----------------

@pytest.mark.parametrize("model,dim,L,algo", [
    (MODEL_ISING, 3, 2, METROPOLIS), (MODEL_ISING, 3, 4, HEATBATH), (MODEL_ISING, 2, 6, METROPOLIS),
    (MODEL_ISING, 2, 2, HEATBATH), (MODEL_ISING, 3, 6, METROPOLIS), (MODEL_POTTS, 3, 4, HEATBATH),
    (MODEL_POTTS, 2, 2, HEATBATH), (MODEL_POTTS, 2, 6, HEATBATH)])
def test_energy_bookkeeping(model, dim, L, algo):
    o = Oracle(model=model, dim=dim, L=L, sample_ids=[0, 5, 70], n_replicas=2, seed=SEED + 9)
    for _ in range(6):
        o.sweep(algo, 0.9, 1)
        assert o.bookkeeping_error() == 0
    # the oracle's energy agrees with an independent energy function, and
    # M and Q with their definitions written out on the read-back spins
    sp, J = o.spins(), o.couplings()
    E, M, Q = o.measure()
    for s in range(o.S):
        for a in range(2):
            if model == MODEL_ISING:
                ref = pins.ising_energy(sp[s, a], J[s], L, dim)
                assert M[s, 0, a] == int(sp[s, a].astype(np.int64).sum())
            else:
                ref = pins.potts_energy(sp[s, a], J[s], L, dim)
                assert np.array_equal(M[s, 0, a], np.bincount(sp[s, a], minlength=4))
            assert E[s, 0, a] == ref
        if model == MODEL_ISING:
            assert Q[s, 0] == int((sp[s, 0].astype(np.int64) * sp[s, 1]).sum())
        else:
            assert Q[s, 0] == int((sp[s, 0] == sp[s, 1]).sum())


# ---------------- exact enumeration ----------------

def _ising_tables(algo, beta, D):
    if algo == METROPOLIS:
        return {dE: oracle.table_metropolis(beta, dE) for dE in range(4, 4 * D + 1, 4)}
    return {x: oracle.table_heatbath(beta, x) for x in range(-2 * D, 2 * D + 1, 2)}


def _enumerate_ising(J, L, D):
    N = L ** D
    states = np.array([[1 - 2 * ((k >> i) & 1) for i in range(N)] for k in range(2 ** N)], dtype=np.int64)
    E = np.array([pins.ising_energy(s, J, L, D) for s in states], dtype=np.float64)
    return states, E


def _ising_sweep_matrix(J, L, D, algo, beta):
    """Exact one-sweep transition matrix of the quantised update rule:
    colour 0 sites, then colour 1 sites; flip probability T / 2^32."""
    N = L ** D
    n = 2 ** N
    states, _ = _enumerate_ising(J, L, D)
    tab = _ising_tables(algo, beta, D)
    bl = pins.bonds(L, D)
    nb = [[] for _ in range(N)]
    for i, j, d in bl:
        nb[i].append((j, int(J[d][i])))
        nb[j].append((i, int(J[d][i])))
    P = np.eye(n)
    for c in (0, 1):
        for i in range(N):
            if pins.colour_of(i, L, D) != c:
                continue
            Ki = np.zeros((n, n))
            for k in range(n):
                s = states[k]
                u = sum(1 for j, Jij in nb[i] if Jij * s[i] * s[j] == -1)
                if algo == METROPOLIS:
                    dE = 4 * D - 4 * u
                    pf = 1.0 if dE <= 0 else tab[dE] / 2.0 ** 32
                else:
                    pf = 1.0 - tab[2 * D - 2 * u] / 2.0 ** 32
                Ki[k, k ^ (1 << i)] += pf
                Ki[k, k] += 1.0 - pf
            P = P @ Ki
    return P


def _stationary(P):
    w, v = np.linalg.eig(P.T)
    pi = np.real(v[:, np.argmin(np.abs(w - 1.0))])
    return pi / pi.sum()


def _closed_classes(P):
    """Communicating classes of the chain.  The Metropolis rule flips a site
    with zero local field (dE = 0) with probability 1, so on tiny lattices a
    site whose field stays zero flips every sweep and the state space splits
    into closed classes; Boltzmann weights restricted to each class must then
    be stationary on that class."""
    n = P.shape[0]
    A = (P > 0).astype(np.int64)
    reach = np.eye(n, dtype=bool)
    for _ in range(n):
        new = reach | ((reach.astype(np.int64) @ A) > 0)
        if np.array_equal(new, reach):
            break
        reach = new
    classes, seen = [], np.zeros(n, dtype=bool)
    for k in range(n):
        if seen[k]:
            continue
        cls = np.where(reach[k] & reach[:, k])[0]
        seen[cls] = True
        classes.append(cls)
    return classes


def _check_boltzmann_stationary(P, E, beta, p_min):
    """Stationary vector vs Boltzmann weights.  Each acceptance probability p
    is applied as floor(2^32 p)/2^32, a relative error of at most 2^-32/p, so
    the tolerance is a small multiple of that for the smallest p in use."""
    tol = max(1e-10, 4.0 * 2.0 ** -32 / p_min)
    boltz = np.exp(-beta * (E - E.min()))
    for cls in _closed_classes(P):
        sub = P[np.ix_(cls, cls)]
        assert np.allclose(sub.sum(axis=1), 1.0)  # closed: no probability leaves
        pi = _stationary(sub)
        b = boltz[cls] / boltz[cls].sum()
        assert np.max(np.abs(pi - b) / b) < tol


@pytest.mark.parametrize("algo,beta", [(METROPOLIS, 0.35), (HEATBATH, 0.35), (METROPOLIS, 1.1), (HEATBATH, 0.9)])
def test_ising_exact_stationary(algo, beta):
    o = Oracle(dim=3, L=2, sample_ids=[3], seed=SEED + 1)
    J = o.couplings()[0]
    P = _ising_sweep_matrix(J, 2, 3, algo, beta)
    assert np.allclose(P.sum(axis=1), 1.0)
    _, E = _enumerate_ising(J, 2, 3)
    p_min = min(math.exp(-beta * 12), 1.0 / (1.0 + math.exp(2 * beta * 6)))
    _check_boltzmann_stationary(P, E, beta, p_min)
    if algo == HEATBATH:  # 0 < p < 1 everywhere: a single class
        assert len(_closed_classes(P)) == 1


def _chain_histogram(o, algo, beta, nsweeps, nstates, encode):
    hist = np.zeros(nstates, dtype=np.int64)
    for _ in range(nsweeps):
        o.sweep(algo, beta, 1)
        hist[encode(o.spins()[0, 0])] += 1
    return hist


def _chi2(hist, p):
    n = hist.sum()
    e = n * p
    m = e > 5
    return float(((hist[m] - e[m]) ** 2 / e[m]).sum()), int(m.sum()) - 1


@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
def test_ising_chain_matches_boltzmann_N8(algo):
    """The oracle's own chain (stream, neighbour and bond indexing, decision)
    reproduces the enumerated Boltzmann weights of the 3D L=2 glass."""
    beta = 0.3
    o = Oracle(dim=3, L=2, sample_ids=[3], seed=SEED + 2)
    J = o.couplings()[0]
    _, E = _enumerate_ising(J, 2, 3)
    p = np.exp(-beta * (E - E.min()))
    p /= p.sum()
    w = 1 << np.arange(8)
    hist = _chain_histogram(o, algo, beta, 60000, 256, lambda s: int(((1 - s) // 2 * w).sum()))
    chi2, dof = _chi2(hist, p)
    assert chi2 / dof < 1.6, (chi2, dof)


@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
def test_ising_energy_histogram_N16(algo):
    """2D L=4 (N=16, 65536 states): energy histogram of a long oracle run
    against the exactly enumerated distribution P(E)."""
    beta = 0.4
    o = Oracle(dim=2, L=4, sample_ids=[1, 2, 3, 4], seed=SEED + 3)
    J = o.couplings()
    o.sweep(algo, beta, 40000, measure_every=1, nthreads=4)
    _, Es, _, _ = o.series()
    N = 16
    ks = np.arange(2 ** N)
    states = 1 - 2 * ((ks[:, None] >> np.arange(N)[None, :]) & 1)
    for s in range(4):
        E = np.zeros(2 ** N, dtype=np.int64)
        for i, j, d in pins.bonds(4, 2):
            E -= int(J[s][d][i]) * states[:, i] * states[:, j]
        levels = np.unique(E)
        w = np.exp(-beta * (E - E.min()).astype(np.float64))
        pE = np.array([w[E == e].sum() for e in levels]) / w.sum()
        h = np.array([(Es[:, s, 0, 0] == e).sum() for e in levels])
        assert h.sum() == len(Es)
        chi2, dof = _chi2(h, pE)
        assert chi2 / max(dof, 1) < 3.0, (s, chi2, dof)


# ---------------- Potts enumeration ----------------

def _potts_sweep_matrix(J, L, D, beta, q=4):
    N = L ** D
    n = q ** N
    states = np.array([[(k // q ** i) % q for i in range(N)] for k in range(n)])
    nb = [[] for _ in range(N)]
    for i, j, d in pins.bonds(L, D):
        nb[i].append((j, int(J[d][i])))
        nb[j].append((i, int(J[d][i])))
    P = np.eye(n)
    cache = {}
    for c in (0, 1):
        for i in range(N):
            if pins.colour_of(i, L, D) != c:
                continue
            Ki = np.zeros((n, n))
            for k in range(n):
                s = states[k]
                cnt = [0] * q
                for j, Jij in nb[i]:
                    cnt[s[j]] += Jij
                key = tuple(cnt)
                if key not in cache:
                    cache[key] = oracle.table_potts(beta, cnt)
                T = [0] + cache[key] + [2 ** 32]
                for knew in range(q):
                    pk = (T[knew + 1] - T[knew]) / 2.0 ** 32
                    k2 = k + (knew - s[i]) * q ** i
                    Ki[k, k2] += pk
            P = P @ Ki
    return P, states


@pytest.mark.parametrize("beta", [0.5, 1.25])
def test_potts_exact_stationary(beta):
    o = Oracle(model=MODEL_POTTS, dim=2, L=2, sample_ids=[6], seed=SEED + 4)
    J = o.couplings()[0]
    P, states = _potts_sweep_matrix(J, 2, 2, beta)
    E = np.array([pins.potts_energy(s, J, 2, 2) for s in states], dtype=np.float64)
    p_min = 1.0 / (1.0 + 3.0 * math.exp(beta * 8))  # smallest state weight share, n in -4..4
    _check_boltzmann_stationary(P, E, beta, p_min)
    assert len(_closed_classes(P)) == 1


def test_potts_chain_matches_boltzmann():
    beta = 0.7
    o = Oracle(model=MODEL_POTTS, dim=2, L=2, sample_ids=[6], seed=SEED + 5)
    J = o.couplings()[0]
    states = np.array([[(k // 4 ** i) % 4 for i in range(4)] for k in range(256)])
    E = np.array([pins.potts_energy(s, J, 2, 2) for s in states], dtype=np.float64)
    p = np.exp(-beta * (E - E.min()))
    p /= p.sum()
    w = 4 ** np.arange(4)
    hist = _chain_histogram(o, HEATBATH, beta, 60000, 256, lambda s: int((s.astype(np.int64) * w).sum()))
    chi2, dof = _chi2(hist, p)
    assert chi2 / dof < 1.6, (chi2, dof)


@pytest.mark.parametrize("dim,L", [(2, 6), (3, 4)])
def test_potts_beta_zero_takes_the_top_bits_of_the_stream(dim, L):
    """At beta = 0 the cumulative thresholds are (k + 1) 2^30, so the new
    state is the top two bits of the site's POTTS word: this fixes the state
    order of the cumulative selection, which the Boltzmann pins cannot see."""
    ids = [0, 5, 70]
    o = Oracle(model=MODEL_POTTS, dim=dim, L=L, sample_ids=ids, n_replicas=2, seed=SEED + 17)
    o.sweep(HEATBATH, 0.0, 1)
    sp = o.spins()
    key = pins.key_of(SEED + 17)
    for k, s in enumerate(ids):
        for slot in range(2):
            for i in range(L ** dim):
                x = pins.philox4x32_10([i, 0, (4 << 28) | (slot << 16) | (s >> 2), 0], key)
                assert sp[k, slot, i] == x[s & 3] >> 30


def test_potts_q2_energy_reduction():
    """delta(s, s') = (1 + sigma sigma')/2 with sigma = 1 - 2s, so
    E_Potts(q=2) = (E_Ising(sigma) - sum J) / 2 exactly."""
    rng = np.random.default_rng(5)
    for dim, L in ((2, 4), (3, 4), (3, 2)):
        o_p = Oracle(model=MODEL_POTTS, q=2, dim=dim, L=L, sample_ids=[0, 1], seed=SEED + 6)
        o_i = Oracle(model=MODEL_ISING, dim=dim, L=L, sample_ids=[0, 1], seed=SEED + 6)
        J = o_i.couplings()
        assert np.array_equal(J, o_p.couplings())
        st = rng.integers(0, 2, size=(2, 1, L ** dim)).astype(np.int8)
        o_p.set_spins(st)
        o_i.set_spins((1 - 2 * st).astype(np.int8))
        Ep, _, _ = o_p.measure()
        Ei, _, _ = o_i.measure()
        for s in range(2):
            assert 2 * Ep[s, 0, 0] == Ei[s, 0, 0] - int(J[s].astype(np.int64).sum())


# ---------------- gauge invariance ----------------

@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
@pytest.mark.parametrize("dim,L", [(3, 4), (2, 6), (3, 2)])
def test_gauge_invariance_bit_for_bit(algo, dim, L):
    """J'_ij = e_i J_ij e_j, s'_i(0) = e_i s_i(0) with the same seed gives
    s'_i(t) = e_i s_i(t) after every sweep, and equal E and Q."""
    N = L ** dim
    rng = np.random.default_rng(17)
    a = Oracle(dim=dim, L=L, sample_ids=[2, 65], n_replicas=2, seed=SEED + 7)
    b = Oracle(dim=dim, L=L, sample_ids=[2, 65], n_replicas=2, seed=SEED + 7)
    eps = rng.choice([-1, 1], size=(2, N)).astype(np.int8)
    J = a.couplings()
    Jg = J.copy()
    for s in range(2):
        for i, j, d in pins.bonds(L, dim):
            Jg[s, d, i] = eps[s, i] * J[s, d, i] * eps[s, j]
    b.set_couplings(Jg)
    b.set_spins(a.spins() * eps[:, None, :])
    for _ in range(8):
        a.sweep(algo, 0.8, 1)
        b.sweep(algo, 0.8, 1)
        assert np.array_equal(b.spins(), a.spins() * eps[:, None, :])
        Ea, _, Qa = a.measure()
        Eb, _, Qb = b.measure()
        assert np.array_equal(Ea, Eb)
        # the overlap of gauge-transformed replicas is invariant too
        assert np.array_equal(Qa, Qb)


# ---------------- closed forms ----------------

@pytest.mark.parametrize("algo,T", [(METROPOLIS, 3.0), (HEATBATH, 2.0), (METROPOLIS, 2.0), (HEATBATH, 3.0)])
def test_onsager_2d_ferromagnet(algo, T):
    beta = 1.0 / T
    o = Oracle(dim=2, L=32, sample_ids=[0, 1, 2, 3], ferro=True, seed=SEED + 8)
    if T < 2.27:
        o.set_spins(np.ones((4, 1, 1024), dtype=np.int8))  # start in the ordered phase
    o.sweep(algo, beta, 300, nthreads=4)
    o.clear_series()
    o.sweep(algo, beta, 2000, measure_every=1, nthreads=4)
    _, E, _, _ = o.series()
    e = E[:, :, 0, 0].astype(np.float64).mean(axis=1) / 1024.0
    mean, err = pins.batch_mean_error(e, nbatch=20)
    exact = pins.onsager_energy_per_site(beta)
    assert abs(mean - exact) < 4 * err + 2e-4, (mean, exact, err)


def test_heatbath_beta_zero_flips_on_plane0():
    """At beta = 0, T_H = 2^31 for every x, so spin i flips in sweep t iff
    plane 0 (the MSB) of its stream is 1."""
    L, dim = 4, 3
    o = Oracle(dim=dim, L=L, sample_ids=[0, 63, 64, 130], n_replicas=2, seed=SEED + 10)
    for t in range(2):
        before = o.spins()
        o.sweep(HEATBATH, 0.0, 1)
        after = o.spins()
        for si, s in enumerate(o.sample_ids):
            for slot in range(2):
                for i in range(L ** dim):
                    bit = (pins.plane_word(SEED + 10, int(s) >> 6, slot, i, t, 0) >> (int(s) & 63)) & 1
                    assert after[si, slot, i] == before[si, slot, i] * (-1 if bit else 1)


def test_metropolis_beta_zero_flips_every_spin():
    """At beta = 0 every Metropolis proposal is accepted (p = exp(0) = 1, the
    threshold 2^32 above every 32-bit random), so one sweep negates every
    spin, whatever the stream."""
    o = Oracle(dim=3, L=4, sample_ids=[0, 70], n_replicas=2, seed=SEED + 18)
    for _ in range(3):
        before = o.spins()
        o.sweep(METROPOLIS, 0.0, 1)
        assert np.array_equal(o.spins(), -before)


def test_metropolis_zero_temperature_never_raises_energy():
    o = Oracle(dim=3, L=6, sample_ids=[0, 1], seed=SEED + 11)
    E0, _, _ = o.measure()
    o.sweep(METROPOLIS, 50.0, 30, measure_every=1)
    _, E, _, _ = o.series()
    seq = np.concatenate([E0[None], E])[:, :, 0, 0]
    assert np.all(np.diff(seq, axis=0) <= 0)
    assert seq[-1].max() < seq[0].max()


def test_energy_differences_are_multiples_of_four():
    """U mod 2 is fixed per sample (every site has even degree), so energies
    of one sample differ by multiples of 4."""
    o = Oracle(dim=3, L=4, sample_ids=[0, 1, 2], n_replicas=2, n_temps=3, seed=SEED + 12)
    o.sweep(HEATBATH, [0.3, 0.6, 0.9], 5)
    E, _, _ = o.measure()
    for s in range(3):
        v = E[s].ravel()
        assert np.all((v - v[0]) % 4 == 0)


# ---------------- parallel tempering ----------------

def test_pt_permutation_and_energy_multiset():
    K = 5
    beta = [1.0 / (0.7 + 0.9 * k / (K - 1)) for k in range(K)]
    o = Oracle(dim=3, L=4, sample_ids=[0, 9, 70], n_replicas=2, n_temps=K, seed=SEED + 13)
    for _ in range(25):
        o.sweep(METROPOLIS, beta, 3)
        Eb, _, _ = o.measure()
        o.pt_swap(beta)
        Ea, _, _ = o.measure()
        slot_at, acc, _ = o.pt_state()
        for s in range(3):
            for a in range(2):
                assert sorted(slot_at[s, a]) == list(range(K))
                assert sorted(Eb[s, :, a]) == sorted(Ea[s, :, a])
    assert acc.sum() > 0


def test_pt_acceptance_frequency():
    """Two temperatures, configurations frozen: whenever the hotter one holds
    the higher energy (d = E_hot - E_cold > 0) the swap is taken with
    probability T_PT(d)/2^32 = floor(2^32 exp(-db d))/2^32, and otherwise
    always (the standard rule min(1, exp(-db d)), db = beta_cold - beta_hot)."""
    beta = [0.75, 0.7]
    o = Oracle(dim=2, L=4, sample_ids=[0], n_replicas=1, n_temps=2, seed=SEED + 14)
    rng = np.random.default_rng(2)
    # choose two configurations whose energies differ by 8
    while True:
        sp = rng.choice([-1, 1], size=(1, 2, 16)).astype(np.int8)
        o.set_spins(sp)
        E, _, _ = o.measure()
        if abs(int(E[0, 1, 0]) - int(E[0, 0, 0])) == 8:
            break
    tries = accepted = 0
    for _ in range(12000):
        E, _, _ = o.measure()
        d = int(E[0, 1, 0]) - int(E[0, 0, 0])
        slot_before = o.pt_state()[0].copy()
        o.pt_swap(beta)
        swapped = not np.array_equal(o.pt_state()[0], slot_before)
        if d > 0:
            tries += 1
            accepted += int(swapped)
        else:
            assert swapped  # db * d <= 0 always swaps
    p = oracle.table_pt(0.05, 8) / 2.0 ** 32
    assert abs(p - math.exp(-0.4)) < 1e-9
    freq = accepted / tries
    assert abs(freq - p) < 5 * math.sqrt(p * (1 - p) / tries), (freq, p, tries)


# ---------------- determinism of the definition ----------------

def test_split_runs_threads_and_subsets_agree():
    kw = dict(dim=3, L=4, n_replicas=2, seed=SEED + 15)
    a = Oracle(sample_ids=list(range(8)), **kw)
    a.sweep(HEATBATH, 0.9, 7, nthreads=1)
    b = Oracle(sample_ids=list(range(8)), **kw)
    b.sweep(HEATBATH, 0.9, 3, nthreads=4)
    b.sweep(HEATBATH, 0.9, 4, nthreads=3)
    assert np.array_equal(a.spins(), b.spins())
    c = Oracle(sample_ids=[5], **kw)
    c.sweep(HEATBATH, 0.9, 7)
    assert np.array_equal(c.spins()[0], a.spins()[5])


def test_series_rows_are_measurements_after_the_sweep():
    """Measurement timing: with measure_every = k the series holds a row
    after every sweep whose absolute count t is a multiple of k (none for the
    initial state), each equal to a measurement of the state after that sweep,
    here taken by stopping a second run there."""
    kw = dict(dim=3, L=4, sample_ids=[0, 3], n_replicas=2, seed=SEED + 16)
    a = Oracle(**kw)
    a.sweep(METROPOLIS, 0.8, 7, measure_every=3)
    sw, E, M, Q = a.series()
    assert [int(t) for t in sw] == [3, 6]
    b = Oracle(**kw)
    done = 0
    for row, t in enumerate(sw):
        b.sweep(METROPOLIS, 0.8, int(t) - done)
        done = int(t)
        Eb, Mb, Qb = b.measure()
        assert np.array_equal(E[row], Eb) and np.array_equal(M[row], Mb) and np.array_equal(Q[row], Qb)
