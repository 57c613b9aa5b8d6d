"""Pins of the oracle's glassy Potts model with permutation couplings (Eq. 3):
H = -sum_<ij> delta(s_i, pi_ij(s_j)), four states, pi_ij one of the 4!
permutations, in 2, 3 and 4 dimensions.

Each test checks the oracle against something the definition fixes:
* the coupling stream and the lexicographic unranking against an independent
  Philox and itertools.permutations, and the 24 permutations equally likely;
* the energy against an independent numpy evaluation of Eq. (3);
* incremental bookkeeping (sum of the update's local energy changes) against
  recomputation, in 2D, 3D and 4D (a wrong backward bond or inverse breaks
  it);
* identity permutations turn Eq. (3) into the ferromagnetic 4-state Potts
  model: the trajectory equals model 1 with every J = +1, bit for bit;
* beta = 0 heat bath: the new state is the top two bits of the stream;
* the exact one-site heat-bath kernels, built from Eq. (3) by enumeration,
  keep the Boltzmann distribution (quantisation tolerance), and the
  oracle's own chain reproduces the enumerated Boltzmann weights (2D L=2)
  and energy distribution (3D L=2);
* beta -> infinity never raises the energy.
"""

import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import HEATBATH, MODEL_PERM, MODEL_POTTS, Oracle
from tests import pins
from tests.test_oracle_physics import _chi2

SEED = 0x0704357300000E00
PERMS = list(itertools.permutations(range(4)))  # lexicographic order


def _index_ref(seed, sample, d, site):
    x = pins.philox4x32_10([site, d, (9 << 28) | (sample >> 2), 0], pins.key_of(seed))
    return (x[sample & 3] * 24) >> 32


def _code(p):
    return p[0] | (p[1] << 2) | (p[2] << 4) | (p[3] << 6)


def _perm_of_code(code):
    c = int(code) & 0xFF
    return [(c >> (2 * v)) & 3 for v in range(4)]


def _energy(states, codes, L, D):
    """Eq. (3) for a batch of configurations: states [n, N] in 0..3."""
    states = np.asarray(states)
    E = np.zeros(states.shape[0], dtype=np.int64)
    for i, j, d in pins.bonds(L, D):
        pi = np.array(_perm_of_code(codes[d][i]))
        E -= (states[:, i] == pi[states[:, j]]).astype(np.int64)
    return E


# ---------------- couplings ----------------

def test_unranking_and_codes_follow_lexicographic_order():
    for k, p in enumerate(PERMS):
        assert oracle.perm_code(k) == _code(p)


def test_coupling_stream_matches_independent_philox():
    o = Oracle(model=MODEL_PERM, dim=3, L=4, sample_ids=[0, 1, 3, 4, 70], seed=SEED)
    J = o.couplings()
    for si, s in enumerate([0, 1, 3, 4, 70]):
        for d in range(3):
            for i in range(0, 64, 5):
                k = _index_ref(SEED, s, d, i)
                assert oracle.perm_coupling_index(SEED, s, d, i) == k
                assert (int(J[si, d, i]) & 0xFF) == _code(PERMS[k])


def test_permutations_equally_likely():
    o = Oracle(model=MODEL_PERM, dim=3, L=16, sample_ids=list(range(8)), seed=SEED + 1)
    codes = (o.couplings().astype(np.int64) & 0xFF).ravel()
    lookup = {_code(p): k for k, p in enumerate(PERMS)}
    idx = np.array([lookup[c] for c in codes])
    hist = np.bincount(idx, minlength=24)
    chi2, dof = _chi2(hist, np.full(24, 1 / 24))
    assert dof == 23 and chi2 < 60, chi2  # p ~ 4e-5 at 60 for 23 dof


def test_set_couplings_rejects_non_permutations():
    o = Oracle(model=MODEL_PERM, dim=2, L=4, seed=SEED)
    J = o.couplings()
    bad = J.copy()
    bad[0, 0, 0] = 0  # (0, 0, 0, 0) is not a permutation
    with pytest.raises(ValueError):
        o.set_couplings(bad)
    assert np.array_equal(o.couplings(), J)


# ---------------- energy and bookkeeping ----------------

@pytest.mark.parametrize("dim,L", [(2, 6), (3, 4), (4, 4), (2, 2), (4, 2)])
def test_energy_and_bookkeeping(dim, L):
    o = Oracle(model=MODEL_PERM, dim=dim, L=L, sample_ids=[0, 5, 9], n_replicas=2, seed=SEED + 2)
    J = o.couplings()
    for beta in (0.4, 1.4, 3.0):
        o.sweep(HEATBATH, beta, 2)
        assert o.bookkeeping_error() == 0
    sp = o.spins()
    E, M, Q = o.measure()
    for s in range(3):
        assert np.array_equal(E[s, 0], _energy(sp[s], J[s], L, dim))
        for a in range(2):
            assert np.array_equal(M[s, 0, a], np.bincount(sp[s, a], minlength=4))
        assert Q[s, 0] == int((sp[s, 0] == sp[s, 1]).sum())


@pytest.mark.parametrize("dim,L", [(2, 4), (3, 4), (4, 4), (3, 2)])
def test_identity_permutations_are_the_ferromagnetic_potts_model(dim, L):
    ident = _code((0, 1, 2, 3))
    a = Oracle(model=MODEL_PERM, dim=dim, L=L, sample_ids=[0, 6], n_replicas=2, seed=SEED + 3)
    b = Oracle(model=MODEL_POTTS, dim=dim, L=L, sample_ids=[0, 6], n_replicas=2, seed=SEED + 3, ferro=True)
    a.set_couplings(np.full((2, dim, L ** dim), ident, dtype=np.uint8).view(np.int8))
    assert np.array_equal(a.spins(), b.spins())
    for beta in (0.5, 1.2):
        a.sweep(HEATBATH, beta, 3)
        b.sweep(HEATBATH, beta, 3)
        assert np.array_equal(a.spins(), b.spins())
        for u, v in zip(a.measure(), b.measure()):
            assert np.array_equal(u, v)


@pytest.mark.parametrize("dim,L", [(3, 4), (4, 2)])
def test_beta_zero_takes_the_top_bits_of_the_stream(dim, L):
    o = Oracle(model=MODEL_PERM, dim=dim, L=L, sample_ids=[0, 3, 6], n_replicas=2, seed=SEED + 4)
    o.sweep(HEATBATH, 0.0, 1)
    sp = o.spins()
    key = pins.key_of(SEED + 4)
    for si, s in enumerate([0, 3, 6]):
        for slot in range(2):
            for i in range(L ** dim):
                x = pins.philox4x32_10([i, 0, (4 << 28) | (slot << 16) | (s >> 2), 0], key)
                assert sp[si, slot, i] == x[s & 3] >> 30


def test_zero_temperature_never_raises_energy():
    o = Oracle(model=MODEL_PERM, dim=3, L=6, sample_ids=[0, 1], seed=SEED + 5)
    E0, _, _ = o.measure()
    o.sweep(HEATBATH, 60.0, 20, measure_every=1)
    _, E, _, _ = o.series()
    seq = np.concatenate([E0[None], E])[:, :, 0, 0]
    assert np.all(np.diff(seq, axis=0) <= 0)
    assert seq[-1].max() < seq[0].max()


# ---------------- exact enumeration ----------------

def _site_kernels_keep_boltzmann(codes, L, D, beta):
    """Heat-bath kernel of every site, from Eq. (3) by enumeration over the
    4^N states, applied to the Boltzmann vector; returns the worst relative
    change (the quantised thresholds allow ~2^-32 / p_min)."""
    N = L ** D
    n = 4 ** N
    k = np.arange(n)
    states = (k[:, None] // (4 ** np.arange(N))[None, :]) % 4
    E = _energy(states, codes, L, D).astype(np.float64)
    boltz = np.exp(-beta * (E - E.min()))
    boltz /= boltz.sum()
    tab_cache = {}
    worst = 0.0
    for i in range(N):
        # bonds at i, from the definition: (i, j) satisfied iff s_i = pi(s_j);
        # (j, i) satisfied iff s_j = pi(s_i)
        cnt = np.zeros((n, 4), dtype=np.int64)
        for a, b, d in pins.bonds(L, D):
            pi = np.array(_perm_of_code(codes[d][a]))
            for c in range(4):
                if a == i and b == i:
                    cnt[:, c] += (c == pi[c])
                elif a == i:
                    cnt[:, c] += (c == pi[states[:, b]])
                elif b == i:
                    cnt[:, c] += (states[:, a] == pi[c])
        out = np.zeros(n)
        base = k - states[:, i] * 4 ** i
        for kk in range(n):
            key = tuple(cnt[kk])
            if key not in tab_cache:
                T = [0] + oracle.table_potts(beta, list(key)) + [1 << 32]
                tab_cache[key] = np.diff(np.array(T, dtype=np.float64)) / 2.0 ** 32
            out[base[kk] + 4 ** i * np.arange(4)] += boltz[kk] * tab_cache[key]
        worst = max(worst, float(np.max(np.abs(out - boltz) / boltz)))
    return worst


@pytest.mark.parametrize("beta", [0.3, 1.0, 2.4])
def test_site_kernels_keep_boltzmann_2d(beta):
    o = Oracle(model=MODEL_PERM, dim=2, L=2, sample_ids=[7], seed=SEED + 6)
    codes = o.couplings()[0].astype(np.int64) & 0xFF
    worst = _site_kernels_keep_boltzmann(codes, 2, 2, beta)
    p_min = 1.0 / (1.0 + 3.0 * math.exp(beta * 4))
    assert worst < 4.0 * 2.0 ** -32 / p_min, worst


def test_chain_matches_boltzmann_2d_L2():
    """2D L=2: 4 sites, 8 bonds (each pair of sites joined by two bonds with
    different permutations), 256 states."""
    beta = 0.8
    o = Oracle(model=MODEL_PERM, dim=2, L=2, sample_ids=[7], seed=SEED + 7)
    codes = o.couplings()[0].astype(np.int64) & 0xFF
    k = np.arange(256)
    states = (k[:, None] // (4 ** np.arange(4))[None, :]) % 4
    E = _energy(states, codes, 2, 2).astype(np.float64)
    p = np.exp(-beta * (E - E.min()))
    p /= p.sum()
    w = 4 ** np.arange(4)
    hist = np.zeros(256, dtype=np.int64)
    for _ in range(60000):
        o.sweep(HEATBATH, beta, 1)
        hist[int((o.spins()[0, 0] * w).sum())] += 1
    chi2, dof = _chi2(hist, p)
    assert chi2 / dof < 1.6, (chi2, dof)


def test_energy_histogram_3d_L2():
    """3D L=2 (8 sites, 24 bonds, 65536 states): energy histogram of long
    oracle runs against the enumerated distribution P(E)."""
    beta = 0.9
    o = Oracle(model=MODEL_PERM, dim=3, L=2, sample_ids=[1, 2, 3, 4], seed=SEED + 8)
    J = o.couplings().astype(np.int64) & 0xFF
    o.sweep(HEATBATH, beta, 30000, measure_every=1, nthreads=4)
    _, Es, _, _ = o.series()
    k = np.arange(4 ** 8)
    states = (k[:, None] // (4 ** np.arange(8))[None, :]) % 4
    for s in range(4):
        E = _energy(states, J[s], 2, 3)
        levels = np.unique(E)
        w = np.exp(-beta * (E - E.min()).astype(np.float64))
        pE = np.array([w[E == e].sum() for e in levels]) / w.sum()
        h = np.array([(Es[:, s, 0, 0] == e).sum() for e in levels])
        assert h.sum() == len(Es)
        chi2, dof = _chi2(h, pE)
        assert chi2 / max(dof, 1) < 3.0, (s, chi2, dof)
