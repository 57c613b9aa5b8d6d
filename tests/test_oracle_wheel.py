"""Pins of the oracle's Parisi-Rapuano wheel stream (Sec. 3.3, Eq. 5):
I(k) = I(k-24) + I(k-55) mod 2^32, R(k) = I(k) xor I(k-61), one wheel per
(sample, slot, row, colour) of the plain Ising-like sweep.

* the recurrence against an independent list-based implementation of Eq. 5;
* the starting values against an independent Philox (WHEEL stream, I(-61)
  made odd);
* output statistics: 64-bin uniformity, bit balance, lag-1 correlation;
* the wiring (which output drives which site in which sweep, empty sites
  consuming theirs): at beta = 0 the heat bath flips a site iff bit 31 of its
  output is set, checked sweep by sweep against the independent generator;
* the physics it drives: the enumerated Boltzmann weights of the 3D L=2
  glass and Onsager's energy of the 2D ferromagnet.
"""

import math

import numpy as np
import pytest

import oracle
from oracle import DIS_DAFF, HEATBATH, METROPOLIS, RNG_WHEEL, Oracle
from tests import pins
from tests.test_oracle_physics import _chi2, _closed_classes, _enumerate_ising, _ising_sweep_matrix

SEED = 0x0704357300000D00


def _start_ref(seed, sample, slot, row, colour):
    key = pins.key_of(seed)
    vals = []
    for n in range(61):
        x = pins.philox4x32_10([row, sample, (10 << 28) | ((n >> 2) << 24) | (slot << 12) | colour, 0], key)
        vals.append(x[n & 3])
    vals[0] |= 1
    return vals


class _RefWheel:
    """Eq. 5 written out on a growing list I, indexed from I(-61)."""

    def __init__(self, start):
        self.I = list(start)

    def next(self):
        k = len(self.I)  # position of the new element I(k) in the list
        Ik = (self.I[k - 24] + self.I[k - 55]) & 0xFFFFFFFF
        self.I.append(Ik)
        return Ik ^ self.I[k - 61]


def test_recurrence_matches_eq5():
    rng = np.random.default_rng(1)
    start = rng.integers(0, 2 ** 32, size=61, dtype=np.uint64).astype(np.uint32)
    ref = _RefWheel([int(v) for v in start])
    want = [ref.next() for _ in range(2000)]
    assert [int(v) for v in oracle.wheel_from(start, 2000)] == want


def test_small_case_by_hand():
    """All zeros but I(-61) = 1.  By hand: the lags 24 and 55 never reach
    back to I(-61), so every I(k), k >= 0, is 0; R(k) = I(k) ^ I(k-61) is 1
    at k = 0 and 0 afterwards."""
    start = np.zeros(61, dtype=np.uint32)
    start[0] = 1
    out = oracle.wheel_from(start, 70)
    assert out[0] == 1 and not out[1:].any()


@pytest.mark.parametrize("sample,slot,row,colour", [(0, 0, 0, 0), (5, 1, 17, 1), (300, 7, 4095, 0)])
def test_seeding_matches_independent_philox(sample, slot, row, colour):
    start, out = oracle.wheel(SEED, sample, slot, row, colour, 500)
    ref_start = _start_ref(SEED, sample, slot, row, colour)
    assert [int(v) for v in start] == ref_start
    ref = _RefWheel(ref_start)
    assert [int(v) for v in out] == [ref.next() for _ in range(500)]


def test_output_statistics():
    _, out = oracle.wheel(SEED, 3, 0, 9, 1, 400000)
    x = out.astype(np.float64) / 2.0 ** 32
    hist = np.bincount((x * 64).astype(int), minlength=64)
    chi2, dof = _chi2(hist, np.full(64, 1 / 64))
    assert chi2 < dof + 6 * math.sqrt(2 * dof)
    bits = (out[:, None] >> np.arange(32, dtype=np.uint32)) & 1
    assert np.all(np.abs(bits.mean(axis=0) - 0.5) < 5 * 0.5 / math.sqrt(len(out)))
    c = np.corrcoef(x[:-1], x[1:])[0, 1]
    assert abs(c) < 5 / math.sqrt(len(out))


@pytest.mark.parametrize("disorder,occ", [(0, 1.0), (DIS_DAFF, 0.6)])
def test_wiring_at_beta_zero(disorder, occ):
    """beta = 0 heat bath keeps s_i iff R < 2^31: a site flips iff bit 31 of
    its output is set.  Each wheel (row, colour) gives its sites one output
    per sweep in increasing x; empty sites (DAFF) consume theirs too."""
    L, D = 4, 3
    ids = [0, 3]
    o = Oracle(dim=D, L=L, sample_ids=ids, n_replicas=2, seed=SEED + 1, rng=RNG_WHEEL, disorder=disorder,
               field=0.5 if disorder else 0.0, occupation=occ)
    _, x = o.sites()
    wheels = {(si, sl, row, c): _RefWheel(_start_ref(SEED + 1, s, sl, row, c))
              for si, s in enumerate(ids) for sl in range(2) for row in range(L * L) for c in range(2)}
    for _ in range(3):
        before = o.spins()
        o.sweep(HEATBATH, 0.0, 1)
        after = o.spins()
        for si in range(len(ids)):
            for sl in range(2):
                for c in range(2):
                    for row in range(L * L):
                        for xx in range(L):
                            i = xx + L * row
                            if pins.colour_of(i, L, D) != c:
                                continue
                            r = wheels[(si, sl, row, c)].next()
                            flip = x[si, i] == 1 and (r >> 31) == 1
                            assert after[si, sl, i] == before[si, sl, i] * (-1 if flip else 1)


@pytest.mark.parametrize("algo", [METROPOLIS, HEATBATH])
def test_wheel_chain_matches_boltzmann_N8(algo):
    beta = 0.3
    o = Oracle(dim=3, L=2, sample_ids=[3], seed=SEED + 2, rng=RNG_WHEEL)
    J = o.couplings()[0]
    _, E = _enumerate_ising(J, 2, 3)
    w = 1 << np.arange(8)
    # Metropolis at L=2 can split into closed classes (zero-field sites flip
    # every sweep): the chain samples Boltzmann weights on its own class
    start = int(((1 - o.spins()[0, 0]) // 2 * w).sum())
    P = _ising_sweep_matrix(J, 2, 3, algo, beta)
    cls = next(c for c in _closed_classes(P) if start in c or P[start, c].sum() > 0)
    p = np.zeros(256)
    p[cls] = np.exp(-beta * (E[cls] - E.min()))
    p /= p.sum()
    hist = np.zeros(256, dtype=np.int64)
    for _ in range(60000):
        o.sweep(algo, beta, 1)
        hist[int(((1 - o.spins()[0, 0]) // 2 * w).sum())] += 1
    chi2, dof = _chi2(hist, p)
    assert chi2 / dof < 1.6, (chi2, dof)


@pytest.mark.parametrize("algo,T", [(METROPOLIS, 3.0), (HEATBATH, 2.0)])
def test_wheel_onsager_2d_ferromagnet(algo, T):
    beta = 1.0 / T
    o = Oracle(dim=2, L=32, sample_ids=[0, 1, 2, 3], ferro=True, seed=SEED + 3, rng=RNG_WHEEL)
    if T < 2.27:
        o.set_spins(np.ones((4, 1, 1024), dtype=np.int8))
    o.sweep(algo, beta, 300, nthreads=4)
    o.clear_series()
    o.sweep(algo, beta, 2000, measure_every=1, nthreads=4)
    _, E, _, _ = o.series()
    e = E[:, :, 0, 0].astype(np.float64).mean(axis=1) / 1024.0
    mean, err = pins.batch_mean_error(e, nbatch=20)
    exact = pins.onsager_energy_per_site(beta)
    assert abs(mean - exact) < 4 * err + 2e-4, (mean, exact, err)


def test_wheel_bookkeeping_and_only_for_ising():
    o = Oracle(dim=3, L=6, sample_ids=[0, 1], n_replicas=2, seed=SEED + 4, rng=RNG_WHEEL)
    for algo in (METROPOLIS, HEATBATH):
        o.sweep(algo, 0.8, 3)
        assert o.bookkeeping_error() == 0
    with pytest.raises(ValueError):
        Oracle(model=oracle.MODEL_POTTS, rng=RNG_WHEEL)
