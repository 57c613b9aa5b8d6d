"""Pins of the oracle's random stream and acceptance tables (CPU only).

Pins used (none is the oracle checking itself):
* Philox4x32-10 known-answer vectors published with the generator
  (tests/golden/philox4x32_10_kat.txt);
* a third, pure-Python implementation of the stream definition for the
  bit-plane assembly, the couplings and the initial states (tests/pins.py),
  itself pinned by the same vectors;
* uniformity of the assembled 32-bit values (chi-square);
* acceptance tables against 60-digit evaluations with sympy, and the
  identities p(x) + p(-x) = 1 and monotonicity in the energy argument.
"""

import math
import os
import random

import numpy as np
import pytest
import sympy

import oracle
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("row", _kat_rows())
def test_philox_known_answers(row):
    ctr, key, expect = row
    assert oracle.philox(ctr, key) == expect
    assert pins.philox4x32_10(ctr, key) == expect


def test_ising_random_is_plane_assembly():
    """r(s, sigma, i, t) = sum_p bit_l(W_p) << (31 - p), W from the SPIN stream."""
    rng = random.Random(7)
    for _ in range(40):
        seed = rng.getrandbits(64)
        s = rng.randrange(0, 300)
        slot = rng.randrange(0, 70)
        site = rng.getrandbits(32)
        t = rng.getrandbits(40)
        lane, g = s & 63, s >> 6
        r = 0
        for p in range(32):
            r |= ((pins.plane_word(seed, g, slot, site, t, p) >> lane) & 1) << (31 - p)
        assert oracle.ising_random(seed, s, slot, site, t) == r


def test_potts_and_pt_random_words():
    rng = random.Random(11)
    for _ in range(40):
        seed = rng.getrandbits(64)
        s = rng.randrange(0, 1000)
        slot = rng.randrange(0, 100)
        site = rng.getrandbits(32)
        t = rng.getrandbits(40)
        x = pins.philox4x32_10([site, t & pins.MASK32, (4 << 28) | (slot << 16) | (s >> 2), t >> 32],
                               pins.key_of(seed))
        assert oracle.potts_random(seed, s, slot, site, t) == x[s & 3]
        k = rng.randrange(0, 40)
        a = rng.randrange(0, 3)
        x = pins.philox4x32_10([k, t & pins.MASK32, (6 << 28) | (a << 16) | (s >> 2), t >> 32], pins.key_of(seed))
        assert oracle.pt_random(seed, s, a, k, t) == x[s & 3]


def _lane_bit(seed, c0, c1, c2, lane):
    x = pins.philox4x32_10([c0, c1, c2, 0], pins.key_of(seed))
    return ((x[0] | (x[1] << 32)) >> lane) & 1


@pytest.mark.parametrize("model", [oracle.MODEL_ISING, oracle.MODEL_POTTS])
def test_disorder_and_initial_state_streams(model):
    """Couplings (J stream: bit l of x0 | x1 << 32 at c0 = i, c1 = d,
    c2 = (2 << 28) | g; set bit = J = -1) and initial states (Ising: INIT
    stream, c2 = (3 << 28) | (sigma << 12) | g; Potts: x_{s & 3} >> 30 of the
    PINIT stream, c2 = (5 << 28) | (sigma << 16) | (s >> 2)), recomputed
    with the independent Philox for samples in three 64-lane groups."""
    seed, ids, dim, L, R = 0x0123456789ABCDEF, [0, 5, 70, 130], 3, 4, 2
    o = oracle.Oracle(model=model, dim=dim, L=L, sample_ids=ids, n_replicas=R, seed=seed)
    J, sp = o.couplings(), o.spins()
    N = L ** dim
    key = pins.key_of(seed)
    for k, s in enumerate(ids):
        g, lane = s >> 6, s & 63
        for d in range(dim):
            for i in range(N):
                assert J[k, d, i] == 1 - 2 * _lane_bit(seed, i, d, (2 << 28) | g, lane)
        for sigma in range(R):
            for i in range(N):
                if model == oracle.MODEL_ISING:
                    want = 1 - 2 * _lane_bit(seed, i, 0, (3 << 28) | (sigma << 12) | g, lane)
                else:
                    x = pins.philox4x32_10([i, 0, (5 << 28) | (sigma << 16) | (s >> 2), 0], key)
                    want = x[s & 3] >> 30
                assert sp[k, sigma, i] == want


def test_ising_random_uniform():
    """Assembled values are uniform on [0, 2^32): chi-square over 64 bins, and
    each bit position is fair.  Catches a lost or duplicated plane."""
    seed = 0x0704357300000001
    vals = np.array([oracle.ising_random(seed, s, 0, i, 3) for s in range(0, 128, 5) for i in range(400)],
                    dtype=np.uint64)
    counts = np.bincount((vals >> np.uint64(26)).astype(np.int64), minlength=64)
    exp = len(vals) / 64.0
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 120.0, chi2  # 63 dof, p ~ 1e-5
    for b in range(32):
        frac = float(((vals >> np.uint64(b)) & np.uint64(1)).mean())
        assert abs(frac - 0.5) < 5 * 0.5 / math.sqrt(len(vals)), (b, frac)


# ---------------- tables vs 60-digit evaluation ----------------

def _exact_floor(expr_value):
    """floor(2^32 p) with p a sympy Float of high precision; also its distance
    to the nearest integer (to allow FP64 rounding at a near-tie)."""
    v = expr_value * sympy.Integer(2) ** 32
    f = int(sympy.floor(v))
    frac = float(v - f)
    return f, min(frac, 1.0 - frac)


def _check(got, exact, dist):
    if dist < 1e-6:
        assert abs(got - exact) <= 1
    else:
        assert got == exact


BETAS = [0.0, 0.1, 0.44068679350977147, 1 / 1.1, 1.0, 1.25, 2.4, 5.0]


@pytest.mark.parametrize("beta", BETAS)
def test_metropolis_table_exact(beta):
    b = sympy.Float(beta, 60)
    prev = None
    for dE in (4, 8, 12):
        exact, dist = _exact_floor(sympy.exp(-b * dE).evalf(60))
        got = oracle.table_metropolis(beta, dE)
        _check(got, exact, dist)
        if prev is not None:
            assert got <= prev
        prev = got


@pytest.mark.parametrize("beta", BETAS)
def test_heatbath_table_exact(beta):
    b = sympy.Float(beta, 60)
    prev = -1
    for x in range(-6, 7, 2):
        exact, dist = _exact_floor((1 / (1 + sympy.exp(-2 * b * x))).evalf(60))
        got = oracle.table_heatbath(beta, x)
        _check(got, exact, dist)
        assert got >= prev
        prev = got
        # p(x) + p(-x) = 1  =>  T(x) + T(-x) is 2^32 - 1 or 2^32
        assert abs(got + oracle.table_heatbath(beta, -x) - (2 ** 32 - 1)) <= 1


def test_heatbath_beta_zero_is_half():
    for x in range(-6, 7, 2):
        assert oracle.table_heatbath(0.0, x) == 2 ** 31


@pytest.mark.parametrize("beta", [0.0, 0.8, 1.25, 2.4])
def test_potts_table_exact(beta):
    b = sympy.Float(beta, 60)
    rng = random.Random(3)
    tuples = [(0, 0, 0, 0), (6, 0, 0, 0), (-6, 0, 0, 0), (0, 0, 0, 6), (1, -2, 3, 0)]
    tuples += [tuple(rng.randint(-6, 6) for _ in range(4)) for _ in range(20)]
    for n in tuples:
        w = [sympy.exp(b * v) for v in n]
        Z = sum(w)
        got = oracle.table_potts(beta, n)
        acc = 0
        for k in range(3):
            acc = acc + w[k]
            exact, dist = _exact_floor((acc / Z).evalf(60))
            _check(got[k], exact, dist)
        assert got[0] <= got[1] <= got[2] <= 2 ** 32


def test_pt_table_exact():
    for db in (0.01, 0.0263, 0.5):
        for d in (4, 8, 40, 400):
            exact, dist = _exact_floor(sympy.exp(-sympy.Float(db, 60) * d).evalf(60))
            _check(oracle.table_pt(db, d), exact, dist)
