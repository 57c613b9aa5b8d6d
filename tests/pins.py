"""Independent helpers used by the oracle pin tests.

Nothing here is shared with the oracle or the CUDA library: the Philox
generator below is a third implementation, in Python integers, of the
published Philox4x32-10 definition (Salmon et al., SC'11), and the exact
enumeration and Onsager helpers are textbook closed forms.
"""

from __future__ import annotations

import itertools
import math

import numpy as np

MASK32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    c = list(ctr)
    k0, k1 = key
    for rnd in range(10):
        if rnd:
            k0 = (k0 + 0x9E3779B9) & MASK32
            k1 = (k1 + 0xBB67AE85) & MASK32
        p0 = 0xD2511F53 * c[0]
        p1 = 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k0) & MASK32, p1 & MASK32, ((p0 >> 32) ^ c[3] ^ k1) & MASK32, p0 & MASK32]
    return c


def key_of(seed):
    return (seed & MASK32, seed >> 32)


def plane_word(seed, group, slot, site, sweep, plane):
    """Bit-plane word W[plane] of the Ising update stream (64 lanes)."""
    m = plane >> 1
    c2 = (1 << 28) | (m << 24) | (slot << 12) | group
    x = philox4x32_10([site, sweep & MASK32, c2, sweep >> 32], key_of(seed))
    if plane & 1:
        return x[2] | (x[3] << 32)
    return x[0] | (x[1] << 32)


# ---- lattice helpers (periodic, site i = x + L*(y + L*z)) ----

def coords(i, L, D):
    out = []
    for _ in range(D):
        out.append(i % L)
        i //= L
    return out


def index(x, L):
    i = 0
    for v in reversed(x):
        i = i * L + v
    return i


def fwd(i, d, L, D):
    x = coords(i, L, D)
    x[d] = (x[d] + 1) % L
    return index(x, L)


def bonds(L, D):
    """List of (i, j, d): forward bond J_d(i) joining i and i + e_d."""
    N = L ** D
    return [(i, fwd(i, d, L, D), d) for i in range(N) for d in range(D)]


def colour_of(i, L, D):
    return sum(coords(i, L, D)) % 2


def ising_energy(spins, J, L, D):
    """E = -sum over bonds J s s; spins [N] of +-1, J [D][N]."""
    E = 0
    for i, j, d in bonds(L, D):
        E -= int(J[d][i]) * int(spins[i]) * int(spins[j])
    return E


def potts_energy(states, J, L, D):
    E = 0
    for i, j, d in bonds(L, D):
        if states[i] == states[j]:
            E -= int(J[d][i])
    return E


# ---- Onsager: exact energy per site of the 2D Ising ferromagnet ----

def _agm(a, b):
    for _ in range(60):
        a, b = (a + b) / 2.0, math.sqrt(a * b)
    return a


def complete_elliptic_k(kappa):
    """K(kappa) = pi / (2 agm(1, sqrt(1 - kappa^2)))."""
    return math.pi / (2.0 * _agm(1.0, math.sqrt(1.0 - kappa * kappa)))


def onsager_energy_per_site(beta):
    """u = -coth(2b) [1 + (2/pi)(2 tanh^2(2b) - 1) K(kappa)], kappa = 2 sinh 2b / cosh^2 2b."""
    t2 = math.tanh(2 * beta)
    kappa = 2.0 * math.sinh(2 * beta) / math.cosh(2 * beta) ** 2
    return -(1.0 / t2) * (1.0 + (2.0 / math.pi) * (2.0 * t2 * t2 - 1.0) * complete_elliptic_k(kappa))


def batch_mean_error(x, nbatch=20):
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nbatch
    means = x[: n * nbatch].reshape(nbatch, n).mean(axis=1)
    return float(means.mean()), float(means.std(ddof=1) / math.sqrt(nbatch))


def all_states(n, q=2):
    return itertools.product(range(q), repeat=n)
