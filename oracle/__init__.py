"""CPU oracle for the checkerboard Metropolis / heat-bath sweep (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The library under
``paper_0704_3573_gb300`` never imports, links or calls it, and it shares no
code with the CUDA path.

The oracle is plain C++17 (``oracle/*.cpp``) compiled with g++ into
``oracle/liboracle.so`` and wrapped here with ctypes.  What it computes, and
the passages it follows, are listed in ``oracle/oracle.h``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["stream.cpp", "model.cpp", "capi.cpp"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (plain -O2, portable: no -march flags)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_LIB_PATH):
        lib_m = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= lib_m for s in srcs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp]
    cmd += [os.path.join(_HERE, s) for s in _SRCS]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        c = ctypes
        L.oracle_create.restype = c.c_void_p
        L.oracle_create.argtypes = [c.c_int, c.c_int, c.c_int, c.c_int, c.POINTER(c.c_int32), c.c_int,
                                    c.c_int, c.c_int, c.c_uint64, c.c_int, c.c_double, c.c_double, c.c_int]
        L.oracle_destroy.argtypes = [c.c_void_p]
        L.oracle_sweep.argtypes = [c.c_void_p, c.c_int, c.POINTER(c.c_double), c.c_uint64, c.c_uint32, c.c_int]
        L.oracle_pt_swap.argtypes = [c.c_void_p, c.POINTER(c.c_double)]
        L.oracle_measure.argtypes = [c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p]
        L.oracle_sweeps.restype = c.c_uint64
        L.oracle_sweeps.argtypes = [c.c_void_p]
        L.oracle_series_rows.restype = c.c_size_t
        L.oracle_series_rows.argtypes = [c.c_void_p]
        L.oracle_series.argtypes = [c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p]
        L.oracle_series_clear.argtypes = [c.c_void_p]
        for f in ("oracle_get_spins", "oracle_set_spins", "oracle_get_couplings", "oracle_set_couplings"):
            getattr(L, f).argtypes = [c.c_void_p, c.c_void_p]
        L.oracle_set_couplings.restype = c.c_int
        L.oracle_perm_coupling_index.restype = c.c_int
        L.oracle_perm_coupling_index.argtypes = [c.c_uint64, c.c_int, c.c_int, c.c_uint32]
        L.oracle_perm_code.restype = c.c_int
        L.oracle_wheel.argtypes = [c.c_uint64, c.c_int, c.c_int, c.c_uint32, c.c_int, c.c_void_p, c.c_uint32,
                                   c.c_void_p]
        L.oracle_wheel_from.argtypes = [c.c_void_p, c.c_uint32, c.c_void_p]
        L.oracle_perm_code.argtypes = [c.c_int]
        L.oracle_get_sites.argtypes = [c.c_void_p, c.c_void_p, c.c_void_p]
        L.oracle_set_sites.argtypes = [c.c_void_p, c.c_void_p, c.c_void_p]
        L.oracle_get_pt.argtypes = [c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p]
        L.oracle_bookkeeping_error.restype = c.c_int64
        L.oracle_bookkeeping_error.argtypes = [c.c_void_p]
        L.oracle_philox.argtypes = [c.c_void_p, c.c_void_p, c.c_void_p]
        L.oracle_ising_random.restype = c.c_uint32
        L.oracle_ising_random.argtypes = [c.c_uint64, c.c_int, c.c_int, c.c_uint32, c.c_uint64]
        L.oracle_potts_random.restype = c.c_uint32
        L.oracle_potts_random.argtypes = [c.c_uint64, c.c_int, c.c_int, c.c_uint32, c.c_uint64]
        L.oracle_pt_random.restype = c.c_uint32
        L.oracle_pt_random.argtypes = [c.c_uint64, c.c_int, c.c_int, c.c_int, c.c_uint64]
        L.oracle_table_metropolis.restype = c.c_uint64
        L.oracle_table_metropolis.argtypes = [c.c_double, c.c_int]
        L.oracle_table_heatbath.restype = c.c_uint64
        L.oracle_table_heatbath.argtypes = [c.c_double, c.c_int]
        L.oracle_table_potts.argtypes = [c.c_double, c.c_int, c.c_void_p, c.c_void_p]
        L.oracle_table_pt.restype = c.c_uint64
        L.oracle_table_pt.argtypes = [c.c_double, c.c_int64]
        L.oracle_table_metropolis_x.restype = c.c_uint64
        L.oracle_table_metropolis_x.argtypes = [c.c_double, c.c_double]
        L.oracle_table_heatbath_x.restype = c.c_uint64
        L.oracle_table_heatbath_x.argtypes = [c.c_double, c.c_double]
        L.oracle_field_sign_bit.restype = c.c_int
        L.oracle_field_sign_bit.argtypes = [c.c_uint64, c.c_int, c.c_uint32]
        L.oracle_occupation_random.restype = c.c_uint32
        L.oracle_occupation_random.argtypes = [c.c_uint64, c.c_int, c.c_uint32]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox(_ptr(c), _ptr(k), _ptr(out))
    return [int(v) for v in out]


def ising_random(seed, sample, slot, site, sweep) -> int:
    return int(lib().oracle_ising_random(seed, sample, slot, site, sweep))


def potts_random(seed, sample, slot, site, sweep) -> int:
    return int(lib().oracle_potts_random(seed, sample, slot, site, sweep))


def pt_random(seed, sample, replica, pair, step) -> int:
    return int(lib().oracle_pt_random(seed, sample, replica, pair, step))


def table_metropolis(beta: float, dE: int) -> int:
    return int(lib().oracle_table_metropolis(beta, dE))


def table_heatbath(beta: float, x: int) -> int:
    return int(lib().oracle_table_heatbath(beta, x))


def table_potts(beta: float, n) -> list[int]:
    q = len(n)
    nn = np.asarray(n, dtype=np.int32)
    T = np.zeros(q - 1, dtype=np.uint64)
    lib().oracle_table_potts(beta, q, _ptr(nn), _ptr(T))
    return [int(v) for v in T]


def table_pt(dbeta_abs: float, dabs: int) -> int:
    return int(lib().oracle_table_pt(dbeta_abs, dabs))


def table_metropolis_x(beta: float, x: float) -> int:
    return int(lib().oracle_table_metropolis_x(beta, x))


def table_heatbath_x(beta: float, x: float) -> int:
    return int(lib().oracle_table_heatbath_x(beta, x))


def field_sign_bit(seed, sample, site) -> int:
    return int(lib().oracle_field_sign_bit(seed, sample, site))


def occupation_random(seed, sample, site) -> int:
    return int(lib().oracle_occupation_random(seed, sample, site))


def perm_coupling_index(seed, sample, d, site) -> int:
    return int(lib().oracle_perm_coupling_index(seed, sample, d, site))


def perm_code(index) -> int:
    return int(lib().oracle_perm_code(index))


def wheel(seed, sample, slot, row, colour, n):
    """(I(-61..-1), R(0..n-1)) of a freshly seeded Parisi-Rapuano wheel."""
    start = np.zeros(61, dtype=np.uint32)
    out = np.zeros(n, dtype=np.uint32)
    lib().oracle_wheel(seed, sample, slot, row, colour, _ptr(start), n, _ptr(out))
    return start, out


def wheel_from(start61, n):
    s = np.ascontiguousarray(start61, dtype=np.uint32)
    out = np.zeros(n, dtype=np.uint32)
    lib().oracle_wheel_from(_ptr(s), n, _ptr(out))
    return out


MODEL_ISING, MODEL_POTTS, MODEL_PERM = 0, 1, 2
METROPOLIS, HEATBATH = 0, 1
DIS_EA, DIS_FERRO, DIS_RFIM, DIS_DAFF = 0, 1, 2, 3
RNG_PHILOX, RNG_WHEEL = 0, 1


class Oracle:
    """One oracle state: the listed samples of a lattice configuration.

    ``sample_ids`` selects which disorder samples are simulated; each keeps its
    true index, so sample s here follows the same streams as sample s of a
    full batch.  ``disorder`` is one of DIS_* (``ferro=True`` is DIS_FERRO);
    ``field`` is |h| (random-field model) and ``occupation`` the site
    occupation probability (diluted antiferromagnet).  Field models measure
    M as [S, K, R, 2] = (sum x s, sum sign(h) x s).  ``rng`` selects the
    Ising update stream: RNG_PHILOX (the plane stream) or RNG_WHEEL (one
    Parisi-Rapuano wheel per sample, slot, row and colour).
    """

    def __init__(self, model=MODEL_ISING, dim=3, L=4, sample_ids=(0,), n_replicas=1, n_temps=1,
                 seed=1, ferro=False, q=4, disorder=None, field=0.0, occupation=1.0, rng=RNG_PHILOX):
        ids = np.asarray(sample_ids, dtype=np.int32)
        if disorder is None:
            disorder = DIS_FERRO if ferro else DIS_EA
        if model == MODEL_PERM:
            q = 4  # the glassy Potts model of Eq. (3) has four states
        self.model, self.q, self.dim, self.L = model, q, dim, L
        self.disorder, self.field, self.occupation = disorder, float(field), float(occupation)
        self.N = L ** dim
        self.S, self.R, self.K = len(ids), n_replicas, n_temps
        self.sample_ids = ids
        self.mq = q if model != MODEL_ISING else (2 if disorder in (DIS_RFIM, DIS_DAFF) else 1)
        h = lib().oracle_create(model, q, dim, L, ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(ids),
                                n_replicas, n_temps, seed, int(disorder), float(field), float(occupation), int(rng))
        if not h:
            raise ValueError("invalid oracle configuration")
        self._h = ctypes.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.oracle_destroy(h)
            self._h = None

    def sweep(self, algo, beta, nsweeps, measure_every=0, nthreads=1):
        b = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float64), (self.K,)))
        lib().oracle_sweep(self._h, algo, b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nsweeps,
                           measure_every, nthreads)

    def pt_swap(self, beta):
        b = np.ascontiguousarray(np.asarray(beta, dtype=np.float64))
        lib().oracle_pt_swap(self._h, b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))

    @property
    def sweeps(self) -> int:
        return int(lib().oracle_sweeps(self._h))

    def measure(self):
        """Returns (E [S,K,R], M [S,K,R] or [S,K,R,q], Q [S,K] or None)."""
        S, K, R = self.S, self.K, self.R
        E = np.zeros((S, K, R), dtype=np.int64)
        M = np.zeros((S, K, R) if self.mq == 1 else (S, K, R, self.mq), dtype=np.int64)
        Q = np.zeros((S, K), dtype=np.int64)
        lib().oracle_measure(self._h, _ptr(E), _ptr(M), _ptr(Q) if R >= 2 else None)
        return E, M, (Q if R >= 2 else None)

    def series(self):
        n = int(lib().oracle_series_rows(self._h))
        S, K, R = self.S, self.K, self.R
        sw = np.zeros(n, dtype=np.uint64)
        E = np.zeros((n, S, K, R), dtype=np.int64)
        M = np.zeros((n, S, K, R) if self.mq == 1 else (n, S, K, R, self.mq), dtype=np.int64)
        Q = np.zeros((n, S, K), dtype=np.int64)
        lib().oracle_series(self._h, _ptr(sw), _ptr(E), _ptr(M), _ptr(Q))
        return sw, E, M, (Q if R >= 2 else None)

    def clear_series(self):
        lib().oracle_series_clear(self._h)

    def spins(self) -> np.ndarray:
        out = np.zeros((self.S, self.K * self.R, self.N), dtype=np.int8)
        lib().oracle_get_spins(self._h, _ptr(out))
        return out

    def set_spins(self, a):
        a = np.ascontiguousarray(a, dtype=np.int8).reshape(self.S, self.K * self.R, self.N)
        lib().oracle_set_spins(self._h, _ptr(a))

    def couplings(self) -> np.ndarray:
        out = np.zeros((self.S, self.dim, self.N), dtype=np.int8)
        lib().oracle_get_couplings(self._h, _ptr(out))
        return out

    def set_couplings(self, a):
        """J = +-1, or for the permutation model the 8-bit codes as int8."""
        a = np.ascontiguousarray(a, dtype=np.int8).reshape(self.S, self.dim, self.N)
        if lib().oracle_set_couplings(self._h, _ptr(a)) != 0:
            raise ValueError("coupling code is not a permutation")

    def sites(self):
        """(sign(h_i) [S, N], x_i [S, N]) as int8."""
        hs = np.zeros((self.S, self.N), dtype=np.int8)
        x = np.zeros((self.S, self.N), dtype=np.int8)
        lib().oracle_get_sites(self._h, _ptr(hs), _ptr(x))
        return hs, x

    def set_sites(self, hs=None, x=None):
        hs = None if hs is None else np.ascontiguousarray(hs, dtype=np.int8).reshape(self.S, self.N)
        x = None if x is None else np.ascontiguousarray(x, dtype=np.int8).reshape(self.S, self.N)
        lib().oracle_set_sites(self._h, None if hs is None else _ptr(hs), None if x is None else _ptr(x))

    def pt_state(self):
        S, R, K = self.S, self.R, self.K
        slot_at = np.zeros((S, R, K), dtype=np.int32)
        acc = np.zeros((S, R, max(K - 1, 0)), dtype=np.uint64)
        steps = np.zeros(1, dtype=np.uint64)
        lib().oracle_get_pt(self._h, _ptr(slot_at), _ptr(acc) if K > 1 else None, _ptr(steps))
        return slot_at, acc, int(steps[0])

    def bookkeeping_error(self) -> int:
        return int(lib().oracle_bookkeeping_error(self._h))
