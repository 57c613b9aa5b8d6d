"""GB300 checkerboard Monte Carlo for the EA +-J spin glass and the q=4 Potts glass.

Thin ctypes binding over ``libianus.so`` (C ABI in ``include/ianus.h``).  This
module only marshals arguments: every step of the sweep, the measurements and
the parallel-tempering swaps run in the library's CUDA kernels.  PyTorch is
used for device memory (the lattice state lives in a ``torch.uint8`` CUDA
tensor handed to the library) and for the current CUDA stream.

There is no CPU fallback: if the library cannot be built or loaded, or no
CUDA device is present, constructing a :class:`Lattice` raises.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

ABI_VERSION = 3

EA_PM_J, POTTS4_J, POTTS4_PERM = 0, 1, 2
METROPOLIS, HEATBATH = 0, 1
LAYOUT_AUTO, LAYOUT_I8, LAYOUT_BITS64, LAYOUT_U8X4 = 0, 1, 2, 3
DISORDER_PM_J, DISORDER_FERRO, DISORDER_RFIM, DISORDER_DAFF = 0, 1, 2, 3
RNG_PHILOX, RNG_WHEEL = 0, 1

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, ESTATE = range(7)

_MODELS = {"ea": EA_PM_J, "potts": POTTS4_J, "potts_perm": POTTS4_PERM}
_ALGOS = {"metropolis": METROPOLIS, "heatbath": HEATBATH}
_LAYOUTS = {"auto": LAYOUT_AUTO, "i8": LAYOUT_I8, "bits64": LAYOUT_BITS64, "u8x4": LAYOUT_U8X4}
_RNGS = {"philox": RNG_PHILOX, "wheel": RNG_WHEEL}
_DISORDERS = {"pm_j": DISORDER_PM_J, "ferro": DISORDER_FERRO, "rfim": DISORDER_RFIM, "daff": DISORDER_DAFF}

EXPORTS = [
    "ianus_required_bytes", "ianus_lattice_create", "ianus_sweep", "ianus_pt_swap", "ianus_sweep_pt",
    "ianus_measure", "ianus_read_series", "ianus_get_spins_i8", "ianus_set_spins_i8", "ianus_get_couplings_i8",
    "ianus_set_couplings_i8", "ianus_get_pt_state", "ianus_get_sweeps", "ianus_get_state", "ianus_set_state",
    "ianus_synchronize", "ianus_destroy", "ianus_status_string", "ianus_table_ising", "ianus_table_potts",
    "ianus_table_pt", "ianus_measure_bits64_noalloc", "ianus_set_variant", "ianus_set_block_words",
    "ianus_set_graphs", "ianus_set_resident", "ianus_get_sites_i8", "ianus_set_sites_i8", "ianus_table_field",
    "ianus_table_potts_counts", "ianus_segment_load", "ianus_segment_release", "ianus_segment_state",
    "ianus_sweep_segments", "ianus_set_persistent_wait", "ianus_prepare_sweep",
]


class IanusConfig(C.Structure):
    _fields_ = [
        ("abi_version", C.c_uint32),
        ("model", C.c_int32),
        ("dim", C.c_int32),
        ("L", C.c_int32),
        ("n_samples", C.c_int32),
        ("n_replicas", C.c_int32),
        ("n_temps", C.c_int32),
        ("layout", C.c_int32),
        ("disorder", C.c_int32),
        ("series_capacity", C.c_uint32),
        ("seed", C.c_uint64),
        ("device_buffer", C.c_void_p),
        ("device_buffer_bytes", C.c_size_t),
        ("cuda_stream", C.c_void_p),
        ("field", C.c_double),
        ("occupation", C.c_double),
        ("rng", C.c_int32),
    ]


class IanusError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libianus.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libianus.so not built at {_build.LIB}")
    L = C.CDLL(_build.LIB)
    vp, i32, u32, u64, sz, dp = C.c_void_p, C.c_int32, C.c_uint32, C.c_uint64, C.c_size_t, C.POINTER(C.c_double)
    cfgp = C.POINTER(IanusConfig)
    sig = {
        "ianus_required_bytes": (sz, [cfgp]),
        "ianus_lattice_create": (i32, [cfgp, C.POINTER(vp)]),
        "ianus_sweep": (i32, [vp, i32, dp, u64, u32]),
        "ianus_pt_swap": (i32, [vp]),
        "ianus_sweep_pt": (i32, [vp, i32, dp, u64, u32, u32]),
        "ianus_measure": (i32, [vp, vp, vp, vp]),
        "ianus_read_series": (i32, [vp, vp, vp, vp, vp, sz, C.POINTER(sz), i32]),
        "ianus_get_spins_i8": (i32, [vp, vp]),
        "ianus_set_spins_i8": (i32, [vp, vp]),
        "ianus_get_couplings_i8": (i32, [vp, vp]),
        "ianus_set_couplings_i8": (i32, [vp, vp]),
        "ianus_get_pt_state": (i32, [vp, vp, vp, C.POINTER(u64)]),
        "ianus_get_sweeps": (i32, [vp, C.POINTER(u64)]),
        "ianus_get_state": (i32, [vp, vp, sz, C.POINTER(sz)]),
        "ianus_set_state": (i32, [vp, vp, sz]),
        "ianus_synchronize": (i32, [vp]),
        "ianus_destroy": (i32, [vp]),
        "ianus_status_string": (C.c_char_p, [i32]),
        "ianus_table_ising": (sz, [i32, i32, C.c_double, vp, sz]),
        "ianus_table_potts": (sz, [C.c_double, vp, sz]),
        "ianus_table_pt": (sz, [C.c_double, C.c_double, vp, sz]),
        "ianus_measure_bits64_noalloc": (i32, [vp, vp, i32, i32, i32, i32, vp, vp, vp]),
        "ianus_set_variant": (i32, [vp, i32]),
        "ianus_set_block_words": (i32, [vp, u32]),
        "ianus_set_persistent_wait": (i32, [vp, u64, i32]),
        "ianus_prepare_sweep": (i32, [vp, i32, vp, i32, vp]),
        "ianus_set_graphs": (i32, [vp, i32]),
        "ianus_set_resident": (i32, [vp, i32]),
        "ianus_get_sites_i8": (i32, [vp, vp, vp]),
        "ianus_set_sites_i8": (i32, [vp, vp, vp]),
        "ianus_table_field": (sz, [i32, i32, C.c_double, C.c_double, vp, sz]),
        "ianus_table_potts_counts": (sz, [C.c_double, vp, vp]),
        "ianus_segment_load": (i32, [vp, i32, i32, i32, u64, i32, i32, C.c_double, u64]),
        "ianus_segment_release": (i32, [vp, i32, i32]),
        "ianus_segment_state": (i32, [vp, i32, i32, C.POINTER(u64), C.POINTER(u64)]),
        "ianus_sweep_segments": (i32, [vp, u64]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def status_string(st: int) -> str:
    return lib().ianus_status_string(st).decode()


def _check(st: int, what: str):
    if st != OK:
        raise IanusError(st, what)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def table_ising(dim: int, algo: int, beta: float) -> np.ndarray:
    out = np.zeros(8, dtype=np.uint64)
    n = lib().ianus_table_ising(dim, algo, beta, _ptr(out), 8)
    return out[:n]


def table_potts(beta: float) -> np.ndarray:
    out = np.zeros(3 * 13 ** 4, dtype=np.uint64)
    n = lib().ianus_table_potts(beta, _ptr(out), out.size)
    if n != out.size:
        raise ValueError("bad beta")
    return out.reshape(13, 13, 13, 13, 3)


def table_pt(beta_k: float, beta_k1: float, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    lib().ianus_table_pt(beta_k, beta_k1, _ptr(out), n)
    return out


def table_potts_counts(beta: float, n) -> list[int]:
    """Potts heat-bath thresholds T_0..T_2 for one tuple of counts n_0..n_3."""
    nn = np.ascontiguousarray(n, dtype=np.int32)
    out = np.zeros(3, dtype=np.uint64)
    if lib().ianus_table_potts_counts(beta, _ptr(nn), _ptr(out)) != 3:
        raise ValueError("bad table arguments")
    return [int(v) for v in out]


def table_field(dim: int, algo: int, beta: float, field: float) -> np.ndarray:
    """Thresholds of the field models, indexed [(v + 2 dim) * 2 + f]."""
    out = np.zeros(32, dtype=np.uint64)
    n = lib().ianus_table_field(dim, algo, beta, field, _ptr(out), out.size)
    if n == 0:
        raise ValueError("bad table arguments")
    return out[:n]


class Lattice:
    """A batch of lattices: n_samples disorder samples x n_temps x n_replicas.

    The device state is held in a torch CUDA byte tensor (``self.buffer``);
    all work is enqueued on ``stream`` (default: torch's current stream).
    """

    def __init__(self, model="ea", dim=3, L=16, n_samples=1, n_replicas=1, n_temps=1, seed=0,
                 layout="auto", ferro=False, series_capacity=0, stream=None, device=None, disorder=None,
                 field=0.0, occupation=1.0, rng="philox"):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("paper_0704_3573_gb300 needs a CUDA device (no CPU fallback)")
        self._lib = lib()
        self.model = _MODELS[model] if isinstance(model, str) else int(model)
        self.dim, self.L = dim, L
        self.N = L ** dim
        self.S, self.R, self.K = n_samples, n_replicas, n_temps
        if disorder is None:
            disorder = DISORDER_FERRO if ferro else DISORDER_PM_J
        self.disorder = _DISORDERS[disorder] if isinstance(disorder, str) else int(disorder)
        self.field, self.occupation = float(field), float(occupation)
        self.mq = 4 if self.model != EA_PM_J else (2 if self.disorder in (DISORDER_RFIM, DISORDER_DAFF) else 1)
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        cfg = IanusConfig()
        cfg.abi_version = ABI_VERSION
        cfg.model = self.model
        cfg.dim, cfg.L = dim, L
        cfg.n_samples, cfg.n_replicas, cfg.n_temps = n_samples, n_replicas, n_temps
        cfg.layout = _LAYOUTS[layout] if isinstance(layout, str) else int(layout)
        cfg.disorder = self.disorder
        cfg.field = self.field
        cfg.occupation = self.occupation
        cfg.rng = _RNGS[rng] if isinstance(rng, str) else int(rng)
        cfg.series_capacity = series_capacity
        cfg.seed = seed & 0xFFFFFFFFFFFFFFFF
        nbytes = self._lib.ianus_required_bytes(C.byref(cfg))
        if nbytes == 0:
            # invalid configuration: ianus_lattice_create validates it the
            # same way (before any allocation) and names the reason
            h = C.c_void_p()
            st = self._lib.ianus_lattice_create(C.byref(cfg), C.byref(h))
            raise IanusError(st if st != OK else EINVAL, "ianus_lattice_create")
        with torch.cuda.device(dev):
            self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        cfg.device_buffer = self.buffer.data_ptr()
        cfg.device_buffer_bytes = nbytes
        cfg.cuda_stream = stream.cuda_stream
        self.cfg = cfg
        self._h = C.c_void_p()
        with torch.cuda.device(dev):
            _check(self._lib.ianus_lattice_create(C.byref(cfg), C.byref(self._h)), "ianus_lattice_create")
        self.device = dev

    # ---- lifetime ----
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.ianus_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- the hot path ----
    def _beta(self, beta) -> np.ndarray:
        return np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float64), (self.K,)))

    def sweep(self, algo, beta, nsweeps: int, measure_every: int = 0):
        a = _ALGOS[algo] if isinstance(algo, str) else int(algo)
        b = self._beta(beta)
        _check(self._lib.ianus_sweep(self._h, a, b.ctypes.data_as(C.POINTER(C.c_double)), nsweeps, measure_every),
               "ianus_sweep")

    def prepare_sweep(self, algo, beta, variant: int = 0) -> bool:
        """Compile (or find cached) the kernel a sweep at (algo, beta) under
        `variant` would specialise, without launching or changing anything;
        True when that kernel is ready.  Safe on a worker thread while other
        threads sweep (the call releases the GIL)."""
        a = _ALGOS[algo] if isinstance(algo, str) else int(algo)
        b = self._beta(beta)
        ready = C.c_int32(0)
        _check(self._lib.ianus_prepare_sweep(self._h, a, b.ctypes.data_as(C.POINTER(C.c_double)), int(variant),
                                             C.byref(ready)), "ianus_prepare_sweep")
        return bool(ready.value)

    def pt_swap(self):
        _check(self._lib.ianus_pt_swap(self._h), "ianus_pt_swap")

    # ---- fused serving (pool lattices) ----
    def segment_load(self, group: int, lane0: int, n: int, seed: int, algo, beta: float, nsweeps: int,
                     job_group: int = 0):
        """Samples 64 job_group .. + n - 1 of the job with this seed into
        lanes lane0 .. lane0 + n - 1 of `group`."""
        a = _ALGOS[algo] if isinstance(algo, str) else int(algo)
        _check(self._lib.ianus_segment_load(self._h, group, lane0, n, seed & 0xFFFFFFFFFFFFFFFF, job_group, a,
                                            float(beta), nsweeps), "ianus_segment_load")

    def segment_release(self, group: int, lane0: int):
        _check(self._lib.ianus_segment_release(self._h, group, lane0), "ianus_segment_release")

    def segment_state(self, group: int, lane0: int) -> tuple[int, int]:
        done, req = C.c_uint64(), C.c_uint64()
        _check(self._lib.ianus_segment_state(self._h, group, lane0, C.byref(done), C.byref(req)),
               "ianus_segment_state")
        return int(done.value), int(req.value)

    def sweep_segments(self, nsweeps: int):
        _check(self._lib.ianus_sweep_segments(self._h, nsweeps), "ianus_sweep_segments")

    def sweep_pt(self, algo, beta, nsweeps: int, swap_every: int, measure_every: int = 0):
        a = _ALGOS[algo] if isinstance(algo, str) else int(algo)
        b = self._beta(beta)
        _check(self._lib.ianus_sweep_pt(self._h, a, b.ctypes.data_as(C.POINTER(C.c_double)), nsweeps, swap_every,
                                        measure_every), "ianus_sweep_pt")

    # ---- observables ----
    def measure(self, overlap: bool | None = None):
        """(E [S,K,R], M [S,K,R] or [S,K,R,4], Q [S,K] or None), exact int64."""
        S, K, R = self.S, self.K, self.R
        E = np.zeros((S, K, R), dtype=np.int64)
        M = np.zeros((S, K, R) if self.mq == 1 else (S, K, R, self.mq), dtype=np.int64)
        want_q = (R >= 2) if overlap is None else overlap
        Q = np.zeros((S, K), dtype=np.int64) if want_q else None
        _check(self._lib.ianus_measure(self._h, _ptr(E), _ptr(M), _ptr(Q)), "ianus_measure")
        return E, M, Q

    def series(self, clear: bool = False, max_rows: int = 1 << 20):
        S, K, R = self.S, self.K, self.R
        cap = min(max_rows, self.cfg.series_capacity or 1024)
        sw = np.zeros(cap, dtype=np.uint64)
        E = np.zeros((cap, S, K, R), dtype=np.int64)
        M = np.zeros((cap, S, K, R) if self.mq == 1 else (cap, S, K, R, self.mq), dtype=np.int64)
        Q = np.zeros((cap, S, K), dtype=np.int64) if R >= 2 else None
        n = C.c_size_t()
        _check(self._lib.ianus_read_series(self._h, _ptr(sw), _ptr(E), _ptr(M), _ptr(Q), cap, C.byref(n),
                                           int(clear)), "ianus_read_series")
        k = n.value
        return sw[:k], E[:k], M[:k], (Q[:k] if Q is not None else None)

    def spins(self) -> np.ndarray:
        out = np.zeros((self.S, self.K * self.R, self.N), dtype=np.int8)
        _check(self._lib.ianus_get_spins_i8(self._h, _ptr(out)), "ianus_get_spins_i8")
        return out

    def set_spins(self, a):
        a = np.ascontiguousarray(a, dtype=np.int8).reshape(self.S, self.K * self.R, self.N)
        _check(self._lib.ianus_set_spins_i8(self._h, _ptr(a)), "ianus_set_spins_i8")

    def couplings(self) -> np.ndarray:
        out = np.zeros((self.S, self.dim, self.N), dtype=np.int8)
        _check(self._lib.ianus_get_couplings_i8(self._h, _ptr(out)), "ianus_get_couplings_i8")
        return out

    def set_couplings(self, a):
        a = np.ascontiguousarray(a, dtype=np.int8).reshape(self.S, self.dim, self.N)
        _check(self._lib.ianus_set_couplings_i8(self._h, _ptr(a)), "ianus_set_couplings_i8")

    def sites(self):
        """(sign of h_i [S, N], x_i [S, N]) as int8 (Ising-like models)."""
        hs = np.zeros((self.S, self.N), dtype=np.int8)
        x = np.zeros((self.S, self.N), dtype=np.int8)
        _check(self._lib.ianus_get_sites_i8(self._h, _ptr(hs), _ptr(x)), "ianus_get_sites_i8")
        return hs, x

    def set_sites(self, hs=None, x=None):
        hs = None if hs is None else np.ascontiguousarray(hs, dtype=np.int8).reshape(self.S, self.N)
        x = None if x is None else np.ascontiguousarray(x, dtype=np.int8).reshape(self.S, self.N)
        _check(self._lib.ianus_set_sites_i8(self._h, _ptr(hs), _ptr(x)), "ianus_set_sites_i8")

    def pt_state(self):
        S, R, K = self.S, self.R, self.K
        slot_at = np.zeros((S, R, K), dtype=np.int32)
        acc = np.zeros((S, R, max(K - 1, 0)), dtype=np.uint64)
        steps = C.c_uint64()
        _check(self._lib.ianus_get_pt_state(self._h, _ptr(slot_at), _ptr(acc) if K > 1 else None, C.byref(steps)),
               "ianus_get_pt_state")
        return slot_at, acc, steps.value

    @property
    def sweeps(self) -> int:
        v = C.c_uint64()
        _check(self._lib.ianus_get_sweeps(self._h, C.byref(v)), "ianus_get_sweeps")
        return v.value

    def get_state(self) -> bytes:
        n = C.c_size_t()
        _check(self._lib.ianus_get_state(self._h, None, 0, C.byref(n)), "ianus_get_state")
        buf = np.zeros(n.value, dtype=np.uint8)
        _check(self._lib.ianus_get_state(self._h, _ptr(buf), n.value, C.byref(n)), "ianus_get_state")
        return buf.tobytes()

    def set_state(self, blob: bytes):
        buf = np.frombuffer(blob, dtype=np.uint8).copy()
        _check(self._lib.ianus_set_state(self._h, _ptr(buf), buf.size), "ianus_set_state")

    def set_variant(self, variant: int):
        """Bit-sliced sweep kernel: 0 automatic, 1 per-lane threshold planes,
        2..27 shapes of the kernel specialised at run time (include/ianus.h)."""
        _check(self._lib.ianus_set_variant(self._h, variant), "ianus_set_variant")

    def set_block_words(self, words: int):
        """Colour words per 256-thread block of the bit-sliced sweep (0 = default)."""
        _check(self._lib.ianus_set_block_words(self._h, words), "ianus_set_block_words")

    def set_persistent_wait(self, timeout_ns: int, absent_block: int = -1):
        """Bound of each wait of the persistent sweep (variants 25..27), and a
        block told to return at once (tests of the timeout path; -1 none)."""
        _check(self._lib.ianus_set_persistent_wait(self._h, int(timeout_ns), int(absent_block)),
               "ianus_set_persistent_wait")

    def set_graphs(self, enable: bool):
        """Replay sweep blocks from captured CUDA graphs (default) or launch directly."""
        _check(self._lib.ianus_set_graphs(self._h, int(bool(enable))), "ianus_set_graphs")

    def set_resident(self, enable):
        """Shared-memory-resident sweeps for small lattices.  Plain layout:
        True / 1 (default: a block cluster per configuration when there are
        few), 2 (one block per configuration always), 3 (a cluster per
        configuration whenever one can be formed), False / 0 (off).
        Bit-sliced layout (automatic variant) and pools: any nonzero value
        on, 0 off."""
        _check(self._lib.ianus_set_resident(self._h, int(enable)), "ianus_set_resident")

    def synchronize(self):
        _check(self._lib.ianus_synchronize(self._h), "ianus_synchronize")
