"""GPU test of ianus_measure_bits64_noalloc, the measurement entry point for
callers that cannot allocate device memory.

Such callers include code running inside a framework that owns all device
memory through its own pool (a direct cudaMalloc would bypass the pool and can
fail once it has reserved the GPU), and serving loops that must not call
cudaMalloc or cudaFree because those synchronise the device and stall other
streams.  The entry point keeps its counters in a fixed device array inside
the library and is handed device pointers for its inputs and outputs.

The test packs a lattice's spins and couplings into the bit-sliced layout
itself, calls the entry point through the C ABI twice in a row (on two
different configurations, so the second call must not see the first call's
counts), and compares each result with what ianus_measure reports for the
same lattice.  Values are exact integers, so the comparison is exact.  The
file is named to be collected last.
"""

import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pack_bits64(a, L, dim):
    """int8 array [n_samples][m][L^dim] of +-1 -> uint64 [groups][m][L^dim]
    in checkerboard-split site order, lane l = sample 64 g + l, bit 1 = -1."""
    S, m, N = a.shape
    G = (S + 63) // 64
    bits = np.zeros((G * 64, m, N), dtype=np.uint64)
    bits[:S] = (a < 0).astype(np.uint64)
    bits = bits.reshape(G, 64, m, N)
    words = np.zeros((G, m, N), dtype=np.uint64)
    for lane in range(64):
        words |= bits[:, lane] << np.uint64(lane)
    i = np.arange(N)
    x, y = i % L, (i // L) % L
    z = i // (L * L) if dim == 3 else np.zeros_like(i)
    split = (2 * (y + L * z) + ((x + y + z) & 1)) * (L // 2) + x // 2
    out = np.zeros_like(words)
    out[:, :, split] = words
    return out


def _call_noalloc(ianus, lat, torch):
    spins = torch.from_numpy(_pack_bits64(lat.spins(), lat.L, lat.dim).view(np.int64)).cuda()
    J = torch.from_numpy(_pack_bits64(lat.couplings(), lat.L, lat.dim).view(np.int64)).cuda()
    slots = lat.K * lat.R
    E = torch.full((lat.S, slots), -7, dtype=torch.int64, device="cuda")
    M = torch.full((lat.S, slots), -7, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    st = ianus.lib().ianus_measure_bits64_noalloc(
        C.c_void_p(spins.data_ptr()), C.c_void_p(J.data_ptr()), lat.dim, lat.L, lat.S, slots,
        C.c_void_p(E.data_ptr()), C.c_void_p(M.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert st == ianus.OK, ianus.status_string(st)
    torch.cuda.synchronize()
    return E.cpu().numpy(), M.cpu().numpy()


# the last case fills the fixed array exactly: 16384 samples x 2 slots = 32768
@pytest.mark.parametrize("dim,L,S,R", [(3, 8, 70, 2), (2, 16, 5, 1), (3, 4, 130, 2), (3, 4, 16384, 2)])
def test_noalloc_measure_matches_ianus_measure_twice(ianus, dim, L, S, R):
    import torch

    lat = ianus.Lattice(dim=dim, L=L, n_samples=S, n_replicas=R, seed=0x0704357300000077, layout="bits64")
    for call in range(2):
        lat.sweep(ianus.HEATBATH, 0.9, 3 + call)
        E_ref, M_ref, _ = lat.measure(overlap=False)  # [S][1][R]: one temperature, slot = replica
        E, M = _call_noalloc(ianus, lat, torch)
        assert np.array_equal(E, E_ref[:, 0, :]), call
        assert np.array_equal(M, M_ref[:, 0, :]), call


def test_noalloc_rejects_sizes_over_the_limit(ianus):
    import torch

    lib = ianus.lib()
    dummy = torch.zeros(8, dtype=torch.int64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    # 32768 (sample, slot) pairs is the stated maximum
    assert lib.ianus_measure_bits64_noalloc(p, p, 3, 4, 16385, 2, p, p, None) == ianus.EINVAL
    assert lib.ianus_measure_bits64_noalloc(p, p, 3, 5, 1, 1, p, p, None) == ianus.EINVAL
    assert lib.ianus_measure_bits64_noalloc(None, p, 3, 4, 1, 1, p, p, None) == ianus.EINVAL


def test_noalloc_allocates_no_device_memory(ianus):
    """After a first call (which looks up the array's device address), a
    second call leaves the device's free memory exactly as it was: nothing is
    allocated, by the library or by the CUDA runtime on its behalf."""
    import torch

    lat = ianus.Lattice(dim=3, L=8, n_samples=70, n_replicas=2, seed=0x0704357300000078, layout="bits64")
    lat.sweep(ianus.HEATBATH, 0.9, 2)
    spins = torch.from_numpy(_pack_bits64(lat.spins(), lat.L, lat.dim).view(np.int64)).cuda()
    J = torch.from_numpy(_pack_bits64(lat.couplings(), lat.L, lat.dim).view(np.int64)).cuda()
    E = torch.zeros((lat.S, 2), dtype=torch.int64, device="cuda")
    M = torch.zeros((lat.S, 2), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    args = (C.c_void_p(spins.data_ptr()), C.c_void_p(J.data_ptr()), lat.dim, lat.L, lat.S, 2,
            C.c_void_p(E.data_ptr()), C.c_void_p(M.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert ianus.lib().ianus_measure_bits64_noalloc(*args) == ianus.OK
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    assert ianus.lib().ianus_measure_bits64_noalloc(*args) == ianus.OK
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
