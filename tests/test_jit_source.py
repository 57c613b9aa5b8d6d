"""The kernels compiled at run time (csrc/jit_sweep.cuh, csrc/jit_field.cuh,
csrc/sweep_planes.cuh) compile with NVRTC for sm_103a for the parameter sets
the library generates, with and without the lattice geometry as constants.
NVRTC needs no GPU, so this runs on the CPU host; the GPU parity tests then
check the compiled kernels' results bit for bit."""

import ctypes as C
import os

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0704_3573_gb300", "csrc")


def _nvrtc():
    for name in ("libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"):
        try:
            return C.CDLL(name)
        except OSError:
            continue
    pytest.skip("NVRTC not available")


@pytest.mark.parametrize("D,algo,R,P2,mode,phase,minb,group,jr,uf", [
    (3, 1, 2, 1, 0, 8, 3, 1, 0, 0), (3, 0, 1, 0, 1, 3, 4, 1, 0, 0), (2, 1, 1, 1, 1, 4, 3, 1, 0, 0),
    (2, 0, 2, 0, 0, 8, 4, 1, 0, 0), (3, 1, 2, 1, 0, 8, 3, 2, 0, 0), (3, 1, 2, 0, 1, 4, 3, 2, 0, 0),
    (2, 0, 1, 1, 1, 6, 3, 2, 0, 0), (3, 1, 2, 1, 1, 4, 4, 2, 1, 0), (3, 0, 2, 0, 0, 8, 4, 1, 1, 0),
    (2, 1, 1, 1, 1, 4, 4, 1, 1, 0), (3, 1, 2, 1, 1, 4, 3, 2, 0, 1), (3, 0, 2, 0, 0, 8, 4, 2, 0, 1),
    (2, 1, 1, 0, 0, 8, 3, 2, 0, 1)])
def test_jit_kernel_compiles_for_sm103a(D, algo, R, P2, mode, phase, minb, group, jr, uf):
    lib = _nvrtc()
    hdrs = [open(os.path.join(CSRC, n), "rb").read() for n in ("common.cuh", "jit_sweep.cuh")]
    luts = ",".join(str((13 * q + 5) & 0x7F) for q in range(32))
    pre = (f"#define IANUS_JIT_D {D}\n#define IANUS_JIT_ALGO {algo}\n#define IANUS_JIT_R {R}\n"
           f"#define IANUS_JIT_P2 {P2}\n#define IANUS_JIT_LUTS {luts}\n#define IANUS_JIT_ALWAYS 0\n"
           f"#define IANUS_JIT_NEED 127\n#define IANUS_JIT_MODE {mode}\n#define IANUS_JIT_PHASEA {phase}\n"
           f"#define IANUS_JIT_MINB {minb}\n#define IANUS_JIT_GROUP {group}\n#define IANUS_JIT_JRELOAD {jr}\n#define IANUS_JIT_UFIRST {uf}\n")
    if mode == 1 or uf:  # geometry as constants: L = 64 (power of two) or 12
        pre += "#define IANUS_JIT_L 64\n#define IANUS_JIT_LH 5\n#define IANUS_JIT_LL 6\n" if P2 else \
            "#define IANUS_JIT_L 12\n#define IANUS_JIT_LH 0\n#define IANUS_JIT_LL 0\n"
    pre = (pre + "#include \"jit_sweep.cuh\"\n").encode()
    prog = C.c_void_p()
    H = (C.c_char_p * 2)(*hdrs)
    N = (C.c_char_p * 2)(b"common.cuh", b"jit_sweep.cuh")
    assert lib.nvrtcCreateProgram(C.byref(prog), pre, b"ianus_jit_sweep.cu", 2, H, N) == 0
    opts = (C.c_char_p * 2)(b"--gpu-architecture=sm_103a", b"-std=c++17")
    rc = lib.nvrtcCompileProgram(prog, 2, opts)
    n = C.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, C.byref(n))
    log = C.create_string_buffer(n.value)
    lib.nvrtcGetProgramLog(prog, log)
    size = C.c_size_t()
    lib.nvrtcGetCUBINSize(prog, C.byref(size))
    lib.nvrtcDestroyProgram(C.byref(prog))
    assert rc == 0, log.value.decode()
    assert size.value > 1000


@pytest.mark.parametrize("D,algo,R,P2,dil", [(3, 1, 1, 1, 0), (3, 0, 2, 0, 0), (2, 1, 2, 1, 0), (3, 0, 1, 1, 1),
                                             (3, 1, 2, 0, 1), (2, 0, 2, 1, 1)])
def test_jit_field_kernel_compiles_for_sm103a(D, algo, R, P2, dil):
    lib = _nvrtc()
    hdrs = [open(os.path.join(CSRC, n), "rb").read() for n in ("common.cuh", "jit_field.cuh")]
    pre = (f"#define IANUS_JIT_D {D}\n#define IANUS_JIT_ALGO {algo}\n#define IANUS_JIT_R {R}\n"
           f"#define IANUS_JIT_P2 {P2}\n#define IANUS_JIT_MINB 3\n#define IANUS_JIT_DILUTE {dil}\n")
    pre += "#define IANUS_JIT_L 32\n#define IANUS_JIT_LH 4\n#define IANUS_JIT_LL 5\n" if P2 else \
        "#define IANUS_JIT_L 10\n#define IANUS_JIT_LH 0\n#define IANUS_JIT_LL 0\n"
    for f in range(2):
        for h in range(2):
            pre += f"#define IANUS_JIT_LUT{f}{h} " + ",".join(str((13 * q + 5 * f + 3 * h) & 0x7F) for q in range(32))
            pre += f"\n#define IANUS_JIT_ALWAYS{f}{h} {64 * f}\n#define IANUS_JIT_NEED{f}{h} {127 - 64 * f}\n"
    pre = (pre + "#include \"jit_field.cuh\"\n").encode()
    prog = C.c_void_p()
    H = (C.c_char_p * 2)(*hdrs)
    N = (C.c_char_p * 2)(b"common.cuh", b"jit_field.cuh")
    assert lib.nvrtcCreateProgram(C.byref(prog), pre, b"ianus_jit.cu", 2, H, N) == 0
    opts = (C.c_char_p * 2)(b"--gpu-architecture=sm_103a", b"-std=c++17")
    rc = lib.nvrtcCompileProgram(prog, 2, opts)
    n = C.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, C.byref(n))
    log = C.create_string_buffer(n.value)
    lib.nvrtcGetProgramLog(prog, log)
    lib.nvrtcDestroyProgram(C.byref(prog))
    assert rc == 0, log.value.decode()


@pytest.mark.parametrize("D,algo,RT,L,Q,minb", [(3, 0, 2, 32, 0, 4), (3, 1, 2, 32, 1, 3), (3, 1, 0, 12, 1, 3),
                                                (2, 0, 1, 64, 0, 4), (2, 1, 0, 10, 0, 4), (3, 0, 0, 6, 0, 4)])
def test_jit_planes_kernel_compiles_for_sm103a(D, algo, RT, L, Q, minb):
    lib = _nvrtc()
    hdrs = [open(os.path.join(CSRC, n), "rb").read() for n in ("common.cuh", "sweep_planes.cuh")]
    p2 = L & (L - 1) == 0
    lh, ll = ((L // 2).bit_length() - 1, L.bit_length() - 1) if p2 else (0, 0)
    pre = (f"#define IANUS_JIT_PLANES 1\n#define IANUS_JIT_D {D}\n#define IANUS_JIT_ALGO {algo}\n"
           f"#define IANUS_JIT_RT {RT}\n#define IANUS_JIT_P2 {int(p2)}\n#define IANUS_JIT_Q {Q}\n"
           f"#define IANUS_JIT_MINB {minb}\n#define IANUS_JIT_L {L}\n#define IANUS_JIT_LH {lh}\n"
           f"#define IANUS_JIT_LL {ll}\n#include \"sweep_planes.cuh\"\n").encode()
    prog = C.c_void_p()
    H = (C.c_char_p * 2)(*hdrs)
    N = (C.c_char_p * 2)(b"common.cuh", b"sweep_planes.cuh")
    assert lib.nvrtcCreateProgram(C.byref(prog), pre, b"ianus_jit.cu", 2, H, N) == 0
    opts = (C.c_char_p * 2)(b"--gpu-architecture=sm_103a", b"-std=c++17")
    rc = lib.nvrtcCompileProgram(prog, 2, opts)
    n = C.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, C.byref(n))
    log = C.create_string_buffer(n.value)
    lib.nvrtcGetProgramLog(prog, log)
    lib.nvrtcDestroyProgram(C.byref(prog))
    assert rc == 0, log.value.decode()
