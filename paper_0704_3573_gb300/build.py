"""In-tree build of libianus.so for sm_103a (GB300) with nvcc.

Each translation unit under ``csrc/`` is compiled in parallel, then linked
into ``paper_0704_3573_gb300/libianus.so`` against the shared CUDA runtime.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libianus.so")
BUILD_DIR = os.path.join(ROOT, "_build")

SOURCES = ["api.cu", "k_plain.cu", "k_msc.cu", "k_potts.cu", "k_pt.cu", "tables.cpp", "noalloc.cu"]
PROBE_SOURCES = ["probe.cu"]
PROBE_LIB = os.path.join(HERE, "libianus_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return cand


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "ianus.h"))
    files.append(os.path.join(INCLUDE, "ianus_probe.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    for lib in (LIB, PROBE_LIB):
        if not os.path.exists(lib):
            return False
        t = os.path.getmtime(lib)
        if not all(os.path.getmtime(f) <= t for f in _deps()):
            return False
    return True


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [cc, "-x", "cu", *cmd[1:]]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) + len(PROBE_SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES + PROBE_SOURCES))
    if verbose or ptxas_verbose:
        for (obj, err) in results:
            if err.strip():
                print(f"== {os.path.basename(obj)}\n{err}")
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(cc)), "lib64")
    objs = [o for o, _ in results]
    for lib, n in ((LIB, len(SOURCES)), (PROBE_LIB, None)):
        part = objs[:n] if n is not None else objs[len(SOURCES):]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *part, "-Xlinker", f"-rpath={cuda_lib}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force=True, ptxas_verbose="-v" in sys.argv))
