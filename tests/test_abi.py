"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every entry point include/ianus.h declares, validates configurations, and its
host table builders agree bytewise with the oracle's independent builders;
without a GPU the product path refuses to run."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_0704_3573_gb300 as ianus

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ianus.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ianus_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = ianus.lib()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(ianus.EXPORTS)


def test_status_strings():
    for st in range(7):
        assert ianus.status_string(st) != "unknown status"
    assert ianus.status_string(99) == "unknown status"


def _cfg(**kw):
    c = ianus.IanusConfig()
    c.abi_version = ianus.ABI_VERSION
    c.model, c.dim, c.L = kw.get("model", 0), kw.get("dim", 3), kw.get("L", 16)
    c.n_samples, c.n_replicas, c.n_temps = kw.get("S", 1), kw.get("R", 1), kw.get("K", 1)
    c.layout, c.disorder, c.seed = kw.get("layout", 0), kw.get("disorder", 0), 1
    c.field, c.occupation = kw.get("field", 0.0), kw.get("occupation", 1.0)
    c.rng = kw.get("rng", 0)
    return c


def test_required_bytes_validation():
    lib = ianus.lib()
    rb = lambda **kw: lib.ianus_required_bytes(ctypes.byref(_cfg(**kw)))
    assert rb() > 0
    assert rb(L=5) == 0                      # odd side
    assert rb(L=0) == 0
    assert rb(dim=4) == 0                    # 4D: the permutation Potts model only
    assert rb(model=1, dim=4) == 0
    assert rb(model=2, dim=4, L=4) > 0
    assert rb(model=2, dim=4, L=4, layout=2) == 0
    assert rb(model=3) == 0
    # Parisi-Rapuano wheels: Ising-like model, plain layout (AUTO picks it)
    W = ianus.RNG_WHEEL
    assert rb(rng=W, layout=1) > rb(layout=1)
    assert rb(rng=W) == rb(rng=W, layout=1)
    assert rb(rng=W, layout=2) == 0
    assert rb(model=1, rng=W) == 0
    assert rb(rng=2) == 0
    # one ring of 64 words per (slot, sample, colour, row)
    assert rb(rng=W, layout=1, L=16, S=3, R=2) - rb(layout=1, L=16, S=3, R=2) >= 6 * 2 * 64 * 256 * 4
    assert rb(S=0) == 0
    assert rb(R=64, K=64) == 0               # slot field limit 4096
    assert rb(model=1, layout=1) == 0        # Potts has no I8 layout
    assert rb(model=0, layout=3) == 0        # Ising has no U8X4 layout
    # BITS64 state: 256 samples x 2 replicas of 64^3 = 16 MiB spins + 24 MiB
    # couplings, plus a 1024-row measurement series of 10 MiB
    n = rb(L=64, S=256, R=2, layout=2)
    assert 40 * 2 ** 20 <= n < 52 * 2 ** 20
    bad = _cfg()
    bad.abi_version = 99
    assert lib.ianus_required_bytes(ctypes.byref(bad)) == 0


def test_field_model_validation():
    lib = ianus.lib()
    rb = lambda **kw: lib.ianus_required_bytes(ctypes.byref(_cfg(**kw)))
    RFIM, DAFF = ianus.DISORDER_RFIM, ianus.DISORDER_DAFF
    assert rb(disorder=RFIM, field=1.5) > 0
    assert rb(disorder=RFIM, field=1.5, layout=1) > 0
    assert rb(disorder=DAFF, field=0.5, occupation=0.7) > 0
    assert rb(disorder=DAFF, field=0.5, occupation=0.7, layout=1) > 0
    assert rb(disorder=DAFF, field=0.5, occupation=0.7, layout=2) > 0   # bit-sliced with dilution
    assert rb(disorder=DAFF, occupation=1.5) == 0
    assert rb(disorder=DAFF, occupation=float("nan")) == 0
    assert rb(disorder=RFIM, field=-1.0) == 0
    assert rb(disorder=RFIM, field=float("inf")) == 0
    assert rb(disorder=0, field=0.5) == 0                                # EA takes no field
    assert rb(disorder=4) == 0
    assert rb(model=1, disorder=RFIM, field=1.0) == 0                    # Potts has no field model
    # the field model adds its sites (64-bit words) and field planes
    assert rb(disorder=RFIM, field=1.0, L=16, S=64, layout=2) > rb(L=16, S=64, layout=2)
    # bit-sliced sweeps stage one block's planes in shared memory: bounded replicas
    assert rb(L=8, S=64, R=110, layout=2) > 0 and rb(L=8, S=64, R=111, layout=2) == 0
    assert rb(disorder=RFIM, field=1.0, L=8, S=64, R=55, layout=2) > 0
    assert rb(disorder=RFIM, field=1.0, L=8, S=64, R=56, layout=2) == 0
    assert rb(disorder=DAFF, field=1.0, L=8, S=64, R=27, layout=2) > 0   # 32 plane classes
    assert rb(disorder=DAFF, field=1.0, L=8, S=64, R=28, layout=2) == 0


@pytest.mark.parametrize("beta", [0.0, 0.25, 1 / 1.1, 1.0, 2.0, 7.5])
def test_ising_tables_match_oracle(beta):
    for dim in (2, 3):
        t = ianus.table_ising(dim, ianus.METROPOLIS, beta)
        assert [int(v) for v in t] == [oracle.table_metropolis(beta, 4 * (j + 1)) for j in range(dim)]
        t = ianus.table_ising(dim, ianus.HEATBATH, beta)
        assert [int(v) for v in t] == [oracle.table_heatbath(beta, -2 * dim + 2 * j) for j in range(2 * dim + 1)]


@pytest.mark.parametrize("beta", [0.0, 0.8, 1.25])
def test_potts_table_matches_oracle(beta):
    t = ianus.table_potts(beta)
    rng = np.random.default_rng(0)
    for _ in range(300):
        n = rng.integers(-6, 7, size=4)
        assert [int(v) for v in t[n[0] + 6, n[1] + 6, n[2] + 6, n[3] + 6]] == oracle.table_potts(beta, list(n))


def test_pt_table_matches_oracle():
    t = ianus.table_pt(1 / 0.7, 1 / (0.7 + 0.9 / 31), 64)
    db = abs(1 / 0.7 - 1 / (0.7 + 0.9 / 31))
    assert [int(v) for v in t] == [oracle.table_pt(db, 4 * m) for m in range(1, 65)]


@pytest.mark.parametrize("beta,h", [(0.0, 0.0), (0.3, 0.5), (1 / 1.1, 1.0), (1.0, 2.25), (4.0, 0.75), (0.5, 13.0)])
def test_field_tables_match_oracle(beta, h):
    for dim in (2, 3):
        for algo, ref in ((ianus.METROPOLIS, oracle.table_metropolis_x), (ianus.HEATBATH, oracle.table_heatbath_x)):
            t = ianus.table_field(dim, algo, beta, h)
            assert len(t) == 2 * (4 * dim + 1)
            for v in range(-2 * dim, 2 * dim + 1):
                for f in (0, 1):
                    w = 0.0 if h == 0 else (h if f else -h)
                    x = float(v) + w
                    if algo == ianus.METROPOLIS and 2 * x <= 0:
                        want = 1 << 32  # dE <= 0 always flips
                    else:
                        want = ref(beta, x)
                    assert int(t[(v + 2 * dim) * 2 + f]) == want, (dim, algo, v, f)
    # at h = 0 the field tables are the EA tables
    for dim in (2, 3):
        t = ianus.table_field(dim, ianus.HEATBATH, beta, 0.0)
        e = ianus.table_ising(dim, ianus.HEATBATH, beta)
        for j in range(2 * dim + 1):
            v = -2 * dim + 2 * j
            assert t[(v + 2 * dim) * 2] == t[(v + 2 * dim) * 2 + 1] == e[j]


@pytest.mark.parametrize("beta", [0.0, 0.7, 1.405, 2.4, 40.0])
def test_potts_count_tables_match_oracle(beta):
    """Permutation model counts n_k in 0..2D (D up to 4) with sum 2D."""
    for D in (2, 3, 4):
        for n0 in range(2 * D + 1):
            for n1 in range(2 * D + 1 - n0):
                for n2 in range(2 * D + 1 - n0 - n1):
                    n = [n0, n1, n2, 2 * D - n0 - n1 - n2]
                    assert ianus.table_potts_counts(beta, n) == oracle.table_potts(beta, n), (D, n)


def test_no_cpu_fallback_without_a_gpu():
    """Without a CUDA device the product path refuses to run: constructing a
    lattice raises instead of computing anywhere else."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        ianus.Lattice(dim=3, L=4, n_samples=1)
