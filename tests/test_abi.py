"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every entry point include/ianus.h declares, validates configurations, and its
host table builders agree bytewise with the oracle's independent builders."""

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
    c.layout, c.disorder, c.seed = kw.get("layout", 0), 0, 1
    return c


def test_required_bytes_validation():
    lib = ianus.lib()
    rb = lambda **kw: lib.ianus_required_bytes(ctypes.byref(_cfg(**kw)))
    assert rb() > 0
    assert rb(L=5) == 0                      # odd side
    assert rb(L=0) == 0
    assert rb(dim=4) == 0
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
