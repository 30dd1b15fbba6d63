"""The C-ABI library builds, loads and exports every entry point include/rr.h declares (CPU only)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rr_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2505_00281_gb300 import build, _lib

    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(rr_[a-z0-9_]+)", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    # the Python binding declares the same names
    assert sorted(_lib.EXPORTED) == declared
    L = _lib.lib()
    for d in declared:
        assert hasattr(L, d)


def test_workspace_queries_run_without_gpu():
    """Size queries do not touch the device."""
    import ctypes

    from paper_2505_00281_gb300 import _lib

    L = _lib.lib()
    assert L.rr_gram_workspace_size(10000, 64, 64) > 0
    assert L.rr_pencil_workspace_size(64, 64) > 64 * 64 * 8
    op = _lib.RrOperator(0, 0, 1000, 200, 1000, 0, 1, None, None)
    p = _lib.RrParams()
    p.k, p.block, p.degree, p.max_sweeps, p.basis, p.refine = 8, 16, 2, 10, 2, 1
    assert L.rr_workspace_size(ctypes.byref(op), ctypes.byref(p), 1) > 0
    bad = _lib.RrOperator(0, 0, 100, 200, 100, 0, 1, None, None)   # m < n for the SVD
    assert L.rr_workspace_size(ctypes.byref(bad), ctypes.byref(p), 1) == 0


def test_autotune_table_host_logic(tmp_path):
    """Size classes and the persisted table (host only)."""
    from paper_2505_00281_gb300 import autotune as AT
    assert AT.size_class(512, 128) == "9,7,bf16" and AT.size_class(1023, 255) == "9,7,bf16"
    assert AT.size_class(1024, 256) == "10,8,bf16"
    t = {"9,7,bf16": {"branches": 8, "max_splits": 1, "order": 1, "ms": 1.0, "default_ms": 2.0}}
    AT.save(t, tmp_path / "t.json")
    assert AT.load(tmp_path / "t.json") == t
    assert all(1 <= c["branches"] <= 64 and c["max_splits"] >= 0 and c["order"] in (0, 1) for c in AT.CANDIDATES)


def test_shipped_tuning_table():
    from paper_2505_00281_gb300 import autotune as AT
    t = AT.load()
    assert t and all(set(v) >= {"branches", "max_splits", "order"} for v in t.values())


def test_autotune_batch_grouping_and_order(monkeypatch):
    """batch_svd splits a batch by size class, runs each class with its tuned
    parameters (defaults for classes the table lacks) and returns the results in
    the caller's order (host logic, the batch call faked)."""
    from types import SimpleNamespace

    from paper_2505_00281_gb300 import autotune as AT
    calls = []

    def fake(ops, params, seed, tuning=None, **kw):
        calls.append(([o.m for o in ops], dict(tuning), seed))
        return [("out", o.m) for o in ops], [0] * len(ops), [{"m": o.m} for o in ops]
    monkeypatch.setattr(AT.api, "rr_batch_svd", fake)
    ops = [SimpleNamespace(m=m, n=m // 4) for m in (300, 1100, 310, 2100, 1200)]
    table = {AT.size_class(300, 75): {"branches": 8, "max_splits": 1, "order": 1, "ms": 1.0, "default_ms": 2.0}}
    outs, st, infos = AT.batch_svd(ops, None, 100, table)
    assert [o[1] for o in outs] == [300, 1100, 310, 2100, 1200] and [i["m"] for i in infos] == [300, 1100, 310, 2100, 1200]
    by_sizes = {tuple(c[0]): c[1] for c in calls}
    assert by_sizes[(300, 310)] == {"branches": 8, "max_splits": 1, "order": 1}
    assert by_sizes[(1100, 1200)] == AT.DEFAULT and by_sizes[(2100,)] == AT.DEFAULT
    assert all(x == 0 for x in st)
