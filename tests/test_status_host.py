"""Host-side argument and workspace checks of the solver entry points, and
the C struct layout the Python binding marshals (no GPU: every call here
returns before anything reaches the device)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")
# the fake device pointers below must never reach a real device
pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="host-only checks (fake pointers)")

FAKE = 0x1000  # never dereferenced: the checks under test return first


@pytest.fixture(scope="module")
def L():
    from paper_2505_00281_gb300 import build, _lib
    build.build()
    return _lib.lib()


def _op(m, n):
    from paper_2505_00281_gb300._lib import RR, RrOperator
    return RrOperator(RR.DENSE, RR.F64, m, n, m, 0, FAKE, None, None)


def _params(k=8, block=16):
    from paper_2505_00281_gb300._lib import RrParams
    p = RrParams()
    p.k, p.block, p.degree, p.max_sweeps, p.basis, p.refine, p.tol = k, block, 2, 10, 2, 1, 1e-10
    p.v0 = FAKE
    return p


def _svd(L, op, p, ws, wsb):
    from paper_2505_00281_gb300._lib import RrInfo
    info = RrInfo()
    return L.rr_svd(ctypes.byref(op), ctypes.byref(p), FAKE, FAKE, FAKE, ws, wsb, ctypes.byref(info), None)


def test_solver_argument_errors(L):
    from paper_2505_00281_gb300._lib import RR, RrInfo
    op = _op(1000, 200)
    assert _svd(L, op, _params(k=20, block=16), FAKE, 1 << 40) == RR.ERR_ARG        # k > block
    assert _svd(L, _op(100, 200), _params(), FAKE, 1 << 40) == RR.ERR_ARG           # m < n
    assert _svd(L, op, _params(k=0), FAKE, 1 << 40) == RR.ERR_ARG                    # k < 1
    p = _params()
    p.basis = 9
    assert _svd(L, op, p, FAKE, 1 << 40) == RR.ERR_ARG                               # unknown dtype
    p = _params(k=8, block=200)
    assert _svd(L, op, p, FAKE, 1 << 40) == RR.ERR_ARG                               # 2b pencil > 335
    info = RrInfo()
    # a non-square dense operator for the symmetric eigensolver
    assert L.rr_eig(ctypes.byref(op), ctypes.byref(_params()), FAKE, FAKE, FAKE, 1 << 40,
                    ctypes.byref(info), None) == RR.ERR_ARG


def test_solver_workspace_errors(L):
    from paper_2505_00281_gb300._lib import RR
    op, p = _op(1000, 200), _params()
    need = L.rr_workspace_size(ctypes.byref(op), ctypes.byref(p), 1)
    assert need > 0
    assert _svd(L, op, p, FAKE, need - 1) == RR.ERR_WORKSPACE                        # too small
    assert _svd(L, op, p, None, need) == RR.ERR_WORKSPACE                            # missing
    assert _svd(L, op, p, FAKE + 8, need) == RR.ERR_WORKSPACE                        # not 256-aligned
    # a start block drawn from the seed needs room for it
    p.v0 = None
    assert L.rr_workspace_size(ctypes.byref(op), ctypes.byref(p), 1) == need + 200 * 16 * 8


def test_gram_noalloc_rejects_bad_dtype_even_when_empty(L):
    from paper_2505_00281_gb300._lib import RR
    for n, p, q in [(0, 1, 1), (10, 0, 4), (10, 4, 0)]:
        assert L.rr_gram_noalloc(n, p, q, 9, FAKE, max(n, 1), 0, FAKE, max(n, 1), FAKE, max(p, 1), 0, None) == RR.ERR_ARG
        assert L.rr_gram(n, p, q, 0, FAKE, max(n, 1), 9, FAKE, max(n, 1), FAKE, max(p, 1), 0, FAKE, 256, None) == RR.ERR_ARG
    assert L.rr_wait_selftest(2, 1000, FAKE, None) == RR.ERR_ARG
    assert L.rr_wait_selftest(0, 0, FAKE, None) == RR.ERR_ARG


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_struct_layout_matches_header(tmp_path):
    """sizeof and field offsets of rr_operator, rr_params, rr_info and
    rr_batch_tuning as the C compiler lays them out from include/rr.h, against
    the ctypes structures."""
    from paper_2505_00281_gb300 import _lib
    classes = (("rr_params", _lib.RrParams), ("rr_info", _lib.RrInfo), ("rr_operator", _lib.RrOperator),
               ("rr_batch_tuning", _lib.RrBatchTuning))
    fields = {t: [f for f, _ in cls._fields_] for t, cls in classes}
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "rr.h"', 'int main(void) {']
    for t, fs in fields.items():
        src.append(f'printf("{t} %zu\\n", sizeof({t}));')
        for f in fs:
            src.append(f'printf("{t}.{f} %zu\\n", offsetof({t}, {f}));')
    src.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for t, cls in classes:
        assert int(got[t]) == ctypes.sizeof(cls), t
        for f in fields[t]:
            assert int(got[f"{t}.{f}"]) == getattr(cls, f).offset, (t, f)


def test_batch_tuning_argument_errors(L):
    """rr_batch_svd_tuned rejects launch parameters out of range (branches
    outside 1..64, order or fixed_sweeps other than 0 / 1) before anything
    reaches the device."""
    from paper_2505_00281_gb300._lib import RR, RrBatchTuning, RrInfo
    op = (type(_op(256, 64)) * 1)(_op(256, 64))
    p = _params(k=8, block=16)
    ptrs = (ctypes.c_void_p * 1)(FAKE)
    per = (ctypes.c_int32 * 1)()
    infos = (RrInfo * 1)()
    for t in (RrBatchTuning(0, 0, 0, 0), RrBatchTuning(65, 0, 0, 0), RrBatchTuning(16, -1, 0, 0),
              RrBatchTuning(16, 0, 2, 0), RrBatchTuning(16, 0, 0, 2)):
        assert L.rr_batch_svd_tuned(1, op, ctypes.byref(p), 7, ptrs, ptrs, ptrs, FAKE, 1 << 40, ctypes.byref(t),
                                    per, infos, None) == RR.ERR_ARG, (t.branches, t.max_splits, t.order,
                                                                      t.fixed_sweeps)
