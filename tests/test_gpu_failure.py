"""Failure detection on the GPU without a GPU fault: every device-side wait of
the library is bounded.  Each of its two kinds of wait (the grid barrier of
the cooperative kernels, the mbarrier wait of the tensor-core kernels) is run
where nothing can release it, with a short limit; the kernel must give up,
report RR_ERR_TIMEOUT and leave the context usable."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rr():
    import paper_2505_00281_gb300 as pkg
    from paper_2505_00281_gb300 import build

    build.build()
    pkg.lib()
    return pkg


@pytest.mark.parametrize("mode", [0, 1])
def test_bounded_wait_expires_and_context_survives(rr, mode):
    from paper_2505_00281_gb300._lib import RR
    t0 = time.perf_counter()
    st = rr.api.rr_wait_selftest(mode, 50_000_000)     # 50 ms
    dt = time.perf_counter() - t0
    assert st == RR.ERR_TIMEOUT
    assert 0.04 <= dt < 5.0, dt
    # the context still runs kernels: a Gram product through the library
    x = np.arange(64 * 3, dtype=np.float64).reshape(64, 3)
    X = rr.fortran(torch.from_numpy(x).cuda())
    G = rr.rr_gram(X, X)
    torch.cuda.synchronize()
    assert np.array_equal(G.cpu().numpy(), x.T @ x)
