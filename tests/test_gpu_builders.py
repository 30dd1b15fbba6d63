"""f4: the comparator basis builders of Table 3 on the GPU (MGS-L, MGS-R, CGS,
CGS-2, Hess-L; Hess-R is Algorithm 8) against the FP64 oracle
(oracle/builders.py): FP64 storage to FP64 accuracy, FP32 and FP16 storage
(FP32 arithmetic) within their precision, on U(0,1) blocks as in Table 3."""
import numpy as np
import pytest

from oracle import builders as B
from oracle import ofrr as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rr():
    import paper_2505_00281_gb300 as pkg
    from paper_2505_00281_gb300 import build

    build.build()
    pkg.lib()
    return pkg


def dev(a, dtype=torch.float64):
    import paper_2505_00281_gb300 as pkg
    return pkg.fortran(torch.from_numpy(np.asfortranarray(a)).cuda().to(dtype))


GS = {"mgs_l": B.mgs_left, "mgs_r": B.mgs_right, "cgs": B.cgs, "cgs2": B.cgs2}


@pytest.mark.parametrize("method", ["mgs_l", "mgs_r", "cgs", "cgs2"])
@pytest.mark.parametrize("n,k", [(2500, 40), (777, 33)])
def test_gram_schmidt_fp64(rr, method, n, k):
    W = np.random.default_rng(n + k).uniform(0, 1, (n, k))
    Qo, Ro = GS[method](W)
    Q, R, _ = rr.rr_basis_builder(dev(W), method)
    Q, R = Q.cpu().numpy(), R.cpu().numpy()
    kappa = np.linalg.cond(W)
    assert np.abs(Q - Qo).max() < 1e-13 * kappa * k
    assert np.abs(R - Ro).max() < 1e-13 * kappa * np.abs(Ro).max()
    assert np.abs(Q @ R - W).max() < 1e-13 * np.abs(W).max() * k


@pytest.mark.parametrize("method", ["mgs_l", "mgs_r", "cgs", "cgs2"])
@pytest.mark.parametrize("dtype,u", [(torch.float32, 2.0 ** -24), (torch.float16, 2.0 ** -11)])
def test_gram_schmidt_low_precision(rr, method, dtype, u):
    n, k = 3000, 24
    W = np.random.default_rng(k).uniform(0, 1, (n, k))
    Wd = dev(W, dtype)
    Ws = Wd.double().cpu().numpy()          # the stored (rounded) input
    Qo, Ro = GS[method](Ws)
    Q, R, _ = rr.rr_basis_builder(Wd, method)
    Q, R = Q.double().cpu().numpy(), R.cpu().numpy()
    kappa = np.linalg.cond(Ws)
    tol_q = 64 * u * kappa * (kappa if method == "cgs" else 1.0) * np.sqrt(k)
    assert np.abs(Q - Qo).max() < tol_q, np.abs(Q - Qo).max()
    assert np.abs(Q @ R - Ws).max() < 64 * u * np.abs(Ws).max() * np.sqrt(k)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_hess_left_and_right(rr, dtype):
    """Left- and right-looking Hessenberg processes on the same block: the
    same pivots; the basis equal to the oracle's to the storage precision."""
    n, k = 4000, 50
    W = np.random.default_rng(7).uniform(0, 1, (n, k))
    Qo, pivo = B.hess_left(W)
    QL, _, pL = rr.rr_basis_builder(dev(W, dtype), "hess_l")
    QR, _, pR = rr.rr_basis_builder(dev(W, dtype), "hess_r")
    assert np.array_equal(pL.cpu().numpy(), pivo) and np.array_equal(pR.cpu().numpy(), pivo)
    u = 2.0 ** -53 if dtype == torch.float64 else 2.0 ** -24
    for Q in (QL, QR):
        assert np.abs(Q.double().cpu().numpy() - Qo).max() < 1e4 * u * k


def test_hess_fp16_storage(rr):
    n, k = 3000, 24
    W = np.random.default_rng(9).uniform(0, 1, (n, k))
    Wd = dev(W, torch.float16)
    Ws = Wd.double().cpu().numpy()
    Qo, pivo = B.hess_left(Ws)
    for m in ("hess_l", "hess_r"):
        Q, _, piv = rr.rr_basis_builder(dev(Ws, torch.float16), m)
        assert np.abs(Q.double().cpu().numpy() - Qo).max() < 4 * 2.0 ** -11 * k
        assert np.array_equal(piv.cpu().numpy()[:8], pivo[:8])
