"""rr_gram_noalloc: the Gram product for callers that cannot allocate device
memory (its scratch is a fixed array inside the library).  Checked through
the C ABI against rr_gram, the workspace-taking entry point, on two calls in
a row: the second call reuses the array the first one left behind.

Kept in a file collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U53 = 2.0 ** -53


@pytest.fixture(scope="module")
def rr():
    import paper_2505_00281_gb300 as pkg
    from paper_2505_00281_gb300 import build

    build.build()
    pkg.lib()
    return pkg


def _dev(rr, a, dtype=None):
    t = torch.from_numpy(np.asfortranarray(a)).cuda()
    if dtype is not None:
        t = t.to(dtype)
    return rr.fortran(t)


def test_gram_noalloc_matches_gram_twice(rr):
    from oracle import ofrr as O

    for call, (n, p, q, seed) in enumerate([(20000, 128, 128, 1), (7001, 37, 50, 2)]):
        rng = np.random.default_rng(seed)
        X = O.round_bf16(rng.standard_normal((n, p)))
        Y = rng.standard_normal((n, q))
        Xd, Yd = _dev(rr, X, torch.bfloat16), _dev(rr, Y)
        G_ws = rr.rr_gram(Xd, Yd)                 # workspace-taking entry point
        G_na = rr.rr_gram_noalloc(Xd, Yd)         # fixed in-library scratch
        torch.cuda.synchronize()
        a, b = G_ws.cpu().numpy(), G_na.cpu().numpy()
        bound = 2 * n * U53 * (np.abs(X).T @ np.abs(Y))
        assert np.all(np.abs(a - b) <= 2 * bound), call
        assert np.all(np.abs(b - X.T @ Y) <= 2 * bound), call


def test_gram_noalloc_largest_size_and_accumulate(rr):
    """The largest accepted product (p q = 262144: the whole array holds one
    chunk, so the partial kernel covers all n rows at once) and the
    accumulating form (G += X^T Y on a nonzero G), both against rr_gram."""
    rng = np.random.default_rng(3)
    n, p, q = 3000, 512, 512
    X, Y = rng.standard_normal((n, p)), rng.standard_normal((n, q))
    Xd, Yd = _dev(rr, X), _dev(rr, Y)
    G_ws = rr.rr_gram(Xd, Yd)
    G_na = rr.rr_gram_noalloc(Xd, Yd)
    torch.cuda.synchronize()
    bound = 2 * n * U53 * (np.abs(X).T @ np.abs(Y))
    assert np.all(np.abs(G_ws.cpu().numpy() - G_na.cpu().numpy()) <= 2 * bound)
    n, p, q = 5000, 40, 24
    X, Y = rng.standard_normal((n, p)), rng.standard_normal((n, q))
    G0 = rng.standard_normal((p, q))
    Xd, Yd = _dev(rr, X), _dev(rr, Y)
    Ga, Gb = _dev(rr, G0), _dev(rr, G0)
    rr.rr_gram(Xd, Yd, G=Ga, accumulate=True)
    rr.rr_gram_noalloc(Xd, Yd, G=Gb, accumulate=True)
    torch.cuda.synchronize()
    bound = 2 * n * U53 * (np.abs(X).T @ np.abs(Y)) + 2 * U53 * np.abs(G0)
    assert np.all(np.abs(Ga.cpu().numpy() - Gb.cpu().numpy()) <= 2 * bound)
    assert np.all(np.abs(Gb.cpu().numpy() - (G0 + X.T @ Y)) <= 2 * bound)


def test_gram_noalloc_rejects_sizes_beyond_its_scratch(rr):
    from paper_2505_00281_gb300._lib import RR, RrError

    with pytest.raises(RrError) as e:
        rr.rr_gram_noalloc(rr.fortran(torch.zeros(16, 600, dtype=torch.float64, device="cuda")),
                           rr.fortran(torch.zeros(16, 600, dtype=torch.float64, device="cuda")))
    assert e.value.status == RR.ERR_ARG
