"""End-to-end parity of the solvers (rr_eig, rr_svd, rr_batch_svd) with the
FP64 oracle: converged values against the closed-form spectra and the
oracle's own solve, residuals recomputed by the oracle in FP64 from the GPU's
vectors, and the theorem's orthonormality."""
import numpy as np
import pytest

import workloads as wl
from oracle import ofrr as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def rr():
    import paper_2505_00281_gb300 as pkg
    from paper_2505_00281_gb300 import build

    build.build()
    pkg.lib()
    return pkg


def dev(a):
    import paper_2505_00281_gb300 as pkg
    return pkg.fortran(torch.from_numpy(np.asfortranarray(a)).to(DEV))


def host(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("basis", ["f32", "bf16", "f64"])
def test_eig_dense_config1_shape(rr, basis):
    """Dense symmetric lambda_i = 1/i (config 1 recipe, n reduced), top 8, block 16."""
    n, k, b = 600, 8, 16
    A, lam = wl.config1(n)
    V0 = wl.uniform_block(n, b, 1001)
    refine = basis != "f64"
    p = rr.api.make_params(k, b, 2, 60, 1e-10, basis=basis, v0=dev(V0), refine=refine, phase1_sweeps=2)
    th, X, info = rr.rr_eig(rr.api.dense_operator(dev(A)), p, n)
    th, X = host(th), host(X)
    assert info["n_converged"] == k, info
    assert np.max(np.abs(th - lam[:k]) / lam[:k]) <= 1e-10
    res = O.residual_eig(O.dense_apply(A)[0], X, th)
    assert res.max() <= 1.5e-10, res
    assert np.abs(X.T @ X - np.eye(k)).max() < 1e-10


def test_eig_fixed_sweeps_trajectory_config1(rr):
    """Fixed work (6 sweeps, no refinement, FP32 basis) against the oracle's
    FP64 trajectory.  The GPU's plain phase projects with the FP32 copy of A
    (Sec. 4.2: working precision = input precision of the products), so its
    Ritz values carry the operator rounding u32 |A|_2 on top of the
    first-order basis term: |dtheta| <= 1e-10 |theta| + 2 u32 |A| + 10 u32 |A| r_oracle."""
    n, k, b = 2000, 8, 16
    A, lam = wl.config1(n)
    V0 = wl.uniform_block(n, b, 1001)
    p = rr.api.make_params(k, b, 1, 6, 1e-30, basis="f32", v0=dev(V0), refine=False)
    th, X, info = rr.rr_eig(rr.api.dense_operator(dev(A)), p, n)
    ora = O.solve_eig(O.dense_apply(A)[0], n, k, V0, degree=1, max_sweeps=6, tol=1e-30)
    assert info["sweeps"] == 6 and ora.sweeps == 6
    th = host(th)
    u32, normA = 2.0 ** -24, 1.0
    bound = 1e-10 * np.abs(ora.values) + 2 * u32 * normA + 10 * u32 * normA * ora.res
    assert np.all(np.abs(th - ora.values) <= bound), (th - ora.values, bound)


def test_svd_dense_bf16_refined(rr):
    """Dense SVD sigma_i = exp(-i/60) (config 2 recipe, reduced), BF16 basis + refinement."""
    m, n, b, k = 2048, 512, 32, 16
    sig = wl.config2_sigma(n)
    A = wl.dense_svd(m, n, sig, 2000)
    V0 = wl.uniform_block(n, b, 2001)
    p = rr.api.make_params(k, b, 4, 30, 1e-10, basis="bf16", v0=dev(V0), refine=True, phase1_sweeps=1)
    s, U, V, info = rr.rr_svd(rr.api.dense_operator(dev(A)), p)
    s, U, V = host(s), host(U), host(V)
    assert info["n_converged"] == k, info
    assert np.max(np.abs(s - sig[:k]) / sig[:k]) <= 1e-10
    Amul, Atmul = O.dense_apply(A)
    assert O.residual_svd(Amul, Atmul, U, V, s).max() <= 1.5e-10
    assert np.abs(U.T @ U - np.eye(k)).max() < 1e-10
    assert np.abs(V.T @ V - np.eye(k)).max() < 1e-10
    ref = O.solve_svd(Amul, Atmul, m, n, k, V0, degree=4, max_sweeps=30, tol=1e-10)
    assert np.max(np.abs(s - ref.values) / ref.values) <= 1e-10
    # singular vectors agree with the oracle's up to the sign convention
    for j in range(k):
        assert min(np.abs(V[:, j] - ref.X[:, j]).max(), np.abs(V[:, j] + ref.X[:, j]).max()) < 1e-8


def test_svd_dense_e4m3_refined(rr):
    """The same SVD with an FP8-E4M3 phase-1 basis (operator and basis in E4M3,
    tcgen05 kind::f8f6f4 products), refined to 1e-10 on BF16 correction blocks."""
    m, n, b, k = 2048, 512, 32, 16
    sig = wl.config2_sigma(n)
    A = wl.dense_svd(m, n, sig, 2000)
    V0 = wl.uniform_block(n, b, 2001)
    p = rr.api.make_params(k, b, 4, 30, 1e-10, basis="e4m3", v0=dev(V0), refine=True, phase1_sweeps=1)
    s, U, V, info = rr.rr_svd(rr.api.dense_operator(dev(A)), p)
    s, U, V = host(s), host(U), host(V)
    assert info["n_converged"] == k, info
    assert np.max(np.abs(s - sig[:k]) / sig[:k]) <= 1e-10
    Amul, Atmul = O.dense_apply(A)
    assert O.residual_svd(Amul, Atmul, U, V, s).max() <= 1.5e-10
    assert np.abs(U.T @ U - np.eye(k)).max() < 1e-10
    assert np.abs(V.T @ V - np.eye(k)).max() < 1e-10


def test_svd_dense_fp64_plain_method(rr):
    m, n, b, k = 800, 200, 24, 8
    sig = wl.config2_sigma(n)
    A = wl.dense_svd(m, n, sig, 2100)
    V0 = wl.uniform_block(n, b, 2101)
    p = rr.api.make_params(k, b, 2, 40, 1e-10, basis="f64", v0=dev(V0), refine=False)
    s, U, V, info = rr.rr_svd(rr.api.dense_operator(dev(A)), p)
    assert info["n_converged"] == k, info
    assert np.max(np.abs(host(s) - sig[:k]) / sig[:k]) <= 1e-10


def test_eig_csr_chebyshev_lowest_constant_potential(rr):
    """Chebyshev-filtered, lowest pairs of -Lap + c on a grid: closed form."""
    N, k, b = 32, 12, 20
    rp, ci, va = wl.grid_potential_csr(N, np.full(N * N, 0.5))
    n = N * N
    V0 = wl.uniform_block(n, b, 3001)
    d = [torch.from_numpy(a).to(DEV) for a in (rp, ci, va)]
    op = rr.api.csr_operator(*d)
    p = rr.api.make_params(k, b, 10, 60, 1e-10, basis="bf16", v0=dev(V0), filter=rr.RR.CHEBYSHEV,
                           which=rr.RR.SMALLEST, refine=True, phase1_sweeps=4)
    th, X, info = rr.rr_eig(op, p, n)
    exact = wl.laplacian_constant_eigs(N, 0.5)[:k]
    th = host(th)
    assert info["n_converged"] == k, info
    assert np.max(np.abs(th - exact) / exact) <= 1e-9
    res = O.residual_eig(O.csr_apply(rp, ci, va), host(X), th)
    assert res.max() <= 1.5e-10


def test_eig_csr_random_potential_vs_oracle(rr):
    N, k, b = 24, 10, 16
    rp, ci, va, v = wl.grid_schrodinger_csr(N, 10.0, 3000)
    n = N * N
    V0 = wl.uniform_block(n, b, 3002)
    d = [torch.from_numpy(a).to(DEV) for a in (rp, ci, va)]
    p = rr.api.make_params(k, b, 8, 80, 1e-10, basis="bf16", v0=dev(V0), filter=rr.RR.CHEBYSHEV,
                           which=rr.RR.SMALLEST, refine=True, phase1_sweeps=4)
    th, X, info = rr.rr_eig(rr.api.csr_operator(*d), p, n)
    Amul = O.csr_apply(rp, ci, va)
    dense = Amul(np.eye(n))
    exact = np.linalg.eigvalsh(dense)[:k]          # brute force
    assert info["n_converged"] == k, info
    assert np.max(np.abs(host(th) - exact) / np.abs(exact)) <= 1e-9


def test_batch_svd_small(rr):
    shapes = [(256, 64), (400, 100), (300, 75), (512, 128), (260, 65)]
    ops, As, sigs = [], [], []
    for i, (m, n) in enumerate(shapes):
        sg = wl.config4_sigma(n)
        A = wl.dense_svd(m, n, sg, 4000 + i)
        t = dev(A)
        As.append((A, t))
        sigs.append(sg)
        ops.append(rr.api.dense_operator(t))
    p = rr.api.make_params(8, 16, 2, 12, 1e-10, basis="bf16", refine=True, phase1_sweeps=2)
    outs, st, infos = rr.rr_batch_svd(ops, p, seed=4000)
    for i, ((s, U, V), (A, _)) in enumerate(zip(outs, As)):
        s = host(s)
        assert np.max(np.abs(s - sigs[i][:8]) / sigs[i][:8]) <= 1e-10, (i, s, sigs[i][:8], infos[i])
        Amul, Atmul = O.dense_apply(A)
        assert O.residual_svd(Amul, Atmul, host(U), host(V), s).max() <= 1.5e-10


def test_batch_autotune_and_tuned_launches(rr):
    """Every launch-parameter choice of the batched SVD gives the converged
    result (sigma to the closed form), and the autotuner's table drives a
    per-class run of a mixed batch."""
    from paper_2505_00281_gb300 import autotune as AT
    shapes = [(256, 64), (300, 75), (512, 128), (520, 130), (1024, 256), (1040, 260)]
    ops, sigs, keep = [], [], []
    for i, (m, n) in enumerate(shapes):
        sg = wl.config4_sigma(n)
        A = dev(wl.dense_svd(m, n, sg, 4100 + i))
        keep.append(A)
        ops.append(rr.api.dense_operator(A))
        sigs.append(sg)
    p = rr.api.make_params(8, 16, 4, 12, 1e-10, basis="bf16", refine=True, phase1_sweeps=1)
    for tuning in ({"branches": 1, "max_splits": 1, "order": 0}, {"branches": 4, "max_splits": 0, "order": 1},
                   {"branches": 64, "max_splits": 2, "order": 1}):
        outs, st, _ = rr.rr_batch_svd(ops, p, 5, tuning=tuning)
        assert all(x == 0 for x in st), (tuning, st)
        for (s, U, V), sg in zip(outs, sigs):
            assert np.max(np.abs(host(s) - sg[:8]) / sg[:8]) <= 1e-10
    samples = {}
    for op in ops:
        samples.setdefault(AT.size_class(op.m, op.n), []).append(op)
    table = AT.tune(samples, p, candidates=[{"branches": 2, "max_splits": 1, "order": 0},
                                            {"branches": 8, "max_splits": 0, "order": 1}], reps=1)
    assert set(table) == set(samples)
    outs, st, infos = AT.batch_svd(ops, p, 5, table)
    assert all(x == 0 for x in st)
    for (s, U, V), sg in zip(outs, sigs):
        assert np.max(np.abs(host(s) - sg[:8]) / sg[:8]) <= 1e-10


def test_batch_problems_keep_converged_triplets(rr):
    """Batched problems iterate for a fixed sweep count: easy problems converge
    within a few sweeps and then run 30 more; their converged triplets must be
    what comes out (no degenerate post-convergence sweep reaches the result)."""
    shapes = [(256, 64), (264, 66), (320, 80), (256, 64)]
    ops, sigs, keep = [], [], []
    for i, (m, n) in enumerate(shapes):
        sg = np.exp(-np.arange(1, n + 1) / 4.0)          # wide gaps: converges in a few sweeps
        A = dev(wl.dense_svd(m, n, sg, 4200 + i))
        keep.append(A)
        ops.append(rr.api.dense_operator(A))
        sigs.append(sg)
    p = rr.api.make_params(4, 8, 2, 36, 1e-10, basis="bf16", refine=True, phase1_sweeps=1)
    outs, st, infos = rr.rr_batch_svd(ops, p, 9)
    assert all(x == 0 for x in st), (st, infos)
    for (s, U, V), sg, A in zip(outs, sigs, keep):
        assert np.max(np.abs(host(s) - sg[:4]) / sg[:4]) <= 1e-10
        Ah = host(A)
        Amul, Atmul = O.dense_apply(Ah)
        assert O.residual_svd(Amul, Atmul, host(U), host(V), host(s)).max() <= 1.5e-10


@pytest.mark.parametrize("basis,refine", [("bf16", True), ("f64", False)])
def test_batch_device_loop_stops_at_tol(rr, basis, refine):
    """Device-side loop control of the batched solver: a problem's sweeps after
    the first run inside WHILE graph nodes whose condition a kernel sets after
    each residual check, so each problem stops on the GPU once its k wanted
    residuals reach tol.  Easy problems (wide gaps) stop after a few of the 36
    allowed sweeps and a harder one (sigma_j = j^-1.5) in the same batch runs
    longer; the triplets match the closed form, as do those of the schedule
    that runs every problem for all 36 sweeps (fixed_sweeps)."""
    shapes = [(256, 64), (264, 66), (320, 80), (1024, 256)]
    ops, sigs, keep = [], [], []
    for i, (m, n) in enumerate(shapes):
        sg = np.exp(-np.arange(1, n + 1) / 4.0) if i < 3 else wl.config4_sigma(n)
        A = wl.dense_svd(m, n, sg, 4300 + i)
        keep.append((A, dev(A)))
        ops.append(rr.api.dense_operator(keep[-1][1]))
        sigs.append(sg)
    p = rr.api.make_params(4, 8, 2, 36, 1e-10, basis=basis, refine=refine, phase1_sweeps=1)
    outs, st, infos = rr.rr_batch_svd(ops, p, 9)
    fixed = {"branches": 16, "max_splits": 0, "order": 0, "fixed_sweeps": 1}
    outs_f, st_f, infos_f = rr.rr_batch_svd(ops, p, 9, tuning=fixed)
    assert all(x == 0 for x in st) and all(x == 0 for x in st_f), (st, st_f, infos)
    sweeps = [inf["sweeps"] for inf in infos]
    assert all(inf["sweeps"] == 36 for inf in infos_f)
    assert max(sweeps[:3]) <= 12 and min(sweeps) >= 1, sweeps
    assert sweeps[3] >= min(sweeps[:3]), sweeps
    for o in (outs, outs_f):
        for (s, U, V), sg, (A, _) in zip(o, sigs, keep):
            s = host(s)
            assert np.max(np.abs(s - sg[:4]) / sg[:4]) <= 1e-10
            Amul, Atmul = O.dense_apply(A)
            assert O.residual_svd(Amul, Atmul, host(U), host(V), s).max() <= 1.5e-10


def test_batch_svd_several_graphs(rr):
    """A batch larger than one captured graph (graphs of 16 problems, launched
    in order while the host captures the next): 40 problems of the batched
    workload's smallest class in three graphs, every one converged to the
    closed form, its sweep count within max_sweeps."""
    sh = [(m, n) for m, n in wl.config4_shapes(512) if m < 512][:40]
    ops, keep, sigs = [], [], []
    for i, (m, n) in enumerate(sh):
        sg = wl.config4_sigma(n)
        A = wl.dense_svd(m, n, sg, 4400 + i)
        keep.append((A, dev(A)))
        ops.append(rr.api.dense_operator(keep[-1][1]))
        sigs.append(sg)
    p = rr.api.make_params(16, 32, 4, 12, 1e-10, basis="bf16", refine=True, phase1_sweeps=1)
    outs, st, infos = rr.rr_batch_svd(ops, p, seed=4400)
    assert all(x == 0 for x in st), [(i, inf) for i, (x, inf) in enumerate(zip(st, infos)) if x]
    assert all(1 <= inf["sweeps"] <= 12 for inf in infos)
    for (s, U, V), sg, (A, _) in zip(outs, sigs, keep):
        s = host(s)
        assert np.max(np.abs(s - sg[:16]) / sg[:16]) <= 1e-10
        Amul, Atmul = O.dense_apply(A)
        assert O.residual_svd(Amul, Atmul, host(U), host(V), s).max() <= 1.5e-10


def test_svd_seeded_start_block_and_info(rr):
    """v0 = NULL draws the start block on the device from params.seed (Alg. 1's
    U(0,1) block) and the solve converges from it.  Runs are not reproducible
    bit for bit (split-K products add FP32 partial tiles with atomics, and the
    BF16 basis amplifies the different roundings), so the same seed gives the
    same triplets and a first-projection residual within a few per cent.
    rr_info's Gram condition estimate is at least 1 (G_ii (G^-1)_ii >= 1 for
    any SPD G) and finite."""
    m, n, b, k = 2048, 512, 32, 16
    sig = wl.config2_sigma(n)
    Ad = dev(wl.dense_svd(m, n, sig, 2000))
    outs = []
    for seed in (7, 7, 8):
        p = rr.api.make_params(k, b, 4, 30, 1e-10, basis="bf16", v0=None, refine=True, phase1_sweeps=1,
                               seed=seed)
        s, U, V, info = rr.rr_svd(rr.api.dense_operator(Ad), p)
        assert info["n_converged"] == k, info
        assert np.max(np.abs(host(s) - sig[:k]) / sig[:k]) <= 1e-10
        assert len(info["cond_history"]) == info["sweeps"]
        assert all(1.0 <= c < 1e16 for c in info["cond_history"]), info["cond_history"]
        assert info["cond_G_est"] == info["cond_history"][-1]
        outs.append((host(s), info["res_history"]))
    assert np.max(np.abs(outs[0][0] - outs[1][0]) / sig[:k]) < 1e-13
    assert abs(outs[0][1][0] / outs[1][1][0] - 1) < 0.05


def test_svd_nan_operator_reports_nan(rr):
    """A NaN in the operator makes every residual NaN: the solver stops with
    RR_ERR_NAN instead of running to max_sweeps."""
    from paper_2505_00281_gb300._lib import RR, RrError
    m, n, b, k = 512, 128, 16, 4
    A = wl.dense_svd(m, n, wl.config2_sigma(n), 2200)
    A[17, 3] = np.nan
    for basis, refine in (("bf16", True), ("f64", False)):
        p = rr.api.make_params(k, b, 2, 10, 1e-10, basis=basis, v0=dev(wl.uniform_block(n, b, 2201)),
                               refine=refine)
        with pytest.raises(RrError) as e:
            rr.rr_svd(rr.api.dense_operator(dev(A)), p)
        assert e.value.status == RR.ERR_NAN


def test_eig_hess_tol_is_used(rr):
    """params.hess_tol reaches Algorithm 8: the default value given explicitly
    changes nothing (to rounding: small FP64 products sum with atomics); a
    skip tolerance of 0.9 (a column is skipped unless elimination left its
    pivot within 10 % of its entry inf-norm) drops columns."""
    n, k, b = 600, 8, 16
    A, lam = wl.config1(n)
    Ad, V0 = dev(A), dev(wl.uniform_block(n, b, 1001))
    runs = []
    for tol in (0.0, 4 * b * 2.0 ** -23, 0.9):
        p = rr.api.make_params(k, b, 2, 8, 1e-30, basis="f32", v0=V0, refine=False, hess_tol=tol)
        th, X, info = rr.rr_eig(rr.api.dense_operator(Ad), p, n)
        runs.append((host(th), info["res_history"], info["cols_dropped"]))
    assert np.max(np.abs(runs[0][0] - runs[1][0]) / lam[:k]) < 1e-12
    assert all(abs(a / b - 1) < 1e-6 for a, b in zip(runs[0][1][:3], runs[1][1][:3]))
    assert runs[0][2] == 0 and runs[2][2] > 0, (runs[0][2], runs[2][2])


def _c4_ragged(count):
    """Problems of the batched workload (m_i = 4 round(64 16^u_i), n_i = m_i/4,
    sigma_j = j^-1.5, seed 4000 + i) from its largest class with m or n not a
    multiple of 8: the shapes that lost the split-BF16 and emulated-FP64 paths
    before operators were zero-padded."""
    sh = wl.config4_shapes(512)
    return [(i, m, n) for i, (m, n) in enumerate(sh) if m >= 2048 and (m % 8 or n % 8)][:count]


def test_svd_ragged_shape_single(rr):
    """One such problem through rr_svd (3172 x 793, zero-padded to 3176 x 800
    inside the library): all 16 triplets to 1e-10, the outputs of A's own
    size."""
    i, m, n = _c4_ragged(1)[0]
    sg = wl.config4_sigma(n)
    A = wl.dense_svd(m, n, sg, 4000 + i)
    p = rr.api.make_params(16, 32, 4, 30, 1e-10, basis="bf16", v0=dev(wl.uniform_block(n, 32, 4500 + i)),
                           refine=True, phase1_sweeps=1)
    s, U, V, info = rr.rr_svd(rr.api.dense_operator(dev(A)), p)
    assert info["n_converged"] == 16, info
    s, U, V = host(s), host(U), host(V)
    assert U.shape == (m, 16) and V.shape == (n, 16)
    assert np.max(np.abs(s - sg[:16]) / sg[:16]) <= 1e-10
    Amul, Atmul = O.dense_apply(A)
    assert O.residual_svd(Amul, Atmul, U, V, s).max() <= 1.5e-10


def test_batch_svd_ragged_largest_class(rr):
    """Eight problems of the batched workload's 2048-4095-row class with m or
    n not a multiple of 8 (the class where most problems used to stall at
    residual 3e-10), batched at the workload's settings (top 16, block 32,
    4 products per sweep, 30 sweeps): every problem converges to 1e-10."""
    probs = _c4_ragged(8)
    ops, keep = [], []
    for i, m, n in probs:
        A = wl.dense_svd(m, n, wl.config4_sigma(n), 4000 + i)
        t = dev(A)
        keep.append((A, t))
        ops.append(rr.api.dense_operator(t))
    p = rr.api.make_params(16, 32, 4, 30, 1e-10, basis="bf16", refine=True, phase1_sweeps=1)
    outs, st, infos = rr.rr_batch_svd(ops, p, seed=4000)
    for (i, m, n), (s, U, V), (A, _), x, inf in zip(probs, outs, keep, st, infos):
        sg = wl.config4_sigma(n)
        s = host(s)
        assert x == 0, ((m, n), inf)
        assert np.max(np.abs(s - sg[:16]) / sg[:16]) <= 1e-10, (m, n)
        Amul, Atmul = O.dense_apply(A)
        assert O.residual_svd(Amul, Atmul, host(U), host(V), s).max() <= 1.5e-10, (m, n)


def test_svd_fp64_polish_after_stall(rr):
    """Asked for a tolerance below what the low-precision corrections reach
    (1e-14; on sigma_j = j^-1.5 with 16 of 32 wanted they stop near 1e-13),
    the solver switches to FP64 polish sweeps once the residual stops
    contracting (largest wanted residual above 0.3 times the previous one).
    The polish sweeps (the correction sweep in FP64-accurate arithmetic) keep
    every triplet at the FP64 level: residual below 1e-12 by the oracle,
    sigma to 1e-13.  Single solves (host stall rule) and the batched solver
    (device-side stall rule inside its WHILE graph nodes) alike."""
    sh = wl.config4_shapes(512)
    probs = [(i, m, n) for i, (m, n) in enumerate(sh) if m >= 2048][:4]
    mats = [(m, n, wl.config4_sigma(n), wl.dense_svd(m, n, wl.config4_sigma(n), 4000 + i)) for i, m, n in probs]

    def check(s, U, V, sg, A):
        s = host(s)
        assert np.max(np.abs(s - sg[:16]) / sg[:16]) <= 1e-13
        Amul, Atmul = O.dense_apply(A)
        assert O.residual_svd(Amul, Atmul, host(U), host(V), s).max() <= 1e-12

    for (i, _, _), (m, n, sg, A) in zip(probs, mats):
        p = rr.api.make_params(16, 32, 4, 10, 1e-14, basis="bf16", v0=dev(wl.uniform_block(n, 32, 4600 + i)),
                               refine=True, phase1_sweeps=1)
        s, U, V, info = rr.rr_svd(rr.api.dense_operator(dev(A)), p)
        assert info["polish_sweeps"] >= 1 and info["sweeps"] == 10, ((m, n), info["res_history"])
        check(s, U, V, sg, A)
    keep = [dev(A) for _, _, _, A in mats]
    p = rr.api.make_params(16, 32, 4, 10, 1e-14, basis="bf16", refine=True, phase1_sweeps=1)
    outs, st, infos = rr.rr_batch_svd([rr.api.dense_operator(t) for t in keep], p, seed=4000)
    for (s, U, V), (m, n, sg, A), inf in zip(outs, mats, infos):
        assert inf["polish_sweeps"] >= 1 and inf["sweeps"] == 10, ((m, n), inf)
        check(s, U, V, sg, A)


@pytest.mark.parametrize("k,b", [(40, 96), (64, 160)])
def test_eig_csr_tall_block_refined(rr, k, b):
    """A tall operator (n = 131072) refined with 3 products per correction:
    the correction blocks are projected against the Ritz vectors by the
    whole-block FP32 Gram and low-rank update kernels of tall blocks."""
    n = 131072
    rp, ci, va, lam = wl.block_diag_csr(n, k, 7100 + b)
    d = [torch.from_numpy(a).to(DEV) for a in (rp, ci, va)]
    V0 = wl.uniform_block(n, b, 7200 + b)
    p = rr.api.make_params(k, b, 2, 40, 1e-10, basis="bf16", v0=dev(V0), refine=True, phase1_sweeps=2,
                           refine_degree=3)
    th, X, info = rr.rr_eig(rr.api.csr_operator(*d), p, n)
    th, X = host(th), host(X)
    assert info["n_converged"] == k, info
    assert np.max(np.abs(th - lam[:k]) / lam[:k]) <= 1e-10
    assert O.residual_eig(O.csr_apply(rp, ci, va), X, th).max() <= 1.5e-10
    assert np.abs(X.T @ X - np.eye(k)).max() < 1e-10
