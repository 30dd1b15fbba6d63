#!/usr/bin/env python
"""Benchmark: converged Ritz triplets per second at 1e-10 relative residual.

Workload (one "step" = one full solve): the dense SVD of
A = U diag(sigma) V^T, 16384 x 4096 FP64, U and V Haar (QR of seeded
Gaussians), sigma_i = exp(-i/60); top k = 64 triplets, block 128, 4 power
sweeps per projection, BF16 basis with FP32 accumulation, FP64 projection,
refinement to relative residual <= 1e-10 (synthetic data, seeded).

Reported: the mixed-precision solve's converged triplets/s (``value``), the
same algorithm all-FP64 on the same GPU (``fp64``), the second run with an
FP8-E4M3 phase-1 basis (``e4m3``), per-stage device times
from CUDA events inside the timed solves (``stages``) and the roofline of the
dominant stage, an end-to-end number through host buffers (``e2e``), and the
FP64 oracle timed on the host cores (``cpu_baseline``).

``--impl reference`` times the oracle (plain FP64 numpy/LAPACK on the host
cores) on the same workload.  N > 1 (torchrun): every rank solves its own
instance (seed + rank), no collective on the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import datetime
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

M, N, B, K, Q = 16384, 4096, 128, 64, 4
TOL = 1e-10
SEED = wl.seed_for(2)
METRIC = "Ritz pairs/s at 1e-10 rel. residual, mixed vs all-FP64 on GB300; % of roofline"
WORKLOAD = ("dense SVD A=U diag(exp(-i/60)) V^T 16384x4096 FP64 (Haar U, V), top 64 triplets, "
            "block 128, 4 power sweeps per projection, BF16 basis + FP32 accumulation, FP64 "
            "projection, refined to rel. residual <= 1e-10")
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")


def bench_config(world: int = 1) -> dict:
    """The workload's config dict, identical in both arms of the bench."""
    return {"workload": WORKLOAD, "m": M, "n": N, "block": B, "k": K, "power_sweeps": Q, "tol": TOL,
            "l2": "inputs larger than L2 (A: 512 MiB FP64 + 256 MiB BF16 copies)",
            "parallelism": f"replicas x{world}"}
# nominal FP64 rate of a GB300 (no measured FP64 figure exists): 1.25 TFLOP/s


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 100 ms; stop(t0, t1) keeps the samples taken
    between the host wall-clock times t0 and t1 (the timed region)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self, t0=None, t1=None):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = []
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if t0 is None or (t0 - 0.05 <= r[0] <= t1 + 0.05)]
        if not inside and rows and t0 is not None:
            # a region shorter than the sampling interval: the sample nearest its middle
            mid = 0.5 * (t0 + t1)
            inside = [min(rows, key=lambda r: abs(r[0] - mid))]
        if not inside:
            return None
        reasons = set()
        for r in inside:
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[3]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median([r[1] for r in inside]), "sm_max_mhz": max(r[2] for r in inside),
                "samples": len(inside), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- oracle legs
def oracle_sweep_seconds(A: np.ndarray, V0: np.ndarray, reps: int = 1) -> float:
    """Time one sweep of the oracle's solve (FP64: q products with A and A^T,
    each followed by Algorithm 8, then Algorithm 5 and the residual check)."""
    from oracle import ofrr as O

    Amul, Atmul = O.dense_apply(A)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        O.solve_svd(Amul, Atmul, A.shape[0], A.shape[1], K, V0, degree=Q, max_sweeps=1, tol=TOL)
        ts.append(time.perf_counter() - t0)
    return statistics.median(ts)


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import ofrr as O

    A = wl.dense_svd(M, N, wl.config2_sigma(N), SEED)
    V0 = wl.uniform_block(N, B, SEED + 1)
    Amul, Atmul = O.dense_apply(A)
    # one full oracle solve fixes the number of sweeps S the method needs here
    t0 = time.perf_counter()
    full = O.solve_svd(Amul, Atmul, M, N, K, V0, degree=Q, max_sweeps=40, tol=TOL)
    t_full = time.perf_counter() - t0
    S = full.sweeps
    for _ in range(args.warmup):
        oracle_sweep_seconds(A, V0)
    ts = [oracle_sweep_seconds(A, V0) for _ in range(args.steps)]
    t_sweep = statistics.median(ts)
    value = full.n_converged / (S * t_sweep)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # one timed step is one oracle sweep: ms_per_step is that sweep's time
        "ms_per_step": t_sweep * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": bench_config(1),
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": "pairs/s", "cores": cores,
                         "sample": f"each timed step = 1 of the {S} sweeps the oracle needs "
                                   f"(median {t_sweep:.2f} s; full solve measured once: {t_full:.1f} s, "
                                   f"{full.n_converged}/{K} converged); value = converged / "
                                   f"(S x median sweep time), a per-sweep extrapolation"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- ranks
def aggregate(seconds: float, converged: int, dist=None, device=None):
    """Whole-job numbers across ranks: the slowest rank's time and the total
    converged pairs (every rank solves its own instance; no data exchange)."""
    if dist is None:
        return seconds, converged
    import torch

    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    c = torch.tensor([float(converged)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


# --------------------------------------------------------------------------- GPU arm
# DRAM bytes per launch of k_gemm_bf16_tc by role (the low-precision products,
# the FP64-emulation passes), mean over one solve of this workload (ncu
# dram__bytes_read.sum + dram__bytes_write.sum, a one-pass capture of every
# launch of the kernel in one solve; profiles/ncu_gemm_bf16_tc_16384x4096x128.md).
# Emptied when the kernel changes, until it is captured again.
TC_TRAFFIC_PER_LAUNCH = {"lowp_product": 221.6e6, "f64_emulation": 231.7e6}


def stage_roofline(info, peaks, src):
    """Per-stage device time (CUDA events inside the library around every
    stage of one solve) with each stage's share, and the roofline of the
    dominant kernel.

    ``roofline`` is the tcgen05 product kernel ``k_gemm_bf16_tc``, the
    dominant kernel, whose launches play two roles: the low-precision
    products (filter products, split-BF16 corrections; HBM-bound at b = 128,
    128 flop per byte of operator against a BF16 ridge near 260) and the
    FP64-emulation passes (all slice pairs of an FP64-accurate product, Gram
    or lift in one launch: 36 pair products per operator slice set, above the
    ridge, so tensor-bound).  The library brackets every launch with CUDA
    events on its stream and adds up, per role, its algorithmic bytes (each
    operand read once -- for an emulation pass the distinct 6-bit slices --
    and the output written once) and flops (2 M N K per product formed).  The
    line carries the role that holds most of the kernel's time against its
    own bound; ``roles`` gives both, and ``kernel_roofline_time_frac`` the
    roofline time of every launch (max of bytes / measured bandwidth and
    flops / measured BF16 rate, per role) over the kernel's measured time.
    """
    ms, calls = info["stage_ms"], info["stage_calls"]
    names = ["lowp_product", "f64_product", "hessenberg", "gram", "pencil", "lift", "other"]
    total = sum(ms[:7])
    stages = {}
    for i, nm in enumerate(names):
        if calls[i] == 0:
            continue
        stages[nm] = {"ms": ms[i], "calls": calls[i], "ms_per_call": ms[i] / calls[i],
                      "share": ms[i] / total if total else None}
    hbm = peaks["hbm_gbs"]
    opb = 2.0 * M * N  # BF16 operator bytes
    if "lowp_product" in stages:
        # the products' stage: plain (2q + 1 per phase-1 sweep) and split (2q + 1 per
        # refinement sweep) products, m n 2 / 2 m n 2 operator bytes each
        ph1 = info["sweeps"] - info["refine_sweeps"]
        prod_bytes = (2 * Q + 1) * (ph1 * opb + info["refine_sweeps"] * 2 * opb)
        ach = prod_bytes / (stages["lowp_product"]["ms"] * 1e-3) / 1e9
        stages["lowp_product"].update({"bound": "hbm", "achieved_gbs": ach, "frac": ach / hbm})
    if "f64_product" in stages:
        # FP64-accurate A X / A^T Y (b = 128): the FP64 operator read once is the
        # algorithmic floor (512 MiB)
        d = stages["f64_product"]
        ach = 8.0 * M * N / (d["ms_per_call"] * 1e-3) / 1e9
        d.update({"bound": "hbm", "achieved_gbs": ach, "frac": ach / hbm,
                  "note": "FP64 operator bytes per product / time"})
    if "hessenberg" in stages:
        d = stages["hessenberg"]
        byts = (M + N) / 2 * B * (4 + 2)
        ach = byts / (d["ms_per_call"] * 1e-3) / 1e9
        d.update({"bound": "latency", "achieved_gbs": ach, "frac": ach / hbm,
                  "note": "floor bytes (read FP32 block, write BF16 basis) / time; b sequential pivots"})
    if "pencil" in stages:
        stages["pencil"].update({"bound": "latency", "us_per_call": stages["pencil"]["ms_per_call"] * 1e3})
    dominant = max(stages, key=lambda k: stages[k]["ms"]) if stages else None
    roof = None
    tc_ms, tc_n = ms[7], calls[7]
    if tc_n:
        tens = peaks["bf16_tflops_sustained"] if "bf16_tflops_sustained" in peaks else peaks["bf16_tflops"]
        rms, rby, rfl = info["tc_role_ms"], info["tc_role_bytes"], info["tc_role_flops"]
        roles = {}
        t_roof = 0.0
        for r, nm in enumerate(["lowp_product", "f64_emulation"]):
            if rms[r] <= 0:
                continue
            t_b = rby[r] / (hbm * 1e9) * 1e3   # ms at the measured copy bandwidth
            t_f = rfl[r] / (tens * 1e12) * 1e3  # ms at the measured BF16 rate
            t_roof += max(t_b, t_f)
            roles[nm] = {"ms": rms[r], "bound": "hbm" if t_b >= t_f else "tensor",
                         "achieved_gbs": rby[r] / (rms[r] * 1e-3) / 1e9,
                         "achieved_tflops": rfl[r] / (rms[r] * 1e-3) / 1e12,
                         "frac": max(t_b, t_f) / rms[r]}
        # the role that holds most of the kernel's time carries the line; the
        # other role and the kernel-wide fraction (roofline time of every
        # launch / its measured time) are reported beside it
        main = max(roles, key=lambda k: roles[k]["ms"])
        d = roles[main]
        if d["bound"] == "tensor":
            roof = {"bound": "tensor", "achieved": d["achieved_tflops"], "peak": tens, "unit": "TFLOP/s",
                    "frac": d["achieved_tflops"] / tens}
        else:
            roof = {"bound": "hbm", "achieved": d["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                    "frac": d["achieved_gbs"] / hbm}
        roof.update({"traffic": TC_TRAFFIC_PER_LAUNCH.get(main),
                     "traffic_scope": "DRAM bytes per launch of this role (mean over one solve, ncu)",
                     "kernel": "k_gemm_bf16_tc", "role": main, "launches": tc_n,
                     "kernel_ms_per_solve": tc_ms, "kernel_share_of_solve": tc_ms / total if total else None,
                     "role_share_of_kernel": d["ms"] / tc_ms, "roles": roles,
                     "kernel_roofline_time_frac": t_roof / tc_ms,
                     "algorithmic_bytes_per_launch": info["tc_bytes"] / tc_n,
                     "dominant_stage": dominant,
                     "peak_source": src + " (of measured; BF16 sustained for the tensor bound)" if src == "measured"
                     else src + " (of fallback)"})
    return roof, stages


def sparse_solve(rr, sweeps=60):
    """The sparse eigenproblem: H = -Lap + diag(v), v_j ~ U[0, 10], 1024 x 1024
    grid (n = 1,048,576), lowest 100 pairs, Chebyshev degree 20, block 160,
    BF16 basis, FP64 projection, residual <= 1e-8; one timed solve plus the
    Chebyshev step timed alone on the same operator (row-major BF16 blocks)."""
    import torch

    peaks, src = load_peaks()
    Ng, k, bs, deg = 1024, 100, 160, 20
    rp, ci, va, _ = wl.grid_schrodinger_csr(Ng, 10.0, wl.seed_for(3))
    n = Ng * Ng
    d = [torch.from_numpy(a).cuda() for a in (rp, ci, va)]
    op = rr.api.csr_operator(*d)
    V0 = rr.fortran(torch.from_numpy(wl.uniform_block(n, bs, wl.seed_for(3) + 1)).cuda())
    p = rr.api.make_params(k, bs, deg, sweeps, 1e-8, basis="bf16", v0=V0, filter=rr.RR.CHEBYSHEV,
                           which=rr.RR.SMALLEST, refine=True, phase1_sweeps=2, profile=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    th, X, info = rr.rr_eig(op, p, n)
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    names = ["lowp_product", "f64_product", "hessenberg", "gram", "pencil", "lift", "other"]
    # the plain filter's step on its own: read Y_j, Y_{j-1}, write Y_{j+1} and the CSR arrays
    L = rr.lib()
    bf = rr.api.DTYPES[torch.bfloat16]
    R = [torch.randn(n, bs, device="cuda", dtype=torch.float32).to(torch.bfloat16) for _ in range(3)]
    stream = torch.cuda.current_stream().cuda_stream

    def step():
        rc = L.rr_chebyshev_step_rows(n, bs, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), bf,
                                      R[1].data_ptr(), R[0].data_ptr(), bs, 0.1, 6.0, 0.5, bf, R[2].data_ptr(),
                                      bs, stream)
        assert rc == 0, rc
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    reps = 10
    e0.record()
    for _ in range(reps):
        step()
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / reps
    nbytes = 4 * (n + 1) + 8 * len(ci) + 3 * 2 * n * bs
    return {"workload": "H = -Lap + diag(v), v ~ U[0,10], 1024x1024 Dirichlet grid (n = 1,048,576, CSR FP32), "
                        "lowest 100 pairs, Chebyshev degree 20, block 160, BF16 basis, tol 1e-8",
            "value": info["n_converged"] / sec, "unit": "pairs/s", "seconds": sec,
            "n_converged": info["n_converged"], "k": k, "tol": 1e-8, "sweeps": info["sweeps"],
            "refine_sweeps": info["refine_sweeps"], "max_res": info["max_res"],
            "theta_first": float(th[0].item()), "theta_last": float(th[-1].item()),
            "stages_ms": dict(zip(names, info["stage_ms"][:7])),
            "cheb_step": {"kernel": "k_csr_cheb_rows", "us": us, "algorithmic_bytes": nbytes,
                          "achieved_gbs": nbytes / us / 1e3, "peak_gbs": peaks["hbm_gbs"],
                          "frac": nbytes / us / 1e3 / peaks["hbm_gbs"], "peak_source": src}}


def run_ours(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2505_00281_gb300 import build

    build.build()
    import paper_2505_00281_gb300 as rr

    L = rr.lib()
    dev = torch.device("cuda", local)
    seed = SEED + 7919 * rank
    sigma = wl.config2_sigma(N)
    At = wl.dense_svd_torch(M, N, sigma, seed, device=str(dev))   # n x m row-major = A col-major
    A = At.t()                                                     # (m, n), stride (1, m)
    V0 = rr.fortran(torch.from_numpy(wl.uniform_block(N, B, seed + 1)).to(dev))
    op = rr.api.dense_operator(A)
    peaks, src = load_peaks()

    def params(basis="bf16", profile=False):
        if basis == "f64":
            return rr.api.make_params(K, B, Q, 40, TOL, basis="f64", v0=V0, refine=False,
                                      profile=profile)
        return rr.api.make_params(K, B, Q, 30, TOL, basis=basis, v0=V0, refine=True,
                                  phase1_sweeps=1, profile=profile)

    p_mixed = params()
    wsb = L.rr_workspace_size(rr.api.ctypes.byref(op), rr.api.ctypes.byref(p_mixed), 1)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    for _ in range(args.warmup):
        rr.rr_svd(op, p_mixed, device=dev, ws=ws)
    # timed steps
    clocks = ClockSampler(local)
    launches0 = L.rr_kernel_launches()
    barrier()
    clocks.start()
    time.sleep(0.3)  # nvidia-smi's first samples come after its start-up
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    wt0 = time.time()
    ev0.record(stream)
    conv = 0
    infos = []
    for _ in range(args.steps):
        s, U, V, info = rr.rr_svd(op, p_mixed, device=dev, ws=ws)
        conv += info["n_converged"]
        infos.append(info)
    ev1.record(stream)
    barrier()
    wt1 = time.time()
    clk = clocks.stop(wt0, wt1)
    launches = L.rr_kernel_launches() - launches0
    t = ev0.elapsed_time(ev1) / 1e3
    t, conv = aggregate(t, conv, dist, dev)
    value = conv / t

    # correctness of the timed result against the closed form (sampled outputs)
    s_h = s.cpu().numpy()
    sig_err = float(np.max(np.abs(s_h - sigma[:K]) / sigma[:K]))

    # stage profile (one more solve, CUDA events around every stage)
    _, _, _, pinfo = rr.rr_svd(op, params(profile=True), device=dev, ws=ws)
    roof, stages = stage_roofline(pinfo, peaks, src)

    # all-FP64 run of the same algorithm
    fp64 = None
    if not args.no_fp64:
        p64 = params("f64")
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s64, _, _, info64 = rr.rr_svd(op, p64, device=dev)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        s64_h = s64.cpu().numpy()
        fp64 = {"value": info64["n_converged"] / t64, "unit": "pairs/s", "seconds": t64,
                "n_converged": info64["n_converged"], "sweeps": info64["sweeps"],
                "mixed_over_fp64": value / (info64["n_converged"] / t64) if info64["n_converged"] else None,
                # the FP64 path's own distance to the prescribed spectrum (the
                # rounding of A to FP64 sets a floor near 1e-14), and the
                # mixed-precision result's distance to it
                "sigma_max_rel_err": float(np.max(np.abs(s64_h - sigma[:K]) / sigma[:K])),
                "sigma_max_rel_diff_mixed": float(np.max(np.abs(s_h - s64_h) / s64_h))}

    # the second run of the workload with an FP8-E4M3 phase-1 basis (operator and basis
    # in E4M3 with power-of-two scales, tcgen05 kind::f8f6f4 products), refined to the same
    # tolerance on BF16 correction blocks: one warm-up solve and one timed solve
    e4m3 = None
    if not args.no_fp8:
        p8 = params("e4m3")
        ws8 = torch.empty(L.rr_workspace_size(rr.api.ctypes.byref(op), rr.api.ctypes.byref(p8), 1),
                          dtype=torch.uint8, device=dev)
        rr.rr_svd(op, p8, device=dev, ws=ws8)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s8, _, _, info8 = rr.rr_svd(op, p8, device=dev, ws=ws8)
        e1.record(stream)
        torch.cuda.synchronize()
        t8 = e0.elapsed_time(e1) / 1e3
        s8_h = s8.cpu().numpy()
        e4m3 = {"value": info8["n_converged"] / t8, "unit": "pairs/s", "seconds": t8,
                "n_converged": info8["n_converged"], "sweeps": info8["sweeps"],
                "refine_sweeps": info8["refine_sweeps"], "res_history": info8["res_history"],
                "sigma_max_rel_err": float(np.max(np.abs(s8_h - sigma[:K]) / sigma[:K]))}
        del ws8

    # end to end through host buffers: H2D of A and V0 from pinned memory,
    # the solve, D2H of sigma, U, V every step
    A_host = torch.empty((N, M), dtype=torch.float64, pin_memory=True)
    A_host.copy_(At)
    V0_host = torch.empty((B, N), dtype=torch.float64, pin_memory=True)
    V0_host.copy_(V0.t())
    A_dev2 = torch.empty_like(At)
    V0_dev2 = torch.empty((B, N), dtype=torch.float64, device=dev)
    op2 = rr.api.dense_operator(A_dev2.t())
    p2 = rr.api.make_params(K, B, Q, 30, TOL, basis="bf16", v0=V0_dev2.t(), refine=True, phase1_sweeps=1)
    s_host = torch.empty(K, dtype=torch.float64, pin_memory=True)
    U_host = torch.empty((K, M), dtype=torch.float64, pin_memory=True)
    V_host = torch.empty((K, N), dtype=torch.float64, pin_memory=True)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    conv2 = 0
    for _ in range(args.steps):
        A_dev2.copy_(A_host, non_blocking=True)
        V0_dev2.copy_(V0_host, non_blocking=True)
        s2, U2, V2, info2 = rr.rr_svd(op2, p2, device=dev, ws=ws)
        s_host.copy_(s2, non_blocking=True)
        U_host.copy_(U2.t(), non_blocking=True)
        V_host.copy_(V2.t(), non_blocking=True)
        conv2 += info2["n_converged"]
    e1.record(stream)
    barrier()
    t2 = e0.elapsed_time(e1) / 1e3
    t2, conv2 = aggregate(t2, conv2, dist, dev)
    e2e = {"value": conv2 / t2, "unit": "pairs/s", "h2d_bytes_per_step": (M * N + N * B) * 8,
           "d2h_bytes_per_step": (K + M * K + N * K) * 8}

    # the sparse eigenproblem of the same family of methods (rank 0, N = 1 only)
    sparse = None
    if rank == 0 and world == 1 and not args.no_sparse:
        del ws
        torch.cuda.empty_cache()
        sparse = sparse_solve(rr)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        A_np = At.t().cpu().numpy()  # column-major view of the same matrix
        V0_np = V0.cpu().numpy()
        t_sweep = oracle_sweep_seconds(np.asfortranarray(A_np), V0_np)
        S = fp64["sweeps"] if fp64 else 4
        cpu = {"value": K / (S * t_sweep), "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one oracle sweep (q={Q} power sweeps with Algorithm 8, Algorithm 5, FP64 "
                         f"residuals) on the full 16384x4096 input took {t_sweep:.2f} s; value = "
                         f"{K} / ({S} sweeps, the count the same algorithm needs in FP64 on the GPU, "
                         f"x sweep time)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic (seeded Haar factors, prescribed spectrum)",
            "config": bench_config(world),
            "converged": conv, "sigma_max_rel_err": sig_err,
            "sweeps": infos[-1]["sweeps"], "refine_sweeps": infos[-1]["refine_sweeps"],
            "res_history": infos[-1]["res_history"],
            "fp64": fp64, "e4m3": e4m3, "sparse": sparse, "stages": stages, "roofline": roof,
            "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk, "gpu_launches": int(launches),
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def run_stage(args):
    """Single-stage driver for profiling (ncu -k on one kernel): runs one
    stage of the bench workload twice (warm-up, then the profiled call)."""
    import torch

    from paper_2505_00281_gb300 import build

    build.build()
    import paper_2505_00281_gb300 as rr

    rng = np.random.default_rng(7)
    b = args.b

    def dev(a, dt=None):
        t = torch.from_numpy(np.asfortranarray(a)).cuda()
        return rr.fortran(t.to(dt) if dt is not None else t)

    if args.stage == "pencil":
        A = rng.standard_normal((3 * b, 2 * b))
        U = rng.uniform(0, 1, (3 * b, b))
        V = rng.uniform(0, 1, (2 * b, b))
        Bp, Gu, Gv = dev(U.T @ A @ V), dev(U.T @ U), dev(V.T @ V)
        for _ in range(2):
            rr.rr_pencil_svd(Bp, Gu, Gv)
    elif args.stage == "hessenberg":
        W0 = torch.randn(b, args.rows, device="cuda", dtype=torch.float32).t()  # rows x b column-major
        for _ in range(2):
            rr.rr_hessenberg(W0.clone(), qtype=torch.bfloat16)
    elif args.stage == "split":
        Af = torch.randn(M, N, device="cuda", dtype=torch.float32)  # row-major M x N: K-major for A V
        Ah = Af.to(torch.bfloat16)
        Al = (Af - Ah.float()).to(torch.bfloat16)
        Xf = torch.randn(B, N, device="cuda", dtype=torch.float32).t()  # N x B column-major
        Xh = rr.fortran(Xf.to(torch.bfloat16))
        Xl = rr.fortran((Xf - Xh.float()).to(torch.bfloat16))
        for _ in range(2):
            rr.rr_gemm_lowp_split(M, B, N, Ah, Al, N, Xh, Xl, N)
    elif args.stage == "cheb":
        # the sparse workload's filter step: H = -Lap + diag(v) on the 1024 x 1024 grid
        # (n = 1,048,576, 5-point stencil, FP32 values), block 160 in BF16
        Ng, bs = 1024, 160
        rp, ci, va, _ = wl.grid_schrodinger_csr(Ng, 10.0, 3001)
        n = Ng * Ng
        d_rp, d_ci, d_va = (torch.from_numpy(a).cuda() for a in (rp, ci, va))
        Y0 = rr.fortran(torch.randn(bs, n, device="cuda", dtype=torch.float32).t().to(torch.bfloat16))
        Y1 = rr.fortran(torch.randn(bs, n, device="cuda", dtype=torch.float32).t().to(torch.bfloat16))
        Y2 = rr.fortran(torch.empty(bs, n, device="cuda", dtype=torch.bfloat16).t())
        L = rr.lib()
        bf = rr.api.DTYPES[torch.bfloat16]
        stream = torch.cuda.current_stream().cuda_stream

        def step():  # the C entry point on preallocated blocks (no allocation in the timed loop)
            rc = L.rr_chebyshev_step(n, bs, d_rp.data_ptr(), d_ci.data_ptr(), d_va.data_ptr(), bf, Y1.data_ptr(),
                                     Y0.data_ptr(), n, 0.1, 6.0, 0.5, None, None, 0, None, bf, Y2.data_ptr(), n,
                                     stream)
            assert rc == 0, rc
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        reps = 10
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            step()
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / reps
        del Y2
        # the same step on row-major blocks (the eigensolver's filter layout)
        R0 = torch.randn(n, bs, device="cuda", dtype=torch.float32).to(torch.bfloat16)
        R1 = torch.randn(n, bs, device="cuda", dtype=torch.float32).to(torch.bfloat16)
        R2 = torch.empty(n, bs, device="cuda", dtype=torch.bfloat16)

        def step_rows():
            rc = L.rr_chebyshev_step_rows(n, bs, d_rp.data_ptr(), d_ci.data_ptr(), d_va.data_ptr(), bf,
                                          R1.data_ptr(), R0.data_ptr(), bs, 0.1, 6.0, 0.5, bf, R2.data_ptr(), bs,
                                          stream)
            assert rc == 0, rc
        for _ in range(3):
            step_rows()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            step_rows()
        e1.record()
        torch.cuda.synchronize()
        us_rows = e0.elapsed_time(e1) * 1e3 / reps
        nbytes = 4 * (n + 1) + 8 * len(ci) + 3 * 2 * n * bs  # CSR, Y_cur, Y_prev, Y_next
        peaks, src = load_peaks()
        print(json.dumps({"stage": "cheb", "n": n, "nnz": int(len(ci)), "b": bs, "algorithmic_bytes": nbytes,
                          "columns": {"us_per_step": us, "achieved_gbs": nbytes / us / 1e3},
                          "rows": {"us_per_step": us_rows, "achieved_gbs": nbytes / us_rows / 1e3,
                                   "frac": nbytes / us_rows / 1e3 / peaks["hbm_gbs"]},
                          "peak_gbs": peaks["hbm_gbs"], "peak_source": src}))
    elif args.stage == "sparse":
        print(json.dumps({"stage": "sparse", **sparse_solve(rr, args.sweeps)}))
    elif args.stage == "project":
        # a tall refined eigensolve whose correction blocks are projected against
        # the Ritz vectors by the whole-block FP32 Gram and low-rank update:
        # block-diagonal CSR (4 x 4 blocks), n rows, 64 largest pairs, block 160,
        # BF16 basis, 3 products per correction, 6 sweeps
        import torch
        n, k, bs = args.rows if args.rows != M else 131072, 64, 160
        rp, ci, va, lam = wl.block_diag_csr(n, k, 7100 + bs)
        d = [torch.from_numpy(a).cuda() for a in (rp, ci, va)]
        V0 = rr.fortran(torch.from_numpy(wl.uniform_block(n, bs, 7200 + bs)).cuda())
        p = rr.api.make_params(k, bs, 2, 6, 1e-10, basis="bf16", v0=V0, refine=True, phase1_sweeps=2,
                               refine_degree=3, profile=True)
        th, X, info = rr.rr_eig(rr.api.csr_operator(*d), p, n)
        torch.cuda.synchronize()
        names = ["lowp_product", "f64_product", "hessenberg", "gram", "pencil", "lift", "other"]
        print(json.dumps({"stage": "project", "n": n, "k": k, "b": bs, "sweeps": info["sweeps"],
                          "res_history": info["res_history"][:info["sweeps"]],
                          "stages_ms": dict(zip(names, info["stage_ms"][:7]))}))
    elif args.stage == "warm":
        # learned warm start: H(p) = -Lap + V_p (8 Gaussian bumps) on a grid x grid mesh,
        # lowest k pairs; train on solves of `train` family members, then solve `test`
        # held-out members from the random, free-mode and learned start blocks
        from paper_2505_00281_gb300 import warmstart as WS
        Ng = args.grid
        k, bs, deg, hidden, depth = (16, 24, 10, 24, 3) if Ng <= 64 else (32, 48, 20, 32, 4)
        hidden = args.hidden or hidden
        depth = args.depth or depth

        def problems(seeds):
            for sd in seeds:
                pot = wl.gaussian_potential(Ng, sd)
                rp, ci, va = wl.grid_potential_csr(Ng, pot.ravel())
                yield pot, rp, ci, va, wl.uniform_block(Ng * Ng, bs, sd + 1)
        t0 = time.perf_counter()
        data = WS.eigen_targets(problems(range(70000, 70000 + args.train)), k, bs, deg)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        params = wl.conv_params(WS.layer_shapes(k, hidden, depth), 44)
        params = [(W * (0.1 if i == depth - 1 else 1.0), b) for i, (W, b) in enumerate(params)]
        net = WS.StartBlockNet(Ng, k, params)
        hist = WS.train(net, [(P, X) for P, X, _ in data], epochs=args.epochs, lr=2e-3, batch=8)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        rows = WS.evaluate(net, problems(range(71000, 71000 + args.test)), k, bs, deg)

        def gmean(v):
            return float(np.exp(np.mean(np.log(np.maximum(v, 1e-300)))))
        arms = {}
        for arm in WS.ARMS:
            arms[arm] = {
                "sweeps": float(np.mean([r[arm]["sweeps"] for r in rows])),
                "ms": float(np.mean([r[arm]["ms"] for r in rows])),
                "res_after_1": gmean([r[arm]["res"][0] for r in rows]),
                "res_after_3": gmean([r[arm]["res"][min(2, len(r[arm]["res"]) - 1)] for r in rows]),
                "converged": [r[arm]["n_converged"] for r in rows]}
        print(json.dumps({"stage": "warm", "grid": Ng, "k": k, "block": bs, "degree": deg,
                          "params": int(sum(W.size + b.size for W, b in params)), "train": args.train,
                          "test": args.test, "epochs": args.epochs,
                          "target_ms_per_solve": 1e3 * (t1 - t0) / max(1, args.train),
                          "train_ms_per_sample_step": 1e3 * (t2 - t1) / max(1, args.epochs * args.train),
                          "loss_first": hist[0] if hist else None, "loss_last": hist[-1] if hist else None,
                          "arms": arms}))
    elif args.stage == "fp8":
        # the dense workload's block product A V (16384 x 4096 operator, block 128) with BF16
        # operands and with E4M3 operands (power-of-two row / column scales), CUDA events
        A = torch.randn(N, M, device="cuda", dtype=torch.float64).t()   # M x N column-major
        V = rr.fortran(torch.randn(N, B, device="cuda", dtype=torch.float64))
        A_row = A.to(torch.bfloat16).contiguous()
        Vb = rr.fortran(V.to(torch.bfloat16))
        Aq, ia = rr.rr_quantize_e4m3(A, by_rows=True)
        Vq, iv = rr.rr_quantize_e4m3(V, by_rows=False)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        out = {}
        for name, fn, nbytes in (("bf16", lambda: rr.rr_gemm_lowp(2, M, B, N, A_row, N, Vb, N), M * N * 2),
                                 ("e4m3", lambda: rr.rr_gemm_e4m3(M, B, N, Aq, ia, Vq, iv), M * N)):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            reps = 20
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / reps
            out[name] = {"us": us, "operator_gbs": nbytes / us / 1e3, "tflops": 2.0 * M * N * B / us / 1e6}
        Cb = rr.rr_gemm_lowp(2, M, B, N, A_row, N, Vb, N)
        C8 = rr.rr_gemm_e4m3(M, B, N, Aq, ia, Vq, iv)
        ref = A @ V
        scale = ref.abs().max().item()
        peaks, src = load_peaks()
        print(json.dumps({"stage": "fp8", "M": M, "N": B, "K": N, **out, "peak_gbs": peaks["hbm_gbs"],
                          "peak_source": src,
                          "max_err_rel": {"bf16": (Cb.double() - ref).abs().max().item() / scale,
                                          "e4m3": (C8.double() - ref).abs().max().item() / scale}}))
    elif args.stage == "batch":
        # the batched workload: 512 SVDs, m_i = 4 round(64 16^u_i), n_i = m_i / 4, sigma_j = j^-1.5,
        # top 16 triplets, block 32, BF16 basis refined to 1e-10; autotuned per size class
        from paper_2505_00281_gb300 import autotune as AT
        shapes = wl.config4_shapes(args.count)
        mats = [wl.dense_svd_torch(m, n, wl.config4_sigma(n), 4000 + i) for i, (m, n) in enumerate(shapes)]
        ops = [rr.api.dense_operator(t.t()) for t in mats]
        params = rr.api.make_params(16, 32, 4, args.batch_sweeps, 1e-10, basis="bf16", refine=True,
                                    phase1_sweeps=1, refine_degree=args.refine_degree)
        by_class = {}
        for op_ in ops:
            by_class.setdefault(AT.size_class(op_.m, op_.n), []).append(op_)
        samples = {k: v[:8] for k, v in by_class.items()}
        cands = [{"branches": b_, "max_splits": c_, "order": 1} for b_ in (8, 32) for c_ in (0, 1, 4)]
        t0 = time.perf_counter()
        table = AT.tune(samples, params, candidates=cands, reps=1) if args.tune else AT.load()
        t_tune = time.perf_counter() - t0 if args.tune else 0.0
        if args.table:
            AT.save(table, args.table)

        def run(fn):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, st, infos = fn()
            torch.cuda.synchronize()
            return time.perf_counter() - t1, st, infos
        t_def, st_def, inf_def = run(lambda: rr.rr_batch_svd(ops, params, 7))
        # the same batch with the all-FP64 method (the same sweeps, no refinement)
        p64 = rr.api.make_params(16, 32, 4, args.batch_sweeps, 1e-10, basis="f64", refine=False)
        t_64, st_64, inf_64 = run(lambda: rr.rr_batch_svd(ops, p64, 7))
        t_tuned, st_tuned, inf_tuned = run(lambda: AT.batch_svd(ops, params, 7, table))
        conv = lambda infos: int(sum(i["n_converged"] for i in infos))

        def failures(st):
            out = {}
            for op_, x in zip(ops, st):
                if x != 0:
                    key = AT.size_class(op_.m, op_.n)
                    out[key] = out.get(key, 0) + 1
            return out
        print(json.dumps({"stage": "batch", "count": len(ops), "sweeps": args.batch_sweeps,
                          "refine_degree": args.refine_degree,
                          "converged_problems": {"default": sum(1 for x in st_def if x == 0),
                                                 "tuned": sum(1 for x in st_tuned if x == 0),
                                                 "fp64": sum(1 for x in st_64 if x == 0)},
                          "fp64": {"seconds": t_64, "problems_per_s": len(ops) / t_64,
                                   "pairs_per_s": conv(inf_64) / t_64, "failed_by_class": failures(st_64)},
                          "classes": {k: len(v) for k, v in by_class.items()}, "tune_seconds": t_tune,
                          "sweeps_mean": {"default": float(np.mean([i["sweeps"] for i in inf_def])),
                                          "fp64": float(np.mean([i["sweeps"] for i in inf_64]))},
                          "default": {"seconds": t_def, "problems_per_s": len(ops) / t_def,
                                      "pairs_per_s": conv(inf_def) / t_def, "failed_by_class": failures(st_def),
                                      "max_res_by_class": {k: max(i["max_res"] for op_, i in zip(ops, inf_def)
                                                                  if AT.size_class(op_.m, op_.n) == k)
                                                           for k in by_class}},
                          "tuned": {"seconds": t_tuned, "problems_per_s": len(ops) / t_tuned,
                                    "pairs_per_s": conv(inf_tuned) / t_tuned, "failed_by_class": failures(st_tuned)},
                          "table": table}))
    elif args.stage == "kernel":
        # the Gaussian kernel-matrix family at scale: n points uniform in the square of side sqrt(n)
        # (one per unit area, as the paper's 1000-point sets), f = 0.2, l = 10, s = 0.01; the 20
        # largest eigenpairs, block 32, 3 products per sweep, BF16 basis refined to 1e-10, through the
        # matrix-free operator; and the operator product alone (FP32 and FP64 evaluation)
        n, f, l, sh, k, bs = args.points, 0.2, 10.0, 0.01, 20, 32
        x = torch.from_numpy(wl.kernel_points(n, 6500)).cuda()
        op = rr.api.kernel_operator(x, f, l, sh)
        V = rr.fortran(torch.rand(n, bs, device="cuda", dtype=torch.float64))
        out = {}
        for name, Xd, odt in (("fp32", V.to(torch.float32), torch.float32), ("fp64", V, torch.float64)):
            for _ in range(2):
                rr.api.rr_kernel_apply(op, rr.fortran(Xd), out_dtype=odt)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            reps = 3
            for _ in range(reps):
                rr.api.rr_kernel_apply(op, rr.fortran(Xd), out_dtype=odt)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            flops = 2.0 * n * n * bs
            out[name] = {"ms": ms, "tflops": flops / ms / 1e9, "entries_per_s": n * n / ms * 1e3}
        # FP32 FMA peak from the unit counts: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
        fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
        out["fp32"]["frac_of_fp32_fma_peak"] = out["fp32"]["tflops"] / fp32_peak
        if args.products_only:
            print(json.dumps({"stage": "kernel", "n": n, "block": bs, "products": out, "fp32_fma_peak_tflops": fp32_peak}))
            torch.cuda.synchronize()
            print("stage", args.stage, "done")
            return 0
        p = rr.api.make_params(k, bs, 3, 40, 1e-10, basis="bf16", v0=None, seed=6501, refine=True, phase1_sweeps=2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        th, X, info = rr.rr_eig(op, p, n)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        print(json.dumps({"stage": "kernel", "n": n, "f": f, "l": l, "s": sh, "k": k, "block": bs,
                          "products": out, "fp32_fma_peak_tflops": fp32_peak, "bound": "alu",
                          "solve": {"seconds": sec, "n_converged": info["n_converged"], "sweeps": info["sweeps"],
                                    "max_res": info["max_res"], "pairs_per_s": info["n_converged"] / sec,
                                    "theta_first": float(th[0].item()), "theta_last": float(th[-1].item())}}))
    elif args.stage == "krylov":
        # Krylov-Hessenberg + OFRR on the sparse workload's operator (1024 x 1024 grid, n = 1,048,576):
        # Krylov dimension 100, 4 restarts from the top Ritz vector, the 20 largest pairs reported
        Ng, m, restarts, k = 1024, 100, 4, 20
        rp, ci, va, _ = wl.grid_schrodinger_csr(Ng, 10.0, wl.seed_for(3))
        d = [torch.from_numpy(a).cuda() for a in (rp, ci, va)]
        op = rr.api.csr_operator(*d)
        v = torch.from_numpy(wl.uniform_block(Ng * Ng, 1, 6601)[:, 0]).cuda()
        out = {}
        for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
            rr.rr_krylov_eig(op, v, m, 0, k, dtype=dt)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            th, X, res = rr.rr_krylov_eig(op, v, m, restarts, k, dtype=dt)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            r = res.cpu().numpy()
            # bytes of one cycle's basis process: every step reads the earlier vectors once
            es = 8 if dt == torch.float64 else 4
            byts = (restarts + 1) * (es * Ng * Ng * m * (m + 1) / 2 + m * (len(ci) * 8 + (Ng * Ng + 1) * 4))
            out[name] = {"ms": ms, "theta_first": float(th[0].item()), "res_first": float(r[0]),
                         "res_median": float(np.median(r)), "converged_1e-8": int((r < 1e-8).sum()),
                         "process_bytes": byts, "process_gbs_over_solve": byts / ms / 1e6}
        print(json.dumps({"stage": "krylov", "n": Ng * Ng, "m": m, "restarts": restarts, "k": k, **out}))
    elif args.stage == "builders":
        # Table 3's comparison on this GPU: MGS-L, MGS-R, CGS, CGS-2, Hess-L, Hess-R on U(0,1)
        # blocks of 25000 x 200, 50000 x 200 and 50000 x 400 in FP64, FP32 and FP16 storage (FP16
        # computes in FP32); CUDA events, median of 3 after one warm-up.  The paper's numbers
        # (RTX 3070 Ti) are context only.
        shapes = [(25000, 200), (50000, 200), (50000, 400)]
        methods = ["mgs_l", "mgs_r", "cgs", "cgs2", "hess_l", "hess_r"]
        out = {}
        for dt, name in ((torch.float64, "fp64"), (torch.float32, "fp32"), (torch.float16, "fp16")):
            for (n, k) in shapes:
                W0 = rr.fortran(torch.rand(k, n, device="cuda", dtype=torch.float64).t()).to(dt)
                W0 = rr.fortran(W0)
                for mth in methods:
                    if args.quick and mth == "mgs_l" and k > 200:
                        continue
                    ts = []
                    for rep in range(4):
                        W = rr.fortran(W0.clone())
                        torch.cuda.synchronize()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record()
                        rr.api.rr_basis_builder(W, mth, want_r=False)
                        e1.record()
                        torch.cuda.synchronize()
                        if rep:
                            ts.append(e0.elapsed_time(e1))
                    out.setdefault(name, {}).setdefault(f"{n}x{k}", {})[mth] = float(np.median(ts))
        print(json.dumps({"stage": "builders", "ms": out}))
    elif args.stage == "prep":
        A = torch.randn(N, M, device="cuda", dtype=torch.float64).t()   # M x N column-major
        X = rr.fortran(torch.randn(N, B, device="cuda", dtype=torch.float64))
        Y = rr.fortran(torch.randn(M, B, device="cuda", dtype=torch.float64))
        for _ in range(2):
            rr.rr_split_operator(A)                  # BF16 hi / lo, both layouts
            rr.rr_gemm_f64_emulated(0, A, X)         # row-scaled slices (+ products)
            rr.rr_gemm_f64_emulated(1, A, Y)         # column-scaled slices (+ products)
    elif args.stage in ("gemm", "f64emu"):
        A = torch.randn(N, M, device="cuda", dtype=torch.float64).t()   # M x N column-major
        X = rr.fortran(torch.randn(N, B, device="cuda", dtype=torch.float64))
        A_row = A.to(torch.bfloat16).contiguous()   # element (i, k) at i*N + k: K-major
        Xb = rr.fortran(X.to(torch.bfloat16))
        for _ in range(2):
            if args.stage == "f64emu":
                rr.rr_gemm_f64_emulated(0, A, X)
            else:
                rr.rr_gemm_lowp(2, M, B, N, A_row, N, Xb, N)
    torch.cuda.synchronize()
    print("stage", args.stage, "done")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp8", action="store_true", help="skip the FP8-E4M3 basis run")
    ap.add_argument("--no-sparse", action="store_true", help="skip the sparse eigenproblem leg")
    ap.add_argument("--stage", choices=["pencil", "hessenberg", "gemm", "split", "f64emu", "prep", "cheb", "warm", "sparse",
                                        "fp8", "batch", "kernel", "krylov", "builders", "project"],
                    help="run one stage of the workload (profiling driver)")
    ap.add_argument("--b", type=int, default=256, help="pencil size for --stage pencil, columns for hessenberg")
    ap.add_argument("--rows", type=int, default=M,
                    help="rows of the block for --stage hessenberg (of the operator for --stage project)")
    ap.add_argument("--grid", type=int, default=64, help="grid side for --stage warm")
    ap.add_argument("--points", type=int, default=65536, help="points of the kernel operator for --stage kernel")
    ap.add_argument("--quick", action="store_true", help="--stage builders: skip MGS-L at k = 400")
    ap.add_argument("--products-only", action="store_true", help="--stage kernel: time the operator products only")
    ap.add_argument("--sweeps", type=int, default=60, help="sweep limit for --stage sparse")
    ap.add_argument("--count", type=int, default=512, help="problems for --stage batch")
    ap.add_argument("--batch-sweeps", type=int, default=12, help="sweeps of every problem for --stage batch")
    ap.add_argument("--table", default="", help="--stage batch: write the tuned table (JSON) here")
    ap.add_argument("--tune", action="store_true", help="--stage batch: tune now instead of the shipped table")
    ap.add_argument("--refine-degree", type=int, default=0,
                    help="--stage batch: products per refinement sweep (0: the power degree)")
    ap.add_argument("--train", type=int, default=48, help="training solves for --stage warm")
    ap.add_argument("--test", type=int, default=8, help="held-out solves for --stage warm")
    ap.add_argument("--epochs", type=int, default=40, help="training epochs for --stage warm")
    ap.add_argument("--hidden", type=int, default=0, help="--stage warm: hidden channels (0: by grid)")
    ap.add_argument("--depth", type=int, default=0, help="--stage warm: convolution layers (0: by grid)")
    args = ap.parse_args()
    if args.stage:
        return run_stage(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
