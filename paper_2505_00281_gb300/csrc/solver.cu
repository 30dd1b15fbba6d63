// Host orchestration of the solvers (rr_eig, rr_svd, rr_batch_svd).
//
// Phase 1 is the paper's method: Algorithm 1 (subspace iteration, the RR
// output restarting the next sweep, Sec. 2) with Algorithm 8 after every
// product and OFRR (Algorithm 3 / 5) in the precision map of Sec. 4.2:
// basis and products in the low precision, projection accumulated in FP64,
// small problem in FP64.
//
// Phase 2 (refinement; the paper reaches only the basis precision, so this
// is an added step) keeps the Ritz vectors X in FP64 and, per sweep:
//   P = A X   (FP64-accurate), R = P - X Theta, residual check (Sec. 5.2.2);
//   the correction block D = p(A) X - X p(Theta) built in the low precision
//   from R by the filter's own recurrence (every low-precision quantity is
//   O(|R|), so its rounding error is relative to the residual, not to X);
//   OFRR over S = [X, D] with FP64-accurate blocks where X is involved.
// The span of [X, D] equals span(X, p(A) X), so a sweep contracts the error
// by the filter rate, limited below by the low precision's unit roundoff.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <vector>

#include "rr_common.cuh"
#include "solver_kernels.cuh"

namespace rr {

struct Op {
  int kind;
  const rr_operator* kop;  // RR_KERNEL: the caller's operator (points, parameters)
  int64_t m, n;
  const double* A;
  int64_t lda;
  const int32_t* rp;
  const int32_t* ci;
  const float* va;
  void* lo_col;  // K-major operand of A^T X (column-major copy), dtype dt
  void* lo_row;  // K-major operand of A X (row-major copy), dtype dt
  // split BF16 operator (refinement of a BF16 basis): the BF16 residuals
  // A - bf16(A), same layouts, for the products of the correction recurrence
  bool split;
  void* lo2_col;
  void* lo2_row;
  int32_t dt;    // basis dtype
  int32_t wt;    // product output type (F32, or F64 when dt is F64)
  // FP64-accurate products on the tensor cores (dense operator, refinement)
  bool has_emu;
  EmuOperator emu;
  void* emu_mem;
  void* emu_blk;
  // FP64-accurate lifts on the tensor cores (low-precision bases)
  void* lift_mem;
  size_t lift_bytes;
  // FP8-E4M3 basis (dense SVD, phase 1): E4M3 copies of the operator with one
  // power-of-two scale per row (row-major, for A V) and per column (column-
  // major, for A^T U), the inverse scales, and the basis scale 2^-8 per column.
  // dt stays BF16 for the refinement phase.
  bool f8;
  void* f8_row;
  void* f8_col;
  int64_t f8_ldr, f8_ldc;
  float* f8_rs;
  float* f8_cs;
  float* f8_bs;
  void* f8_scratch;
};

constexpr int kEmuSlices = 8;

static size_t dsz(int32_t t) { return dtype_size(t); }

// Per-stage device timing with CUDA events on the solver's stream (enabled by
// rr_params.profile; read once, after the solve's final synchronisation).
struct Prof {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<int, size_t>> recs;  // (stage, index of the start event)
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  TcProf tc;  // kernel-level timing of the tensor-core product kernel
  void start() {
    if (on) tc_prof_attach(&tc);
  }
  void finish(rr_info* inf) {
    tc_prof_attach(nullptr);
    if (on && inf) {
      cudaStreamSynchronize(s);
      for (auto& r : recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pool[r.second], pool[r.second + 1]) == cudaSuccess) {
          inf->stage_ms[r.first] += ms;
          inf->stage_calls[r.first] += 1;
        }
      }
      for (size_t i = 0; i + 1 < tc.ev.size(); i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, tc.ev[i], tc.ev[i + 1]) == cudaSuccess) {
          inf->stage_ms[RR_KERNEL_TC] += ms;
          inf->stage_calls[RR_KERNEL_TC] += 1;
          inf->tc_role_ms[tc.role[i / 2]] += ms;
        }
      }
      inf->tc_bytes = tc.bytes;
      for (int r = 0; r < 2; ++r) {
        inf->tc_role_bytes[r] = tc.role_bytes[r];
        inf->tc_role_flops[r] = tc.role_flops[r];
      }
    }
    for (auto e : pool) cudaEventDestroy(e);
    for (auto e : tc.ev) cudaEventDestroy(e);
    tc.ev.clear();
    tc.role.clear();
    tc.bytes = 0.0;
    tc.role_bytes[0] = tc.role_bytes[1] = tc.role_flops[0] = tc.role_flops[1] = 0.0;
    tc.launches = 0;
    pool.clear();
    recs.clear();
    used = 0;
  }
  ~Prof() { finish(nullptr); }
};

struct StageScope {
  Prof* p;
  int st;
  size_t i0;
  StageScope(Prof* p_, int st_) : p(p_), st(st_), i0(0) {
    if (p->on) {
      i0 = p->used;
      cudaEventRecord(p->get(), p->s);
    }
  }
  ~StageScope() {
    if (p->on) {
      cudaEventRecord(p->get(), p->s);
      p->recs.push_back({st, i0});
    }
  }
};

#define STAGE(st, expr)              \
  do {                               \
    StageScope _sc(&prof, (st));     \
    RR_TRY(expr);                    \
  } while (0)

// ---------------------------------------------------------------------------
// products
// ---------------------------------------------------------------------------
// out (m x b, wt) = A X (+ coef_j R(:,j)),  X (n x b, dt)
static rr_status apply_lowp(const Op& op, int64_t b, const void* X, int64_t ldx, void* out,
                            int64_t ldo, const double* R, int64_t ldr, const double* coef,
                            cudaStream_t s) {
  if (op.kind == RR_KERNEL) return kernel_apply(s, op.kop, 0, b, op.dt, X, ldx, op.wt, out, ldo, R, ldr, coef);
  if (op.kind == RR_DENSE) {
    if (op.dt == RR_F64) {
      RR_TRY(rr_gemm_f64(0, op.m, b, op.n, op.A, op.lda, (const double*)X, ldx, (double*)out, ldo, 0, s));
      if (R) {
        // out += coef * R  (FP64 path: lift-style axpy via residual kernel is not needed; use lift)
        return RR_ERR_ARG;
      }
      return RR_OK;
    }
    return rr_gemm_lowp(op.dt, op.m, b, op.n, op.lo_row, op.n, X, ldx, (float*)out, ldo, R, ldr,
                        coef, s);
  }
  // CSR: Y = A X via the Chebyshev step with alpha = 1, c = 0, beta = 0
  return rr_chebyshev_step(op.n, b, op.rp, op.ci, op.va, op.dt, X, nullptr, ldx, 1.0, 0.0, 0.0,
                           nullptr, R, ldr, coef, op.wt, out, ldo, s);
}

// Phase-1 products of the SVD: E4M3 operands when the basis is E4M3 (X holds
// codes of 256 x, the basis scale 2^-8 undoes it), else as apply_lowp(_T).
static rr_status apply_ph1(const Op& op, int64_t b, const void* X, int64_t ldx, float* out, int64_t ldo,
                           cudaStream_t s) {
  if (!op.f8) return apply_lowp(op, b, X, ldx, out, ldo, nullptr, 0, nullptr, s);
  return gemm_e4m3_tc(op.m, b, op.n, op.f8_row, op.f8_ldr, op.f8_rs, X, ldx, op.f8_bs, out, ldo, s);
}

// out (n x b, wt) = A^T X (+ coef_j R(:,j)),  X (m x b, dt)
static rr_status apply_lowp_T(const Op& op, int64_t b, const void* X, int64_t ldx, void* out,
                              int64_t ldo, const double* R, int64_t ldr, const double* coef,
                              cudaStream_t s) {
  if (op.kind == RR_KERNEL) return kernel_apply(s, op.kop, 1, b, op.dt, X, ldx, op.wt, out, ldo, R, ldr, coef);
  if (op.kind != RR_DENSE) return RR_ERR_ARG;
  if (op.dt == RR_F64) {
    if (R) return RR_ERR_ARG;
    return rr_gemm_f64(1, op.n, b, op.m, op.A, op.lda, (const double*)X, ldx, (double*)out, ldo, 0, s);
  }
  return rr_gemm_lowp(op.dt, op.n, b, op.m, op.lo_col, op.m, X, ldx, (float*)out, ldo, R, ldr, coef, s);
}

static rr_status apply_ph1_T(const Op& op, int64_t b, const void* X, int64_t ldx, float* out, int64_t ldo,
                             cudaStream_t s) {
  if (!op.f8) return apply_lowp_T(op, b, X, ldx, out, ldo, nullptr, 0, nullptr, s);
  return gemm_e4m3_tc(op.n, b, op.m, op.f8_col, op.f8_ldc, op.f8_cs, X, ldx, op.f8_bs, out, ldo, s);
}

// Split-BF16 products for the correction recurrence: (A_hi + A_lo) applied to
// a block stored as X_hi + X_lo (BF16 rounding and residual), lo.lo dropped:
// out (m x b, FP32) = A X (+ coef_j R(:,j)); the _T form computes A^T X.
static rr_status apply_lowp_split(const Op& op, int64_t b, const void* Xh, const void* Xl, int64_t ldx,
                                  void* out, int64_t ldo, const double* R, int64_t ldr, const double* coef,
                                  cudaStream_t s) {
  return gemm_bf16_tc_split(op.m, b, op.n, (const __nv_bfloat16*)op.lo_row, (const __nv_bfloat16*)op.lo2_row,
                            op.n, (const __nv_bfloat16*)Xh, (const __nv_bfloat16*)Xl, ldx, (float*)out, ldo,
                            R, ldr, coef, s);
}
static rr_status apply_lowp_T_split(const Op& op, int64_t b, const void* Xh, const void* Xl, int64_t ldx,
                                    void* out, int64_t ldo, const double* R, int64_t ldr,
                                    const double* coef, cudaStream_t s) {
  return gemm_bf16_tc_split(op.n, b, op.m, (const __nv_bfloat16*)op.lo_col, (const __nv_bfloat16*)op.lo2_col,
                            op.m, (const __nv_bfloat16*)Xh, (const __nv_bfloat16*)Xl, ldx, (float*)out, ldo,
                            R, ldr, coef, s);
}

// FP64-accurate products with the given operator: on the tensor cores by
// error-free slicing when the operator was sliced (mixed precision with
// refinement), otherwise FP64 arithmetic (the all-FP64 mode, CSR operators).
static rr_status apply_f64(const Op& op, int64_t b, const double* X, int64_t ldx, double* out,
                           int64_t ldo, cudaStream_t s) {
  if (op.kind == RR_KERNEL)
    return kernel_apply(s, op.kop, 0, b, RR_F64, X, ldx, RR_F64, out, ldo, nullptr, 0, nullptr);
  if (op.kind == RR_DENSE) {
    if (op.has_emu && b <= 256) return emu_gemm(s, op.emu, 0, b, X, ldx, out, ldo, op.emu_blk);
    return rr_gemm_f64(0, op.m, b, op.n, op.A, op.lda, X, ldx, out, ldo, 0, s);
  }
  return rr_csr_spmm(op.n, b, op.rp, op.ci, op.va, RR_F64, X, ldx, RR_F64, out, ldo, s);
}
static rr_status apply_f64_T(const Op& op, int64_t b, const double* X, int64_t ldx, double* out,
                             int64_t ldo, cudaStream_t s) {
  if (op.kind == RR_KERNEL)
    return kernel_apply(s, op.kop, 1, b, RR_F64, X, ldx, RR_F64, out, ldo, nullptr, 0, nullptr);
  if (op.kind != RR_DENSE) return RR_ERR_ARG;
  if (op.has_emu && op.emu.cols && b <= 256) return emu_gemm(s, op.emu, 1, b, X, ldx, out, ldo, op.emu_blk);
  return rr_gemm_f64(1, op.n, b, op.m, op.A, op.lda, X, ldx, out, ldo, 0, s);
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
struct Common {
  void* hess_ws;
  size_t hess_bytes;
  void* hess_ws2;   // a second Algorithm 8 workspace (for a process running concurrently)
  int32_t* piv2;
  void* gram_ws;
  size_t gram_bytes;
  void* pen_ws;
  size_t pen_bytes;
  int32_t* piv;
  double* scale;  // b
  double* hres;   // unused host mirror placeholder
  int hess_grid;  // 0 = full GPU, 1 = one CTA
  double hess_tol;  // Algorithm 8's skip tolerance (<= 0: the default)
  int pen_b1, pen_b2;  // sizes of the last pencil solved on pen_ws (0: none yet)
};

static void carve_common(Arena& ar, int64_t rows, int64_t b2, int32_t wt, Common& c) {
  // room for the FP64-arithmetic process on b2 columns too (the SVD's FP64
  // polish sweep runs Algorithm 8 in FP64 on b <= b2 columns)
  c.hess_bytes = std::max(rr_hessenberg_workspace_size(rows, b2, wt), rr_hessenberg_workspace_size(rows, b2, RR_F64));
  c.hess_ws = ar.take_bytes(c.hess_bytes);
  c.hess_ws2 = ar.take_bytes(c.hess_bytes);
  c.gram_bytes = rr_gram_workspace_size(rows, b2, b2);
  c.gram_ws = ar.take_bytes(c.gram_bytes);
  c.pen_bytes = rr_pencil_workspace_size(b2, b2);
  c.pen_ws = ar.take_bytes(c.pen_bytes);
  c.piv = ar.take<int32_t>(b2);
  c.piv2 = ar.take<int32_t>(b2);
  c.scale = ar.take<double>(b2);
  c.hess_grid = 0;
  c.hess_tol = 0.0;
  c.pen_b1 = c.pen_b2 = 0;
}

static rr_status basis_step(const Common& c, bool hess, int32_t wt, int32_t dt, int64_t rows,
                            int64_t b, void* W, int64_t ldw, void* Q, int64_t ldq, cudaStream_t s) {
  if (hess)
    return hessenberg_ex(wt, rows, b, W, ldw, dt, Q, ldq, c.piv, c.hess_tol, c.hess_ws, c.hess_bytes, s,
                         c.hess_grid);
  return scale_cast(s, wt, rows, b, W, ldw, c.scale, dt, Q, ldq, nullptr, nullptr);
}

// The same Common with the second Algorithm 8 workspace and pivot array.
static Common second_hess(const Common& c) {
  Common d = c;
  d.hess_ws = c.hess_ws2;
  d.piv = c.piv2;
  return d;
}

static rr_status gram(const Common& c, int64_t n, int64_t p, int64_t q, int32_t xt, const void* X,
                      int64_t ldx, int32_t yt, const void* Y, int64_t ldy, double* G, int64_t ldg,
                      cudaStream_t s) {
  return rr_gram(n, p, q, xt, X, ldx, yt, Y, ldy, G, ldg, 0, c.gram_ws, c.gram_bytes, s);
}

// Remove the span of the orthonormal Ritz vectors X (n x b, their FP32 copy)
// from the FP32 block T (n x b): T <- T - X (X^T T), in FP32 arithmetic (the block is
// stored in BF16 next; FP32 leaves components along X of ~1e-7 relative).
// Keeps the correction blocks of the refinement phase away from the
// converged directions, which the power / Chebyshev steps would otherwise
// amplify until [X, D] is numerically dependent.  K is b x b FP64 scratch.
static rr_status project_out(const Common& c, cudaStream_t s, int64_t n, int64_t b, const float* X,
                             int64_t ldx, float* T, int64_t ldt, double* K) {
  RR_TRY(gram_f32acc(s, n, b, b, X, ldx, T, ldt, K, b, c.gram_ws, c.gram_bytes));
  return sub_lowrank_f32(s, n, b, b, X, ldx, K, b, T, ldt);
}

// Scratch of the tensor-core form of project_out for tall blocks: the Ritz
// vectors as split BF16 pairs, column-major and row-major (taken once per
// sweep), the block T as split BF16 pairs, the FP32 Gram and its split
// pair, the product X K.
struct ProjTc {
  __nv_bfloat16 *Xh = nullptr, *Xl = nullptr, *Xrh = nullptr, *Xrl = nullptr, *Th = nullptr, *Tl = nullptr;
  __nv_bfloat16 *Kh = nullptr, *Kl = nullptr;
  float *K32 = nullptr, *P = nullptr;
};

// Tall blocks (n >= 65536, n a multiple of 8, b <= 256) of a BF16 basis: both
// products of the projection on the tensor cores from split BF16 operands
// (X = X_hi + X_lo, T = T_hi + T_lo, K likewise; the lo.lo products dropped:
// about 2^-16 relative, against FP32's 2^-24 with the FP32-pipe kernels at
// more than twice the time): K = X^T T, then P = X K and T -= P.  The block
// is stored in BF16 right after the projection, so components along X at
// 1e-5 of the block are far below its own rounding.
static bool proj_tc_applies(int64_t n, int64_t b) { return n >= 65536 && n % 8 == 0 && b <= 256; }

// The split pairs of the Ritz vectors X (n x b, FP64) in both layouts.
static rr_status proj_tc_prepare(const ProjTc& pt, cudaStream_t s, int64_t n, int64_t b, const double* X,
                                 int64_t ldx) {
  RR_TRY(scale_split(s, RR_F64, n, b, X, ldx, nullptr, pt.Xh, pt.Xl, n, nullptr, nullptr));
  RR_TRY(block_to_rows(s, RR_BF16, n, b, b, pt.Xh, n, pt.Xrh, b));
  return block_to_rows(s, RR_BF16, n, b, b, pt.Xl, n, pt.Xrl, b);
}

static rr_status project_out_tc(const ProjTc& pt, cudaStream_t s, int64_t n, int64_t b, float* T, int64_t ldt) {
  RR_TRY(scale_split(s, RR_F32, n, b, T, ldt, nullptr, pt.Th, pt.Tl, n, nullptr, nullptr));
  RR_TRY(gemm_bf16_tc_split(b, b, n, pt.Xh, pt.Xl, n, pt.Th, pt.Tl, n, pt.K32, b, nullptr, 0, nullptr, s));
  RR_TRY(scale_split(s, RR_F32, b, b, pt.K32, b, nullptr, pt.Kh, pt.Kl, b, nullptr, nullptr));
  RR_TRY(gemm_bf16_tc_split(n, b, b, pt.Xrh, pt.Xrl, b, pt.Kh, pt.Kl, b, pt.P, n, nullptr, 0, nullptr, s));
  return sub_block_f32(s, n, b, pt.P, n, T, ldt);
}

// Pencil solves that record which sizes ran, so the condition estimate of
// the last one can be found in the pencil workspace.
static rr_status pencil_svd(Common& c, int64_t b1, int64_t b2, const double* B, const double* Gu,
                            const double* Gv, double* s_, double* Y, double* Z, cudaStream_t s) {
  c.pen_b1 = (int)b1;
  c.pen_b2 = (int)b2;
  return rr_pencil_svd(b1, b2, B, Gu, Gv, s_, Y, Z, c.pen_ws, c.pen_bytes, nullptr, s);
}
static rr_status pencil_eig(Common& c, int64_t b, const double* H, const double* G, double* th,
                            double* Y, cudaStream_t s) {
  c.pen_b1 = c.pen_b2 = (int)b;
  return rr_pencil_eig(b, H, G, th, Y, c.pen_ws, c.pen_bytes, nullptr, s);
}
// Queue the copy of the last pencil's condition estimates and drop counts
// (4 doubles) into host memory (valid after the next stream synchronisation).
static rr_status queue_cond(const Common& c, cudaStream_t s, double* host4) {
  host4[0] = host4[1] = host4[2] = host4[3] = 0.0;
  if (!c.pen_b1) return RR_OK;
  const double* d = pencil_cond_slot(c.pen_ws, c.pen_bytes, c.pen_b1, c.pen_b2);
  if (!d) return RR_OK;
  RR_CUDA(cudaMemcpyAsync(host4, d, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  return RR_OK;
}
static void note_cond(rr_info& inf, int sweep, const double* host4) {
  const double c = fmax(host4[0], host4[1]);
  inf.cond_G_est = c;
  inf.cols_dropped = (int32_t)(host4[2] + host4[3]);
  if (sweep >= 1 && sweep <= 64) inf.cond_history[sweep - 1] = c;
}
// every one of the k wanted residuals is NaN: a NaN or infinity in the
// operator (or a basis that collapsed entirely)
static bool all_nan(const double* res, int k) {
  for (int i = 0; i < k; ++i)
    if (!std::isnan(res[i])) return false;
  return k > 0;
}

// An operator with a NaN or infinity makes every later quantity NaN and
// gives the data-dependent steps (argmax, sorts, cluster detection) no
// meaningful input: check the values once, before the first product, and
// stop with RR_ERR_NAN.  One read of the operator and one synchronisation.
static rr_status check_operator_finite(const rr_operator* A, const Common& c, cudaStream_t s) {
  RR_CUDA(cudaMemsetAsync(c.piv, 0, sizeof(int), s));
  if (A->kind == RR_KERNEL) {
    // the points of both sides (m x d, n x d)
    RR_TRY(operator_nonfinite(s, RR_DENSE, A->m, A->nnz, A->values, A->ld, 0, c.piv));
    if (A->points_y) RR_TRY(operator_nonfinite(s, RR_DENSE, A->n, A->nnz, A->points_y, A->n, 0, c.piv));
  } else {
    const int64_t m = A->kind == RR_DENSE ? A->m : A->n;
    RR_TRY(operator_nonfinite(s, A->kind, m, A->n, A->values, A->ld, A->nnz, c.piv));
  }
  int h = 0;
  RR_CUDA(cudaMemcpyAsync(&h, c.piv, sizeof(int), cudaMemcpyDeviceToHost, s));
  RR_CUDA(cudaStreamSynchronize(s));
  return h ? RR_ERR_NAN : RR_OK;
}

static int count_converged(const double* res, int k, double tol, double* maxres) {
  int n = 0;
  double mx = 0.0;
  for (int i = 0; i < k; ++i) {
    if (res[i] <= tol) ++n;
    mx = std::isnan(res[i]) ? INFINITY : fmax(mx, res[i]);
  }
  *maxres = mx;
  return n;
}

static rr_status read_err(const Common& c, cudaStream_t s) {
  int e = 0, e2 = 0;
  RR_CUDA(cudaMemcpyAsync(&e, c.hess_ws, sizeof(int), cudaMemcpyDeviceToHost, s));
  RR_CUDA(cudaMemcpyAsync(&e2, c.hess_ws2, sizeof(int), cudaMemcpyDeviceToHost, s));
  RR_CUDA(cudaStreamSynchronize(s));
  if (e) return (rr_status)e;
  if (e2) return (rr_status)e2;
  return tc_take_error(s);
}

static rr_status check_params(const rr_params* p, int64_t rows_min) {
  if (!p) return RR_ERR_ARG;
  if (p->k <= 0 || p->block < p->k || p->block > rows_min || p->block > 1024) return RR_ERR_ARG;
  if (p->degree <= 0 || p->max_sweeps <= 0 || p->max_sweeps > 10000) return RR_ERR_ARG;
  if (p->basis != RR_F64 && p->basis != RR_F32 && p->basis != RR_BF16 && p->basis != RR_E4M3) return RR_ERR_ARG;
  // the projected pencil (2 block with refinement) must fit the small solver
  const bool refine = p->refine != 0 && p->basis != RR_F64;
  if ((refine ? 2 * p->block : p->block) > 335) return RR_ERR_ARG;
  return RR_OK;
}

// ===========================================================================
// SVD (Algorithm 5 with Algorithm 1/8 and the refinement phase)
// ===========================================================================
struct SvdBufs {
  Common c;
  void *Ulo, *Vlo, *W, *Pw, *Elo, *Flo, *AF;
  double *Gu, *Gv, *Bm, *Ys, *Zs, *sig2;
  double *Ut, *Vt, *Ut2, *Vt2, *sig, *P, *Qm, *Rv, *Ru, *ss, *res, *mu, *coef;
  // split mode: lo halves of the correction blocks, FP32 final blocks
  void *Elo2, *Flo2, *E32, *F32;
  float *Ut32, *Vt32;  // FP32 copies of the singular vectors for the refinement's projections
  // batch mode: [0] the problem reached tol (frozen), [1] sweeps done, [2]
  // FP64 polish sweeps done, [4..5] the previous sweep's largest residual
  // (a double; device-side loop control)
  int* frozen;
};

static void carve_svd(Arena& ar, const Op& op, int64_t b, bool refine, SvdBufs& w) {
  const int64_t m = op.m, n = op.n, mx = m > n ? m : n, b2 = refine ? 2 * b : b;
  const size_t ds = dsz(op.dt), ws_ = dsz(op.wt);
  carve_common(ar, mx, b2, op.wt, w.c);
  w.Ulo = ar.take_bytes(m * b * ds);
  w.Vlo = ar.take_bytes(n * b * ds);
  w.W = ar.take_bytes(mx * b * ws_);
  w.Pw = ar.take_bytes(m * b * ws_);
  w.Gu = ar.take<double>(b2 * b2);
  w.Gv = ar.take<double>(b2 * b2);
  w.Bm = ar.take<double>(b2 * b2);
  w.Ys = ar.take<double>(b2 * b2);
  w.Zs = ar.take<double>(b2 * b2);
  w.sig2 = ar.take<double>(b2);
  w.Ut = ar.take<double>(m * b);
  w.Vt = ar.take<double>(n * b);
  w.frozen = ar.take<int>(8);
  w.sig = ar.take<double>(b);
  w.P = ar.take<double>(m * b);
  w.Qm = ar.take<double>(n * b);
  w.ss = ar.take<double>(b);
  w.res = ar.take<double>(b);
  if (refine) {
    w.Ut2 = ar.take<double>(m * b);
    w.Vt2 = ar.take<double>(n * b);
    w.Rv = ar.take<double>(m * b);
    w.Ru = ar.take<double>(n * b);
    w.Elo = ar.take_bytes(m * b * ds);
    w.Flo = ar.take_bytes(n * b * ds);
    w.AF = ar.take_bytes(m * b * ws_);
    w.mu = ar.take<double>(b);
    w.coef = ar.take<double>(b);
    w.Ut32 = ar.take<float>(m * b);
    w.Vt32 = ar.take<float>(n * b);
  } else {
    w.Ut2 = w.Vt2 = w.Rv = w.Ru = w.mu = w.coef = nullptr;
    w.Elo = w.Flo = w.AF = nullptr;
    w.Ut32 = w.Vt32 = nullptr;
  }
  w.Elo2 = w.Flo2 = w.E32 = w.F32 = nullptr;
  if (refine && op.split) {
    w.Elo2 = ar.take_bytes(m * b * 2);
    w.Flo2 = ar.take_bytes(n * b * 2);
    w.E32 = ar.take_bytes(m * b * 4);
    w.F32 = ar.take_bytes(n * b * 4);
  }
}

static void make_op(const rr_operator* A, int32_t basis, Op& op) {
  const int32_t dt = basis == RR_E4M3 ? RR_BF16 : basis;
  op.f8 = basis == RR_E4M3;
  op.f8_row = op.f8_col = op.f8_scratch = nullptr;
  op.f8_rs = op.f8_cs = op.f8_bs = nullptr;
  op.f8_ldr = op.f8_ldc = 0;
  op.kind = A->kind;
  op.kop = A;
  op.m = A->kind == RR_CSR ? A->n : A->m;
  op.n = A->n;
  op.A = (const double*)A->values;
  op.lda = A->ld;
  op.rp = A->row_ptr;
  op.ci = A->col_idx;
  op.va = (const float*)A->values;
  op.lo_col = op.lo_row = nullptr;
  op.split = false;
  op.lo2_col = op.lo2_row = nullptr;
  op.dt = dt;
  op.wt = dt == RR_F64 ? RR_F64 : RR_F32;
  op.has_emu = false;
  op.emu_mem = op.emu_blk = nullptr;
  op.lift_mem = nullptr;
  op.lift_bytes = 0;
}

// The operator copies live at the front of the workspace: the low-precision
// copies for the filter and, with refinement, the BF16 slices of the FP64
// operator for the FP64-accurate products (row-scaled for A X, and
// column-scaled for A^T Y when the operator is not symmetric).
static void carve_op(Arena& ar, Op& op, bool symmetric, bool refine, int64_t b) {
  if (op.dt != RR_F64 && b <= 256) {
    // lifts of up to 2b columns ([X, D] Y in the refinement)
    op.lift_bytes = lift_emu_bytes(op.m > op.n ? op.m : op.n, b, 2 * b);
    op.lift_mem = ar.take_bytes(op.lift_bytes);
  }
  if (op.kind != RR_DENSE || op.dt == RR_F64) return;
  if (op.f8) {
    op.f8_ldr = (op.n + 15) / 16 * 16;
    op.f8_ldc = (op.m + 15) / 16 * 16;
    op.f8_row = ar.take_bytes(op.m * op.f8_ldr);
    op.f8_col = ar.take_bytes(op.n * op.f8_ldc);
    op.f8_rs = ar.take<float>(op.m);
    op.f8_cs = ar.take<float>(op.n);
    op.f8_bs = ar.take<float>(b);
    op.f8_scratch = ar.take<uint64_t>(op.m > op.n ? op.m : op.n);
  }
  op.lo_col = ar.take_bytes(op.m * op.n * dsz(op.dt));
  op.lo_row = symmetric ? op.lo_col : ar.take_bytes(op.m * op.n * dsz(op.dt));
  if (refine && !symmetric && op.dt == RR_BF16 && op.m % 8 == 0 && op.n % 8 == 0 && b <= 256) {
    op.split = true;
    op.lo2_col = ar.take_bytes(op.m * op.n * 2);
    op.lo2_row = symmetric ? op.lo2_col : ar.take_bytes(op.m * op.n * 2);
  }
  if (refine && op.m % 8 == 0 && op.n % 8 == 0 && b <= 256) {
    op.has_emu = true;
    op.emu_mem = ar.take_bytes(emu_operator_bytes(op.m, op.n, kEmuSlices, true, !symmetric));
    op.emu_blk = ar.take_bytes(emu_block_bytes(op.m > op.n ? op.m : op.n, b, kEmuSlices));
  }
}

static rr_status prepare_f8(const Op& op, int64_t b, cudaStream_t s) {
  RR_TRY(rr_quantize_e4m3(op.m, op.n, op.A, op.lda, 1, op.f8_row, op.f8_ldr, op.f8_rs, op.f8_scratch, s));
  RR_TRY(rr_quantize_e4m3(op.m, op.n, op.A, op.lda, 0, op.f8_col, op.f8_ldc, op.f8_cs, op.f8_scratch, s));
  return fill_f32(s, b, 1.0f / 256.0f, op.f8_bs);
}

static rr_status prepare_op(const Op& op_in, Op& op, bool symmetric, cudaStream_t s) {
  (void)op_in;
  if (op.kind == RR_DENSE && op.dt == RR_BF16 && op.lo_col && (!op.has_emu || kEmuSlices == 8)) {
    // every copy and slice of the operator from two passes over A
    return op_prepare(s, op.A, op.m, op.n, op.lda, (__nv_bfloat16*)op.lo_col,
                      symmetric ? nullptr : (__nv_bfloat16*)op.lo_row,
                      op.split ? (__nv_bfloat16*)op.lo2_col : nullptr,
                      op.split && !symmetric ? (__nv_bfloat16*)op.lo2_row : nullptr, kEmuSlices,
                      op.has_emu ? &op.emu : nullptr, op.emu_mem, true, !symmetric);
  }
  if (op.lo_col)
    RR_TRY(rr_cast_operator(op.m, op.n, op.A, op.lda, op.dt, op.lo_col, symmetric ? nullptr : op.lo_row, s));
  if (op.split) RR_TRY(cast_operator_lo(op.m, op.n, op.A, op.lda, op.lo2_col, op.lo2_row, s));
  if (op.has_emu)
    RR_TRY(emu_prepare(s, op.A, op.m, op.n, op.lda, kEmuSlices, op.emu, op.emu_mem, true, !symmetric));
  return RR_OK;
}

// X (n x b, FP64) = S1 Y(0:p1, :) + S2 Y(p1:p1+p2, :) (S2 may be null): the
// FP64-accurate tensor-core lift when the shape allows, else FP64 arithmetic
static rr_status lift2(const Op& op, cudaStream_t s, int64_t n, int64_t b, int32_t t1, const void* S1, int64_t ld1,
                       int64_t p1, int32_t t2, const void* S2, int64_t ld2, int64_t p2, const double* Y, int64_t ldy,
                       double* X, int64_t ldx) {
  bool done = false;
  RR_TRY(lift_emu(s, n, b, t1, S1, ld1, p1, t2, S2, ld2, p2, Y, ldy, X, ldx, op.lift_mem, op.lift_bytes, &done));
  if (done) return RR_OK;
  RR_TRY(lift(s, t1, n, b, p1, S1, ld1, Y, ldy, X, ldx, 0));
  if (S2 && p2 > 0) RR_TRY(lift(s, t2, n, b, p2, S2, ld2, Y + p1, ldy, X, ldx, 1));
  return RR_OK;
}

// FP64 residual of the first kk triplets: res = sqrt(|A v - s u|^2 + |A^T u - s v|^2) / s
static rr_status svd_residual(const Op& op, SvdBufs& w, int64_t kk, double* R1, double* R2,
                              cudaStream_t s) {
  const int64_t m = op.m, n = op.n;
  RR_TRY(apply_f64(op, kk, w.Vt, n, w.P, m, s));
  RR_TRY(apply_f64_T(op, kk, w.Ut, m, w.Qm, n, s));
  RR_TRY(residual_block(s, m, kk, w.P, m, w.Ut, m, w.sig, R1, m, w.ss, 0));
  RR_TRY(residual_block(s, n, kk, w.Qm, n, w.Vt, n, w.sig, R2, n, w.ss, 1));
  return res_finish(s, kk, w.ss, w.sig, w.res);
}

// Dense operators in the mixed-precision path are solved zero-padded to a
// multiple of 8 rows and columns (16 for the E4M3 basis): the tensor-core
// products, the split-BF16 corrections and the FP64-emulated products need
// strides in whole 16-byte vectors.  Zero rows and columns add only zero
// singular values, and the iteration keeps the padded entries of every
// basis exactly zero after the first product (A's zero columns and rows
// contribute exact zeros), so the top triplets are those of A with the
// padded entries of u and v equal to zero.
static int svd_pad_quantum(const rr_operator* A, const rr_params* p) {
  if (A->kind != RR_DENSE || p->basis == RR_F64) return 0;
  const int q = p->basis == RR_E4M3 ? 16 : 8;
  return (A->m % q || A->n % q) ? q : 0;
}

// The FP64 polish of the refinement phase: one correction sweep carried in
// FP64-accurate arithmetic (FP64 blocks, FP64-accurate products, Algorithm 8
// in FP64 arithmetic) from the residual blocks of the current triplets:
//   F = A^T R_v + R_u Sigma    (= A^T A V~ - V~ Sigma^2),
//   E = A F + R_v Sigma^2      (= A A^T A V~ - U~ Sigma^3),
// each scaled to unit column inf-norm and projected against the orthonormal
// V~ / U~ (F <- F - V~ (V~^T F), FP64-accurate: exactly, R_v and R_u are
// orthogonal to U~ and V~, but their rounding noise is not, and relative to a
// residual of 1e-11 it would leave S_u = [U~, E] with a Gram condition of
// 1e11 and more), then Algorithm 8, Algorithm 5 over S_u = [U~, E],
// S_v = [V~, F] and the lift into (Ut2, Vt2, sig2).  The low-precision
// corrections stop improving at a level set by their precision and the
// ratio of the largest to the smallest wanted singular value (near 2e-10 for
// sigma_j = j^-1.5 with 16 wanted); this sweep contracts to the FP64
// rounding level (about 1e-14 there, against 1e-11 to 1e-10 for the paper's
// method run in FP64).  Needs P = A V~, Q = A^T U~, R_v, R_u from the
// residual check before it; overwrites R_v, R_u, P, Q and the pencil blocks.
static rr_status svd_polish_f64(const Op& op, SvdBufs& w, int64_t b, cudaStream_t s, Prof& prof) {
  const int64_t m = op.m, n = op.n, b2 = 2 * b;
  double* F0 = w.Vt2;  // n x b
  double* E0 = w.Ut2;  // m x b
  STAGE(RR_STAGE_F64_PRODUCT, apply_f64_T(op, b, w.Rv, m, F0, n, s));         // A^T R_v
  STAGE(RR_STAGE_OTHER, add_cols_scaled(s, n, b, w.Ru, n, w.sig, 1, F0, n));   // + R_u Sigma
  STAGE(RR_STAGE_F64_PRODUCT, apply_f64(op, b, F0, n, E0, m, s));               // A F
  STAGE(RR_STAGE_OTHER, add_cols_scaled(s, m, b, w.Rv, m, w.sig, 2, E0, m));   // + R_v Sigma^2
  // unit inf-norm columns (R_v and R_u are free now), then the projections:
  // [T, X] [I; -X^T T] = T - X (X^T T) by the FP64-accurate lift
  double* Fs = w.Ru;
  double* Es = w.Rv;
  STAGE(RR_STAGE_OTHER, scale_cast(s, RR_F64, n, b, F0, n, w.mu, RR_F64, Fs, n, nullptr, nullptr));
  STAGE(RR_STAGE_OTHER, scale_cast(s, RR_F64, m, b, E0, m, w.mu, RR_F64, Es, m, nullptr, nullptr));
  STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, w.Vt, n, RR_F64, Fs, n, w.Ys, b, s));
  STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, RR_F64, w.Ut, m, RR_F64, Es, m, w.Zs, b, s));
  STAGE(RR_STAGE_OTHER, eye_neg(s, b, w.Ys, b, w.Gv, b2));
  STAGE(RR_STAGE_OTHER, eye_neg(s, b, w.Zs, b, w.Gu, b2));
  double* F = w.Vt2;
  double* E = w.Ut2;
  STAGE(RR_STAGE_LIFT, lift2(op, s, n, b, RR_F64, Fs, n, b, RR_F64, w.Vt, n, b, w.Gv, b2, F, n));
  STAGE(RR_STAGE_LIFT, lift2(op, s, m, b, RR_F64, Es, m, b, RR_F64, w.Ut, m, b, w.Gu, b2, E, m));
  STAGE(RR_STAGE_HESSENBERG, basis_step(w.c, true, RR_F64, RR_F64, m, b, E, m, E, m, s));
  STAGE(RR_STAGE_HESSENBERG, basis_step(w.c, true, RR_F64, RR_F64, n, b, F, n, F, n, s));
  double* AF = w.Rv;
  STAGE(RR_STAGE_F64_PRODUCT, apply_f64(op, b, F, n, AF, m, s));                // A F of the basis
  // projected blocks over S_u = [U~, E], S_v = [V~, F]  (ld 2b)
  double* B = w.Bm;
  STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, RR_F64, w.Ut, m, RR_F64, w.P, m, B, b2, s));             // U~^T A V~
  STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, w.Qm, n, RR_F64, F, n, B + b * b2, b2, s));      // U~^T A F
  STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, RR_F64, E, m, RR_F64, w.P, m, B + b, b2, s));            // E^T A V~
  STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, RR_F64, E, m, RR_F64, AF, m, B + b + b * b2, b2, s));    // E^T A F
  STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, RR_F64, w.Ut, m, RR_F64, w.Ut, m, w.Gu, b2, s));
  STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, RR_F64, w.Ut, m, RR_F64, E, m, w.Gu + b * b2, b2, s));
  STAGE(RR_STAGE_OTHER, transpose(s, b, b, w.Gu + b * b2, b2, w.Gu + b, b2));
  STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, RR_F64, E, m, RR_F64, E, m, w.Gu + b + b * b2, b2, s));
  STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, w.Vt, n, RR_F64, w.Vt, n, w.Gv, b2, s));
  STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, w.Vt, n, RR_F64, F, n, w.Gv + b * b2, b2, s));
  STAGE(RR_STAGE_OTHER, transpose(s, b, b, w.Gv + b * b2, b2, w.Gv + b, b2));
  STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, F, n, RR_F64, F, n, w.Gv + b + b * b2, b2, s));
  STAGE(RR_STAGE_PENCIL, pencil_svd(w.c, b2, b2, B, w.Gu, w.Gv, w.sig2, w.Ys, w.Zs, s));
  // lift the leading b triplets (into P and Q, which the blocks above no
  // longer need), then into the sweep's outputs
  STAGE(RR_STAGE_LIFT, lift2(op, s, m, b, RR_F64, w.Ut, m, b, RR_F64, E, m, b, w.Ys, b2, w.P, m));
  STAGE(RR_STAGE_LIFT, lift2(op, s, n, b, RR_F64, w.Vt, n, b, RR_F64, F, n, b, w.Zs, b2, w.Qm, n));
  RR_CUDA(cudaMemcpyAsync(w.Ut2, w.P, (size_t)m * b * sizeof(double), cudaMemcpyDeviceToDevice, s));
  RR_CUDA(cudaMemcpyAsync(w.Vt2, w.Qm, (size_t)n * b * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return RR_OK;
}

// Device-side loop of the batched solver.  At this point of the capture on
// `outer` a WHILE node is added whose body, captured on `body_s` (a stream
// that is not capturing), is `body(body_s)` followed by the loop-control
// kernel: sweeps repeat on the GPU while the problem is not frozen and its
// sweep count is below max_sweeps (and below stop_at when stop_at >= 0) and,
// with stall != 0, while the largest of the k residuals res keeps falling
// below 0.3 times the previous sweep's.  ctl = [frozen, sweeps, polish
// sweeps, -, previous largest residual (double)]; before the node, inc_first
// sweeps are added to the count and the condition is set for the first
// iteration; each iteration adds one sweep (and one polish sweep when
// polish != 0).
template <class F>
static rr_status device_loop(cudaStream_t outer, cudaStream_t body_s, int* ctl, int max_sweeps, int stop_at,
                             int inc_first, int polish, const double* res, int k, int stall, F&& body) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  RR_CUDA(cudaStreamGetCaptureInfo(outer, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive || !g) return RR_ERR_ARG;
  cudaGraphConditionalHandle h;
  RR_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  RR_TRY(loop_ctl(outer, h, ctl, inc_first, 0, max_sweeps, stop_at, res, k, 0));
  RR_CUDA(cudaStreamGetCaptureInfo(outer, &cs, nullptr, &g, &deps, &ed, &nd));
  // (a union with members that have no default constructor: zeroed storage)
  alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
  memset(npbuf, 0, sizeof(npbuf));
  cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(npbuf);
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  RR_CUDA(cudaGraphAddNode(&node, g, deps, ed, nd, &np));
  RR_CUDA(cudaStreamUpdateCaptureDependencies(outer, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  RR_CUDA(cudaStreamBeginCaptureToGraph(body_s, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal));
  rr_status st = body(body_s);
  if (st == RR_OK) st = loop_ctl(body_s, h, ctl, 1, polish, max_sweeps, stop_at, res, k, stall);
  cudaGraph_t bg = nullptr;
  const cudaError_t e = cudaStreamEndCapture(body_s, &bg);  // the body graph stays owned by the node
  if (st == RR_OK && e != cudaSuccess) {
    set_last_error("device_loop end capture", e);
    st = RR_ERR_CUDA;
  }
  return st;
}

// The padded operator of a problem (svd_pad_quantum) and, when padding, its
// buffer taken from the front of the workspace: every user of a problem's
// workspace layout (the solve, its size query, the batch's read-back) carves
// it the same way.
static const rr_operator* svd_operator(const rr_operator* A_in, const rr_params* p, Arena& ar,
                                       rr_operator& Apad, double** Abuf) {
  const int padq = svd_pad_quantum(A_in, p);
  Apad = *A_in;
  if (Abuf) *Abuf = nullptr;
  if (!padq) return A_in;
  Apad.m = (A_in->m + padq - 1) / padq * padq;
  Apad.n = (A_in->n + padq - 1) / padq * padq;
  Apad.ld = Apad.m;
  double* buf = ar.take<double>(Apad.m * Apad.n);
  Apad.values = buf;
  if (Abuf) *Abuf = buf;
  return &Apad;
}

static rr_status svd_run(const rr_operator* Aop_in, const rr_params* p, double* sigma_out,
                         double* U_out, double* V_out, void* ws, size_t ws_bytes, rr_info* info,
                         cudaStream_t s, bool batch_mode, int hess_grid, uint64_t seed,
                         cudaStream_t body_s) {
  Arena ar(ws, ws_bytes);
  const int64_t m0 = Aop_in->m, n0 = Aop_in->n;
  const int padq = svd_pad_quantum(Aop_in, p);
  rr_operator Apad;
  double* Abuf = nullptr;
  const rr_operator* Aop = svd_operator(Aop_in, p, ar, Apad, &Abuf);
  Op op;
  make_op(Aop, p->basis, op);
  const int32_t dt = op.dt;                 // refinement blocks (BF16 for an E4M3 basis)
  const int32_t dt1 = p->basis;             // phase-1 basis
  if (op.f8 && (batch_mode || op.m % 16 || op.n % 16)) return RR_ERR_ARG;
  const int64_t m = op.m, n = op.n, b = p->block, k = p->k;
  const int q = p->degree;
  const int qr = p->refine_degree > 0 ? p->refine_degree : q;  // products per refinement sweep
  const bool hess = p->hessenberg != 0;
  const bool refine = p->refine != 0 && dt != RR_F64;
  const int ph1 = refine ? (p->phase1_sweeps > 0 ? p->phase1_sweeps : 1) : p->max_sweeps;
  carve_op(ar, op, false, refine, b);
  SvdBufs w;
  carve_svd(ar, op, b, refine, w);
  double* v0buf = (batch_mode || !p->v0 || padq) ? ar.take<double>(n * b) : nullptr;
  if (ar.overflow) return RR_ERR_WORKSPACE;
  Prof prof;
  prof.on = p->profile != 0 && !batch_mode;
  prof.s = s;
  prof.start();
  w.c.hess_grid = hess_grid;
  w.c.hess_tol = p->hess_tol;
  RR_CUDA(cudaMemsetAsync(w.c.hess_ws, 0, 512, s));
  RR_CUDA(cudaMemsetAsync(w.c.hess_ws2, 0, 512, s));
  RR_CUDA(cudaMemsetAsync(w.frozen, 0, 8 * sizeof(int), s));
  if (!batch_mode) STAGE(RR_STAGE_OTHER, check_operator_finite(Aop_in, w.c, s));
  if (padq) {
    // the zero-padded copy of A (counted with the one-time operator casts)
    RR_CUDA(cudaMemsetAsync(Abuf, 0, (size_t)m * n * sizeof(double), s));
    RR_CUDA(cudaMemcpy2DAsync(Abuf, m * sizeof(double), Aop_in->values, Aop_in->ld * sizeof(double),
                              m0 * sizeof(double), n0, cudaMemcpyDeviceToDevice, s));
  }

  // one-time operator casts and slicing (counted in the solve time)
  STAGE(RR_STAGE_OTHER, prepare_op(op, op, false, s));
  if (op.f8) STAGE(RR_STAGE_OTHER, prepare_f8(op, b, s));

  // a1: start block
  const double* v0 = p->v0;
  if (batch_mode || !v0) {
    STAGE(RR_STAGE_OTHER, uniform_block(s, n, b, batch_mode ? seed : p->seed, v0buf, n));
    v0 = v0buf;
  } else if (padq) {
    // the caller's n0 x b start block with zero rows up to n
    RR_CUDA(cudaMemsetAsync(v0buf, 0, (size_t)n * b * sizeof(double), s));
    RR_CUDA(cudaMemcpy2DAsync(v0buf, n * sizeof(double), v0, n0 * sizeof(double), n0 * sizeof(double), b,
                              cudaMemcpyDeviceToDevice, s));
    v0 = v0buf;
  }
  STAGE(RR_STAGE_OTHER, rr_colscale_cast(n, b, v0, n, dt1, w.Vlo, n, w.c.scale, s));

  rr_info inf;
  memset(&inf, 0, sizeof(inf));
  std::vector<double> hres(b);
  double hcond[4] = {0.0, 0.0, 0.0, 0.0};
  int sweep = 0;
  bool converged = false, nan_seen = false;

  // ---------------- phase 1: the paper's method ----------------
  // One sweep: q times { U = Alg. 8(A V), V = Alg. 8(A^T U) }, then
  // Algorithm 5 over (U, V) and the lift into (Ut, Vt, sig); `recast` starts
  // from the previous sweep's Ritz vectors.
  auto ph1_sweep = [&](cudaStream_t s, bool recast) -> rr_status {
    if (recast) STAGE(RR_STAGE_OTHER, rr_colscale_cast(n, b, w.Vt, n, dt1, w.Vlo, n, w.c.scale, s));
    for (int it = 0; it < q; ++it) {
      STAGE(RR_STAGE_LOWP_PRODUCT, apply_ph1(op, b, w.Vlo, n, (float*)w.W, m, s));                      // W = A V
      STAGE(RR_STAGE_HESSENBERG, basis_step(w.c, hess, op.wt, dt1, m, b, w.W, m, w.Ulo, m, s));         // U = basis(W)
      STAGE(RR_STAGE_LOWP_PRODUCT, apply_ph1_T(op, b, w.Ulo, m, (float*)w.W, n, s));                    // Z = A^T U
      STAGE(RR_STAGE_HESSENBERG, basis_step(w.c, hess, op.wt, dt1, n, b, w.W, n, w.Vlo, n, s));         // V = basis(Z)
    }
    // Algorithm 5: B = U^T (A V), Gu = U^T U, Gv = V^T V (FP64 accumulation)
    STAGE(RR_STAGE_LOWP_PRODUCT, apply_ph1(op, b, w.Vlo, n, (float*)w.Pw, m, s));
    STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, dt1, w.Ulo, m, dt1, w.Ulo, m, w.Gu, b, s));
    STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, dt1, w.Vlo, n, dt1, w.Vlo, n, w.Gv, b, s));
    STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, dt1, w.Ulo, m, op.wt, w.Pw, m, w.Bm, b, s));
    STAGE(RR_STAGE_PENCIL, pencil_svd(w.c, b, b, w.Bm, w.Gu, w.Gv, w.sig2, w.Ys, w.Zs, s));
    STAGE(RR_STAGE_LIFT, lift2(op, s, m, b, dt1, w.Ulo, m, b, 0, nullptr, 0, 0, w.Ys, b, w.Ut, m));
    STAGE(RR_STAGE_LIFT, lift2(op, s, n, b, dt1, w.Vlo, n, b, 0, nullptr, 0, 0, w.Zs, b, w.Vt, n));
    RR_CUDA(cudaMemcpyAsync(w.sig, w.sig2, b * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return RR_OK;
  };
  // batched problems: sweeps after the first run in WHILE nodes of the graph
  // (device-side loop control), each problem stopping at tol
  const bool dloop = batch_mode && body_s != nullptr;

  if (dloop && !refine) {
    // the plain method in a batch: the residual check after every sweep
    RR_TRY(ph1_sweep(s, false));
    ++sweep;
    STAGE(RR_STAGE_F64_PRODUCT, svd_residual(op, w, k, w.P, w.Qm, s));
    STAGE(RR_STAGE_OTHER, freeze_update(s, k, w.res, p->tol, w.frozen));
    RR_TRY(device_loop(s, body_s, w.frozen, p->max_sweeps, -1, sweep, 0, w.res, (int)k, 0,
                       [&](cudaStream_t bs) -> rr_status {
      RR_TRY(ph1_sweep(bs, true));
      RR_TRY(svd_residual(op, w, k, w.P, w.Qm, bs));
      return freeze_update(bs, k, w.res, p->tol, w.frozen);
    }));
  } else {
    for (int ps = 0; ps < ph1 && sweep < p->max_sweeps; ++ps) {
      RR_TRY(ph1_sweep(s, ps > 0));
      ++sweep;
      if (!refine && !batch_mode) {
        // plain method: FP64 residual check of the wanted triplets every sweep
        STAGE(RR_STAGE_F64_PRODUCT, svd_residual(op, w, k, w.Rv ? w.Rv : w.P, w.Ru ? w.Ru : w.Qm, s));
        RR_CUDA(cudaMemcpyAsync(hres.data(), w.res, k * sizeof(double), cudaMemcpyDeviceToHost, s));
        RR_TRY(queue_cond(w.c, s, hcond));
        RR_CUDA(cudaStreamSynchronize(s));
        RR_TRY(read_err(w.c, s));
        double mx;
        inf.n_converged = count_converged(hres.data(), (int)k, p->tol, &mx);
        inf.max_res = mx;
        if (sweep <= 64) inf.res_history[sweep - 1] = mx;
        note_cond(inf, sweep, hcond);
        if (all_nan(hres.data(), (int)k)) {
          nan_seen = true;
          break;
        }
        if (inf.n_converged == k) {
          converged = true;
          break;
        }
      }
    }
  }

  // ---------------- phase 2: refinement ----------------
  // residual of all b Ritz triplets, FP64-accurate (P, Q, R_v, R_u, res)
  auto residual_all = [&](cudaStream_t s) -> rr_status {
    STAGE(RR_STAGE_F64_PRODUCT, apply_f64(op, b, w.Vt, n, w.P, m, s));      // P = A V~
    STAGE(RR_STAGE_F64_PRODUCT, apply_f64_T(op, b, w.Ut, m, w.Qm, n, s));   // Q = A^T U~
    STAGE(RR_STAGE_OTHER, residual_block(s, m, b, w.P, m, w.Ut, m, w.sig, w.Rv, m, w.ss, 0));
    STAGE(RR_STAGE_OTHER, residual_block(s, n, b, w.Qm, n, w.Vt, n, w.sig, w.Ru, n, w.ss, 1));
    STAGE(RR_STAGE_OTHER, res_finish(s, b, w.ss, w.sig, w.res));
    if (batch_mode) STAGE(RR_STAGE_OTHER, freeze_update(s, k, w.res, p->tol, w.frozen));
    return RR_OK;
  };
  // One refinement sweep from the residual blocks into (Ut2, Vt2, sig2).
  auto corr_sweep = [&](cudaStream_t s) -> rr_status {
    const int64_t b2 = 2 * b;
    // correction recurrence (low precision):
    //   E_1 = R_v;  F_j = A^T E_j + R_u S^(2j-1);  E_{j+1} = A F_j + R_v S^(2j)
    // each block kept at unit column inf-norm, the injection coefficient
    // tracked per column (coef <- coef * sigma / mu after each scaling).
    STAGE(RR_STAGE_OTHER, fill(s, b, 1.0, w.coef));
    // FP32 copies of the singular vectors for the projections of this sweep
    STAGE(RR_STAGE_OTHER, cast_f32(s, n, b, w.Vt, n, w.Vt32, n));
    STAGE(RR_STAGE_OTHER, cast_f32(s, m, b, w.Ut, m, w.Ut32, m));
    // split mode: blocks and operator carried as BF16 pairs (hi + lo), the
    // final correction blocks kept in FP32 for the projection and the lift
    const bool sp = op.split;
    const int32_t et = sp ? RR_F32 : dt;
    void* Eg = sp ? w.E32 : w.Elo;
    void* Fg = sp ? w.F32 : w.Flo;
    if (sp) STAGE(RR_STAGE_OTHER, scale_split(s, RR_F64, m, b, w.Rv, m, w.mu, w.Elo, w.Elo2, m, w.coef, w.sig));
    else STAGE(RR_STAGE_OTHER, scale_cast(s, RR_F64, m, b, w.Rv, m, w.mu, dt, w.Elo, m, w.coef, w.sig));
    for (int j = 0; j < qr; ++j) {
      if (sp) STAGE(RR_STAGE_LOWP_PRODUCT, apply_lowp_T_split(op, b, w.Elo, w.Elo2, m, w.W, n, w.Ru, n, w.coef, s));
      else STAGE(RR_STAGE_LOWP_PRODUCT, apply_lowp_T(op, b, w.Elo, m, w.W, n, w.Ru, n, w.coef, s));
      STAGE(RR_STAGE_GRAM, project_out(w.c, s, n, b, w.Vt32, n, (float*)w.W, n, w.Ys));
      if (sp) STAGE(RR_STAGE_OTHER, scale_split(s, op.wt, n, b, w.W, n, w.mu, w.Flo, w.Flo2, n, w.coef, w.sig));
      else STAGE(RR_STAGE_OTHER, scale_cast(s, op.wt, n, b, w.W, n, w.mu, dt, w.Flo, n, w.coef, w.sig));
      if (sp) STAGE(RR_STAGE_LOWP_PRODUCT, apply_lowp_split(op, b, w.Flo, w.Flo2, n, w.AF, m, w.Rv, m, w.coef, s));
      else STAGE(RR_STAGE_LOWP_PRODUCT, apply_lowp(op, b, w.Flo, n, w.AF, m, w.Rv, m, w.coef, s));
      STAGE(RR_STAGE_GRAM, project_out(w.c, s, m, b, w.Ut32, m, (float*)w.AF, m, w.Ys));
      if (j + 1 < qr) {
        if (sp) STAGE(RR_STAGE_OTHER, scale_split(s, op.wt, m, b, w.AF, m, w.mu, w.Elo, w.Elo2, m, w.coef, w.sig));
        else STAGE(RR_STAGE_OTHER, scale_cast(s, op.wt, m, b, w.AF, m, w.mu, dt, w.Elo, m, w.coef, w.sig));
      }
    }
    // conditioning of the correction blocks (Algorithm 8; the two blocks'
    // processes run at the same time, F's on the side stream with the second
    // workspace: each is a chain of b latency-bound pivot steps), then A F
    // for the low-precision block of the projected matrix
    STAGE(RR_STAGE_HESSENBERG, [&]() -> rr_status {
      cudaStream_t s2;
      RR_TRY(side_fork(s, &s2));
      RR_TRY(basis_step(w.c, hess, op.wt, et, m, b, w.AF, m, Eg, m, s));
      RR_TRY(basis_step(second_hess(w.c), hess, op.wt, et, n, b, w.W, n, Fg, n, s2));
      return side_join(s);
    }());
    if (sp) {
      STAGE(RR_STAGE_OTHER, scale_split(s, RR_F32, n, b, w.F32, n, nullptr, w.Flo, w.Flo2, n, nullptr, nullptr));
      STAGE(RR_STAGE_LOWP_PRODUCT, apply_lowp_split(op, b, w.Flo, w.Flo2, n, w.AF, m, nullptr, 0, nullptr, s));
    } else {
      STAGE(RR_STAGE_LOWP_PRODUCT, apply_lowp(op, b, w.Flo, n, w.AF, m, nullptr, 0, nullptr, s));
    }
    // projected blocks over S_u = [U~, E], S_v = [V~, F]  (ld 2b)
    double* B = w.Bm;
    STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, RR_F64, w.Ut, m, RR_F64, w.P, m, B, b2, s));                   // U~^T A V~
    STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, w.Qm, n, et, Fg, n, B + b * b2, b2, s));             // U~^T A F
    STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, et, Eg, m, RR_F64, w.P, m, B + b, b2, s));                   // E^T A V~
    STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, et, Eg, m, op.wt, w.AF, m, B + b + b * b2, b2, s));          // E^T A F
    STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, RR_F64, w.Ut, m, RR_F64, w.Ut, m, w.Gu, b2, s));
    STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, RR_F64, w.Ut, m, et, Eg, m, w.Gu + b * b2, b2, s));
    STAGE(RR_STAGE_OTHER, transpose(s, b, b, w.Gu + b * b2, b2, w.Gu + b, b2));
    STAGE(RR_STAGE_GRAM, gram(w.c, m, b, b, et, Eg, m, et, Eg, m, w.Gu + b + b * b2, b2, s));
    STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, w.Vt, n, RR_F64, w.Vt, n, w.Gv, b2, s));
    STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, w.Vt, n, et, Fg, n, w.Gv + b * b2, b2, s));
    STAGE(RR_STAGE_OTHER, transpose(s, b, b, w.Gv + b * b2, b2, w.Gv + b, b2));
    STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, et, Fg, n, et, Fg, n, w.Gv + b + b * b2, b2, s));
    STAGE(RR_STAGE_PENCIL, pencil_svd(w.c, b2, b2, B, w.Gu, w.Gv, w.sig2, w.Ys, w.Zs, s));
    // lift the leading b triplets
    STAGE(RR_STAGE_LIFT, lift2(op, s, m, b, RR_F64, w.Ut, m, b, et, Eg, m, b, w.Ys, b2, w.Ut2, m));
    STAGE(RR_STAGE_LIFT, lift2(op, s, n, b, RR_F64, w.Vt, n, b, et, Fg, n, b, w.Zs, b2, w.Vt2, n));
    return RR_OK;
  };
  // the device loops' fixed buffers: the sweep's output becomes the current
  // Ritz triplets (the host loop swaps the pointers instead)
  auto adopt = [&](cudaStream_t s) -> rr_status {
    RR_CUDA(cudaMemcpyAsync(w.Ut, w.Ut2, (size_t)m * b * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RR_CUDA(cudaMemcpyAsync(w.Vt, w.Vt2, (size_t)n * b * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RR_CUDA(cudaMemcpyAsync(w.sig, w.sig2, (size_t)b * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return RR_OK;
  };

  if (refine && !nan_seen && dloop) {
    // correction sweeps while the problem is not frozen and they contract
    // the residual (the single solve's stall rule), at most up to the sweep
    // where the fixed schedule polishes (its last two sweeps), then FP64
    // polish sweeps while the problem is still not frozen
    RR_TRY(residual_all(s));
    const int polish_from = std::max(p->max_sweeps - 2, ph1 + 1);
    RR_TRY(device_loop(s, body_s, w.frozen, p->max_sweeps, polish_from, sweep, 0, w.res, (int)k, 1,
                       [&](cudaStream_t bs) -> rr_status {
      RR_TRY(corr_sweep(bs));
      RR_TRY(adopt(bs));
      return residual_all(bs);
    }));
    RR_TRY(device_loop(s, body_s, w.frozen, p->max_sweeps, -1, 0, 1, w.res, (int)k, 0,
                       [&](cudaStream_t bs) -> rr_status {
      RR_TRY(svd_polish_f64(op, w, b, bs, prof));
      RR_TRY(adopt(bs));
      return residual_all(bs);
    }));
  } else if (refine && !nan_seen) {
    double prev_mx = INFINITY;
    bool polish = false;
    for (;;) {
      RR_TRY(residual_all(s));
      if (!batch_mode) {
        RR_CUDA(cudaMemcpyAsync(hres.data(), w.res, k * sizeof(double), cudaMemcpyDeviceToHost, s));
        RR_TRY(queue_cond(w.c, s, hcond));
        RR_CUDA(cudaStreamSynchronize(s));
        RR_TRY(read_err(w.c, s));
        double mx;
        inf.n_converged = count_converged(hres.data(), (int)k, p->tol, &mx);
        inf.max_res = mx;
        if (sweep >= 1 && sweep <= 64) inf.res_history[sweep - 1] = mx;
        note_cond(inf, sweep, hcond);
        if (all_nan(hres.data(), (int)k)) {
          nan_seen = true;
          break;
        }
        if (inf.n_converged == k) {
          converged = true;
          break;
        }
        // the corrections stopped contracting the residual: polish in FP64
        polish = inf.refine_sweeps >= 1 && mx > 0.3 * prev_mx;
        prev_mx = mx;
      }
      if (sweep >= p->max_sweeps) break;
      // batched problems (no host check) polish on their last two sweeps
      if (batch_mode) polish = sweep >= p->max_sweeps - 2 && sweep >= ph1 + 1;
      if (polish) {
        RR_TRY(svd_polish_f64(op, w, b, s, prof));
        ++inf.polish_sweeps;
        polish = false;
        prev_mx = INFINITY;
      } else {
        RR_TRY(corr_sweep(s));
      }
      if (batch_mode)
        STAGE(RR_STAGE_OTHER, keep_frozen(s, w.frozen, m, n, b, w.Ut, w.Ut2, w.Vt, w.Vt2, w.sig, w.sig2));
      std::swap(w.Ut, w.Ut2);
      std::swap(w.Vt, w.Vt2);
      RR_CUDA(cudaMemcpyAsync(w.sig, w.sig2, b * sizeof(double), cudaMemcpyDeviceToDevice, s));
      ++sweep;
      ++inf.refine_sweeps;
    }
  }
  if (batch_mode && !refine && !dloop) {
    // final residual for the caller's convergence count (read after the graph)
    STAGE(RR_STAGE_F64_PRODUCT, svd_residual(op, w, k, w.P, w.Qm, s));
  }
  // outputs: sigma, U, V (first k; the rows of A's own size), unit columns,
  // sign fixed on V
  RR_CUDA(cudaMemcpyAsync(sigma_out, w.sig, k * sizeof(double), cudaMemcpyDeviceToDevice, s));
  RR_CUDA(cudaMemcpy2DAsync(U_out, m0 * sizeof(double), w.Ut, m * sizeof(double), m0 * sizeof(double), k,
                            cudaMemcpyDeviceToDevice, s));
  RR_CUDA(cudaMemcpy2DAsync(V_out, n0 * sizeof(double), w.Vt, n * sizeof(double), n0 * sizeof(double), k,
                            cudaMemcpyDeviceToDevice, s));
  STAGE(RR_STAGE_OTHER, normalize_sign(s, n0, k, V_out, n0, m0, U_out, m0));
  inf.sweeps = sweep;
  if (batch_mode) {
    if (info) *info = inf;
    return RR_OK;
  }
  prof.finish(&inf);
  if (info) *info = inf;
  RR_CUDA(cudaStreamSynchronize(s));
  RR_TRY(read_err(w.c, s));
  if (nan_seen) return RR_ERR_NAN;
  return converged ? RR_OK : RR_ERR_NO_CONV;
}

static size_t svd_ws(const rr_operator* A_in, const rr_params* p, bool batch) {
  Arena ar(nullptr, 0);
  const int padq = svd_pad_quantum(A_in, p);
  rr_operator Apad;
  const rr_operator* A = svd_operator(A_in, p, ar, Apad, nullptr);
  Op op;
  make_op(A, p->basis, op);
  const bool refine = p->refine != 0 && p->basis != RR_F64;
  carve_op(ar, op, false, refine, p->block);
  SvdBufs w;
  carve_svd(ar, op, p->block, refine, w);
  if (batch || !p->v0 || padq) ar.take<double>(op.n * p->block);
  return ar.off + 4096;
}

// ===========================================================================
// symmetric eigenproblem (Algorithm 3 with Algorithm 1/8, power or Chebyshev
// filter, and the refinement phase)
// ===========================================================================
struct EigBufs {
  Common c;
  void *Vlo, *W, *Pw, *Dlo, *Dprev, *AD;
  double *G, *H, *Y, *Ysel, *th2;
  double *X, *X2, *theta, *P, *R, *ss, *res, *mu, *coef, *kap, *kap_prev, *rho, *gam, *gersh;
  float* X32;  // FP32 copy of the Ritz vectors for the refinement's projections
  ProjTc ptc;  // tensor-core projections of tall blocks (null when they do not apply)
};

// Row stride of the filter's row-major blocks: b rounded up to 8 columns
// (one 16-byte vector of BF16; a multiple of the FP32 and FP64 widths too).
static inline int64_t rows_width(int64_t b) { return (b + 7) / 8 * 8; }

static void carve_eig(Arena& ar, const Op& op, int64_t b, bool refine, EigBufs& w) {
  const int64_t n = op.n, b2 = refine ? 2 * b : b;
  const size_t ds = dsz(op.dt), ws_ = dsz(op.wt);
  const int64_t bp = rows_width(b);  // the filter's row-major blocks use these buffers too
  carve_common(ar, n, b2, op.wt, w.c);
  w.Vlo = ar.take_bytes(n * bp * ds);
  w.W = ar.take_bytes(n * bp * ws_);
  w.Pw = ar.take_bytes(n * bp * ws_);
  w.Dprev = ar.take_bytes(n * bp * ds);
  w.G = ar.take<double>(b2 * b2);
  w.H = ar.take<double>(b2 * b2);
  w.Y = ar.take<double>(b2 * b2);
  w.Ysel = ar.take<double>(b2 * b);
  w.th2 = ar.take<double>(b2);
  w.X = ar.take<double>(n * b);
  w.theta = ar.take<double>(b);
  w.P = ar.take<double>(n * b);
  w.R = ar.take<double>(n * b);
  w.ss = ar.take<double>(b);
  w.res = ar.take<double>(b);
  w.gersh = ar.take<double>(520);
  w.mu = ar.take<double>(b);
  w.coef = ar.take<double>(b);
  w.kap = ar.take<double>(b);
  w.kap_prev = ar.take<double>(b);
  w.rho = ar.take<double>(b);
  w.gam = ar.take<double>(b);
  if (refine) {
    w.X2 = ar.take<double>(n * b);
    w.Dlo = ar.take_bytes(n * b * ds);
    w.AD = ar.take_bytes(n * b * ws_);
    w.X32 = ar.take<float>(n * b);
    if (op.dt == RR_BF16 && proj_tc_applies(n, b)) {
      w.ptc.Xh = (__nv_bfloat16*)ar.take_bytes(n * b * 2);
      w.ptc.Xl = (__nv_bfloat16*)ar.take_bytes(n * b * 2);
      w.ptc.Xrh = (__nv_bfloat16*)ar.take_bytes(n * b * 2);
      w.ptc.Xrl = (__nv_bfloat16*)ar.take_bytes(n * b * 2);
      w.ptc.Th = (__nv_bfloat16*)ar.take_bytes(n * b * 2);
      w.ptc.Tl = (__nv_bfloat16*)ar.take_bytes(n * b * 2);
      w.ptc.Kh = (__nv_bfloat16*)ar.take_bytes(b * b * 2);
      w.ptc.Kl = (__nv_bfloat16*)ar.take_bytes(b * b * 2);
      w.ptc.K32 = ar.take<float>(b * b);
      w.ptc.P = ar.take<float>(n * b);
    }
  } else {
    w.X2 = nullptr;
    w.Dlo = w.AD = nullptr;
    w.X32 = nullptr;
  }
}

// Plain scaled Chebyshev filter of the block V (dt) into W (wt, Y_d,
// unscaled).  Bounds: damp [a, up], normalised at a0.  The d steps run on
// row-major copies (row stride bp = b rounded up to 8 columns): V is
// transposed once into Dprev, the steps ping-pong among Dprev, Vlo and W
// (Vlo is rewritten by the basis step afterwards), the last step writes Pw
// in wt, and Pw is transposed back into W.
static rr_status cheb_filter(const Op& op, EigBufs& w, int64_t b, int d, double a, double up,
                             double a0, cudaStream_t s) {
  const int64_t n = op.n;
  const double e = (up - a) / 2, c = (up + a) / 2, s1 = e / (a0 - c);
  const int64_t bp = rows_width(b);
  RR_TRY(block_to_rows(s, op.dt, n, b, bp, w.Vlo, n, w.Dprev, bp));
  if (d == 1) {
    RR_TRY(cheb_rows(s, n, b, op.rp, op.ci, op.va, op.dt, w.Dprev, nullptr, bp, s1 / e, c, 0.0, op.wt, w.Pw, bp));
  } else {
    RR_TRY(cheb_rows(s, n, b, op.rp, op.ci, op.va, op.dt, w.Dprev, nullptr, bp, s1 / e, c, 0.0, op.dt, w.Vlo, bp));
    double sg = s1;
    void *pm1 = w.Dprev, *p0 = w.Vlo, *p1 = w.W;
    for (int j = 2; j <= d; ++j) {
      const double sn = 1.0 / (2.0 / s1 - sg);
      const bool last = (j == d);
      RR_TRY(cheb_rows(s, n, b, op.rp, op.ci, op.va, op.dt, p0, pm1, bp, 2.0 * sn / e, c, sg * sn,
                       last ? op.wt : op.dt, last ? w.Pw : p1, bp));
      void* t = pm1;
      pm1 = p0;
      p0 = p1;
      p1 = t;
      sg = sn;
    }
  }
  return block_from_rows(s, op.wt, n, b, w.Pw, bp, w.W, n);
}


static rr_status eig_run(const rr_operator* Aop, const rr_params* p, double* theta_out,
                         double* X_out, void* ws, size_t ws_bytes, rr_info* info, cudaStream_t s) {
  const int32_t dt = p->basis;
  if (dt == RR_E4M3) return RR_ERR_ARG;  // the FP8 basis is built for the SVD
  Op op;
  make_op(Aop, dt, op);
  const int64_t n = op.n, b = p->block, k = p->k;
  const int q = p->degree;
  const bool hess = p->hessenberg != 0;
  const bool cheb = p->filter == RR_CHEBYSHEV;
  const bool refine = p->refine != 0 && dt != RR_F64;
  const int ph1 = refine ? (p->phase1_sweeps > 0 ? p->phase1_sweeps : 1) : p->max_sweeps;
  if (cheb && op.kind != RR_CSR) return RR_ERR_ARG;
  if (!cheb && p->which != RR_LARGEST) return RR_ERR_ARG;
  Arena ar(ws, ws_bytes);
  carve_op(ar, op, true, refine, b);
  EigBufs w;
  carve_eig(ar, op, b, refine, w);
  double* v0buf = p->v0 ? nullptr : ar.take<double>(n * b);
  if (ar.overflow) return RR_ERR_WORKSPACE;
  Prof prof;
  prof.on = p->profile != 0;
  prof.s = s;
  prof.start();
  w.c.hess_tol = p->hess_tol;
  RR_CUDA(cudaMemsetAsync(w.c.hess_ws, 0, 512, s));
  RR_CUDA(cudaMemsetAsync(w.c.hess_ws2, 0, 512, s));
  STAGE(RR_STAGE_OTHER, check_operator_finite(Aop, w.c, s));
  STAGE(RR_STAGE_OTHER, prepare_op(op, op, true, s));

  double lo = p->bounds[0], up = p->bounds[1];
  if (cheb && !(lo < up)) {
    STAGE(RR_STAGE_OTHER, csr_gershgorin(s, n, op.rp, op.ci, op.va, w.gersh));
    double h2[2];
    RR_CUDA(cudaMemcpyAsync(h2, w.gersh + 512, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaStreamSynchronize(s));
    lo = h2[0];
    up = h2[1];
  }
  double ca = lo + 0.1 * (up - lo), ca0 = lo;  // Chebyshev cut and scaling point

  const double* v0 = p->v0;
  if (!v0) {
    STAGE(RR_STAGE_OTHER, uniform_block(s, n, b, p->seed, v0buf, n));
    v0 = v0buf;
  }
  STAGE(RR_STAGE_OTHER, rr_colscale_cast(n, b, v0, n, dt, w.Vlo, n, w.c.scale, s));
  rr_info inf;
  memset(&inf, 0, sizeof(inf));
  std::vector<double> hres(b), hth(b);
  double hcond[4] = {0.0, 0.0, 0.0, 0.0};
  int sweep = 0;
  bool converged = false, nan_seen = false;

  auto update_bounds = [&]() -> rr_status {
    if (!cheb) return RR_OK;
    RR_CUDA(cudaMemcpyAsync(hth.data(), w.theta, b * sizeof(double), cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaStreamSynchronize(s));
    double mn = INFINITY, mxv = -INFINITY;
    for (int i = 0; i < b; ++i)
      if (!std::isnan(hth[i])) {
        mn = fmin(mn, hth[i]);
        mxv = fmax(mxv, hth[i]);
      }
    if (mn < mxv && mxv < up) {
      ca = mxv;
      ca0 = mn;
    }
    return RR_OK;
  };

  // ---------------- phase 1 ----------------
  for (int ps = 0; ps < ph1 && sweep < p->max_sweeps; ++ps) {
    if (ps > 0) STAGE(RR_STAGE_OTHER, rr_colscale_cast(n, b, w.X, n, dt, w.Vlo, n, w.c.scale, s));
    if (cheb) {
      STAGE(RR_STAGE_LOWP_PRODUCT, cheb_filter(op, w, b, q, ca, up, ca0, s));
      STAGE(RR_STAGE_HESSENBERG, basis_step(w.c, hess, op.wt, dt, n, b, w.W, n, w.Vlo, n, s));
    } else {
      for (int it = 0; it < q; ++it) {
        STAGE(RR_STAGE_LOWP_PRODUCT, apply_lowp(op, b, w.Vlo, n, w.W, n, nullptr, 0, nullptr, s));
        STAGE(RR_STAGE_HESSENBERG, basis_step(w.c, hess, op.wt, dt, n, b, w.W, n, w.Vlo, n, s));
      }
    }
    // Algorithm 3: H = V^T (A V), G = V^T V, H Y = G Y Theta, X = V Y
    STAGE(RR_STAGE_LOWP_PRODUCT, apply_lowp(op, b, w.Vlo, n, w.Pw, n, nullptr, 0, nullptr, s));
    STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, dt, w.Vlo, n, dt, w.Vlo, n, w.G, b, s));
    STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, dt, w.Vlo, n, op.wt, w.Pw, n, w.H, b, s));
    STAGE(RR_STAGE_PENCIL, pencil_eig(w.c, b, w.H, w.G, w.th2, w.Y, s));
    STAGE(RR_STAGE_PENCIL, select_eig(s, b, b, p->which, w.th2, w.Y, b, w.theta, w.Ysel, b));
    STAGE(RR_STAGE_LIFT, lift2(op, s, n, b, dt, w.Vlo, n, b, 0, nullptr, 0, 0, w.Ysel, b, w.X, n));
    ++sweep;
    STAGE(RR_STAGE_OTHER, update_bounds());
    if (!refine) {
      // FP64 residual of the wanted pairs.  With an FP64 basis A X = (A V) Y exactly.
      if (dt == RR_F64) STAGE(RR_STAGE_LIFT, lift(s, RR_F64, n, k, b, w.Pw, n, w.Ysel, b, w.P, n, 0));
      else RR_TRY(apply_f64(op, k, w.X, n, w.P, n, s));
      STAGE(RR_STAGE_OTHER, residual_block(s, n, k, w.P, n, w.X, n, w.theta, w.R, n, w.ss, 0));
      STAGE(RR_STAGE_OTHER, res_finish(s, k, w.ss, w.theta, w.res));
      RR_CUDA(cudaMemcpyAsync(hres.data(), w.res, k * sizeof(double), cudaMemcpyDeviceToHost, s));
      RR_TRY(queue_cond(w.c, s, hcond));
      RR_CUDA(cudaStreamSynchronize(s));
      RR_TRY(read_err(w.c, s));
      double mx;
      inf.n_converged = count_converged(hres.data(), (int)k, p->tol, &mx);
      inf.max_res = mx;
      if (sweep <= 64) inf.res_history[sweep - 1] = mx;
      note_cond(inf, sweep, hcond);
      if (all_nan(hres.data(), (int)k)) {
        nan_seen = true;
        break;
      }
      if (inf.n_converged == k) {
        converged = true;
        break;
      }
    }
  }

  // ---------------- phase 2 ----------------
  if (refine && !nan_seen) {
    const int64_t b2 = 2 * b;
    double prev_mx = INFINITY;
    for (;;) {
      STAGE(RR_STAGE_F64_PRODUCT, apply_f64(op, b, w.X, n, w.P, n, s));  // P = A X, FP64-accurate
      STAGE(RR_STAGE_OTHER, residual_block(s, n, b, w.P, n, w.X, n, w.theta, w.R, n, w.ss, 0));
      STAGE(RR_STAGE_OTHER, res_finish(s, b, w.ss, w.theta, w.res));
      RR_CUDA(cudaMemcpyAsync(hres.data(), w.res, k * sizeof(double), cudaMemcpyDeviceToHost, s));
      RR_TRY(queue_cond(w.c, s, hcond));
      RR_CUDA(cudaStreamSynchronize(s));
      RR_TRY(read_err(w.c, s));
      double mx;
      inf.n_converged = count_converged(hres.data(), (int)k, p->tol, &mx);
      inf.max_res = mx;
      if (sweep >= 1 && sweep <= 64) inf.res_history[sweep - 1] = mx;
      note_cond(inf, sweep, hcond);
      if (all_nan(hres.data(), (int)k)) {
        nan_seen = true;
        break;
      }
      if (inf.n_converged == k) {
        converged = true;
        break;
      }
      if (sweep >= p->max_sweeps) break;
      // the corrections stopped contracting the residual (power filter): one
      // sweep of the method in FP64-accurate arithmetic from the Ritz vectors
      // (q products, each followed by Algorithm 8 in FP64, then Algorithm 3).
      // A stall is a sweep that keeps more than 0.7 of the residual: the power
      // filter's own rate is often 0.3-0.4 per sweep on clustered spectra (the
      // Gaussian kernel matrix), where the FP64 sweep contracts no faster and
      // costs q FP64-accurate products (a 0.3 threshold took that solve through
      // 7 polish sweeps: 28 s against 14 s)
      const bool stalled = !cheb && inf.refine_sweeps >= 1 && mx > 0.7 * prev_mx;
      prev_mx = mx;
      if (stalled) {
        double* V = w.X2;
        double* Wb = w.P;
        RR_CUDA(cudaMemcpyAsync(V, w.X, (size_t)n * b * sizeof(double), cudaMemcpyDeviceToDevice, s));
        for (int it = 0; it < q; ++it) {
          STAGE(RR_STAGE_F64_PRODUCT, apply_f64(op, b, V, n, Wb, n, s));
          STAGE(RR_STAGE_HESSENBERG, basis_step(w.c, true, RR_F64, RR_F64, n, b, Wb, n, V, n, s));
        }
        STAGE(RR_STAGE_F64_PRODUCT, apply_f64(op, b, V, n, w.R, n, s));
        STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, V, n, RR_F64, V, n, w.G, b, s));
        STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, V, n, RR_F64, w.R, n, w.H, b, s));
        STAGE(RR_STAGE_PENCIL, pencil_eig(w.c, b, w.H, w.G, w.th2, w.Y, s));
        STAGE(RR_STAGE_PENCIL, select_eig(s, b, b, p->which, w.th2, w.Y, b, w.theta, w.Ysel, b));
        STAGE(RR_STAGE_LIFT, lift2(op, s, n, b, RR_F64, V, n, b, 0, nullptr, 0, 0, w.Ysel, b, w.P, n));
        RR_CUDA(cudaMemcpyAsync(w.X, w.P, (size_t)n * b * sizeof(double), cudaMemcpyDeviceToDevice, s));
        ++sweep;
        ++inf.refine_sweeps;
        ++inf.polish_sweeps;
        prev_mx = INFINITY;
        continue;
      }
      // FP32 copy (for tall BF16-basis blocks split BF16 pairs) of the Ritz
      // vectors for the projections of this sweep
      if (w.ptc.Xh) STAGE(RR_STAGE_OTHER, proj_tc_prepare(w.ptc, s, n, b, w.X, n));
      else STAGE(RR_STAGE_OTHER, cast_f32(s, n, b, w.X, n, w.X32, n));
      auto proj = [&](float* T) -> rr_status {
        return w.ptc.Xh ? project_out_tc(w.ptc, s, n, b, T, n) : project_out(w.c, s, n, b, w.X32, n, T, n, w.Y);
      };
      if (cheb) {
        // D_1 = (s1/e) R;  D_{j+1} = (2 s_{j+1}/e)(A - cI) D_j - s_j s_{j+1} D_{j-1}
        //                           + (2 s_{j+1}/e) phi_j(theta) R
        // with D_j = s_j * Dhat_j, kappa_j = phi_j / s_j, rho_j = s_{j-1} / s_j.
        const double e = (up - ca) / 2, c = (up + ca) / 2, s1 = e / (ca0 - c);
        STAGE(RR_STAGE_OTHER, scale_cast(s, RR_F64, n, b, w.R, n, w.mu, dt, w.Vlo, n, nullptr, nullptr));
        // kappa_1 = (theta - c)/mu_1 ; kappa_0 rho_1 = e/(s1 mu_1)  (phi_0 / s_1)
        // computed by the coefficient kernel from kappa=1/(mu s1/e) seeds:
        STAGE(RR_STAGE_OTHER, fill(s, b, 0.0, w.kap));
        STAGE(RR_STAGE_OTHER, fill(s, b, 0.0, w.kap_prev));
        STAGE(RR_STAGE_OTHER, fill(s, b, 1.0, w.rho));
        // kap <- ((s1/e)(theta - c)*1 - 0)/((s1/e) mu) : an = 1, bn = 0 with kap = 1, then divide
        STAGE(RR_STAGE_OTHER, fill(s, b, e / s1, w.kap));
        STAGE(RR_STAGE_OTHER, cheb_coef_update(s, b, w.theta, w.mu, s1 / e, c, 0.0, w.kap, w.kap_prev, w.rho));
        // now kap = (theta - c)/mu_1, kap_prev = e/s1, rho = 1/mu_1 -> kap_prev*rho = e/(s1 mu_1)
        void* dm1 = nullptr;  // Dhat_0 = 0
        void* d0 = w.Vlo;
        void* d1 = w.Dprev;
        double sg = s1;
        for (int j = 1; j < q; ++j) {
          const double sn = 1.0 / (2.0 / s1 - sg);
          const double an = 2.0 * sn / e, bn = sg * sn;
          STAGE(RR_STAGE_OTHER, vec_scale(s, b, an, w.kap, w.gam));
          STAGE(RR_STAGE_LOWP_PRODUCT, rr_chebyshev_step(n, b, op.rp, op.ci, op.va, dt, d0, dm1, n, an, c, bn, w.rho, w.R, n,
                                   w.gam, op.wt, w.W, n, s));
          STAGE(RR_STAGE_GRAM, proj((float*)w.W));
          if (j + 1 < q) {
            // Dhat_{j+1} = T / mu into the buffer of Dhat_{j-1}
            void* dst = dm1 ? dm1 : d1;
            STAGE(RR_STAGE_OTHER, scale_cast(s, op.wt, n, b, w.W, n, w.mu, dt, dst, n, nullptr, nullptr));
            STAGE(RR_STAGE_OTHER, cheb_coef_update(s, b, w.theta, w.mu, an, c, bn, w.kap, w.kap_prev, w.rho));
            dm1 = d0;
            d0 = dst;
          }
          sg = sn;
        }
        if (q == 1) STAGE(RR_STAGE_OTHER, scale_cast(s, RR_F64, n, b, w.R, n, w.mu, op.wt, w.W, n, nullptr, nullptr));
      } else {
        // D_1 = R;  D_{j+1} = A D_j + R Theta^j  (coef <- coef theta / mu)
        STAGE(RR_STAGE_OTHER, fill(s, b, 1.0, w.coef));
        if (q == 1) {
          STAGE(RR_STAGE_OTHER, scale_cast(s, RR_F64, n, b, w.R, n, w.mu, op.wt, w.W, n, nullptr, nullptr));
        } else {
          STAGE(RR_STAGE_OTHER, scale_cast(s, RR_F64, n, b, w.R, n, w.mu, dt, w.Vlo, n, w.coef, w.theta));
          for (int j = 1; j < q; ++j) {
            STAGE(RR_STAGE_LOWP_PRODUCT, apply_lowp(op, b, w.Vlo, n, w.W, n, w.R, n, w.coef, s));
            STAGE(RR_STAGE_GRAM, proj((float*)w.W));
            if (j + 1 < q) STAGE(RR_STAGE_OTHER, scale_cast(s, op.wt, n, b, w.W, n, w.mu, dt, w.Vlo, n, w.coef, w.theta));
          }
        }
      }
      STAGE(RR_STAGE_HESSENBERG, basis_step(w.c, hess, op.wt, dt, n, b, w.W, n, w.Dlo, n, s));
      STAGE(RR_STAGE_LOWP_PRODUCT, apply_lowp(op, b, w.Dlo, n, w.AD, n, nullptr, 0, nullptr, s));
      // projected pencil over S = [X, D] (ld 2b)
      STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, w.X, n, RR_F64, w.X, n, w.G, b2, s));
      STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, w.X, n, dt, w.Dlo, n, w.G + b * b2, b2, s));
      STAGE(RR_STAGE_OTHER, transpose(s, b, b, w.G + b * b2, b2, w.G + b, b2));
      STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, dt, w.Dlo, n, dt, w.Dlo, n, w.G + b + b * b2, b2, s));
      STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, w.X, n, RR_F64, w.P, n, w.H, b2, s));
      STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, RR_F64, w.P, n, dt, w.Dlo, n, w.H + b * b2, b2, s));
      STAGE(RR_STAGE_OTHER, transpose(s, b, b, w.H + b * b2, b2, w.H + b, b2));
      STAGE(RR_STAGE_GRAM, gram(w.c, n, b, b, dt, w.Dlo, n, op.wt, w.AD, n, w.H + b + b * b2, b2, s));
      STAGE(RR_STAGE_PENCIL, pencil_eig(w.c, b2, w.H, w.G, w.th2, w.Y, s));
      STAGE(RR_STAGE_PENCIL, select_eig(s, b2, b, p->which, w.th2, w.Y, b2, w.theta, w.Ysel, b2));
      STAGE(RR_STAGE_LIFT, lift2(op, s, n, b, RR_F64, w.X, n, b, dt, w.Dlo, n, b, w.Ysel, b2, w.X2, n));
      std::swap(w.X, w.X2);
      ++sweep;
      ++inf.refine_sweeps;
      STAGE(RR_STAGE_OTHER, update_bounds());
    }
  }

  RR_CUDA(cudaMemcpyAsync(theta_out, w.theta, k * sizeof(double), cudaMemcpyDeviceToDevice, s));
  RR_CUDA(cudaMemcpy2DAsync(X_out, n * sizeof(double), w.X, n * sizeof(double), n * sizeof(double), k,
                            cudaMemcpyDeviceToDevice, s));
  STAGE(RR_STAGE_OTHER, normalize_sign(s, n, k, X_out, n, 0, nullptr, 0));
  RR_CUDA(cudaStreamSynchronize(s));
  RR_TRY(read_err(w.c, s));
  inf.sweeps = sweep;
  prof.finish(&inf);
  if (info) *info = inf;
  if (nan_seen) return RR_ERR_NAN;
  return converged ? RR_OK : RR_ERR_NO_CONV;
}

static size_t eig_ws(const rr_operator* A, const rr_params* p) {
  Op op;
  make_op(A, p->basis, op);
  Arena ar(nullptr, 0);
  const bool refine = p->refine != 0 && p->basis != RR_F64;
  carve_op(ar, op, true, refine, p->block);
  EigBufs w;
  carve_eig(ar, op, p->block, refine, w);
  if (!p->v0) ar.take<double>(op.n * p->block);
  return ar.off + 4096;
}

static rr_status check_op(const rr_operator* A, bool svd) {
  if (!A || !A->values) return RR_ERR_ARG;
  if (A->kind == RR_DENSE) {
    if (A->dtype != RR_F64 || A->m <= 0 || A->n <= 0 || A->ld < A->m) return RR_ERR_ARG;
    if (svd && A->m < A->n) return RR_ERR_ARG;
    if (!svd && A->m != A->n) return RR_ERR_ARG;
    return RR_OK;
  }
  if (A->kind == RR_KERNEL) {
    RR_TRY(check_kernel_operator(A));
    if (svd && A->m < A->n) return RR_ERR_ARG;
    if (!svd && A->points_y) return RR_ERR_ARG;  // the eigensolver takes the symmetric operator
    return RR_OK;
  }
  if (A->kind == RR_CSR) {
    if (svd || A->dtype != RR_F32 || A->n <= 0 || !A->row_ptr || !A->col_idx) return RR_ERR_ARG;
    if (A->n > 0x7fffffff || A->nnz > 0x7fffffff) return RR_ERR_ARG;
    return RR_OK;
  }
  return RR_ERR_ARG;
}

}  // namespace rr

using namespace rr;

extern "C" size_t rr_workspace_size(const rr_operator* A, const rr_params* p, int svd) {
  if (check_op(A, svd != 0) != RR_OK || !p) return 0;
  return svd ? svd_ws(A, p, false) : eig_ws(A, p);
}

extern "C" rr_status rr_eig(const rr_operator* A, const rr_params* p, double* theta, double* X,
                            void* ws, size_t ws_bytes, rr_info* info, void* stream) {
  RR_TRY(check_op(A, false));
  RR_TRY(check_params(p, A->n));
  if (p->basis == RR_E4M3) return RR_ERR_ARG;
  if (!theta || !X) return RR_ERR_ARG;
  if (!ws || ws_bytes < eig_ws(A, p) || ((uintptr_t)ws & 255)) return RR_ERR_WORKSPACE;
  return eig_run(A, p, theta, X, ws, ws_bytes, info, as_stream(stream));
}

extern "C" rr_status rr_svd(const rr_operator* A, const rr_params* p, double* sigma, double* U,
                            double* V, void* ws, size_t ws_bytes, rr_info* info, void* stream) {
  RR_TRY(check_op(A, true));
  RR_TRY(check_params(p, A->n));
  if (!sigma || !U || !V) return RR_ERR_ARG;
  if (!ws || ws_bytes < svd_ws(A, p, false) || ((uintptr_t)ws & 255)) return RR_ERR_WORKSPACE;
  return svd_run(A, p, sigma, U, V, ws, ws_bytes, info, as_stream(stream), false, 0, 0, nullptr);
}

extern "C" size_t rr_batch_workspace_size(int32_t count, const rr_operator* A, const rr_params* p) {
  if (count <= 0 || !A || !p) return 0;
  size_t tot = 0;
  for (int i = 0; i < count; ++i) {
    if (check_op(&A[i], true) != RR_OK) return 0;
    tot += align_up(svd_ws(&A[i], p, true), 4096);
  }
  return tot + 4096;
}

// All problems are captured into one CUDA graph: NS streams fork from the
// caller's stream, problems are dealt round-robin to them, each problem runs
// with no host synchronisation, its Hessenberg steps on one CTA (plain
// launches), and the branches join back before the single graph launch
// completes.  A problem's first sweep is captured as plain nodes; its later
// sweeps run in WHILE nodes whose condition a kernel sets on the GPU after
// each sweep's residual check, so a problem stops at tol (device-side loop
// control).  With tuning->fixed_sweeps every sweep is captured instead and
// every problem runs max_sweeps sweeps, keeping the triplets it froze at.
extern "C" rr_status rr_batch_svd(int32_t count, const rr_operator* A, const rr_params* p,
                                  uint64_t seed, double* const* sigma, double* const* U,
                                  double* const* V, void* ws, size_t ws_bytes,
                                  rr_status* per_problem, rr_info* info, void* stream) {
  return rr_batch_svd_tuned(count, A, p, seed, sigma, U, V, ws, ws_bytes, nullptr, per_problem, info, stream);
}

extern "C" rr_status rr_batch_svd_tuned(int32_t count, const rr_operator* A, const rr_params* p, uint64_t seed,
                                        double* const* sigma, double* const* U, double* const* V, void* ws,
                                        size_t ws_bytes, const rr_batch_tuning* tuning, rr_status* per_problem,
                                        rr_info* info, void* stream) {
  if (count <= 0 || !A || !p || !sigma || !U || !V || !ws || p->basis == RR_E4M3) return RR_ERR_ARG;
  const rr_batch_tuning tune = tuning ? *tuning : rr_batch_tuning{16, 0, 0, 0};
  if (tune.branches < 1 || tune.branches > kBatchMaxBranches || tune.max_splits < 0 ||
      (tune.order != 0 && tune.order != 1) || (tune.fixed_sweeps != 0 && tune.fixed_sweeps != 1))
    return RR_ERR_ARG;
  const bool dloop = tune.fixed_sweeps == 0;
  for (int i = 0; i < count; ++i) {
    RR_TRY(check_op(&A[i], true));
    RR_TRY(check_params(p, A[i].n));
  }
  if (ws_bytes < rr_batch_workspace_size(count, A, p)) return RR_ERR_WORKSPACE;
  RR_TRY(tc_prepare_attributes());
  cudaStream_t s = as_stream(stream);
  const int NS = tune.branches;
  // launch order: as given, or largest problems first (each branch then
  // finishes its big problems before its small ones)
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  if (tune.order == 1)
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return A[a].m * A[a].n > A[b].m * A[b].n; });
  // Capture on a private stream (the legacy default stream cannot be
  // captured); the instantiated graph is launched on the caller's stream.
  cudaStream_t cap = nullptr, body = nullptr;
  cudaStream_t br[kBatchMaxBranches] = {};
  cudaEvent_t fork = nullptr, join[kBatchMaxBranches] = {};
  rr_params pp = *p;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaGraphExec_t> execs;
  rr_status st = RR_OK;
  std::vector<size_t> offs(count);
  size_t off = 0;
  for (int i = 0; i < count; ++i) {
    offs[i] = off;
    off += align_up(svd_ws(&A[i], p, true), 4096);
  }
  std::vector<rr_info> infos(count);
  auto cu = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == RR_OK) {
      set_last_error(what, e);
      st = RR_ERR_CUDA;
    }
  };
  cu(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "rr_batch_svd stream");
  for (int i = 0; i < NS && st == RR_OK; ++i) {
    cu(cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking), "rr_batch_svd stream");
    cu(cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming), "rr_batch_svd event");
    if (st == RR_OK && pencil_side_prepare(br[i]) != RR_OK) st = RR_ERR_CUDA;  // before the capture
  }
  cu(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "rr_batch_svd event");
  // the stream the loop bodies are captured on (one body at a time)
  if (dloop && st == RR_OK) {
    cu(cudaStreamCreateWithFlags(&body, cudaStreamNonBlocking), "rr_batch_svd stream");
    if (st == RR_OK && pencil_side_prepare(body) != RR_OK) st = RR_ERR_CUDA;
  }
  // one graph per chunk of problems, launched in order on `s` (the host
  // captures and instantiates the next chunk while the GPU runs the earlier
  // ones).  With every sweep captured: at most kBatchSweepBudget
  // problem-sweeps per graph (a few hundred thousand nodes).  With device
  // loops (a problem captures its phase-1 sweeps, one correction sweep, one
  // polish sweep and three residual checks): kBatchLoopChunk problems per
  // graph.  Capture and instantiation take about as long as the GPU work, so
  // one graph for the whole batch left the GPU idle for half the call (512
  // problems: 2.8 s; graphs of 64 problems 2.6 s, of 32 2.0 s, of 16 1.8 s).
  const int ph1c = p->refine != 0 && p->basis != RR_F64 ? std::max(1, (int)p->phase1_sweeps) : 1;
  const int captured = dloop ? std::min((int)p->max_sweeps, ph1c + 3) : (int)p->max_sweeps;
  const int per_graph = dloop ? kBatchLoopChunk : std::max(1, kBatchSweepBudget / std::max(1, captured));
  for (int r0 = 0; r0 < count && st == RR_OK; r0 += per_graph) {
    const int r1 = std::min(count, r0 + per_graph);
    bool capturing = false;
    if (st == RR_OK) {
      cu(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "rr_batch_svd capture");
      capturing = st == RR_OK;
    }
    if (capturing) {
      cu(cudaEventRecord(fork, cap), "rr_batch_svd fork");
      for (int i = 0; i < NS; ++i) cu(cudaStreamWaitEvent(br[i], fork, 0), "rr_batch_svd fork wait");
      GemmSplitCap cap_scope(tune.max_splits);  // K splits of the products captured below
      for (int r = r0; r < r1 && st == RR_OK; ++r) {
        const int i = order[r];
        size_t need = align_up(svd_ws(&A[i], p, true), 4096);
        st = svd_run(&A[i], &pp, sigma[i], U[i], V[i], (char*)ws + offs[i], need, &infos[i], br[(r - r0) % NS],
                     true, 1, seed + (uint64_t)i, dloop ? body : nullptr);
      }
      for (int i = 0; i < NS; ++i) {
        cudaEventRecord(join[i], br[i]);
        cudaStreamWaitEvent(cap, join[i], 0);
      }
      cudaError_t ce = cudaStreamEndCapture(cap, &graph);
      cu(ce, "rr_batch_svd end capture");
    }
    if (st == RR_OK) cu(cudaGraphInstantiate(&exec, graph, 0), "rr_batch_svd instantiate");
    if (st == RR_OK) cu(cudaGraphLaunch(exec, s), "rr_batch_svd launch");
    if (exec) execs.push_back(exec);  // destroyed after the final synchronisation
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
  cu(cudaStreamSynchronize(s), "rr_batch_svd sync");
  for (cudaGraphExec_t e : execs) cudaGraphExecDestroy(e);
  if (cap) cudaStreamDestroy(cap);
  if (body) {
    pencil_side_release(body);
    cudaStreamDestroy(body);
  }
  for (int i = 0; i < NS; ++i) {
    if (br[i]) pencil_side_release(br[i]);
    if (br[i]) cudaStreamDestroy(br[i]);
    if (join[i]) cudaEventDestroy(join[i]);
  }
  if (fork) cudaEventDestroy(fork);
  if (st != RR_OK) return st;
  // per-problem residuals (device) -> convergence counts
  int nbad = 0;
  for (int i = 0; i < count; ++i) {
    Op op;
    Arena ar((char*)ws + offs[i], align_up(svd_ws(&A[i], p, true), 4096));
    rr_operator Apad;
    make_op(svd_operator(&A[i], p, ar, Apad, nullptr), p->basis, op);
    carve_op(ar, op, false, p->refine != 0 && p->basis != RR_F64, p->block);
    SvdBufs w;
    carve_svd(ar, op, p->block, p->refine != 0 && p->basis != RR_F64, w);
    std::vector<double> hres(p->k);
    RR_CUDA(cudaMemcpy(hres.data(), w.res, p->k * sizeof(double), cudaMemcpyDeviceToHost));
    int e = 0;
    RR_CUDA(cudaMemcpy(&e, w.c.hess_ws, sizeof(int), cudaMemcpyDeviceToHost));
    if (!e) RR_CUDA(cudaMemcpy(&e, w.c.hess_ws2, sizeof(int), cudaMemcpyDeviceToHost));
    if (dloop) {
      // sweeps the problem ran (device-side loop control)
      int ctl[3] = {0, 0, 0};
      RR_CUDA(cudaMemcpy(ctl, w.frozen, sizeof(ctl), cudaMemcpyDeviceToHost));
      infos[i].sweeps = ctl[1];
      infos[i].polish_sweeps = ctl[2];
      infos[i].refine_sweeps = p->refine != 0 && p->basis != RR_F64 ? std::max(0, ctl[1] - ph1c) : 0;
    }
    double mx;
    infos[i].n_converged = count_converged(hres.data(), p->k, p->tol, &mx);
    infos[i].max_res = mx;
    rr_status ps = e ? (rr_status)e : (infos[i].n_converged == p->k ? RR_OK : RR_ERR_NO_CONV);
    if (ps != RR_OK) ++nbad;
    if (per_problem) per_problem[i] = ps;
    if (info) info[i] = infos[i];
  }
  return nbad ? RR_ERR_NO_CONV : RR_OK;
}
