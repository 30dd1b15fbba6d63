// Internal launchers shared between the kernel files and the host solver.
#pragma once
#include <vector>
#include "rr_common.cuh"

namespace rr {
rr_status lift(cudaStream_t s, int32_t stype, int64_t n, int64_t b, int64_t p, const void* S,
               int64_t lds, const double* Y, int64_t ldy, double* X, int64_t ldx, int accum);
rr_status residual_block(cudaStream_t s, int64_t n, int64_t b, const double* P, int64_t ldp,
                         const double* X, int64_t ldx, const double* theta, double* R, int64_t ldr,
                         double* ss, int accum_ss);
rr_status res_finish(cudaStream_t s, int64_t b, const double* ss, const double* theta, double* res);
rr_status scale_cast(cudaStream_t s, int32_t ttype, int64_t n, int64_t b, const void* T, int64_t ldt,
                     double* mu, int32_t dtype, void* D, int64_t ldd, double* coef,
                     const double* sig);
rr_status scale_split(cudaStream_t s, int32_t ttype, int64_t n, int64_t b, const void* T, int64_t ldt,
                      double* mu, void* D_hi, void* D_lo, int64_t ldd, double* coef, const double* sig);
rr_status cast_operator_lo(int64_t m, int64_t n, const double* A, int64_t lda, void* lo_col, void* lo_row,
                           cudaStream_t s);
rr_status transpose(cudaStream_t s, int64_t p, int64_t q, const double* src, int64_t lds, double* dst,
                    int64_t ldd);
rr_status select_eig(cudaStream_t s, int64_t nb, int64_t b, int which, const double* theta,
                     const double* Y, int64_t ldy, double* tsel, double* Ysel, int64_t ldys);
rr_status normalize_sign(cudaStream_t s, int64_t n, int64_t k, double* X, int64_t ldx, int64_t m,
                         double* U, int64_t ldu);
rr_status vec_mul(cudaStream_t s, int64_t n, const double* a, const double* b, double* d);
rr_status fill(cudaStream_t s, int64_t n, double v, double* d);
rr_status side_fork(cudaStream_t s, cudaStream_t* s2);
rr_status side_join(cudaStream_t s);
rr_status eye_neg(cudaStream_t s, int64_t b, const double* K, int64_t ldk, double* Y, int64_t ldy);
rr_status add_cols_scaled(cudaStream_t s, int64_t n, int64_t b, const double* X, int64_t ldx, const double* c, int pw,
                          double* Y, int64_t ldy);
rr_status freeze_update(cudaStream_t s, int64_t k, const double* res, double tol, int* frozen);
rr_status loop_ctl(cudaStream_t s, cudaGraphConditionalHandle h, int* ctl, int inc, int inc_polish, int max_sweeps,
                   int stop_at, const double* res, int k, int stall);
rr_status keep_frozen(cudaStream_t s, const int* frozen, int64_t m, int64_t n, int64_t b, const double* U, double* U2,
                      const double* V, double* V2, const double* sig, double* sig2);
rr_status operator_nonfinite(cudaStream_t s, int kind, int64_t m, int64_t n, const void* values, int64_t lda,
                             int64_t nnz, int* flag);
// left-looking Hessenberg process on a block (k_krylov.cu)
size_t hess_left_ws_bytes(int64_t n, int64_t k, int32_t arith);
rr_status hess_left_run(cudaStream_t s, int32_t arith, int64_t n, int64_t k, void* W, int64_t ldw, int* piv,
                        void* ws, size_t ws_bytes);
// matrix-free Gaussian kernel operator (k_kernel.cu)
rr_status kernel_apply(cudaStream_t s, const rr_operator* A, int trans, int64_t b, int32_t xtype, const void* X,
                       int64_t ldx, int32_t otype, void* Y, int64_t ldy, const double* R, int64_t ldr,
                       const double* coef);
rr_status check_kernel_operator(const rr_operator* A);
rr_status uniform_block(cudaStream_t s, int64_t n, int64_t b, uint64_t seed, double* V, int64_t ldv);
rr_status cheb_coef_update(cudaStream_t s, int64_t b, const double* theta, const double* mu,
                           double alpha_next, double cshift, double beta_next, double* kappa,
                           double* kappa_prev, double* rho);
const double* pencil_cond_slot(void* ws, size_t ws_bytes, int b1, int b2);
void small_gemm(cudaStream_t s, int ta, int tb, int M, int N, int K, double alpha, const double* A,
                int lda, const double* B, int ldb, double beta, double* C, int ldc);
rr_status fill_f32(cudaStream_t s, int64_t n, float v, float* d);
// Upper bound on the K splits of the plain / split tensor-core products
// (0: none) while an instance is alive on this thread; the batched solver
// sets it around its graph capture.
// Kernel-level timing of the tensor-core product kernel (k_gemm_bf16_tc in
// every role: filter products, split corrections, FP64 emulation passes,
// E4M3 products): while a TcProf is attached to the calling thread, each
// launch is bracketed by CUDA events on its stream and its algorithmic bytes
// (each operand read once, the output written once) are added up.
struct TcProf {
  std::vector<cudaEvent_t> ev;  // start / end per launch
  std::vector<int> role;        // per launch: 0 low-precision product, 1 FP64-emulation pass
  double bytes = 0.0;
  double role_bytes[2] = {0.0, 0.0};
  double role_flops[2] = {0.0, 0.0};
  int launches = 0;
};
void tc_prof_attach(TcProf* p);  // nullptr detaches
// the small pencils' side stream for the caller stream s (created here if new;
// call before capturing work on s)
rr_status pencil_side_prepare(cudaStream_t s);
void pencil_side_release(cudaStream_t s);  // before s is destroyed, its work complete
int& gemm_split_cap();
struct GemmSplitCap {
  int prev;
  explicit GemmSplitCap(int cap) : prev(gemm_split_cap()) { gemm_split_cap() = cap; }
  ~GemmSplitCap() { gemm_split_cap() = prev; }
};
constexpr int kBatchMaxBranches = 64;
constexpr int kBatchSweepBudget = 4096;  // problem-sweeps captured in one graph of the batched SVD
constexpr int kBatchLoopChunk = 16;      // problems per graph with device-side loop control
// E4M3 x E4M3 tensor-core product with row / column scales (k_gemm_tc.cu)
rr_status gemm_e4m3_tc(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const float* rscale,
                       const void* B, int64_t ldb, const float* cscale, float* C, int64_t ldc, cudaStream_t s);
// row-major blocks for the plain Chebyshev filter (k_sparse.cu): transposes
// (pad columns b .. bp - 1 zeroed) and the row-major fused step
rr_status block_to_rows(cudaStream_t s, int32_t t, int64_t n, int64_t b, int64_t bp, const void* src,
                        int64_t ld, void* dst, int64_t ldr);
rr_status block_from_rows(cudaStream_t s, int32_t t, int64_t n, int64_t b, const void* src, int64_t ldr, void* dst,
                          int64_t ld);
rr_status cheb_rows(cudaStream_t s, int64_t n, int64_t b, const int32_t* rp, const int32_t* ci, const float* va,
                    int32_t ytype, const void* Yc, const void* Yp, int64_t ldr, double alpha, double c, double beta,
                    int32_t out_type, void* Yn, int64_t ldn);
rr_status csr_gershgorin(cudaStream_t s, int64_t n, const int32_t* rp, const int32_t* ci,
                         const float* va, double* out2);
}  // namespace rr

namespace rr {
rr_status hessenberg_ex(int32_t arith, int64_t n, int64_t k, void* W, int64_t ldw, int32_t qtype,
                        void* Q, int64_t ldq, int32_t* piv, double tol, void* ws, size_t ws_bytes,
                        cudaStream_t s, int max_grid);
rr_status gram_f32acc(cudaStream_t s, int64_t n, int64_t p, int64_t q, const float* X, int64_t ldx,
                      const float* Y, int64_t ldy, double* G, int64_t ldg, void* ws, size_t ws_bytes);
rr_status sub_lowrank_f32(cudaStream_t s, int64_t n, int64_t b, int64_t p, const float* X, int64_t ldx,
                          const double* K, int64_t ldk, float* T, int64_t ldt);
rr_status cast_f32(cudaStream_t s, int64_t n, int64_t b, const double* X, int64_t ldx, float* Y, int64_t ldy);
rr_status sub_block_f32(cudaStream_t s, int64_t n, int64_t b, const float* P, int64_t ldp, float* T, int64_t ldt);
rr_status tc_take_error(cudaStream_t s);
rr_status tc_prepare_attributes();

// Tensor-core launch of an FP64-emulation product (k_gemm_tc.cu): the sum
// over slice pairs (pair[z] = p0 | q0 << 8 | nq << 16, 0-based) of the A
// slice p0 times B slices q0 (and q0 + 1 when nq = 2), element (row, col)
// scaled by 2^(rexp[row] + cexp[col] - 6 (p0 + 1) - 6 (q0 + nq)); added into
// C64 (ld ldc64) or written as one M x nb partial (ld M) per (pair, K split).
struct TcEmu {
  double* C64;
  int64_t ldc64;
  double* part;
  const int* rexp;
  const int* cexp;
  int nb;
  int a_slices, b_slices;          // slices stacked in the A / B operands
  int a_slice_rows, b_slice_rows;  // rows of one slice in the tensor-map outer dimension
  int npairs;                      // <= 48
  const uint32_t* pair;            // host array
  int max_kchunk;                  // K elements per exact FP32 accumulation
  // > 0: a lift's anti-diagonal products in one launch (pair z codes diagonal
  // d = p0 + 2 of lift_s): A's K range [0, (p0 + 1) lift_k0), B's
  // [(lift_s - 1 - p0) lift_k0, lift_s lift_k0); K = lift_s lift_k0
  int lift_k0, lift_s;
};
rr_status gemm_bf16_tc_emu(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A, int64_t lda,
                           const __nv_bfloat16* B, int64_t ldb, const TcEmu& e, cudaStream_t s);
int tc_emu_partial_splits(int64_t M, int64_t K, int npairs, int max_kchunk);
rr_status gemm_bf16_tc_split(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A_hi,
                             const __nv_bfloat16* A_lo, int64_t lda, const __nv_bfloat16* B_hi,
                             const __nv_bfloat16* B_lo, int64_t ldb, float* C, int64_t ldc,
                             const double* R, int64_t ldr, const double* coef, cudaStream_t s);

// FP64-accurate products on the tensor cores (k_f64emu.cu)
struct EmuOperator {
  int64_t m, n;
  int S;
  __nv_bfloat16* rows;  // S row-scaled slices, row-major (for A X)
  int* rexp;
  __nv_bfloat16* cols;  // S column-scaled slices, column-major (for A^T Y)
  int* cexp;
};
size_t emu_operator_bytes(int64_t m, int64_t n, int S, bool rows, bool cols);
size_t emu_block_bytes(int64_t K, int64_t N, int S);
rr_status emu_prepare(cudaStream_t s, const double* A, int64_t m, int64_t n, int64_t lda, int S,
                      EmuOperator& op, void* mem, bool rows, bool cols);
size_t lift_emu_bytes(int64_t n, int64_t b, int64_t K);
rr_status lift_emu(cudaStream_t s, int64_t n, int64_t b, int32_t t1, const void* S1, int64_t ld1, int64_t p1,
                   int32_t t2, const void* S2, int64_t ld2, int64_t p2, const double* Y, int64_t ldy, double* X,
                   int64_t ldx, void* mem, size_t mem_bytes, bool* done);
rr_status op_prepare(cudaStream_t s, const double* A, int64_t m, int64_t n, int64_t lda,
                     __nv_bfloat16* hi_col, __nv_bfloat16* hi_row, __nv_bfloat16* lo_col, __nv_bfloat16* lo_row,
                     int S, EmuOperator* emu, void* emu_mem, bool rows, bool cols);
rr_status emu_gemm(cudaStream_t s, const EmuOperator& op, int trans, int64_t N, const double* X,
                   int64_t ldx, double* C, int64_t ldc, void* mem);
rr_status vec_scale(cudaStream_t s, int64_t n, double alpha, const double* a, double* d);
bool emu_gram_supported(int64_t n, int64_t p, int64_t q);
size_t emu_gram_bytes(int64_t n, int64_t p, int64_t q);
rr_status emu_gram(cudaStream_t s, int64_t n, int64_t p, int64_t q, int32_t xt, const void* X, int64_t ldx,
                   int32_t yt, const void* Y, int64_t ldy, double* G, int64_t ldg, int accum, void* mem,
                   size_t bytes);
}  // namespace rr
