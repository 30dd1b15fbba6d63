// Dense stages: start-block scaling and casts (Sec. 2 column scaling; Sec. 5.2
// U(0,1) start cast to the working precision), the low-precision block
// product (Sec. 2, X_iter = A X; Fig. 4 "W = AV"), FP64 products and the
// projection Gram products (Alg. 3 / Alg. 5).
#include <atomic>
#include <cstdio>
#include <cstring>

#include "rr_common.cuh"
#include "solver_kernels.cuh"

namespace rr {

static thread_local char g_last_error[512] = "";

void set_last_error(const char* what, cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
}

static std::atomic<uint64_t> g_launches{0};
void note_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

rr_status check_launch(const char* what) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(what, e);
    return RR_ERR_CUDA;
  }
  return RR_OK;
}

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// ---------------------------------------------------------------------------
// a1: column inf-norm scaling + cast
// ---------------------------------------------------------------------------
__global__ void k_colmax_f64(int64_t rows, const double* __restrict__ X, int64_t ldx,
                             double* __restrict__ out) {
  int64_t j = blockIdx.x;
  const double* x = X + j * ldx;
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) m = fmax(m, fabs(x[i]));
  __shared__ double sm[32];
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? sm[threadIdx.x] : 0.0;
    m = warp_max(m);
    if (threadIdx.x == 0) out[j] = m;
  }
}

template <typename TO>
__global__ void k_scale_cast(int64_t rows, int64_t cols, const double* __restrict__ X, int64_t ldx,
                             const double* __restrict__ mx, TO* __restrict__ Y, int64_t ldy) {
  int64_t j = blockIdx.y;
  double m = mx[j];
  if (!(m > 0.0)) m = 1.0;  // zero column stays zero
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x)
    Y[i + j * ldy] = from_f64<TO>(X[i + j * ldx] / m);
}

}  // namespace rr

using namespace rr;

extern "C" const char* rr_last_error(void) { return g_last_error; }
extern "C" uint64_t rr_kernel_launches(void) { return g_launches.load(); }

extern "C" rr_status rr_colscale_cast(int64_t rows, int64_t cols, const double* X, int64_t ldx,
                                      int32_t dtype, void* Y, int64_t ldy, double* scale,
                                      void* stream) {
  if (rows < 0 || cols < 0 || ldx < rows || ldy < rows || !X || !Y) return RR_ERR_ARG;
  if (!scale) return RR_ERR_ARG;  // caller provides the cols-long scale buffer
  if (rows == 0 || cols == 0) return RR_OK;
  cudaStream_t s = as_stream(stream);
  k_colmax_f64<<<(unsigned)cols, 256, 0, s>>>(rows, X, ldx, scale);
  dim3 g((unsigned)std::min<int64_t>((rows + 255) / 256, 1024), (unsigned)cols);
  switch (dtype) {
    case RR_F64: k_scale_cast<double><<<g, 256, 0, s>>>(rows, cols, X, ldx, scale, (double*)Y, ldy); break;
    case RR_F32: k_scale_cast<float><<<g, 256, 0, s>>>(rows, cols, X, ldx, scale, (float*)Y, ldy); break;
    case RR_BF16: k_scale_cast<__nv_bfloat16><<<g, 256, 0, s>>>(rows, cols, X, ldx, scale, (__nv_bfloat16*)Y, ldy); break;
    case RR_E4M3: k_scale_cast<e4m3b_t><<<g, 256, 0, s>>>(rows, cols, X, ldx, scale, (e4m3b_t*)Y, ldy); break;
    default: return RR_ERR_ARG;
  }
  note_launches(1);
  return check_launch("rr_colscale_cast");
}

// ---------------------------------------------------------------------------
// operator cast: FP64 column-major -> dtype column-major (+ row-major copy)
// 32x32 tiles through shared memory so both the read and the transposed
// write are coalesced.
// ---------------------------------------------------------------------------
namespace rr {
template <typename TO>
__global__ void k_cast_operator(int64_t m, int64_t n, const double* __restrict__ A, int64_t lda,
                                TO* __restrict__ out_col, TO* __restrict__ out_row) {
  __shared__ TO tile[32][33];
  int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    int64_t i = i0 + tx, j = j0 + r;
    if (i < m && j < n) {
      TO v = from_f64<TO>(A[i + j * lda]);
      out_col[i + j * m] = v;
      tile[r][tx] = v;
    }
  }
  if (!out_row) return;
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    int64_t i = i0 + r, j = j0 + tx;
    if (i < m && j < n) out_row[i * n + j] = tile[tx][r];
  }
}
}  // namespace rr

namespace rr {
// BF16 residual of the operator cast: lo = bf16(a - bf16(a)), column-major
// and row-major copies (the second half of a split BF16 operator)
__global__ void k_cast_operator_lo(int64_t m, int64_t n, const double* __restrict__ A, int64_t lda,
                                   __nv_bfloat16* __restrict__ out_col, __nv_bfloat16* __restrict__ out_row) {
  __shared__ __nv_bfloat16 tile[32][33];
  int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    int64_t i = i0 + tx, j = j0 + r;
    if (i < m && j < n) {
      const double a = A[i + j * lda];
      const __nv_bfloat16 v = __double2bfloat16(a - (double)__bfloat162float(__double2bfloat16(a)));
      out_col[i + j * m] = v;
      tile[r][tx] = v;
    }
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    int64_t i = i0 + r, j = j0 + tx;
    if (i < m && j < n) out_row[i * n + j] = tile[tx][r];
  }
}

rr_status cast_operator_lo(int64_t m, int64_t n, const double* A, int64_t lda, void* lo_col, void* lo_row,
                           cudaStream_t s) {
  if (m == 0 || n == 0) return RR_OK;
  dim3 g((unsigned)((m + 31) / 32), (unsigned)((n + 31) / 32)), b(32, 8);
  k_cast_operator_lo<<<g, b, 0, s>>>(m, n, A, lda, (__nv_bfloat16*)lo_col, (__nv_bfloat16*)lo_row);
  return check_launch("cast_operator_lo");
}
}  // namespace rr

extern "C" rr_status rr_cast_operator(int64_t m, int64_t n, const double* A, int64_t lda,
                                      int32_t dtype, void* out_col, void* out_row, void* stream) {
  if (m < 0 || n < 0 || lda < m || !A || !out_col) return RR_ERR_ARG;
  if (m == 0 || n == 0) return RR_OK;
  dim3 g((unsigned)((m + 31) / 32), (unsigned)((n + 31) / 32)), b(32, 8);
  cudaStream_t s = as_stream(stream);
  switch (dtype) {
    case RR_F32: k_cast_operator<float><<<g, b, 0, s>>>(m, n, A, lda, (float*)out_col, (float*)out_row); break;
    case RR_BF16:
      return op_prepare(s, A, m, n, lda, (__nv_bfloat16*)out_col, (__nv_bfloat16*)out_row, nullptr, nullptr, 0,
                        nullptr, nullptr, false, false);
    case RR_F64: k_cast_operator<double><<<g, b, 0, s>>>(m, n, A, lda, (double*)out_col, (double*)out_row); break;
    default: return RR_ERR_ARG;
  }
  return check_launch("rr_cast_operator");
}

// ---------------------------------------------------------------------------
// SIMT block product with FP32 accumulation (portable baseline kernel; the
// tcgen05 path in k_gemm_tc.cu takes BF16 shapes it supports)
// C(M x N) = A_k^T B (+ coef_j R(:,j)),  A_k: K x M K-contiguous, B: K x N.
// ---------------------------------------------------------------------------
namespace rr {
constexpr int GBM = 64, GBN = 64, GBK = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_lowp_simt(
    int64_t M, int64_t N, int64_t K, const T* __restrict__ A, int64_t lda,
    const T* __restrict__ B, int64_t ldb, float* __restrict__ C, int64_t ldc,
    const double* __restrict__ R, int64_t ldr, const double* __restrict__ coef) {
  __shared__ float As[GBK][GBM + 1];
  __shared__ float Bs[GBK][GBN + 1];
  int64_t m0 = (int64_t)blockIdx.x * GBM, n0 = (int64_t)blockIdx.y * GBN;
  int tid = threadIdx.x;
  int tm = tid % 16, tn = tid / 16;  // 16 x 16 threads, 4 x 4 outputs each
  float acc[4][4] = {};
  for (int64_t k0 = 0; k0 < K; k0 += GBK) {
    for (int e = tid; e < GBK * GBM; e += 256) {
      int kk = e % GBK, i = e / GBK;
      int64_t gk = k0 + kk, gi = m0 + i;
      As[kk][i] = (gk < K && gi < M) ? Ld<T>::f32(A + gk + gi * lda) : 0.f;
    }
    for (int e = tid; e < GBK * GBN; e += 256) {
      int kk = e % GBK, j = e / GBK;
      int64_t gk = k0 + kk, gj = n0 + j;
      Bs[kk][j] = (gk < K && gj < N) ? Ld<T>::f32(B + gk + gj * ldb) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][tm + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tn + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int64_t j = n0 + tn + 16 * c;
    if (j >= N) continue;
    float cf = (R && coef) ? (float)coef[j] : 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int64_t i = m0 + tm + 16 * r;
      if (i >= M) continue;
      float v = acc[r][c];
      if (R && coef) v += (float)((double)cf * R[i + j * ldr]);
      C[i + j * ldc] = v;
    }
  }
}
}  // namespace rr

// tcgen05 path (k_gemm_tc.cu); returns RR_ERR_ARG when the shape is unsupported
namespace rr {
rr_status gemm_bf16_tc(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A, int64_t lda,
                       const __nv_bfloat16* B, int64_t ldb, float* C, int64_t ldc,
                       const double* R, int64_t ldr, const double* coef, cudaStream_t s);
bool gemm_bf16_tc_supported(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb,
                            const void* A, const void* B);
int& gemm_force_simt();
}  // namespace rr

extern "C" rr_status rr_gemm_lowp_split(int64_t M, int64_t N, int64_t K, const void* A_hi,
                                        const void* A_lo, int64_t lda, const void* B_hi, const void* B_lo,
                                        int64_t ldb, float* C, int64_t ldc, const double* R, int64_t ldr,
                                        const double* coef, void* stream) {
  if (M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldc < M || !C) return RR_ERR_ARG;
  if (!A_hi || !A_lo || !B_hi || !B_lo) return RR_ERR_ARG;
  if (M == 0 || N == 0) return RR_OK;
  if ((R != nullptr) != (coef != nullptr)) return RR_ERR_ARG;
  if (R && ldr < M) return RR_ERR_ARG;
  if (!gemm_bf16_tc_supported(M, N, K, lda, ldb, A_hi, B_hi) ||
      !gemm_bf16_tc_supported(M, N, K, lda, ldb, A_lo, B_lo))
    return RR_ERR_ARG;
  return gemm_bf16_tc_split(M, N, K, (const __nv_bfloat16*)A_hi, (const __nv_bfloat16*)A_lo, lda,
                            (const __nv_bfloat16*)B_hi, (const __nv_bfloat16*)B_lo, ldb, C, ldc, R, ldr,
                            coef, as_stream(stream));
}

extern "C" rr_status rr_gemm_lowp(int32_t dtype, int64_t M, int64_t N, int64_t K, const void* A_k,
                                  int64_t lda, const void* B, int64_t ldb, float* C, int64_t ldc,
                                  const double* R, int64_t ldr, const double* coef, void* stream) {
  if (M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldc < M || !C) return RR_ERR_ARG;
  if (M == 0 || N == 0) return RR_OK;
  if ((R != nullptr) != (coef != nullptr)) return RR_ERR_ARG;
  if (R && ldr < M) return RR_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  if (dtype == RR_BF16 && !gemm_force_simt() &&
      gemm_bf16_tc_supported(M, N, K, lda, ldb, A_k, B))
    return gemm_bf16_tc(M, N, K, (const __nv_bfloat16*)A_k, lda, (const __nv_bfloat16*)B, ldb,
                        C, ldc, R, ldr, coef, s);
  dim3 g((unsigned)((M + GBM - 1) / GBM), (unsigned)((N + GBN - 1) / GBN));
  switch (dtype) {
    case RR_BF16:
      k_gemm_lowp_simt<__nv_bfloat16><<<g, 256, 0, s>>>(M, N, K, (const __nv_bfloat16*)A_k, lda,
                                                         (const __nv_bfloat16*)B, ldb, C, ldc, R, ldr, coef);
      break;
    case RR_F32:
      k_gemm_lowp_simt<float><<<g, 256, 0, s>>>(M, N, K, (const float*)A_k, lda, (const float*)B,
                                                ldb, C, ldc, R, ldr, coef);
      break;
    default: return RR_ERR_ARG;
  }
  return check_launch("rr_gemm_lowp");
}

// ---------------------------------------------------------------------------
// FP64 products C = op(A) B (+C): SIMT, 64 x 64 tiles, 4 x 4 per thread.
// FP64 issue rate, not memory, bounds this on GB300.
// ---------------------------------------------------------------------------
namespace rr {
constexpr int DBM = 64, DBN = 64, DBK = 16;
__global__ void __launch_bounds__(256) k_gemm_f64(
    int trans, int64_t M, int64_t N, int64_t K, const double* __restrict__ A, int64_t lda,
    const double* __restrict__ B, int64_t ldb, double* __restrict__ C, int64_t ldc, int accum) {
  __shared__ double As[DBK][DBM + 1];
  __shared__ double Bs[DBK][DBN + 1];
  int64_t m0 = (int64_t)blockIdx.x * DBM, n0 = (int64_t)blockIdx.y * DBN;
  int tid = threadIdx.x;
  int tm = tid % 16, tn = tid / 16;
  double acc[4][4] = {};
  for (int64_t k0 = 0; k0 < K; k0 += DBK) {
    if (trans) {
      for (int e = tid; e < DBK * DBM; e += 256) {
        int kk = e % DBK, i = e / DBK;
        int64_t gk = k0 + kk, gi = m0 + i;
        As[kk][i] = (gk < K && gi < M) ? A[gk + gi * lda] : 0.0;
      }
    } else {
      for (int e = tid; e < DBK * DBM; e += 256) {
        int i = e % DBM, kk = e / DBM;
        int64_t gk = k0 + kk, gi = m0 + i;
        As[kk][i] = (gk < K && gi < M) ? A[gi + gk * lda] : 0.0;
      }
    }
    for (int e = tid; e < DBK * DBN; e += 256) {
      int kk = e % DBK, j = e / DBK;
      int64_t gk = k0 + kk, gj = n0 + j;
      Bs[kk][j] = (gk < K && gj < N) ? B[gk + gj * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DBK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][tm + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tn + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int64_t j = n0 + tn + 16 * c;
    if (j >= N) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int64_t i = m0 + tm + 16 * r;
      if (i >= M) continue;
      double v = acc[r][c];
      if (accum) v += C[i + j * ldc];
      C[i + j * ldc] = v;
    }
  }
}
}  // namespace rr

extern "C" rr_status rr_gemm_f64(int32_t trans, int64_t M, int64_t N, int64_t K, const double* A,
                                 int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                                 int32_t accumulate, void* stream) {
  if (M < 0 || N < 0 || K < 0 || ldb < K || ldc < M || !C) return RR_ERR_ARG;
  if (trans ? lda < K : lda < M) return RR_ERR_ARG;
  if (M == 0 || N == 0) return RR_OK;
  dim3 g((unsigned)((M + DBM - 1) / DBM), (unsigned)((N + DBN - 1) / DBN));
  k_gemm_f64<<<g, 256, 0, as_stream(stream)>>>(trans, M, N, K, A, lda, B, ldb, C, ldc, accumulate);
  return check_launch("rr_gemm_f64");
}

// ---------------------------------------------------------------------------
// Gram products G = X^T Y for tall X (n x p), Y (n x q), FP64 accumulation,
// split over rows into chunks with deterministic second-pass reduction.
// ---------------------------------------------------------------------------
namespace rr {
constexpr int GT = 32;      // output tile GT x GT
constexpr int GROWS = 32;   // rows per smem stage

template <typename TX, typename TY, typename TA = double>
__global__ void __launch_bounds__(256) k_gram_partial(
    int64_t n, int64_t p, int64_t q, const TX* __restrict__ X, int64_t ldx,
    const TY* __restrict__ Y, int64_t ldy, int64_t rows_per_chunk, double* __restrict__ part) {
  __shared__ TA Xs[GROWS][GT + 1];
  __shared__ TA Ys[GROWS][GT + 1];
  int64_t p0 = (int64_t)blockIdx.x * GT, q0 = (int64_t)blockIdx.y * GT;
  int64_t r0 = (int64_t)blockIdx.z * rows_per_chunk;
  int64_t r1 = r0 + rows_per_chunk < n ? r0 + rows_per_chunk : n;
  int tid = threadIdx.x;
  int ti = tid % 16, tj = tid / 16;  // 2 x 2 outputs per thread
  TA acc[2][2] = {};
  for (int64_t rs = r0; rs < r1; rs += GROWS) {
    for (int e = tid; e < GROWS * GT; e += 256) {
      int rr_ = e % GROWS, c = e / GROWS;
      int64_t row = rs + rr_;
      Xs[rr_][c] = (row < r1 && p0 + c < p) ? LdAs<TA, TX>::get(X + row + (p0 + c) * ldx) : TA(0);
      Ys[rr_][c] = (row < r1 && q0 + c < q) ? LdAs<TA, TY>::get(Y + row + (q0 + c) * ldy) : TA(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr_ = 0; rr_ < GROWS; ++rr_) {
      TA x0 = Xs[rr_][ti], x1 = Xs[rr_][ti + 16];
      TA y0 = Ys[rr_][tj], y1 = Ys[rr_][tj + 16];
      acc[0][0] = fma(x0, y0, acc[0][0]);
      acc[0][1] = fma(x0, y1, acc[0][1]);
      acc[1][0] = fma(x1, y0, acc[1][0]);
      acc[1][1] = fma(x1, y1, acc[1][1]);
    }
    __syncthreads();
  }
  double* out = part + (size_t)blockIdx.z * p * q;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int64_t i = p0 + ti + 16 * a, j = q0 + tj + 16 * b;
      if (i < p && j < q) out[i + j * p] = (double)acc[a][b];
    }
}

__global__ void k_gram_reduce(int64_t p, int64_t q, int64_t chunks, const double* __restrict__ part,
                              double* __restrict__ G, int64_t ldg, int accum) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= p * q) return;
  double s = 0.0;
  for (int64_t c = 0; c < chunks; ++c) s += part[c * p * q + e];
  int64_t i = e % p, j = e / p;
  if (accum) s += G[i + j * ldg];
  G[i + j * ldg] = s;
}

static int64_t gram_chunks(int64_t n, int64_t p, int64_t q) {
  int64_t tiles = ((p + GT - 1) / GT) * ((q + GT - 1) / GT);
  int64_t want = (4 * (int64_t)num_sms() + tiles - 1) / tiles;
  int64_t maxc = (n + 255) / 256;
  int64_t c = want < maxc ? want : maxc;
  return c < 1 ? 1 : c;
}
}  // namespace rr

// Workspace: the SIMT path's split-K partials, or the tensor-core path's
// slices and partials when the shape qualifies (for q > 128 the calls with
// q' <= 128 columns qualify)
extern "C" size_t rr_gram_workspace_size(int64_t n, int64_t p, int64_t q) {
  size_t b = align_up((size_t)gram_chunks(n, p, q) * p * q * sizeof(double)) + 256;
  const int64_t qe = q < 128 ? q : 128;
  if (emu_gram_supported(n, p, qe)) {
    const size_t e = emu_gram_bytes(n, p, qe);
    if (e > b) b = e;
  }
  return b;
}

namespace rr {
template <typename TX>
static rr_status gram_dispatch_y(int32_t ytype, dim3 g, cudaStream_t s, int64_t n, int64_t p,
                                 int64_t q, const TX* X, int64_t ldx, const void* Y, int64_t ldy,
                                 int64_t rpc, double* part) {
  switch (ytype) {
    case RR_F64: k_gram_partial<TX, double><<<g, 256, 0, s>>>(n, p, q, X, ldx, (const double*)Y, ldy, rpc, part); break;
    case RR_F32: k_gram_partial<TX, float><<<g, 256, 0, s>>>(n, p, q, X, ldx, (const float*)Y, ldy, rpc, part); break;
    case RR_BF16: k_gram_partial<TX, __nv_bfloat16><<<g, 256, 0, s>>>(n, p, q, X, ldx, (const __nv_bfloat16*)Y, ldy, rpc, part); break;
    case RR_E4M3: k_gram_partial<TX, e4m3b_t><<<g, 256, 0, s>>>(n, p, q, X, ldx, (const e4m3b_t*)Y, ldy, rpc, part); break;
    default: return RR_ERR_ARG;
  }
  return RR_OK;
}
}  // namespace rr

namespace rr {
// FP32 Gram partials for tall blocks (the refinement's projection of the
// Ritz vectors out of a correction block): a CTA takes a 64 x 64 tile of
// X^T Y over one chunk of rows, 4 x 4 outputs per thread; the chunk's 32 rows
// of both tiles are staged in shared memory row by row (a row's 64 values
// contiguous), so a thread reads its 4 X and 4 Y values as two 16-byte loads
// per 16 FMAs.  part[chunk][i + j p] (FP64, summed by k_gram_reduce).
constexpr int kG32 = 64, kG32R = 32;
__global__ void __launch_bounds__(256) k_gram32(int64_t n, int64_t p, int64_t q, const float* __restrict__ X,
                                                int64_t ldx, const float* __restrict__ Y, int64_t ldy, int64_t rpc,
                                                double* __restrict__ part) {
  // rows padded by 4 floats: the column-wise staging stores meet 4-way
  // instead of 32-way bank conflicts, the 16-byte row loads stay aligned
  __shared__ __align__(16) float Xs[kG32R][kG32 + 4];
  __shared__ __align__(16) float Ys[kG32R][kG32 + 4];
  const int64_t p0 = (int64_t)blockIdx.x * kG32, q0 = (int64_t)blockIdx.y * kG32;
  const int64_t r0 = (int64_t)blockIdx.z * rpc, r1 = r0 + rpc < n ? r0 + rpc : n;
  const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4;  // outputs 4 ti.., 4 tj..
  float acc[4][4] = {};
  for (int64_t rs = r0; rs < r1; rs += kG32R) {
    // stage: thread e loads row (e % 32) of column (e / 32) of both tiles (rows contiguous in HBM)
    for (int e = tid; e < kG32R * kG32; e += 256) {
      const int rr_ = e % kG32R, c = e / kG32R;
      const int64_t row = rs + rr_;
      Xs[rr_][c] = (row < r1 && p0 + c < p) ? X[row + (p0 + c) * ldx] : 0.f;
      Ys[rr_][c] = (row < r1 && q0 + c < q) ? Y[row + (q0 + c) * ldy] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr_ = 0; rr_ < kG32R; ++rr_) {
      const float4 xv = reinterpret_cast<const float4*>(&Xs[rr_][0])[ti];
      const float4 yv = reinterpret_cast<const float4*>(&Ys[rr_][0])[tj];
      const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, ya[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(xa[a], ya[c], acc[a][c]);
    }
    __syncthreads();
  }
  double* out = part + (size_t)blockIdx.z * p * q;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t i = p0 + 4 * ti + a, j = q0 + 4 * tj + c;
      if (i < p && j < q) out[i + j * p] = (double)acc[a][c];
    }
}

// The same partials with the whole p x q result in one CTA (p, q <= TP =
// 16 PT): every row of X and Y is read once.  A thread owns PT x PT outputs
// (rows 2 ti + 32 a' + {0, 1} of G, a' < PT / 2, and columns PT tj ..); each
// staged row gives it PT X values (8-byte shared loads, 16 distinct per
// warp: one wavefront) and PT Y values (broadcast 8-byte loads) per PT^2
// FMAs, issued as packed FP32 pairs (each component rounded as one fmaf),
// and the next rows' global loads are issued before the current rows are
// used.
template <int PT>
__global__ void __launch_bounds__(256, 1) k_gram32_full(int64_t n, int p, int q, const float* __restrict__ X,
                                                        int64_t ldx, const float* __restrict__ Y, int64_t ldy,
                                                        int64_t rpc, double* __restrict__ part) {
  constexpr int TP = 16 * PT, R = 16;
  __shared__ __align__(16) float Xs[R][TP + 2];
  __shared__ __align__(16) float Ys[R][TP + 2];
  const int64_t r0 = (int64_t)blockIdx.x * rpc, r1 = r0 + rpc < n ? r0 + rpc : n;
  const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4;
  static_assert(PT % 2 == 0, "column pairs");
  float2 acc[PT][PT / 2];
#pragma unroll
  for (int a = 0; a < PT; ++a)
#pragma unroll
    for (int c = 0; c < PT / 2; ++c) acc[a][c] = make_float2(0.f, 0.f);
  // staging: R rows x TP columns of each operand, thread e -> (row e % R, column e / R)
  constexpr int PER = R * TP / 256;
  float xr[PER], yr[PER];
  auto fetch = [&](int64_t rs) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + 256 * u, rr_ = e % R, c = e / R;
      const int64_t row = rs + rr_;
      xr[u] = (row < r1 && c < p) ? X[row + c * ldx] : 0.f;
      yr[u] = (row < r1 && c < q) ? Y[row + c * ldy] : 0.f;
    }
  };
  fetch(r0);
  for (int64_t rs = r0; rs < r1; rs += R) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + 256 * u, rr_ = e % R, c = e / R;
      Xs[rr_][c] = xr[u];
      Ys[rr_][c] = yr[u];
    }
    __syncthreads();
    if (rs + R < r1) fetch(rs + R);  // in flight while the tile is used
#pragma unroll 2
    for (int rr_ = 0; rr_ < R; ++rr_) {
      float xa[PT];
      float2 ya[PT / 2];
#pragma unroll
      for (int a = 0; a < PT; a += 2) {
        const float2 xv = *reinterpret_cast<const float2*>(&Xs[rr_][2 * ti + 16 * a]);
        xa[a] = xv.x;
        xa[a + 1] = xv.y;
      }
#pragma unroll
      for (int c = 0; c < PT / 2; ++c) ya[c] = *reinterpret_cast<const float2*>(&Ys[rr_][PT * tj + 2 * c]);
#pragma unroll
      for (int a = 0; a < PT; ++a) {
        const float2 xx = make_float2(xa[a], xa[a]);
#pragma unroll
        for (int c = 0; c < PT / 2; ++c) acc[a][c] = __ffma2_rn(xx, ya[c], acc[a][c]);
      }
    }
  }
  double* out = part + (size_t)blockIdx.x * p * q;
#pragma unroll
  for (int a = 0; a < PT; ++a)
#pragma unroll
    for (int c = 0; c < PT; ++c) {
      const int i = 2 * ti + 16 * (a & ~1) + (a & 1), j = PT * tj + c;
      if (i < p && j < q) out[i + (int64_t)j * p] = (double)((c & 1) ? acc[a][c >> 1].y : acc[a][c >> 1].x);
    }
}

// G = X^T Y with FP32 products and FP32 accumulation per row chunk (chunk
// sums added in FP64), X and Y FP32, where FP32 accuracy is all the caller
// needs.
rr_status gram_f32acc(cudaStream_t s, int64_t n, int64_t p, int64_t q, const float* X, int64_t ldx,
                      const float* Y, int64_t ldy, double* G, int64_t ldg, void* ws, size_t ws_bytes) {
  if (p == 0 || q == 0) return RR_OK;
  if (!ws) return RR_ERR_WORKSPACE;
  const int64_t fitc = (int64_t)(ws_bytes / ((size_t)p * q * sizeof(double)));
  if (p <= 160 && q <= 160 && n >= 64 * 1024 && fitc >= num_sms()) {
    // tall blocks: one CTA per row chunk holds the whole product
    const int64_t chunks = num_sms();
    const int64_t rpc = ((n + chunks - 1) / chunks + 15) / 16 * 16;
    const int64_t used = (n + rpc - 1) / rpc;
    if (p <= 128 && q <= 128)
      k_gram32_full<8><<<(unsigned)used, 256, 0, s>>>(n, (int)p, (int)q, X, ldx, Y, ldy, rpc, (double*)ws);
    else
      k_gram32_full<10><<<(unsigned)used, 256, 0, s>>>(n, (int)p, (int)q, X, ldx, Y, ldy, rpc, (double*)ws);
    RR_TRY(check_launch("gram_f32acc partial"));
    k_gram_reduce<<<(unsigned)((p * q + 255) / 256), 256, 0, s>>>(p, q, used, (const double*)ws, G, ldg, 0);
    return check_launch("gram_f32acc reduce");
  }
  const int64_t tiles = ((p + kG32 - 1) / kG32) * ((q + kG32 - 1) / kG32);
  int64_t chunks = (2 * (int64_t)num_sms() + tiles - 1) / tiles;
  const int64_t fit = (int64_t)(ws_bytes / ((size_t)p * q * sizeof(double)));
  if (chunks > fit) chunks = fit;
  if (chunks > (n + kG32R - 1) / kG32R) chunks = (n + kG32R - 1) / kG32R;
  if (chunks < 1) return RR_ERR_WORKSPACE;
  int64_t rpc = (n + chunks - 1) / chunks;
  rpc = (rpc + kG32R - 1) / kG32R * kG32R;
  chunks = (n + rpc - 1) / rpc;
  dim3 g((unsigned)((p + kG32 - 1) / kG32), (unsigned)((q + kG32 - 1) / kG32), (unsigned)chunks);
  k_gram32<<<g, 256, 0, s>>>(n, p, q, X, ldx, Y, ldy, rpc, (double*)ws);
  RR_TRY(check_launch("gram_f32acc partial"));
  k_gram_reduce<<<(unsigned)((p * q + 255) / 256), 256, 0, s>>>(p, q, chunks, (const double*)ws, G, ldg, 0);
  return check_launch("gram_f32acc reduce");
}
}  // namespace rr

extern "C" rr_status rr_gram(int64_t n, int64_t p, int64_t q, int32_t xtype, const void* X,
                             int64_t ldx, int32_t ytype, const void* Y, int64_t ldy, double* G,
                             int64_t ldg, int32_t accumulate, void* ws, size_t ws_bytes,
                             void* stream) {
  if (n < 0 || p < 0 || q < 0 || ldx < n || ldy < n || ldg < p || !G) return RR_ERR_ARG;
  auto valid = [](int32_t t) { return t == RR_F64 || t == RR_F32 || t == RR_BF16 || t == RR_E4M3; };
  if (!valid(xtype) || !valid(ytype)) return RR_ERR_ARG;
  if (p == 0 || q == 0) return RR_OK;
  cudaStream_t s = as_stream(stream);
  if (n == 0) {
    if (!accumulate)
      for (int64_t j = 0; j < q; ++j) RR_CUDA(cudaMemsetAsync(G + j * ldg, 0, p * sizeof(double), s));
    return RR_OK;
  }
  // FP64-accurate products on the tensor cores when the shape qualifies and
  // the workspace holds the slices
  if (emu_gram_supported(n, p, q) && ws && ws_bytes >= emu_gram_bytes(n, p, q))
    return emu_gram(s, n, p, q, xtype, X, ldx, ytype, Y, ldy, G, ldg, accumulate, ws, ws_bytes);
  // wider Y: the same products on column chunks of at most 128
  constexpr int64_t kQc = 128;
  if (q > kQc && emu_gram_supported(n, p, kQc) && ws && ws_bytes >= emu_gram_bytes(n, p, kQc)) {
    const size_t ys = dtype_size(ytype);
    for (int64_t j0 = 0; j0 < q; j0 += kQc) {
      const int64_t qc = std::min<int64_t>(kQc, q - j0);
      RR_TRY(emu_gram(s, n, p, qc, xtype, X, ldx, ytype, (const char*)Y + (size_t)j0 * ldy * ys, ldy, G + j0 * ldg,
                      ldg, accumulate, ws, ws_bytes));
    }
    return RR_OK;
  }
  int64_t chunks = gram_chunks(n, p, q);
  if (ws_bytes < (size_t)chunks * p * q * sizeof(double) || !ws) return RR_ERR_WORKSPACE;
  int64_t rpc = (n + chunks - 1) / chunks;
  chunks = (n + rpc - 1) / rpc;
  double* part = (double*)ws;
  dim3 g((unsigned)((p + GT - 1) / GT), (unsigned)((q + GT - 1) / GT), (unsigned)chunks);
  rr_status st;
  switch (xtype) {
    case RR_F64: st = gram_dispatch_y<double>(ytype, g, s, n, p, q, (const double*)X, ldx, Y, ldy, rpc, part); break;
    case RR_F32: st = gram_dispatch_y<float>(ytype, g, s, n, p, q, (const float*)X, ldx, Y, ldy, rpc, part); break;
    case RR_BF16: st = gram_dispatch_y<__nv_bfloat16>(ytype, g, s, n, p, q, (const __nv_bfloat16*)X, ldx, Y, ldy, rpc, part); break;
    case RR_E4M3: st = gram_dispatch_y<e4m3b_t>(ytype, g, s, n, p, q, (const e4m3b_t*)X, ldx, Y, ldy, rpc, part); break;
    default: return RR_ERR_ARG;
  }
  if (st != RR_OK) return st;
  RR_TRY(check_launch("rr_gram partial"));
  k_gram_reduce<<<(unsigned)((p * q + 255) / 256), 256, 0, s>>>(p, q, chunks, part, G, ldg, accumulate);
  return check_launch("rr_gram reduce");
}

// ---------------------------------------------------------------------------
// rr_gram_noalloc: the Gram product for callers that cannot allocate device
// memory.  Its split-K partial sums live in a fixed array compiled into the
// library instead of a caller-provided workspace.
// ---------------------------------------------------------------------------
#include <cuda.h>
#include <mutex>

namespace rr {

// Scratch of rr_gram_noalloc: 2 MiB of FP64 partial sums per GPU, held by
// every GPU that loads the library until the process exits.
constexpr size_t kNoAllocDoubles = (size_t)1 << 18;
static __device__ __align__(256) double g_gram_scratch[kNoAllocDoubles];

// Device address of g_gram_scratch in the current context.  Host code may
// not use the symbol itself as a device pointer, so the address is looked up
// with cudaGetSymbolAddress and cached per device together with the context
// it was taken in: after a device reset (a new primary context, the module
// loaded again) the context differs and the address is looked up afresh
// instead of reusing a pointer into memory that no longer exists.
// (cuCtxGetCurrent is taken through the runtime's driver entry-point lookup,
// so the library keeps no load-time dependency on the driver library.)
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
static CUcontext current_context() {
  static CtxGetCurrentFn fn = []() -> CtxGetCurrentFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return (CtxGetCurrentFn)p;
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

static rr_status noalloc_scratch(double** out) {
  static std::mutex mu;
  static double* addr[64] = {};
  static CUcontext ctx_of[64] = {};
  int dev = 0;
  RR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RR_ERR_ARG;
  std::lock_guard<std::mutex> lk(mu);
  CUcontext cur = current_context();
  if (!addr[dev] || !cur || cur != ctx_of[dev]) {
    void* p = nullptr;
    RR_CUDA(cudaGetSymbolAddress(&p, g_gram_scratch));
    addr[dev] = (double*)p;
    ctx_of[dev] = current_context();
  }
  *out = addr[dev];
  return RR_OK;
}

}  // namespace rr

extern "C" rr_status rr_gram_noalloc(int64_t n, int64_t p, int64_t q, int32_t xtype, const void* X,
                                     int64_t ldx, int32_t ytype, const void* Y, int64_t ldy, double* G,
                                     int64_t ldg, int32_t accumulate, void* stream) {
  if (n < 0 || p < 0 || q < 0 || ldx < n || ldy < n || ldg < p || !G) return RR_ERR_ARG;
  if ((size_t)p * (size_t)q > kNoAllocDoubles) return RR_ERR_ARG;  // beyond the fixed scratch
  auto valid = [](int32_t t) { return t == RR_F64 || t == RR_F32 || t == RR_BF16 || t == RR_E4M3; };
  if (!valid(xtype) || !valid(ytype)) return RR_ERR_ARG;              // as rr_gram
  if (p == 0 || q == 0) return RR_OK;
  if (n > 0 && (!X || !Y)) return RR_ERR_ARG;
  double* scratch = nullptr;
  RR_TRY(noalloc_scratch(&scratch));
  cudaStream_t s = as_stream(stream);
  if (n == 0) {
    if (!accumulate)
      for (int64_t j = 0; j < q; ++j) RR_CUDA(cudaMemsetAsync(G + j * ldg, 0, p * sizeof(double), s));
    return RR_OK;
  }
  // as many row chunks as the scratch holds (every slot used is written by
  // the partial kernel before the reduction reads it: nothing to clear)
  int64_t chunks = gram_chunks(n, p, q);
  const int64_t cap = (int64_t)(kNoAllocDoubles / ((size_t)p * (size_t)q));
  if (chunks > cap) chunks = cap;
  int64_t rpc = (n + chunks - 1) / chunks;
  chunks = (n + rpc - 1) / rpc;
  dim3 g((unsigned)((p + GT - 1) / GT), (unsigned)((q + GT - 1) / GT), (unsigned)chunks);
  rr_status st;
  switch (xtype) {
    case RR_F64: st = gram_dispatch_y<double>(ytype, g, s, n, p, q, (const double*)X, ldx, Y, ldy, rpc, scratch); break;
    case RR_F32: st = gram_dispatch_y<float>(ytype, g, s, n, p, q, (const float*)X, ldx, Y, ldy, rpc, scratch); break;
    case RR_BF16: st = gram_dispatch_y<__nv_bfloat16>(ytype, g, s, n, p, q, (const __nv_bfloat16*)X, ldx, Y, ldy, rpc, scratch); break;
    case RR_E4M3: st = gram_dispatch_y<e4m3b_t>(ytype, g, s, n, p, q, (const e4m3b_t*)X, ldx, Y, ldy, rpc, scratch); break;
    default: return RR_ERR_ARG;
  }
  if (st != RR_OK) return st;
  RR_TRY(check_launch("rr_gram_noalloc partial"));
  k_gram_reduce<<<(unsigned)((p * q + 255) / 256), 256, 0, s>>>(p, q, chunks, scratch, G, ldg, accumulate);
  return check_launch("rr_gram_noalloc reduce");
}
