// Matrix-free Gaussian kernel operator (Sec. 2's kernel-matrix family, the
// setups of the kernel-matrix experiments in Sec. 5):
//   A(i, j) = f (exp(-|x_i - y_j|^2 / (2 l^2)) + s [i == j])
// over points x_i (rows) and y_j (columns) in d dimensions; the shift s only
// on a square operator whose two point sets are the same.  The product
//   Y = op(A) X (+ coef_j R(:, j)),  op(A) = A or A^T
// evaluates each entry where it is used and never stores A: a CTA takes 128
// output rows, walks the columns in tiles of 32 points, computes the 128 x 32
// tile of A in shared memory (each entry once: d subtractions and squares, one
// exponential) and accumulates the tile times the matching 32 rows of X,
// 2 rows x 16 output columns per thread (16-byte shared-memory loads of X).  Work per entry: one exponential and 2 b
// multiply-adds, against 8 bytes per point row read once per tile: bound by
// the exponential unit and the FMA pipe, not by memory.  FP32 evaluation for
// the low-precision products, FP64 for the FP64-accurate ones.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "rr_common.cuh"
#include "solver_kernels.cuh"

namespace rr {
namespace {

constexpr int kKR = 128;  // output rows per CTA (2 per thread)
// columns (points) per tile: 32 in FP32, 16 in FP64 (static shared memory)
template <typename TC> constexpr int kcols() { return sizeof(TC) == 8 ? 16 : 32; }
constexpr int kKB = 64;   // output columns per pass (16 per thread)
constexpr int kKD = 8;    // largest point dimension

template <typename T> __device__ __forceinline__ T kexp(T x);
template <> __device__ __forceinline__ float kexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double kexp<double>(double x) { return exp(x); }

template <typename TX> __device__ __forceinline__ float ldx_f(const TX* p);
template <> __device__ __forceinline__ float ldx_f<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ldx_f<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <> __device__ __forceinline__ float ldx_f<double>(const double* p) { return (float)*p; }

template <typename TC, typename TX>
__device__ __forceinline__ TC load_x(const TX* p) {
  if constexpr (std::is_same<TC, double>::value) {
    if constexpr (std::is_same<TX, double>::value) return *p;
    else return (double)ldx_f<TX>(p);
  } else {
    return ldx_f<TX>(p);
  }
}

// 16 consecutive values of a shared-memory row (16-byte aligned) into registers
__device__ __forceinline__ void ld16(const float* p, float (&v)[16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 t = reinterpret_cast<const float4*>(p)[q];
    v[4 * q] = t.x;
    v[4 * q + 1] = t.y;
    v[4 * q + 2] = t.z;
    v[4 * q + 3] = t.w;
  }
}
__device__ __forceinline__ void ld16(const double* p, double (&v)[16]) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double2 t = reinterpret_cast<const double2*>(p)[q];
    v[2 * q] = t.x;
    v[2 * q + 1] = t.y;
  }
}

template <typename TC, typename TX, typename TO, int kKC = kcols<TC>()>
__global__ void __launch_bounds__(256) k_kernel_mv(int64_t rows, int64_t cols, int d, const double* __restrict__ P,
                                                   int64_t ldp, const double* __restrict__ Q, int64_t ldq, TC f,
                                                   TC inv2l2, TC shift, int square, int b, const TX* __restrict__ X,
                                                   int64_t ldx, TO* __restrict__ Y, int64_t ldy,
                                                   const double* __restrict__ R, int64_t ldr,
                                                   const double* __restrict__ coef) {
  __shared__ TC sq[kKC][kKD];                       // the column tile's points
  __shared__ TC sa[kKC][kKR + 1];                   // A tile, transposed (column j, row r)
  __shared__ __align__(16) TC sx[kKC][kKB];         // X rows of the tile, this pass's columns
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * kKR;
  const int c0 = blockIdx.y * kKB;
  const int nb = min(kKB, b - c0);
  // this thread: rows r0 + lr and r0 + lr + 64, columns c0 + 16 cg .. + 15;
  // it evaluates the A-tile entries of its two rows in tile columns cg + 4 t
  const int lr = tid & 63, cg = tid >> 6;
  TC pr[2][kKD];
  int64_t gr[2] = {r0 + lr, r0 + lr + 64};
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int t = 0; t < kKD; ++t) pr[h][t] = (t < d && gr[h] < rows) ? (TC)P[gr[h] + (int64_t)t * ldp] : TC(0);
  TC acc[2][16];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[h][c] = TC(0);
  for (int64_t j0 = 0; j0 < cols; j0 += kKC) {
    const int nc = cols - j0 < kKC ? (int)(cols - j0) : kKC;
    __syncthreads();
    for (int e = tid; e < kKC * d; e += 256) {
      const int j = e / d, t = e % d;
      sq[j][t] = j < nc ? (TC)Q[(j0 + j) + (int64_t)t * ldq] : TC(0);
    }
    for (int e = tid; e < kKC * kKB; e += 256) {
      const int j = e / kKB, c = e % kKB;
      sx[j][c] = (j < nc && c < nb) ? load_x<TC, TX>(X + (j0 + j) + (int64_t)(c0 + c) * ldx) : TC(0);
    }
    __syncthreads();
#pragma unroll
    for (int t8 = 0; t8 < kKC / 4; ++t8) {
      const int j = cg + 4 * t8;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        TC dist = TC(0);
#pragma unroll
        for (int t = 0; t < kKD; ++t) {
          if (t < d) {
            const TC df = pr[h][t] - sq[j][t];
            dist += df * df;
          }
        }
        TC a = kexp<TC>(-dist * inv2l2);
        if (square && gr[h] == j0 + j) a += shift;
        sa[j][lr + 64 * h] = (j < nc && gr[h] < rows) ? f * a : TC(0);
      }
    }
    __syncthreads();
    for (int j = 0; j < nc; ++j) {
      TC xv[16];
      ld16(&sx[j][cg * 16], xv);
      const TC a0 = sa[j][lr], a1 = sa[j][lr + 64];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        acc[0][c] += a0 * xv[c];
        acc[1][c] += a1 * xv[c];
      }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (gr[h] >= rows) continue;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int col = c0 + cg * 16 + c;
      if (col >= b) break;
      TC v = acc[h][c];
      if (R && coef) v += (TC)(coef[col] * R[gr[h] + (int64_t)col * ldr]);
      Y[gr[h] + (int64_t)col * ldy] = (TO)v;
    }
  }
}

template <typename TC, typename TX, typename TO>
rr_status launch_kernel_mv(cudaStream_t s, int64_t rows, int64_t cols, int d, const double* P, int64_t ldp,
                           const double* Q, int64_t ldq, double f, double l, double shift, int square, int64_t b,
                           const TX* X, int64_t ldx, TO* Y, int64_t ldy, const double* R, int64_t ldr,
                           const double* coef) {
  dim3 g((unsigned)((rows + kKR - 1) / kKR), (unsigned)((b + kKB - 1) / kKB));
  k_kernel_mv<TC, TX, TO><<<g, 256, 0, s>>>(rows, cols, d, P, ldp, Q, ldq, (TC)f, (TC)(1.0 / (2.0 * l * l)),
                                            (TC)shift, square, (int)b, X, ldx, Y, ldy, R, ldr, coef);
  return check_launch("kernel operator product");
}

template <typename TC, typename TX>
rr_status dispatch_out(cudaStream_t s, int32_t otype, int64_t rows, int64_t cols, int d, const double* P,
                       int64_t ldp, const double* Q, int64_t ldq, double f, double l, double shift, int square,
                       int64_t b, const TX* X, int64_t ldx, void* Y, int64_t ldy, const double* R, int64_t ldr,
                       const double* coef) {
  switch (otype) {
    case RR_F32:
      return launch_kernel_mv<TC, TX, float>(s, rows, cols, d, P, ldp, Q, ldq, f, l, shift, square, b, X, ldx,
                                             (float*)Y, ldy, R, ldr, coef);
    case RR_F64:
      return launch_kernel_mv<TC, TX, double>(s, rows, cols, d, P, ldp, Q, ldq, f, l, shift, square, b, X, ldx,
                                              (double*)Y, ldy, R, ldr, coef);
  }
  return RR_ERR_ARG;
}

}  // namespace

// Y = op(A) X (+ coef R) for a kernel operator (internal form used by the
// solver; the C entry below checks its arguments)
rr_status kernel_apply(cudaStream_t s, const rr_operator* A, int trans, int64_t b, int32_t xtype, const void* X,
                       int64_t ldx, int32_t otype, void* Y, int64_t ldy, const double* R, int64_t ldr,
                       const double* coef) {
  const double* px = (const double*)A->values;
  const double* py = A->points_y ? A->points_y : px;
  const int64_t ldpx = A->ld, ldpy = A->points_y ? A->n : A->ld;
  const bool square = A->points_y == nullptr;
  const int d = (int)A->nnz;
  const double f = A->kparams[0], l = A->kparams[1], sh = square ? A->kparams[2] : 0.0;
  const int64_t rows = trans ? A->n : A->m, cols = trans ? A->m : A->n;
  const double* P = trans ? py : px;
  const double* Q = trans ? px : py;
  const int64_t ldp = trans ? ldpy : ldpx, ldq = trans ? ldpx : ldpy;
  if (b == 0 || rows == 0) return RR_OK;
  const bool f64 = xtype == RR_F64 || otype == RR_F64;
  if (f64) {
    switch (xtype) {
      case RR_F64: return dispatch_out<double, double>(s, otype, rows, cols, d, P, ldp, Q, ldq, f, l, sh, square, b,
                                                       (const double*)X, ldx, Y, ldy, R, ldr, coef);
      case RR_F32: return dispatch_out<double, float>(s, otype, rows, cols, d, P, ldp, Q, ldq, f, l, sh, square, b,
                                                      (const float*)X, ldx, Y, ldy, R, ldr, coef);
      case RR_BF16:
        return dispatch_out<double, __nv_bfloat16>(s, otype, rows, cols, d, P, ldp, Q, ldq, f, l, sh, square, b,
                                                   (const __nv_bfloat16*)X, ldx, Y, ldy, R, ldr, coef);
    }
    return RR_ERR_ARG;
  }
  switch (xtype) {
    case RR_F32: return dispatch_out<float, float>(s, otype, rows, cols, d, P, ldp, Q, ldq, f, l, sh, square, b,
                                                   (const float*)X, ldx, Y, ldy, R, ldr, coef);
    case RR_BF16: return dispatch_out<float, __nv_bfloat16>(s, otype, rows, cols, d, P, ldp, Q, ldq, f, l, sh,
                                                            square, b, (const __nv_bfloat16*)X, ldx, Y, ldy, R,
                                                            ldr, coef);
  }
  return RR_ERR_ARG;
}

rr_status check_kernel_operator(const rr_operator* A) {
  if (!A || A->kind != RR_KERNEL || A->dtype != RR_F64 || !A->values) return RR_ERR_ARG;
  if (A->m <= 0 || A->n <= 0 || A->ld < A->m || A->nnz < 1 || A->nnz > kKD) return RR_ERR_ARG;
  if (!(A->kparams[1] > 0.0) || !std::isfinite(A->kparams[0]) || !std::isfinite(A->kparams[2])) return RR_ERR_ARG;
  if (!A->points_y && A->m != A->n) return RR_ERR_ARG;
  return RR_OK;
}

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_kernel_apply(int32_t trans, const rr_operator* A, int64_t b, int32_t xtype, const void* X,
                                     int64_t ldx, int32_t otype, void* Y, int64_t ldy, const double* R, int64_t ldr,
                                     const double* coef, void* stream) {
  RR_TRY(check_kernel_operator(A));
  const int64_t cols = trans ? A->m : A->n, rows = trans ? A->n : A->m;
  if (b < 0 || !X || !Y || ldx < cols || ldy < rows || (R && ldr < rows) || (R && !coef)) return RR_ERR_ARG;
  if (xtype != RR_F64 && xtype != RR_F32 && xtype != RR_BF16) return RR_ERR_ARG;
  if (otype != RR_F64 && otype != RR_F32) return RR_ERR_ARG;
  return kernel_apply(as_stream(stream), A, trans, b, xtype, X, ldx, otype, Y, ldy, R, ldr, coef);
}
