// Matrix-free Gaussian kernel operator (Sec. 2's kernel-matrix family, the
// setups of the kernel-matrix experiments in Sec. 5):
//   A(i, j) = f (exp(-|x_i - y_j|^2 / (2 l^2)) + s [i == j])
// over points x_i (rows) and y_j (columns) in d dimensions; the shift s only
// on a square operator whose two point sets are the same.  The product
//   Y = op(A) X (+ coef_j R(:, j)),  op(A) = A or A^T
// evaluates each entry where it is used and never stores A: a CTA takes 128
// or 256 output rows (64 or 32 output columns per pass), walks the
// columns in tiles of 32 points (16 in FP64), computes that tile of A in
// shared memory (each entry once: d subtractions and squares, one
// exponential) and accumulates the tile times the matching rows of X, 2 rows
// x 16 output columns per thread (16-byte shared-memory loads of X).  Small
// grids split the points over CTAs and add their partial sums atomically.  Work per entry: one exponential and 2 b
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

// output rows per CTA: 2 per thread, 256 / CG threads per column group
// columns (points) per tile: 32 in FP32, 16 in FP64 (static shared memory)
template <typename TC> constexpr int kcols() { return sizeof(TC) == 8 ? 16 : 32; }
// output columns per pass: 16 per thread, CG column groups (CG = 1, 2 or 4:
// b up to 16, 32 or 64 per pass)
constexpr int kKD = 8;    // largest point dimension

template <typename T> __device__ __forceinline__ T kexp(T x);
template <> __device__ __forceinline__ float kexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double kexp<double>(double x) { return exp(x); }

template <typename TX> __device__ __forceinline__ float ldx_f(const TX* p);
template <> __device__ __forceinline__ float ldx_f<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ldx_f<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

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

template <typename TC, typename TX, typename TO, int CG, int kKC = kcols<TC>()>
__global__ void __launch_bounds__(256) k_kernel_mv(int64_t rows, int64_t cols, int d, const double* __restrict__ P,
                                                   int64_t ldp, const double* __restrict__ Q, int64_t ldq, TC f,
                                                   TC inv2l2, TC shift, int square, int b, const TX* __restrict__ X,
                                                   int64_t ldx, TO* __restrict__ Y, int64_t ldy,
                                                   const double* __restrict__ R, int64_t ldr,
                                                   const double* __restrict__ coef, int64_t jspan) {
  constexpr int TR = 256 / CG;      // threads per column group (rows / 2)
  constexpr int kKR = 2 * TR;       // output rows per CTA
  constexpr int kKB = 16 * CG;      // output columns per pass
  __shared__ TC sq[kKC][kKD];                       // the column tile's points
  __shared__ TC sa[kKC][kKR + 1];                   // A tile, transposed (column j, row r)
  __shared__ __align__(16) TC sx[kKC][kKB];         // X rows of the tile, this pass's columns
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * kKR;
  const int c0 = blockIdx.y * kKB;
  const int nb = min(kKB, b - c0);
  // the points of this CTA's share of the columns (blockIdx.z of the split)
  const int64_t jb = (int64_t)blockIdx.z * jspan, je = jb + jspan < cols ? jb + jspan : cols;
  // this thread: rows r0 + lr and r0 + lr + TR, columns c0 + 16 cg .. + 15;
  // it evaluates the A-tile entries of its two rows in tile columns cg + CG t
  const int lr = tid % TR, cg = tid / TR;
  TC pr[2][kKD];
  int64_t gr[2] = {r0 + lr, r0 + lr + TR};
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int t = 0; t < kKD; ++t) pr[h][t] = (t < d && gr[h] < rows) ? (TC)P[gr[h] + (int64_t)t * ldp] : TC(0);
  TC acc[2][16];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[h][c] = TC(0);
  for (int64_t j0 = jb; j0 < je; j0 += kKC) {
    const int nc = je - j0 < kKC ? (int)(je - j0) : kKC;
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
    for (int t8 = 0; t8 < kKC / CG; ++t8) {
      const int j = cg + CG * t8;
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
        sa[j][lr + TR * h] = (j < nc && gr[h] < rows) ? f * a : TC(0);
      }
    }
    __syncthreads();
    for (int j = 0; j < nc; ++j) {
      TC xv[16];
      ld16(&sx[j][cg * 16], xv);
      const TC a0 = sa[j][lr], a1 = sa[j][lr + TR];
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
      if (gridDim.z > 1) {
        // split over the points: partial sums added into Y, which the
        // launcher initialised with the added term (or zero)
        atomicAdd(Y + gr[h] + (int64_t)col * ldy, (TO)v);
        continue;
      }
      if (R && coef) v += (TC)(coef[col] * R[gr[h] + (int64_t)col * ldr]);
      Y[gr[h] + (int64_t)col * ldy] = (TO)v;
    }
  }
}

// Y(:, j) = coef_j R(:, j) or 0: the starting value of a split product
template <typename TO>
__global__ void k_kmv_init(int64_t rows, int64_t b, TO* __restrict__ Y, int64_t ldy, const double* __restrict__ R,
                           int64_t ldr, const double* __restrict__ coef) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * b; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % rows, j = e / rows;
    Y[i + j * ldy] = (R && coef) ? (TO)(coef[j] * R[i + j * ldr]) : TO(0);
  }
}

template <typename TC, typename TX, typename TO, int CG>
rr_status launch_cg(cudaStream_t s, int64_t rows, int64_t cols, int d, const double* P, int64_t ldp, const double* Q,
                    int64_t ldq, double f, double l, double shift, int square, int64_t b, const TX* X, int64_t ldx, TO* Y,
                    int64_t ldy, const double* R, int64_t ldr, const double* coef) {
  constexpr int kKR = 2 * (256 / CG), kKB = 16 * CG, KC = kcols<TC>();
  const int64_t gx = (rows + kKR - 1) / kKR, gy = (b + kKB - 1) / kKB;
  // split the points over CTAs until the grid covers the GPU twice
  int64_t split = 1;
  const int64_t want = 2 * (int64_t)num_sms();
  while (gx * gy * split < want && split < 64 && cols / (split * 2) >= 4 * KC) split *= 2;
  const int64_t jspan = ((cols + split - 1) / split + KC - 1) / KC * KC;
  split = (cols + jspan - 1) / jspan;
  if (split > 1) {
    k_kmv_init<TO><<<(unsigned)std::min<int64_t>((rows * b + 255) / 256, 4096), 256, 0, s>>>(rows, b, Y, ldy, R, ldr,
                                                                                          coef);
    note_launches(1);
  }
  dim3 g((unsigned)gx, (unsigned)gy, (unsigned)split);
  k_kernel_mv<TC, TX, TO, CG><<<g, 256, 0, s>>>(rows, cols, d, P, ldp, Q, ldq, (TC)f, (TC)(1.0 / (2.0 * l * l)),
                                                (TC)shift, square, (int)b, X, ldx, Y, ldy, R, ldr, coef, jspan);
  return check_launch("kernel operator product");
}

// column groups per pass from b: 32 columns (b <= 32), else 64 (static
// shared memory keeps a CTA at 512 threads' worth of rows at most)
template <typename TC, typename TX, typename TO>
rr_status launch_kernel_mv(cudaStream_t s, int64_t rows, int64_t cols, int d, const double* P, int64_t ldp,
                           const double* Q, int64_t ldq, double f, double l, double shift, int square, int64_t b,
                           const TX* X, int64_t ldx, TO* Y, int64_t ldy, const double* R, int64_t ldr,
                           const double* coef) {
  if (b <= 32)
    return launch_cg<TC, TX, TO, 2>(s, rows, cols, d, P, ldp, Q, ldq, f, l, shift, square, b, X, ldx, Y, ldy, R, ldr, coef);
  return launch_cg<TC, TX, TO, 4>(s, rows, cols, d, P, ldp, Q, ldq, f, l, shift, square, b, X, ldx, Y, ldy, R, ldr, coef);
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
