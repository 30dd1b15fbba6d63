// Small projected problems in FP64 (Alg. 3 "B Y = M Y Lambda"; Alg. 5's block
// pencil; Sec. 4.2: the projected problem is solved in FP64).
//
// Pencil (H, G) -> whitening by Cholesky with column dropping -> symmetric
// (or rectangular, for the SVD) whitened matrix -> one-sided Jacobi
// (Hestenes) -> back-transformation.  The SVD pencil of Alg. 5 is solved
// through the whitened b1 x b2 SVD, which has the same positive spectrum and
// gives the sqrt(2)-scaled lift of the theorem in Sec. 3.2 directly.
//
// Small O(b^3) steps run in one CTA per problem; the triangular transforms
// are small FP64 GEMMs spread over the GPU.
#include <cfloat>
#include <climits>
#include <map>
#include <mutex>
#include <utility>

#include <cooperative_groups.h>

#include "rr_common.cuh"

namespace rr {

constexpr int kSmallThreads = 1024;
// largest pencil side: the packed FP32 Cholesky factor must fit in shared
// memory (b (b + 1) / 2 floats <= 227 KB)
constexpr int kMaxPencil = 335;

// Cholesky G = L L^T (lower), dropping column j when its pivot
// L_jj^2 <= 64 u64 max_i G_ii (or is not positive).  A dropped index gets a
// unit diagonal and zero row/column, so it is decoupled from the rest.
__global__ void __launch_bounds__(kSmallThreads) k_chol_drop(int b, const double* __restrict__ G,
                                                             int ldg, double* __restrict__ L,
                                                             int* __restrict__ dropped) {
  const int tid = threadIdx.x;
  __shared__ double s_maxd;
  __shared__ int s_keep;
  for (int e = tid; e < b * b; e += kSmallThreads) {
    int i = e % b, j = e / b;
    L[i + j * b] = (i >= j) ? 0.5 * (G[i + j * ldg] + G[j + i * ldg]) : 0.0;
  }
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < b; ++i) m = fmax(m, G[i + i * ldg]);
    s_maxd = m;
  }
  __syncthreads();
  const double thr = 64.0 * DBL_EPSILON * 0.5 * s_maxd;
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      double d = L[j + j * b];
      s_keep = (d > thr && d > 0.0) ? 1 : 0;
      dropped[j] = s_keep ? 0 : 1;
      L[j + j * b] = s_keep ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double ljj = L[j + j * b];
    if (s_keep) {
      for (int i = j + 1 + tid; i < b; i += kSmallThreads) L[i + j * b] /= ljj;
    } else {
      for (int i = j + 1 + tid; i < b; i += kSmallThreads) L[i + j * b] = 0.0;
      for (int l = tid; l < j; l += kSmallThreads) L[j + l * b] = 0.0;
    }
    __syncthreads();
    if (s_keep) {
      const int m = b - j - 1;
      const int total = m * m;
      for (int e = tid; e < total; e += kSmallThreads) {
        int ii = e % m, ll = e / m;
        if (ii < ll) continue;
        int i = j + 1 + ii, l = j + 1 + ll;
        L[i + l * b] -= L[i + j * b] * L[l + j * b];
      }
    }
    __syncthreads();
  }
}

// Inverse of a lower-triangular L (one thread per column of the inverse).
__global__ void __launch_bounds__(kSmallThreads) k_tri_inv_lower(int b, const double* __restrict__ L,
                                                                 double* __restrict__ Li) {
  for (int e = threadIdx.x; e < b * b; e += kSmallThreads) Li[e] = 0.0;
  __syncthreads();
  for (int c = threadIdx.x; c < b; c += kSmallThreads) {
    Li[c + c * b] = 1.0 / L[c + c * b];
    for (int i = c + 1; i < b; ++i) {
      double s = 0.0;
      for (int l = c; l < i; ++l) s = fma(L[i + l * b], Li[l + c * b], s);
      Li[i + c * b] = -s / L[i + i * b];
    }
  }
}

// Small products C = alpha op(A) op(B) + beta C (op = transpose when ta / tb),
// 16 x 16 output tiles, one output per thread, K in panels of KP staged in
// shared memory with all of a panel's loads in flight at once.  On GB300 the
// FP64 units of an SM are the limit (a 16 x 16 x 256 tile is 65k FP64 FMAs,
// ~16 us on one SM), so the work is cut into (tile, K-range) pieces spread
// evenly over the SMs: 1-D grid of ntiles x ks CTAs; with ks > 1 (beta = 0)
// the K ranges' partial sums add into a zeroed C with FP64 atomics.  sym:
// the result is symmetric (M == N): only tiles with bx <= by are computed,
// the off-diagonal ones write their mirror image too.
template <typename TA, int KP>
__global__ void __launch_bounds__(256) k_gemm_small(int ta, int tb, int M, int N, int K, double alpha,
                                                    const double* __restrict__ A, int lda,
                                                    const double* __restrict__ B, int ldb, double beta,
                                                    double* __restrict__ C, int ldc, int sym, int ks, int kc) {
  const int tm = (M + 15) / 16;
  const int tile = blockIdx.x / ks, split = blockIdx.x - tile * ks;
  int bx, by;
  if (sym) {  // tile = by (by + 1) / 2 + bx, bx <= by
    by = (int)((sqrtf(8.f * (float)tile + 1.f) - 1.f) * 0.5f);
    while ((by + 1) * (by + 2) / 2 <= tile) ++by;
    while (by * (by + 1) / 2 > tile) --by;
    bx = tile - by * (by + 1) / 2;
  } else {
    bx = tile % tm;
    by = tile / tm;
  }
  __shared__ TA As[KP][17];
  __shared__ TA Bs[KP][17];
  const int m0 = bx * 16, n0 = by * 16;
  const int kbeg = split * kc, kend = min(K, kbeg + kc);
  const int tid = threadIdx.x, ti = tid % 16, tj = tid / 16;
  TA acc = TA(0);
  for (int k0 = kbeg; k0 < kend; k0 += KP) {
    for (int e = tid; e < KP * 16; e += 256) {
      // consecutive threads along the operand's contiguous dimension
      const int ka = ta ? e % KP : e / 16, ia = ta ? e / KP : e % 16;
      const int gk = k0 + ka, gi = m0 + ia;
      As[ka][ia] = (gk < kend && gi < M) ? (TA)(ta ? A[gk + (size_t)gi * lda] : A[gi + (size_t)gk * lda]) : TA(0);
      const int kb = tb ? e / 16 : e % KP, jb = tb ? e % 16 : e / KP;
      const int gkb = k0 + kb, gj = n0 + jb;
      Bs[kb][jb] = (gkb < kend && gj < N) ? (TA)(tb ? B[gj + (size_t)gkb * ldb] : B[gkb + (size_t)gj * ldb]) : TA(0);
    }
    __syncthreads();
    const int kn = kend - k0 < KP ? kend - k0 : KP;
#pragma unroll 8
    for (int kk = 0; kk < kn; ++kk) acc = fma(As[kk][ti], Bs[kk][tj], acc);
    __syncthreads();
  }
  const int i = m0 + ti, j = n0 + tj;
  if (i < M && j < N) {
    const double v0 = alpha * (double)acc;
    if (ks > 1) {
      atomicAdd(C + i + (size_t)j * ldc, v0);
      if (sym && bx != by) atomicAdd(C + j + (size_t)i * ldc, v0);
    } else {
      double v = v0;
      if (beta != 0.0) v += beta * C[i + (size_t)j * ldc];
      C[i + (size_t)j * ldc] = v;
      if (sym && bx != by) C[j + (size_t)i * ldc] = v;
    }
  }
}

__global__ void k_zero_small(int M, int N, double* __restrict__ C, int ldc) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * N; e += gridDim.x * blockDim.x)
    C[e % M + (size_t)(e / M) * ldc] = 0.0;
}

template <typename TA, int KP>
static void gemm_small_launch(cudaStream_t s, int ta, int tb, int M, int N, int K, double alpha,
                              const double* A, int lda, const double* B, int ldb, double beta, double* C,
                              int ldc, int sym) {
  const int tm = (M + 15) / 16, tn = (N + 15) / 16;
  const int ntiles = sym ? tm * (tm + 1) / 2 : tm * tn;
  // about six CTAs per SM, each K range at least 64 long
  int ks = 1;
  if (beta == 0.0) {
    const int want = (6 * num_sms() + ntiles - 1) / ntiles;
    const int most = K / 64 > 1 ? K / 64 : 1;
    ks = want < most ? want : most;
    if (ks < 1) ks = 1;
  }
  const int kc = (K + ks - 1) / ks;
  ks = (K + kc - 1) / kc;
  if (ks > 1) {
    k_zero_small<<<(M * N + 255) / 256, 256, 0, s>>>(M, N, C, ldc);
    note_launches(1);
  }
  k_gemm_small<TA, KP><<<ntiles * ks, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sym, ks,
                                                   kc);
}

static void gemm_small(cudaStream_t s, int ta, int tb, int M, int N, int K, double alpha,
                       const double* A, int lda, const double* B, int ldb, double beta, double* C,
                       int ldc) {
  gemm_small_launch<double, 128>(s, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 0);
}

// C (n x n) = A^T B for a product known to be symmetric (W^T G W, N^T N,
// V^T V): half the tiles
static void gemm_small_sym(cudaStream_t s, int n, int K, const double* A, int lda, const double* B, int ldb,
                           double* C, int ldc) {
  gemm_small_launch<double, 128>(s, 1, 0, n, n, K, 1.0, A, lda, B, ldb, 0.0, C, ldc, 1);
}

static void gemm_mixed(cudaStream_t s, int ta, int tb, int M, int N, int K, double alpha,
                       const double* A, int lda, const double* B, int ldb, double beta, double* C,
                       int ldc) {
  // FP32 products are not FP64-unit bound: whole-K tiles
  dim3 g((unsigned)(((M + 15) / 16) * ((N + 15) / 16)));
  const int tm = (M + 15) / 16;
  (void)tm;
  k_gemm_small<float, 256><<<g, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, 0, 1, K);
}

// Symmetrise C and decouple dropped indices (zero row and column; their
// singular value is then exactly 0), and bracket lambda_min of the kept part
// for the shift that makes it positive definite: sh[0] = the Gershgorin lower
// bound (a valid shift), sh[1] = min_i C_ii (an upper bound on lambda_min),
// sh[2] = max_i sum_j |C_ij|, sh[3] = the span of the Gershgorin interval.
__global__ void __launch_bounds__(kSmallThreads) k_eig_prep(int b, double* __restrict__ C,
                                                            const int* __restrict__ dropped,
                                                            double* __restrict__ sh) {
  const int tid = threadIdx.x;
  for (int e = tid; e < b * b; e += kSmallThreads) {
    int i = e % b, j = e / b;
    if (i < j) {
      double v = 0.5 * (C[i + j * b] + C[j + i * b]);
      if (dropped[i] || dropped[j]) v = 0.0;
      C[i + j * b] = v;
      C[j + i * b] = v;
    }
  }
  __syncthreads();
  __shared__ double red[4][32];
  double lo = DBL_MAX, hi = -DBL_MAX, dmin = DBL_MAX, rmax = 0.0;
  for (int i = tid; i < b; i += kSmallThreads) {
    if (dropped[i]) continue;
    double r = 0.0;
    for (int j = 0; j < b; ++j)
      if (j != i) r += fabs(C[i + j * b]);
    const double d = C[i + i * b];
    lo = fmin(lo, d - r);
    hi = fmax(hi, d + r);
    dmin = fmin(dmin, d);
    rmax = fmax(rmax, fabs(d) + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    dmin = fmin(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
    rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = lo;
    red[1][tid >> 5] = hi;
    red[2][tid >> 5] = dmin;
    red[3][tid >> 5] = rmax;
  }
  __syncthreads();
  if (tid == 0) {
    double l = DBL_MAX, h = -DBL_MAX, u = DBL_MAX, rm = 0.0;
    for (int w = 0; w < kSmallThreads / 32; ++w) {
      l = fmin(l, red[0][w]);
      h = fmax(h, red[1][w]);
      u = fmin(u, red[2][w]);
      rm = fmax(rm, red[3][w]);
    }
    if (l > h) {  // everything dropped
      l = 0.0;
      h = 1.0;
      u = 0.0;
    }
    double span = fmax(h - l, fmax(fabs(l), fabs(h)));
    if (span == 0.0) span = 1.0;
    sh[0] = l;
    sh[1] = u;
    sh[2] = rm;
    sh[3] = span;
  }
}

// A tighter shift than the Gershgorin bound.  The one-sided Jacobi works on
// C - mu I, whose singular values lambda - mu all lie near |mu| when mu is far
// below the spectrum; FP32 Jacobi then resolves close eigenvalues only to
// u32 (lambda - mu)^2 / gap, which the FP64 refinement cannot recover from
// once the resulting angles are large.  The shift is found by a parallel search
// with definiteness tests: CTA p factors C - sigma_p I by FP32 LDL^T
// (no pivoting; the Schur-complement pivots are all positive iff the FP32
// matrix is positive definite, up to rounding), sigma_p spread uniformly over
// the bracket [sh[0], sh[1]].  Dropped indices take a unit diagonal.  The
// packed lower triangle lives in shared memory (b (b + 1) / 2 floats).
constexpr int kShiftTrials = 64, kShiftThreads = 256;
__global__ void __launch_bounds__(kShiftThreads) k_shift_trials(int b, const double* __restrict__ C,
                                                                const int* __restrict__ dropped,
                                                                const double* __restrict__ sh,
                                                                int* __restrict__ ok) {
  extern __shared__ float sh_pk[];  // column j at off(j) = j (2b - j + 1) / 2, rows j..b-1
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double l = sh[0], u = sh[1];
  const double sigma = l + (u - l) * (double)(blockIdx.x + 1) / (double)(kShiftTrials + 1);
  for (int j = warp; j < b; j += kShiftThreads / 32) {
    const size_t off = (size_t)j * (2 * b - j + 1) / 2;
    for (int i = j + lane; i < b; i += 32) {
      double v;
      if (dropped[i] || dropped[j]) v = i == j ? 1.0 : 0.0;
      else v = C[i + (size_t)j * b] - (i == j ? sigma : 0.0);
      sh_pk[off + (i - j)] = (float)v;
    }
  }
  int good = 1;
  for (int j = 0; j < b; ++j) {
    __syncthreads();
    const size_t oj = (size_t)j * (2 * b - j + 1) / 2;
    const float d = sh_pk[oj];
    if (!(d > 0.f)) {  // every thread reads the same pivot: a uniform exit
      good = 0;
      break;
    }
    const float rd = 1.f / d;
    for (int k = j + 1 + warp; k < b; k += kShiftThreads / 32) {
      const float lk = sh_pk[oj + (k - j)] * rd;
      const size_t ok_ = (size_t)k * (2 * b - k + 1) / 2;
      for (int i = k + lane; i < b; i += 32) sh_pk[ok_ + (i - k)] = fmaf(-sh_pk[oj + (i - j)], lk, sh_pk[ok_ + (i - k)]);
    }
  }
  if (tid == 0) ok[blockIdx.x] = good;
}

// Narrow the bracket to the trials that passed: the largest passing sigma is
// the new lower end, the next trial the new upper end (64 trials place the
// shift within 1/65 of the bracket below lambda_min, which keeps the relative
// gaps of the singular values those of the spectrum).  On the last round the
// shift is that lower end less the FP32 backward error of the test,
// (b + 1) b u32 |C - sigma I|, and 1e-3 of the span (which keeps the smallest
// singular value clear of the Jacobi's norm floor); mu goes to mu_out and the
// diagonal of C is shifted.
__global__ void k_shift_pick(int b, double* __restrict__ C, const int* __restrict__ dropped, double* __restrict__ sh,
                             const int* __restrict__ ok, int last, double* __restrict__ mu_out) {
  __shared__ double s_mu;
  if (threadIdx.x == 0) {
    const double l = sh[0], u = sh[1];
    int best = -1;
    for (int p = 0; p < kShiftTrials; ++p)
      if (ok[p]) best = p;
    auto sig = [&](int p) { return l + (u - l) * (double)(p + 1) / (double)(kShiftTrials + 1); };
    const double nl = best >= 0 ? sig(best) : l;
    const double nu = best + 1 < kShiftTrials ? sig(best + 1) : u;
    sh[0] = nl;
    sh[1] = nu;
    if (last) {
      const double tol = 1.1 * (double)(b + 1) * (double)b * 0x1p-24 * (sh[2] + fabs(nl));
      // a passing trial is only trusted to its backward error; the Gershgorin
      // bound needs no margin, but the same one is harmless
      s_mu = nl - tol - 1e-3 * sh[3];
      *mu_out = s_mu;
    }
  }
  if (!last) return;
  __syncthreads();
  for (int i = threadIdx.x; i < b; i += blockDim.x) C[i + (size_t)i * b] = dropped[i] ? 0.0 : C[i + (size_t)i * b] - s_mu;
}

static size_t shift_trial_smem(int b) { return (size_t)b * (b + 1) / 2 * sizeof(float); }

// Symmetrise, bracket, one round of trials, shift.
static rr_status eig_shift(cudaStream_t s, int b, double* C, const int* dropped, double* sh, int* ok, double* mu) {
  k_eig_prep<<<1, kSmallThreads, 0, s>>>(b, C, dropped, sh);
  const size_t sm = shift_trial_smem(b);
  if (sm > 48 * 1024)
    RR_CUDA(cudaFuncSetAttribute(k_shift_trials, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_shift_trials<<<kShiftTrials, kShiftThreads, sm, s>>>(b, C, dropped, sh, ok);
  k_shift_pick<<<1, 256, 0, s>>>(b, C, dropped, sh, ok, 1, mu);
  note_launches(2);  // with check_launch's one: prep, the trials, the pick
  return check_launch("eigen shift");
}

// Zero the rows (drop_r) and columns (drop_c) of a rectangular b1 x b2 matrix.
__global__ void k_zero_dropped(int b1, int b2, double* __restrict__ C, const int* __restrict__ dr,
                               const int* __restrict__ dc) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= b1 * b2) return;
  int i = e % b1, j = e / b1;
  if (dr[i] || dc[j]) C[i + j * b1] = 0.0;
}

// Column norms sigma_j of M (r x c), descending order with ties by index;
// zero columns (dropped directions) sort last and are flagged invalid.
__global__ void __launch_bounds__(kSmallThreads) k_colnorm_sort(int r, int c, const double* __restrict__ M,
                                                                int ldm, double* __restrict__ sig,
                                                                int* __restrict__ order) {
  extern __shared__ double sh[];
  double* nrm = sh;  // [c]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = warp; j < c; j += kSmallThreads / 32) {
    double s = 0.0;
    for (int i = lane; i < r; i += 32) s = fma(M[i + j * ldm], M[i + j * ldm], s);
    s = warp_sum(s);
    if (lane == 0) nrm[j] = sqrt(s);
  }
  __syncthreads();
  // a total order (a NaN norm counts as -1: last, flagged invalid with 0), so
  // the ranks form a permutation whatever the data
  for (int j = tid; j < c; j += kSmallThreads) {
    const double v = nrm[j] >= 0.0 ? nrm[j] : -1.0;
    int rank = 0;
    for (int l = 0; l < c; ++l) {
      const double w = nrm[l] >= 0.0 ? nrm[l] : -1.0;
      if (w > v || (w == v && l < j)) ++rank;
    }
    order[rank] = j;
    sig[rank] = v >= 0.0 ? v : 0.0;
  }
}

// Eigen finish: theta_rank = sigma + mu for valid columns, ascending order;
// Z(:, out) = V(:, order) for valid, 0 for dropped.
__global__ void k_eig_finish(int b, const double* __restrict__ sig_desc,
                             const int* __restrict__ order_desc, const double* __restrict__ mu,
                             const double* __restrict__ V, double* __restrict__ theta,
                             double* __restrict__ Z, int* __restrict__ nvalid) {
  // count valid (sigma > 0): they are the first ones in descending order
  __shared__ int s_nv;
  if (threadIdx.x == 0) {
    int nv = 0;
    for (int i = 0; i < b; ++i) nv += sig_desc[i] > 0.0;
    s_nv = nv;
    if (nvalid) *nvalid = nv;
  }
  __syncthreads();
  const int nv = s_nv;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    int i = e % b, out = e / b;
    double v = 0.0;
    if (out < nv) {
      int src = order_desc[nv - 1 - out];  // ascending theta
      v = V[i + src * b];
    }
    Z[i + out * b] = v;
  }
  for (int out = threadIdx.x; out < b; out += blockDim.x)
    theta[out] = out < nv ? sig_desc[nv - 1 - out] + *mu : nan("");
}

// SVD finish: Uw(:, out) = M(:, src)/sigma (left vectors of the whitened
// matrix), Vw(:, out) = V(:, src); invalid (sigma == 0) columns zeroed.
__global__ void k_svd_finish(int b1, int b2, const double* __restrict__ sig_desc,
                             const int* __restrict__ order_desc, const double* __restrict__ M,
                             const double* __restrict__ V, double* __restrict__ s_out,
                             double* __restrict__ Uw, double* __restrict__ Vw, int r) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < (b1 + b2) * r; e += gridDim.x * blockDim.x) {
    int out = e / (b1 + b2), i = e % (b1 + b2);
    int src = order_desc[out];
    double sg = sig_desc[out];
    if (i < b1) {
      Uw[i + out * b1] = sg > 0.0 ? M[i + src * b1] / sg : 0.0;
    } else {
      int ii = i - b1;
      Vw[ii + out * b2] = sg > 0.0 ? V[ii + src * b2] : 0.0;
    }
    if (i == 0) s_out[out] = sg;
  }
}

// ---------------------------------------------------------------------------
// FP32 Cholesky with column dropping, then the inverse of the factor, in one
// CTA with the lower triangle packed in shared memory (b(b+1)/2 floats).
// A column j is dropped when its Schur-complement pivot is below 64 u32 times
// its original diagonal (its new content is below ~1e-3 of its length:
// rounding noise for a basis stored in BF16/FP32) or not positive; dropped
// indices get a unit diagonal and zero row/column.  Output W0 = L^-T (FP64)
// with dropped columns zeroed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pk(int i, int j, int b) { return j * b - (j * (j - 1)) / 2 + (i - j); }

__global__ void __launch_bounds__(kSmallThreads) k_chol_inv_f32(int b, const double* __restrict__ G, int ldg,
                                                                int* __restrict__ dropped,
                                                                double* __restrict__ W) {
  extern __shared__ float Ls[];  // packed lower triangle, column-major
  float* gd = Ls + (size_t)b * (b + 1) / 2;  // [b] original diagonal
  float* cb = gd + b;                        // [b] column buffer
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kSmallThreads / 32;
  // symmetrised copy, one warp per column
  for (int j = warp; j < b; j += nw) {
    for (int i = j + lane; i < b; i += 32)
      Ls[pk(i, j, b)] = (float)(0.5 * (G[i + (size_t)j * ldg] + G[j + (size_t)i * ldg]));
    if (lane == 0) gd[j] = (float)G[j + (size_t)j * ldg];
  }
  __syncthreads();
  // right-looking factorisation; every thread takes the pivot decision itself
  for (int j = 0; j < b; ++j) {
    const float d = Ls[pk(j, j, b)];
    const float g0 = gd[j];
    const bool keep = g0 > 0.f && d > 64.f * 0x1p-24f * g0;
    const float ljj = keep ? sqrtf(d) : 1.f;
    const int bj = pk(j, j, b) - j;  // column j starts at bj + j
    for (int i = j + 1 + tid; i < b; i += kSmallThreads) Ls[bj + i] = keep ? Ls[bj + i] / ljj : 0.f;
    if (!keep)
      for (int l = tid; l < j; l += kSmallThreads) Ls[pk(j, l, b)] = 0.f;
    __syncthreads();
    if (tid == 0) {
      Ls[bj + j] = ljj;
      dropped[j] = keep ? 0 : 1;
    }
    if (keep) {
      // trailing update, one warp per column l, lanes over rows i >= l
      for (int l = j + 1 + warp; l < b; l += nw) {
        const float llj = Ls[bj + l];
        const int bl = pk(l, l, b) - l;
        for (int i = l + lane; i < b; i += 32) Ls[bl + i] = fmaf(-Ls[bj + i], llj, Ls[bl + i]);
      }
    }
    __syncthreads();
  }
  // in-place inverse X = L^-1 by right-looking forward substitution: at step
  // l row l of X is final up to the factor 1 / L_ll; then every row i > l
  // takes -L(i, l) X(l, :).  Slot (i, k), k < i, holds L(i, k) until step k
  // and the accumulating X(i, k) afterwards; column l of L is staged in cb.
  for (int l = 0; l < b; ++l) {
    const float ill = 1.f / Ls[pk(l, l, b)];
    const int bl = pk(l, l, b) - l;
    for (int i = l + 1 + tid; i < b; i += kSmallThreads) cb[i] = Ls[bl + i];
    for (int k = tid; k < l; k += kSmallThreads) Ls[pk(l, k, b)] *= ill;
    __syncthreads();
    if (tid == 0) Ls[bl + l] = ill;
    for (int k = warp; k <= l; k += nw) {
      const int bk = pk(k, k, b) - k;
      if (k == l) {
        for (int i = l + 1 + lane; i < b; i += 32) Ls[bk + i] = -cb[i] * ill;
      } else {
        const float xlk = Ls[bk + l];
        for (int i = l + 1 + lane; i < b; i += 32) Ls[bk + i] = fmaf(-cb[i], xlk, Ls[bk + i]);
      }
    }
    __syncthreads();
  }
  // W0 = (L^-1)^T, dropped columns zero
  for (int e = tid; e < b * b; e += kSmallThreads) {
    int i = e % b, j = e / b;
    W[i + j * b] = (dropped[j] || j < i) ? 0.0 : (double)Ls[pk(j, i, b)];
  }
}

// Blocked variant for b <= 256 (the same factorisation, drop rule and
// output), 32 x 32 tiles of the lower triangle in shared memory, one CTA:
//   per 32-wide panel k: warp 0 factors the diagonal tile (warp-synchronous,
//   the pivot test of the unblocked kernel per column); one thread per row
//   solves the panel's tiles below against it (dropped columns zero); every
//   warp applies tile products of the trailing update (register-blocked);
//   inverse: diagonal tiles inverted by one warp each (column per lane), then
//   block row I of L^-1 from X(I,K) = -X(I,I) sum_{J=K..I-1} L(I,J) X(J,K).
// About 40 CTA barriers instead of 4 per column.
constexpr int kCT = 32;      // tile
constexpr int kCLd = 33;     // padded row length
constexpr int kCTMax = 8;    // tiles per side (b <= 256)
constexpr int kChThreads = 512;  // 128 registers per thread: the 32-entry row stays in registers
__device__ __forceinline__ int ctile(int I, int J) { return I * (I + 1) / 2 + J; }

// C[r][c] += sgn * sum_l A[r][l] * Bop(l, c) for 32 x 32 tiles, one warp,
// lane = c.  btrans: Bop(l, c) = B[c][l] (A B^T), else B[l][c] (A B).
__device__ __forceinline__ void warp_tile_mac(float* C, const float* A, const float* B, bool btrans,
                                              float sgn, int lane) {
  float bv[kCT];
#pragma unroll
  for (int l = 0; l < kCT; ++l) bv[l] = btrans ? B[lane * kCLd + l] : B[l * kCLd + lane];
  for (int r = 0; r < kCT; ++r) {
    float acc = 0.f;
#pragma unroll
    for (int l = 0; l < kCT; ++l) acc = fmaf(A[r * kCLd + l], bv[l], acc);
    C[r * kCLd + lane] = fmaf(sgn, acc, C[r * kCLd + lane]);
  }
}

__global__ void __launch_bounds__(kChThreads, 1) k_chol_inv_blocked(int b, const double* __restrict__ G, int ldg,
                                                                    int* __restrict__ dropped,
                                                                    double* __restrict__ W) {
  extern __shared__ float cs_raw[];
  const int nt = (b + kCT - 1) / kCT;
  const int ntiles = nt * (nt + 1) / 2;
  float* Ts = cs_raw;                                   // [ntiles][32][33]
  float* Ss = Ts + (size_t)ntiles * kCT * kCLd;         // [nt - 1][32][33] scratch
  float* gd = Ss + (size_t)(nt > 1 ? nt - 1 : 1) * kCT * kCLd;  // [32 nt]
  int* sdrop = reinterpret_cast<int*>(gd + kCT * nt);   // [32 nt]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kChThreads / 32;
  auto T = [&](int I, int J) { return Ts + (size_t)ctile(I, J) * kCT * kCLd; };
  // symmetrised copy, thread = (r, c) of every tile (kCT x kCT / kChThreads
  // passes); rows/columns beyond b padded with the identity
  for (int rc = tid; rc < kCT * kCT; rc += kChThreads) {
    const int r = rc % kCT, c = rc / kCT;
    int I = 0, J = 0;
#pragma unroll 4
    for (int t = 0; t < ntiles; ++t) {
      const int gi = I * kCT + r, gj = J * kCT + c;
      float v;
      if (gi < b && gj < b) v = (float)(0.5 * (G[gi + (size_t)gj * ldg] + G[gj + (size_t)gi * ldg]));
      else v = (gi == gj) ? 1.f : 0.f;
      Ts[(size_t)t * kCT * kCLd + r * kCLd + c] = v;
      if (++J > I) {
        ++I;
        J = 0;
      }
    }
  }
  for (int i = tid; i < kCT * nt; i += kChThreads) gd[i] = i < b ? (float)G[i + (size_t)i * ldg] : 1.f;
  __syncthreads();
  for (int k = 0; k < nt; ++k) {
    float* D = T(k, k);
    if (warp == 0) {
      // lane r holds the trailing part of row r (columns j..31 in a[0..31-j],
      // shifted left after every column, so the current column is a[0] and
      // the loop over j stays rolled); column j travels by shuffle
      float a[kCT];
#pragma unroll
      for (int c = 0; c < kCT; ++c) a[c] = D[lane * kCLd + c];
      for (int j = 0; j < kCT; ++j) {
        const float d = __shfl_sync(0xffffffffu, a[0], j);
        const float g0 = gd[k * kCT + j];
        const bool keep = g0 > 0.f && d > 64.f * 0x1p-24f * g0;
        const float ljj = keep ? sqrtf(d) : 1.f;
        if (lane > j) a[0] = keep ? a[0] / ljj : 0.f;
        if (lane == j) {
          a[0] = ljj;
          if (!keep)
            for (int c = 0; c < j; ++c) D[j * kCLd + c] = 0.f;
        }
        if (lane == 0) sdrop[k * kCT + j] = keep ? 0 : 1;
        if (lane >= j) D[lane * kCLd + j] = a[0];  // column j of L (and the diagonal)
#pragma unroll
        for (int u = 1; u < kCT; ++u) {
          const float lcj = __shfl_sync(0xffffffffu, a[0], (j + u) & 31);
          if (keep && j + u < kCT && lane >= j + u) a[u] = fmaf(-a[0], lcj, a[u]);
        }
#pragma unroll
        for (int u = 0; u < kCT - 1; ++u) a[u] = a[u + 1];
      }
    }
    __syncthreads();
    // dropped columns of this panel: zero their rows in the earlier panels
    for (int e = tid; e < k * kCT * kCT; e += kChThreads) {
      const int J = e / (kCT * kCT), rc = e % (kCT * kCT), r = rc / kCT, c = rc % kCT;
      if (sdrop[k * kCT + r]) T(k, J)[r * kCLd + c] = 0.f;
    }
    // panel tiles below: row x of tile (I, k) solves x L(k,k)^T = a
    for (int row = tid; row < (nt - 1 - k) * kCT; row += kChThreads) {
      const int I = k + 1 + row / kCT, r = row % kCT;
      float* a = T(I, k) + r * kCLd;
      float x[kCT];
#pragma unroll
      for (int j = 0; j < kCT; ++j) {
        float v = a[j];
#pragma unroll
        for (int l = 0; l < j; ++l) v = fmaf(-x[l], D[j * kCLd + l], v);
        x[j] = sdrop[k * kCT + j] ? 0.f : v / D[j * kCLd + j];
      }
#pragma unroll
      for (int j = 0; j < kCT; ++j) a[j] = x[j];
    }
    __syncthreads();
    // trailing update A(I,J) -= L(I,k) L(J,k)^T, k < J <= I
    {
      const int m = nt - 1 - k;  // tiles below the panel
      for (int t = warp; t < m * (m + 1) / 2; t += nw) {
        int I = 0;
        while ((I + 1) * (I + 2) / 2 <= t) ++I;
        const int J = t - I * (I + 1) / 2;
        warp_tile_mac(T(k + 1 + I, k + 1 + J), T(k + 1 + I, k), T(k + 1 + J, k), true, -1.f, lane);
      }
    }
    __syncthreads();
  }
  // inverse of the diagonal tiles, one warp each, lane = column
  for (int k = warp; k < nt; k += nw) {
    float* D = T(k, k);
    float x[kCT];
#pragma unroll
    for (int r = 0; r < kCT; ++r) {
      float v = (r == lane) ? 1.f : 0.f;
#pragma unroll
      for (int l = 0; l < r; ++l) v = fmaf(-D[r * kCLd + l], x[l], v);
      x[r] = (r < lane) ? 0.f : v / D[r * kCLd + r];
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kCT; ++r) D[r * kCLd + lane] = x[r];
  }
  __syncthreads();
  // block rows of L^-1: S(K) = sum_{J=K..I-1} L(I,J) X(J,K), then
  // X(I,K) = -X(I,I) S(K); one warp per (K, 8-row slice)
  for (int I = 1; I < nt; ++I) {
    for (int t = warp; t < I * 4; t += nw) {
      const int K = t >> 2, r0 = (t & 3) * 8;
      float* S = Ss + (size_t)K * kCT * kCLd;
      float acc[8] = {};
      for (int J = K; J < I; ++J) {
        const float* A = T(I, J);
        const float* B = T(J, K);
        float bv[kCT];
#pragma unroll
        for (int l = 0; l < kCT; ++l) bv[l] = B[l * kCLd + lane];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
#pragma unroll
          for (int l = 0; l < kCT; ++l) acc[rr] = fmaf(A[(r0 + rr) * kCLd + l], bv[l], acc[rr]);
        }
      }
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) S[(r0 + rr) * kCLd + lane] = acc[rr];
    }
    __syncthreads();
    for (int t = warp; t < I * 4; t += nw) {
      const int K = t >> 2, r0 = (t & 3) * 8;
      const float* A = T(I, I);
      const float* B = Ss + (size_t)K * kCT * kCLd;
      float bv[kCT];
#pragma unroll
      for (int l = 0; l < kCT; ++l) bv[l] = B[l * kCLd + lane];
      float* X = T(I, K);
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        float acc = 0.f;
#pragma unroll
        for (int l = 0; l < kCT; ++l) acc = fmaf(A[(r0 + rr) * kCLd + l], bv[l], acc);
        X[(r0 + rr) * kCLd + lane] = -acc;
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < b; i += kChThreads) dropped[i] = sdrop[i];
  // W0 = (L^-1)^T, dropped columns zero
  for (int e = tid; e < b * b; e += kChThreads) {
    const int i = e % b, j = e / b;
    float v = 0.f;
    if (!sdrop[j] && j >= i) v = T(j / kCT, i / kCT)[(j % kCT) * kCLd + (i % kCT)];
    W[i + (size_t)j * b] = (double)v;
  }
}

static size_t chol_blocked_smem(int b) {
  const int nt = (b + kCT - 1) / kCT;
  return ((size_t)(nt * (nt + 1) / 2 + (nt > 1 ? nt - 1 : 1)) * kCT * kCLd + 2 * (size_t)kCT * nt) * sizeof(float);
}

// mode 0: E <- E - diag(kept)  (E = W^T G W, so E becomes W^T G W - I on the
// kept part); mode 1: F = E/2 - 3/8 E2, the correction of
// W <- W (I - E/2 + 3/8 E^2) = W - W F
__global__ void k_whiten_corr(int b, double* __restrict__ E, const double* __restrict__ E2,
                              const int* __restrict__ dropped, double* __restrict__ F, int stage) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= b * b) return;
  int i = e % b, j = e / b;
  double v = E[e];
  if (stage == 0) {
    if (i == j && !dropped[i]) v -= 1.0;
    E[e] = v;
    return;
  }
  F[e] = 0.5 * v - 0.375 * E2[e];
}

// One-sided block Jacobi (Hestenes) on the columns of M (r x cpad, FP32):
// M <- M V, V orthogonal (cpad x cpad, initialised to I by the launcher).
// The cpad columns form 2P blocks of w; CTA g takes one block pair per round
// (circle method over the blocks, 2P-1 rounds per sweep), loads its 2w
// columns of M and V into shared memory and orthogonalises column pairs
// among them, and writes them back; a bounded grid barrier separates rounds.
// Round 0 of a sweep takes every pair among the 2w local columns (circle
// method, w pairs per sub-round), which also covers every block's internal
// pairs once per sweep; later rounds only the w x w pairs across the two
// blocks (sub-round t pairs column i of block a with column (i + t) mod w of
// block b), c - 1 sub-rounds per sweep in all.
//
// In a sub-round warp i forms the inner product of its pair (in the cross
// rounds column i of block a stays in warp i's registers for the whole
// round), computes the rotation, carries the squared column norms through it
// (|x'|^2 = |x|^2 - t g, |y'|^2 = |y|^2 + t g; the norms are computed when
// the block is loaded) and applies it to the pair and to the round's 2w x 2w
// accumulated rotation Q, which is applied to the V block once at the end of
// the round (V_blk <- V_blk Q); the pairs of a sub-round are disjoint, so one
// __syncthreads separates sub-rounds.  A pair whose
// inner product is exactly zero, or below tol relative to the column norms
// (floored, so rounding-level columns count as converged against
// everything), is not rotated; zero columns (dropped directions, padding)
// stay decoupled.  Converged when a sweep rotates nothing.
constexpr int kBJThreads = 512;
constexpr int kBJMaxChunks = 3;  // float4 row chunks per lane: r, cpad <= 384

// (x + y) mod m for 0 <= x, y < m
__device__ __forceinline__ int add_mod(int x, int y, int m) {
  const int s = x + y;
  return s >= m ? s - m : s;
}

// pair pi of sub-round sr: round 0 circle method over the 2w local columns
// (p < q), later rounds column pi of block a with column (pi + sr) mod w of b
__device__ __forceinline__ void bj_pair(int round, int pi, int sr, int w, int& p, int& q) {
  const int w2 = 2 * w;
  if (round == 0) {
    const int a = (pi == 0) ? 0 : 1 + add_mod(pi - 1, sr, w2 - 1);
    const int bq = 1 + add_mod(w2 - 2 - pi, sr, w2 - 1);
    p = a < bq ? a : bq;
    q = a < bq ? bq : a;
  } else {
    p = pi;
    q = w + add_mod(pi, sr, w);
  }
}

// One round's pair work on the 2w columns in shared memory (Ms [2w][rp],
// tracked squared norms nrm, Q accumulated in Qs [2w][ldq]); every thread of
// the block calls it, and it ends with the columns back in Ms.
template <int NCH>
__device__ __forceinline__ void bj_round(int round, int w, int rp, float* __restrict__ Ms, float* __restrict__ Qs,
                                         int ldq, float* __restrict__ nrm, float nfloor, float tol2,
                                         int* s_rot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int w2 = 2 * w, rch = rp >> 2;
  const bool resident = round > 0;  // column `warp` of block a lives in registers
  float4 xr[NCH];
  if (resident && warp < w) {
    const float4* mp = reinterpret_cast<const float4*>(Ms + (size_t)warp * rp);
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
      const int c = lane + 32 * t;
      xr[t] = c < rch ? mp[c] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  const int nsub = (round == 0) ? w2 - 1 : w;
  for (int sr = 0; sr < nsub; ++sr) {
    // warp `warp` owns pair `warp` of the sub-round: inner product, its
    // rotation (every lane computes it from the reduced sums), the update
    // of the two columns, their tracked norms and Q's two columns; pairs
    // of a sub-round are disjoint, so one barrier per sub-round suffices
    if (warp < w) {
      int p, q;
      bj_pair(round, warp, sr, w, p, q);
      float4 x[NCH], y[NCH];
      const float4* mp = reinterpret_cast<const float4*>(Ms + (size_t)p * rp);
      const float4* mq = reinterpret_cast<const float4*>(Ms + (size_t)q * rp);
      float ga = 0.f;
#pragma unroll
      for (int t = 0; t < NCH; ++t) {
        const int c = lane + 32 * t;
        x[t] = resident ? xr[t] : (c < rch ? mp[c] : make_float4(0.f, 0.f, 0.f, 0.f));
        y[t] = c < rch ? mq[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        ga = fmaf(x[t].x, y[t].x, ga);
        ga = fmaf(x[t].y, y[t].y, ga);
        ga = fmaf(x[t].z, y[t].z, ga);
        ga = fmaf(x[t].w, y[t].w, ga);
      }
      ga = warp_sum(ga);
      const float al = nrm[p], be = nrm[q];
      const float fa = fmaxf(al, nfloor), fb = fmaxf(be, nfloor);
      // rotate unless |g| <= tol |x| |y| (squared form; the block is scaled
      // so that squared norms stay far from the FP32 range limits)
      if (ga != 0.f && ga * ga > tol2 * fa * fb) {
        // t the smaller root of t^2 + 2 zeta t - 1 = 0, zeta = (|y|^2 - |x|^2) / (2 g)
        const float zeta = __fdividef(be - al, 2.f * ga);
        const float az = fabsf(zeta);
        float tt;
        if (az > 1e18f) {
          tt = __fdividef(0.5f, az);
        } else {
          const float s2 = fmaf(az, az, 1.f);
          tt = __fdividef(1.f, az + s2 * rsqrtf(s2));
        }
        tt = copysignf(tt, zeta);
        const float u = fmaf(tt, tt, 1.f);
        float cs = rsqrtf(u);
        cs = cs * fmaf(-0.5f * u, cs * cs, 1.5f);  // one Newton step: cs^2 (1 + t^2) = 1
        const float sn = cs * tt;
        float4* mpw = reinterpret_cast<float4*>(Ms + (size_t)p * rp);
        float4* mqw = reinterpret_cast<float4*>(Ms + (size_t)q * rp);
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
          const int c = lane + 32 * t;
          float4 a4, b4;
          a4.x = cs * x[t].x - sn * y[t].x;
          a4.y = cs * x[t].y - sn * y[t].y;
          a4.z = cs * x[t].z - sn * y[t].z;
          a4.w = cs * x[t].w - sn * y[t].w;
          b4.x = sn * x[t].x + cs * y[t].x;
          b4.y = sn * x[t].y + cs * y[t].y;
          b4.z = sn * x[t].z + cs * y[t].z;
          b4.w = sn * x[t].w + cs * y[t].w;
          if (resident) xr[t] = a4;
          else if (c < rch) mpw[c] = a4;
          if (c < rch) mqw[c] = b4;
        }
        if (lane < w2) {
          const float qp = Qs[lane * ldq + p], qq = Qs[lane * ldq + q];
          Qs[lane * ldq + p] = cs * qp - sn * qq;
          Qs[lane * ldq + q] = sn * qp + cs * qq;
        }
        if (lane == 0) {
          nrm[p] = al - tt * ga;
          nrm[q] = be + tt * ga;
          *s_rot = 1;
        }
      }
    }
    __syncthreads();
  }
  if (resident && warp < w) {
    float4* mp = reinterpret_cast<float4*>(Ms + (size_t)warp * rp);
#pragma unroll
    for (int t = 0; t < NCH; ++t) {
      const int c = lane + 32 * t;
      if (c < rch) mp[c] = xr[t];
    }
  }
}

// Shared-memory layout: Ms [2w][rp] and Vs [2w][cp4] with rp, cp4 the row
// counts rounded up to 4 (zero rows; float4 access), Qs [2w][ldq], nrm [2w].
// NCH = row chunks of 4 per lane (rp <= 128 NCH).
template <int NCH>
__global__ void __launch_bounds__(kBJThreads) k_block_jacobi(int r, int cpad, int w, float* __restrict__ M,
                                                             int ldm, float* __restrict__ V, int ldv,
                                                             float tol, int max_sweeps, int* __restrict__ rot,
                                                             GridBarrier* bar, int* err,
                                                             int* __restrict__ sweeps_out,
                                                             const float* __restrict__ floor_ptr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w2 = 2 * w;
  const int rp = (r + 3) & ~3, cp4 = (cpad + 3) & ~3;
  const int ldq = (w2 + 7) & ~3;  // multiple of 4, >= 2w + 4
  float* Ms = reinterpret_cast<float*>(smem_raw);
  float* Vs = Ms + (size_t)w2 * rp;
  float* Qs = Vs + (size_t)w2 * cp4;
  float* nrm = Qs + w2 * ldq;
  const int P = gridDim.x, g = blockIdx.x, nblk = 2 * P;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kBJThreads / 32;
  const float nfloor = floor_ptr ? *floor_ptr : 0.f;
  const float tol2 = tol * tol;
  __shared__ int s_rot;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    for (int round = 0; round < nblk - 1; ++round) {
      const int ba = (g == 0) ? 0 : 1 + add_mod(g - 1, round, nblk - 1);
      const int bb = 1 + add_mod(nblk - 2 - g, round, nblk - 1);
      // load the 2w columns of M (with their squared norms) and of V; Q = I
      for (int l = warp; l < w2; l += nw) {
        const int gc = (l < w ? ba * w + l : bb * w + (l - w));
        const float* src = M + (size_t)gc * ldm;
        float* dst = Ms + (size_t)l * rp;
        float s2 = 0.f;
        for (int i = lane; i < rp; i += 32) {
          const float v = i < r ? src[i] : 0.f;
          dst[i] = v;
          s2 = fmaf(v, v, s2);
        }
        s2 = warp_sum(s2);
        if (lane == 0) nrm[l] = s2;
        const float* vsrc = V + (size_t)gc * ldv;
        float* vdst = Vs + (size_t)l * cp4;
        for (int i = lane; i < cp4; i += 32) vdst[i] = i < cpad ? vsrc[i] : 0.f;
      }
      for (int e = tid; e < w2 * ldq; e += kBJThreads) {
        const int i = e / ldq, j = e - i * ldq;
        Qs[e] = (i == j) ? 1.f : 0.f;
      }
      __syncthreads();
      bj_round<NCH>(round, w, rp, Ms, Qs, ldq, nrm, nfloor, tol2, &s_rot);
      __syncthreads();
      // store back M
      for (int l = warp; l < w2; l += nw) {
        const int gc = (l < w ? ba * w + l : bb * w + (l - w));
        const float* src = Ms + (size_t)l * rp;
        float* dst = M + (size_t)gc * ldm;
        for (int i = lane; i < r; i += 32) dst[i] = src[i];
      }
      // V_blk <- V_blk Q: thread = (float4 row chunk, 4 output columns)
      {
        const int vch = cp4 >> 2, ngrp = (w2 + 3) >> 2;
        for (int e = tid; e < vch * ngrp; e += kBJThreads) {
          const int ch = e % vch, c0 = (e / vch) * 4;
          float4 acc[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int k2 = 0; k2 < w2; ++k2) {
            const float4 v = reinterpret_cast<const float4*>(Vs + (size_t)k2 * cp4)[ch];
            const float4 qv = *reinterpret_cast<const float4*>(Qs + k2 * ldq + c0);
            const float qq[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              acc[j].x = fmaf(v.x, qq[j], acc[j].x);
              acc[j].y = fmaf(v.y, qq[j], acc[j].y);
              acc[j].z = fmaf(v.z, qq[j], acc[j].z);
              acc[j].w = fmaf(v.w, qq[j], acc[j].w);
            }
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int l = c0 + j;
            if (l < w2) {
              const int gc = (l < w ? ba * w + l : bb * w + (l - w));
              float* dst = V + (size_t)gc * ldv + 4 * ch;
              const float a4[4] = {acc[j].x, acc[j].y, acc[j].z, acc[j].w};
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (4 * ch + u < cpad) dst[u] = a4[u];
            }
          }
        }
      }
      if (P > 1) {
        if (!grid_barrier(bar, P, err)) return;
      } else {
        __syncthreads();
      }
    }
    // convergence test over the whole grid
    if (P > 1) {
      if (tid == 0 && s_rot) atomicAdd(&rot[sweep], 1);
      if (!grid_barrier(bar, P, err)) return;
      if (__ldcg(&rot[sweep]) == 0) break;
    } else {
      __syncthreads();
      if (!s_rot) break;
    }
    __syncthreads();
  }
  if (g == 0 && tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// The same block Jacobi on one thread-block cluster (P <= 8 CTAs): the
// columns stay in shared memory for the whole solve.  At the end of a round
// each CTA sends its two blocks straight into the shared memory of the CTAs
// that take them in the next round (double-buffered by round parity), the V
// block as V_blk Q, so a round costs one cluster barrier and no global
// traffic.  Shared memory: Mb [2][2w][rp], Vb [2][2w][cp4], Qs [2w][ldq],
// nrm [2w].
constexpr int kBJMaxCluster = 8;

__device__ __forceinline__ void bj_blocks(int g, int round, int nblk, int& ba, int& bb) {
  ba = (g == 0) ? 0 : 1 + add_mod(g - 1, round, nblk - 1);
  bb = 1 + add_mod(nblk - 2 - g, round, nblk - 1);
}

template <int NCH>
__global__ void __launch_bounds__(kBJThreads) k_block_jacobi_cl(int r, int cpad, int w, float* __restrict__ M,
                                                                int ldm, float* __restrict__ V, int ldv,
                                                                float tol, int max_sweeps,
                                                                int* __restrict__ sweeps_out,
                                                                const float* __restrict__ floor_ptr) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w2 = 2 * w;
  const int rp = (r + 3) & ~3, cp4 = (cpad + 3) & ~3;
  const int ldq = (w2 + 7) & ~3;
  float* Mb = reinterpret_cast<float*>(smem_raw);
  float* Vb = Mb + 2 * (size_t)w2 * rp;
  float* Qs = Vb + 2 * (size_t)w2 * cp4;
  float* nrm = Qs + w2 * ldq;
  __shared__ int s_rot;
  __shared__ int rotf[2][kBJMaxCluster];  // per-CTA "rotated" flags, by sweep parity
  const int P = (int)cl.num_blocks(), g = (int)cl.block_rank(), nblk = 2 * P;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kBJThreads / 32;
  const float nfloor = floor_ptr ? *floor_ptr : 0.f;
  const float tol2 = tol * tol;
  int ba, bb;
  bj_blocks(g, 0, nblk, ba, bb);
  // round 0's blocks into buffer 0
  for (int l = warp; l < w2; l += nw) {
    const int gc = (l < w ? ba * w + l : bb * w + (l - w));
    const float* src = M + (size_t)gc * ldm;
    float* dst = Mb + (size_t)l * rp;
    for (int i = lane; i < rp; i += 32) dst[i] = i < r ? src[i] : 0.f;
    const float* vsrc = V + (size_t)gc * ldv;
    float* vdst = Vb + (size_t)l * cp4;
    for (int i = lane; i < cp4; i += 32) vdst[i] = i < cpad ? vsrc[i] : 0.f;
  }
  __syncthreads();
  int buf = 0, sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    for (int round = 0; round < nblk - 1; ++round) {
      bj_blocks(g, round, nblk, ba, bb);
      float* Ms = Mb + (size_t)buf * w2 * rp;
      float* Vs = Vb + (size_t)buf * w2 * cp4;
      // squared norms of the 2w columns; Q = I
      for (int l = warp; l < w2; l += nw) {
        const float4* col = reinterpret_cast<const float4*>(Ms + (size_t)l * rp);
        float s2 = 0.f;
        for (int c = lane; c < (rp >> 2); c += 32) {
          const float4 v = col[c];
          s2 = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, s2))));
        }
        s2 = warp_sum(s2);
        if (lane == 0) nrm[l] = s2;
      }
      for (int e = tid; e < w2 * ldq; e += kBJThreads) {
        const int i = e / ldq, j = e - i * ldq;
        Qs[e] = (i == j) ? 1.f : 0.f;
      }
      __syncthreads();
      bj_round<NCH>(round, w, rp, Ms, Qs, ldq, nrm, nfloor, tol2, &s_rot);
      __syncthreads();
      // where this CTA's blocks go next (round 0 of the next sweep after the last round)
      const int nr = (round + 1 == nblk - 1) ? 0 : round + 1;
      int dst_cta[2], dst_slot[2];
      {
        const int mine[2] = {ba, bb};
        for (int s = 0; s < 2; ++s) {
          dst_cta[s] = 0;
          dst_slot[s] = 0;
          for (int q = 0; q < P; ++q) {
            int qa, qb;
            bj_blocks(q, nr, nblk, qa, qb);
            if (qa == mine[s]) { dst_cta[s] = q; dst_slot[s] = 0; }
            if (qb == mine[s]) { dst_cta[s] = q; dst_slot[s] = 1; }
          }
        }
      }
      float* Mn = Mb + (size_t)(buf ^ 1) * w2 * rp;
      float* Vn = Vb + (size_t)(buf ^ 1) * w2 * cp4;
      // M columns: copy into the receivers' next buffer
      {
        const int rch = rp >> 2;
        for (int e = tid; e < w2 * rch; e += kBJThreads) {
          const int l = e / rch, ch = e - l * rch, s = l < w ? 0 : 1, li = l - s * w;
          float4* dst = reinterpret_cast<float4*>(
              cl.map_shared_rank(Mn + (size_t)(dst_slot[s] * w + li) * rp, dst_cta[s]));
          dst[ch] = reinterpret_cast<const float4*>(Ms + (size_t)l * rp)[ch];
        }
      }
      // V columns: V_blk Q into the receivers' next buffer
      {
        const int vch = cp4 >> 2, ngrp = (w2 + 3) >> 2;
        for (int e = tid; e < vch * ngrp; e += kBJThreads) {
          const int ch = e % vch, c0 = (e / vch) * 4;
          float4 acc[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int k2 = 0; k2 < w2; ++k2) {
            const float4 v = reinterpret_cast<const float4*>(Vs + (size_t)k2 * cp4)[ch];
            const float4 qv = *reinterpret_cast<const float4*>(Qs + k2 * ldq + c0);
            const float qq[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              acc[j].x = fmaf(v.x, qq[j], acc[j].x);
              acc[j].y = fmaf(v.y, qq[j], acc[j].y);
              acc[j].z = fmaf(v.z, qq[j], acc[j].z);
              acc[j].w = fmaf(v.w, qq[j], acc[j].w);
            }
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int l = c0 + j;
            if (l < w2) {
              const int s = l < w ? 0 : 1, li = l - s * w;
              float4* dst = reinterpret_cast<float4*>(
                  cl.map_shared_rank(Vn + (size_t)(dst_slot[s] * w + li) * cp4, dst_cta[s]));
              dst[ch] = acc[j];
            }
          }
        }
      }
      if (round == nblk - 2 && tid < P) *cl.map_shared_rank(&rotf[sweep & 1][g], tid) = s_rot;
      cl.sync();
      buf ^= 1;
    }
    int any = 0;
    for (int q = 0; q < P; ++q) any |= rotf[sweep & 1][q];
    if (!any) break;
  }
  // the current buffer holds round 0's blocks
  __syncthreads();
  bj_blocks(g, 0, nblk, ba, bb);
  const float* Ms = Mb + (size_t)buf * w2 * rp;
  const float* Vs = Vb + (size_t)buf * w2 * cp4;
  for (int l = warp; l < w2; l += nw) {
    const int gc = (l < w ? ba * w + l : bb * w + (l - w));
    float* dst = M + (size_t)gc * ldm;
    for (int i = lane; i < r; i += 32) dst[i] = Ms[(size_t)l * rp + i];
    float* vdst = V + (size_t)gc * ldv;
    for (int i = lane; i < cpad; i += 32) vdst[i] = Vs[(size_t)l * cp4 + i];
  }
  if (g == 0 && tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// identity (cpad x cpad) and copy/convert of an r x c matrix into an r x cpad
// padded one (zero padding columns)
// Power of two 2^-e with 2^(e-1) <= max |A| < 2^e (1 for a zero matrix), one block.
__global__ void k_pow2_scale(int r, int c, const double* __restrict__ A, int lda, float* __restrict__ out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int j = threadIdx.x >> 5; j < c; j += blockDim.x >> 5)
    for (int i = threadIdx.x & 31; i < r; i += 32) m = fmax(m, fabs(A[i + (size_t)j * lda]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v = fmax(v, red[k]);
    int e = 0;
    if (v > 0.0) frexp(v, &e);
    *out = (float)ldexp(1.0, -e);
  }
}

// M (r x cpad, ld r) = scale * A padded with zero columns; V = I (cpad x cpad)
template <typename TI, typename TO>
__global__ void k_pad_copy(int r, int c, int cpad, const TI* __restrict__ A, int lda,
                           TO* __restrict__ M, TO* __restrict__ V, const float* __restrict__ scale) {
  const TI sc = scale ? (TI)*scale : TI(1);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * cpad; e += gridDim.x * blockDim.x) {
    int i = e % r, j = e / r;
    M[e] = j < c ? (TO)(sc * A[i + j * lda]) : TO(0);
  }
  if (V)
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cpad * cpad; e += gridDim.x * blockDim.x) {
      int i = e % cpad, j = e / cpad;
      V[e] = i == j ? TO(1) : TO(0);
    }
}

// V64 (c x c, ld c) = V32 (top-left of cpad x cpad)
__global__ void k_v32_to_64(int c, int cpad, const float* __restrict__ V32, double* __restrict__ V) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c * c; e += gridDim.x * blockDim.x) {
    int i = e % c, j = e / c;
    V[e] = (double)V32[i + j * cpad];
  }
}


// scratch of one whitening (whiten())
struct WhitenScratch {
  double *W1, *W2, *T, *E, *E2, *F;
};

struct PencilWs {
  double *W1, *W2, *T, *E, *E2, *F, *C, *V, *Vp, *M, *Mp, *sig, *mu;
  WhitenScratch wb;                    // the SVD pencil's second whitening (beside the first)
  double* sh;                          // [4] bracket and scales of the eigen shift
  int* shok;                           // [kShiftTrials] definiteness trials
  double* cond;                        // [4] condition estimates of the whitened Grams, drop counts
  float *L32, *Li32, *M32, *V32, *fs;  // fs: [0] Jacobi norm floor, [1] scale
  float *Hq, *tq;                      // QR preconditioner: reflectors (c x c), taus
  int *drop1, *drop2, *order, *nvalid, *rot, *err, *sweeps, *cid, *cst;
  GridBarrier* bar;
};

// Block layout of the Jacobi columns: 2P blocks of w <= 16 columns (a block
// pair's 2w columns index the lanes of the round's Q), P CTAs.
static int bj_cpad(int c, int* w_out, int* P_out, size_t elt, int r) {
  int w, P;
  if (c <= 32) {
    w = (c + 1) / 2;
    if (w < 1) w = 1;
    P = 1;
  } else {
    w = 16;
    size_t per_w = 2 * (size_t)(r + c + 64) * elt;
    while (w > 1 && per_w * w > 200 * 1024) --w;
    P = (c + 2 * w - 1) / (2 * w);
  }
  *w_out = w;
  *P_out = P;
  return 2 * P * w;
}

static bool carve_pencil(Arena& ar, int b1, int b2, PencilWs& w) {
  int bm = b1 > b2 ? b1 : b2;
  int ww, P;
  int cp8 = bj_cpad(b2 > b1 ? b2 : b1, &ww, &P, 8, bm);
  int cp4 = bj_cpad(b2 > b1 ? b2 : b1, &ww, &P, 4, bm);
  int cp = cp8 > cp4 ? cp8 : cp4;
  size_t bb = (size_t)bm * bm, cc = (size_t)cp * cp, rc = (size_t)bm * cp;
  w.W1 = ar.take<double>(bb);
  w.W2 = ar.take<double>(bb);
  w.T = ar.take<double>(bb);
  w.E = ar.take<double>(bb);
  w.E2 = ar.take<double>(bb);
  w.F = ar.take<double>(bb);
  w.C = ar.take<double>(bb);
  w.V = ar.take<double>(bb);
  w.wb.W1 = ar.take<double>(bb);
  w.wb.W2 = ar.take<double>(bb);
  w.wb.T = ar.take<double>(bb);
  w.wb.E = ar.take<double>(bb);
  w.wb.E2 = ar.take<double>(bb);
  w.wb.F = ar.take<double>(bb);
  w.Vp = ar.take<double>(cc);
  w.M = ar.take<double>(rc);
  w.Mp = ar.take<double>(rc);
  w.sig = ar.take<double>(cp);
  w.mu = ar.take<double>(2);
  w.sh = ar.take<double>(4);
  w.shok = ar.take<int>(kShiftTrials);
  w.cond = ar.take<double>(4);
  w.fs = ar.take<float>(4);
  w.L32 = ar.take<float>(bb);
  w.Li32 = ar.take<float>(bb);
  w.M32 = ar.take<float>(rc);
  w.V32 = ar.take<float>(cc);
  w.Hq = ar.take<float>(cc);
  w.tq = ar.take<float>(cp);
  w.drop1 = ar.take<int>(bm);
  w.drop2 = ar.take<int>(bm);
  w.order = ar.take<int>(cp);
  w.nvalid = ar.take<int>(1);
  w.rot = ar.take<int>(64);
  w.err = ar.take<int>(1);
  w.sweeps = ar.take<int>(2);
  w.cid = ar.take<int>(cp);
  w.cst = ar.take<int>(cp + 1);
  w.bar = ar.take<GridBarrier>(1);
  return !ar.overflow;
}

// Condition estimate of a whitened Gram matrix G (b x b) from its whitener
// W (W^T G W = I on the kept part, so G^-1 = W W^T there):
//   out = max_i G_ii * max_i sum_j W_ij^2 = max_i G_ii * max_i (G^-1)_ii.
// Each factor is at most the matching extreme eigenvalue and at least 1/b of
// it, so out lies in [cond_2(G) / b^2, cond_2(G)].  Also writes the number
// of dropped columns (drop flags) to out[2].  One block.
__global__ void k_cond_est(int b, const double* __restrict__ G, const double* __restrict__ W,
                           const int* __restrict__ drop, double* __restrict__ out) {
  __shared__ double sg[32], sw[32];
  __shared__ int sd[32];
  double mg = 0.0, mw = 0.0;
  int nd = 0;
  for (int i = threadIdx.x; i < b; i += blockDim.x) {
    nd += drop[i] != 0;
    mg = fmax(mg, G[i + (size_t)i * b]);
    double acc = 0.0;
    for (int j = 0; j < b; ++j) {
      const double w = W[i + (size_t)j * b];
      acc = fma(w, w, acc);
    }
    mw = fmax(mw, acc);
  }
  mg = warp_max(mg);
  mw = warp_max(mw);
  nd = warp_sum(nd);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sg[wid] = mg;
    sw[wid] = mw;
    sd[wid] = nd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      mg = fmax(mg, sg[i]);
      mw = fmax(mw, sw[i]);
      nd += sd[i];
    }
    out[0] = mg * mw;
    out[2] = (double)nd;
  }
}

// Whitening matrix W (b x b) with W^T G W = I on the kept part: FP32
// Cholesky for W0 = L^-T, then three steps of iterative refinement
// W <- W (I - E/2 + 3/8 E^2), E = W^T G W - I, whose error cubes per step.
// E is formed in FP64; the correction W (E/2 - 3/8 E^2) only needs FP32
// relative accuracy (its rounding, u32 |E|, is what the next step removes),
// so E^2 and W F are FP32 products.
static void whiten(cudaStream_t s, int b, const double* G, const WhitenScratch& w, int* dropped, double* Wout) {
  const int g1 = (b * b + 255) / 256;
  if (b <= kCT * kCTMax) {
    const size_t sm = chol_blocked_smem(b);
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(k_chol_inv_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_chol_inv_blocked<<<1, kChThreads, sm, s>>>(b, G, b, dropped, w.W1);
  } else {
    const size_t sm = ((size_t)b * (b + 1) / 2 + 2 * (size_t)b) * sizeof(float);
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(k_chol_inv_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_chol_inv_f32<<<1, kSmallThreads, sm, s>>>(b, G, b, dropped, w.W1);
  }
  // every step writes the other buffer (the products never run in place);
  // the result is copied to Wout at the end (which may be either buffer)
  double* Wc = w.W1;
  double* Wn = w.W2;
  for (int it = 0; it < 3; ++it) {
    gemm_small(s, 0, 0, b, b, b, 1.0, G, b, Wc, b, 0.0, w.T, b);        // T = G W
    gemm_small_sym(s, b, b, Wc, b, w.T, b, w.E, b);                       // E = W^T T (symmetric)
    k_whiten_corr<<<g1, 256, 0, s>>>(b, w.E, nullptr, dropped, nullptr, 0);
    gemm_mixed(s, 0, 0, b, b, b, 1.0, w.E, b, w.E, b, 0.0, w.E2, b);    // E^2
    k_whiten_corr<<<g1, 256, 0, s>>>(b, w.E, w.E2, dropped, w.F, 1);    // F = E/2 - 3/8 E^2
    cudaMemcpyAsync(Wn, Wc, (size_t)b * b * sizeof(double), cudaMemcpyDeviceToDevice, s);
    gemm_mixed(s, 0, 0, b, b, b, -1.0, Wc, b, w.F, b, 1.0, Wn, b);      // W - W F
    double* t = Wc;
    Wc = Wn;
    Wn = t;
  }
  if (Wc != Wout) cudaMemcpyAsync(Wout, Wc, (size_t)b * b * sizeof(double), cudaMemcpyDeviceToDevice, s);
  note_launches(16);
}

// A second stream per caller stream (and device) for independent small steps
// (the SVD pencil's two whitenings), created on first use and kept for the
// life of the process; work forks to it and joins back through events, which
// stream capture records as two parallel branches.
struct SideStream {
  cudaStream_t s2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

static std::mutex g_side_mu;
static std::map<std::pair<int, cudaStream_t>, SideStream> g_side_pool;

static rr_status side_stream(cudaStream_t s, SideStream* out) {
  auto& mu = g_side_mu;
  auto& pool = g_side_pool;
  int dev = 0;
  RR_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = pool.find({dev, s});
  if (it == pool.end()) {
    SideStream ss;
    RR_CUDA(cudaStreamCreateWithFlags(&ss.s2, cudaStreamNonBlocking));
    RR_CUDA(cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming));
    RR_CUDA(cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming));
    it = pool.emplace(std::make_pair(dev, s), ss).first;
  }
  *out = it->second;
  return RR_OK;
}

// Fork independent work of the caller's stream s onto its side stream (*s2
// runs after s's work so far) and join it back (s waits for *s2's work).
rr_status side_fork(cudaStream_t s, cudaStream_t* s2) {
  SideStream ss;
  RR_TRY(side_stream(s, &ss));
  RR_CUDA(cudaEventRecord(ss.fork, s));
  RR_CUDA(cudaStreamWaitEvent(ss.s2, ss.fork, 0));
  *s2 = ss.s2;
  return RR_OK;
}

rr_status side_join(cudaStream_t s) {
  SideStream ss;
  RR_TRY(side_stream(s, &ss));
  RR_CUDA(cudaEventRecord(ss.join, ss.s2));
  RR_CUDA(cudaStreamWaitEvent(s, ss.join, 0));
  return RR_OK;
}

rr_status pencil_side_prepare(cudaStream_t s) {
  SideStream ss;
  return side_stream(s, &ss);
}

// Destroy the side stream of s (before s itself is destroyed; its work must be
// complete).
void pencil_side_release(cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lock(g_side_mu);
  auto it = g_side_pool.find({dev, s});
  if (it == g_side_pool.end()) return;
  cudaStreamDestroy(it->second.s2);
  cudaEventDestroy(it->second.fork);
  cudaEventDestroy(it->second.join);
  g_side_pool.erase(it);
}

// floor[0] = scale * max_j |M(:, j)|^2 (one block)
template <typename T>
__global__ void k_colnorm_floor(int r, int c, const T* __restrict__ M, int ldm, T scale, T* __restrict__ floor_out) {
  __shared__ T red[32];
  T mx = T(0);
  for (int j = threadIdx.x >> 5; j < c; j += blockDim.x >> 5) {
    T sacc = T(0);
    for (int i = threadIdx.x & 31; i < r; i += 32) sacc = fma(M[i + (size_t)j * ldm], M[i + (size_t)j * ldm], sacc);
    sacc = warp_sum(sacc);
    mx = fmax(mx, sacc);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    T m = T(0);
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmax(m, red[k]);
    *floor_out = scale * m;
  }
}

static size_t bj_smem(int r, int cpad, int w) {
  const size_t rp = (r + 3) & ~3, cp4 = (cpad + 3) & ~3;
  const size_t ldq = (2 * w + 7) & ~3;
  return ((size_t)2 * w * (rp + cp4) + (size_t)2 * w * ldq + 2 * (size_t)w) * sizeof(float);
}

static size_t bj_cl_smem(int r, int cpad, int w) {
  const size_t rp = (r + 3) & ~3, cp4 = (cpad + 3) & ~3;
  const size_t ldq = (2 * w + 7) & ~3;
  return ((size_t)4 * w * (rp + cp4) + (size_t)2 * w * ldq + 2 * (size_t)w) * sizeof(float);
}

static rr_status launch_bj(cudaStream_t s, int r, int cpad, int w, int P, float* M, float* V, float tol,
                           int max_sweeps, PencilWs& ws, const float* floor_ptr = nullptr) {
  const int rp = (r + 3) & ~3;
  if (rp > 128 * kBJMaxChunks || cpad > 128 * kBJMaxChunks || 2 * w > 32 || w < 1) return RR_ERR_ARG;
  const size_t csm = bj_cl_smem(r, cpad, w);
  if (P <= kBJMaxCluster && csm <= 220 * 1024) {
    // one cluster: columns stay in shared memory, no global barrier
    const void* fn = rp <= 128 ? (const void*)k_block_jacobi_cl<1>
                     : rp <= 256 ? (const void*)k_block_jacobi_cl<2>
                                 : (const void*)k_block_jacobi_cl<3>;
    if (csm > 48 * 1024)
      RR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P);
    cfg.blockDim = dim3(kBJThreads);
    cfg.dynamicSmemBytes = csm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = P;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ld = r, ldv = cpad;
    int* sw = ws.sweeps;
    void* args[] = {&r, &cpad, &w, &M, &ld, &V, &ldv, &tol, &max_sweeps, &sw, &floor_ptr};
    RR_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
    note_launches(1);
    return RR_OK;
  }
  const size_t smem = bj_smem(r, cpad, w);
  const void* fn = rp <= 128 ? (const void*)k_block_jacobi<1>
                   : rp <= 256 ? (const void*)k_block_jacobi<2>
                               : (const void*)k_block_jacobi<3>;
  if (smem > 48 * 1024)
    RR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  RR_CUDA(cudaMemsetAsync(ws.rot, 0, 64 * sizeof(int), s));
  RR_CUDA(cudaMemsetAsync(ws.bar, 0, sizeof(GridBarrier), s));
  int ld = r, ldv = cpad;
  int* rot = ws.rot;
  GridBarrier* bar = ws.bar;
  int* err = ws.err;
  int* sw = ws.sweeps;
  const float* fl = floor_ptr;
  void* args[] = {&r, &cpad, &w, &M, &ld, &V, &ldv, &tol, &max_sweeps, &rot, &bar, &err, &sw, &fl};
  if (P == 1) {
    // a single CTA never waits on another one: plain launch
    RR_CUDA(cudaLaunchKernel(fn, dim3(1), dim3(kBJThreads), args, smem, s));
    return check_launch("block_jacobi");
  }
  RR_CUDA(cudaLaunchCooperativeKernel(fn, dim3(P), dim3(kBJThreads), args, smem, s));
  note_launches(1);
  return RR_OK;
}

// ---------------------------------------------------------------------------
// QR preconditioning of the one-sided Jacobi (the preconditioned Jacobi SVD
// of Drmac and Veselic).  With the column-pivoted Householder QR
// C^T P = Q R, the Jacobi runs on X = C Q (whose columns are the rows of R,
// graded by the pivoting) and accumulates its rotations onto Q, so that
// X J = C (Q J) and V = Q J.  Graded columns need about half the sweeps of
// C's own columns.
//
// One cluster of NC CTAs holds A = s C^T (c x r, s the power-of-two scale) in
// registers: CTA z owns the columns k = z 16 CPW + 16 u + warp (u < CPW),
// lane l the rows t 32 + l (t < RPL).  Step j takes the reflector of the
// column with the largest remaining norm (rows >= j; ties to the lower
// column), applies it to every column not yet pivoted, recomputes their
// remaining norms exactly (rows > j), and each CTA publishes the reflector of
// its best column into every CTA's shared memory (double-buffered by step
// parity: one cluster barrier per step).  The reflector of x (rows >= j) is
// v = x - beta e_j, beta = -sign(x_j) |x|, tau = 1 / (beta (beta - x_j)), so
// that (I - tau v v^T) x = beta e_j.  Q = H_0 H_1 ... H_{c-1} is formed
// afterwards by backward accumulation from the stored reflectors; every CTA
// owns whole columns of Q, so that part needs no barrier.
constexpr int kQrThreads = 512;
constexpr int kQrWarps = kQrThreads / 32;
constexpr int kQrMaxNC = 8;
constexpr int kQrMaxRows = 384;  // 32 x 12

struct QrCand {
  float nrm2;  // squared norm of the candidate's remaining part (-1: none)
  int col;
  float tau, beta;
};

__device__ __forceinline__ bool qr_better(float n, int k, float bn, int bk) {
  return n > bn || (n == bn && k < bk);
}

// Warp sums of N (a power of two <= 32) per-lane values at once
// (reduce-scatter: halving exchanges over the top lane bits, then butterflies
// over the rest): on return lane l holds the sum of value l >> (5 - log2 N).
template <int N>
__device__ __forceinline__ float qr_rs(float d[N]) {
  static_assert(N >= 1 && N <= 32 && (N & (N - 1)) == 0, "power of two");
  constexpr int L = N >= 32 ? 5 : N >= 16 ? 4 : N >= 8 ? 3 : N >= 4 ? 2 : N >= 2 ? 1 : 0;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int st = 0; st < L; ++st) {
    const int h = N >> (st + 1), b = 16 >> st;
    const bool up = lane & b;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? d[i] : d[i + h], keep = up ? d[i + h] : d[i];
      d[i] = keep + __shfl_xor_sync(0xffffffffu, send, b);
    }
  }
  float v = d[0];
#pragma unroll
  for (int b = 16 >> L; b >= 1; b >>= 1) v += __shfl_xor_sync(0xffffffffu, v, b);
  return v;
}
// lane holding value u after qr_rs<N>
template <int N>
__device__ __forceinline__ int qr_rs_lane(int u) {
  return u * (32 / N);
}

// (squared norm, column) as one key, larger norm first, then lower column;
// 0 = no candidate
__device__ __forceinline__ unsigned long long qr_key(float n2, int col) {
  return ((unsigned long long)__float_as_uint(n2) << 32) | (unsigned)(~col);
}

template <int RPL, int CPW>
__global__ void __launch_bounds__(kQrThreads, 1)
    k_qr_precond(int r, int c, const double* __restrict__ C, const float* __restrict__ scale,
                 float* __restrict__ X, int cpad, float* __restrict__ Vq, float* __restrict__ Hv,
                 float* __restrict__ tq) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ __align__(16) float vbuf[2][kQrMaxNC][kQrMaxRows];
  __shared__ QrCand cand[2][kQrMaxNC];
  __shared__ unsigned long long s_key[2];
  const int NC = (int)cl.num_blocks();
  const int z = (int)cl.block_rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float sc = *scale;
  const int col0 = z * kQrWarps * CPW + warp;  // column of slot u: col0 + 16 u
  if (threadIdx.x < 2) s_key[threadIdx.x] = 0ull;

  float a[CPW][RPL];
  unsigned done = 0;  // slot u pivoted already (or beyond the last column)
#pragma unroll
  for (int u = 0; u < CPW; ++u) {
    const int k = col0 + kQrWarps * u;
    if (k >= r) done |= 1u << u;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int i = t * 32 + lane;
      a[u][t] = (k < r && i < c) ? (float)((double)sc * C[k + (size_t)i * r]) : 0.f;
    }
  }
  __syncthreads();

  // best remaining column of this CTA (rows > j) -> reflector for step j + 1
  // into buffer `par` of every CTA
  auto publish = [&](int j, int par) {
    float d[CPW];
#pragma unroll
    for (int u = 0; u < CPW; ++u) {
      float s2 = 0.f;
#pragma unroll
      for (int t = 0; t < RPL; ++t)
        if (t * 32 + lane > j) s2 = fmaf(a[u][t], a[u][t], s2);
      d[u] = s2;
    }
    const float n2 = qr_rs<CPW>(d);          // lane l: slot l / (32 / CPW)
    const int us = lane / (32 / CPW);
    const bool live = !((done >> us) & 1u);
    const unsigned long long key = live ? qr_key(n2, col0 + kQrWarps * us) : 0ull;
    const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
    const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
    const unsigned long long wk = ((unsigned long long)mhi << 32) | mlo;
    if (lane == 0 && wk) atomicMax(&s_key[par], wk);
    __syncthreads();
    const unsigned long long bk = s_key[par];
    if (bk == 0ull) {  // every column of this CTA is pivoted: publish "none"
      if (threadIdx.x < NC) {
        QrCand* dst = cl.map_shared_rank(&cand[par][z], (int)threadIdx.x);
        *dst = QrCand{-1.f, INT_MAX, 0.f, 0.f};
      }
      return;
    }
    const int ck = (int)(~(unsigned)bk);
    const float cn = __uint_as_float((unsigned)(bk >> 32));
    const int rel = ck - z * kQrWarps * CPW;
    if (warp != rel % kQrWarps) return;
    const int bu = rel / kQrWarps;
    const int j1 = j + 1;
    float x[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) x[t] = 0.f;
#pragma unroll
    for (int u = 0; u < CPW; ++u)
      if (u == bu) {
#pragma unroll
        for (int t = 0; t < RPL; ++t) x[t] = a[u][t];
      }
    float xj = 0.f;
#pragma unroll
    for (int t = 0; t < RPL; ++t)
      if (t == (j1 >> 5)) xj = x[t];
    xj = __shfl_sync(0xffffffffu, xj, j1 & 31);
    const float beta = -copysignf(sqrtf(cn), xj);
    const float tau = cn > 0.f ? 1.f / (beta * (beta - xj)) : 0.f;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int i = t * 32 + lane;
      x[t] = i > j1 ? x[t] : (i == j1 ? xj - beta : 0.f);
    }
    for (int q = 0; q < NC; ++q) {
      float* dst = cl.map_shared_rank(&vbuf[par][z][0], q);
#pragma unroll
      for (int t = 0; t < RPL; ++t) dst[t * 32 + lane] = x[t];
      if (lane == 0) *cl.map_shared_rank(&cand[par][z], q) = QrCand{cn, ck, tau, beta};
    }
  };

  publish(-1, 0);
  for (int j = 0; j < c; ++j) {
    cl.sync();
    const int par = j & 1;
    // the key publish(j - 1) filled (read before this step's cluster barrier;
    // filled next by publish(j + 1), after the next one)
    if (threadIdx.x == 0) s_key[par] = 0ull;
    QrCand b = cand[par][0];
    int zs = 0;
    for (int q = 1; q < NC; ++q) {
      const QrCand m = cand[par][q];
      if (qr_better(m.nrm2, m.col, b.nrm2, b.col)) {
        b = m;
        zs = q;
      }
    }
    const float* v = &vbuf[par][zs][0];
    float vr[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) vr[t] = v[t * 32 + lane];
    if (z == j % NC) {
      for (int i = threadIdx.x; i < c; i += kQrThreads) Hv[(size_t)j * c + i] = v[i];
      if (threadIdx.x == 0) tq[j] = b.tau;
    }
    // w_u = tau v^T a_u for the warp's 8 columns at once, then a_u -= w_u v
    // (pivoted columns have zero entries at rows >= j: no change)
    float d[CPW];
#pragma unroll
    for (int u = 0; u < CPW; ++u) {
      float s2 = 0.f;
#pragma unroll
      for (int t = 0; t < RPL; ++t) s2 = fmaf(vr[t], a[u][t], s2);
      d[u] = s2;
    }
    const float wsum = qr_rs<CPW>(d) * b.tau;
#pragma unroll
    for (int u = 0; u < CPW; ++u) {
      const float wu = __shfl_sync(0xffffffffu, wsum, qr_rs_lane<CPW>(u));
      const int k = col0 + kQrWarps * u;
      if (k == b.col) {  // the pivot column becomes beta e_j
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
          const int i = t * 32 + lane;
          a[u][t] = i == j ? b.beta : (i > j ? 0.f : a[u][t]);
        }
        done |= 1u << u;
      } else if (!((done >> u) & 1u)) {
#pragma unroll
        for (int t = 0; t < RPL; ++t) a[u][t] = fmaf(-wu, vr[t], a[u][t]);
      }
    }
    if (j + 1 < c) publish(j, par ^ 1);
  }

  // X (r x cpad, ld r) = (Q^T A)^T = s C Q; zero padding columns
#pragma unroll
  for (int u = 0; u < CPW; ++u) {
    const int k = col0 + kQrWarps * u;
    if (k >= r) continue;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int i = t * 32 + lane;
      if (i < c) X[k + (size_t)i * r] = a[u][t];
    }
  }
  if (z == 0) {
    for (int e = threadIdx.x; e < (cpad - c) * r; e += kQrThreads) X[(size_t)c * r + e] = 0.f;
    // V padding: rows >= c of the first c columns zero, identity beyond
    for (int e = threadIdx.x; e < cpad * cpad; e += kQrThreads) {
      const int i = e % cpad, k = e / cpad;
      if (i >= c || k >= c) Vq[e] = (i == k) ? 1.f : 0.f;
    }
  }
  __threadfence();
  cl.sync();  // every reflector stored

  // Q by backward accumulation: Q^(j) = H_j Q^(j+1); columns k < j of
  // Q^(j+1) are e_k, which H_j leaves alone (v_k = 0 for k < j)
#pragma unroll
  for (int u = 0; u < CPW; ++u) {
    const int k = col0 + kQrWarps * u;
#pragma unroll
    for (int t = 0; t < RPL; ++t) a[u][t] = (t * 32 + lane == k) ? 1.f : 0.f;
  }
  float vn[RPL];
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int i = t * 32 + lane;
    vn[t] = i < c ? __ldcg(&Hv[(size_t)(c - 1) * c + i]) : 0.f;
  }
  float taun = __ldcg(&tq[c - 1]);
  for (int j = c - 1; j >= 0; --j) {
    float vr[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) vr[t] = vn[t];
    const float tau = taun;
    if (j > 0) {  // prefetch the next reflector
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int i = t * 32 + lane;
        vn[t] = i < c ? __ldcg(&Hv[(size_t)(j - 1) * c + i]) : 0.f;
      }
      taun = __ldcg(&tq[j - 1]);
    }
    if (tau == 0.f) continue;
    float d[CPW];
#pragma unroll
    for (int u = 0; u < CPW; ++u) {
      float s2 = 0.f;
#pragma unroll
      for (int t = 0; t < RPL; ++t) s2 = fmaf(vr[t], a[u][t], s2);
      d[u] = s2;
    }
    const float wsum = qr_rs<CPW>(d) * tau;
#pragma unroll
    for (int u = 0; u < CPW; ++u) {
      const int k = col0 + kQrWarps * u;
      const float wu = __shfl_sync(0xffffffffu, wsum, qr_rs_lane<CPW>(u));
      if (k < j || k >= c) continue;
#pragma unroll
      for (int t = 0; t < RPL; ++t) a[u][t] = fmaf(-wu, vr[t], a[u][t]);
    }
  }
  // V (cpad x cpad, ld cpad): Q in the leading c x c block
#pragma unroll
  for (int u = 0; u < CPW; ++u) {
    const int k = col0 + kQrWarps * u;
    if (k >= c) continue;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int i = t * 32 + lane;
      if (i < c) Vq[i + (size_t)k * cpad] = a[u][t];
    }
  }
}

// the preconditioner applies for r >= c (A = C^T has at least as many
// columns as rows) and pencils wide enough for the saved sweeps to pay
constexpr int kQrMinCols = 160;

static bool qr_precond_applies(int r, int c) { return r >= c && c >= kQrMinCols && c <= kQrMaxRows; }

static rr_status launch_qr_precond(cudaStream_t s, int r, int c, const double* C, const float* scale, float* X,
                                   int cpad, float* V, float* Hv, float* tq) {
  const int rpl = c <= 128 ? 4 : c <= 256 ? 8 : 12;
  const int cpw = rpl <= 8 ? 8 : 4;
  const int NC = (r + kQrWarps * cpw - 1) / (kQrWarps * cpw);
  if (c > r || c > kQrMaxRows || NC > kQrMaxNC || cpad < c) return RR_ERR_ARG;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(NC);
  cfg.blockDim = dim3(kQrThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = NC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (rpl == 4)
    RR_CUDA(cudaLaunchKernelEx(&cfg, k_qr_precond<4, 8>, r, c, C, scale, X, cpad, V, Hv, tq));
  else if (rpl == 8)
    RR_CUDA(cudaLaunchKernelEx(&cfg, k_qr_precond<8, 8>, r, c, C, scale, X, cpad, V, Hv, tq));
  else
    RR_CUDA(cudaLaunchKernelEx(&cfg, k_qr_precond<12, 4>, r, c, C, scale, X, cpad, V, Hv, tq));
  note_launches(1);
  return RR_OK;
}

// ---------------------------------------------------------------------------
// FP64 refinement of the FP32 Jacobi result (a Newton-type correction built
// from small GEMMs, in the manner of Ogita and Aishima's refinement of
// eigenvector bases).  With N = C V, K = N^T N (FP64), T = V^T V,
// lam_i = K_ii / T_ii and the coupling corrected for non-orthogonality
// c_ij = K_ij - (lam_i + lam_j) T_ij / 2, the update is V <- V (I + E),
//   E = (I - T)/2 + W,   W_ij = atan(2 c_ij / (lam_j - lam_i)) / 2 (skew),
// the exact angle of each pair (first order in the pairs' interaction), which
// orthogonalises V and diagonalises K with both defects squaring per step
// (applied as V (I + (I - T)/2 + W), the cross term being second order).
// Pairs that need a large rotation (|W_ij| > kBigAngle: close values with a
// coupling above rounding level) interact, and composing such rotations
// simultaneously diverges; they join clusters (runs of close values in sorted order, at
// most kClMax), and each cluster's block is diagonalised exactly instead
// (two-sided FP64 Jacobi, one warp per cluster), its rotation taking the
// place of W on the block.
// ---------------------------------------------------------------------------
constexpr double kBigAngle = 0.003;
// couplings at the rounding level of K (relative to the pair's lam) carry no
// direction information: such pairs are neither rotated nor linked (for
// (near-)equal lam their exact angle would be an arbitrary large rotation)
constexpr double kCoupleNoise = 1e-13;
// ... but a pair whose values are well apart (relative gap above kSepGap)
// is always rotated: its angle c_ij / (lam_j - lam_i) is small and fixed by
// c_ij even at the rounding level, and an angle left behind between a large
// and a small singular value returns in the small one's residual multiplied
// by (sigma_large / sigma_small)^2 (u = C v / sigma takes the v error into u
// amplified by sigma_large / sigma_small, and A^T u again): a skipped 1e-13
// coupling between sigma_1 and sigma_16 = sigma_1 / 64 alone leaves that
// pair at residual 4e-10.
constexpr double kSepGap = 1e-3;
constexpr int kClMax = 32;          // largest cluster resolved as one block
constexpr int kClWarps = 8;         // clusters resolved at once

__device__ __forceinline__ double oa_coupling(const double* K, const double* T, int c, int i, int j,
                                              double li, double lj) {
  return K[i + (size_t)j * c] - 0.5 * (li + lj) * T[i + (size_t)j * c];
}

// F1 = I + (I - T)/2 + W, W the exact pair angles outside the clusters
// (cid: cluster ids, -1 none); within a cluster only the orthogonality part.
// W itself goes to Wout: the caller adds W^2 / 2, so that I + W + W^2 / 2
// (exp(W) to second order) is orthogonal up to W^4 / 4 — with I + W alone
// the rotations' own W^2 defect (up to c kBigAngle^2) would have to be
// squared away by the following steps.
__global__ void k_oa_update(int c, const double* __restrict__ K, const double* __restrict__ T,
                            const int* __restrict__ cid, double* __restrict__ F1, double* __restrict__ Wout) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= c * c) return;
  const int i = e % c, j = e / c;
  const double Tij = T[e];
  double f = (i == j) ? 1.0 + 0.5 * (1.0 - Tij) : -0.5 * Tij;
  double wij = 0.0;
  if (i != j && !(cid[i] >= 0 && cid[i] == cid[j])) {
    const double li = K[i + (size_t)i * c] / T[i + (size_t)i * c];
    const double lj = K[j + (size_t)j * c] / T[j + (size_t)j * c];
    const double cij = oa_coupling(K, T, c, i, j, li, lj);
    const double big = fmax(fabs(li), fabs(lj));
    if (fabs(lj - li) > kSepGap * big || fabs(cij) > kCoupleNoise * big) wij = 0.5 * atan(2.0 * cij / (lj - li));
  }
  F1[e] = f + wij;
  Wout[e] = wij;
}

// Cluster detection and resolution (one CTA).  Sorted by lam, a pair
// needing |W_ij| > kBigAngle links every sorted position between its two
// members; the linked runs (at most kClMax) are the clusters.  The ordering
// and the link test are thresholds and run in FP32.  Each cluster's block
// B - mean(lam) I (B_ab = c_ab, B_aa = lam_a, formed in FP64) has entries of
// the size of the cluster's spread and couplings, so FP32 two-sided Jacobi on
// it gives the rotation Q to FP32 relative accuracy (the next FP64 step
// squares the rest away).  Outputs: cid (cluster id per index, -1 none),
// ord / st (members of cluster q: ord[st[q] .. st[q+1]-1]) and Qb (c x c,
// only the cluster blocks are written).
__global__ void __launch_bounds__(1024) k_cluster_rot(int c, const double* __restrict__ K,
                                                      const double* __restrict__ T,
                                                      double* __restrict__ Qb, int* __restrict__ cid,
                                                      int* __restrict__ ord, int* __restrict__ st) {
  extern __shared__ double cl_smem[];
  double* Sw = cl_smem;                                        // [kClWarps][kClMax][kClMax + 1]
  double* lam = Sw + kClWarps * kClMax * (kClMax + 1);         // [c]
  float* Bw = reinterpret_cast<float*>(lam + c);               // [kClWarps][kClMax][kClMax + 1]
  float* Qw = Bw + kClWarps * kClMax * (kClMax + 1);
  float* lamf = Qw + kClWarps * kClMax * (kClMax + 1);         // [c]
  int* order = reinterpret_cast<int*>(lamf + c);               // [c]
  int* pos = order + c;                                        // [c]
  int* link = pos + c;                                         // [c + 1] difference array of links
  int* start = link + c + 1;                                   // [c + 1]
  __shared__ int s_ncl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < c; i += blockDim.x) {
    // a zero (dropped) column has T_ii = 0: lambda 0 keeps the ranks below a permutation
    const double t = T[i + (size_t)i * c], li = t > 0.0 ? K[i + (size_t)i * c] / t : 0.0;
    lam[i] = isfinite(li) ? li : 0.0;
    lamf[i] = (float)lam[i];
  }
  for (int i = tid; i <= c; i += blockDim.x) link[i] = 0;
  __syncthreads();
  for (int i = tid; i < c; i += blockDim.x) {
    const float li = lamf[i];
    int rank = 0;
    for (int j = 0; j < c; ++j) rank += (lamf[j] < li || (lamf[j] == li && j < i)) ? 1 : 0;
    order[rank] = i;
    pos[i] = rank;
  }
  __syncthreads();
  const float tb = (float)tan(2.0 * kBigAngle);
  // every pair (i < j) once; four entries of K and T per thread in flight at
  // a time (one load after another made this pass most of the kernel's time)
  const int cc = c * c;
  for (int e0 = tid; e0 < cc; e0 += 4 * (int)blockDim.x) {
    float kv[4], tv[4];
    int ii[4], jj[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      ii[u] = e % c;
      jj[u] = e / c;
      ok[u] = e < cc && ii[u] < jj[u];
      kv[u] = ok[u] ? (float)K[e] : 0.f;
      tv[u] = ok[u] ? (float)T[e] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!ok[u]) continue;
      const int i = ii[u], j = jj[u];
      const float cij = kv[u] - 0.5f * (lamf[i] + lamf[j]) * tv[u];
      if (fabsf(2.f * cij) > tb * fabsf(lamf[j] - lamf[i]) &&
          fabsf(cij) > (float)kCoupleNoise * fmaxf(fabsf(lamf[i]), fabsf(lamf[j]))) {
        const int a = min(pos[i], pos[j]), b = max(pos[i], pos[j]);
        atomicAdd(&link[a], 1);
        atomicAdd(&link[b], -1);
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    int n = 0, len = 1, run = link[0];
    start[0] = 0;
    for (int k = 1; k < c; ++k) {
      // positions k-1 and k are linked when a large pair spans them
      if (run > 0 && len < kClMax) {
        ++len;
      } else {
        start[++n] = k;
        len = 1;
      }
      run += link[k];
    }
    start[++n] = c;
    s_ncl = n;
  }
  __syncthreads();
  const int ncl = s_ncl;
  for (int q = tid; q < ncl; q += blockDim.x)
    for (int k = start[q]; k < start[q + 1]; ++k) cid[order[k]] = (start[q + 1] - start[q] > 1) ? q : -1;
  for (int k = tid; k < c; k += blockDim.x) ord[k] = order[k];
  for (int q = tid; q <= ncl; q += blockDim.x) st[q] = start[q];
  if (warp >= kClWarps) return;
  float* B = Bw + (size_t)warp * kClMax * (kClMax + 1);
  float* Q = Qw + (size_t)warp * kClMax * (kClMax + 1);
  const int ld = kClMax + 1;
  for (int q = warp; q < ncl; q += kClWarps) {
    const int k0 = start[q], m = start[q + 1] - k0;
    if (m < 2) continue;
    double mean = 0.0;
    for (int a = 0; a < m; ++a) mean += lam[order[k0 + a]];
    mean /= m;
    for (int a = 0; a < m; ++a)
      if (lane < m) {
        const int ia = order[k0 + a], ib = order[k0 + lane];
        B[a * ld + lane] = (float)((a == lane) ? lam[ia] - mean : oa_coupling(K, T, c, ia, ib, lam[ia], lam[ib]));
        Q[a * ld + lane] = (a == lane) ? 1.f : 0.f;
      }
    __syncwarp();
    for (int sweep = 0; sweep < 12; ++sweep) {
      float offm = 0.f, bm = 0.f;
      for (int a = 0; a < m; ++a)
        if (lane < m) {
          if (lane != a) offm = fmaxf(offm, fabsf(B[a * ld + lane]));
          bm = fmaxf(bm, fabsf(B[a * ld + lane]));
        }
      offm = warp_max(offm);
      bm = warp_max(bm);
      if (offm <= 0x1p-24f * bm) break;
      for (int pp = 0; pp < m - 1; ++pp)
        for (int qq = pp + 1; qq < m; ++qq) {
          const float g = B[pp * ld + qq];
          if (g == 0.f) continue;
          const float zeta = (B[qq * ld + qq] - B[pp * ld + pp]) / (2.f * g);
          const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float cs = rsqrtf(1.f + t * t), sn = cs * t;
          __syncwarp();
          if (lane < m) {  // rows p, q
            const float x = B[pp * ld + lane], y = B[qq * ld + lane];
            B[pp * ld + lane] = cs * x - sn * y;
            B[qq * ld + lane] = sn * x + cs * y;
          }
          __syncwarp();
          if (lane < m) {  // columns p, q, and Q
            const float x = B[lane * ld + pp], y = B[lane * ld + qq];
            B[lane * ld + pp] = cs * x - sn * y;
            B[lane * ld + qq] = sn * x + cs * y;
            const float u = Q[lane * ld + pp], v = Q[lane * ld + qq];
            Q[lane * ld + pp] = cs * u - sn * v;
            Q[lane * ld + qq] = sn * u + cs * v;
          }
          __syncwarp();
          if (lane == 0) {
            B[pp * ld + qq] = 0.f;
            B[qq * ld + pp] = 0.f;
          }
          __syncwarp();
        }
    }
    // FP64 polish of the FP32 rotation, Q <- Q (I - E/2) with E = Q^T Q - I
    // (a Newton-Schulz step): its orthogonality defect (FP32 rounding times
    // the rotation's size) squares, so a cluster rotation taken in the last
    // refinement step leaves V orthogonal to FP64 accuracy
    double* S = Sw + (size_t)warp * kClMax * (kClMax + 1);
    if (lane < m)
      for (int a = 0; a < m; ++a) {
        double e = (a == lane) ? -1.0 : 0.0;
        for (int k = 0; k < m; ++k) e = fma((double)Q[k * ld + a], (double)Q[k * ld + lane], e);
        S[a * ld + lane] = e;
      }
    __syncwarp();
    if (lane < m)
      for (int k = 0; k < m; ++k) {
        double acc = 0.0;
        for (int a = 0; a < m; ++a) acc = fma((double)Q[k * ld + a], S[a * ld + lane], acc);
        Qb[order[k0 + k] + (size_t)order[k0 + lane] * c] = (double)Q[k * ld + lane] - 0.5 * acc;
      }
    __syncwarp();
  }
}

// F = F1 Qb with Qb block-diagonal over the clusters (identity elsewhere):
// a singleton column is copied, a cluster column mixes its members' columns
__global__ void k_block_apply(int c, const double* __restrict__ F1, const double* __restrict__ Qb,
                              const int* __restrict__ cid, const int* __restrict__ ord,
                              const int* __restrict__ st, double* __restrict__ F) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= c * c) return;
  const int i = e % c, j = e / c;
  const int q = cid[j];
  if (q < 0) {
    F[e] = F1[e];
    return;
  }
  double acc = 0.0;
  for (int k = st[q]; k < st[q + 1]; ++k) {
    const int a = ord[k];
    acc = fma(F1[i + (size_t)a * c], Qb[a + (size_t)j * c], acc);
  }
  F[e] = acc;
}

static size_t cluster_smem(int c) {
  return ((size_t)kClWarps * kClMax * (kClMax + 1) + c) * sizeof(double) +
         (2 * (size_t)kClWarps * kClMax * (kClMax + 1) + c) * sizeof(float) + (4 * (size_t)c + 2) * sizeof(int);
}

// SVD of the r x c matrix C (FP64, ld r): on exit Mout (r x c) = C V with
// orthogonal columns, Vout (c x c) orthogonal.  FP32 block one-sided Jacobi
// (relative orthogonality 1e-4, column norms floored at 1e-10 of the largest
// so rounding-level directions do not stall it; for wide pencils on the
// QR-preconditioned C Q, starting from V = Q), then four FP64 refinement
// steps (N = C V, K = N^T N, T = V^T V, clusters, V <- V (I + E)) and
// M = C V.  The steps square the defects (1e-4 from the Jacobi, 1e-8, 1e-16):
// two reach rounding level on the dense benchmark's pencils, but a pencil
// whose clusters take their rotation late needs all four (a 200-column
// pencil with clustered values: orthogonality 2.6e-11 after three, 1e-15
// after four).
static rr_status jacobi_svd(cudaStream_t s, int r, int c, const double* C, PencilWs& w, double* Mout,
                            double* Vout) {
  int ww, P;
  const int cpad = bj_cpad(c, &ww, &P, 4, r);
  const int g = 256, gc = (c * c + 255) / 256;
  // FP32 copy scaled by a power of two to max entry in [1/2, 1): squared
  // column norms stay well inside the FP32 range
  k_pow2_scale<<<1, 1024, 0, s>>>(r, c, C, r, w.fs + 1);
  const bool qr = qr_precond_applies(r, c);
  if (qr) {
    // Jacobi on s C Q with V starting at Q (C^T P = Q R)
    RR_TRY(launch_qr_precond(s, r, c, C, w.fs + 1, w.M32, cpad, w.V32, w.Hq, w.tq));
  } else {
    k_pad_copy<double, float><<<g, 256, 0, s>>>(r, c, cpad, C, r, w.M32, w.V32, w.fs + 1);
  }
  float* fl = w.fs;
  k_colnorm_floor<float><<<1, 1024, 0, s>>>(r, cpad, w.M32, r, 1e-10f, fl);
  RR_TRY(launch_bj(s, r, cpad, ww, P, w.M32, w.V32, 1e-4f, 15, w, fl));
  k_v32_to_64<<<g, 256, 0, s>>>(c, cpad, w.V32, w.V);
  const size_t csm = cluster_smem(c);
  if (csm > 48 * 1024)
    RR_CUDA(cudaFuncSetAttribute(k_cluster_rot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
  constexpr int kRefineSteps = 4;
  for (int it = 0; it < kRefineSteps; ++it) {
    gemm_small(s, 0, 0, r, c, c, 1.0, C, r, w.V, c, 0.0, w.Mp, r);          // N = C V
    gemm_small_sym(s, c, r, w.Mp, r, w.Mp, r, w.E2, c);                     // K = N^T N
    gemm_small_sym(s, c, c, w.V, c, w.V, c, w.T, c);                        // T = V^T V
    k_cluster_rot<<<1, 1024, csm, s>>>(c, w.E2, w.T, w.F, w.cid, w.order, w.cst);  // Qb
    k_oa_update<<<gc, 256, 0, s>>>(c, w.E2, w.T, w.cid, w.Vp, w.E);         // F1, W
    gemm_mixed(s, 0, 0, c, c, c, 0.5, w.E, c, w.E, c, 1.0, w.Vp, c);        // F1 += W^2 / 2
    // V <- V (I + (I - T)/2 + W) Qb: orthogonalise, the small pair rotations,
    // then the clusters' rotations
    k_block_apply<<<gc, 256, 0, s>>>(c, w.Vp, w.F, w.cid, w.order, w.cst, w.T);  // F = F1 Qb
    gemm_small(s, 0, 0, c, c, c, 1.0, w.V, c, w.T, c, 0.0, w.E, c);         // V F
    RR_CUDA(cudaMemcpyAsync(w.V, w.E, (size_t)c * c * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  gemm_small(s, 0, 0, r, c, c, 1.0, C, r, w.V, c, 0.0, Mout, r);            // M = C V
  if (Vout != w.V)
    RR_CUDA(cudaMemcpyAsync(Vout, w.V, (size_t)c * c * sizeof(double), cudaMemcpyDeviceToDevice, s));
  // setup (scale, pad copy unless the QR preconditioner ran, norm floor, V to
  // FP64; the QR and Jacobi launchers count their own), 8 refinement kernels
  // per step, the final product (in check_launch)
  note_launches((qr ? 3 : 4) + 8 * kRefineSteps);
  return check_launch("jacobi_svd");
}

}  // namespace rr

using namespace rr;

extern "C" size_t rr_pencil_workspace_size(int64_t b1, int64_t b2) {
  Arena ar(nullptr, 0);
  PencilWs w;
  carve_pencil(ar, (int)b1, (int)b2, w);
  return ar.off + 256;
}

static rr_status count_dropped(const int* d, int b, int32_t* out, cudaStream_t s) {
  if (!out) return RR_OK;
  int host[4096];
  RR_CUDA(cudaMemcpyAsync(host, d, b * sizeof(int), cudaMemcpyDeviceToHost, s));
  RR_CUDA(cudaStreamSynchronize(s));
  int n = 0;
  for (int i = 0; i < b; ++i) n += host[i];
  *out += n;
  return RR_OK;
}

extern "C" rr_status rr_pencil_eig(int64_t b, const double* H, const double* G, double* theta,
                                   double* Y, void* ws, size_t ws_bytes, int32_t* dropped,
                                   void* stream) {
  if (b <= 0 || b > kMaxPencil || !H || !G || !theta || !Y) return RR_ERR_ARG;
  Arena ar(ws, ws_bytes);
  PencilWs w;
  if (!ws || !carve_pencil(ar, (int)b, (int)b, w)) return RR_ERR_WORKSPACE;
  cudaStream_t s = as_stream(stream);
  const int n = (int)b;
  RR_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), s));
  whiten(s, n, G, WhitenScratch{w.W1, w.W2, w.T, w.E, w.E2, w.F}, w.drop1, w.W1);
  RR_CUDA(cudaMemsetAsync(w.cond, 0, 4 * sizeof(double), s));
  k_cond_est<<<1, 256, 0, s>>>(n, G, w.W1, w.drop1, w.cond);
  // C = W^T H W, symmetrised and shifted positive definite (C - mu I)
  gemm_small(s, 0, 0, n, n, n, 1.0, H, n, w.W1, n, 0.0, w.T, n);
  gemm_small_sym(s, n, n, w.W1, n, w.T, n, w.C, n);  // W^T H W (symmetric)
  RR_TRY(eig_shift(s, n, w.C, w.drop1, w.sh, w.shok, w.mu));
  RR_TRY(jacobi_svd(s, n, n, w.C, w, w.M, w.V));
  k_colnorm_sort<<<1, kSmallThreads, n * sizeof(double), s>>>(n, n, w.M, n, w.sig, w.order);
  k_eig_finish<<<1, 256, 0, s>>>(n, w.sig, w.order, w.mu, w.V, theta, w.T, w.nvalid);
  // Y = W Z
  gemm_small(s, 0, 0, n, n, n, 1.0, w.W1, n, w.T, n, 0.0, Y, n);
  note_launches(5);
  RR_TRY(check_launch("rr_pencil_eig"));
  if (dropped) {
    *dropped = 0;
    RR_TRY(count_dropped(w.drop1, n, dropped, s));
  }
  return RR_OK;
}

extern "C" rr_status rr_pencil_svd(int64_t b1, int64_t b2, const double* B, const double* Gu,
                                   const double* Gv, double* sv, double* Y, double* Z, void* ws,
                                   size_t ws_bytes, int32_t* dropped, void* stream) {
  if (b1 <= 0 || b2 <= 0 || b1 > kMaxPencil || b2 > kMaxPencil || !B || !Gu || !Gv || !sv || !Y || !Z)
    return RR_ERR_ARG;
  Arena ar(ws, ws_bytes);
  PencilWs w;
  if (!ws || !carve_pencil(ar, (int)b1, (int)b2, w)) return RR_ERR_WORKSPACE;
  cudaStream_t s = as_stream(stream);
  const int n1 = (int)b1, n2 = (int)b2, r = n1 < n2 ? n1 : n2;
  RR_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), s));
  // whitening of both sides, at the same time on two streams (each is a
  // chain of latency-bound small kernels): Wu -> C on s, Wv -> V on the side
  // stream, each with its own scratch
  SideStream ss;
  RR_TRY(side_stream(s, &ss));
  RR_CUDA(cudaEventRecord(ss.fork, s));
  RR_CUDA(cudaStreamWaitEvent(ss.s2, ss.fork, 0));
  whiten(s, n1, Gu, WhitenScratch{w.W1, w.W2, w.T, w.E, w.E2, w.F}, w.drop1, w.C);
  whiten(ss.s2, n2, Gv, w.wb, w.drop2, w.V);
  k_cond_est<<<1, 256, 0, ss.s2>>>(n2, Gv, w.V, w.drop2, w.cond + 1);  // cond[1], drops[3]
  RR_CUDA(cudaEventRecord(ss.join, ss.s2));
  RR_CUDA(cudaStreamWaitEvent(s, ss.join, 0));
  RR_CUDA(cudaMemcpyAsync(w.W1, w.C, (size_t)n1 * n1 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  RR_CUDA(cudaMemcpyAsync(w.W2, w.V, (size_t)n2 * n2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  k_cond_est<<<1, 256, 0, s>>>(n1, Gu, w.W1, w.drop1, w.cond);      // cond[0], drops[2]
  // Cw = Wu^T B Wv (b1 x b2) -> C
  gemm_small(s, 0, 0, n1, n2, n2, 1.0, B, n1, w.W2, n2, 0.0, w.T, n1);
  gemm_small(s, 1, 0, n1, n2, n1, 1.0, w.W1, n1, w.T, n1, 0.0, w.C, n1);
  k_zero_dropped<<<(n1 * n2 + 255) / 256, 256, 0, s>>>(n1, n2, w.C, w.drop1, w.drop2);
  RR_TRY(jacobi_svd(s, n1, n2, w.C, w, w.M, w.V));   // M = Cw V (b1 x b2), V (b2 x b2)
  k_colnorm_sort<<<1, kSmallThreads, n2 * sizeof(double), s>>>(n1, n2, w.M, n1, w.sig, w.order);
  double* Uw = w.T;   // b1 x r
  double* Vw = w.E;   // b2 x r
  k_svd_finish<<<64, 256, 0, s>>>(n1, n2, w.sig, w.order, w.M, w.V, sv, Uw, Vw, r);
  // Y = Wu Uw, Z = Wv Vw
  gemm_small(s, 0, 0, n1, r, n1, 1.0, w.W1, n1, Uw, n1, 0.0, Y, n1);
  gemm_small(s, 0, 0, n2, r, n2, 1.0, w.W2, n2, Vw, n2, 0.0, Z, n2);
  note_launches(9);
  RR_TRY(check_launch("rr_pencil_svd"));
  if (dropped) {
    *dropped = 0;
    RR_TRY(count_dropped(w.drop1, n1, dropped, s));
    RR_TRY(count_dropped(w.drop2, n2, dropped, s));
  }
  return RR_OK;
}

// exported for the solver (same translation unit helpers)
namespace rr {
// Device address of the condition estimates and drop counts the last
// rr_pencil_eig / rr_pencil_svd on this workspace wrote: [0], [1] the
// estimates (eig: [1] = 0; SVD: U and V side), [2], [3] the dropped columns.
const double* pencil_cond_slot(void* ws, size_t ws_bytes, int b1, int b2) {
  Arena ar(ws, ws_bytes);
  PencilWs w;
  if (!ws || !carve_pencil(ar, b1, b2, w)) return nullptr;
  return w.cond;
}

void small_gemm(cudaStream_t s, int ta, int tb, int M, int N, int K, double alpha, const double* A,
                int lda, const double* B, int ldb, double beta, double* C, int ldc) {
  gemm_small(s, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}
}  // namespace rr
