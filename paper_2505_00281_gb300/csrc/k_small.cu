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

#include "rr_common.cuh"

namespace rr {

constexpr int kSmallThreads = 1024;

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

// Small FP64 GEMM: C = alpha op(A) op(B) + beta C (32 x 32 tiles).
__global__ void __launch_bounds__(256) k_gemm_f64_small(int ta, int tb, int M, int N, int K,
                                                        double alpha, const double* __restrict__ A,
                                                        int lda, const double* __restrict__ B,
                                                        int ldb, double beta, double* __restrict__ C,
                                                        int ldc) {
  __shared__ double As[16][33];
  __shared__ double Bs[16][33];
  const int m0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
  const int tid = threadIdx.x, ti = tid % 16, tj = tid / 16;
  double acc[2][2] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = tid; e < 16 * 32; e += 256) {
      int kk = e % 16, i = e / 16;
      int gk = k0 + kk, gi = m0 + i, gj = n0 + i;
      As[kk][i] = (gk < K && gi < M) ? (ta ? A[gk + gi * lda] : A[gi + gk * lda]) : 0.0;
      Bs[kk][i] = (gk < K && gj < N) ? (tb ? B[gj + gk * ldb] : B[gk + gj * ldb]) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a0 = As[kk][ti], a1 = As[kk][ti + 16], b0 = Bs[kk][tj], b1 = Bs[kk][tj + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      int i = m0 + ti + 16 * a, j = n0 + tj + 16 * c;
      if (i < M && j < N) {
        double v = alpha * acc[a][c];
        if (beta != 0.0) v += beta * C[i + j * ldc];
        C[i + j * ldc] = v;
      }
    }
}

static void gemm_small(cudaStream_t s, int ta, int tb, int M, int N, int K, double alpha,
                       const double* A, int lda, const double* B, int ldb, double beta, double* C,
                       int ldc) {
  dim3 g((M + 31) / 32, (N + 31) / 32);
  k_gemm_f64_small<<<g, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

// Symmetrise C, shift it to positive definite by a Gershgorin bound
// (C - mu I, mu < lambda_min), and decouple dropped indices (zero row and
// column; their singular value is then exactly 0).
__global__ void __launch_bounds__(kSmallThreads) k_eig_prep(int b, double* __restrict__ C,
                                                            const int* __restrict__ dropped,
                                                            double* __restrict__ mu_out) {
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
  __shared__ double red_lo[32], red_hi[32];
  double lo = DBL_MAX, hi = -DBL_MAX;
  for (int i = tid; i < b; i += kSmallThreads) {
    if (dropped[i]) continue;
    double r = 0.0;
    for (int j = 0; j < b; ++j)
      if (j != i) r += fabs(C[i + j * b]);
    lo = fmin(lo, C[i + i * b] - r);
    hi = fmax(hi, C[i + i * b] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((tid & 31) == 0) {
    red_lo[tid >> 5] = lo;
    red_hi[tid >> 5] = hi;
  }
  __syncthreads();
  __shared__ double s_mu;
  if (tid == 0) {
    double l = DBL_MAX, h = -DBL_MAX;
    for (int w = 0; w < kSmallThreads / 32; ++w) {
      l = fmin(l, red_lo[w]);
      h = fmax(h, red_hi[w]);
    }
    if (l > h) {  // everything dropped
      l = 0.0;
      h = 1.0;
    }
    double span = fmax(h - l, fmax(fabs(l), fabs(h)));
    if (span == 0.0) span = 1.0;
    s_mu = l - 1e-3 * span;
    *mu_out = s_mu;
  }
  __syncthreads();
  for (int i = tid; i < b; i += kSmallThreads) C[i + i * b] = dropped[i] ? 0.0 : C[i + i * b] - s_mu;
}

// Zero the rows (drop_r) and columns (drop_c) of a rectangular b1 x b2 matrix.
__global__ void k_zero_dropped(int b1, int b2, double* __restrict__ C, const int* __restrict__ dr,
                               const int* __restrict__ dc) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= b1 * b2) return;
  int i = e % b1, j = e / b1;
  if (dr[i] || dc[j]) C[i + j * b1] = 0.0;
}

// One-sided Jacobi (Hestenes) on the columns of M (r x c): M <- M V with V
// orthogonal, until every column pair is orthogonal to relative tol.
// Parallel round-robin ordering: c'/2 disjoint pairs per round, one warp per
// pair, rounds separated by __syncthreads.  A pair whose inner product is
// exactly zero is never rotated, so exactly-zero (dropped) columns stay
// decoupled.
template <typename T>
__global__ void __launch_bounds__(kSmallThreads) k_jacobi1s(int r, int c, T* __restrict__ M, int ldm,
                                                            T* __restrict__ V, int ldv, int max_sweeps,
                                                            T tol, int* __restrict__ sweeps_out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kSmallThreads / 32;
  for (int e = tid; e < c * c; e += kSmallThreads) {
    int i = e % c, j = e / c;
    V[i + j * ldv] = (i == j) ? T(1) : T(0);
  }
  const int cp = c + (c & 1);  // padded to even; index c (if odd) is a dummy
  __shared__ int s_rot;
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < cp - 1; ++round) {
      for (int pi = warp; pi < cp / 2; pi += nw) {
        // round-robin (circle method): position 0 fixed, others rotate
        int a = (pi == 0) ? 0 : 1 + (pi - 1 + round) % (cp - 1);
        int bq = 1 + (cp - 2 - pi + round) % (cp - 1);
        int p = a < bq ? a : bq, q = a < bq ? bq : a;
        if (q >= c) continue;
        T* mp = M + (size_t)p * ldm;
        T* mq = M + (size_t)q * ldm;
        T al = T(0), be = T(0), ga = T(0);
        for (int i = lane; i < r; i += 32) {
          T x = mp[i], y = mq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga == T(0) || fabs(ga) <= tol * sqrt(al * be)) continue;
        T zeta = (be - al) / (T(2) * ga);
        T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        T cs = T(1) / sqrt(T(1) + t * t), sn = cs * t;
        for (int i = lane; i < r; i += 32) {
          T x = mp[i], y = mq[i];
          mp[i] = cs * x - sn * y;
          mq[i] = sn * x + cs * y;
        }
        T* vp = V + (size_t)p * ldv;
        T* vq = V + (size_t)q * ldv;
        for (int i = lane; i < c; i += 32) {
          T x = vp[i], y = vq[i];
          vp[i] = cs * x - sn * y;
          vq[i] = sn * x + cs * y;
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    if (!s_rot) break;
    __syncthreads();
  }
  if (tid == 0 && sweeps_out) *sweeps_out = sweep;
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
  for (int j = tid; j < c; j += kSmallThreads) {
    double v = nrm[j];
    int rank = 0;
    for (int l = 0; l < c; ++l) {
      double w = nrm[l];
      if (w > v || (w == v && l < j)) ++rank;
    }
    order[rank] = j;
    sig[rank] = v;
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

struct PencilWs {
  double *L1, *Li1, *L2, *Li2, *T, *C, *V, *sig, *mu;
  int *drop1, *drop2, *order, *nvalid;
};

static bool carve_pencil(Arena& ar, int b1, int b2, PencilWs& w) {
  int bm = b1 > b2 ? b1 : b2;
  w.L1 = ar.take<double>((size_t)b1 * b1);
  w.Li1 = ar.take<double>((size_t)b1 * b1);
  w.L2 = ar.take<double>((size_t)b2 * b2);
  w.Li2 = ar.take<double>((size_t)b2 * b2);
  w.T = ar.take<double>((size_t)bm * bm);
  w.C = ar.take<double>((size_t)bm * bm);
  w.V = ar.take<double>((size_t)bm * bm);
  w.sig = ar.take<double>(bm);
  w.mu = ar.take<double>(1);
  w.drop1 = ar.take<int>(b1);
  w.drop2 = ar.take<int>(b2);
  w.order = ar.take<int>(bm);
  w.nvalid = ar.take<int>(1);
  return !ar.overflow;
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
  if (b <= 0 || b > 4096 || !H || !G || !theta || !Y) return RR_ERR_ARG;
  Arena ar(ws, ws_bytes);
  PencilWs w;
  if (!ws || !carve_pencil(ar, (int)b, (int)b, w)) return RR_ERR_WORKSPACE;
  cudaStream_t s = as_stream(stream);
  const int n = (int)b;
  k_chol_drop<<<1, kSmallThreads, 0, s>>>(n, G, n, w.L1, w.drop1);
  k_tri_inv_lower<<<1, kSmallThreads, 0, s>>>(n, w.L1, w.Li1);
  // C = Li H Li^T
  gemm_small(s, 0, 0, n, n, n, 1.0, w.Li1, n, H, n, 0.0, w.T, n);
  gemm_small(s, 0, 1, n, n, n, 1.0, w.T, n, w.Li1, n, 0.0, w.C, n);
  k_eig_prep<<<1, kSmallThreads, 0, s>>>(n, w.C, w.drop1, w.mu);
  k_jacobi1s<double><<<1, kSmallThreads, 0, s>>>(n, n, w.C, n, w.V, n, 40, 4.0 * DBL_EPSILON, nullptr);
  k_colnorm_sort<<<1, kSmallThreads, n * sizeof(double), s>>>(n, n, w.C, n, w.sig, w.order);
  k_eig_finish<<<1, 256, 0, s>>>(n, w.sig, w.order, w.mu, w.V, theta, w.T, w.nvalid);
  // Y = Li^T Z
  gemm_small(s, 1, 0, n, n, n, 1.0, w.Li1, n, w.T, n, 0.0, Y, n);
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
  if (b1 <= 0 || b2 <= 0 || b1 > 4096 || b2 > 4096 || !B || !Gu || !Gv || !sv || !Y || !Z)
    return RR_ERR_ARG;
  Arena ar(ws, ws_bytes);
  PencilWs w;
  if (!ws || !carve_pencil(ar, (int)b1, (int)b2, w)) return RR_ERR_WORKSPACE;
  cudaStream_t s = as_stream(stream);
  const int n1 = (int)b1, n2 = (int)b2, r = n1 < n2 ? n1 : n2;
  k_chol_drop<<<1, kSmallThreads, 0, s>>>(n1, Gu, n1, w.L1, w.drop1);
  k_tri_inv_lower<<<1, kSmallThreads, 0, s>>>(n1, w.L1, w.Li1);
  k_chol_drop<<<1, kSmallThreads, 0, s>>>(n2, Gv, n2, w.L2, w.drop2);
  k_tri_inv_lower<<<1, kSmallThreads, 0, s>>>(n2, w.L2, w.Li2);
  // C = Lu^-1 B Lv^-T  (b1 x b2)
  gemm_small(s, 0, 0, n1, n2, n1, 1.0, w.Li1, n1, B, n1, 0.0, w.T, n1);
  gemm_small(s, 0, 1, n1, n2, n2, 1.0, w.T, n1, w.Li2, n2, 0.0, w.C, n1);
  k_zero_dropped<<<(n1 * n2 + 255) / 256, 256, 0, s>>>(n1, n2, w.C, w.drop1, w.drop2);
  k_jacobi1s<double><<<1, kSmallThreads, 0, s>>>(n1, n2, w.C, n1, w.V, n2, 40, 4.0 * DBL_EPSILON, nullptr);
  k_colnorm_sort<<<1, kSmallThreads, n2 * sizeof(double), s>>>(n1, n2, w.C, n1, w.sig, w.order);
  // whitened singular vectors (Uw in T, Vw in L1-sized scratch reuse: use Li? no: dedicated)
  double* Uw = w.T;   // b1 x r
  double* Vw = w.L2;  // b2 x r (L2 no longer needed)
  k_svd_finish<<<64, 256, 0, s>>>(n1, n2, w.sig, w.order, w.C, w.V, sv, Uw, Vw, r);
  // Y = Lu^-T Uw, Z = Lv^-T Vw
  gemm_small(s, 1, 0, n1, r, n1, 1.0, w.Li1, n1, Uw, n1, 0.0, Y, n1);
  gemm_small(s, 1, 0, n2, r, n2, 1.0, w.Li2, n2, Vw, n2, 0.0, Z, n2);
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
void small_gemm(cudaStream_t s, int ta, int tb, int M, int N, int K, double alpha, const double* A,
                int lda, const double* B, int ldb, double beta, double* C, int ldc) {
  gemm_small(s, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}
}  // namespace rr
