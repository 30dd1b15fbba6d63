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

// Small FP64 GEMM: C = alpha op(A) op(B) + beta C.  16 x 16 output tiles,
// one output per thread, so a 256 x 256 product spreads over 256 CTAs (FP64
// issue rate per SM is the limit on GB300, so the work must cover the GPU).
__global__ void __launch_bounds__(256) k_gemm_f64_small(int ta, int tb, int M, int N, int K,
                                                        double alpha, const double* __restrict__ A,
                                                        int lda, const double* __restrict__ B,
                                                        int ldb, double beta, double* __restrict__ C,
                                                        int ldc) {
  __shared__ double As[32][17];
  __shared__ double Bs[32][17];
  const int m0 = blockIdx.x * 16, n0 = blockIdx.y * 16;
  const int tid = threadIdx.x, ti = tid % 16, tj = tid / 16;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int e = tid; e < 32 * 16; e += 256) {
      int kk = e % 32, i = e / 32;
      int gk = k0 + kk, gi = m0 + i, gj = n0 + i;
      As[kk][i] = (gk < K && gi < M) ? (ta ? A[gk + gi * lda] : A[gi + gk * lda]) : 0.0;
      Bs[kk][i] = (gk < K && gj < N) ? (tb ? B[gj + gk * ldb] : B[gk + gj * ldb]) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) acc = fma(As[kk][ti], Bs[kk][tj], acc);
    __syncthreads();
  }
  int i = m0 + ti, j = n0 + tj;
  if (i < M && j < N) {
    double v = alpha * acc;
    if (beta != 0.0) v += beta * C[i + j * ldc];
    C[i + j * ldc] = v;
  }
}

static void gemm_small(cudaStream_t s, int ta, int tb, int M, int N, int K, double alpha,
                       const double* A, int lda, const double* B, int ldb, double beta, double* C,
                       int ldc) {
  dim3 g((M + 15) / 16, (N + 15) / 16);
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
  const int tid = threadIdx.x;
  __shared__ int s_keep;
  for (int j = 0; j < b; ++j)
    for (int i = j + tid; i < b; i += kSmallThreads)
      Ls[pk(i, j, b)] = (float)(0.5 * (G[i + j * ldg] + G[j + i * ldg]));
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      float d = Ls[pk(j, j, b)];
      float g0 = (float)G[j + j * ldg];
      s_keep = (g0 > 0.f && d > 64.f * 0x1p-24f * g0) ? 1 : 0;
      dropped[j] = s_keep ? 0 : 1;
      Ls[pk(j, j, b)] = s_keep ? sqrtf(d) : 1.f;
    }
    __syncthreads();
    const float ljj = Ls[pk(j, j, b)];
    if (s_keep) {
      for (int i = j + 1 + tid; i < b; i += kSmallThreads) Ls[pk(i, j, b)] /= ljj;
    } else {
      for (int i = j + 1 + tid; i < b; i += kSmallThreads) Ls[pk(i, j, b)] = 0.f;
      for (int l = tid; l < j; l += kSmallThreads) Ls[pk(j, l, b)] = 0.f;
    }
    __syncthreads();
    if (s_keep) {
      // trailing update, one warp per column l, lanes over rows i >= l
      const int lane = tid & 31, warp = tid >> 5;
      const int bj = pk(j, j, b) - j;  // column j starts at bj + j
      for (int l = j + 1 + warp; l < b; l += kSmallThreads / 32) {
        const float llj = Ls[bj + l];
        const int bl = pk(l, l, b) - l;
        for (int i = l + lane; i < b; i += 32) Ls[bl + i] = fmaf(-Ls[bj + i], llj, Ls[bl + i]);
      }
    }
    __syncthreads();
  }
  // in-place inverse, last column first: column j of L^-1 from the already
  // inverted trailing block, x = -(Linv[j+1:, j+1:] L[j+1:, j]) / L_jj; one
  // warp per row, lanes split the dot product.  New values are staged in
  // xbuf (the old column j is read by every row).
  {
    float* xbuf = Ls + (size_t)b * (b + 1) / 2;  // [b]
    const int lane = tid & 31, warp = tid >> 5, nw = kSmallThreads / 32;
    for (int j = b - 1; j >= 0; --j) {
      const float ajj = 1.f / Ls[pk(j, j, b)];
      for (int i = j + 1 + warp; i < b; i += nw) {
        float sum = 0.f;
        for (int l = j + 1 + lane; l <= i; l += 32) sum = fmaf(Ls[pk(i, l, b)], Ls[pk(l, j, b)], sum);
        sum = warp_sum(sum);
        if (lane == 0) xbuf[i] = -sum * ajj;
      }
      __syncthreads();
      for (int i = j + 1 + tid; i < b; i += kSmallThreads) Ls[pk(i, j, b)] = xbuf[i];
      if (tid == 0) Ls[pk(j, j, b)] = ajj;
      __syncthreads();
    }
  }
  // W0 = (L^-1)^T, dropped columns zero
  for (int e = tid; e < b * b; e += kSmallThreads) {
    int i = e % b, j = e / b;
    W[i + j * b] = (dropped[j] || j < i) ? 0.0 : (double)Ls[pk(j, i, b)];
  }
}

// E <- E - diag(kept)  (E = W^T G W, so E becomes W^T G W - I on the kept part)
// then F = I - E/2 (+ 3/8 E2 if given)
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
  double f = (i == j ? 1.0 : 0.0) - 0.5 * v;
  if (E2) f += 0.375 * E2[e];
  F[e] = f;
}

// One-sided block Jacobi (Hestenes) on the columns of M (r x cpad):
// M <- M V, V orthogonal (cpad x cpad, initialised to I by the launcher).
// The cpad columns form 2P blocks of w; CTA g takes one block pair per round
// (circle method over the blocks, 2P-1 rounds per sweep), loads its 2w
// columns of M and V into shared memory, orthogonalises every column pair
// among them (circle method over the 2w columns, one warp per pair), and
// writes them back; a bounded grid barrier separates rounds.  A pair whose
// inner product is exactly zero is never rotated, so zero columns (dropped
// directions, padding) stay decoupled.  Converged when a sweep rotates
// nothing (rotation counts per sweep in rot[]).
constexpr int kBJThreads = 512;
template <typename T>
__global__ void __launch_bounds__(kBJThreads) k_block_jacobi(int r, int cpad, int w, T* __restrict__ M,
                                                             int ldm, T* __restrict__ V, int ldv, T tol,
                                                             int max_sweeps, int* __restrict__ rot,
                                                             GridBarrier* bar, int* err,
                                                             int* __restrict__ sweeps_out,
                                                             const T* __restrict__ floor_ptr) {
  extern __shared__ unsigned char smem_raw[];
  T* Ms = reinterpret_cast<T*>(smem_raw);   // [2w][r]
  T* Vs = Ms + (size_t)2 * w * r;           // [2w][cpad]
  const int P = gridDim.x, g = blockIdx.x, nblk = 2 * P;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kBJThreads / 32;
  const int w2 = 2 * w;
  // columns whose squared norm is below the floor (rounding-level directions)
  // count as converged against everything
  const T nfloor = floor_ptr ? *floor_ptr : T(0);
  __shared__ int s_rot;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    for (int round = 0; round < nblk - 1; ++round) {
      const int ba = (g == 0) ? 0 : 1 + (g - 1 + round) % (nblk - 1);
      const int bb = 1 + (nblk - 2 - g + round) % (nblk - 1);
      // load the 2w columns
      for (int e = tid; e < w2 * r; e += kBJThreads) {
        int l = e / r, i = e % r;
        int gc = (l < w ? ba * w + l : bb * w + (l - w));
        Ms[(size_t)l * r + i] = M[i + (size_t)gc * ldm];
      }
      for (int e = tid; e < w2 * cpad; e += kBJThreads) {
        int l = e / cpad, i = e % cpad;
        int gc = (l < w ? ba * w + l : bb * w + (l - w));
        Vs[(size_t)l * cpad + i] = V[i + (size_t)gc * ldv];
      }
      __syncthreads();
      // Round 0 of a sweep: all pairs among the 2w local columns (circle
      // method, w pairs per sub-round), which also covers every block's
      // internal pairs once per sweep.  Later rounds: only the w x w pairs
      // across the two blocks (sub-round t pairs column i of block a with
      // column (i + t) mod w of block b).  Per sweep that is c - 1 sub-rounds.
      const int nsub = (round == 0) ? w2 - 1 : w;
      for (int sr = 0; sr < nsub; ++sr) {
        for (int pi = warp; pi < w; pi += nw) {
          int p, q;
          if (round == 0) {
            int a = (pi == 0) ? 0 : 1 + (pi - 1 + sr) % (w2 - 1);
            int bq = 1 + (w2 - 2 - pi + sr) % (w2 - 1);
            p = a < bq ? a : bq;
            q = a < bq ? bq : a;
          } else {
            p = pi;
            q = w + (pi + sr) % w;
          }
          T* mp = Ms + (size_t)p * r;
          T* mq = Ms + (size_t)q * r;
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
          if (ga == T(0) || fabs(ga) <= tol * sqrt(fmax(al, nfloor) * fmax(be, nfloor))) continue;
          T zeta = (be - al) / (T(2) * ga);
          T t = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          T cs = T(1) / sqrt(T(1) + t * t), sn = cs * t;
          for (int i = lane; i < r; i += 32) {
            T x = mp[i], y = mq[i];
            mp[i] = cs * x - sn * y;
            mq[i] = sn * x + cs * y;
          }
          T* vp = Vs + (size_t)p * cpad;
          T* vq = Vs + (size_t)q * cpad;
          for (int i = lane; i < cpad; i += 32) {
            T x = vp[i], y = vq[i];
            vp[i] = cs * x - sn * y;
            vq[i] = sn * x + cs * y;
          }
          if (lane == 0) s_rot = 1;
        }
        __syncthreads();
      }
      // store back
      for (int e = tid; e < w2 * r; e += kBJThreads) {
        int l = e / r, i = e % r;
        int gc = (l < w ? ba * w + l : bb * w + (l - w));
        M[i + (size_t)gc * ldm] = Ms[(size_t)l * r + i];
      }
      for (int e = tid; e < w2 * cpad; e += kBJThreads) {
        int l = e / cpad, i = e % cpad;
        int gc = (l < w ? ba * w + l : bb * w + (l - w));
        V[i + (size_t)gc * ldv] = Vs[(size_t)l * cpad + i];
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

// identity (cpad x cpad) and copy/convert of an r x c matrix into an r x cpad
// padded one (zero padding columns)
template <typename TI, typename TO>
__global__ void k_pad_copy(int r, int c, int cpad, const TI* __restrict__ A, int lda,
                           TO* __restrict__ M, TO* __restrict__ V) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * cpad; e += gridDim.x * blockDim.x) {
    int i = e % r, j = e / r;
    M[e] = j < c ? (TO)A[i + j * lda] : TO(0);
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

// F = 1.5 I - 0.5 T
__global__ void k_ns_coef(int c, const double* __restrict__ T, double* __restrict__ F) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= c * c) return;
  int i = e % c, j = e / c;
  F[e] = (i == j ? 1.5 : 0.0) - 0.5 * T[e];
}

struct PencilWs {
  double *W1, *W2, *T, *E, *E2, *F, *C, *V, *Vp, *M, *Mp, *sig, *mu;
  float *L32, *Li32, *M32, *V32;
  int *drop1, *drop2, *order, *nvalid, *rot, *err, *sweeps;
  GridBarrier* bar;
};

static int bj_cpad(int c, int* w_out, int* P_out, size_t elt, int r) {
  int w, P;
  if (c <= 64) {
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
  w.Vp = ar.take<double>(cc);
  w.M = ar.take<double>(rc);
  w.Mp = ar.take<double>(rc);
  w.sig = ar.take<double>(cp);
  w.mu = ar.take<double>(2);
  w.L32 = ar.take<float>(bb);
  w.Li32 = ar.take<float>(bb);
  w.M32 = ar.take<float>(rc);
  w.V32 = ar.take<float>(cc);
  w.drop1 = ar.take<int>(bm);
  w.drop2 = ar.take<int>(bm);
  w.order = ar.take<int>(cp);
  w.nvalid = ar.take<int>(1);
  w.rot = ar.take<int>(64);
  w.err = ar.take<int>(1);
  w.sweeps = ar.take<int>(2);
  w.bar = ar.take<GridBarrier>(1);
  return !ar.overflow;
}

// Whitening matrix W (b x b) with W^T G W = I on the kept part: FP32
// Cholesky for W0 = L^-T, then two steps of FP64 iterative refinement,
// W <- W (I - E/2 + 3/8 E^2), E = W^T G W - I, whose error squares per step.
static void whiten(cudaStream_t s, int b, const double* G, PencilWs& w, int* dropped, double* Wout) {
  const int g1 = (b * b + 255) / 256;
  const size_t sm = ((size_t)b * (b + 1) / 2 + b) * sizeof(float);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_chol_inv_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_chol_inv_f32<<<1, kSmallThreads, sm, s>>>(b, G, b, dropped, w.W1);
  // three refinement steps W <- W (I - E/2 + 3/8 E^2), E = W^T G W - I;
  // each cubes the error (|E| ~ u32 cond(G) after the FP32 factorisation)
  double* Wc = w.W1;
  double* Wn = w.W2;
  for (int it = 0; it < 3; ++it) {
    gemm_small(s, 0, 0, b, b, b, 1.0, G, b, Wc, b, 0.0, w.T, b);
    gemm_small(s, 1, 0, b, b, b, 1.0, Wc, b, w.T, b, 0.0, w.E, b);
    k_whiten_corr<<<g1, 256, 0, s>>>(b, w.E, nullptr, dropped, nullptr, 0);
    gemm_small(s, 0, 0, b, b, b, 1.0, w.E, b, w.E, b, 0.0, w.E2, b);
    k_whiten_corr<<<g1, 256, 0, s>>>(b, w.E, w.E2, dropped, w.F, 1);
    gemm_small(s, 0, 0, b, b, b, 1.0, Wc, b, w.F, b, 0.0, it == 2 ? Wout : Wn, b);
    double* t = Wc;
    Wc = Wn;
    Wn = t;
  }
  note_launches(17);
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

template <typename T>
static rr_status launch_bj(cudaStream_t s, int r, int cpad, int w, int P, T* M, T* V, T tol,
                           int max_sweeps, PencilWs& ws, const T* floor_ptr = nullptr) {
  size_t smem = (size_t)2 * w * (r + cpad) * sizeof(T);
  const void* fn = (const void*)k_block_jacobi<T>;
  if (smem > 48 * 1024)
    RR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  RR_CUDA(cudaMemsetAsync(ws.rot, 0, 64 * sizeof(int), s));
  RR_CUDA(cudaMemsetAsync(ws.bar, 0, sizeof(GridBarrier), s));
  int ld = r, ldv = cpad;
  if (P == 1) {
    k_block_jacobi<T><<<1, kBJThreads, smem, s>>>(r, cpad, w, M, ld, V, ldv, tol, max_sweeps, ws.rot,
                                                  ws.bar, ws.err, ws.sweeps, floor_ptr);
    return check_launch("block_jacobi");
  }
  int* rot = ws.rot;
  GridBarrier* bar = ws.bar;
  int* err = ws.err;
  int* sw = ws.sweeps;
  const T* fl = floor_ptr;
  void* args[] = {&r, &cpad, &w, &M, &ld, &V, &ldv, &tol, &max_sweeps, &rot, &bar, &err, &sw, &fl};
  RR_CUDA(cudaLaunchCooperativeKernel(fn, dim3(P), dim3(kBJThreads), args, smem, s));
  note_launches(1);
  return RR_OK;
}

// Omega (c x c) from K = N^T N: for i < j the exact one-sided Jacobi angle
// that makes columns i and j of N orthogonal, Omega_ij = phi, Omega_ji = -phi
// (V <- V (I + Omega) to first order).  Zero columns are never rotated.
__global__ void k_polish_angles(int c, const double* __restrict__ K, double* __restrict__ Om) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= c * c) return;
  int i = e % c, j = e / c;
  if (i == j) {
    Om[e] = 0.0;
    return;
  }
  int p = i < j ? i : j, q = i < j ? j : i;
  double al = K[p + p * c], be = K[q + q * c], ga = K[p + q * c];
  double phi = 0.0;
  if (ga != 0.0 && al > 0.0 && be > 0.0) {
    double zeta = (be - al) / (2.0 * ga);
    double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    phi = atan(t);
  }
  Om[e] = (i < j) ? phi : -phi;
}

// F = I + Om + Om2/2
__global__ void k_expm2(int c, const double* __restrict__ Om, const double* __restrict__ Om2,
                        double* __restrict__ F) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= c * c) return;
  int i = e % c, j = e / c;
  F[e] = (i == j ? 1.0 : 0.0) + Om[e] + 0.5 * Om2[e];
}

// V <- V (3I - V^T V)/2, twice (Newton-Schulz polar step; orthogonality error
// d -> ~3d^2/4 per step).  Uses T, F, E as scratch.
static void ns_orthonormalize(cudaStream_t s, int c, double* V, PencilWs& w) {
  for (int it = 0; it < 2; ++it) {
    gemm_small(s, 1, 0, c, c, c, 1.0, V, c, V, c, 0.0, w.T, c);
    k_ns_coef<<<(c * c + 255) / 256, 256, 0, s>>>(c, w.T, w.F);
    gemm_small(s, 0, 0, c, c, c, 1.0, V, c, w.F, c, 0.0, w.E, c);
    cudaMemcpyAsync(V, w.E, (size_t)c * c * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  note_launches(6);
}

// SVD of the r x c matrix C (FP64, ld r): on exit Mout (r x c) = C V with
// orthogonal columns, Vout (c x c) orthogonal.  FP32 block one-sided Jacobi
// (relative orthogonality 1e-4, column norms floored at 1e-10 of the largest
// so rounding-level directions do not stall it), then an FP64 polish made
// only of small parallel GEMMs: V <- NS(V); N = C V; K = N^T N; rotate every
// pair by its exact Jacobi angle at once (V <- V (I + Om + Om^2/2)); three
// times.  Each polish step roughly squares the relative off-diagonal of K.
static rr_status jacobi_svd(cudaStream_t s, int r, int c, const double* C, PencilWs& w, double* Mout,
                            double* Vout) {
  int ww, P;
  const int cpad = bj_cpad(c, &ww, &P, 4, r);
  const int g = 256, gc = (c * c + 255) / 256;
  k_pad_copy<double, float><<<g, 256, 0, s>>>(r, c, cpad, C, r, w.M32, w.V32);
  float* fl = (float*)(w.mu + 1);  // scratch slot after mu
  k_colnorm_floor<float><<<1, 1024, 0, s>>>(r, cpad, w.M32, r, 1e-10f, fl);
  RR_TRY(launch_bj<float>(s, r, cpad, ww, P, w.M32, w.V32, 1e-4f, 15, w, fl));
  k_v32_to_64<<<g, 256, 0, s>>>(c, cpad, w.V32, w.V);
  for (int it = 0; it < 3; ++it) {
    ns_orthonormalize(s, c, w.V, w);
    gemm_small(s, 0, 0, r, c, c, 1.0, C, r, w.V, c, 0.0, w.Mp, r);          // N = C V
    gemm_small(s, 1, 0, c, c, r, 1.0, w.Mp, r, w.Mp, r, 0.0, w.Vp, c);      // K = N^T N
    k_polish_angles<<<gc, 256, 0, s>>>(c, w.Vp, w.E2);
    gemm_small(s, 0, 0, c, c, c, 1.0, w.E2, c, w.E2, c, 0.0, w.T, c);       // Om^2
    k_expm2<<<gc, 256, 0, s>>>(c, w.E2, w.T, w.F);
    gemm_small(s, 0, 0, c, c, c, 1.0, w.V, c, w.F, c, 0.0, w.E, c);         // V (I + Om + Om^2/2)
    RR_CUDA(cudaMemcpyAsync(w.V, w.E, (size_t)c * c * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  ns_orthonormalize(s, c, w.V, w);
  gemm_small(s, 0, 0, r, c, c, 1.0, C, r, w.V, c, 0.0, Mout, r);            // M = C V
  if (Vout != w.V)
    RR_CUDA(cudaMemcpyAsync(Vout, w.V, (size_t)c * c * sizeof(double), cudaMemcpyDeviceToDevice, s));
  note_launches(18);
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
  whiten(s, n, G, w, w.drop1, w.W1);
  // C = W^T H W, symmetrised and shifted positive definite (C - mu I)
  gemm_small(s, 0, 0, n, n, n, 1.0, H, n, w.W1, n, 0.0, w.T, n);
  gemm_small(s, 1, 0, n, n, n, 1.0, w.W1, n, w.T, n, 0.0, w.C, n);
  k_eig_prep<<<1, kSmallThreads, 0, s>>>(n, w.C, w.drop1, w.mu);
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
  // whitening of both sides: Wu -> C, Wv -> V (whiten() uses W1/W2/T/E/E2/F as scratch)
  whiten(s, n1, Gu, w, w.drop1, w.C);
  whiten(s, n2, Gv, w, w.drop2, w.V);
  RR_CUDA(cudaMemcpyAsync(w.W1, w.C, (size_t)n1 * n1 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  RR_CUDA(cudaMemcpyAsync(w.W2, w.V, (size_t)n2 * n2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
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
  note_launches(7);
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
