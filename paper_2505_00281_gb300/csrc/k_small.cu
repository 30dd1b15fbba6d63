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
// A sub-round has three phases separated by __syncthreads: (1) warp i forms
// the inner product of its pair (in the cross rounds column i of block a
// stays in warp i's registers for the whole round); (2) one warp computes the
// w rotations, lane j for pair j, and carries the squared column norms
// through them (|x'|^2 = |x|^2 - t g, |y'|^2 = |y|^2 + t g; the norms are
// computed when the block is loaded); (3) warp i applies its rotation to the
// pair and to the round's 2w x 2w accumulated rotation Q, which is applied to
// the V block once at the end of the round (V_blk <- V_blk Q).  A pair whose
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

// Shared-memory layout: Ms [2w][rp] and Vs [2w][cp4] with rp, cp4 the row
// counts rounded up to 4 (zero rows; float4 access), Qs [2w][ldq], nrm [2w],
// gam / rc / rs [w] (inner products and rotations of the sub-round).
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
  float* gam = nrm + w2;
  float* rc = gam + w;
  float* rs = rc + w;
  const int P = gridDim.x, g = blockIdx.x, nblk = 2 * P;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kBJThreads / 32;
  const int rch = rp >> 2;  // float4 chunks per M column
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
        // (1) inner products
        int p = 0, q = 0;
        float4 x[NCH], y[NCH];
        if (warp < w) {
          bj_pair(round, warp, sr, w, p, q);
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
          if (lane == 0) gam[warp] = ga;
        }
        __syncthreads();
        // (2) the rotations, lane j for pair j
        if (warp == 0 && lane < w) {
          int pj, qj;
          bj_pair(round, lane, sr, w, pj, qj);
          const float ga = gam[lane];
          const float al = nrm[pj], be = nrm[qj];
          const float fa = fmaxf(al, nfloor), fb = fmaxf(be, nfloor);
          float cs = 1.f, sn = 0.f;
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
            cs = rsqrtf(u);
            cs = cs * fmaf(-0.5f * u, cs * cs, 1.5f);  // one Newton step: cs^2 (1 + t^2) = 1
            sn = cs * tt;
            nrm[pj] = al - tt * ga;
            nrm[qj] = be + tt * ga;
            s_rot = 1;
          }
          rc[lane] = cs;
          rs[lane] = sn;
        }
        __syncthreads();
        // (3) apply
        if (warp < w) {
          const float cs = rc[warp], sn = rs[warp];
          if (sn != 0.f) {
            float4* mp = reinterpret_cast<float4*>(Ms + (size_t)p * rp);
            float4* mq = reinterpret_cast<float4*>(Ms + (size_t)q * rp);
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
              else if (c < rch) mp[c] = a4;
              if (c < rch) mq[c] = b4;
            }
            if (lane < w2) {
              const float qp = Qs[lane * ldq + p], qq = Qs[lane * ldq + q];
              Qs[lane * ldq + p] = cs * qp - sn * qq;
              Qs[lane * ldq + q] = sn * qp + cs * qq;
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

// F = 1.5 I - 0.5 T
__global__ void k_ns_coef(int c, const double* __restrict__ T, double* __restrict__ F) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= c * c) return;
  int i = e % c, j = e / c;
  F[e] = (i == j ? 1.5 : 0.0) - 0.5 * T[e];
}

struct PencilWs {
  double *W1, *W2, *T, *E, *E2, *F, *C, *V, *Vp, *M, *Mp, *sig, *mu;
  float *L32, *Li32, *M32, *V32, *fs;  // fs: [0] Jacobi norm floor, [1] scale
  int *drop1, *drop2, *order, *nvalid, *rot, *err, *sweeps;
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
  w.Vp = ar.take<double>(cc);
  w.M = ar.take<double>(rc);
  w.Mp = ar.take<double>(rc);
  w.sig = ar.take<double>(cp);
  w.mu = ar.take<double>(2);
  w.fs = ar.take<float>(4);
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
  const size_t sm = ((size_t)b * (b + 1) / 2 + 2 * (size_t)b) * sizeof(float);
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

static size_t bj_smem(int r, int cpad, int w) {
  const size_t rp = (r + 3) & ~3, cp4 = (cpad + 3) & ~3;
  const size_t ldq = (2 * w + 7) & ~3;
  return ((size_t)2 * w * (rp + cp4) + (size_t)2 * w * ldq + 2 * w + 3 * (size_t)w) * sizeof(float);
}

static rr_status launch_bj(cudaStream_t s, int r, int cpad, int w, int P, float* M, float* V, float tol,
                           int max_sweeps, PencilWs& ws, const float* floor_ptr = nullptr) {
  const int rp = (r + 3) & ~3;
  if (rp > 128 * kBJMaxChunks || cpad > 128 * kBJMaxChunks || 2 * w > 32 || w < 1) return RR_ERR_ARG;
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
  // FP32 copy scaled by a power of two to max entry in [1/2, 1): squared
  // column norms stay well inside the FP32 range
  k_pow2_scale<<<1, 1024, 0, s>>>(r, c, C, r, w.fs + 1);
  k_pad_copy<double, float><<<g, 256, 0, s>>>(r, c, cpad, C, r, w.M32, w.V32, w.fs + 1);
  float* fl = w.fs;
  k_colnorm_floor<float><<<1, 1024, 0, s>>>(r, cpad, w.M32, r, 1e-10f, fl);
  RR_TRY(launch_bj(s, r, cpad, ww, P, w.M32, w.V32, 1e-4f, 15, w, fl));
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
  note_launches(22);  // 4 setup kernels, 3 x 6 polish kernels (+ the final product in check_launch)
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
