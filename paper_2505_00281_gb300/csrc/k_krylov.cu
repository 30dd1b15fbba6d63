// Krylov-Hessenberg process (Sec. 4.1, Alg. 7) and the Krylov eigensolver
// built on it with OFRR (Alg. 3), for sparse symmetric operators.
//
// Alg. 7 builds a basis of K_k(A, v) without inner products: each new vector
// A v_j is reduced at the pivot rows of the earlier vectors (the preselected
// vectors z_i = e_{pi_i}) and scaled so that its largest-magnitude entry (its
// pivot, found by one argmax reduction) is 1.  Step j on the GPU:
//   w = A v_j (CSR product; kept as column j of AV, the raw products the
//       projection needs);
//   coefficients h_ij = w^(i-1)(pi_i), i = 1..j: the value at pivot row pi_i
//       after the first i-1 subtractions, a forward substitution over the j x j
//       unit lower triangle of pivot-row entries (one thread: sequential, as
//       the process is);
//   every row: w(r) <- w(r) - h_1j v_1(r) - ... - h_jj v_j(r) in that order,
//       each a separately rounded multiply and subtract, so the rows see the
//       operations of the literal loop; per-CTA argmax of |w| (first index on
//       ties) as partials;
//   the pivot from the partials (one CTA), then v_{j+1} = w / w(pi).
// The whole process is arithmetic-exact against a sequential loop in the same
// precision (FP64, or FP32 for the low-precision basis of Sec. 4.2).
#include <algorithm>
#include <cmath>
#include <vector>

#include "rr_common.cuh"
#include "solver_kernels.cuh"

namespace rr {
namespace {

template <typename T> __device__ __forceinline__ T kmul(T a, T b);
template <> __device__ __forceinline__ float kmul<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ double kmul<double>(double a, double b) { return __dmul_rn(a, b); }
template <typename T> __device__ __forceinline__ T ksub(T a, T b);
template <> __device__ __forceinline__ float ksub<float>(float a, float b) { return __fsub_rn(a, b); }
template <> __device__ __forceinline__ double ksub<double>(double a, double b) { return __dsub_rn(a, b); }
template <typename T> __device__ __forceinline__ T kdiv(T a, T b);
template <> __device__ __forceinline__ float kdiv<float>(float a, float b) { return __fdiv_rn(a, b); }
template <> __device__ __forceinline__ double kdiv<double>(double a, double b) { return __ddiv_rn(a, b); }

constexpr int kKhThreads = 256;

// v (FP64, the caller's start vector) -> T
template <typename T>
__global__ void k_kh_load(int64_t n, const double* __restrict__ v, T* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = (T)v[i];
}

// h_ij = w^(i-1)(pi_i) for i < j1 by forward substitution, written to c[i]
// and to column `hcol` of H (FP64).  Pr holds the pivot rows' entries
// column-major, Pr[l k + i] = v_l(pi_i) for l < i.  The substitution runs by
// columns of the triangle: once c_l is final, every later row i subtracts
// c_l v_l(pi_i) (threads over i, one barrier per l), so each c_i sees
// exactly the subtractions of the sequential loop in its order, with the
// triangle's columns read coalesced from global memory.
template <typename T>
__global__ void k_kh_coeffs(int j1, int k, const T* __restrict__ Pr, const int* __restrict__ piv,
                            const T* __restrict__ w, T* __restrict__ c, double* __restrict__ Hcol) {
  extern __shared__ unsigned char kh_smem[];
  T* sw = reinterpret_cast<T*>(kh_smem);  // [j1]: w(pi_i), then c_i
  for (int i = threadIdx.x; i < j1; i += blockDim.x) sw[i] = w[piv[i]];
  __syncthreads();
  for (int l = 0; l + 1 < j1; ++l) {
    const T cl = sw[l];
    const T* col = Pr + (size_t)l * k;
    for (int i = l + 1 + threadIdx.x; i < j1; i += blockDim.x) sw[i] = ksub<T>(sw[i], kmul<T>(cl, col[i]));
    __syncthreads();
  }
  for (int i = threadIdx.x; i < j1; i += blockDim.x) {
    c[i] = sw[i];
    Hcol[i] = (double)sw[i];
  }
}

// after pivot pi_j of the new vector v_j is known: Pr[l k + j] = v_l(pi_j),
// l < j (the new pivot row's entries in the earlier vectors)
template <typename T>
__global__ void k_kh_pivot_row(int j, int k, const T* __restrict__ V, int64_t ldv, const int* __restrict__ piv,
                               T* __restrict__ Pr) {
  const int p = piv[j];
  for (int l = threadIdx.x; l < j; l += blockDim.x) Pr[(size_t)l * k + j] = V[p + (int64_t)l * ldv];
}

// w(r) <- w(r) - sum_{i < j1} c_i v_i(r) (in order), and the per-CTA argmax
// of |w| (first index on ties) into (pv, pi)[blockIdx.x]
template <typename T>
__global__ void __launch_bounds__(kKhThreads) k_kh_update(int64_t n, int j1, const T* __restrict__ V, int64_t ldv,
                                                          const T* __restrict__ c, T* __restrict__ w,
                                                          T* __restrict__ pv, int64_t* __restrict__ pi) {
  __shared__ T rv[kKhThreads / 32];
  __shared__ int64_t ri[kKhThreads / 32];
  T bv = T(-1);
  int64_t bi = INT64_MAX;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T t = w[i];
    // the loads of 8 columns go out before their ordered subtractions
    int l = 0;
    for (; l + 8 <= j1; l += 8) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = V[i + (int64_t)(l + u) * ldv];
#pragma unroll
      for (int u = 0; u < 8; ++u) t = ksub<T>(t, kmul<T>(c[l + u], v[u]));
    }
    for (; l < j1; ++l) t = ksub<T>(t, kmul<T>(c[l], V[i + (int64_t)l * ldv]));
    w[i] = t;
    const T a = fabs(t);
    if (a > bv) {
      bv = a;
      bi = i;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  if (lane == 0) {
    rv[wid] = bv;
    ri[wid] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < kKhThreads / 32; ++q)
      if (rv[q] > bv || (rv[q] == bv && ri[q] < bi)) {
        bv = rv[q];
        bi = ri[q];
      }
    pv[blockIdx.x] = bv;
    pi[blockIdx.x] = bi;
  }
}

// pivot of the new vector from the per-CTA partials (first index on ties);
// piv[j] = row, H(j, j-1) = w(row) (skipped when j == 0), *pw = w(row)
// (one CTA of 256 threads: strided partials, then warp and block merges)
template <typename T>
__global__ void __launch_bounds__(256) k_kh_pivot(int nparts, const T* __restrict__ pv, const int64_t* __restrict__ pi,
                                                  const T* __restrict__ w, int j, int* __restrict__ piv,
                                                  double* __restrict__ Hsub, T* __restrict__ pw) {
  __shared__ T rv[8];
  __shared__ int64_t ri[8];
  T bv = T(-1);
  int64_t bi = INT64_MAX;
  for (int q = threadIdx.x; q < nparts; q += blockDim.x)
    if (pv[q] > bv || (pv[q] == bv && pi[q] < bi)) {
      bv = pv[q];
      bi = pi[q];
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    rv[threadIdx.x >> 5] = bv;
    ri[threadIdx.x >> 5] = bi;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
    if (rv[q] > bv || (rv[q] == bv && ri[q] < bi)) {
      bv = rv[q];
      bi = ri[q];
    }
  const int r = bi == INT64_MAX ? 0 : (int)bi;
  piv[j] = r;
  *pw = w[r];
  if (Hsub) *Hsub = (double)w[r];
}

// v_j = w / w(pivot)
template <typename T>
__global__ void k_kh_scale(int64_t n, const T* __restrict__ w, const T* __restrict__ pw, T* __restrict__ vj) {
  const T d = *pw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    vj[i] = kdiv<T>(w[i], d);
}

template <typename T>
size_t kh_ws_bytes(int64_t n, int k) {
  const int nparts = 8 * 160;
  return align_up((size_t)n * sizeof(T)) + align_up((size_t)k * sizeof(T)) + align_up(nparts * sizeof(T)) +
         align_up(nparts * sizeof(int64_t)) + align_up(sizeof(T)) + align_up((size_t)k * k * sizeof(T)) + 256;
}

template <typename T>
rr_status kh_run(cudaStream_t s, int64_t n, int k, const int32_t* rp, const int32_t* ci, const float* va,
                 const double* v, T* V, T* AV, int64_t ldv, double* H, int* piv, void* ws, size_t ws_bytes) {
  if (ws_bytes < kh_ws_bytes<T>(n, k) || !ws) return RR_ERR_WORKSPACE;
  Arena ar(ws, ws_bytes);
  T* w = ar.take<T>(n);
  T* c = ar.take<T>(k);
  const int nparts = (int)std::min<int64_t>((n + kKhThreads - 1) / kKhThreads, 8 * (int64_t)num_sms());
  T* pv = ar.take<T>(8 * 160);
  int64_t* pi = ar.take<int64_t>(8 * 160);
  T* pw = ar.take<T>(1);
  T* Pr = ar.take<T>((size_t)k * k);
  if (nparts > 8 * 160) return RR_ERR_ARG;
  const int32_t dt = sizeof(T) == 8 ? RR_F64 : RR_F32;
  const unsigned g = (unsigned)nparts;
  RR_CUDA(cudaMemsetAsync(H, 0, (size_t)k * k * sizeof(double), s));
  // v_1 = v / v(pivot)
  k_kh_load<T><<<g, kKhThreads, 0, s>>>(n, v, w);
  k_kh_update<T><<<g, kKhThreads, 0, s>>>(n, 0, V, ldv, c, w, pv, pi);  // no subtraction: argmax only
  k_kh_pivot<T><<<1, 256, 0, s>>>(nparts, pv, pi, w, 0, piv, nullptr, pw);
  k_kh_scale<T><<<g, kKhThreads, 0, s>>>(n, w, pw, V);
  note_launches(4);
  for (int j = 0; j < k; ++j) {
    // w = A v_j (kept as the raw product column j)
    RR_TRY(rr_csr_spmm(n, 1, rp, ci, va, dt, V + (int64_t)j * ldv, ldv, dt, AV + (int64_t)j * ldv, ldv, s));
    if (j + 1 == k) break;
    RR_CUDA(cudaMemcpyAsync(w, AV + (int64_t)j * ldv, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    const int j1 = j + 1;
    k_kh_coeffs<T><<<1, 256, (size_t)j1 * sizeof(T), s>>>(j1, k, Pr, piv, w, c, H + (int64_t)j * k);
    k_kh_update<T><<<g, kKhThreads, 0, s>>>(n, j1, V, ldv, c, w, pv, pi);
    k_kh_pivot<T><<<1, 256, 0, s>>>(nparts, pv, pi, w, j1, piv, H + (int64_t)j * k + j1, pw);
    k_kh_scale<T><<<g, kKhThreads, 0, s>>>(n, w, pw, V + (int64_t)j1 * ldv);
    k_kh_pivot_row<T><<<1, 128, 0, s>>>(j1, k, V, ldv, piv, Pr);
    note_launches(5);
  }
  return check_launch("krylov_hessenberg");
}

// Left-looking Hessenberg process on a block (the Hess-L comparator of
// Table 3): column j takes all earlier columns' eliminations at once when it
// is reached (coefficients by forward substitution at the earlier pivot rows,
// then the ordered subtraction), then its argmax and scaling -- the Krylov
// process's step with the next column of W in place of A v_j.  In place: W
// becomes Q.  No column skip (the comparator is timed on full-rank blocks).
template <typename T>
rr_status hess_left_t(cudaStream_t s, int64_t n, int k, T* W, int64_t ldw, int* piv, void* ws, size_t ws_bytes) {
  if (ws_bytes < kh_ws_bytes<T>(n, k) + align_up((size_t)k * k * sizeof(double)) || !ws) return RR_ERR_WORKSPACE;
  Arena ar(ws, ws_bytes);
  ar.take<T>(n);
  T* c = ar.take<T>(k);
  const int nparts = (int)std::min<int64_t>((n + kKhThreads - 1) / kKhThreads, 8 * (int64_t)num_sms());
  T* pv = ar.take<T>(8 * 160);
  int64_t* pi = ar.take<int64_t>(8 * 160);
  T* pw = ar.take<T>(1);
  T* Pr = ar.take<T>((size_t)k * k);
  double* H = ar.take<double>((size_t)k * k);
  const unsigned g = (unsigned)nparts;
  for (int j = 0; j < k; ++j) {
    T* wj = W + (int64_t)j * ldw;
    if (j > 0)
      k_kh_coeffs<T><<<1, 256, (size_t)j * sizeof(T), s>>>(j, k, Pr, piv, wj, c, H + (int64_t)j * k);
    k_kh_update<T><<<g, kKhThreads, 0, s>>>(n, j, W, ldw, c, wj, pv, pi);
    k_kh_pivot<T><<<1, 256, 0, s>>>(nparts, pv, pi, wj, j, piv, nullptr, pw);
    k_kh_scale<T><<<g, kKhThreads, 0, s>>>(n, wj, pw, wj);
    k_kh_pivot_row<T><<<1, 128, 0, s>>>(j, k, W, ldw, piv, Pr);
    note_launches(5);
  }
  return check_launch("hess_left");
}

// H (b x b) <- (H + H^T) / 2 in place (one thread per entry pair)
__global__ void k_symmetrize(int b, double* __restrict__ H) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= b * b) return;
  const int i = e % b, j = e / b;
  if (i < j) {
    const double a = 0.5 * (H[i + (size_t)j * b] + H[j + (size_t)i * b]);
    H[i + (size_t)j * b] = a;
    H[j + (size_t)i * b] = a;
  }
}

// X(:, j) /= |X(:, j)|_2: CTA (j, chunk) writes the chunk's sum of squares,
// then every CTA of the scaling pass sums its column's chunks (fixed order)
constexpr int kNrmChunks = 64;
__global__ void k_colnorm_parts(int64_t n, const double* __restrict__ X, int64_t ldx, double* __restrict__ parts) {
  const double* x = X + (int64_t)blockIdx.x * ldx;
  const int64_t per = (n + kNrmChunks - 1) / kNrmChunks;
  const int64_t i0 = (int64_t)blockIdx.y * per, i1 = i0 + per < n ? i0 + per : n;
  double acc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc = fma(x[i], x[i], acc);
  __shared__ double red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    parts[(size_t)blockIdx.x * kNrmChunks + blockIdx.y] = t;
  }
}
__global__ void k_normalize_cols(int64_t n, double* __restrict__ X, int64_t ldx, const double* __restrict__ parts) {
  __shared__ double sc;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int c = 0; c < kNrmChunks; ++c) t += parts[(size_t)blockIdx.x * kNrmChunks + c];
    sc = t > 0 ? 1.0 / sqrt(t) : 0.0;
  }
  __syncthreads();
  double* x = X + (int64_t)blockIdx.x * ldx;
  for (int64_t i = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.y * blockDim.x)
    x[i] *= sc;
}

// Ysel rows 0..m-1 (ld m) into a zero-padded (mp x k) copy (the lift's K must
// be a multiple of 8 for the tensor-core path; the basis has zero columns
// m..mp-1)
__global__ void k_pad_rows(int m, int mp, int k, const double* __restrict__ Y, double* __restrict__ Yp) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= mp * k) return;
  const int i = e % mp, j = e / mp;
  Yp[e] = i < m ? Y[i + (size_t)j * m] : 0.0;
}

struct KrylovWs {
  void *V, *AV, *kh;
  size_t kh_bytes;
  int mp;  // m rounded up to 8 (columns of V: the extra ones stay zero)
  double *H, *P, *G, *Y, *th, *tsel, *Ysel, *Ypad, *nparts, *X, *AX, *R, *ss;
  int* piv;
  void *gram_ws, *pen_ws, *lift_ws;
  size_t gram_bytes, pen_bytes, lift_bytes;
};

static bool carve_krylov(Arena& ar, int64_t n, int m, int k, int32_t arith, KrylovWs& w) {
  const size_t es = arith == RR_F64 ? 8 : 4;
  w.mp = (m + 7) / 8 * 8;
  w.V = ar.take_bytes((size_t)n * w.mp * es);
  w.AV = ar.take_bytes((size_t)n * m * es);
  w.kh_bytes = arith == RR_F64 ? kh_ws_bytes<double>(n, m) : kh_ws_bytes<float>(n, m);
  w.kh = ar.take_bytes(w.kh_bytes);
  w.H = ar.take<double>((size_t)m * m);
  w.P = ar.take<double>((size_t)m * m);
  w.G = ar.take<double>((size_t)m * m);
  w.Y = ar.take<double>((size_t)m * m);
  w.th = ar.take<double>(m);
  w.tsel = ar.take<double>(m);
  w.Ysel = ar.take<double>((size_t)m * m);
  w.Ypad = ar.take<double>((size_t)w.mp * k);
  w.nparts = ar.take<double>((size_t)k * kNrmChunks);
  w.X = ar.take<double>((size_t)n * k);
  w.AX = ar.take<double>((size_t)n * k);
  w.R = ar.take<double>((size_t)n * k);
  w.ss = ar.take<double>(k);
  w.piv = ar.take<int>(m);
  w.gram_bytes = rr_gram_workspace_size(n, m, m);
  w.gram_ws = ar.take_bytes(w.gram_bytes);
  w.pen_bytes = rr_pencil_workspace_size(m, m);
  w.pen_ws = ar.take_bytes(w.pen_bytes);
  w.lift_bytes = rr_lift_workspace_size(n, k, w.mp);
  w.lift_ws = ar.take_bytes(w.lift_bytes);
  return !ar.overflow;
}

}  // namespace
}  // namespace rr

namespace rr {
size_t hess_left_ws_bytes(int64_t n, int64_t k, int32_t arith) {
  return (arith == RR_F64 ? kh_ws_bytes<double>(n, (int)k) : kh_ws_bytes<float>(n, (int)k)) +
         align_up((size_t)k * k * sizeof(double)) + 256;
}
rr_status hess_left_run(cudaStream_t s, int32_t arith, int64_t n, int64_t k, void* W, int64_t ldw, int* piv,
                        void* ws, size_t ws_bytes) {
  if (arith == RR_F64) return hess_left_t<double>(s, n, (int)k, (double*)W, ldw, piv, ws, ws_bytes);
  if (arith == RR_F32) return hess_left_t<float>(s, n, (int)k, (float*)W, ldw, piv, ws, ws_bytes);
  return RR_ERR_ARG;
}
}  // namespace rr

using namespace rr;

extern "C" size_t rr_krylov_hessenberg_workspace_size(int64_t n, int32_t k, int32_t arith) {
  return arith == RR_F64 ? kh_ws_bytes<double>(n, k) : kh_ws_bytes<float>(n, k);
}

extern "C" rr_status rr_krylov_hessenberg(int32_t arith, int64_t n, int32_t k, const int32_t* row_ptr,
                                          const int32_t* col_idx, const float* values, const double* v, void* V,
                                          void* AV, int64_t ldv, double* H, int32_t* piv, void* ws, size_t ws_bytes,
                                          void* stream) {
  if (n <= 0 || k < 1 || k > n || ldv < n || !row_ptr || !col_idx || !values || !v || !V || !AV || !H || !piv)
    return RR_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  if (arith == RR_F64)
    return kh_run<double>(s, n, k, row_ptr, col_idx, values, v, (double*)V, (double*)AV, ldv, H, piv, ws, ws_bytes);
  if (arith == RR_F32)
    return kh_run<float>(s, n, k, row_ptr, col_idx, values, v, (float*)V, (float*)AV, ldv, H, piv, ws, ws_bytes);
  return RR_ERR_ARG;
}

extern "C" size_t rr_krylov_workspace_size(int64_t n, int32_t m, int32_t k, int32_t arith) {
  if (n <= 0 || m < 1 || k < 1 || k > m || (arith != RR_F64 && arith != RR_F32)) return 0;
  Arena ar(nullptr, 0);
  KrylovWs w;
  carve_krylov(ar, n, m, k, arith, w);
  return ar.off + 4096;
}

extern "C" rr_status rr_krylov_eig(const rr_operator* A, int32_t m, int32_t restarts, int32_t k, int32_t arith,
                                   const double* v0, double* theta, double* X, double* res, void* ws,
                                   size_t ws_bytes, void* stream) {
  if (!A || A->kind != RR_CSR || A->dtype != RR_F32 || !A->row_ptr || !A->col_idx || !A->values) return RR_ERR_ARG;
  const int64_t n = A->n;
  if (n <= 0 || m < 2 || m > n || m > 335 || k < 1 || k > m || restarts < 0 || !v0 || !theta || !X || !res)
    return RR_ERR_ARG;
  if (arith != RR_F64 && arith != RR_F32) return RR_ERR_ARG;
  Arena ar(ws, ws_bytes);
  KrylovWs w;
  if (!ws || ((uintptr_t)ws & 255) || !carve_krylov(ar, n, m, k, arith, w)) return RR_ERR_WORKSPACE;
  cudaStream_t s = as_stream(stream);
  const float* va = (const float*)A->values;
  const double* v = v0;
  const size_t es = arith == RR_F64 ? 8 : 4;
  if (w.mp > m)
    RR_CUDA(cudaMemset2DAsync((char*)w.V + (size_t)m * n * es, n * es, 0, n * es, w.mp - m, s));
  for (int cyc = 0; cyc <= restarts; ++cyc) {
    // Alg. 7: the basis of K_m(A, v) and the raw products A V
    RR_TRY(rr_krylov_hessenberg(arith, n, m, A->row_ptr, A->col_idx, va, v, w.V, w.AV, n, w.H, w.piv, w.kh,
                                w.kh_bytes, stream));
    // Alg. 3: (V^T A V) y = theta (V^T V) y, FP64-accurate projection
    RR_TRY(rr_gram(n, m, m, arith, w.V, n, arith, w.AV, n, w.P, m, 0, w.gram_ws, w.gram_bytes, stream));
    RR_TRY(rr_gram(n, m, m, arith, w.V, n, arith, w.V, n, w.G, m, 0, w.gram_ws, w.gram_bytes, stream));
    k_symmetrize<<<(m * m + 255) / 256, 256, 0, s>>>(m, w.P);
    RR_TRY(check_launch("krylov symmetrize"));
    RR_TRY(rr_pencil_eig(m, w.P, w.G, w.th, w.Y, w.pen_ws, w.pen_bytes, nullptr, stream));
    RR_TRY(select_eig(s, m, m, RR_LARGEST, w.th, w.Y, m, w.tsel, w.Ysel, m));
    // Ritz vectors of the k largest values (unit columns); the next cycle
    // restarts from the first
    k_pad_rows<<<(unsigned)((w.mp * k + 255) / 256), 256, 0, s>>>(m, w.mp, k, w.Ysel, w.Ypad);
    RR_TRY(check_launch("krylov pad"));
    RR_TRY(rr_lift(n, k, arith, w.V, n, w.mp, 0, nullptr, n, 0, w.Ypad, w.mp, w.X, n, w.lift_ws, w.lift_bytes,
                   stream));
    k_colnorm_parts<<<dim3((unsigned)k, kNrmChunks), 256, 0, s>>>(n, w.X, n, w.nparts);
    k_normalize_cols<<<dim3((unsigned)k, 64), 256, 0, s>>>(n, w.X, n, w.nparts);
    note_launches(1);
    RR_TRY(check_launch("krylov normalize"));
    v = w.X;
  }
  // relative residuals |A x - theta x| / |theta| in FP64
  RR_TRY(rr_csr_spmm(n, k, A->row_ptr, A->col_idx, va, RR_F64, w.X, n, RR_F64, w.AX, n, stream));
  RR_TRY(residual_block(s, n, k, w.AX, n, w.X, n, w.tsel, w.R, n, w.ss, 0));
  RR_TRY(res_finish(s, k, w.ss, w.tsel, res));
  RR_CUDA(cudaMemcpyAsync(theta, w.tsel, (size_t)k * sizeof(double), cudaMemcpyDeviceToDevice, s));
  RR_CUDA(cudaMemcpy2DAsync(X, n * sizeof(double), w.X, n * sizeof(double), n * sizeof(double), k,
                            cudaMemcpyDeviceToDevice, s));
  RR_TRY(normalize_sign(s, n, k, X, n, 0, nullptr, 0));
  return RR_OK;
}
