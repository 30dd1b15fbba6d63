// Sparse operator stages: CSR block product (Sec. 5.1 uses CSR for sparse
// operators) and the fused scaled-Chebyshev filter step (the chebfsi filter
// the paper cites in Sec. 2), one warp per row.
#include <cfloat>
#include <cstdint>
#include <type_traits>

#include "rr_common.cuh"
#include "solver_kernels.cuh"

namespace rr {

template <typename TA> struct AccT { using type = float; };
template <> struct AccT<double> { using type = double; };

// Thread per row, lanes on consecutive rows: with column-major blocks a
// warp's load of Y(i, j) for 32 consecutive rows is contiguous, and so are the
// gathers Y(col_e, j) of a stencil's neighbours.  The row's first kRowE CSR
// entries stay in registers for all b columns (longer rows loop over the
// rest).  Arithmetic in the accumulation type (FP32 for FP32 / BF16 blocks,
// FP64 for FP64 ones: no FP64 instruction on the low-precision path).
constexpr int kRowE = 8;
constexpr int64_t kChebMaxCols = 3072;  // per-column coefficients in 48 KB of shared memory

template <typename A, typename T>
__device__ __forceinline__ A ld_acc(const T* p) {
  return LdAs<A, T>::get(p);
}
template <typename TO, typename A> __device__ __forceinline__ TO st_cvt(A v);
template <> __device__ __forceinline__ float st_cvt<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 st_cvt<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ double st_cvt<double, float>(float v) { return (double)v; }
template <> __device__ __forceinline__ double st_cvt<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float st_cvt<float, double>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 st_cvt<__nv_bfloat16, double>(double v) {
  return __double2bfloat16(v);
}

// Y_next(i,j) = alpha*(sum_e v_e Y_cur(col_e, j) - c*Y_cur(i,j)) - beta*bc_j*Y_prev(i,j) + g_j R(i,j)
// The shift folds into the row's diagonal entry (held in registers), so the
// row's own Y_cur(i, j) is not loaded again; sixteen columns per iteration
// give sixteen independent sums and more loads in flight.
// The per-column coefficients beta * bc_j and gamma_j (FP64 inputs) are
// formed once per CTA in shared memory, in the accumulation type: on the
// FP32 path no FP64 instruction (multiply or conversion) runs per element.
template <typename TY, typename TO>
__global__ void __launch_bounds__(256, std::is_same<TY, double>::value ? 2 : 4) k_csr_cheb(
    int64_t n, int64_t b, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const float* __restrict__ va, const TY* __restrict__ Yc, const TY* __restrict__ Yp, int64_t ld,
    double alpha, double cshift, double beta, const double* __restrict__ bc,
    const double* __restrict__ R, int64_t ldr, const double* __restrict__ gam, TO* __restrict__ Yn,
    int64_t ldn) {
  using A = typename AccT<TY>::type;
  extern __shared__ __align__(16) unsigned char cheb_smem[];
  A* s_pb = reinterpret_cast<A*>(cheb_smem);   // beta * bc_j
  A* s_g = s_pb + b;                           // gamma_j
  __shared__ A s_sc[2];                        // alpha, shift c
  for (int64_t j = threadIdx.x; j < b; j += blockDim.x) {
    s_pb[j] = (A)(beta * (bc ? bc[j] : 1.0));
    s_g[j] = gam ? (A)gam[j] : A(0);
  }
  if (threadIdx.x == 0) {
    s_sc[0] = (A)alpha;
    s_sc[1] = (A)cshift;
  }
  __syncthreads();
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const int e0 = rp[row], e1 = rp[row + 1];
  const int ne = e1 - e0 < kRowE ? e1 - e0 : kRowE;
  int cie[kRowE];
  A vae[kRowE];
  bool diag = false;  // the shift folded into a diagonal entry in registers
#pragma unroll
  for (int t = 0; t < kRowE; ++t) {
    cie[t] = t < ne ? ci[e0 + t] : (int)row;
    vae[t] = t < ne ? (A)va[e0 + t] : A(0);
    if (t < ne && cie[t] == (int)row && !diag) {
      vae[t] -= s_sc[1];
      diag = true;
    }
  }
  const A shift = diag ? A(0) : s_sc[1];  // no diagonal among the first entries
  const A al = s_sc[0];
  // column-group base pointers advance by kC columns per iteration; the
  // per-column offsets u * ld are compile-time multiples shared by all entries
  constexpr int kC = std::is_same<A, double>::value ? 8 : 16;  // columns per iteration
  const TY* yc = Yc;
  int64_t j = 0;
  for (; j + kC <= b; j += kC, yc += kC * ld) {
    A acc[kC];
#pragma unroll
    for (int u = 0; u < kC; ++u) acc[u] = A(0);
#pragma unroll
    for (int t = 0; t < kRowE; ++t)
      if (t < ne) {
#pragma unroll
        for (int u = 0; u < kC; ++u) acc[u] = fma(vae[t], ld_acc<A>(yc + u * ld + cie[t]), acc[u]);
      }
    for (int e = e0 + kRowE; e < e1; ++e) {
      const A ve = (A)va[e];
      const int c = ci[e];
#pragma unroll
      for (int u = 0; u < kC; ++u) acc[u] = fma(ve, ld_acc<A>(yc + u * ld + c), acc[u]);
    }
#pragma unroll
    for (int u = 0; u < kC; ++u) {
      const int64_t jj = j + u;
      A a = acc[u];
      if (!diag) a -= shift * ld_acc<A>(yc + u * ld + row);
      A v = al * a;
      if (Yp) v -= s_pb[jj] * ld_acc<A>(Yp + row + jj * ld);
      if (R && gam) v += s_g[jj] * ld_acc<A>(R + row + jj * ldr);
      Yn[row + jj * ldn] = st_cvt<TO, A>(v);
    }
  }
  for (; j < b; ++j, yc += ld) {
    A acc = A(0);
#pragma unroll
    for (int t = 0; t < kRowE; ++t)
      if (t < ne) acc = fma(vae[t], ld_acc<A>(yc + cie[t]), acc);
    for (int e = e0 + kRowE; e < e1; ++e) acc = fma((A)va[e], ld_acc<A>(yc + ci[e]), acc);
    if (!diag) acc -= shift * ld_acc<A>(yc + row);
    A v = al * acc;
    if (Yp) v -= s_pb[j] * ld_acc<A>(Yp + row + j * ld);
    if (R && gam) v += s_g[j] * ld_acc<A>(R + row + j * ldr);
    Yn[row + j * ldn] = st_cvt<TO, A>(v);
  }
}

// Y = A X, thread per row (same access pattern)
template <typename TX, typename TO>
__global__ void __launch_bounds__(256) k_csr_spmm(int64_t n, int64_t b, const int32_t* __restrict__ rp,
                                                  const int32_t* __restrict__ ci,
                                                  const float* __restrict__ va,
                                                  const TX* __restrict__ X, int64_t ldx,
                                                  TO* __restrict__ Y, int64_t ldy) {
  using A = typename AccT<TX>::type;
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const int e0 = rp[row], e1 = rp[row + 1];
  const int ne = e1 - e0 < kRowE ? e1 - e0 : kRowE;
  int cie[kRowE];
  A vae[kRowE];
#pragma unroll
  for (int t = 0; t < kRowE; ++t) {
    cie[t] = t < ne ? ci[e0 + t] : (int)row;
    vae[t] = t < ne ? (A)va[e0 + t] : A(0);
  }
  for (int64_t j = 0; j < b; ++j) {
    const TX* x = X + j * ldx;
    A acc = A(0);
#pragma unroll
    for (int t = 0; t < kRowE; ++t) acc += vae[t] * ld_acc<A>(x + cie[t]);
    for (int e = e0 + kRowE; e < e1; ++e) acc += (A)va[e] * ld_acc<A>(x + ci[e]);
    Y[row + j * ldy] = st_cvt<TO, A>(acc);
  }
}

template <typename TY>
static rr_status cheb_out(int32_t out_type, dim3 g, cudaStream_t s, int64_t n, int64_t b,
                          const int32_t* rp, const int32_t* ci, const float* va, const TY* Yc,
                          const TY* Yp, int64_t ld, double alpha, double c, double beta,
                          const double* bc, const double* R, int64_t ldr, const double* gam,
                          void* Yn, int64_t ldn) {
  using A = typename AccT<TY>::type;
  const size_t smem = 2 * (size_t)b * sizeof(A);
  switch (out_type) {
    case RR_F64: k_csr_cheb<TY, double><<<g, 256, smem, s>>>(n, b, rp, ci, va, Yc, Yp, ld, alpha, c, beta, bc, R, ldr, gam, (double*)Yn, ldn); break;
    case RR_F32: k_csr_cheb<TY, float><<<g, 256, smem, s>>>(n, b, rp, ci, va, Yc, Yp, ld, alpha, c, beta, bc, R, ldr, gam, (float*)Yn, ldn); break;
    case RR_BF16: k_csr_cheb<TY, __nv_bfloat16><<<g, 256, smem, s>>>(n, b, rp, ci, va, Yc, Yp, ld, alpha, c, beta, bc, R, ldr, gam, (__nv_bfloat16*)Yn, ldn); break;
    default: return RR_ERR_ARG;
  }
  return check_launch("rr_chebyshev_step");
}

template <typename TX>
static rr_status spmm_out(int32_t ytype, dim3 g, cudaStream_t s, int64_t n, int64_t b,
                          const int32_t* rp, const int32_t* ci, const float* va, const TX* X,
                          int64_t ldx, void* Y, int64_t ldy) {
  switch (ytype) {
    case RR_F64: k_csr_spmm<TX, double><<<g, 256, 0, s>>>(n, b, rp, ci, va, X, ldx, (double*)Y, ldy); break;
    case RR_F32: k_csr_spmm<TX, float><<<g, 256, 0, s>>>(n, b, rp, ci, va, X, ldx, (float*)Y, ldy); break;
    case RR_BF16: k_csr_spmm<TX, __nv_bfloat16><<<g, 256, 0, s>>>(n, b, rp, ci, va, X, ldx, (__nv_bfloat16*)Y, ldy); break;
    default: return RR_ERR_ARG;
  }
  return check_launch("rr_csr_spmm");
}

// ---------------------------------------------------------------------------
// Row-major blocks for the plain Chebyshev filter: element (i, j) at
// Y[i * ldr + j].  A thread takes one row and one 16-byte vector of columns
// (8 BF16, 4 FP32 or 2 FP64), so every gather of a neighbour row is one
// 16-byte load and the lanes of a warp read whole rows contiguously.  The
// row's CSR entries go in chunks of kRowChunk: the chunk's vector loads are
// issued together, then its FMAs.  Pad columns (b up to the vector width)
// are read and written like the others.
// ---------------------------------------------------------------------------
constexpr int kRowChunk = 5;
constexpr int64_t kRowsMaxUnits = 256;  // vectors per row: at most one CTA row of threads

template <typename T> struct VecW { static constexpr int V = 16 / (int)sizeof(T); };

// one 16-byte vector of T (raw bits) -> V values of the accumulation type
template <typename T>
__device__ __forceinline__ void unpack_vec(const uint4 u, typename AccT<T>::type (&o)[VecW<T>::V]) {
  if constexpr (std::is_same<T, __nv_bfloat16>::value) {
    const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      o[2 * k] = __uint_as_float(w[k] << 16);
      o[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
    }
  } else if constexpr (std::is_same<T, float>::value) {
    o[0] = __uint_as_float(u.x);
    o[1] = __uint_as_float(u.y);
    o[2] = __uint_as_float(u.z);
    o[3] = __uint_as_float(u.w);
  } else {
    o[0] = __longlong_as_double(((long long)u.y << 32) | u.x);
    o[1] = __longlong_as_double(((long long)u.w << 32) | u.z);
  }
}

template <typename TO, typename A, int V>
__device__ __forceinline__ void st_vec(TO* p, const A (&v)[V]) {
  if constexpr (std::is_same<TO, __nv_bfloat16>::value && V == 8) {
    uint4 u;
    unsigned* w = reinterpret_cast<unsigned*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
      w[k] = *reinterpret_cast<const unsigned*>(&h);
    }
    *reinterpret_cast<uint4*>(p) = u;
  } else if constexpr (std::is_same<TO, float>::value && V == 8) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
  } else if constexpr (std::is_same<TO, float>::value && V == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    static_assert(std::is_same<TO, double>::value && V == 2, "row-major output type");
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
}

// Y_next(i, :) = alpha ((A - c I) Y_cur)(i, :) - beta Y_prev(i, :)   (Y_prev may be null)
// CTA (units, R): threadIdx.x is the column vector, threadIdx.y the row, so
// consecutive lanes cover a row's vectors and then the next row's.  The
// CTA's CSR entries are staged in shared memory (coalesced loads by all
// threads), so a thread's gathers depend on no global load; Y_prev is
// requested before the barrier.  A CTA whose rows hold more than kRowsStage
// entries leaves them to a second kernel that stages them in windows.
constexpr int kRowsStage = 1024;

template <typename TY, typename A, int V>
__device__ __forceinline__ void rows_gather(int e0, int e1, const int* __restrict__ sci, const float* __restrict__ sva,
                                            const TY* __restrict__ Yc, int64_t ldr, int64_t j0, A (&acc)[V]) {
  for (int e = e0; e < e1; e += kRowChunk) {
    uint4 y[kRowChunk];
    A v[kRowChunk];
#pragma unroll
    for (int t = 0; t < kRowChunk; ++t) {
      const bool ok = e + t < e1;
      v[t] = ok ? (A)sva[e + t] : A(0);
      const int c = ok ? sci[e + t] : 0;
      y[t] = ok ? __ldg(reinterpret_cast<const uint4*>(Yc + (int64_t)c * ldr + j0)) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int t = 0; t < kRowChunk; ++t) {
      A f[V];
      unpack_vec<TY>(y[t], f);
#pragma unroll
      for (int k = 0; k < V; ++k) acc[k] = fma(v[t], f[k], acc[k]);
    }
  }
}

// Resident CTAs per SM the row kernel is compiled for (BF16 blocks have a
// kernel of their own below).
template <typename T> struct kRowsMinBlocks { static constexpr int value = 5; };
template <> struct kRowsMinBlocks<double> { static constexpr int value = 3; };

// A row group (the R rows of one CTA of the step kernels) whose rows hold
// more entries than one stage: windows of kRowsStage entries, one gather at a
// time, by every thread of the CTA (the barriers are the CTA's).
template <typename TY, typename TO>
__device__ __forceinline__ void cheb_rows_windows(int g, int n, const int32_t* __restrict__ rp,
                                                  const int32_t* __restrict__ ci, const float* __restrict__ va,
                                                  const TY* __restrict__ Yc, const TY* __restrict__ Yp, int64_t ldr,
                                                  typename AccT<TY>::type alpha, typename AccT<TY>::type cshift,
                                                  typename AccT<TY>::type beta, TO* __restrict__ Yn, int64_t ldn,
                                                  int* s_ci, float* s_va) {
  using A = typename AccT<TY>::type;
  constexpr int V = VecW<TY>::V;
  const int R = blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  const int r0 = g * R, rows = n - r0 < R ? n - r0 : R;
  const int base = __ldg(rp + r0), E = __ldg(rp + r0 + rows) - base;
  const int row = r0 + threadIdx.y;
  const bool mine = (int)threadIdx.y < rows;
  const int64_t j0 = (int64_t)threadIdx.x * V;
  const int e0 = mine ? __ldg(rp + row) - base : 0, e1 = mine ? __ldg(rp + row + 1) - base : 0;
  A acc[V];
#pragma unroll
  for (int k = 0; k < V; ++k) acc[k] = A(0);
  for (int ws = 0; ws < E; ws += kRowsStage) {
    const int we = E - ws < kRowsStage ? E : ws + kRowsStage;
    __syncthreads();  // the previous window (or group) is read
    for (int t = tid; t < we - ws; t += nth) {
      s_ci[t] = __ldg(ci + base + ws + t);
      s_va[t] = __ldg(va + base + ws + t);
    }
    __syncthreads();
    const int lo = e0 > ws ? e0 : ws, hi = e1 < we ? e1 : we;
    for (int e = lo - ws; e < hi - ws; ++e) {
      A f[V];
      unpack_vec<TY>(__ldg(reinterpret_cast<const uint4*>(Yc + (int64_t)s_ci[e] * ldr + j0)), f);
      const A v = (A)s_va[e];
#pragma unroll
      for (int k = 0; k < V; ++k) acc[k] = fma(v, f[k], acc[k]);
    }
  }
  if (!mine) return;
  A f[V];
  unpack_vec<TY>(__ldg(reinterpret_cast<const uint4*>(Yc + row * ldr + j0)), f);
#pragma unroll
  for (int k = 0; k < V; ++k) acc[k] = fma(-cshift, f[k], acc[k]);
  unpack_vec<TY>(__ldg(reinterpret_cast<const uint4*>(Yp + row * ldr + j0)), f);
  A out[V];
#pragma unroll
  for (int k = 0; k < V; ++k) out[k] = fma(-beta, f[k], alpha * acc[k]);
  st_vec<TO, A, V>(Yn + row * ldn + j0, out);
}

// The groups the step kernels skip (more than kRowsStage entries): each
// thread tests one group, the CTA lists the long ones and processes them in
// turn.  Same CTA shape as the step kernel; launched after it on the same
// stream, it costs one pass over the group boundaries when there are none.
template <typename TY, typename TO>
__global__ void __launch_bounds__(256) k_csr_cheb_rows_long(int n, const int32_t* __restrict__ rp,
                                                            const int32_t* __restrict__ ci,
                                                            const float* __restrict__ va, const TY* __restrict__ Yc,
                                                            const TY* __restrict__ Yp, int64_t ldr,
                                                            typename AccT<TY>::type alpha,
                                                            typename AccT<TY>::type cshift,
                                                            typename AccT<TY>::type beta, TO* __restrict__ Yn,
                                                            int64_t ldn) {
  __shared__ int s_ci[kRowsStage];
  __shared__ float s_va[kRowsStage];
  __shared__ int s_list[256];
  __shared__ int s_cnt;
  const int R = blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  const int groups = (n + R - 1) / R;
  for (int g0 = blockIdx.x * nth; g0 < groups; g0 += gridDim.x * nth) {
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    const int g = g0 + tid;
    if (g < groups) {
      const int r0 = g * R, rows = n - r0 < R ? n - r0 : R;
      if (__ldg(rp + r0 + rows) - __ldg(rp + r0) > kRowsStage) s_list[atomicAdd(&s_cnt, 1)] = g;
    }
    __syncthreads();
    const int cnt = s_cnt;
    for (int k = 0; k < cnt; ++k)
      cheb_rows_windows<TY, TO>(s_list[k], n, rp, ci, va, Yc, Yp, ldr, alpha, cshift, beta, Yn, ldn, s_ci, s_va);
    __syncthreads();  // s_cnt and s_list are reused
  }
}

template <typename TY, typename TO>
__global__ void __launch_bounds__(256, kRowsMinBlocks<TY>::value) k_csr_cheb_rows(
    int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const float* __restrict__ va, const TY* __restrict__ Yc, const TY* __restrict__ Yp, int64_t ldr,
    typename AccT<TY>::type alpha, typename AccT<TY>::type cshift, typename AccT<TY>::type beta,
    TO* __restrict__ Yn, int64_t ldn) {
  using A = typename AccT<TY>::type;
  constexpr int V = VecW<TY>::V;
  __shared__ int s_ci[kRowsStage];
  __shared__ float s_va[kRowsStage];
  const int R = blockDim.y;
  const int r0 = blockIdx.x * R;
  const int rows = n - r0 < R ? n - r0 : R;
  const int base = __ldg(rp + r0), E = __ldg(rp + r0 + rows) - base;
  if (E > kRowsStage) return;  // the same for the whole CTA: k_csr_cheb_rows_long takes it
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  const bool mine = (int)threadIdx.y < rows;
  const int row = r0 + threadIdx.y;
  const int64_t j0 = (int64_t)threadIdx.x * V;
  int e0 = 0, e1 = 0;
  uint4 praw = make_uint4(0, 0, 0, 0);
  if (mine) {  // independent of the stage: in flight across the barrier
    e0 = __ldg(rp + row);
    e1 = __ldg(rp + row + 1);
    praw = __ldg(reinterpret_cast<const uint4*>(Yp + row * ldr + j0));  // never null here
  }
  for (int t = tid; t < E; t += nth) {
    s_ci[t] = __ldg(ci + base + t);
    s_va[t] = __ldg(va + base + t);
  }
  __syncthreads();
  if (!mine) return;
  A acc[V];
#pragma unroll
  for (int k = 0; k < V; ++k) acc[k] = A(0);
  rows_gather<TY, A, V>(e0 - base, e1 - base, s_ci, s_va, Yc, ldr, j0, acc);
  // the shift: the row's own vector, usually just gathered as the diagonal entry (an L1 hit)
  A f[V];
  unpack_vec<TY>(__ldg(reinterpret_cast<const uint4*>(Yc + row * ldr + j0)), f);
#pragma unroll
  for (int k = 0; k < V; ++k) acc[k] = fma(-cshift, f[k], acc[k]);
  unpack_vec<TY>(praw, f);
  A out[V];
#pragma unroll
  for (int k = 0; k < V; ++k) out[k] = fma(-beta, f[k], alpha * acc[k]);
  st_vec<TO, A, V>(Yn + row * ldn + j0, out);
}

// BF16 blocks: the same step written for the register budget of eight
// resident CTAs per SM (32 registers, no spills), which is what hides the
// latency of the staged entries and the gathers: FP32 accumulators in pairs
// (a BF16 pair unpacks into one), the output packed pair by pair.
__device__ __forceinline__ float2 bf16x2_unpack(unsigned w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
}

template <typename TO>
__global__ void __launch_bounds__(256, 8) k_csr_cheb_rows_bf16(int n, const int32_t* __restrict__ rp,
                                                               const int32_t* __restrict__ ci,
                                                               const float* __restrict__ va,
                                                               const __nv_bfloat16* __restrict__ Yc,
                                                               const __nv_bfloat16* __restrict__ Yp, int64_t ldr,
                                                               float alpha, float cshift, float beta,
                                                               TO* __restrict__ Yn, int64_t ldn) {
  __shared__ int s_ci[kRowsStage];
  __shared__ float s_va[kRowsStage];
  const int R = blockDim.y;
  const int r0 = blockIdx.x * R;
  const int rows = n - r0 < R ? n - r0 : R;
  const int base = __ldg(rp + r0), E = __ldg(rp + r0 + rows) - base;
  if (E > kRowsStage) return;  // the same for the whole CTA: k_csr_cheb_rows_long takes it
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  const bool mine = (int)threadIdx.y < rows;
  const int row = r0 + threadIdx.y;
  const int64_t j0 = (int64_t)threadIdx.x * 8;
  int e0 = 0, e1 = 0;
  uint4 praw = make_uint4(0, 0, 0, 0);
  if (mine) {  // independent of the stage: in flight across the barrier
    e0 = __ldg(rp + row) - base;
    e1 = __ldg(rp + row + 1) - base;
    praw = __ldg(reinterpret_cast<const uint4*>(Yp + row * ldr + j0));
  }
  for (int t = tid; t < E; t += nth) {
    s_ci[t] = __ldg(ci + base + t);
    s_va[t] = __ldg(va + base + t);
  }
  __syncthreads();
  if (!mine) return;
  float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  for (int e = e0; e < e1; e += kRowChunk) {
    uint4 y[kRowChunk];
    float v[kRowChunk];
#pragma unroll
    for (int t = 0; t < kRowChunk; ++t) {
      const bool ok = e + t < e1;
      const int c = ok ? s_ci[e + t] : 0;
      v[t] = ok ? s_va[e + t] : 0.f;
      y[t] = ok ? __ldg(reinterpret_cast<const uint4*>(Yc + (int64_t)c * ldr + j0)) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int t = 0; t < kRowChunk; ++t) {
      const unsigned w[4] = {y[t].x, y[t].y, y[t].z, y[t].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 f = bf16x2_unpack(w[q]);
        acc[q].x = fmaf(v[t], f.x, acc[q].x);
        acc[q].y = fmaf(v[t], f.y, acc[q].y);
      }
    }
  }
  // the shift: the row's own vector, usually just gathered as the diagonal entry (an L1 hit)
  const uint4 u = __ldg(reinterpret_cast<const uint4*>(Yc + row * ldr + j0));
  const unsigned wu[4] = {u.x, u.y, u.z, u.w}, wp[4] = {praw.x, praw.y, praw.z, praw.w};
  float o[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 f = bf16x2_unpack(wu[q]), pp = bf16x2_unpack(wp[q]);
    o[2 * q] = fmaf(-beta, pp.x, alpha * fmaf(-cshift, f.x, acc[q].x));
    o[2 * q + 1] = fmaf(-beta, pp.y, alpha * fmaf(-cshift, f.y, acc[q].y));
  }
  st_vec<TO, float, 8>(Yn + row * ldn + j0, o);
}

// column-major (ld) <-> row-major (row stride ldr, pad columns b .. bp - 1
// written as zero), 32 x 32 tiles through shared memory
template <typename T>
__global__ void k_cols_to_rows(int64_t n, int64_t b, int64_t bp, const T* __restrict__ src, int64_t ld,
                               T* __restrict__ dst, int64_t ldr) {
  __shared__ T tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + threadIdx.x, j = j0 + r;
    tile[r][threadIdx.x] = (i < n && j < b) ? src[i + j * ld] : T(0);
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + threadIdx.x;
    if (i < n && j < bp) dst[i * ldr + j] = tile[threadIdx.x][r];
  }
}

template <typename T>
__global__ void k_rows_to_cols(int64_t n, int64_t b, const T* __restrict__ src, int64_t ldr, T* __restrict__ dst,
                               int64_t ld) {
  __shared__ T tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + threadIdx.x;
    if (i < n && j < b) tile[r][threadIdx.x] = src[i * ldr + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + threadIdx.x, j = j0 + r;
    if (i < n && j < b) dst[i + j * ld] = tile[threadIdx.x][r];
  }
}

rr_status block_to_rows(cudaStream_t s, int32_t t, int64_t n, int64_t b, int64_t bp, const void* src,
                        int64_t ld, void* dst, int64_t ldr) {
  if (n == 0 || bp == 0) return RR_OK;
  dim3 g((unsigned)((n + 31) / 32), (unsigned)((bp + 31) / 32)), th(32, 8);
  switch (t) {
    case RR_F64: k_cols_to_rows<double><<<g, th, 0, s>>>(n, b, bp, (const double*)src, ld, (double*)dst, ldr); break;
    case RR_F32: k_cols_to_rows<float><<<g, th, 0, s>>>(n, b, bp, (const float*)src, ld, (float*)dst, ldr); break;
    case RR_BF16:
      k_cols_to_rows<__nv_bfloat16><<<g, th, 0, s>>>(n, b, bp, (const __nv_bfloat16*)src, ld, (__nv_bfloat16*)dst, ldr);
      break;
    default: return RR_ERR_ARG;
  }
  return check_launch("block_to_rows");
}

rr_status block_from_rows(cudaStream_t s, int32_t t, int64_t n, int64_t b, const void* src, int64_t ldr, void* dst,
                          int64_t ld) {
  if (n == 0 || b == 0) return RR_OK;
  dim3 g((unsigned)((n + 31) / 32), (unsigned)((b + 31) / 32)), th(32, 8);
  switch (t) {
    case RR_F64: k_rows_to_cols<double><<<g, th, 0, s>>>(n, b, (const double*)src, ldr, (double*)dst, ld); break;
    case RR_F32: k_rows_to_cols<float><<<g, th, 0, s>>>(n, b, (const float*)src, ldr, (float*)dst, ld); break;
    case RR_BF16:
      k_rows_to_cols<__nv_bfloat16><<<g, th, 0, s>>>(n, b, (const __nv_bfloat16*)src, ldr, (__nv_bfloat16*)dst, ld);
      break;
    default: return RR_ERR_ARG;
  }
  return check_launch("block_from_rows");
}

template <typename TY, typename TO>
static rr_status cheb_rows_launch(cudaStream_t s, int64_t n, int64_t b, const int32_t* rp, const int32_t* ci,
                                  const float* va, const void* Yc, const void* Yp, int64_t ldr, double alpha,
                                  double c, double beta, void* Yn, int64_t ldn) {
  using A = typename AccT<TY>::type;
  constexpr int V = VecW<TY>::V;
  const int64_t units = (b + V - 1) / V;
  if (units > kRowsMaxUnits || n > INT32_MAX) return RR_ERR_ARG;
  if (n == 0 || units == 0) return RR_OK;
  const int64_t R = std::max<int64_t>(1, 256 / units);
  dim3 th((unsigned)units, (unsigned)R);
  // without Y_prev the kernels read Y_cur in its place, times beta = 0
  const TY* yp = (const TY*)(Yp ? Yp : Yc);
  const A bt = (A)(Yp ? beta : 0.0);
  const int64_t groups = (n + R - 1) / R;
  if constexpr (std::is_same<TY, __nv_bfloat16>::value && !std::is_same<TO, double>::value)
    k_csr_cheb_rows_bf16<TO><<<(unsigned)groups, th, 0, s>>>((int)n, rp, ci, va, (const TY*)Yc, yp, ldr, (A)alpha,
                                                           (A)c, bt, (TO*)Yn, ldn);
  else
    k_csr_cheb_rows<TY, TO><<<(unsigned)groups, th, 0, s>>>((int)n, rp, ci, va, (const TY*)Yc, yp, ldr, (A)alpha,
                                                            (A)c, bt, (TO*)Yn, ldn);
  RR_TRY(check_launch("rr_chebyshev_step_rows"));
  const int64_t per = (int64_t)th.x * th.y, lg = (groups + per - 1) / per;
  k_csr_cheb_rows_long<TY, TO><<<(unsigned)(lg < 4 * num_sms() ? lg : 4 * num_sms()), th, 0, s>>>(
      (int)n, rp, ci, va, (const TY*)Yc, yp, ldr, (A)alpha, (A)c, bt, (TO*)Yn, ldn);
  return check_launch("rr_chebyshev_step_rows long rows");
}

// row-major step: (ytype, out_type) in {(BF16, BF16), (BF16, F32), (F32, F32), (F64, F64)}
rr_status cheb_rows(cudaStream_t s, int64_t n, int64_t b, const int32_t* rp, const int32_t* ci, const float* va,
                    int32_t ytype, const void* Yc, const void* Yp, int64_t ldr, double alpha, double c, double beta,
                    int32_t out_type, void* Yn, int64_t ldn) {
  if (ytype == RR_BF16 && out_type == RR_BF16)
    return cheb_rows_launch<__nv_bfloat16, __nv_bfloat16>(s, n, b, rp, ci, va, Yc, Yp, ldr, alpha, c, beta, Yn, ldn);
  if (ytype == RR_BF16 && out_type == RR_F32)
    return cheb_rows_launch<__nv_bfloat16, float>(s, n, b, rp, ci, va, Yc, Yp, ldr, alpha, c, beta, Yn, ldn);
  if (ytype == RR_F32 && out_type == RR_F32)
    return cheb_rows_launch<float, float>(s, n, b, rp, ci, va, Yc, Yp, ldr, alpha, c, beta, Yn, ldn);
  if (ytype == RR_F64 && out_type == RR_F64)
    return cheb_rows_launch<double, double>(s, n, b, rp, ci, va, Yc, Yp, ldr, alpha, c, beta, Yn, ldn);
  return RR_ERR_ARG;
}

// Gershgorin bounds of a symmetric CSR matrix: per-block partial min/max,
// then one block reduces (deterministic).
__global__ void k_gersh_partial(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const float* __restrict__ va, double* __restrict__ part) {
  double lo = DBL_MAX, hi = -DBL_MAX;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0, r = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      if (ci[e] == i) d += va[e];
      else r += fabs((double)va[e]);
    }
    lo = fmin(lo, d - r);
    hi = fmax(hi, d + r);
  }
  __shared__ double sl[32], sh[32];
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    sl[threadIdx.x >> 5] = lo;
    sh[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lo = fmin(lo, sl[w]);
      hi = fmax(hi, sh[w]);
    }
    part[2 * blockIdx.x] = fmin(lo, sl[0]);
    part[2 * blockIdx.x + 1] = fmax(hi, sh[0]);
  }
}

__global__ void k_gersh_final(int nb, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double lo = DBL_MAX, hi = -DBL_MAX;
    for (int i = 0; i < nb; ++i) {
      lo = fmin(lo, part[2 * i]);
      hi = fmax(hi, part[2 * i + 1]);
    }
    out[0] = lo;
    out[1] = hi;
  }
}

rr_status csr_gershgorin(cudaStream_t s, int64_t n, const int32_t* rp, const int32_t* ci,
                         const float* va, double* scratch) {
  // scratch: 2*256 partials followed by the 2 outputs
  k_gersh_partial<<<256, 256, 0, s>>>(n, rp, ci, va, scratch);
  k_gersh_final<<<1, 32, 0, s>>>(256, scratch, scratch + 512);
  note_launches(1);
  return check_launch("csr_gershgorin");
}

// Scalars of the Chebyshev difference recurrence (see solver.cu):
// kappa_next = (alpha_next (theta - c) kappa - beta_next kappa_prev rho) / mu,
// rho_next = 1/mu, kappa_prev <- kappa, kappa <- kappa_next.
__global__ void k_cheb_coef(int64_t b, const double* __restrict__ theta, const double* __restrict__ mu,
                            double an, double cs, double bn, double* __restrict__ kap,
                            double* __restrict__ kap_prev, double* __restrict__ rho) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= b) return;
  double kn = (an * (theta[j] - cs) * kap[j] - bn * kap_prev[j] * rho[j]) / mu[j];
  kap_prev[j] = kap[j];
  kap[j] = kn;
  rho[j] = 1.0 / mu[j];
}

rr_status cheb_coef_update(cudaStream_t s, int64_t b, const double* theta, const double* mu,
                           double alpha_next, double cshift, double beta_next, double* kappa,
                           double* kappa_prev, double* rho) {
  k_cheb_coef<<<(unsigned)((b + 127) / 128), 128, 0, s>>>(b, theta, mu, alpha_next, cshift, beta_next,
                                                         kappa, kappa_prev, rho);
  return check_launch("cheb_coef_update");
}

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_csr_spmm(int64_t n, int64_t b, const int32_t* row_ptr, const int32_t* col_idx,
                                 const float* values, int32_t xtype, const void* X, int64_t ldx,
                                 int32_t ytype, void* Y, int64_t ldy, void* stream) {
  if (n < 0 || b < 0 || ldx < n || ldy < n || !row_ptr || !X || !Y) return RR_ERR_ARG;
  if (n == 0 || b == 0) return RR_OK;
  dim3 g((unsigned)((n + 255) / 256));
  cudaStream_t s = as_stream(stream);
  switch (xtype) {
    case RR_F64: return spmm_out<double>(ytype, g, s, n, b, row_ptr, col_idx, values, (const double*)X, ldx, Y, ldy);
    case RR_F32: return spmm_out<float>(ytype, g, s, n, b, row_ptr, col_idx, values, (const float*)X, ldx, Y, ldy);
    case RR_BF16: return spmm_out<__nv_bfloat16>(ytype, g, s, n, b, row_ptr, col_idx, values, (const __nv_bfloat16*)X, ldx, Y, ldy);
  }
  return RR_ERR_ARG;
}

extern "C" rr_status rr_chebyshev_step(int64_t n, int64_t b, const int32_t* row_ptr,
                                       const int32_t* col_idx, const float* values, int32_t ytype,
                                       const void* Y_cur, const void* Y_prev, int64_t ld, double alpha,
                                       double c, double beta, const double* beta_col, const double* R,
                                       int64_t ldr, const double* gamma, int32_t out_type, void* Y_next,
                                       int64_t ld_next, void* stream) {
  if (n < 0 || b < 0 || ld < n || ld_next < n || !row_ptr || !Y_cur || !Y_next) return RR_ERR_ARG;
  if ((R != nullptr) != (gamma != nullptr)) return RR_ERR_ARG;
  if (b > kChebMaxCols) return RR_ERR_ARG;
  if (n == 0 || b == 0) return RR_OK;
  dim3 g((unsigned)((n + 255) / 256));
  cudaStream_t s = as_stream(stream);
  switch (ytype) {
    case RR_F64: return cheb_out<double>(out_type, g, s, n, b, row_ptr, col_idx, values, (const double*)Y_cur, (const double*)Y_prev, ld, alpha, c, beta, beta_col, R, ldr, gamma, Y_next, ld_next);
    case RR_F32: return cheb_out<float>(out_type, g, s, n, b, row_ptr, col_idx, values, (const float*)Y_cur, (const float*)Y_prev, ld, alpha, c, beta, beta_col, R, ldr, gamma, Y_next, ld_next);
    case RR_BF16: return cheb_out<__nv_bfloat16>(out_type, g, s, n, b, row_ptr, col_idx, values, (const __nv_bfloat16*)Y_cur, (const __nv_bfloat16*)Y_prev, ld, alpha, c, beta, beta_col, R, ldr, gamma, Y_next, ld_next);
  }
  return RR_ERR_ARG;
}

extern "C" rr_status rr_chebyshev_step_rows(int64_t n, int64_t b, const int32_t* row_ptr, const int32_t* col_idx,
                                            const float* values, int32_t ytype, const void* Y_cur,
                                            const void* Y_prev, int64_t ldr, double alpha, double c, double beta,
                                            int32_t out_type, void* Y_next, int64_t ldr_next, void* stream) {
  if (n < 0 || b < 0 || !row_ptr || !col_idx || !values || !Y_cur || !Y_next) return RR_ERR_ARG;
  if (ytype != RR_BF16 && ytype != RR_F32 && ytype != RR_F64) return RR_ERR_ARG;
  if (out_type != RR_BF16 && out_type != RR_F32 && out_type != RR_F64) return RR_ERR_ARG;
  const int64_t ys = (int64_t)dtype_size(ytype), os = (int64_t)dtype_size(out_type);
  const int64_t V = 16 / ys, bp = (b + V - 1) / V * V;
  if (ldr < bp || ldr_next < bp || (ldr * ys) % 16 || (ldr_next * os) % 16) return RR_ERR_ARG;
  auto al16 = [](const void* p) { return p == nullptr || ((uintptr_t)p & 15) == 0; };
  if (!al16(Y_cur) || !al16(Y_prev) || !al16(Y_next)) return RR_ERR_ARG;
  if (n == 0 || b == 0) return RR_OK;
  return cheb_rows(as_stream(stream), n, b, row_ptr, col_idx, values, ytype, Y_cur, Y_prev, ldr, alpha, c, beta,
                   out_type, Y_next, ldr_next);
}
