// Sparse operator stages: CSR block product (Sec. 5.1 uses CSR for sparse
// operators) and the fused scaled-Chebyshev filter step (the chebfsi filter
// the paper cites in Sec. 2), one warp per row.
#include <cfloat>

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
// row's own Y_cur(i, j) is not loaded again; eight columns per iteration give
// eight independent sums and more loads in flight.
template <typename TY, typename TO>
__global__ void __launch_bounds__(256) k_csr_cheb(
    int64_t n, int64_t b, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const float* __restrict__ va, const TY* __restrict__ Yc, const TY* __restrict__ Yp, int64_t ld,
    double alpha, double cshift, double beta, const double* __restrict__ bc,
    const double* __restrict__ R, int64_t ldr, const double* __restrict__ gam, TO* __restrict__ Yn,
    int64_t ldn) {
  using A = typename AccT<TY>::type;
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
      vae[t] -= (A)cshift;
      diag = true;
    }
  }
  const A shift = diag ? A(0) : (A)cshift;  // no diagonal among the first entries
  const A al = (A)alpha;
  int64_t j = 0;
  constexpr int kC = 8;  // columns per iteration
  for (; j + kC <= b; j += kC) {
    A acc[kC];
#pragma unroll
    for (int u = 0; u < kC; ++u) acc[u] = A(0);
#pragma unroll
    for (int t = 0; t < kRowE; ++t)
      if (t < ne) {
#pragma unroll
        for (int u = 0; u < kC; ++u) acc[u] += vae[t] * ld_acc<A>(Yc + (j + u) * ld + cie[t]);
      }
    for (int e = e0 + kRowE; e < e1; ++e) {
      const A ve = (A)va[e];
#pragma unroll
      for (int u = 0; u < kC; ++u) acc[u] += ve * ld_acc<A>(Yc + (j + u) * ld + ci[e]);
    }
#pragma unroll
    for (int u = 0; u < kC; ++u) {
      const int64_t jj = j + u;
      A a = acc[u];
      if (!diag) a -= shift * ld_acc<A>(Yc + jj * ld + row);
      A v = al * a;
      if (Yp) v -= (A)(beta * (bc ? bc[jj] : 1.0)) * ld_acc<A>(Yp + row + jj * ld);
      if (R && gam) v += (A)gam[jj] * ld_acc<A>(R + row + jj * ldr);
      Yn[row + jj * ldn] = st_cvt<TO, A>(v);
    }
  }
  for (; j < b; ++j) {
    const TY* yc = Yc + j * ld;
    A acc = A(0);
#pragma unroll
    for (int t = 0; t < kRowE; ++t)
      if (t < ne) acc += vae[t] * ld_acc<A>(yc + cie[t]);
    for (int e = e0 + kRowE; e < e1; ++e) acc += (A)va[e] * ld_acc<A>(yc + ci[e]);
    if (!diag) acc -= shift * ld_acc<A>(yc + row);
    A v = al * acc;
    if (Yp) v -= (A)(beta * (bc ? bc[j] : 1.0)) * ld_acc<A>(Yp + row + j * ld);
    if (R && gam) v += (A)gam[j] * ld_acc<A>(R + row + j * ldr);
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
  switch (out_type) {
    case RR_F64: k_csr_cheb<TY, double><<<g, 256, 0, s>>>(n, b, rp, ci, va, Yc, Yp, ld, alpha, c, beta, bc, R, ldr, gam, (double*)Yn, ldn); break;
    case RR_F32: k_csr_cheb<TY, float><<<g, 256, 0, s>>>(n, b, rp, ci, va, Yc, Yp, ld, alpha, c, beta, bc, R, ldr, gam, (float*)Yn, ldn); break;
    case RR_BF16: k_csr_cheb<TY, __nv_bfloat16><<<g, 256, 0, s>>>(n, b, rp, ci, va, Yc, Yp, ld, alpha, c, beta, bc, R, ldr, gam, (__nv_bfloat16*)Yn, ldn); break;
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
