// Solver-side block kernels: Ritz lift (Alg. 3 "U~ = U Y", Alg. 5 lift),
// residual blocks and norms (Sec. 5.2.2), per-column scaling of correction
// blocks, selection and output normalisation.
#include <cfloat>

#include <type_traits>

#include <algorithm>

#include "rr_common.cuh"
#include "solver_kernels.cuh"

namespace rr {

// X (n x b, TO, ld ldx) = [X +] alpha * S (n x p, TS, ld lds) * Y (p x b FP64, ld ldy)
constexpr int LBM = 64, LBN = 64, LBK = 16;
template <typename TS, typename TO = double, typename TA = double>
__global__ void __launch_bounds__(256) k_lift(int64_t n, int64_t b, int64_t p, const TS* __restrict__ S,
                                             int64_t lds, const double* __restrict__ Y, int64_t ldy,
                                             TO* __restrict__ X, int64_t ldx, int accum, double alpha = 1.0) {
  __shared__ TA Ss[LBK][LBM + 1];
  __shared__ TA Ys[LBK][LBN + 1];
  const int64_t m0 = (int64_t)blockIdx.x * LBM, n0 = (int64_t)blockIdx.y * LBN;
  const int tid = threadIdx.x, tm = tid % 16, tn = tid / 16;
  TA acc[4][4] = {};
  for (int64_t k0 = 0; k0 < p; k0 += LBK) {
    for (int e = tid; e < LBK * LBM; e += 256) {
      int i = e % LBM, kk = e / LBM;
      int64_t gi = m0 + i, gk = k0 + kk;
      Ss[kk][i] = (gi < n && gk < p) ? LdAs<TA, TS>::get(S + gi + gk * lds) : TA(0);
    }
    for (int e = tid; e < LBK * LBN; e += 256) {
      int kk = e % LBK, j = e / LBK;
      int64_t gk = k0 + kk, gj = n0 + j;
      Ys[kk][j] = (gk < p && gj < b) ? LdAs<TA, double>::get(Y + gk + gj * ldy) : TA(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < LBK; ++kk) {
      TA a[4], c[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = Ss[kk][tm + 16 * r];
#pragma unroll
      for (int q = 0; q < 4; ++q) c[q] = Ys[kk][tn + 16 * q];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = fma(a[r], c[q], acc[r][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int64_t j = n0 + tn + 16 * q;
    if (j >= b) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int64_t i = m0 + tm + 16 * r;
      if (i >= n) continue;
      if constexpr (std::is_same<TA, float>::value && std::is_same<TO, float>::value) {
        // FP32 result of an FP32 product (alpha = +-1, exact in FP32): one
        // rounding, as through FP64, without FP64 instructions
        const float v = fmaf((float)alpha, acc[r][q], accum ? (float)X[i + j * ldx] : 0.f);
        X[i + j * ldx] = (TO)v;
      } else {
        double v = alpha * (double)acc[r][q];
        if (accum) v += (double)X[i + j * ldx];
        X[i + j * ldx] = (TO)v;
      }
    }
  }
}

// T (n x b, FP32) -= X (n x p, FP32) K (p x b, FP64 read as FP32), FP32
// accumulation: a CTA takes 128 rows x 64 columns of T, 8 x 4
// outputs per thread, the p dimension in steps of 32 staged in shared memory
// (X rows contiguous per column, K columns contiguous per row) so a thread's
// operands are three 16-byte loads per 32 FMAs.
constexpr int kSL_M = 128, kSL_N = 64, kSL_K = 32;
__global__ void __launch_bounds__(256) k_sub_lowrank32(int64_t n, int64_t b, int64_t p, const float* __restrict__ X,
                                                       int64_t ldx, const double* __restrict__ K, int64_t ldk,
                                                       float* __restrict__ T, int64_t ldt) {
  __shared__ __align__(16) float Xs[kSL_K][kSL_M];
  __shared__ __align__(16) float Ks[kSL_K][kSL_N + 4];  // padded: see k_gram32
  const int64_t m0 = (int64_t)blockIdx.x * kSL_M, n0 = (int64_t)blockIdx.y * kSL_N;
  const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4;  // rows 8 ti.., columns 4 tj..
  float acc[8][4] = {};
  for (int64_t k0 = 0; k0 < p; k0 += kSL_K) {
    for (int e = tid; e < kSL_K * kSL_M; e += 256) {
      const int r = e % kSL_M, kk = e / kSL_M;
      Xs[kk][r] = (m0 + r < n && k0 + kk < p) ? X[(m0 + r) + (k0 + kk) * ldx] : 0.f;
    }
    for (int e = tid; e < kSL_K * kSL_N; e += 256) {
      const int kk = e % kSL_K, c = e / kSL_K;
      Ks[kk][c] = (k0 + kk < p && n0 + c < b) ? (float)K[(k0 + kk) + (n0 + c) * ldk] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kSL_K; ++kk) {
      const float4 x0 = reinterpret_cast<const float4*>(&Xs[kk][0])[2 * ti];
      const float4 x1 = reinterpret_cast<const float4*>(&Xs[kk][0])[2 * ti + 1];
      const float4 kv = reinterpret_cast<const float4*>(&Ks[kk][0])[tj];
      const float xa[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const float ka[4] = {kv.x, kv.y, kv.z, kv.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(xa[a], ka[c], acc[a][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int64_t j = n0 + 4 * tj + c;
    if (j >= b) continue;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t i = m0 + 8 * ti + a;
      if (i < n) T[i + j * ldt] -= acc[a][c];
    }
  }
}

// The same update for narrow T (b <= 16 CT): K (p x b) stays in shared memory
// (FP32, row stride 16 CT + 2), and a persistent CTA walks tiles of 128 rows
// holding all b columns, so X is read once.  Thread (ti, tj) owns rows
// ti + 16 a (a < 8) and columns CT tj .. CT tj + CT - 1: the shared X loads are
// conflict-free and each T store of a warp covers 16 consecutive rows.  The p
// dimension goes in steps of 32, the next step's X loads issued before the
// current step is used; the tile of T itself is copied to shared memory by
// asynchronous 4-byte copies issued with the tile's first step, so the
// epilogue's read of T does not wait on HBM.  The FMAs are issued as packed
// FP32 pairs over the columns (each component rounded as one fmaf).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 4 : 0;  // 0: fill with zeros, nothing read
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr int kSLF_M = 128, kSLF_K = 32;
template <int CT>
__global__ void __launch_bounds__(256, 1) k_sub_lowrank32_full(int64_t n, int b, int p, const float* __restrict__ X,
                                                               int64_t ldx, const double* __restrict__ K, int64_t ldk,
                                                               float* __restrict__ T, int64_t ldt) {
  constexpr int TB = 16 * CT, KS = TB + 2;
  extern __shared__ __align__(16) float sm_slf[];
  float* Ks = sm_slf;                                        // [p][KS]
  float* Xs = Ks + (((size_t)p * KS + 3) & ~(size_t)3);      // [kSLF_K][kSLF_M]
  float* Ts = Xs + kSLF_K * kSLF_M;                          // [b][kSLF_M]
  const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4;
  for (int e = tid; e < p * TB; e += 256) {
    const int kk = e % p, c = e / p;
    Ks[kk * KS + c] = c < b ? (float)K[kk + (int64_t)c * ldk] : 0.f;
  }
  const int64_t tiles = (n + kSLF_M - 1) / kSLF_M;
  const int ksteps = (p + kSLF_K - 1) / kSLF_K;
  constexpr int PER = kSLF_K * kSLF_M / 256;
  float xr[PER];
  auto fetch = [&](int64_t tile, int step) {
    const int64_t m0 = tile * kSLF_M;
    const int k0 = step * kSLF_K;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + 256 * u, r = e % kSLF_M, kk = e / kSLF_M;
      xr[u] = (m0 + r < n && k0 + kk < p) ? X[(m0 + r) + (int64_t)(k0 + kk) * ldx] : 0.f;
    }
  };
  int64_t tile = blockIdx.x;
  if (tile < tiles) fetch(tile, 0);
  for (; tile < tiles; tile += gridDim.x) {
    const int64_t m0 = tile * kSLF_M;
    static_assert(CT % 2 == 0, "column pairs");
    float2 acc[8][CT / 2];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < CT / 2; ++c) acc[a][c] = make_float2(0.f, 0.f);
    for (int step = 0; step < ksteps; ++step) {
      __syncthreads();
#pragma unroll
      for (int u = 0; u < PER; ++u) Xs[tid + 256 * u] = xr[u];  // e = kk * M + r
      if (step == 0) {
        // every thread is past the previous tile's epilogue: refill Ts
        for (int e = tid; e < b * kSLF_M; e += 256) {
          const int r = e % kSLF_M, c = e / kSLF_M;
          const bool in = m0 + r < n;
          cp_async4(Ts + e, in ? T + (m0 + r) + (int64_t)c * ldt : T, in);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
      }
      __syncthreads();
      if (step + 1 < ksteps)
        fetch(tile, step + 1);
      else if (tile + gridDim.x < tiles)
        fetch(tile + gridDim.x, 0);
      const int k0 = step * kSLF_K, kn = p - k0 < kSLF_K ? p - k0 : kSLF_K;
#pragma unroll 2
      for (int kk = 0; kk < kn; ++kk) {
        float xa[8];
        float2 ka[CT / 2];
#pragma unroll
        for (int a = 0; a < 8; ++a) xa[a] = Xs[kk * kSLF_M + ti + 16 * a];
        const float* kr = Ks + (size_t)(k0 + kk) * KS + CT * tj;
#pragma unroll
        for (int c = 0; c < CT / 2; ++c) ka[c] = *reinterpret_cast<const float2*>(kr + 2 * c);
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const float2 xx = make_float2(xa[a], xa[a]);
#pragma unroll
          for (int c = 0; c < CT / 2; ++c) acc[a][c] = __ffma2_rn(xx, ka[c], acc[a][c]);
        }
      }
    }
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CT; ++c) {
      const int j = CT * tj + c;
      if (j >= b) continue;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int64_t i = m0 + ti + 16 * a;
        if (i < n) T[i + j * ldt] = Ts[j * kSLF_M + ti + 16 * a] - ((c & 1) ? acc[a][c >> 1].y : acc[a][c >> 1].x);
      }
    }
  }
}

template <int CT>
static rr_status launch_sub_lowrank32_full(cudaStream_t s, int64_t n, int64_t b, int64_t p, const float* X,
                                           int64_t ldx, const double* K, int64_t ldk, float* T, int64_t ldt) {
  const size_t smem =
      ((((size_t)p * (16 * CT + 2) + 3) & ~(size_t)3) + (size_t)kSLF_K * kSLF_M + (size_t)b * kSLF_M) * sizeof(float);
  RR_CUDA(cudaFuncSetAttribute(k_sub_lowrank32_full<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t tiles = (n + kSLF_M - 1) / kSLF_M;
  const int64_t grid = tiles < num_sms() ? tiles : num_sms();
  k_sub_lowrank32_full<CT><<<(unsigned)grid, 256, smem, s>>>(n, (int)b, (int)p, X, ldx, K, ldk, T, ldt);
  return check_launch("sub_lowrank_f32 full");
}

rr_status sub_lowrank_f32(cudaStream_t s, int64_t n, int64_t b, int64_t p, const float* X, int64_t ldx,
                          const double* K, int64_t ldk, float* T, int64_t ldt) {
  if (n == 0 || b == 0 || p == 0) return RR_OK;
  if (b <= 160 && p <= 160 && n >= 64 * 1024) {
    if (b <= 128) return launch_sub_lowrank32_full<8>(s, n, b, p, X, ldx, K, ldk, T, ldt);
    return launch_sub_lowrank32_full<10>(s, n, b, p, X, ldx, K, ldk, T, ldt);
  }
  dim3 g((unsigned)((n + kSL_M - 1) / kSL_M), (unsigned)((b + kSL_N - 1) / kSL_N));
  k_sub_lowrank32<<<g, 256, 0, s>>>(n, b, p, X, ldx, K, ldk, T, ldt);
  return check_launch("sub_lowrank_f32");
}

// Y (n x b, FP32) = X (n x b, FP64) rounded to nearest.
__global__ void k_cast_f32(int64_t n, int64_t b, const double* __restrict__ X, int64_t ldx, float* __restrict__ Y,
                           int64_t ldy) {
  const int64_t tot = n * b;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    Y[i + j * ldy] = (float)X[i + j * ldx];
  }
}

// T (n x b, FP32, ld ldt) -= P (n x b, FP32, ld ldp)
__global__ void k_sub_block_f32(int64_t n, int64_t b, const float* __restrict__ P, int64_t ldp, float* __restrict__ T,
                                int64_t ldt) {
  const int64_t tot = n * b;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    T[i + j * ldt] -= P[i + j * ldp];
  }
}

rr_status sub_block_f32(cudaStream_t s, int64_t n, int64_t b, const float* P, int64_t ldp, float* T, int64_t ldt) {
  if (n <= 0 || b <= 0) return RR_OK;
  const int64_t want = (n * b + 255) / 256, cap = 8 * (int64_t)num_sms();
  k_sub_block_f32<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(n, b, P, ldp, T, ldt);
  return check_launch("sub_block_f32");
}

rr_status cast_f32(cudaStream_t s, int64_t n, int64_t b, const double* X, int64_t ldx, float* Y, int64_t ldy) {
  if (n == 0 || b == 0) return RR_OK;
  const int64_t want = (n * b + 255) / 256, cap = 8 * (int64_t)num_sms();
  k_cast_f32<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(n, b, X, ldx, Y, ldy);
  return check_launch("cast_f32");
}

rr_status lift(cudaStream_t s, int32_t stype, int64_t n, int64_t b, int64_t p, const void* S,
               int64_t lds, const double* Y, int64_t ldy, double* X, int64_t ldx, int accum) {
  if (n == 0 || b == 0) return RR_OK;
  if (p == 0) {
    if (!accum)
      for (int64_t j = 0; j < b; ++j) RR_CUDA(cudaMemsetAsync(X + j * ldx, 0, n * sizeof(double), s));
    return RR_OK;
  }
  dim3 g((unsigned)((n + LBM - 1) / LBM), (unsigned)((b + LBN - 1) / LBN));
  switch (stype) {
    case RR_F64: k_lift<double><<<g, 256, 0, s>>>(n, b, p, (const double*)S, lds, Y, ldy, X, ldx, accum); break;
    case RR_F32: k_lift<float><<<g, 256, 0, s>>>(n, b, p, (const float*)S, lds, Y, ldy, X, ldx, accum); break;
    case RR_BF16: k_lift<__nv_bfloat16><<<g, 256, 0, s>>>(n, b, p, (const __nv_bfloat16*)S, lds, Y, ldy, X, ldx, accum); break;
    case RR_E4M3: k_lift<e4m3b_t><<<g, 256, 0, s>>>(n, b, p, (const e4m3b_t*)S, lds, Y, ldy, X, ldx, accum); break;
    default: return RR_ERR_ARG;
  }
  return check_launch("lift");
}

// R = P - X diag(theta); ss[j] += sum_i R(i,j)^2 (one block per column)
__global__ void k_residual_block(int64_t n, const double* __restrict__ P, int64_t ldp,
                                 const double* __restrict__ X, int64_t ldx,
                                 const double* __restrict__ theta, double* __restrict__ R,
                                 int64_t ldr, double* __restrict__ ss, int accum_ss) {
  const int64_t j = blockIdx.x;
  const double t = theta[j];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double r = P[i + j * ldp] - t * X[i + j * ldx];
    R[i + j * ldr] = r;
    acc = fma(r, r, acc);
  }
  __shared__ double sm[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = (threadIdx.x < (blockDim.x >> 5)) ? sm[threadIdx.x] : 0.0;
    acc = warp_sum(acc);
    if (threadIdx.x == 0) ss[j] = (accum_ss ? ss[j] : 0.0) + acc;
  }
}

rr_status residual_block(cudaStream_t s, int64_t n, int64_t b, const double* P, int64_t ldp,
                         const double* X, int64_t ldx, const double* theta, double* R, int64_t ldr,
                         double* ss, int accum_ss) {
  if (b == 0) return RR_OK;
  k_residual_block<<<(unsigned)b, 512, 0, s>>>(n, P, ldp, X, ldx, theta, R, ldr, ss, accum_ss);
  return check_launch("residual_block");
}

// res[j] = sqrt(ss[j]) / |theta[j]|
__global__ void k_res_finish(int64_t b, const double* __restrict__ ss, const double* __restrict__ theta,
                             double* __restrict__ res) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < b) {
    double t = fabs(theta[j]);
    res[j] = t > 0 ? sqrt(ss[j]) / t : INFINITY;
  }
}

rr_status res_finish(cudaStream_t s, int64_t b, const double* ss, const double* theta, double* res) {
  k_res_finish<<<(unsigned)((b + 127) / 128), 128, 0, s>>>(b, ss, theta, res);
  return check_launch("res_finish");
}

// Column inf-norm of a block T (FP32 or FP64), then D = T / mu cast to TO.
// If coef/sig given: coef[j] *= sig[j] / mu[j] (the correction recurrence's
// injection coefficient, see solver.cu).  Zero columns: mu = 1.
// FP32 blocks take the maximum in FP32 (exact) and convert once: no FP64
// instruction per element on the low-precision path.
template <typename TI>
__global__ void k_colmax_any(int64_t n, const TI* __restrict__ T, int64_t ldt, double* __restrict__ mu) {
  const int64_t j = blockIdx.x;
  TI mt = TI(0);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mt = fmax(mt, fabs(T[i + j * ldt]));
  double m = (double)mt;
  __shared__ double sm[32];
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? sm[threadIdx.x] : 0.0;
    m = warp_max(m);
    if (threadIdx.x == 0) mu[j] = m > 0.0 ? m : 1.0;
  }
}

// Column scale 1 / mu_j formed once per CTA; an FP32 block is scaled and
// rounded in FP32 (one FP32 multiply, one rounding to TO per element).
template <typename TI, typename TO>
__global__ void k_scale_cast2(int64_t n, int64_t b, const TI* __restrict__ T, int64_t ldt,
                              const double* __restrict__ mu, TO* __restrict__ D, int64_t ldd) {
  const int64_t j = blockIdx.y;
  __shared__ TI s_sc;
  if (threadIdx.x == 0) s_sc = (TI)(1.0 / mu[j]);
  __syncthreads();
  const TI sc = s_sc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (std::is_same<TI, float>::value) D[i + j * ldd] = from_f32<TO>(T[i + j * ldt] * sc);
    else D[i + j * ldd] = from_f64<TO>(T[i + j * ldt] * sc);
  }
}

__global__ void k_coef_update(int64_t b, const double* __restrict__ mu, const double* __restrict__ sig,
                              double* __restrict__ coef) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < b) coef[j] = coef[j] * sig[j] / mu[j];
}

template <typename TI>
static rr_status scale_cast_t(cudaStream_t s, int64_t n, int64_t b, const TI* T, int64_t ldt,
                              double* mu, int32_t dtype, void* D, int64_t ldd) {
  k_colmax_any<TI><<<(unsigned)b, 512, 0, s>>>(n, T, ldt, mu);
  dim3 g((unsigned)std::min<int64_t>((n + 255) / 256, 512), (unsigned)b);
  switch (dtype) {
    case RR_F64: k_scale_cast2<TI, double><<<g, 256, 0, s>>>(n, b, T, ldt, mu, (double*)D, ldd); break;
    case RR_F32: k_scale_cast2<TI, float><<<g, 256, 0, s>>>(n, b, T, ldt, mu, (float*)D, ldd); break;
    case RR_BF16: k_scale_cast2<TI, __nv_bfloat16><<<g, 256, 0, s>>>(n, b, T, ldt, mu, (__nv_bfloat16*)D, ldd); break;
    case RR_E4M3: k_scale_cast2<TI, e4m3b_t><<<g, 256, 0, s>>>(n, b, T, ldt, mu, (e4m3b_t*)D, ldd); break;
    default: return RR_ERR_ARG;
  }
  note_launches(1);
  return check_launch("scale_cast");
}

// D_hi + D_lo = T(:, j) / mu_j to 16 bits: D_hi = bf16(v), D_lo = bf16(v - D_hi)
template <typename TI>
__global__ void k_scale_split(int64_t n, int64_t b, const TI* __restrict__ T, int64_t ldt,
                              const double* __restrict__ mu, __nv_bfloat16* __restrict__ Dh,
                              __nv_bfloat16* __restrict__ Dl, int64_t ldd) {
  const int64_t j = blockIdx.y;
  __shared__ TI s_sc;
  if (threadIdx.x == 0) s_sc = (TI)(mu ? 1.0 / mu[j] : 1.0);
  __syncthreads();
  const TI sc = s_sc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const TI v = T[i + j * ldt] * sc;
    if constexpr (std::is_same<TI, float>::value) {
      // FP32 split: v - hi is exact in FP32 (hi is v rounded to 8 bits)
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      Dh[i + j * ldd] = h;
      Dl[i + j * ldd] = __float2bfloat16_rn(v - __bfloat162float(h));
    } else {
      const __nv_bfloat16 h = __double2bfloat16(v);
      Dh[i + j * ldd] = h;
      Dl[i + j * ldd] = __double2bfloat16(v - (double)__bfloat162float(h));
    }
  }
}

rr_status scale_split(cudaStream_t s, int32_t ttype, int64_t n, int64_t b, const void* T, int64_t ldt,
                      double* mu, void* D_hi, void* D_lo, int64_t ldd, double* coef, const double* sig) {
  if (b == 0) return RR_OK;
  dim3 g((unsigned)std::min<int64_t>((n + 255) / 256, 512), (unsigned)b);
  if (ttype == RR_F64) {
    if (mu) k_colmax_any<double><<<(unsigned)b, 512, 0, s>>>(n, (const double*)T, ldt, mu);
    k_scale_split<double><<<g, 256, 0, s>>>(n, b, (const double*)T, ldt, mu, (__nv_bfloat16*)D_hi,
                                            (__nv_bfloat16*)D_lo, ldd);
  } else {
    if (mu) k_colmax_any<float><<<(unsigned)b, 512, 0, s>>>(n, (const float*)T, ldt, mu);
    k_scale_split<float><<<g, 256, 0, s>>>(n, b, (const float*)T, ldt, mu, (__nv_bfloat16*)D_hi,
                                           (__nv_bfloat16*)D_lo, ldd);
  }
  note_launches(mu ? 1 : 0);
  RR_TRY(check_launch("scale_split"));
  if (coef && mu) {
    k_coef_update<<<(unsigned)((b + 127) / 128), 128, 0, s>>>(b, mu, sig, coef);
    return check_launch("coef_update");
  }
  return RR_OK;
}

rr_status scale_cast(cudaStream_t s, int32_t ttype, int64_t n, int64_t b, const void* T, int64_t ldt,
                     double* mu, int32_t dtype, void* D, int64_t ldd, double* coef,
                     const double* sig) {
  if (b == 0) return RR_OK;
  rr_status st = ttype == RR_F64
                     ? scale_cast_t<double>(s, n, b, (const double*)T, ldt, mu, dtype, D, ldd)
                     : scale_cast_t<float>(s, n, b, (const float*)T, ldt, mu, dtype, D, ldd);
  if (st != RR_OK) return st;
  if (coef) {
    k_coef_update<<<(unsigned)((b + 127) / 128), 128, 0, s>>>(b, mu, sig, coef);
    return check_launch("coef_update");
  }
  return RR_OK;
}

// dst (q x p, ld ldd) = src^T (src p x q, ld lds)
__global__ void k_transpose(int64_t p, int64_t q, const double* __restrict__ src, int64_t lds,
                            double* __restrict__ dst, int64_t ldd) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= p * q) return;
  int64_t i = e % p, j = e / p;
  dst[j + i * ldd] = src[i + j * lds];
}

rr_status transpose(cudaStream_t s, int64_t p, int64_t q, const double* src, int64_t lds, double* dst,
                    int64_t ldd) {
  if (p * q == 0) return RR_OK;
  k_transpose<<<(unsigned)((p * q + 255) / 256), 256, 0, s>>>(p, q, src, lds, dst, ldd);
  return check_launch("transpose");
}

// Select b eigenpairs from an ascending theta (NaN = dropped, last) in the
// wanted order: largest -> descending from the top valid; smallest ->
// ascending from the bottom.  Ysel(:, out) = Y(:, src).
__global__ void k_select_eig(int64_t nb, int64_t b, int which, const double* __restrict__ theta,
                             const double* __restrict__ Y, int64_t ldy, double* __restrict__ tsel,
                             double* __restrict__ Ysel, int64_t ldys, int* __restrict__ nsel) {
  __shared__ int s_nv;
  if (threadIdx.x == 0) {
    int nv = 0;
    for (int64_t i = 0; i < nb; ++i) nv += !isnan(theta[i]);
    s_nv = nv;
    if (nsel) *nsel = nv < b ? nv : (int)b;
  }
  __syncthreads();
  const int64_t nv = s_nv;
  for (int64_t e = threadIdx.x + blockIdx.x * (int64_t)blockDim.x; e < nb * b;
       e += (int64_t)blockDim.x * gridDim.x) {
    int64_t i = e % nb, out = e / nb;
    double v = 0.0;
    if (out < nv) {
      int64_t src = which == RR_LARGEST ? nv - 1 - out : out;
      v = Y[i + src * ldy];
    }
    Ysel[i + out * ldys] = v;
  }
  if (blockIdx.x == 0)
    for (int64_t out = threadIdx.x; out < b; out += blockDim.x) {
      int64_t src = which == RR_LARGEST ? nv - 1 - out : out;
      tsel[out] = out < nv ? theta[src] : nan("");
    }
}

rr_status select_eig(cudaStream_t s, int64_t nb, int64_t b, int which, const double* theta,
                     const double* Y, int64_t ldy, double* tsel, double* Ysel, int64_t ldys) {
  k_select_eig<<<1, 1024, 0, s>>>(nb, b, which, theta, Y, ldy, tsel, Ysel, ldys, nullptr);
  return check_launch("select_eig");
}

// Normalise columns to unit 2-norm and fix the sign so the largest-|.| entry
// (first on ties) of X's column is positive; the same sign flips U's column.
// One block per column.
__global__ void k_normalize_sign(int64_t n, double* __restrict__ X, int64_t ldx, int64_t m,
                                 double* __restrict__ U, int64_t ldu) {
  const int64_t j = blockIdx.x;
  double* x = X + j * ldx;
  double ss = 0.0, bv = -1.0;
  int64_t bi = INT64_MAX;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double v = x[i];
    ss = fma(v, v, ss);
    if (fabs(v) > bv) {
      bv = fabs(v);
      bi = i;
    }
  }
  __shared__ double s_ss[32], s_bv[32];
  __shared__ int64_t s_bi[32];
  __shared__ double s_scale;
  for (int o = 16; o > 0; o >>= 1) {
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
    double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    s_ss[threadIdx.x >> 5] = ss;
    s_bv[threadIdx.x >> 5] = bv;
    s_bi[threadIdx.x >> 5] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, v = -1.0;
    int64_t id = INT64_MAX;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t += s_ss[w];
      if (s_bv[w] > v || (s_bv[w] == v && s_bi[w] < id)) {
        v = s_bv[w];
        id = s_bi[w];
      }
    }
    double nr = sqrt(t);
    double sg = (id != INT64_MAX && x[id] < 0) ? -1.0 : 1.0;
    s_scale = nr > 0 ? sg / nr : 1.0;
  }
  __syncthreads();
  const double sc = s_scale;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] *= sc;
  if (U) {
    // U's column: same sign, its own norm
    double* u = U + j * ldu;
    double us = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) us = fma(u[i], u[i], us);
    __shared__ double s_us[32];
    us = warp_sum(us);
    if ((threadIdx.x & 31) == 0) s_us[threadIdx.x >> 5] = us;
    __syncthreads();
    __shared__ double s_uscale;
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_us[w];
      double nr = sqrt(t);
      s_uscale = nr > 0 ? (sc > 0 ? 1.0 : -1.0) / nr : 1.0;
    }
    __syncthreads();
    const double us2 = s_uscale;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) u[i] *= us2;
  }
}

rr_status normalize_sign(cudaStream_t s, int64_t n, int64_t k, double* X, int64_t ldx, int64_t m,
                         double* U, int64_t ldu) {
  if (k == 0) return RR_OK;
  k_normalize_sign<<<(unsigned)k, 512, 0, s>>>(n, X, ldx, m, U, ldu);
  return check_launch("normalize_sign");
}

// d[j] = a[j] * b[j] (or copy if b == NULL)
__global__ void k_vec_mul(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                          double* __restrict__ d) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) d[j] = b ? a[j] * b[j] : a[j];
}

rr_status vec_mul(cudaStream_t s, int64_t n, const double* a, const double* b, double* d) {
  if (n == 0) return RR_OK;
  k_vec_mul<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, a, b, d);
  return check_launch("vec_mul");
}

// Y(:, j) += c_j^pw X(:, j) (n x b, FP64; pw = 1 or 2): the residual blocks'
// injection terms of the FP64 correction sweep
__global__ void k_add_cols_scaled(int64_t n, int64_t b, const double* __restrict__ X, int64_t ldx,
                                  const double* __restrict__ c, int pw, double* __restrict__ Y, int64_t ldy) {
  const int64_t j = blockIdx.y;
  const double cj = pw == 2 ? c[j] * c[j] : c[j];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Y[i + j * ldy] += cj * X[i + j * ldx];
}

rr_status add_cols_scaled(cudaStream_t s, int64_t n, int64_t b, const double* X, int64_t ldx, const double* c, int pw,
                          double* Y, int64_t ldy) {
  if (n <= 0 || b <= 0) return RR_OK;
  k_add_cols_scaled<<<dim3((unsigned)std::min<int64_t>((n + 255) / 256, 256), (unsigned)b), 256, 0, s>>>(
      n, b, X, ldx, c, pw, Y, ldy);
  return check_launch("add_cols_scaled");
}

// Y (2b x b, ld ldy) = [I; -K]: the coefficients that take [T, X] to
// T - X K (the projection of a block against an orthonormal X by the lift)
__global__ void k_eye_neg(int64_t b, const double* __restrict__ K, int64_t ldk, double* __restrict__ Y, int64_t ldy) {
  const int64_t j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * b; i += (int64_t)gridDim.x * blockDim.x)
    Y[i + j * ldy] = i < b ? (i == j ? 1.0 : 0.0) : -K[(i - b) + j * ldk];
}

rr_status eye_neg(cudaStream_t s, int64_t b, const double* K, int64_t ldk, double* Y, int64_t ldy) {
  if (b <= 0) return RR_OK;
  k_eye_neg<<<dim3((unsigned)((2 * b + 127) / 128), (unsigned)b), 128, 0, s>>>(b, K, ldk, Y, ldy);
  return check_launch("eye_neg");
}

__global__ void k_fill(int64_t n, double v, double* __restrict__ d) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) d[j] = v;
}

// Batched solves run a fixed number of sweeps inside one graph: a problem
// whose k wanted residuals all reached tol is frozen (the flag only rises),
// and every later lift is replaced by the frozen Ritz vectors and values.
__global__ void k_freeze(int64_t k, const double* __restrict__ res, double tol, int* __restrict__ frozen) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x)
    if (!(res[i] <= tol)) bad = 1;  // NaN fails the test
  __syncthreads();
  if (threadIdx.x == 0 && !bad) *frozen = 1;
}

__global__ void k_keep_frozen(const int* __restrict__ frozen, int64_t m, int64_t n, int64_t b,
                              const double* __restrict__ U, double* __restrict__ U2, const double* __restrict__ V,
                              double* __restrict__ V2, const double* __restrict__ sig, double* __restrict__ sig2) {
  if (!*frozen) return;
  const int64_t nu = m * b, nv = n * b, tot = nu + nv + b;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nu) U2[e] = U[e];
    else if (e < nu + nv) V2[e - nu] = V[e - nu];
    else sig2[e - nu - nv] = sig[e - nu - nv];
  }
}

rr_status freeze_update(cudaStream_t s, int64_t k, const double* res, double tol, int* frozen) {
  k_freeze<<<1, 128, 0, s>>>(k, res, tol, frozen);
  return check_launch("freeze_update");
}

rr_status keep_frozen(cudaStream_t s, const int* frozen, int64_t m, int64_t n, int64_t b, const double* U, double* U2,
                      const double* V, double* V2, const double* sig, double* sig2) {
  const int64_t tot = (m + n) * b + b;
  k_keep_frozen<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 1024), 256, 0, s>>>(frozen, m, n, b, U, U2, V, V2,
                                                                                   sig, sig2);
  return check_launch("keep_frozen");
}

// Device-side loop control of the batched solver: each problem's sweeps run
// as the body of a WHILE node of the captured graph, and this one-thread
// kernel, at the end of every body (and once before the node), sets the
// node's condition.  ctl[0] = the frozen flag (k_freeze), ctl[1] = sweeps
// done, ctl[2] = FP64 polish sweeps done, ctl[4..5] = the previous sweep's
// largest wanted residual (a double); (inc, inc_polish) are added to the
// counts first.  Another sweep runs while the problem is not frozen, fewer
// than max_sweeps sweeps are done and, when stop_at >= 0, fewer than
// stop_at.  With stall != 0 the loop also ends when the largest of the k
// residuals res[0..k) is above 0.3 times the previous one (the correction
// sweeps stopped contracting; the FP64 polish takes over); res == nullptr
// (before the first sweep of a loop) only records the residual.
__global__ void k_loop_ctl(cudaGraphConditionalHandle h, int* __restrict__ ctl, int inc, int inc_polish,
                           int max_sweeps, int stop_at, const double* __restrict__ res, int k, int stall) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int sw = ctl[1] + inc;
  ctl[1] = sw;
  ctl[2] += inc_polish;
  double* prev = reinterpret_cast<double*>(ctl + 4);
  bool stalled = false;
  if (res) {
    double mx = 0.0;
    for (int i = 0; i < k; ++i) mx = fmax(mx, res[i]);  // a NaN residual is skipped by fmax
    stalled = stall != 0 && mx > 0.3 * *prev;
    *prev = mx;
  }
  const bool go = ctl[0] == 0 && sw < max_sweeps && (stop_at < 0 || sw < stop_at) && !stalled;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

rr_status loop_ctl(cudaStream_t s, cudaGraphConditionalHandle h, int* ctl, int inc, int inc_polish, int max_sweeps,
                   int stop_at, const double* res, int k, int stall) {
  k_loop_ctl<<<1, 32, 0, s>>>(h, ctl, inc, inc_polish, max_sweeps, stop_at, res, k, stall);
  return check_launch("loop_ctl");
}

rr_status fill(cudaStream_t s, int64_t n, double v, double* d) {
  if (n == 0) return RR_OK;
  k_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, v, d);
  return check_launch("fill");
}

// Counter-based U(0,1) start block: splitmix64 of (seed, index), top 53 bits.
__global__ void k_uniform(int64_t n, int64_t b, uint64_t seed, double* __restrict__ V, int64_t ldv) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * b;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed * 0x9E3779B97F4A7C15ull + (uint64_t)e + 1;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    int64_t i = e % n, j = e / n;
    V[i + j * ldv] = (double)(z >> 11) * 0x1.0p-53;
  }
}

rr_status uniform_block(cudaStream_t s, int64_t n, int64_t b, uint64_t seed, double* V, int64_t ldv) {
  k_uniform<<<256, 256, 0, s>>>(n, b, seed, V, ldv);
  return check_launch("uniform_block");
}

}  // namespace rr

namespace rr {
__global__ void k_vec_scale(int64_t n, double alpha, const double* __restrict__ a, double* __restrict__ d) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) d[j] = alpha * a[j];
}
rr_status vec_scale(cudaStream_t s, int64_t n, double alpha, const double* a, double* d) {
  if (n == 0) return RR_OK;
  k_vec_scale<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, alpha, a, d);
  return check_launch("vec_scale");
}
}  // namespace rr

// ---------------------------------------------------------------------------
// Non-finite operator entries (an operator with a NaN or infinity makes every
// later quantity NaN): one read of the values, *flag set to 1 if any entry
// has the all-ones exponent.  Dense: one CTA per column (grid-stride),
// threads over rows; CSR: grid-stride over the nnz values.
// ---------------------------------------------------------------------------
namespace rr {
__global__ void k_nonfinite_dense(int64_t m, int64_t n, const double* __restrict__ A, int64_t lda,
                                  int* __restrict__ flag) {
  int bad = 0;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x)
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
      const unsigned long long u = (unsigned long long)__double_as_longlong(A[i + j * lda]);
      bad |= ((u >> 52) & 0x7FFull) == 0x7FFull;
    }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}
__global__ void k_nonfinite_f32(int64_t cnt, const float* __restrict__ v, int* __restrict__ flag) {
  int bad = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
    bad |= ((__float_as_uint(v[e]) >> 23) & 0xFFu) == 0xFFu;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}
rr_status operator_nonfinite(cudaStream_t s, int kind, int64_t m, int64_t n, const void* values, int64_t lda,
                             int64_t nnz, int* flag) {
  if (kind == RR_DENSE) {
    const unsigned g = (unsigned)std::min<int64_t>(n, 8 * (int64_t)num_sms());
    if (g == 0) return RR_OK;
    k_nonfinite_dense<<<g, 256, 0, s>>>(m, n, (const double*)values, lda, flag);
  } else {
    if (nnz <= 0) return RR_OK;
    const unsigned g = (unsigned)std::min<int64_t>((nnz + 255) / 256, 8 * (int64_t)num_sms());
    k_nonfinite_f32<<<g, 256, 0, s>>>(nnz, (const float*)values, flag);
  }
  return check_launch("operator_nonfinite");
}
}  // namespace rr
