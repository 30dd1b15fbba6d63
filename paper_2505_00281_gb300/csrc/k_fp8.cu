// FP8-E4M3 operands for the low-precision block product (the FP8 option of
// the precision map, Sec. 4.2 and Fig. 4: storage below half precision with
// higher-precision accumulation).  Every row (operator) or column (basis
// block) gets a power-of-two scale 2^e, the largest with max|x| 2^e <= 448
// (the E4M3 maximum), so dequantisation is exact.  A value is quantised as
// e4m3_rn(fp32_rn(x 2^e)), round to nearest even with saturation, in two
// steps: FP64 -> FP32 on the bit pattern, then the hardware FP32 -> E4M3
// conversion.  No FP64 instruction runs per element.
#include <cuda_fp8.h>

#include "rr_common.cuh"
#include "solver_kernels.cuh"

namespace rr {

// |x| as ordered 64-bit keys (NaN excluded by the caller's data)
__device__ __forceinline__ unsigned long long abs_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// e with m 2^e <= 448 < m 2^(e+1) for the maximum m (as its key), within
// [-126, 126]; 0 for m = 0 (a subnormal maximum takes the clamp, 126)
__device__ __forceinline__ int e4m3_exp(unsigned long long key) {
  if (key == 0) return 0;
  if ((key >> 52) == 0) return 126;
  const int E = (int)(key >> 52) - 1023;
  // 448 = 1.75 2^8: e = 8 - E, minus one when the mantissa exceeds 1.75
  const int e = 8 - E - ((key & 0xFFFFFFFFFFFFFull) > 0xC000000000000ull ? 1 : 0);
  return e > 126 ? 126 : (e < -126 ? -126 : e);
}

__device__ __forceinline__ double times_pow2(double x, int e) {
  const long long b = __double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7FF);
  if (be != 0 && be + e > 0 && be + e < 2047) return __longlong_as_double(b + ((long long)e << 52));
  return x == 0.0 ? x : ldexp(x, e);
}

__device__ __forceinline__ unsigned char to_e4m3(double x, int e) {
  const float f = f64_to_f32_rn(times_pow2(x, e));
  return (unsigned char)__nv_cvt_float_to_fp8(f, __NV_SATFINITE, __NV_E4M3);
}

__device__ __forceinline__ float inv_pow2f(int e) { return __uint_as_float((unsigned)(127 - e) << 23); }

// column maxima: one CTA per column
__global__ void k_e4m3_colmax(int64_t rows, const double* __restrict__ X, int64_t ldx,
                              unsigned long long* __restrict__ key) {
  const int64_t j = blockIdx.x;
  unsigned long long m = 0;
  for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
    const unsigned long long k = abs_key(X[i + j * ldx]);
    m = k > m ? k : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  __shared__ unsigned long long sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = sm[w] > m ? sm[w] : m;
    key[j] = m > sm[0] ? m : sm[0];
  }
}

// row maxima: 32 x 32 tiles, one atomic max per row and tile (key zeroed first)
__global__ void k_e4m3_rowmax(int64_t rows, int64_t cols, const double* __restrict__ X, int64_t ldx,
                              unsigned long long* __restrict__ key) {
  const int64_t i = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * 32;
  unsigned long long m = 0;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t j = j0 + r;
    if (i < rows && j < cols) {
      const unsigned long long k = abs_key(X[i + j * ldx]);
      m = k > m ? k : m;
    }
  }
  __shared__ unsigned long long sm[8][33];
  sm[threadIdx.y][threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.y == 0) {
    for (int r = 1; r < 8; ++r) m = sm[r][threadIdx.x] > m ? sm[r][threadIdx.x] : m;
    if (m && i < rows) atomicMax(key + i, m);
  }
}

__global__ void k_e4m3_inv(int64_t count, const unsigned long long* __restrict__ key, float* __restrict__ inv) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) inv[t] = inv_pow2f(e4m3_exp(key[t]));
}

// per-column scales, column-major output
__global__ void k_e4m3_cols(int64_t rows, const double* __restrict__ X, int64_t ldx,
                            const unsigned long long* __restrict__ key, unsigned char* __restrict__ Q, int64_t ldq) {
  const int64_t j = blockIdx.y;
  const int e = e4m3_exp(key[j]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
    Q[i + j * ldq] = to_e4m3(X[i + j * ldx], e);
}

// per-row scales, row-major output (the transpose through shared memory)
__global__ void k_e4m3_rows(int64_t rows, int64_t cols, const double* __restrict__ X, int64_t ldx,
                            const unsigned long long* __restrict__ key, unsigned char* __restrict__ Q, int64_t ldq) {
  __shared__ unsigned char tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  const int64_t i = i0 + threadIdx.x;
  const int e = i < rows ? e4m3_exp(key[i]) : 0;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t j = j0 + r;
    tile[threadIdx.x][r] = (i < rows && j < cols) ? to_e4m3(X[i + j * ldx], e) : (unsigned char)0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t ii = i0 + r, j = j0 + threadIdx.x;
    if (ii < rows && j < cols) Q[ii * ldq + j] = tile[r][threadIdx.x];
  }
}

__global__ void k_fill_f32(int64_t n, float v, float* __restrict__ d) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) d[t] = v;
}

rr_status fill_f32(cudaStream_t s, int64_t n, float v, float* d) {
  if (n <= 0) return RR_OK;
  k_fill_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, v, d);
  return check_launch("fill_f32");
}

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_quantize_e4m3(int64_t rows, int64_t cols, const double* X, int64_t ldx, int32_t by_rows,
                                      void* Q, int64_t ldq, float* inv_scale, void* scratch, void* stream) {
  if (rows < 0 || cols < 0 || ldx < rows || !X || !Q || !inv_scale || !scratch) return RR_ERR_ARG;
  if (by_rows ? ldq < cols : ldq < rows) return RR_ERR_ARG;
  if (rows == 0 || cols == 0) return RR_OK;
  cudaStream_t s = as_stream(stream);
  unsigned long long* key = (unsigned long long*)scratch;
  if (by_rows) {
    RR_CUDA(cudaMemsetAsync(key, 0, rows * sizeof(unsigned long long), s));
    dim3 g((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32)), th(32, 8);
    k_e4m3_rowmax<<<g, th, 0, s>>>(rows, cols, X, ldx, key);
    k_e4m3_rows<<<g, th, 0, s>>>(rows, cols, X, ldx, key, (unsigned char*)Q, ldq);
    k_e4m3_inv<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(rows, key, inv_scale);
  } else {
    k_e4m3_colmax<<<(unsigned)cols, 256, 0, s>>>(rows, X, ldx, key);
    dim3 g((unsigned)std::min<int64_t>((rows + 255) / 256, 1024), (unsigned)cols);
    k_e4m3_cols<<<g, 256, 0, s>>>(rows, X, ldx, key, (unsigned char*)Q, ldq);
    k_e4m3_inv<<<(unsigned)((cols + 255) / 256), 256, 0, s>>>(cols, key, inv_scale);
  }
  note_launches(2);
  return check_launch("rr_quantize_e4m3");
}

extern "C" rr_status rr_gemm_e4m3(int64_t M, int64_t N, int64_t K, const void* A_k, int64_t lda,
                                  const float* a_scale, const void* B, int64_t ldb, const float* b_scale,
                                  float* C, int64_t ldc, void* stream) {
  if (M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldc < M || !C) return RR_ERR_ARG;
  if (M == 0 || N == 0) return RR_OK;
  if (!A_k || !B || !a_scale || !b_scale) return RR_ERR_ARG;
  return gemm_e4m3_tc(M, N, K, A_k, lda, a_scale, B, ldb, b_scale, C, ldc, as_stream(stream));
}
