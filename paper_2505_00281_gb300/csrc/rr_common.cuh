// Shared device helpers: status, bounded grid barrier, reductions, casts.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>
#include <math.h>

#include "../../include/rr.h"

namespace rr {

// ---------------------------------------------------------------------------
// host-side status plumbing
// ---------------------------------------------------------------------------
void set_last_error(const char* what, cudaError_t e);
rr_status check_launch(const char* what);  // counts one launch
void note_launches(int n);                  // counts n further launches

#define RR_TRY(expr)                                   \
  do {                                                 \
    rr_status _s = (expr);                             \
    if (_s != RR_OK) return _s;                        \
  } while (0)

#define RR_CUDA(expr)                                  \
  do {                                                 \
    cudaError_t _e = (expr);                           \
    if (_e != cudaSuccess) {                           \
      ::rr::set_last_error(#expr, _e);                 \
      return RR_ERR_CUDA;                              \
    }                                                  \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int num_sms();

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Upper bound on any single device-side wait (2 s): after it the waiting
// thread records RR_ERR_TIMEOUT in *err and the kernel returns early.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};

// Grid-wide barrier for cooperative launches, with a bounded wait (limit_ns,
// kWaitLimitNs unless a self-test passes a shorter one).
// Returns false (and all later calls return false at once) when *err is set.
__device__ __forceinline__ bool grid_barrier(GridBarrier* gb, unsigned nblocks, int* err,
                                             uint64_t limit_ns = kWaitLimitNs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &gb->gen;
    volatile int* verr = err;
    if (*verr == 0) {
      unsigned int g = *vgen;
      __threadfence();
      unsigned int prev = atomicAdd(&gb->count, 1u);
      if (prev == nblocks - 1) {
        atomicExch(&gb->count, 0u);
        __threadfence();
        atomicAdd(&gb->gen, 1u);
      } else {
        uint64_t t0 = global_timer_ns();
        while (*vgen == g) {
          if (*verr != 0) break;
          if (global_timer_ns() - t0 > limit_ns) {
            atomicCAS(err, 0, (int)RR_ERR_TIMEOUT);
            break;
          }
          __nanosleep(32);
        }
      }
      __threadfence();
    }
  }
  __syncthreads();
  return *(volatile int*)err == 0;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// load/store with conversion for the basis storage types
// FP64 -> FP32, round to nearest even, on the bit pattern (the conversion
// instruction runs on the FP64 units, of which this GPU has few); values
// outside FP32's normal range (and zero, Inf, NaN) take the instruction
__device__ __forceinline__ float f64_to_f32_rn(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int E = (int)((u >> 52) & 0x7FF);
  if (E < 897 || E > 1150) return (float)d;
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  const unsigned q = (unsigned)((m + 0xFFFFFFFull + ((m >> 29) & 1ull)) >> 29);  // may carry into the exponent
  return __uint_as_float(((unsigned)(u >> 63) << 31) | (((unsigned)(E - 896) << 23) + q));
}

// FP8-E4M3 basis entry.  The stored code is e4m3_rn(256 v): Alg. 8's basis
// columns and the infinity-normalised start block have |v| <= 1, so 256 |v| <=
// 448 (the E4M3 maximum) without a per-column scale; a load returns code 2^-8.
struct e4m3b_t {
  unsigned char c;
};
__device__ __forceinline__ float e4m3b_value(unsigned char c) {
  const unsigned e = (c >> 3) & 15u, m = c & 7u;
  // normal: (1 + m/8) 2^(e - 7) 2^-8 -> FP32 exponent field e + 112; subnormal: m 2^-9 2^-8
  const float v = e ? __uint_as_float(((e + 112u) << 23) | (m << 20)) : (float)m * 7.62939453125e-06f;
  return (c & 0x80u) ? -v : v;
}
__device__ __forceinline__ e4m3b_t e4m3b_from_f32(float v) {
  return e4m3b_t{(unsigned char)__nv_cvt_float_to_fp8(v * 256.f, __NV_SATFINITE, __NV_E4M3)};
}

template <typename T> struct Ld;
template <> struct Ld<e4m3b_t> {
  static __device__ __forceinline__ double f64(const e4m3b_t* p) { return (double)e4m3b_value(p->c); }
  static __device__ __forceinline__ float f32(const e4m3b_t* p) { return e4m3b_value(p->c); }
};
template <> struct Ld<double> {
  static __device__ __forceinline__ double f64(const double* p) { return *p; }
  static __device__ __forceinline__ float f32(const double* p) { return f64_to_f32_rn(*p); }
};
template <> struct Ld<float> {
  static __device__ __forceinline__ double f64(const float* p) { return (double)*p; }
  static __device__ __forceinline__ float f32(const float* p) { return *p; }
};
template <> struct Ld<__nv_bfloat16> {
  static __device__ __forceinline__ double f64(const __nv_bfloat16* p) {
    return (double)__bfloat162float(*p);
  }
  static __device__ __forceinline__ float f32(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
  }
};

// load a stored entry as the arithmetic type TA (FP32: no FP64 instruction)
template <typename TA, typename T> struct LdAs;
template <typename T> struct LdAs<float, T> {
  static __device__ __forceinline__ float get(const T* p) { return Ld<T>::f32(p); }
};
template <typename T> struct LdAs<double, T> {
  static __device__ __forceinline__ double get(const T* p) { return Ld<T>::f64(p); }
};

template <typename T> __device__ __forceinline__ T from_f64(double v);
template <> __device__ __forceinline__ double from_f64<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_f64<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f64<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn((float)v);
}
template <> __device__ __forceinline__ e4m3b_t from_f64<e4m3b_t>(double v) { return e4m3b_from_f32(f64_to_f32_rn(v)); }
template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ e4m3b_t from_f32<e4m3b_t>(float v) { return e4m3b_from_f32(v); }
template <> __device__ __forceinline__ double from_f32<double>(float v) { return v; }
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

inline size_t dtype_size(int32_t dt) {
  switch (dt) {
    case RR_F64: return 8;
    case RR_F32: return 4;
    case RR_BF16: return 2;
    case RR_E4M3: return 1;
  }
  return 0;
}

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Simple bump allocator over the caller's workspace.
struct Arena {
  char* base;
  size_t cap;
  size_t off;
  bool overflow;
  explicit Arena(void* b, size_t c) : base((char*)b), cap(c), off(0), overflow(false) {}
  template <typename T>
  T* take(size_t count) {
    size_t bytes = align_up(count * sizeof(T));
    if (off + bytes > cap) {
      overflow = true;
      off += bytes;
      return nullptr;
    }
    T* p = (T*)(base + off);
    off += bytes;
    return p;
  }
  void* take_bytes(size_t bytes) {
    bytes = align_up(bytes);
    if (off + bytes > cap) {
      overflow = true;
      off += bytes;
      return nullptr;
    }
    void* p = base + off;
    off += bytes;
    return p;
  }
};

}  // namespace rr
