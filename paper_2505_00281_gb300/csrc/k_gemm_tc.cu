// tcgen05 tensor-core block product for the low-precision filter (Sec. 2's
// X_iter = A X with the BF16 basis of the precision map in Sec. 4.2):
//   C (M x N, FP32, column-major) = A_k^T B  [+ coef_j R(:, j)]
// A_k: K x M BF16, K contiguous (the K-major "A" operand: rows of A for
// A V, columns of A for A^T W); B: K x N BF16, K contiguous.
//
// One CTA per 128-row tile of C and K-split, 4 warps:
//   warp 0 (one lane): TMA producer, 128B-swizzled 64-wide K slabs of A and
//                      B into an S-stage shared-memory ring (mbarrier
//                      complete_tx per stage);
//   warp 1 (one lane): issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32,
//                      M = 128, N = padded N, K = 16 per instruction) into a
//                      TMEM accumulator, tcgen05.commit frees each stage;
//   warps 0-3:        epilogue, tcgen05.ld 32x32b from TMEM (warp w owns
//                      lanes 32w..32w+31 = rows), coalesced column stores.
// K splits (small M) add their partial tiles with FP32 atomics into a C
// pre-initialised to the added term.
// FP8 variant (kF8): E4M3 x E4M3 -> FP32 (tcgen05 kind::f8f6f4, K = 32 per
// instruction), the same 128-byte swizzle rows (128 elements per K step); the
// epilogue multiplies by a per-row scale of A and a per-column scale of B.
// Every mbarrier wait is bounded (2 s); on expiry the kernel records an error
// (read by the host), stops issuing, waits (bounded) for its in-flight copies,
// frees its TMEM and returns.
#include <cuda.h>

#include "rr_common.cuh"
#include "solver_kernels.cuh"

namespace rr {

__device__ int g_tc_error = 0;

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;  // bf16 elements per 128-byte swizzle row

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on `bar` reaching `parity`; returns false on timeout (after
// recording RR_ERR_TIMEOUT in *err) or when *err is already set
__device__ __forceinline__ bool mbar_wait_on(uint64_t* bar, uint32_t parity, int* err, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (*(volatile int*)err) return false;
    if (global_timer_ns() - t0 > limit_ns) {
      atomicCAS(err, 0, (int)RR_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// the kernels' wait: the library-wide error word, 2 s limit
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  return mbar_wait_on(bar, parity, &g_tc_error, kWaitLimitNs);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// shared-memory matrix descriptor, K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SM100 descriptor format, version 1)
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_e4m3(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

template <bool kF8>
__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t accumulate) {
  if constexpr (kF8) umma_e4m3(dtmem, adesc, bdesc, idesc, accumulate);
  else umma_bf16(dtmem, adesc, bdesc, idesc, accumulate);
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace

struct TcArgs {
  int64_t M, N, K;
  int npad;        // N rounded up to 16 (UMMA N)
  int tmem_cols;   // power of two >= max(32, npad)
  int stages;
  int ksteps_per_split;
  int nk;          // K steps (K / 64 rounded up)
  int nk1;         // same (kept for the launch record)
  int segs;        // 1, or 3 for the split product: per K step A_hi B_hi + A_lo B_hi + A_hi B_lo
  float* C;
  int64_t ldc;
  const double* R;
  int64_t ldr;
  const double* coef;
  int atomic;      // 1: K-split, add into C
  const float* rscale;  // FP8: C(i, j) = rscale[i] cscale[j] acc(i, j)
  const float* cscale;
  // FP64-emulation epilogue (Ozaki-style slices, see k_f64emu.cu).  Launch z
  // multiplies A slice p0 by nq = 1 or 2 consecutive B slices q0, q0 + 1
  // (pair[z] = p0 | q0 << 8 | nq << 16, 0-based); A rows / B rows of slice s
  // start at s * a_slice_rows / s * b_slice_rows in the operands' tensor maps.
  // The exact FP32 sums v0, v1 combine into 64 v0 + v1 at the second slice's
  // scale, and element (row, col) is scaled by
  //   2^(rexp[row] + cexp[col] - 6 (p0 + 1) - 6 (q0 + nq)).
  // Output: C64 (!= nullptr) takes += (atomically under a K-split), else part
  // receives one M x nb block (ld M) per (z, split).
  double* C64;
  int64_t ldc64;
  double* part;
  const int* rexp;
  const int* cexp;
  int nb;
  int a_slice_rows, b_slice_rows;
  int npairs;
  int pair_major;  // grid (pair, split, tile) instead of (tile, split, pair)
  int lift_ksteps, lift_s;  // > 0: a lift's anti-diagonals, pair z = diagonal p0 + 2
  uint32_t pair[48];
};

// d * 2^e, exact: an exponent-field add when the result stays normal
// (ldexp otherwise: zero, subnormal or overflowing results)
__device__ __forceinline__ double mul_pow2(double d, int e) {
  const long long b = __double_as_longlong(d);
  const int be = (int)((b >> 52) & 0x7FF);
  if (be != 0 && be + e > 0 && be + e < 2047) return __longlong_as_double(b + ((long long)e << 52));
  return d == 0.0 ? d : ldexp(d, e);
}

template <bool kF8, bool kEmu>
__global__ void __launch_bounds__(128, 1) k_gemm_bf16_tc(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB,
                                                          const __grid_constant__ CUtensorMap tmA2,
                                                          const __grid_constant__ CUtensorMap tmB2,
                                                          TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t a_bytes = kBM * kBK * 2;            // 16 KB
  const uint32_t b_bytes = (uint32_t)a.npad * kBK * 2;
  // split product: a stage holds A_hi, B_hi, A_lo, B_lo of one K step
  const bool spl = a.segs > 1;
  const uint32_t stage_bytes = (a_bytes + b_bytes) * (spl ? 2 : 1);  // multiple of 1024
  uint64_t* full = (uint64_t*)(base + (size_t)a.stages * stage_bytes);
  uint64_t* empty = full + a.stages;
  uint64_t* accum = empty + a.stages;
  __shared__ uint32_t s_tmem;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // pair-major grids (x = slice pair, z = row tile) put the CTAs of one row
  // tile's slice pairs side by side, so a tile of an operator slice read by
  // several pairs comes from HBM once and from L2 for the others
  const int tile = a.pair_major ? (int)blockIdx.z : (int)blockIdx.x;
  const int zi = a.pair_major ? (int)blockIdx.x : (int)blockIdx.z;
  const int64_t m0 = (int64_t)tile * kBM;
  const int split = blockIdx.y;
  // slice pair of this launch row (FP64 emulation; 0 otherwise)
  const uint32_t pz = a.npairs > 0 ? a.pair[zi] : 0u;
  const int p0 = (int)(pz & 0xFF), q0 = (int)((pz >> 8) & 0xFF), nq = (int)((pz >> 16) & 0xFF);
  const int a_off = p0 * a.a_slice_rows, b_off = q0 * a.b_slice_rows;
  // K steps of this pair: all of K, or for a lift's anti-diagonal d = p0 + 2
  // the first (p0 + 1) lift_ksteps of A and as many of B from its step
  // (lift_s - 1 - p0) lift_ksteps
  const int nkz = a.lift_ksteps ? (p0 + 1) * a.lift_ksteps : a.nk;
  const int bk0 = a.lift_ksteps ? (a.lift_s - 1 - p0) * a.lift_ksteps : 0;
  const int ks0 = split * a.ksteps_per_split;
  int ks1 = ks0 + a.ksteps_per_split;
  if (ks1 > nkz) ks1 = nkz;
  const int nks = ks1 > ks0 ? ks1 - ks0 : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (nks > 0) {
    if (warp == 0 && lane == 0) {
      // ---------------- TMA producer ----------------
      int issued = 0;
      for (int i = 0; i < nks; ++i) {
        const int s = i % a.stages;
        if (i >= a.stages && !mbar_wait(&empty[s], ((i / a.stages) - 1) & 1)) break;
        unsigned char* sa = base + (size_t)s * stage_bytes;
        unsigned char* sb = sa + a_bytes;
        mbar_expect_tx(&full[s], stage_bytes);
        const int kx = (ks0 + i) * (kF8 ? 2 * kBK : kBK);  // elements per 128-byte row
        tma_load_2d(sa, &tmA, &full[s], kx, (int)m0 + a_off);
        tma_load_2d(sb, &tmB, &full[s], kx + bk0 * kBK, b_off);
        if (spl) {
          tma_load_2d(sb + b_bytes, &tmA2, &full[s], kx, (int)m0 + a_off);
          tma_load_2d(sb + b_bytes + a_bytes, &tmB2, &full[s], kx, b_off);
        }
        ++issued;
      }
      if (issued < nks) {
        // error: drain the copies still in flight (bounded) before leaving
        for (int i = (issued > a.stages ? issued - a.stages : 0); i < issued; ++i) {
          const int s = i % a.stages;
          const uint64_t t0 = global_timer_ns();
          while (!mbar_try_wait(&full[s], (i / a.stages) & 1) && global_timer_ns() - t0 < kWaitLimitNs) {
          }
        }
      }
    } else if (warp == 1 && lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = (1u << 4)                                  // D: FP32
                             | (kF8 ? 0u : (1u << 7) | (1u << 10))       // A, B: BF16 (kind::f16) or E4M3 (0)
                             | ((uint32_t)(a.npad >> 3) << 17)          // N / 8
                             | ((uint32_t)(kBM >> 4) << 24);            // M / 16
      for (int i = 0; i < nks; ++i) {
        const int s = i % a.stages;
        if (!mbar_wait(&full[s], (i / a.stages) & 1)) {
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = smem_u32(base + (size_t)s * stage_bytes);
        const uint32_t sb = sa + a_bytes;
        const uint64_t ad = sdesc_sw128(sa), bd = sdesc_sw128(sb);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk)  // 32 bytes of K per instruction (16 BF16 / 32 E4M3)
          umma<kF8>(tmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (i > 0 || kk > 0) ? 1u : 0u);
        if (spl) {
          // A_lo B_hi and A_hi B_lo from the same stage (each operand read once)
          const uint64_t ad2 = sdesc_sw128(sb + b_bytes), bd2 = sdesc_sw128(sb + b_bytes + a_bytes);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            umma_bf16(tmem, ad2 + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, 1u);
            umma_bf16(tmem, ad + (uint64_t)(kk * 2), bd2 + (uint64_t)(kk * 2), idesc, 1u);
          }
        }
        umma_commit(&empty[s]);
      }
      // the final commit arrives once every MMA issued above has completed,
      // also after an error, so TMEM is never freed under a running MMA
      umma_commit(accum);
    }
    // ---------------- epilogue (all 4 warps) ----------------
    __syncwarp();
    bool ready = mbar_wait(accum, 0);
    __syncwarp();
    ready = __all_sync(0xffffffffu, ready) && *(volatile int*)&g_tc_error == 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (kEmu) {
      if (ready) {
        // FP64-emulation epilogue; the 32 C loads of a chunk are issued before
        // any store (read-modify-write mode)
        const int64_t row = m0 + warp * 32 + lane;
        const bool rv = row < a.M;
        const int er = rv ? __ldg(a.rexp + row) - 6 * (p0 + 1) - 6 * (q0 + nq) : 0;
        double* __restrict__ Cr = a.C64 ? a.C64 + row
                                        : a.part + ((size_t)zi * gridDim.y + blockIdx.y) * a.M * a.nb + row;
        const int64_t ldo = a.C64 ? a.ldc64 : a.M;
        const bool rmw = a.C64 && !a.atomic;
        for (int c0 = 0; c0 < a.nb; c0 += 32) {
          uint32_t r0[32], r1[32];
          tmem_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r0);
          if (nq > 1) tmem_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a.nb + c0), r1);
          if (rv) {
            const int cnt = a.nb - c0 < 32 ? a.nb - c0 : 32;
            double cv[32];
            if (rmw) {
  #pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < cnt) cv[j] = Cr[(int64_t)(c0 + j) * ldo];
            }
  #pragma unroll
            for (int j = 0; j < 32; ++j) {
              if (j < cnt) {
                int iv = __float2int_rn(__uint_as_float(r0[j]));
                if (nq > 1) iv = iv * 64 + __float2int_rn(__uint_as_float(r1[j]));
                const double t = mul_pow2(__int2double_rn(iv), er + __ldg(a.cexp + c0 + j));
                if (rmw) cv[j] += t;
                else if (a.C64) atomicAdd(Cr + (int64_t)(c0 + j) * ldo, t);
                else Cr[(int64_t)(c0 + j) * ldo] = t;
              }
            }
            if (rmw) {
  #pragma unroll
              for (int j = 0; j < 32; ++j)
                if (j < cnt) Cr[(int64_t)(c0 + j) * ldo] = cv[j];
            }
          }
        }
      }
    } else if (ready) {
      const int64_t row = m0 + warp * 32 + lane;
      const float rs = (kF8 && row < a.M) ? __ldg(a.rscale + row) : 1.f;
      for (int c0 = 0; c0 < a.npad; c0 += 32) {
        uint32_t r[32];
        tmem_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
        if (row < a.M) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int64_t col = c0 + j;
            if (col < a.N) {
              float v = __uint_as_float(r[j]);
              if constexpr (kF8) v = v * rs * __ldg(a.cscale + col);
              float* dst = a.C + row + col * a.ldc;
              if (a.atomic) {
                atomicAdd(dst, v);
              } else {
                if (a.R) v += (float)(a.coef[col] * a.R[row + col * a.ldr]);
                *dst = v;
              }
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                 : "memory");
  }
}

// C = coef_j R(:, j) (or 0): the starting value for K-split accumulation
__global__ void k_tc_init_c(int64_t M, int64_t N, float* __restrict__ C, int64_t ldc,
                            const double* __restrict__ R, int64_t ldr, const double* __restrict__ coef) {
  const int64_t j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
    C[i + j * ldc] = R ? (float)(coef[j] * R[i + j * ldr]) : 0.f;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int& gemm_force_simt() {
  static int v = 0;
  return v;
}

static thread_local TcProf* t_tc_prof = nullptr;
void tc_prof_attach(TcProf* p) { t_tc_prof = p; }

// event pair around one launch of the product kernel (profiling only)
struct TcProfScope {
  TcProf* p;
  cudaStream_t s;
  TcProfScope(cudaStream_t s_, double bytes, double flops, int role) : p(t_tc_prof), s(s_) {
    if (!p) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    p->ev.push_back(e);
    p->role.push_back(role);
    p->bytes += bytes;
    p->role_bytes[role] += bytes;
    p->role_flops[role] += flops;
    p->launches += 1;
  }
  ~TcProfScope() {
    if (!p) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    p->ev.push_back(e);
  }
};

int& gemm_split_cap() {
  static thread_local int v = 0;
  return v;
}

// Raise the kernel's dynamic shared-memory limit once (outside any stream
// capture: rr_batch_svd calls this before it starts capturing).
rr_status tc_prepare_attributes() {
  static bool done = false;
  if (!done) {
    RR_CUDA(cudaFuncSetAttribute(k_gemm_bf16_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    RR_CUDA(cudaFuncSetAttribute(k_gemm_bf16_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    RR_CUDA(cudaFuncSetAttribute(k_gemm_bf16_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    done = true;
  }
  return RR_OK;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

bool gemm_bf16_tc_supported(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, const void* A,
                            const void* B) {
  if (M <= 0 || N <= 0 || N > 256 || K <= 0) return false;
  if (lda % 8 || ldb % 8) return false;                          // 16-byte strides
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return false;  // 16-byte aligned bases
  if (M > 0x7fffffff || K > 0x7fffffff) return false;
  return encode_fn() != nullptr;
}

static bool make_map(CUtensorMap* m, const void* base, int64_t inner, int64_t outer, int64_t ld_elems,
                     uint32_t box_inner, uint32_t box_outer, bool f8 = false) {
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)ld_elems * (f8 ? 1 : 2)};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(m, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                           const_cast<void*>(base), dims, strides,
                           box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int64_t tc_nk(int64_t K) { return (K + kBK - 1) / kBK; }

// K splits of a partial-output emulation launch: enough for exact FP32
// sums, and about one CTA per SM over tiles x pairs x splits
int tc_emu_partial_splits(int64_t M, int64_t K, int npairs, int max_kchunk) {
  const int64_t tiles = (M + kBM - 1) / kBM, nk = tc_nk(K);
  const int64_t per_max = max_kchunk / kBK;
  if (per_max < 1 || npairs < 1) return 0;
  int64_t splits = (nk + per_max - 1) / per_max;
  const int64_t want = (num_sms() + tiles * npairs - 1) / (tiles * npairs);
  if (want > splits) splits = want < nk ? want : nk;
  const int64_t per = (nk + splits - 1) / splits;
  return (int)((nk + per - 1) / per);
}

static rr_status gemm_bf16_tc_impl(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A, int64_t lda,
                                   const __nv_bfloat16* B, int64_t ldb, float* C, int64_t ldc,
                                   const double* R, int64_t ldr, const double* coef, const TcEmu* emu,
                                   cudaStream_t s, const __nv_bfloat16* A2 = nullptr,
                                   const __nv_bfloat16* B2 = nullptr);

rr_status gemm_bf16_tc(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A, int64_t lda,
                       const __nv_bfloat16* B, int64_t ldb, float* C, int64_t ldc, const double* R,
                       int64_t ldr, const double* coef, cudaStream_t s) {
  return gemm_bf16_tc_impl(M, N, K, A, lda, B, ldb, C, ldc, R, ldr, coef, nullptr, s);
}

// Split-BF16 product: C (M x N, FP32) = (A_hi + A_lo)^T (B_hi + B_lo) without
// the lo.lo term (+ coef_j R(:, j)), FP32 accumulation; each operand pair is
// the BF16 rounding of a wider value and its BF16 residual.
rr_status gemm_bf16_tc_split(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A_hi,
                             const __nv_bfloat16* A_lo, int64_t lda, const __nv_bfloat16* B_hi,
                             const __nv_bfloat16* B_lo, int64_t ldb, float* C, int64_t ldc,
                             const double* R, int64_t ldr, const double* coef, cudaStream_t s) {
  if (!A_lo || !B_lo) return RR_ERR_ARG;
  return gemm_bf16_tc_impl(M, N, K, A_hi, lda, B_hi, ldb, C, ldc, R, ldr, coef, nullptr, s, A_lo, B_lo);
}

// FP64 emulation launch (TcEmu in solver_kernels.cuh); N = nb or 2 nb
rr_status gemm_bf16_tc_emu(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A, int64_t lda,
                           const __nv_bfloat16* B, int64_t ldb, const TcEmu& e, cudaStream_t s) {
  if (e.npairs < 1 || e.npairs > 48 || (!e.C64) == (!e.part) || !e.rexp || !e.cexp || !e.pair)
    return RR_ERR_ARG;
  if (N != e.nb && N != 2 * (int64_t)e.nb) return RR_ERR_ARG;
  return gemm_bf16_tc_impl(M, N, K, A, lda, B, ldb, nullptr, 0, nullptr, 0, nullptr, &e, s);
}

// Split product (A2, B2 non-null): C = A^T B + A2^T B + A^T B2 (+ coef R);
// every pipeline stage carries the four tiles of one K step and three MMAs
// consume them, so each operand is read once.
static rr_status gemm_bf16_tc_impl(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A, int64_t lda,
                                   const __nv_bfloat16* B, int64_t ldb, float* C, int64_t ldc,
                                   const double* R, int64_t ldr, const double* coef, const TcEmu* emu,
                                   cudaStream_t s, const __nv_bfloat16* A2, const __nv_bfloat16* B2) {
  const bool split = A2 && B2;
  if ((A2 || B2) && (!split || emu)) return RR_ERR_ARG;
  const int npad = (int)((N + 15) / 16 * 16);
  // TMEM columns: the accumulator, and for a two-slice emulation launch the
  // epilogue's 32-column reads of the second slice up to nb + 32 ceil(nb / 32)
  int need = npad;
  if (emu && N > emu->nb) {
    const int nb2 = emu->nb + 32 * ((emu->nb + 31) / 32);
    if (nb2 > need) need = nb2;
  }
  if (need > 512) return RR_ERR_ARG;
  int tcols = 32;
  while (tcols < need) tcols <<= 1;
  // tensor maps over the whole slice stacks (emulation) or the operands
  const int64_t a_outer = emu && emu->a_slices > 1 ? (int64_t)emu->a_slices * emu->a_slice_rows : M;
  const int64_t b_outer = emu && emu->b_slices > 1 ? (int64_t)emu->b_slices * emu->b_slice_rows : N;
  CUtensorMap ta, tb, ta2, tb2;
  if (!make_map(&ta, A, K, a_outer, lda, kBK, kBM)) return RR_ERR_ARG;
  if (!make_map(&tb, B, K, b_outer, ldb, kBK, (uint32_t)npad)) return RR_ERR_ARG;
  if (split) {
    if (!make_map(&ta2, A2, K, a_outer, lda, kBK, kBM)) return RR_ERR_ARG;
    if (!make_map(&tb2, B2, K, b_outer, ldb, kBK, (uint32_t)npad)) return RR_ERR_ARG;
  } else {
    ta2 = ta;
    tb2 = tb;
  }
  const int64_t tiles = (M + kBM - 1) / kBM;
  const int nk1 = (int)tc_nk(K);
  const int segs = split ? 3 : 1;
  const int nk = nk1;
  const int sms = num_sms();
  const int npairs = emu ? emu->npairs : 1;
  int splits = 1;
  if (emu && emu->part) {
    splits = tc_emu_partial_splits(M, K, npairs, emu->max_kchunk);
    if (splits < 1) return RR_ERR_ARG;
  } else if (tiles * npairs < sms && !(emu && emu->lift_k0 > 0)) {  // a lift's diagonals: whole K ranges
    splits = (int)(sms / (tiles * npairs));
    if (splits > nk) splits = nk;
    if (gemm_split_cap() > 0 && splits > gemm_split_cap()) splits = gemm_split_cap();
    if (splits < 1) splits = 1;
  }
  int per = (nk + splits - 1) / splits;
  if (emu && per * kBK > emu->max_kchunk) per = emu->max_kchunk / kBK;  // exactness of the FP32 sums
  if (per < 1) return RR_ERR_ARG;
  splits = (nk + per - 1) / per;
  if (emu && emu->part && splits != tc_emu_partial_splits(M, K, npairs, emu->max_kchunk)) return RR_ERR_ARG;
  const uint32_t stage_bytes = (kBM * kBK * 2 + (uint32_t)npad * kBK * 2) * (split ? 2 : 1);
  int stages = (int)((200 * 1024) / stage_bytes);
  if (stages > 8) stages = 8;
  if (stages < 2) return RR_ERR_ARG;
  const size_t smem = 1024 + (size_t)stages * stage_bytes + (2 * stages + 1) * sizeof(uint64_t);
  RR_TRY(tc_prepare_attributes());
  TcArgs a{};
  a.M = M;
  a.N = N;
  a.K = K;
  a.npad = npad;
  a.tmem_cols = tcols;
  a.stages = stages;
  a.ksteps_per_split = per;
  a.nk = nk;
  a.nk1 = nk1;
  a.segs = segs;
  a.C = C;
  a.ldc = ldc;
  a.R = R;
  a.ldr = ldr;
  a.coef = coef;
  a.atomic = splits > 1 || npairs > 1;
  a.C64 = emu ? emu->C64 : nullptr;
  a.ldc64 = emu ? emu->ldc64 : 0;
  a.part = emu ? emu->part : nullptr;
  a.rexp = emu ? emu->rexp : nullptr;
  a.cexp = emu ? emu->cexp : nullptr;
  a.nb = emu ? emu->nb : 1;
  a.a_slice_rows = emu ? emu->a_slice_rows : 0;
  a.b_slice_rows = emu ? emu->b_slice_rows : 0;
  a.npairs = emu ? npairs : 0;
  for (int z = 0; z < 48; ++z) a.pair[z] = (emu && z < npairs) ? emu->pair[z] : 0u;
  if (splits > 1 && !emu) {
    dim3 gi((unsigned)std::min<int64_t>((M + 255) / 256, 256), (unsigned)N);
    k_tc_init_c<<<gi, 256, 0, s>>>(M, N, C, ldc, R, ldr, coef);
    note_launches(1);
  }
  a.lift_ksteps = emu && emu->lift_k0 > 0 ? emu->lift_k0 / kBK : 0;
  a.lift_s = emu ? emu->lift_s : 0;
  if (a.lift_ksteps && (emu->lift_k0 % kBK || (int64_t)emu->lift_s * emu->lift_k0 != K || splits != 1))
    return RR_ERR_ARG;
  a.pair_major = emu && emu->C64 && npairs > 1 && tiles <= 65535;
  dim3 grid = a.pair_major ? dim3((unsigned)npairs, (unsigned)splits, (unsigned)tiles)
                           : dim3((unsigned)tiles, (unsigned)splits, (unsigned)npairs);
  a.rscale = a.cscale = nullptr;
  // algorithmic bytes of this launch: every operand tile it needs read once
  // (the distinct slices of an emulation launch), the output written once;
  // algorithmic flops: 2 M N K per product it forms (per slice pair of an
  // emulation launch, with that pair's own slice count)
  double abytes, aflops = 0.0;
  if (emu) {
    uint64_t amask = 0, bmask = 0;
    for (int z = 0; z < npairs; ++z) {
      const uint32_t pz = emu->pair[z];
      amask |= 1ull << (pz & 0xFF);
      for (uint32_t q = 0; q < ((pz >> 16) & 0xFF); ++q) bmask |= 1ull << (((pz >> 8) & 0xFF) + q);
      const double kz = emu->lift_k0 > 0 ? (double)(((pz & 0xFF) + 1) * emu->lift_k0) : (double)K;
      aflops += 2.0 * (double)M * (double)emu->nb * (double)((pz >> 16) & 0xFF) * kz;
    }
    abytes = 2.0 * K * ((double)M * __builtin_popcountll(amask) + (double)emu->nb * __builtin_popcountll(bmask)) +
             8.0 * M * emu->nb;
  } else {
    abytes = (split ? 2.0 : 1.0) * 2.0 * K * ((double)M + (double)N) + 4.0 * M * N;
    aflops = (split ? 3.0 : 1.0) * 2.0 * (double)M * (double)N * (double)K;
  }
  TcProfScope prof_scope(s, abytes, aflops, emu ? 1 : 0);
  if (emu)  // the FP64-emulation passes: an instantiation of their own (epilogue, profiles)
    k_gemm_bf16_tc<false, true><<<grid, 128, smem, s>>>(ta, tb, ta2, tb2, a);
  else
    k_gemm_bf16_tc<false, false><<<grid, 128, smem, s>>>(ta, tb, ta2, tb2, a);
  return check_launch("gemm_bf16_tc");
}

// E4M3 product: C (M x N, FP32) = diag(rscale) A_k^T B diag(cscale), A_k
// K x M and B K x N E4M3 with K contiguous (ld in elements, multiples of 16),
// FP32 accumulation.
rr_status gemm_e4m3_tc(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const float* rscale,
                       const void* B, int64_t ldb, const float* cscale, float* C, int64_t ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0 || N > 256 || K <= 0 || !rscale || !cscale || !C) return RR_ERR_ARG;
  if (lda % 16 || ldb % 16 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return RR_ERR_ARG;
  if (M > 0x7fffffff || K > 0x7fffffff || !encode_fn()) return RR_ERR_ARG;
  constexpr int kBK8 = 2 * kBK;  // E4M3 elements per 128-byte row
  const int npad = (int)((N + 15) / 16 * 16);
  int tcols = 32;
  while (tcols < npad) tcols <<= 1;
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, K, M, lda, kBK8, kBM, true)) return RR_ERR_ARG;
  if (!make_map(&tb, B, K, N, ldb, kBK8, (uint32_t)npad, true)) return RR_ERR_ARG;
  const int64_t tiles = (M + kBM - 1) / kBM;
  const int nk = (int)((K + kBK8 - 1) / kBK8);
  const int sms = num_sms();
  int splits = 1;
  if (tiles < sms) {
    splits = (int)(sms / tiles);
    if (splits > nk) splits = nk;
    if (splits < 1) splits = 1;
  }
  const int per = (nk + splits - 1) / splits;
  splits = (nk + per - 1) / per;
  const uint32_t stage_bytes = kBM * kBK8 + (uint32_t)npad * kBK8;
  int stages = (int)((200 * 1024) / stage_bytes);
  if (stages > 8) stages = 8;
  if (stages < 2) return RR_ERR_ARG;
  const size_t smem = 1024 + (size_t)stages * stage_bytes + (2 * stages + 1) * sizeof(uint64_t);
  RR_TRY(tc_prepare_attributes());
  TcArgs a{};
  a.M = M;
  a.N = N;
  a.K = K;
  a.npad = npad;
  a.tmem_cols = tcols;
  a.stages = stages;
  a.ksteps_per_split = per;
  a.nk = nk;
  a.nk1 = nk;
  a.segs = 1;
  a.C = C;
  a.ldc = ldc;
  a.atomic = splits > 1;
  a.rscale = rscale;
  a.cscale = cscale;
  if (splits > 1) {
    dim3 gi((unsigned)std::min<int64_t>((M + 255) / 256, 256), (unsigned)N);
    k_tc_init_c<<<gi, 256, 0, s>>>(M, N, C, ldc, nullptr, 0, nullptr);
    note_launches(1);
  }
  dim3 grid((unsigned)tiles, (unsigned)splits, 1u);
  TcProfScope prof_scope(s, (double)K * ((double)M + (double)N) + 4.0 * M * N, 2.0 * (double)M * N * K, 0);
  k_gemm_bf16_tc<true, false><<<grid, 128, smem, s>>>(ta, tb, ta, tb, a);
  return check_launch("gemm_e4m3_tc");
}

// error word of the tensor-core kernels (0 = ok); cleared on read
rr_status tc_take_error(cudaStream_t s) {
  int e = 0;
  RR_CUDA(cudaMemcpyFromSymbolAsync(&e, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  RR_CUDA(cudaStreamSynchronize(s));
  if (e) {
    int z = 0;
    RR_CUDA(cudaMemcpyToSymbolAsync(g_tc_error, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    return (rr_status)e;
  }
  return RR_OK;
}

}  // namespace rr

// ---------------------------------------------------------------------------
// Failure-detection self-test: each bounded wait of the library, made to run
// out on purpose.  mode 0: one CTA enters the grid barrier of the cooperative
// kernels for a grid of two CTAs that has only itself; mode 1: one thread
// waits on an mbarrier that nothing arrives on (the wait of the tensor-core
// kernels).  Both give up after limit_ns, record RR_ERR_TIMEOUT in err and
// return; the kernel ends normally.
// ---------------------------------------------------------------------------
namespace rr {
namespace {
__global__ void k_wait_selftest(int mode, uint64_t limit_ns, GridBarrier* gb, int* err) {
  if (mode == 0) {
    grid_barrier(gb, 2u, err, limit_ns);   // the second CTA never arrives
    return;
  }
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_wait_on(&bar, 0, err, limit_ns);  // phase 0 never completes
  }
}
}  // namespace
}  // namespace rr

extern "C" rr_status rr_wait_selftest(int32_t mode, int64_t limit_ns, void* scratch, void* stream) {
  using namespace rr;
  if ((mode != 0 && mode != 1) || limit_ns <= 0 || limit_ns > 10000000000ll || !scratch ||
      ((uintptr_t)scratch & 15))
    return RR_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  GridBarrier* gb = (GridBarrier*)scratch;
  int* err = (int*)((char*)scratch + sizeof(GridBarrier));
  RR_CUDA(cudaMemsetAsync(scratch, 0, 16, s));
  k_wait_selftest<<<1, 32, 0, s>>>(mode, (uint64_t)limit_ns, gb, err);
  RR_TRY(check_launch("rr_wait_selftest"));
  int h = 0;
  RR_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  RR_CUDA(cudaStreamSynchronize(s));
  return (rr_status)h;
}
