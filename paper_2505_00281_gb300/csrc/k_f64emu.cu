// FP64-accurate block products on the BF16 tensor cores (error-free fixed-
// point slicing, the Ozaki scheme), for the refinement phase's residual
// products A X and A^T Y (FP64 operator, FP64 Ritz vectors).  GB300 has few
// FP64 units; its BF16 tensor cores are ~1500x faster.
//
// Slicing: every row of A (for A X) or column of A (for A^T Y) and every
// column of X is scaled by a power of two 2^e so its entries lie in (-1, 1),
// then split into S integer slices of beta = 6 bits (balanced digits of the
// rounded fixed-point value, computed with integer operations only):
//   x = 2^e (sum_{p=1..S} s_p 2^(-beta p) + r),  |s_1| <= 64, |s_p| <= 32,
//   |r| <= 2^(-beta S - 1);
// each s_p is an integer exactly representable in BF16.  The product of two
// slices, summed over a K-chunk of at most 4096, is an integer of magnitude
// at most 4096 * 64 * 64 = 2^24, which the tensor core's FP32 accumulator
// holds exactly.  The epilogue multiplies each exact partial product by the
// power of two 2^(e_row + e_col - beta (p + q)) and adds it into the FP64
// result.  Slice pairs with p + q <= S + 1 are kept; the dropped ones and the
// remainders contribute below 2^(-beta (S + 1)) relative to the row and
// column scales (S = 8: ~2^-54).
#include "rr_common.cuh"
#include "solver_kernels.cuh"

namespace rr {

bool gemm_bf16_tc_supported(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, const void* A,
                            const void* B);

constexpr int kBeta = 6;
constexpr int kMaxSlices = 10;

// Exponent e with |x| < 2^e from the IEEE bit pattern (integer work only):
// for a normal x = 1.f 2^(E-1023), e = E - 1022; zero and subnormals -> -1100.
__device__ __forceinline__ int exp_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7FF);
  return E == 0 ? -1100 : E - 1022;
}

// exponent of the largest |entry| of every row of a column-major matrix
// (max over the entries' exponents = exponent of the largest entry)
__global__ void k_row_exp(int64_t m, int64_t n, const double* __restrict__ A, int64_t lda,
                          int* __restrict__ e) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int mx = -1100;
  for (int64_t j = 0; j < n; ++j) mx = max(mx, exp_bits(A[i + j * lda]));
  e[i] = mx;
}

// exponent of the largest |entry| of every column (one block per column)
__global__ void k_col_exp(int64_t m, const double* __restrict__ A, int64_t lda, int* __restrict__ e) {
  const int64_t j = blockIdx.x;
  int mx = -1100;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) mx = max(mx, exp_bits(A[i + j * lda]));
  __shared__ int sm[32];
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : -1100;
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) e[j] = mx;
  }
}

// Error-free slicing of x relative to 2^e (|x| < 2^e) in integer arithmetic:
// F = round(|x| 2^(6S - e)) (a fixed-point integer below 2^(6S) + 1), then
// balanced base-64 digits from the least significant end (each in
// [-32, 31]; the leading one in [-32, 64]), signed like x:
//   x = 2^e sum_{p=1..S} out[p-1] 2^(-6p) + r,  |r| <= 2^(e - 6S - 1).
__device__ __forceinline__ void slice_value(double x, int e, int S, float* out) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7FF);
  long long F = 0;
  if (E != 0) {
    const unsigned long long M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    // |x| 2^(6S - e) = M 2^(E - 1075 + 6S - e)
    const int sh = E - 1075 + kBeta * S - e;  // <= 6S - 53 - 1 (|x| < 2^e)
    if (sh >= 0) F = (long long)(M << sh);
    else if (sh > -63) F = (long long)((M + (1ull << (-sh - 1))) >> (-sh));
  }
  // digits in 32-bit integers (a 64-bit integer to float conversion is not
  // a full-rate instruction)
  for (int p = S - 1; p >= 1; --p) {
    int d = (int)(F & 63);
    F >>= 6;
    if (d >= 32) {
      d -= 64;
      F += 1;
    }
    out[p] = (float)d;
  }
  out[0] = (float)(int)F;
  if (u >> 63)
    for (int p = 0; p < S; ++p) out[p] = -out[p];
}

// BF16 bits of a small integer-valued float (|v| <= 256: exact)
__device__ __forceinline__ unsigned bf16_bits_exact(float v) { return __float_as_uint(v) >> 16; }

// BF16 bits (sign excluded) of v = k 2^s (0 < k < 2^62) rounded the way an
// FP64 value is cast to BF16 here: to FP32 (nearest even), then the FP32
// pattern to BF16 (nearest even; a carry may reach the exponent).  Integer
// operations only (this GPU has few FP64 units).  False when the FP32
// rounding is not a normal number (the caller then uses the conversion
// instructions).
__device__ __forceinline__ bool bf16_of_scaled(unsigned long long k, int s, unsigned& out) {
  int msb = 63 - __clzll((long long)k);
  unsigned long long k24;
  if (msb > 23) {
    const int sh = msb - 23;
    k24 = k >> sh;
    const unsigned long long rem = k & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (k24 & 1ull))) ++k24;
    if (k24 == (1ull << 24)) {
      k24 >>= 1;
      ++msb;
    }
  } else {
    k24 = k << (23 - msb);
  }
  const int e32 = msb + s + 127;  // v rounded = (k24 / 2^23) 2^(msb + s)
  if (e32 < 1 || e32 > 254) return false;
  const unsigned f = ((unsigned)e32 << 23) | (unsigned)(k24 & 0x7FFFFFull);
  out = (f + 0x7FFFu + ((f >> 16) & 1u)) >> 16;
  return true;
}

// hi = bf16(a) and lo = bf16(a - hi) with the cast above (a - hi is exact
// in FP64), as BF16 bit patterns.
__device__ __forceinline__ void bf16_split_bits(double a, unsigned& hi, unsigned& lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const unsigned sgn = (unsigned)(u >> 63);
  const int E = (int)((u >> 52) & 0x7FF);
  const unsigned long long M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // a = M 2^(E - 1075)
  unsigned hb, lb;
  if (E == 0 || E == 0x7FF || !bf16_of_scaled(M, E - 1075, hb)) {
    const __nv_bfloat16 h = __float2bfloat16_rn((float)a);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__float2bfloat16_rn((float)(a - (double)__bfloat162float(h))));
    return;
  }
  hi = (sgn << 15) | hb;
  // hi in units of a's last place: (128 + m7) 2^(e8 - 134 - (E - 1075))
  const int e8 = (int)(hb >> 7), sh = e8 + 941 - E;  // 45, or 46 after a carry
  const long long d = (long long)M - (long long)((128ull + (hb & 127u)) << sh);
  if (d == 0) {
    lo = 0;
    return;
  }
  if (!bf16_of_scaled((unsigned long long)(d < 0 ? -d : d), E - 1075, lb)) {
    const double hv = (double)__bfloat162float(__ushort_as_bfloat16((unsigned short)hi));
    lo = __bfloat16_as_ushort(__float2bfloat16_rn((float)(a - hv)));
    return;
  }
  lo = ((sgn ^ (d < 0 ? 1u : 0u)) << 15) | lb;
}

// hi only (the same cast)
__device__ __forceinline__ unsigned bf16_bits_of(double a) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const int E = (int)((u >> 52) & 0x7FF);
  unsigned hb;
  if (E == 0 || E == 0x7FF || !bf16_of_scaled((u & 0xFFFFFFFFFFFFFull) | (1ull << 52), E - 1075, hb))
    return __bfloat16_as_ushort(__float2bfloat16_rn((float)a));
  return ((unsigned)(u >> 63) << 15) | hb;
}

constexpr int kExpNone = -1100;  // exponent of zero (below every finite one)

__global__ void k_exp_init(int64_t count, int* __restrict__ e) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    e[i] = kExpNone;
}

// First pass over a dense FP64 operator (m x n, column-major): the BF16 hi /
// lo split in column-major and row-major copies, and the exponents of the
// largest entry of every row and column (atomic max into rexp / cexp, which
// start at kExpNone).  Every output may be null.  A block takes a 32-row x
// 256-column tile, a warp 32 x 32 (lane = row) in two halves of 16 columns
// (62 registers instead of 120: four blocks per SM, twice the resident
// warps; the pass is bound by the loads in flight): column
// loads are coalesced, a lane writes its row's 16 entries of a half to the
// row-major copies as two 16-byte stores.
__global__ void __launch_bounds__(256, 4) k_op_pass1(int64_t m, int64_t n, const double* __restrict__ A, int64_t lda,
                                                  __nv_bfloat16* __restrict__ hi_col, __nv_bfloat16* __restrict__ hi_row,
                                                  __nv_bfloat16* __restrict__ lo_col, __nv_bfloat16* __restrict__ lo_row,
                                                  int* __restrict__ rexp, int* __restrict__ cexp) {
  __shared__ int rmax[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  const bool rv = i < m;
  const bool need_lo = lo_col || lo_row;
  int emx = kExpNone;
#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    const int64_t jw = (int64_t)blockIdx.y * 256 + warp * 32 + 16 * half;
    unsigned hp[8], lp[8];
    double av[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int64_t j = jw + c;
      av[c] = (rv && j < n) ? A[i + j * lda] : 0.0;
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int64_t j = jw + c;
      const double a = av[c];
      const unsigned long long u = (unsigned long long)__double_as_longlong(a);
      const int E = (int)((u >> 52) & 0x7FF);
      const int e = E == 0 ? kExpNone : E - 1022;
      emx = max(emx, e);
      if (cexp) {
        int ce = e;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ce = max(ce, __shfl_xor_sync(0xffffffffu, ce, o));
        if (lane == 0 && j < n) atomicMax(cexp + j, ce);
      }
      unsigned h = 0, l = 0;
      if (need_lo) {
        bf16_split_bits(a, h, l);
      } else {
        h = bf16_bits_of(a);
      }
      if (c & 1) {
        hp[c >> 1] |= h << 16;
        lp[c >> 1] |= l << 16;
      } else {
        hp[c >> 1] = h;
        lp[c >> 1] = l;
      }
      if (rv && j < n) {
        if (hi_col) hi_col[i + j * m] = __ushort_as_bfloat16((unsigned short)h);
        if (lo_col) lo_col[i + j * m] = __ushort_as_bfloat16((unsigned short)l);
      }
    }
    if (rv) {
      const bool vec = (jw + 16 <= n) && (n % 8 == 0);
      if (hi_row) {
        if (vec) {
          uint4* dst = reinterpret_cast<uint4*>(hi_row + i * n + jw);
#pragma unroll
          for (int k = 0; k < 2; ++k) dst[k] = make_uint4(hp[4 * k], hp[4 * k + 1], hp[4 * k + 2], hp[4 * k + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (jw + c < n) hi_row[i * n + jw + c] = __ushort_as_bfloat16((unsigned short)(hp[c >> 1] >> (16 * (c & 1))));
        }
      }
      if (lo_row) {
        if (vec) {
          uint4* dst = reinterpret_cast<uint4*>(lo_row + i * n + jw);
#pragma unroll
          for (int k = 0; k < 2; ++k) dst[k] = make_uint4(lp[4 * k], lp[4 * k + 1], lp[4 * k + 2], lp[4 * k + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (jw + c < n) lo_row[i * n + jw + c] = __ushort_as_bfloat16((unsigned short)(lp[c >> 1] >> (16 * (c & 1))));
        }
      }
    }
  }
  if (rexp) {
    rmax[warp][lane] = emx;
    __syncthreads();
    if (warp == 0 && rv) {
      int r = rmax[0][lane];
#pragma unroll
      for (int w = 1; w < 8; ++w) r = max(r, rmax[w][lane]);
      atomicMax(rexp + i, r);
    }
  }
}

// Second pass: the S slices of every entry, row-scaled (2^rexp[i], written
// row-major: element (i, j) of slice p at rows[p m n + i n + j]) and / or
// column-scaled (2^cexp[j], column-major: cols[p m n + i + j m]).  A block
// takes 32 rows x 64 columns, a warp 32 x 8 (lane = row); a lane packs its
// row's 8 digits of each slice into one 16-byte store.  Small per-warp work
// and three resident blocks per SM keep many loads in flight (the earlier
// 32 x 32 warp tile at two blocks per SM ran the 16384 x 4096 operator in
// 1.45 ms, this one in 0.80 ms).
constexpr int kSliceCols = 64;
template <int S>
__global__ void __launch_bounds__(256, 3) k_op_slices(int64_t m, int64_t n, const double* __restrict__ A, int64_t lda,
                                                   const int* __restrict__ rexp, const int* __restrict__ cexp,
                                                   __nv_bfloat16* __restrict__ rows, __nv_bfloat16* __restrict__ cols) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  const int64_t jw = (int64_t)blockIdx.y * kSliceCols + warp * 8;
  const bool rv = i < m;
  const int er = (rows && rv) ? rexp[i] : 0;
  const size_t plane = (size_t)m * n;
  const bool vec = (n % 8 == 0);
  {
    const int64_t j0 = jw;
    double av[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) av[c] = (rv && j0 + c < n) ? A[i + (j0 + c) * lda] : 0.0;
    if (rows) {
      unsigned pk[S][4];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        float sl[S];
        slice_value(av[c], er, S, sl);
#pragma unroll
        for (int p = 0; p < S; ++p) {
          const unsigned b = bf16_bits_exact(sl[p]);
          if (c & 1) pk[p][c >> 1] |= b << 16;
          else pk[p][c >> 1] = b;
        }
      }
      if (rv && j0 < n) {
        if (vec && j0 + 8 <= n) {
#pragma unroll
          for (int p = 0; p < S; ++p)
            *reinterpret_cast<uint4*>(rows + (size_t)p * plane + i * n + j0) =
                make_uint4(pk[p][0], pk[p][1], pk[p][2], pk[p][3]);
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (j0 + c < n) {
#pragma unroll
              for (int p = 0; p < S; ++p)
                rows[(size_t)p * plane + i * n + j0 + c] =
                    __ushort_as_bfloat16((unsigned short)(pk[p][c >> 1] >> (16 * (c & 1))));
            }
        }
      }
    }
    if (cols) {
      // the column-scaled digits re-read the entries (cache hits), which
      // keeps the loop rolled and the register count low
#pragma unroll 1
      for (int c = 0; c < 8; ++c) {
        const int64_t j = j0 + c;
        if (j >= n) break;
        float sl[S];
        slice_value(rv ? A[i + j * lda] : 0.0, cexp[j], S, sl);
        if (rv) {
#pragma unroll
          for (int p = 0; p < S; ++p)
            cols[(size_t)p * plane + i + j * m] = __ushort_as_bfloat16((unsigned short)bf16_bits_exact(sl[p]));
        }
      }
    }
  }
}

// column-scaled slices, same layout as the input: out[p] (m x n, ld m)
__global__ void k_slice_cols(int64_t m, int64_t n, const double* __restrict__ A, int64_t lda,
                             const int* __restrict__ cexp, int S, __nv_bfloat16* __restrict__ out) {
  const int64_t j = blockIdx.y;
  const int e = cexp[j];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    float sl[kMaxSlices];
    slice_value(A[i + j * lda], e, S, sl);
    for (int p = 0; p < S; ++p) out[(size_t)p * m * n + i + j * m] = __float2bfloat16_rn(sl[p]);
  }
}

// row-scaled slices written row-major (element (i, j) at i*n + j): the
// K-major operand of A X.  32 x 32 tiles through shared memory.
__global__ void k_slice_rows(int64_t m, int64_t n, const double* __restrict__ A, int64_t lda,
                             const int* __restrict__ rexp, int S, __nv_bfloat16* __restrict__ out) {
  __shared__ __nv_bfloat16 tile[kMaxSlices][32][34];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + tx, j = j0 + r;
    float sl[kMaxSlices];
    if (i < m && j < n) {
      slice_value(A[i + j * lda], rexp[i], S, sl);
    } else {
      for (int p = 0; p < S; ++p) sl[p] = 0.f;
    }
    for (int p = 0; p < S; ++p) tile[p][r][tx] = __float2bfloat16_rn(sl[p]);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + tx;
    if (i < m && j < n)
      for (int p = 0; p < S; ++p) out[(size_t)p * m * n + i * n + j] = tile[p][tx][r];
  }
}

__global__ void k_zero_f64(int64_t M, int64_t N, double* __restrict__ C, int64_t ldc) {
  const int64_t j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
    C[i + j * ldc] = 0.0;
}

// ---------------------------------------------------------------------------
size_t emu_operator_bytes(int64_t m, int64_t n, int S, bool rows, bool cols) {
  size_t b = 0;
  if (rows) b += align_up((size_t)S * m * n * 2) + align_up((size_t)m * 4);
  if (cols) b += align_up((size_t)S * m * n * 2) + align_up((size_t)n * 4);
  return b;
}

size_t emu_block_bytes(int64_t K, int64_t N, int S) {
  return align_up((size_t)S * K * N * 2) + align_up((size_t)N * 4);
}

// All preparation of a dense FP64 operator in two passes over A: BF16 hi / lo
// copies (any of the four may be null) and, when emu is given, the slices
// for FP64-accurate products (row-scaled row-major for A X, column-scaled
// column-major for A^T Y) in emu_mem.
rr_status op_prepare(cudaStream_t s, const double* A, int64_t m, int64_t n, int64_t lda,
                     __nv_bfloat16* hi_col, __nv_bfloat16* hi_row, __nv_bfloat16* lo_col, __nv_bfloat16* lo_row,
                     int S, EmuOperator* emu, void* emu_mem, bool rows, bool cols) {
  if (m <= 0 || n <= 0) return RR_OK;
  int *rexp = nullptr, *cexp = nullptr;
  if (emu) {
    if (S != 8) return RR_ERR_ARG;
    Arena ar(emu_mem, emu_operator_bytes(m, n, S, rows, cols));
    emu->m = m;
    emu->n = n;
    emu->S = S;
    emu->rows = nullptr;
    emu->rexp = nullptr;
    emu->cols = nullptr;
    emu->cexp = nullptr;
    if (rows) {
      emu->rows = (__nv_bfloat16*)ar.take_bytes((size_t)S * m * n * 2);
      emu->rexp = rexp = ar.take<int>(m);
      k_exp_init<<<(unsigned)std::min<int64_t>((m + 255) / 256, 1024), 256, 0, s>>>(m, rexp);
      note_launches(1);
    }
    if (cols) {
      emu->cols = (__nv_bfloat16*)ar.take_bytes((size_t)S * m * n * 2);
      emu->cexp = cexp = ar.take<int>(n);
      k_exp_init<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(n, cexp);
      note_launches(1);
    }
  }
  const dim3 g((unsigned)((m + 31) / 32), (unsigned)((n + 255) / 256));
  if (hi_col || hi_row || lo_col || lo_row || rexp || cexp) {
    k_op_pass1<<<g, 256, 0, s>>>(m, n, A, lda, hi_col, hi_row, lo_col, lo_row, rexp, cexp);
    RR_TRY(check_launch("op_prepare pass 1"));
  }
  if (emu && (rows || cols)) {
    const dim3 g2((unsigned)((m + 31) / 32), (unsigned)((n + kSliceCols - 1) / kSliceCols));
    k_op_slices<8><<<g2, 256, 0, s>>>(m, n, A, lda, rexp, cexp, emu->rows, emu->cols);
    RR_TRY(check_launch("op_prepare slices"));
  }
  return RR_OK;
}

// Slice the FP64 operator A (m x n, column-major) once: row-scaled slices
// (row-major) for A X and/or column-scaled slices (column-major) for A^T Y.
rr_status emu_prepare(cudaStream_t s, const double* A, int64_t m, int64_t n, int64_t lda, int S,
                      EmuOperator& op, void* mem, bool rows, bool cols) {
  if (S < 1 || S > kMaxSlices) return RR_ERR_ARG;
  if (S == 8) return op_prepare(s, A, m, n, lda, nullptr, nullptr, nullptr, nullptr, S, &op, mem, rows, cols);
  Arena ar(mem, emu_operator_bytes(m, n, S, rows, cols));
  op.m = m;
  op.n = n;
  op.S = S;
  op.rows = nullptr;
  op.rexp = nullptr;
  op.cols = nullptr;
  op.cexp = nullptr;
  if (rows) {
    op.rows = (__nv_bfloat16*)ar.take_bytes((size_t)S * m * n * 2);
    op.rexp = ar.take<int>(m);
    k_row_exp<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, n, A, lda, op.rexp);
    dim3 g((unsigned)((m + 31) / 32), (unsigned)((n + 31) / 32)), b(32, 8);
    k_slice_rows<<<g, b, 0, s>>>(m, n, A, lda, op.rexp, S, op.rows);
    note_launches(1);
    RR_TRY(check_launch("emu_prepare rows"));
  }
  if (cols) {
    op.cols = (__nv_bfloat16*)ar.take_bytes((size_t)S * m * n * 2);
    op.cexp = ar.take<int>(n);
    k_col_exp<<<(unsigned)n, 512, 0, s>>>(m, A, lda, op.cexp);
    dim3 g((unsigned)std::min<int64_t>((m + 255) / 256, 1024), (unsigned)n);
    k_slice_cols<<<g, 256, 0, s>>>(m, n, A, lda, op.cexp, S, op.cols);
    note_launches(1);
    RR_TRY(check_launch("emu_prepare cols"));
  }
  return RR_OK;
}

// exact FP64 value of a stored entry, through integer operations (FP32 / BF16
// to FP64 conversions would use the few FP64 units)
__device__ __forceinline__ double f32_to_f64_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned E = (u >> 23) & 0xFFu;
  if (E == 0 || E == 255) return (double)f;  // zero, subnormal, Inf / NaN
  return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                          ((unsigned long long)(E + 896) << 52) |
                                          ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
template <typename T> __device__ __forceinline__ double exact_f64(T v);
template <> __device__ __forceinline__ double exact_f64<double>(double v) { return v; }
template <> __device__ __forceinline__ double exact_f64<float>(float v) { return f32_to_f64_exact(v); }
template <> __device__ __forceinline__ double exact_f64<__nv_bfloat16>(__nv_bfloat16 v) {
  return f32_to_f64_exact(__bfloat162float(v));
}
template <> __device__ __forceinline__ double exact_f64<e4m3b_t>(e4m3b_t v) {
  return f32_to_f64_exact(e4m3b_value(v.c));
}

constexpr int kGramSlices = 8;
constexpr int kGramKChunk = 4096;

// Column exponents and column-scaled slices of a Gram operand (n x c, any
// storage type, n % 8 == 0): a thread takes 8 consecutive rows of one column,
// the values reach FP64 exactly through integer operations (exact_f64), and
// each slice's 8 digits leave as one 16-byte store.
template <typename T>
__global__ void k_col_exp8(int64_t n, const T* __restrict__ X, int64_t ldx, int* __restrict__ e) {
  const int64_t j = blockIdx.x;
  int mx = kExpNone;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = max(mx, exp_bits(exact_f64<T>(X[i + j * ldx])));
  __shared__ int sm[32];
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : kExpNone;
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (threadIdx.x == 0) e[j] = mx;
  }
}

template <typename T>
__global__ void k_slice_cols8(int64_t n, int64_t c, const T* __restrict__ X, int64_t ldx,
                              const int* __restrict__ cexp, __nv_bfloat16* __restrict__ out) {
  constexpr int S = kGramSlices;
  const int64_t j = blockIdx.y;
  const int e = cexp[j];
  const size_t plane = (size_t)n * c;
  for (int64_t i0 = 8 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); i0 < n;
       i0 += 8 * (int64_t)gridDim.x * blockDim.x) {
    unsigned pk[S][4];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      float sl[S];
      slice_value(exact_f64<T>(X[i0 + r + j * ldx]), e, S, sl);
#pragma unroll
      for (int q = 0; q < S; ++q) {
        const unsigned bb = bf16_bits_exact(sl[q]);
        if (r & 1) pk[q][r >> 1] |= bb << 16;
        else pk[q][r >> 1] = bb;
      }
    }
#pragma unroll
    for (int q = 0; q < S; ++q)
      *reinterpret_cast<uint4*>(out + q * plane + j * n + i0) = make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
  }
}

template <typename T>
static void emu_slice_block(cudaStream_t s, int64_t n, int64_t c, const T* X, int64_t ldx, int* e,
                            __nv_bfloat16* out) {
  k_col_exp8<T><<<(unsigned)c, 512, 0, s>>>(n, X, ldx, e);
  dim3 g((unsigned)std::min<int64_t>((n / 8 + 127) / 128, 1024), (unsigned)c);
  k_slice_cols8<T><<<g, 128, 0, s>>>(n, c, X, ldx, e, out);
}

// The slice pairs (p, q), p + q <= S + 1 (1-based), grouped by p into runs
// of one or two consecutive q: pair codes p0 | q0 << 8 | nq << 16 (0-based).
static int emu_pairs(int S, bool two, uint32_t* out) {
  int n = 0;
  for (int p = 1; p <= S; ++p)
    for (int q = 1; q <= S + 1 - p;) {
      const int nq = (two && q + 1 <= S + 1 - p) ? 2 : 1;
      out[n++] = (uint32_t)(p - 1) | ((uint32_t)(q - 1) << 8) | ((uint32_t)nq << 16);
      q += nq;
    }
  return n;
}

// C (FP64, M x N) = A X (trans = 0, M = m, K = n) or A^T X (trans = 1, M = n,
// K = m), X FP64 K x N column-major; mem: emu_block_bytes(K, N, S).
rr_status emu_gemm(cudaStream_t s, const EmuOperator& op, int trans, int64_t N, const double* X,
                   int64_t ldx, double* C, int64_t ldc, void* mem) {
  const int S = op.S;
  const int64_t M = trans ? op.n : op.m, K = trans ? op.m : op.n;
  const __nv_bfloat16* As = trans ? op.cols : op.rows;
  const int* rexp = trans ? op.cexp : op.rexp;
  if (!As || N <= 0 || N > 256) return RR_ERR_ARG;
  Arena ar(mem, emu_block_bytes(K, N, S));
  __nv_bfloat16* T = (__nv_bfloat16*)ar.take_bytes((size_t)S * K * N * 2);
  int* xe = ar.take<int>(N);
  if (S == kGramSlices && K % 8 == 0) {
    emu_slice_block<double>(s, K, N, X, ldx, xe, T);
  } else {
    k_col_exp<<<(unsigned)N, 512, 0, s>>>(K, X, ldx, xe);
    dim3 g((unsigned)std::min<int64_t>((K + 255) / 256, 1024), (unsigned)N);
    k_slice_cols<<<g, 256, 0, s>>>(K, N, X, ldx, xe, S, T);
  }
  dim3 gz((unsigned)std::min<int64_t>((M + 255) / 256, 1024), (unsigned)N);
  k_zero_f64<<<gz, 256, 0, s>>>(M, N, C, ldc);
  note_launches(2);
  RR_TRY(check_launch("emu_gemm slices"));
  const int64_t lda = trans ? op.m : op.n;  // K-contiguous leading dimension of the A slices
  uint32_t pairs[64];
  const bool two = 2 * N <= 256;
  const int np = emu_pairs(S, two, pairs);
  // one launch for every pair (grid z = pair): the tiles of all pairs share
  // the GPU, no SM idles between passes, and each CTA adds its exactly scaled
  // products into C with FP64 atomics (C starts at zero).  A one-slice pair
  // of a two-slice launch also reads the next X slice (present: nq = 1 only
  // where q0 + 1 < S) and ignores it.
  TcEmu e{C, ldc, nullptr, rexp, xe, (int)N, S, S, (int)M, (int)N, np, pairs, 4096};
  return gemm_bf16_tc_emu(M, two ? 2 * N : N, K, As, lda, T, K, e, s);
}

// ---------------------------------------------------------------------------
// FP64-accurate lift X = [S1 S2] Y (Alg. 3 / Alg. 5 "U~ = U Y": the n x K
// basis, K = p1 + p2 columns from two blocks of any storage type, times the
// K x b FP64 Ritz coefficients) on the tensor cores.  [S1 S2] is sliced by
// rows (one exponent per row across both blocks) into A_cat (row-major, row i
// = the S digit blocks of the row, most significant first), Y by columns into
// Y_rev (column j = its digit blocks, least significant first).  With K small
// every product sum of one anti-diagonal p + q = d of slice pairs is exact in
// FP32 (at most 8 K 2^12 <= 2^24 for K <= 512), so diagonal d is one plain
// product A_cat(:, 0:(d-1)K) Y_rev((S-d+1)K : S K, :) whose epilogue adds
// 2^(e_row + e_col - 6d) times it into X: S launches instead of one per pair.
// ---------------------------------------------------------------------------

// Row exponents of [S1 S2] (atomic max over 32-column chunks; rexp starts at
// kExpNone), then the row-scaled slices: a thread takes 8 rows of an
// 8-column group, lane = row (coalesced column loads), and writes each
// slice's 8 digits of a row as one 16-byte store.  K % 8 == 0.
template <typename T1, typename T2>
__global__ void k_lift_rexp(int64_t n, int p1, const T1* __restrict__ S1, int64_t ld1, int p2,
                            const T2* __restrict__ S2, int64_t ld2, int* __restrict__ rexp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int K = p1 + p2, k0 = blockIdx.y * 32, k1 = min(K, k0 + 32);
  int e = kExpNone;
  for (int kk = k0; kk < k1; ++kk)
    e = max(e, exp_bits(kk < p1 ? exact_f64<T1>(S1[i + kk * ld1]) : exact_f64<T2>(S2[i + (kk - p1) * ld2])));
  atomicMax(rexp + i, e);
}

template <typename T1, typename T2>
__global__ void __launch_bounds__(128) k_lift_slices(int64_t n, int p1, const T1* __restrict__ S1, int64_t ld1,
                                                     int p2, const T2* __restrict__ S2, int64_t ld2,
                                                     const int* __restrict__ rexp, __nv_bfloat16* __restrict__ out) {
  constexpr int S = 8;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int K = p1 + p2, k0 = blockIdx.y * 8;
  const int e = rexp[i];
  unsigned pk[S][4];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int kk = k0 + c;
    const double x = kk < p1 ? exact_f64<T1>(S1[i + kk * ld1]) : exact_f64<T2>(S2[i + (kk - p1) * ld2]);
    float sl[S];
    slice_value(x, e, S, sl);
#pragma unroll
    for (int q = 0; q < S; ++q) {
      const unsigned bb = bf16_bits_exact(sl[q]);
      if (c & 1) pk[q][c >> 1] |= bb << 16;
      else pk[q][c >> 1] = bb;
    }
  }
  __nv_bfloat16* row = out + i * (int64_t)(S * K);
#pragma unroll
  for (int q = 0; q < S; ++q)
    *reinterpret_cast<uint4*>(row + q * K + k0) = make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
}

// Y_rev (S K x b, column-major): column j holds Y(:, j)'s digit blocks,
// least significant first, scaled by 2^cexp[j]
__global__ void k_slice_cols_rev(int64_t K, int64_t b, const double* __restrict__ Y, int64_t ldy,
                                 const int* __restrict__ cexp, __nv_bfloat16* __restrict__ out) {
  constexpr int S = 8;
  const int64_t j = blockIdx.y;
  const int e = cexp[j];
  for (int64_t kk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; kk < K; kk += (int64_t)gridDim.x * blockDim.x) {
    float sl[S];
    slice_value(Y[kk + j * ldy], e, S, sl);
#pragma unroll
    for (int q = 0; q < S; ++q)
      out[j * (S * K) + (S - 1 - q) * K + kk] = __ushort_as_bfloat16((unsigned short)bf16_bits_exact(sl[q]));
  }
}

size_t lift_emu_bytes(int64_t n, int64_t b, int64_t K) {
  return align_up((size_t)8 * n * K * 2) + align_up((size_t)8 * K * b * 2) + align_up((size_t)n * 4) +
         align_up((size_t)b * 4) + 256;
}

template <typename T1, typename T2>
static void launch_lift_slices2(cudaStream_t s, int64_t n, int p1, const T1* S1, int64_t ld1, int p2, const T2* S2,
                                int64_t ld2, int* rexp, __nv_bfloat16* out) {
  const int K = p1 + p2;
  k_exp_init<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(n, rexp);
  k_lift_rexp<T1, T2><<<dim3((unsigned)((n + 255) / 256), (unsigned)((K + 31) / 32)), 256, 0, s>>>(
      n, p1, S1, ld1, p2, S2, ld2, rexp);
  k_lift_slices<T1, T2><<<dim3((unsigned)((n + 127) / 128), (unsigned)(K / 8)), 128, 0, s>>>(n, p1, S1, ld1, p2, S2,
                                                                                              ld2, rexp, out);
  note_launches(2);
}

template <typename T1>
static void launch_lift_slices(cudaStream_t s, int64_t n, int p1, const T1* S1, int64_t ld1, int p2, int32_t t2,
                               const void* S2, int64_t ld2, int* rexp, __nv_bfloat16* out) {
  switch (t2) {
    case RR_F32: launch_lift_slices2<T1, float>(s, n, p1, S1, ld1, p2, (const float*)S2, ld2, rexp, out); break;
    case RR_BF16:
      launch_lift_slices2<T1, __nv_bfloat16>(s, n, p1, S1, ld1, p2, (const __nv_bfloat16*)S2, ld2, rexp, out);
      break;
    default: launch_lift_slices2<T1, double>(s, n, p1, S1, ld1, p2, (const double*)S2, ld2, rexp, out); break;
  }
}

static rr_status lift_emu_one(cudaStream_t s, int64_t n, int64_t b, int32_t t1, const void* S1, int64_t ld1,
                              int64_t p1, int32_t t2, const void* S2, int64_t ld2, int64_t p2, const double* Y,
                              int64_t ldy, double* X, int64_t ldx, void* mem, size_t mem_bytes, bool* done,
                              bool accumulate);

// X (n x b FP64) = S1 (n x p1, type t1) Y(0:p1, :) + S2 (n x p2, type t2)
// Y(p1:K, :); *done = false (nothing launched) when the shape is outside the
// tensor-core path (the caller then lifts in FP64 arithmetic).  With both
// blocks present (the refinement's [X, D] lifts, whose correction columns are
// scaled to unit inf-norm while X's unit 2-norm columns have entries of
// 1/sqrt(n)), each block is sliced with its own row exponents and the two
// products add into X: one exponent per row across both would leave X's
// entries only the bits below the correction block's, an error of
// 2^-48 max|D(i,:)| per row instead of 2^-48 max|X(i,:)|.
rr_status lift_emu(cudaStream_t s, int64_t n, int64_t b, int32_t t1, const void* S1, int64_t ld1, int64_t p1,
                   int32_t t2, const void* S2, int64_t ld2, int64_t p2, const double* Y, int64_t ldy, double* X,
                   int64_t ldx, void* mem, size_t mem_bytes, bool* done) {
  *done = false;
  if (S2 && p2 > 0 && p1 % 8 == 0 && p2 % 8 == 0 && p1 > 0) {
    bool d1 = false, d2 = false;
    RR_TRY(lift_emu_one(s, n, b, t1, S1, ld1, p1, t2, nullptr, 0, 0, Y, ldy, X, ldx, mem, mem_bytes, &d1, false));
    if (!d1) return RR_OK;
    RR_TRY(lift_emu_one(s, n, b, t2, S2, ld2, p2, t2, nullptr, 0, 0, Y + p1, ldy, X, ldx, mem, mem_bytes, &d2,
                        true));
    if (!d2) return RR_ERR_ARG;  // the second block fits whenever the first did (same n, b, K <= p1 + p2)
    *done = true;
    return RR_OK;
  }
  return lift_emu_one(s, n, b, t1, S1, ld1, p1, t2, S2, ld2, p2, Y, ldy, X, ldx, mem, mem_bytes, done, false);
}

static rr_status lift_emu_one(cudaStream_t s, int64_t n, int64_t b, int32_t t1, const void* S1, int64_t ld1,
                              int64_t p1, int32_t t2, const void* S2, int64_t ld2, int64_t p2, const double* Y,
                              int64_t ldy, double* X, int64_t ldx, void* mem, size_t mem_bytes, bool* done,
                              bool accumulate) {
  constexpr int S = 8;
  *done = false;
  const int64_t K = p1 + (S2 ? p2 : 0);
  if (!mem || n <= 0 || b <= 0 || b > 256 || K <= 0 || K % 8 || K > 512 || p1 <= 0) return RR_OK;
  if (mem_bytes < lift_emu_bytes(n, b, K)) return RR_OK;
  Arena ar(mem, lift_emu_bytes(n, b, K));
  __nv_bfloat16* Acat = (__nv_bfloat16*)ar.take_bytes((size_t)S * n * K * 2);
  __nv_bfloat16* Yrev = (__nv_bfloat16*)ar.take_bytes((size_t)S * K * b * 2);
  int* rexp = ar.take<int>(n);
  int* yexp = ar.take<int>(b);
  if (!gemm_bf16_tc_supported(n, b, (S - 1) * K, S * K, S * K, Acat, Yrev)) return RR_OK;
  const int ip1 = (int)p1, ip2 = (int)(S2 ? p2 : 0);
  switch (t1) {
    case RR_F64: launch_lift_slices<double>(s, n, ip1, (const double*)S1, ld1, ip2, t2, S2, ld2, rexp, Acat); break;
    case RR_F32: launch_lift_slices<float>(s, n, ip1, (const float*)S1, ld1, ip2, t2, S2, ld2, rexp, Acat); break;
    case RR_E4M3:
      launch_lift_slices<e4m3b_t>(s, n, ip1, (const e4m3b_t*)S1, ld1, ip2, t2, S2, ld2, rexp, Acat);
      break;
    case RR_BF16:
      launch_lift_slices<__nv_bfloat16>(s, n, ip1, (const __nv_bfloat16*)S1, ld1, ip2, t2, S2, ld2, rexp, Acat);
      break;
    default: return RR_ERR_ARG;
  }
  k_col_exp<<<(unsigned)b, 512, 0, s>>>(K, Y, ldy, yexp);
  k_slice_cols_rev<<<dim3((unsigned)((K + 255) / 256), (unsigned)b), 256, 0, s>>>(K, b, Y, ldy, yexp, Yrev);
  dim3 gz((unsigned)std::min<int64_t>((n + 255) / 256, 1024), (unsigned)b);
  if (!accumulate) k_zero_f64<<<gz, 256, 0, s>>>(n, b, X, ldx);
  note_launches(accumulate ? 2 : 3);
  RR_TRY(check_launch("lift_emu slices"));
  uint32_t codes[S];
  for (int d = 2; d <= S + 1; ++d)
    codes[d - 2] = (uint32_t)(d - 2) | (1u << 16);  // p0 = d - 2, q0 = 0, nq = 1: scale 2^(-6d)
  if (K % 64 == 0) {
    // every diagonal in one launch (pair-major: the diagonals of a row tile
    // share its A_cat tiles in L2), adding into X with FP64 atomics
    TcEmu e{X, ldx, nullptr, rexp, yexp, (int)b, 1, 1, 0, 0, S, codes, 4096, (int)K, S};
    RR_TRY(gemm_bf16_tc_emu(n, b, S * K, Acat, S * K, Yrev, S * K, e, s));
  } else {
    for (int d = 2; d <= S + 1; ++d) {
      TcEmu e{X, ldx, nullptr, rexp, yexp, (int)b, 1, 1, 0, 0, 1, codes + (d - 2), 4096};
      RR_TRY(gemm_bf16_tc_emu(n, b, (d - 1) * K, Acat, S * K, Yrev + (size_t)(S - d + 1) * K, S * K, e, s));
    }
  }
  *done = true;
  return RR_OK;
}

// ---------------------------------------------------------------------------
// FP64-accurate Gram products G = X^T Y (X n x p, Y n x q, any storage type)
// on the tensor cores: both operands sliced by columns, every slice pair in
// one launch with exact FP32 sums over K chunks, FP64 partials per (pair, K
// chunk), then a fixed-order FP64 reduction.
// ---------------------------------------------------------------------------
__global__ void k_emu_reduce(int64_t p, int64_t q, int64_t nparts, const double* __restrict__ part,
                             double* __restrict__ G, int64_t ldg, int accum) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= p * q) return;
  double s = 0.0;
  for (int64_t c = 0; c < nparts; ++c) s += part[c * p * q + e];
  const int64_t i = e % p, j = e / p;
  if (accum) s += G[i + j * ldg];
  G[i + j * ldg] = s;
}


static int emu_gram_npairs() {
  uint32_t pr[64];
  return emu_pairs(kGramSlices, true, pr);
}

bool emu_gram_supported(int64_t n, int64_t p, int64_t q) {
  return n >= 64 && n % 8 == 0 && p >= 1 && q >= 1 && p <= 4096 && q <= 128 && n <= ((int64_t)1 << 30);
}

// Workspace of emu_gram, monotone in n, p and q (so one size serves every
// smaller call): slices of both operands, exponents, and the partials for the
// largest K-split count a launch of this size can take.
size_t emu_gram_bytes(int64_t n, int64_t p, int64_t q) {
  const int S = kGramSlices;
  const int64_t np = emu_gram_npairs();
  const int64_t nk = (n + 63) / 64;
  const int64_t kmin = (n + kGramKChunk - 1) / kGramKChunk;
  int64_t smax = (num_sms() + np - 1) / np;
  if (smax < kmin) smax = kmin;
  if (smax > nk) smax = nk;
  return align_up((size_t)S * n * p * 2) + align_up((size_t)S * n * q * 2) + align_up((size_t)p * 4) +
         align_up((size_t)q * 4) + align_up((size_t)(np * smax) * p * q * 8) + 256;
}

static void emu_slice_any(cudaStream_t s, int32_t t, int64_t n, int64_t c, const void* X, int64_t ldx,
                          int* e, __nv_bfloat16* out) {
  switch (t) {
    case RR_F64: emu_slice_block<double>(s, n, c, (const double*)X, ldx, e, out); break;
    case RR_F32: emu_slice_block<float>(s, n, c, (const float*)X, ldx, e, out); break;
    case RR_E4M3: emu_slice_block<e4m3b_t>(s, n, c, (const e4m3b_t*)X, ldx, e, out); break;
    default: emu_slice_block<__nv_bfloat16>(s, n, c, (const __nv_bfloat16*)X, ldx, e, out); break;
  }
}

rr_status emu_gram(cudaStream_t s, int64_t n, int64_t p, int64_t q, int32_t xt, const void* X, int64_t ldx,
                   int32_t yt, const void* Y, int64_t ldy, double* G, int64_t ldg, int accum, void* mem,
                   size_t bytes) {
  if (!emu_gram_supported(n, p, q)) return RR_ERR_ARG;
  if (bytes < emu_gram_bytes(n, p, q) || !mem) return RR_ERR_WORKSPACE;
  const int S = kGramSlices;
  Arena ar(mem, bytes);
  __nv_bfloat16* Xs = (__nv_bfloat16*)ar.take_bytes((size_t)S * n * p * 2);
  __nv_bfloat16* Ys = (__nv_bfloat16*)ar.take_bytes((size_t)S * n * q * 2);
  int* ex = ar.take<int>(p);
  int* ey = ar.take<int>(q);
  uint32_t pairs[64];
  const int np = emu_pairs(S, true, pairs);
  const int splits = tc_emu_partial_splits(p, n, np, kGramKChunk);
  double* part = ar.take<double>((size_t)np * splits * p * q);
  if (ar.overflow) return RR_ERR_WORKSPACE;
  emu_slice_any(s, xt, n, p, X, ldx, ex, Xs);
  const bool same = X == Y && xt == yt && ldx == ldy && p == q;  // X^T X: slice once
  if (!same) emu_slice_any(s, yt, n, q, Y, ldy, ey, Ys);
  note_launches(same ? 1 : 3);
  RR_TRY(check_launch("emu_gram slices"));
  TcEmu e{nullptr, 0, part, ex, same ? ex : ey, (int)q, S, S, (int)p, (int)q, np, pairs, kGramKChunk};
  RR_TRY(gemm_bf16_tc_emu(p, 2 * q, n, Xs, n, same ? Xs : Ys, n, e, s));
  k_emu_reduce<<<(unsigned)((p * q + 255) / 256), 256, 0, s>>>(p, q, (int64_t)np * splits, part, G, ldg, accum);
  return check_launch("emu_gram reduce");
}

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_split_operator(int64_t m, int64_t n, const double* A, int64_t lda, void* hi_col,
                                       void* hi_row, void* lo_col, void* lo_row, void* stream) {
  if (m < 0 || n < 0 || lda < m || !A) return RR_ERR_ARG;
  return op_prepare(as_stream(stream), A, m, n, lda, (__nv_bfloat16*)hi_col, (__nv_bfloat16*)hi_row,
                    (__nv_bfloat16*)lo_col, (__nv_bfloat16*)lo_row, 0, nullptr, nullptr, false, false);
}

extern "C" size_t rr_lift_workspace_size(int64_t n, int64_t b, int64_t K) {
  if (n < 0 || b < 0 || K < 0) return 0;
  return lift_emu_bytes(n, b, K);
}

extern "C" rr_status rr_lift(int64_t n, int64_t b, int32_t t1, const void* S1, int64_t ld1, int64_t p1,
                             int32_t t2, const void* S2, int64_t ld2, int64_t p2, const double* Y, int64_t ldy,
                             double* X, int64_t ldx, void* ws, size_t ws_bytes, void* stream) {
  auto ok_type = [](int32_t t) { return t == RR_F64 || t == RR_F32 || t == RR_BF16; };
  if (n < 0 || b < 1 || p1 < 1 || !S1 || !Y || !X || !ok_type(t1) || ld1 < n || ldx < n) return RR_ERR_ARG;
  if (S2 && (p2 < 0 || !ok_type(t2) || ld2 < n)) return RR_ERR_ARG;
  const int64_t p2e = S2 ? p2 : 0;
  if (ldy < p1 + p2e) return RR_ERR_ARG;
  if (n == 0) return RR_OK;
  cudaStream_t s = as_stream(stream);
  bool done = false;
  RR_TRY(lift_emu(s, n, b, t1, S1, ld1, p1, t2, S2, ld2, p2e, Y, ldy, X, ldx, ws, ws_bytes, &done));
  if (done) return RR_OK;
  RR_TRY(lift(s, t1, n, b, p1, S1, ld1, Y, ldy, X, ldx, 0));
  if (S2 && p2e > 0) RR_TRY(lift(s, t2, n, b, p2e, S2, ld2, Y + p1, ldy, X, ldx, 1));
  return RR_OK;
}

extern "C" size_t rr_gemm_f64_emulated_workspace_size(int32_t trans, int64_t M, int64_t N, int64_t K,
                                                      int32_t slices) {
  const int64_t m = trans ? K : M, n = trans ? M : K;
  return emu_operator_bytes(m, n, slices, !trans, trans != 0) + emu_block_bytes(K, N, slices) + 512;
}

extern "C" rr_status rr_gemm_f64_emulated(int32_t trans, int64_t M, int64_t N, int64_t K, const double* A,
                                          int64_t lda, const double* B, int64_t ldb, double* C,
                                          int64_t ldc, int32_t slices, void* ws, size_t ws_bytes,
                                          void* stream) {
  if (M <= 0 || N <= 0 || N > 256 || K <= 0 || !A || !B || !C || ldb < K || ldc < M) return RR_ERR_ARG;
  if (slices < 1 || slices > kMaxSlices) return RR_ERR_ARG;
  if (trans ? lda < K : lda < M) return RR_ERR_ARG;
  const int64_t m = trans ? K : M, n = trans ? M : K;
  if (!ws || ws_bytes < rr_gemm_f64_emulated_workspace_size(trans, M, N, K, slices)) return RR_ERR_WORKSPACE;
  if (n % 8 || m % 8) return RR_ERR_ARG;  // 16-byte row strides of the BF16 slices (TMA)
  cudaStream_t s = as_stream(stream);
  EmuOperator op;
  const size_t ob = emu_operator_bytes(m, n, slices, !trans, trans != 0);
  RR_TRY(emu_prepare(s, A, m, n, lda, slices, op, ws, !trans, trans != 0));
  return emu_gemm(s, op, trans, N, B, ldb, C, ldc, (char*)ws + align_up(ob));
}
