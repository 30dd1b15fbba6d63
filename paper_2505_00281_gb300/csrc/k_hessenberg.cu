// Algorithm 8: the right-looking Hessenberg process for a block (Sec. 4.2.2),
// the paper's inner-product-free basis step.  Its output equals P^T L of
// row-pivoted LU.
//
// GB300 design: one cooperative launch; each CTA owns a contiguous slab of
// rows (kept in shared memory when it fits).  Per column j:
//   (a) every CTA finds the largest |W(r, j)| in its slab (first index on
//       ties) and publishes (value, row) plus that row's trailing entries,
//       then releases its flag (step j + 1);
//   (b) every CTA acquires all flags (bounded wait) — an all-gather, not a
//       barrier followed by reads;
//   (c) every CTA reduces the published candidates itself and gets the
//       pivot r, W(r, j) and the weights W(r, j+1:k);
//   (d) every CTA scales its part of column j by 1/W(r, j) and applies the
//       rank-1 update to its rows of the trailing columns.
// The candidate buffers are double-buffered by column parity so no CTA can
// overwrite a buffer another CTA still reads.  Arithmetic: IEEE divide,
// multiply and subtract, each rounded separately (no FMA contraction), so the
// result is bit-reproducible and equals a plain FP32/FP64 loop.
#include <climits>
#include <type_traits>

#include <cooperative_groups.h>

#include "rr_common.cuh"

namespace rr {

template <typename T>
struct HessWs {
  int* err;
  GridBarrier* bar;
  T* pval;      // [2][G] signed candidate pivot value
  int* pidx;    // [2][G] candidate row
  T* prow;      // [2][G][k] candidate row's entries
  T* pcolmax;   // [G][k] per-slab column inf-norms
  int* flags;   // [G] column steps published by each CTA (j + 1 after column j)
  unsigned long long* cand;  // [2][G] packed candidates (FP32 path)
  int64_t rpc;               // rows per CTA (FP32 path; 0: ceil(n / G))
  const T* colmax_ext;       // [k] column inf-norms on entry to the whole process
                             // (the blocked process's panels), or null: computed here
};

// Publish/await the per-column candidates: CTA g releases flags[g] = step once
// its candidate is written; readers acquire every flag before reading.
__device__ __forceinline__ void flag_release(int* f, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(f), "r"(v) : "memory");
}
__device__ __forceinline__ void word_release(unsigned long long* f, unsigned long long v) {
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(f), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long word_acquire(const unsigned long long* f) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(f) : "memory");
  return v;
}
__device__ __forceinline__ int flag_acquire(const int* f) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
  return v;
}

// the same exchange through distributed shared memory (one thread-block
// cluster): release / acquire at cluster scope on generic addresses
// (the publishing lanes' row writes reach the releasing lane through
// __syncwarp; a release store is cumulative over them)
__device__ __forceinline__ void word_release_cl(unsigned long long* f, unsigned long long v) {
  asm volatile("st.release.cluster.b64 [%0], %1;" ::"l"(f), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long word_acquire_cl(const unsigned long long* f) {
  unsigned long long v;
  asm volatile("ld.acquire.cluster.b64 %0, [%1];" : "=l"(v) : "l"(f) : "memory");
  return v;
}

template <typename T> __device__ __forceinline__ T ld_cg(const T* p);
template <> __device__ __forceinline__ float ld_cg<float>(const float* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double ld_cg<double>(const double* p) { return __ldcg(p); }
__device__ __forceinline__ int ld_cg_i(const int* p) { return __ldcg(p); }

template <typename T> __device__ __forceinline__ T rn_div(T a, T b);
template <> __device__ __forceinline__ float rn_div<float>(float a, float b) { return __fdiv_rn(a, b); }
template <> __device__ __forceinline__ double rn_div<double>(double a, double b) { return __ddiv_rn(a, b); }
template <typename T> __device__ __forceinline__ T rn_mul(T a, T b);
template <> __device__ __forceinline__ float rn_mul<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ double rn_mul<double>(double a, double b) { return __dmul_rn(a, b); }
template <typename T> __device__ __forceinline__ T rn_sub(T a, T b);
template <> __device__ __forceinline__ float rn_sub<float>(float a, float b) { return __fsub_rn(a, b); }
template <> __device__ __forceinline__ double rn_sub<double>(double a, double b) { return __dsub_rn(a, b); }

// (|v|, idx) with "larger |v| wins, then smaller idx"
template <typename T>
__device__ __forceinline__ void argmax_merge(T& av, int& ai, T bv, int bi) {
  if (bv > av || (bv == av && bi < ai)) {
    av = bv;
    ai = bi;
  }
}

constexpr int kHessThreads = 512;

// The kernel works on "Wv": the CTA's slab of W, either in shared memory
// (slab mode: rows r0..r1 of all k columns, column-major with ld = rows per
// CTA; loaded once, written back at the end) or W itself in global memory.
//
// Look-ahead: after the pivot of column j is known, a CTA scales column j,
// updates column j+1 only, picks and publishes its candidate for column j+1
// (the candidate row's trailing entries get the same rank-1 update, computed
// with the same operations), and only then applies the rank-1 update to
// columns j+2.. — so that update overlaps the other CTAs' progress instead of
// sitting on the per-column critical path.  Loop indices are 32-bit: lanes run
// over rows (consecutive addresses), warps over columns.
template <typename T, typename TO>
__global__ void __launch_bounds__(kHessThreads) k_hessenberg(
    int64_t n, int k, T* __restrict__ W, int64_t ldw, TO* __restrict__ Q, int64_t ldq,
    int* __restrict__ piv, T tol, HessWs<T> ws, int slab) {
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = kHessThreads / 32;
  const int64_t rpc = (n + G - 1) / G;
  const int64_t r0 = (int64_t)g * rpc;
  const int64_t r1 = r0 + rpc < n ? r0 + rpc : n;
  const int nr = r1 > r0 ? (int)(r1 - r0) : 0;

  extern __shared__ unsigned char smem_raw[];
  T* thr = reinterpret_cast<T*>(smem_raw);   // [k]
  T* wgt = thr + k;                          // [k]
  T* slabp = wgt + k;                        // [k][rpc] in slab mode
  // column c of this CTA's rows: col(c)[i], i = 0..nr-1 (row r0 + i)
  T* const base = slab ? slabp : W + r0;
  const int64_t ldv = slab ? rpc : ldw;
  auto col = [&](int c) -> T* { return base + (int64_t)c * ldv; };
  if (slab) {
    for (int c = warp; c < k; c += nwarps) {
      const T* src = W + r0 + (int64_t)c * ldw;
      T* dst = col(c);
      for (int i = lane; i < nr; i += 32) dst[i] = src[i];
    }
    __syncthreads();
  }
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  __shared__ T s_qr;
  __shared__ int s_r, s_win, s_keep;

  // ---- column inf-norms on entry (relative skip threshold) ----
  for (int c = warp; c < k; c += nwarps) {
    T m = T(0);
    const T* cc = col(c);
    for (int i = lane; i < nr; i += 32) m = fmax(m, fabs(cc[i]));
    m = warp_max(m);
    if (lane == 0) ws.pcolmax[(size_t)g * k + c] = m;
  }
  if (!grid_barrier(ws.bar, G, ws.err)) return;
  for (int c = tid; c < k; c += kHessThreads) {
    T m = T(0);
    for (int h = 0; h < G; ++h) m = fmax(m, ld_cg(ws.pcolmax + (size_t)h * k + c));
    thr[c] = rn_mul(tol, m);
  }
  __syncthreads();

  // local argmax of |column jc| over this CTA's rows, then publish the
  // candidate (value, global row, row entries jc+1..k-1).  When upd is set,
  // the row entries are published as they will be after the pending rank-1
  // update by column jc-1 (weights wgt, multiplier column jc-1).
  auto publish = [&](int jc, bool upd) {
    const int par = jc & 1;
    const T* cj = col(jc);
    T bv = T(-1);
    int bi = INT_MAX;
    for (int i = tid; i < nr; i += kHessThreads) {
      T v = fabs(cj[i]);
      if (v > bv) {  // strictly greater: first index wins within a thread
        bv = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      argmax_merge(bv, bi, ov, oi);
    }
    if (lane == 0) {
      red_v[warp] = bv;
      red_i[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
      bv = lane < nwarps ? red_v[lane] : T(-1);
      bi = lane < nwarps ? red_i[lane] : INT_MAX;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        argmax_merge(bv, bi, ov, oi);
      }
      if (lane == 0) {
        s_r = bi;
        ws.pidx[par * G + g] = (bi != INT_MAX) ? (int)(r0 + bi) : INT_MAX;
        ws.pval[par * G + g] = (bi != INT_MAX) ? cj[bi] : T(0);
      }
    }
    __syncthreads();
    const int rl = s_r;
    T* prow = ws.prow + ((size_t)par * G + g) * k;
    if (rl != INT_MAX) {
      const T m = upd ? col(jc - 1)[rl] : T(0);
      for (int c = jc + 1 + tid; c < k; c += kHessThreads) {
        T v = col(c)[rl];
        if (upd) v = rn_sub(v, rn_mul(wgt[c], m));
        prow[c] = v;
      }
    } else {
      for (int c = jc + 1 + tid; c < k; c += kHessThreads) prow[c] = T(0);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      flag_release(ws.flags + g, jc + 1);
    }
  };

  publish(0, false);
  for (int j = 0; j < k; ++j) {
    const int par = j & 1;
    // (b) wait for every CTA's candidate for column j (bounded)
    if (warp == 0) {
      const uint64_t t0 = global_timer_ns();
      bool ok = true;
      for (int h = lane; h < G && ok; h += 32) {
        while (flag_acquire(ws.flags + h) < j + 1) {
          if (*(volatile int*)ws.err != 0 || global_timer_ns() - t0 > kWaitLimitNs) {
            atomicCAS(ws.err, 0, (int)RR_ERR_TIMEOUT);
            ok = false;
            break;
          }
        }
      }
      __syncwarp();
    }
    __syncthreads();
    if (*(volatile int*)ws.err != 0) return;
    // (c) global winner, computed redundantly by every CTA
    if (warp == 0) {
      T av = T(-1);
      int ai = INT_MAX, ag = -1;
      for (int h = lane; h < G; h += 32) {
        int hi = ld_cg_i(ws.pidx + par * G + h);
        T hv = fabs(ld_cg(ws.pval + par * G + h));
        if (hi == INT_MAX) continue;
        if (hv > av || (hv == av && hi < ai)) {
          av = hv;
          ai = hi;
          ag = h;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, av, o);
        int oi = __shfl_xor_sync(0xffffffffu, ai, o);
        int og = __shfl_xor_sync(0xffffffffu, ag, o);
        if (ov > av || (ov == av && oi < ai)) {
          av = ov;
          ai = oi;
          ag = og;
        }
      }
      if (lane == 0) {
        T qr = (ag >= 0) ? ld_cg(ws.pval + par * G + ag) : T(0);
        s_qr = qr;
        s_r = ai;
        s_win = ag;
        s_keep = (ag >= 0 && qr != T(0) && fabs(qr) >= thr[j]) ? 1 : 0;
        if (g == 0) piv[j] = s_keep ? ai : -1;
      }
    }
    __syncthreads();
    const bool keep = s_keep != 0;
    T* cj = col(j);
    // (d) scale column j, update column j+1, publish column j+1's candidate,
    // then update columns j+2..k-1
    if (keep) {
      const T qr = s_qr;
      const T* prow = ws.prow + ((size_t)par * G + s_win) * k;
      for (int c = j + 1 + tid; c < k; c += kHessThreads) wgt[c] = ld_cg(prow + c);
      for (int i = tid; i < nr; i += kHessThreads) cj[i] = rn_div(cj[i], qr);
      __syncthreads();
      if (j + 1 < k) {
        T* cn = col(j + 1);
        const T wn = wgt[j + 1];
        for (int i = tid; i < nr; i += kHessThreads) cn[i] = rn_sub(cn[i], rn_mul(wn, cj[i]));
      }
    } else {
      for (int i = tid; i < nr; i += kHessThreads) cj[i] = T(0);
    }
    __syncthreads();
    if (j + 1 < k) publish(j + 1, keep);
    if (keep) {
      for (int c = j + 2 + warp; c < k; c += nwarps) {
        T* cc = col(c);
        const T wc = wgt[c];
        for (int i = lane; i < nr; i += 32) cc[i] = rn_sub(cc[i], rn_mul(wc, cj[i]));
      }
    }
    __syncthreads();
  }
  // write the result in the requested storage type (and W itself in slab mode)
  for (int c = warp; c < k; c += nwarps) {
    const T* src = col(c);
    T* dw = W + r0 + (int64_t)c * ldw;
    TO* dq = Q + r0 + (int64_t)c * ldq;
    for (int i = lane; i < nr; i += 32) {
      const T v = src[i];
      if (slab) dw[i] = v;
      if ((void*)Q != (void*)W) dq[i] = from_f64<TO>((double)v);
    }
  }
}

// the block's argmax from the per-warp candidates (the same merge order as
// the warp-shuffle reduction, so every warp gets the same row)
template <typename T>
__device__ __forceinline__ int bi_of_block(const T* red_v, const int* red_i, int nwarps) {
  T bv = T(-1);
  int bi = INT_MAX;
  const int lane = threadIdx.x & 31;
  bv = lane < nwarps ? red_v[lane] : T(-1);
  bi = lane < nwarps ? red_i[lane] : INT_MAX;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T ov = __shfl_xor_sync(0xffffffffu, bv, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    argmax_merge(bv, bi, ov, oi);
  }
  return bi;
}

// FP32-arithmetic variant (the basis step of the low-precision path), same
// per-element arithmetic and results as k_hessenberg<float, TO>.  Two
// changes to the per-column exchange:
//   - a CTA's candidate is one 64-bit word (value bits, global row, column
//     tag), written with a single release store and double-buffered by column
//     parity, so the wait for the candidates also delivers them;
//   - warp 0 reduces and publishes the next candidate (its row's trailing
//     entries, updated, go both to the published copy and back to the slab)
//     while the other warps apply the rank-1 update to every other row.
// Needs n < 2^24 - 1 (row field of the word).
constexpr unsigned kNoRow = 0xFFFFFFu;

__device__ __forceinline__ unsigned long long pack_cand(float v, unsigned row, int col) {
  return ((unsigned long long)__float_as_uint(v) << 32) | ((unsigned long long)(row & 0xFFFFFFu) << 8) |
         (unsigned long long)((col + 1) & 0xFF);
}

// Block argmax of (|value|, local row) with ties to the lower row as one
// 64-bit key: |value| bits above the complemented row (0: no candidate;
// value < 0 marks "none", NaN never wins).  A warp reduces with redux.sync,
// lane 0 folds the warp's key into a shared atomicMax.
__device__ __forceinline__ unsigned long long am_key(float av, int row) {
  return av >= 0.f ? ((unsigned long long)__float_as_uint(av) << 32) | (unsigned)(~row) : 0ull;
}
__device__ __forceinline__ unsigned long long warp_key_max(unsigned long long key) {
  const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
  const unsigned mhi = __reduce_max_sync(0xffffffffu, hi);
  const unsigned mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  return ((unsigned long long)mhi << 32) | mlo;
}

// CL: the CTAs form one thread-block cluster (G <= kHessMaxCluster): the
// candidate words and rows go through distributed shared memory instead of
// global memory (the same arithmetic, pivots and results).
constexpr int kHessMaxCluster = 16;

template <typename TO, bool CL>
__global__ void __launch_bounds__(kHessThreads) k_hessenberg_f32(
    int64_t n, int k, float* __restrict__ W, int64_t ldw, TO* __restrict__ Q, int64_t ldq,
    int* __restrict__ piv, float tol, HessWs<float> ws, int slab) {
  using T = float;
  namespace cg = cooperative_groups;
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = kHessThreads / 32;
  const int64_t rpc = ws.rpc > 0 ? ws.rpc : (n + G - 1) / G;
  const int64_t r0 = (int64_t)g * rpc;
  const int64_t r1 = r0 + rpc < n ? r0 + rpc : n;
  const int nr = r1 > r0 ? (int)(r1 - r0) : 0;

  extern __shared__ unsigned char smem_raw[];
  // cluster exchange buffers first (8-byte aligned): candidate words
  // [2][kHessMaxCluster], candidate rows [2][k], column maxima [k]
  unsigned long long* cw = reinterpret_cast<unsigned long long*>(smem_raw);
  T* prs = reinterpret_cast<T*>(cw + (CL ? 2 * kHessMaxCluster : 0));
  T* cmx = prs + (CL ? 2 * k : 0);
  T* thr = cmx + (CL ? k : 0);               // [k]
  T* wgt = thr + k;                          // [2][k] weights, by column parity
  // [k][ldv] in slab mode, 16-byte aligned; with rpc a multiple of 128 the
  // stride is rpc + 4 (column starts 4 banks apart: the candidate row's
  // entries, read across columns, meet 4-way instead of 32-way conflicts)
  // and the rank-1 update moves float4 chunks
  T* slabp = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(wgt + 2 * k) + 15) & ~(uintptr_t)15);
  T* const base = slab ? slabp : W + r0;
  const bool vec = slab && rpc % 128 == 0 && rpc <= 512;
  const int64_t ldv = slab ? (vec ? rpc + 4 : rpc) : ldw;
  auto col = [&](int c) -> T* { return base + (int64_t)c * ldv; };
  if constexpr (CL) {
    // word slots start at 0 (no column tag); the cluster barrier below orders
    // this before any other CTA's first word
    for (int i = tid; i < 2 * kHessMaxCluster; i += kHessThreads) cw[i] = 0ull;
  }
  if (slab) {
    for (int c = warp; c < k; c += nwarps) {
      const T* src = W + r0 + (int64_t)c * ldw;
      T* dst = col(c);
      for (int i = lane; i < (int)ldv; i += 32) dst[i] = i < nr ? src[i] : T(0);  // zero padding rows
    }
    __syncthreads();
  }
  __shared__ T red_v[32];
  __shared__ int red_i[32];
  __shared__ T s_qr;
  __shared__ int s_r, s_keep;
  __shared__ unsigned long long s_key[2];  // block argmax keys, by column parity
  if (tid < 2) s_key[tid] = 0ull;

  for (int c = warp; c < k; c += nwarps) {
    T m = T(0);
    const T* cc = col(c);
    for (int i = lane; i < nr; i += 32) m = fmax(m, fabs(cc[i]));
    m = warp_max(m);
    if (lane == 0) {
      if constexpr (CL) cmx[c] = m;
      else ws.pcolmax[(size_t)g * k + c] = m;
    }
  }
  if constexpr (CL) {
    cg::this_cluster().sync();
    for (int c = tid; c < k; c += kHessThreads) {
      T m = T(0);
      for (int h = 0; h < G; ++h) m = fmax(m, cg::this_cluster().map_shared_rank(cmx, h)[c]);
      thr[c] = rn_mul(tol, ws.colmax_ext ? ws.colmax_ext[c] : m);
    }
  } else {
    if (!grid_barrier(ws.bar, G, ws.err)) return;
    for (int c = tid; c < k; c += kHessThreads) {
      T m = T(0);
      for (int h = 0; h < G; ++h) m = fmax(m, ld_cg(ws.pcolmax + (size_t)h * k + c));
      thr[c] = rn_mul(tol, ws.colmax_ext ? ws.colmax_ext[c] : m);
    }
  }
  __syncthreads();

  // local argmax of |column jc| (first index on ties) -> s_r (local row or
  // INT_MAX); two CTA barriers
  auto local_argmax = [&](int jc) {
    const T* cj = col(jc);
    T bv = T(-1);
    int bi = INT_MAX;
    for (int i = tid; i < nr; i += kHessThreads) {
      T v = fabs(cj[i]);
      if (v > bv) {
        bv = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, bv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      argmax_merge(bv, bi, ov, oi);
    }
    if (lane == 0) {
      red_v[warp] = bv;
      red_i[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
      bv = lane < nwarps ? red_v[lane] : T(-1);
      bi = lane < nwarps ? red_i[lane] : INT_MAX;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        argmax_merge(bv, bi, ov, oi);
      }
      if (lane == 0) s_r = bi;
    }
    __syncthreads();
  };
  // warp 0: publish the candidate of column jc (row rl): its entries jc+1..
  // after the pending update by column jc-1 (upd) go to the published row and
  // back to the slab; then the packed word
  auto publish_w0 = [&](int jc, bool upd, int rl) {
    const int par = jc & 1;
    T* prow = CL ? prs + (size_t)par * k : ws.prow + ((size_t)par * G + g) * k;
    if (rl != INT_MAX) {
      const T m = upd ? col(jc - 1)[rl] : T(0);
      for (int c = jc + 1 + lane; c < k; c += 32) {
        T v = col(c)[rl];
        if (upd) {
          v = rn_sub(v, rn_mul(wgt[c], m));
          col(c)[rl] = v;
        }
        prow[c] = v;
      }
    }
    __syncwarp();
    if constexpr (CL) {
      if (lane < G) {  // into every CTA's word slot g
        const T v = rl != INT_MAX ? col(jc)[rl] : T(0);
        const unsigned row = rl != INT_MAX ? (unsigned)(r0 + rl) : kNoRow;
        word_release_cl(cg::this_cluster().map_shared_rank(cw + par * kHessMaxCluster + g, lane),
                        pack_cand(v, row, jc));
      }
    } else if (lane == 0) {
      const T v = rl != INT_MAX ? col(jc)[rl] : T(0);
      const unsigned row = rl != INT_MAX ? (unsigned)(r0 + rl) : kNoRow;
      __threadfence();
      word_release(ws.cand + (size_t)par * G + g, pack_cand(v, row, jc));
    }
  };

  // warp 0: wait (bounded) for every CTA's word for column jc, reduce to the
  // pivot, and load the pivot row's entries jc+1.. into the weight buffer of
  // column jc's parity; returns false on error
  auto await_pivot = [&](int jc) -> bool {
    const int par = jc & 1;
    const unsigned tag = (unsigned)((jc + 1) & 0xFF);
    const uint64_t t0 = global_timer_ns();
    T av = T(-1), sv = T(0);
    int ai = INT_MAX, ag = -1;
    bool ok = true;
    for (int h = lane; h < G; h += 32) {
      unsigned long long wv;
      while (((wv = CL ? word_acquire_cl(cw + par * kHessMaxCluster + h)
                       : word_acquire(ws.cand + (size_t)par * G + h)) & 0xFFull) != tag) {
        if (*(volatile int*)ws.err != 0 || global_timer_ns() - t0 > kWaitLimitNs) {
          atomicCAS(ws.err, 0, (int)RR_ERR_TIMEOUT);
          ok = false;
          break;
        }
      }
      if (!ok) break;
      const unsigned row = (unsigned)((wv >> 8) & 0xFFFFFFull);
      if (row == kNoRow) continue;
      const T hv = __uint_as_float((unsigned)(wv >> 32));
      const T ah = fabs(hv);
      if (ah > av || (ah == av && (int)row < ai)) {
        av = ah;
        ai = (int)row;
        ag = h;
        sv = hv;
      }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) return false;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T ov = __shfl_xor_sync(0xffffffffu, av, o);
      int oi = __shfl_xor_sync(0xffffffffu, ai, o);
      int og = __shfl_xor_sync(0xffffffffu, ag, o);
      T osv = __shfl_xor_sync(0xffffffffu, sv, o);
      if (ov > av || (ov == av && oi < ai)) {
        av = ov;
        ai = oi;
        ag = og;
        sv = osv;
      }
    }
    const bool kp = ag >= 0 && sv != T(0) && fabs(sv) >= thr[jc];
    if (kp) {
      T* wb = wgt + (size_t)par * k;
      if constexpr (CL) {
        __syncwarp();  // the acquiring lane's order for the whole warp
        const T* prow = cg::this_cluster().map_shared_rank(prs + (size_t)par * k, ag);
        for (int c = jc + 1 + lane; c < k; c += 32) wb[c] = prow[c];
      } else {
        const T* prow = ws.prow + ((size_t)par * G + ag) * k;
        for (int c = jc + 1 + lane; c < k; c += 32) wb[c] = ld_cg(prow + c);
      }
    }
    if (lane == 0) {
      s_qr = sv;
      s_keep = kp ? 1 : 0;
      if (g == 0) piv[jc] = kp ? ai : -1;
    }
    return true;
  };

  __shared__ int s_ok;
  local_argmax(0);
  if (warp == 0) {
    publish_w0(0, false, s_r);
    const bool ok = await_pivot(0);
    if (lane == 0) s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  bool failed = !s_ok;
  for (int j = 0; j < k && !failed; ++j) {
    const bool keep = s_keep != 0;
    const T qr = s_qr;
    const T* wj = wgt + (size_t)(j & 1) * k;  // weights of column j
    T* cj = col(j);
    // (d) scale column j and update column j+1 row by row, tracking the local
    // argmax of the new column j+1 (first index on ties)
    {
      T* cn = j + 1 < k ? col(j + 1) : nullptr;
      const T wn = (keep && cn) ? wj[j + 1] : T(0);
      T bv = T(-1);
      int bi = INT_MAX;
      for (int i = tid; i < nr; i += kHessThreads) {
        T v = T(0);
        if (keep) v = rn_div(cj[i], qr);
        cj[i] = v;
        if (cn) {
          T u = cn[i];
          if (keep) u = rn_sub(u, rn_mul(wn, v));
          cn[i] = u;
          const T au = fabs(u);
          if (au > bv) {
            bv = au;
            bi = i;
          }
        }
      }
      const unsigned long long wk = warp_key_max(am_key(bv, bi));
      if (lane == 0 && wk) atomicMax(&s_key[j & 1], wk);
    }
    __syncthreads();
    const unsigned long long bkey = s_key[j & 1];
    const int bcand = bkey ? (int)(~(unsigned)bkey) : INT_MAX;  // the CTA's candidate row
    if (tid == 0) s_key[(j + 1) & 1] = 0ull;                    // read last in step j - 1
    if (j + 1 < k) {
      if (warp == 0) {
        // publish the candidate (its row takes column j's pending update,
        // written back to the slab), then wait for the pivot of column j+1
        // while the other warps apply column j's update
        const int rl = bcand;
        const int par = (j + 1) & 1;
        T* prow = CL ? prs + (size_t)par * k : ws.prow + ((size_t)par * G + g) * k;
        if (rl != INT_MAX) {
          const T m = cj[rl];
          for (int c = j + 2 + lane; c < k; c += 32) {
            T v = col(c)[rl];
            if (keep) {
              v = rn_sub(v, rn_mul(wj[c], m));
              col(c)[rl] = v;
            }
            prow[c] = v;
          }
        }
        __syncwarp();
        if constexpr (CL) {
          if (lane < G) {
            const T v = rl != INT_MAX ? col(j + 1)[rl] : T(0);
            const unsigned row = rl != INT_MAX ? (unsigned)(r0 + rl) : kNoRow;
            word_release_cl(cg::this_cluster().map_shared_rank(cw + par * kHessMaxCluster + g, lane),
                            pack_cand(v, row, j + 1));
          }
        } else if (lane == 0) {
          const T v = rl != INT_MAX ? col(j + 1)[rl] : T(0);
          const unsigned row = rl != INT_MAX ? (unsigned)(r0 + rl) : kNoRow;
          __threadfence();
          word_release(ws.cand + (size_t)par * G + g, pack_cand(v, row, j + 1));
        }
        // the published candidate is what the other CTAs wait for: the bulk
        // update starts only now, so its shared-memory traffic does not delay it
        asm volatile("bar.arrive 1, %0;" ::"r"(kHessThreads) : "memory");
        const bool ok = await_pivot(j + 1);
        if (lane == 0) s_ok = ok ? 1 : 0;
      } else {
        asm volatile("bar.sync 1, %0;" ::"r"(kHessThreads) : "memory");
      }
      if (warp != 0 && keep) {
        // rank-1 update of columns j+2.. (all rows but the candidate's, which
        // warp 0 updates): the multiplier column in registers, independent
        // loads per target column
        const T* cj_c = cj;
        const int rl = bcand;
        constexpr int kR = 16;  // rows per lane held in registers (nr <= 512)
        // float4 chunks: lane rows 4 lane + 128 t (t < NC = rpc / 128); the
        // padding rows beyond nr are zero and stay finite
        auto upd4 = [&](auto nc) {
          constexpr int NC = decltype(nc)::value;
          float4 xr[NC];
#pragma unroll
          for (int t = 0; t < NC; ++t) xr[t] = reinterpret_cast<const float4*>(cj_c)[lane + 32 * t];
          for (int c = j + 2 + (warp - 1); c < k; c += nwarps - 1) {
            float4* cc = reinterpret_cast<float4*>(col(c));
            const T wc = wj[c];
            float4 yv[NC];
#pragma unroll
            for (int t = 0; t < NC; ++t) yv[t] = cc[lane + 32 * t];
#pragma unroll
            for (int t = 0; t < NC; ++t) {
              const int i0 = 4 * lane + 128 * t;
              float4 o = yv[t];
              o.x = i0 == rl ? yv[t].x : rn_sub(yv[t].x, rn_mul(wc, xr[t].x));
              o.y = i0 + 1 == rl ? yv[t].y : rn_sub(yv[t].y, rn_mul(wc, xr[t].y));
              o.z = i0 + 2 == rl ? yv[t].z : rn_sub(yv[t].z, rn_mul(wc, xr[t].z));
              o.w = i0 + 3 == rl ? yv[t].w : rn_sub(yv[t].w, rn_mul(wc, xr[t].w));
              if ((rl >> 2) == lane + 32 * t) {
                // the candidate's chunk: warp 0 writes row rl concurrently,
                // so only the other three rows are stored
                float* cs = reinterpret_cast<float*>(cc + lane + 32 * t);
                if (i0 != rl) cs[0] = o.x;
                if (i0 + 1 != rl) cs[1] = o.y;
                if (i0 + 2 != rl) cs[2] = o.z;
                if (i0 + 3 != rl) cs[3] = o.w;
              } else {
                cc[lane + 32 * t] = o;
              }
            }
          }
        };
        if (vec) {
          switch (rpc / 128) {
            case 1: upd4(std::integral_constant<int, 1>{}); break;
            case 2: upd4(std::integral_constant<int, 2>{}); break;
            case 3: upd4(std::integral_constant<int, 3>{}); break;
            default: upd4(std::integral_constant<int, 4>{}); break;
          }
        } else if (nr <= 32 * kR) {
          T xr[kR];
#pragma unroll
          for (int t = 0; t < kR; ++t) {
            const int i = lane + 32 * t;
            xr[t] = i < nr ? cj_c[i] : T(0);
          }
          for (int c = j + 2 + (warp - 1); c < k; c += nwarps - 1) {
            T* cc = col(c);
            const T wc = wj[c];
            T yv[kR];
#pragma unroll
            for (int t = 0; t < kR; ++t) {
              const int i = lane + 32 * t;
              yv[t] = i < nr ? cc[i] : T(0);
            }
#pragma unroll
            for (int t = 0; t < kR; ++t) {
              const int i = lane + 32 * t;
              if (i < nr && i != rl) cc[i] = rn_sub(yv[t], rn_mul(wc, xr[t]));
            }
          }
        } else {
          for (int c = j + 2 + (warp - 1); c < k; c += nwarps - 1) {
            T* cc = col(c);
            const T wc = wj[c];
            for (int i = lane; i < nr; i += 32)
              if (i != rl) cc[i] = rn_sub(cc[i], rn_mul(wc, cj_c[i]));
          }
        }
      }
      __syncthreads();
      if (!s_ok) failed = true;
    }
  }
  if constexpr (CL) {
    // no CTA leaves while another may still read its shared memory
    cg::this_cluster().sync();
  }
  if (failed) return;
  for (int c = warp; c < k; c += nwarps) {
    const T* src = col(c);
    T* dw = W + r0 + (int64_t)c * ldw;
    TO* dq = Q + r0 + (int64_t)c * ldq;
    for (int i = lane; i < nr; i += 32) {
      const T v = src[i];
      if (slab) dw[i] = v;
      if ((void*)Q != (void*)W) dq[i] = from_f32<TO>(v);
    }
  }
}

template <typename T>
static size_t hess_ws_bytes(int64_t k, int G) {
  size_t b = 0;
  b += align_up(sizeof(int));
  b += align_up(sizeof(GridBarrier));
  b += align_up(2 * (size_t)G * sizeof(T));
  b += align_up(2 * (size_t)G * sizeof(int));
  b += align_up(2 * (size_t)G * k * sizeof(T));
  b += align_up((size_t)G * k * sizeof(T));
  b += align_up((size_t)G * sizeof(int));
  b += align_up(2 * (size_t)G * sizeof(unsigned long long));
  return b;
}

template <typename T, typename TO>
static rr_status hess_launch(int64_t n, int64_t k, T* W, int64_t ldw, TO* Q, int64_t ldq, int* piv,
                             double tol, void* ws, size_t ws_bytes, cudaStream_t s, int max_grid,
                             const T* colmax_ext = nullptr, bool reset_err = true) {
  // FP32 arithmetic: the packed-candidate kernel (rows must fit its 24-bit field)
  const bool packed = sizeof(T) == 4 && n < (int64_t)kNoRow;
  const void* fn = packed ? (const void*)k_hessenberg_f32<TO, false> : (const void*)k_hessenberg<T, TO>;
  // Grid: about 256 rows per CTA (fewer CTAs make the per-column barrier and
  // candidate reduction cheaper), more CTAs if a slab would not fit in shared
  // memory; slab mode when the CTA's rows of all k columns fit in 200 KB.
  const size_t kSlabLimit = 200 * 1024;
  int G;
  int slab = 0;
  if (max_grid == 1) {
    G = 1;
  } else {
    int64_t g = (n + 255) / 256;
    const int64_t fit = (int64_t)(kSlabLimit / ((size_t)k * sizeof(T)));  // rows per CTA that fit
    if (fit > 0 && (n + g - 1) / g > fit) g = (n + fit - 1) / fit;
    if (g > num_sms()) g = num_sms();
    if (g < 1) g = 1;
    G = (int)g;
  }
  int64_t rpc = (n + G - 1) / G;
  if (packed) {
    // rows per CTA a multiple of 128 where the slab still fits: the FP32
    // kernel's float4 update and padded stride (fewer CTAs when it rounds up)
    const int64_t r128 = (rpc + 127) / 128 * 128;
    if (r128 <= 512 && (size_t)(r128 + 4) * k * sizeof(T) <= kSlabLimit) {
      rpc = r128;
      G = (int)((n + rpc - 1) / rpc);
    }
  }
  const int64_t ldv = (packed && rpc % 128 == 0 && rpc <= 512) ? rpc + 4 : rpc;
  const size_t fixed = (packed ? 3 : 2) * (size_t)k * sizeof(T) + 16;  // thresholds, weights, alignment
  if ((size_t)ldv * k * sizeof(T) <= kSlabLimit && (size_t)ldv * k * sizeof(T) + fixed <= 220 * 1024) slab = 1;
  size_t smem = fixed + (slab ? (size_t)ldv * k * sizeof(T) : 0);
  // one thread-block cluster when every CTA's rows fit in shared memory and
  // the CTAs fit one cluster: the exchange goes through distributed shared
  // memory (checked against the GPU's cluster occupancy; otherwise the
  // cooperative grid)
  bool cl = false;
  const size_t clbytes = 2 * kHessMaxCluster * sizeof(unsigned long long) + 3 * (size_t)k * sizeof(T);
  if (packed && slab && G <= kHessMaxCluster && smem + clbytes <= 227 * 1024) {
    const void* fcl = (const void*)k_hessenberg_f32<TO, true>;
    RR_CUDA(cudaFuncSetAttribute(fcl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem + clbytes)));
    if (G > 8) RR_CUDA(cudaFuncSetAttribute(fcl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3(G);
    q.blockDim = dim3(kHessThreads);
    q.dynamicSmemBytes = smem + clbytes;
    cudaLaunchAttribute qa[1];
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = G;
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.attrs = qa;
    q.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fcl, &q) == cudaSuccess && nclusters >= 1) {
      cl = true;
      fn = fcl;
      smem += clbytes;
    } else {
      (void)cudaGetLastError();
    }
  }
  if (smem > 48 * 1024)
    RR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (ws_bytes < hess_ws_bytes<T>(k, G) || !ws) return RR_ERR_WORKSPACE;
  Arena ar(ws, ws_bytes);
  HessWs<T> h;
  h.err = ar.take<int>(1);
  h.bar = ar.take<GridBarrier>(1);
  h.pval = ar.take<T>(2 * (size_t)G);
  h.pidx = ar.take<int>(2 * (size_t)G);
  h.prow = ar.take<T>(2 * (size_t)G * k);
  h.pcolmax = ar.take<T>((size_t)G * k);
  h.flags = ar.take<int>(G);
  h.cand = ar.take<unsigned long long>(2 * (size_t)G);
  h.rpc = packed ? rpc : 0;
  h.colmax_ext = packed ? colmax_ext : nullptr;
  if (reset_err) RR_CUDA(cudaMemsetAsync(ws, 0, 512, s));  // err + barrier
  RR_CUDA(cudaMemsetAsync(h.flags, 0, (size_t)G * sizeof(int), s));
  RR_CUDA(cudaMemsetAsync(h.cand, 0, 2 * (size_t)G * sizeof(unsigned long long), s));
  T t = tol > 0 ? (T)tol : (T)(4.0 * (double)k * (sizeof(T) == 4 ? 0x1p-23 : 0x1p-52));
  int kk = (int)k;
  void* args[] = {&n, &kk, &W, &ldw, &Q, &ldq, &piv, &t, &h, &slab};
  if (cl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kHessThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = G;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    RR_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
    note_launches(1);
    return RR_OK;
  }
  if (G == 1) {
    // a single CTA never waits on another one: plain launch (graph-capturable,
    // safe to run concurrently with other work)
    RR_CUDA(cudaLaunchKernel(fn, dim3(1), dim3(kHessThreads), args, smem, s));
    return check_launch("rr_hessenberg");
  }
  RR_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kHessThreads), args, smem, s));
  note_launches(1);
  return RR_OK;
}

// ---------------------------------------------------------------------------
// Blocked (level-3) Hessenberg process for blocks too tall for the slab
// kernel's shared memory (the panel form of Algorithm 8 that Table 1's "Block"
// row and the closing future-work passage point to).  Columns go in panels of
// r: the panel is factored by the right-looking kernel above on its r columns
// only (thresholds from the column norms on entry to the whole process), then
// the trailing columns T take the whole panel at once:
//   weights  w_j(c) = T(pi_j, c) - sum_{i < j} L(pi_j, i) w_i(c)   (forward
//            substitution with the panel's unit lower triangle at its pivot rows)
//   update   T(:, c) <- T(:, c) - sum_j L(:, j) w_j(c)
// Every entry sees the same operations in the same order as in the
// right-looking process (the weights are exactly the pivot-row entries it
// would read; each step a separately rounded multiply and subtract, j
// ascending), so the blocked result equals it bit for bit, while the trailing
// columns are streamed once per panel instead of once per column.
// ---------------------------------------------------------------------------
constexpr int kPanelMax = 32;

// colmax[c] = max_i |W(i, c)| (non-negative floats order like their bits):
// CTA (c, chunk) reduces 64K rows and merges with an atomic max
__global__ void k_hess_colmax(int64_t n, int k, const float* __restrict__ W, int64_t ldw,
                              unsigned* __restrict__ colmax_bits) {
  const int c = blockIdx.x;
  const int64_t i0 = (int64_t)blockIdx.y * 65536, i1 = i0 + 65536 < n ? i0 + 65536 : n;
  float m = 0.f;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) m = fmaxf(m, fabsf(W[i + c * ldw]));
  m = warp_max(m);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    atomicMax(colmax_bits + c, __float_as_uint(m));
  }
}

// weights of the panel (r columns at L, pivots piv[0..r)) for the nt trailing
// columns T: w[j * nt + c]; a skipped panel column (pivot -1) has weight 0
// and takes no part in the substitution.  One thread per trailing column.
__global__ void k_hess_weights(int r, int nt, const float* __restrict__ L, const float* __restrict__ T,
                               int64_t ldw, const int* __restrict__ piv, float* __restrict__ w) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nt) return;
  float wr[kPanelMax];
#pragma unroll
  for (int j = 0; j < kPanelMax; ++j) {
    if (j >= r) break;
    const int pj = piv[j];
    float v = 0.f;
    if (pj >= 0) {
      v = T[pj + (int64_t)c * ldw];
#pragma unroll
      for (int i = 0; i < kPanelMax; ++i) {
        if (i >= j) break;
        if (piv[i] >= 0) v = __fsub_rn(v, __fmul_rn(wr[i], L[pj + (int64_t)i * ldw]));
      }
    }
    wr[j] = v;
    w[(size_t)j * nt + c] = v;
  }
}

// T(i, c) <- T(i, c) - sum_j L(i, j) w_j(c), j ascending, every row i; one
// thread per row (grid-stride), the row's panel entries in registers, the
// weights in shared memory; column-major T and L (consecutive threads,
// consecutive rows)
template <int R>
__global__ void __launch_bounds__(256) k_hess_trail(int64_t n, int r, int nt, const float* __restrict__ L,
                                                    float* __restrict__ T, int64_t ldw, const float* __restrict__ w,
                                                    int wld, const int* __restrict__ piv) {
  extern __shared__ float sw[];  // [r][nt]
  __shared__ int keep[R];
  for (int e = threadIdx.x; e < r * nt; e += blockDim.x) sw[e] = w[(e / nt) * (size_t)wld + e % nt];
  if (threadIdx.x < R) keep[threadIdx.x] = (int)threadIdx.x < r && piv[threadIdx.x] >= 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float l[R];
#pragma unroll
    for (int j = 0; j < R; ++j) l[j] = (j < r) ? L[i + (int64_t)j * ldw] : 0.f;
    // 8 columns at a time: their loads go out together, then each column's
    // subtractions in panel order
    int c = 0;
    for (; c + 8 <= nt; c += 8) {
      float t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = T[i + (int64_t)(c + u) * ldw];
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (keep[j]) {
#pragma unroll
          for (int u = 0; u < 8; ++u) t[u] = __fsub_rn(t[u], __fmul_rn(sw[j * nt + c + u], l[j]));
        }
#pragma unroll
      for (int u = 0; u < 8; ++u) T[i + (int64_t)(c + u) * ldw] = t[u];
    }
    for (; c < nt; ++c) {
      float t = T[i + (int64_t)c * ldw];
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (keep[j]) t = __fsub_rn(t, __fmul_rn(sw[j * nt + c], l[j]));
      T[i + (int64_t)c * ldw] = t;
    }
  }
}

// The extra workspace of the blocked process, after the kernel's own part:
// column maxima (k) and panel weights (kPanelMax x k).
static size_t hess_blocked_extra(int64_t k) {
  return align_up((size_t)k * sizeof(float)) + align_up((size_t)kPanelMax * k * sizeof(float));
}

template <typename TO>
static rr_status hess_blocked(int64_t n, int64_t k, float* W, int64_t ldw, TO* Q, int64_t ldq, int* piv,
                              double tol, int r, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (r < 1 || r > kPanelMax) return RR_ERR_ARG;
  const size_t base = hess_ws_bytes<float>(k, num_sms());
  if (!ws || ws_bytes < base + hess_blocked_extra(k)) return RR_ERR_WORKSPACE;
  float* colmax = (float*)((char*)ws + base);
  float* wts = (float*)((char*)ws + base + align_up((size_t)k * sizeof(float)));
  RR_CUDA(cudaMemsetAsync(colmax, 0, (size_t)k * sizeof(float), s));
  k_hess_colmax<<<dim3((unsigned)k, (unsigned)((n + 65535) / 65536)), 256, 0, s>>>(n, (int)k, W, ldw,
                                                                                 (unsigned*)colmax);
  RR_TRY(check_launch("hessenberg colmax"));
  // the default tolerance scales with the whole block's width, as the
  // unblocked process's does
  const double t = tol > 0 ? tol : 4.0 * (double)k * 0x1p-23;
  for (int64_t c0 = 0; c0 < k; c0 += r) {
    const int64_t c1 = c0 + r < k ? c0 + r : k;
    const int pr = (int)(c1 - c0);
    const rr_status st = hess_launch<float, TO>(n, pr, W + c0 * ldw, ldw, Q + c0 * ldq, ldq, piv + c0, t, ws, base,
                                                s, 0, colmax + c0, c0 == 0);
    if (st != RR_OK) return st;
    if (c1 == k) break;
    const int nt = (int)(k - c1);
    k_hess_weights<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(pr, nt, W + c0 * ldw, W + c1 * ldw, ldw, piv + c0,
                                                               wts);
    RR_TRY(check_launch("hessenberg panel weights"));
    // trailing columns in chunks whose weights fit 96 KB of shared memory
    const int ncmax = (int)((96 * 1024) / ((size_t)pr * sizeof(float)));
    const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 8 * (int64_t)num_sms());
    for (int cc0 = 0; cc0 < nt; cc0 += ncmax) {
      const int ntc = nt - cc0 < ncmax ? nt - cc0 : ncmax;
      const size_t sm = (size_t)pr * ntc * sizeof(float);
      float* Tc = W + (c1 + cc0) * ldw;
      if (pr <= 16) {
        if (sm > 48 * 1024) RR_CUDA(cudaFuncSetAttribute(k_hess_trail<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_hess_trail<16><<<g, 256, sm, s>>>(n, pr, ntc, W + c0 * ldw, Tc, ldw, wts + cc0, nt, piv + c0);
      } else {
        if (sm > 48 * 1024) RR_CUDA(cudaFuncSetAttribute(k_hess_trail<kPanelMax>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_hess_trail<kPanelMax><<<g, 256, sm, s>>>(n, pr, ntc, W + c0 * ldw, Tc, ldw, wts + cc0, nt, piv + c0);
      }
      RR_TRY(check_launch("hessenberg trailing update"));
    }
  }
  return RR_OK;
}

// The blocked form replaces the slab kernel where a CTA's rows of all k
// columns do not fit its shared memory (the kernel would stream the whole
// trailing block once per column).
static bool hess_use_blocked(int64_t n, int64_t k, int max_grid) {
  if (max_grid == 1 || k <= 16 || n >= (int64_t)kNoRow) return false;
  const int64_t rpc = (n + num_sms() - 1) / num_sms();
  return (size_t)rpc * k * sizeof(float) > 200 * 1024;
}

}  // namespace rr

using namespace rr;

extern "C" size_t rr_hessenberg_workspace_size(int64_t n, int64_t k, int32_t arith) {
  int G = num_sms();
  return arith == RR_F64 ? hess_ws_bytes<double>(k, G) : hess_ws_bytes<float>(k, G) + hess_blocked_extra(k);
}

namespace rr {
rr_status hessenberg_ex(int32_t arith, int64_t n, int64_t k, void* W, int64_t ldw, int32_t qtype,
                        void* Q, int64_t ldq, int32_t* piv, double tol, void* ws, size_t ws_bytes,
                        cudaStream_t s, int max_grid);
}
extern "C" rr_status rr_hessenberg(int32_t arith, int64_t n, int64_t k, void* W, int64_t ldw,
                                   int32_t qtype, void* Q, int64_t ldq, int32_t* piv, double tol,
                                   void* ws, size_t ws_bytes, void* stream) {
  return hessenberg_ex(arith, n, k, W, ldw, qtype, Q, ldq, piv, tol, ws, ws_bytes,
                       as_stream(stream), 0);
}

rr_status rr::hessenberg_ex(int32_t arith, int64_t n, int64_t k, void* W, int64_t ldw,
                            int32_t qtype, void* Q, int64_t ldq, int32_t* piv, double tol,
                            void* ws, size_t ws_bytes, cudaStream_t s, int max_grid) {
  if (n < 0 || k < 0 || k > 4096 || ldw < n || ldq < n || !W || !Q || !piv) return RR_ERR_ARG;
  if (n > INT_MAX) return RR_ERR_ARG;
  if (k == 0) return RR_OK;
  if (arith == RR_F32 && hess_use_blocked(n, k, max_grid)) {
    float* w = (float*)W;
    constexpr int r = 16;
    switch (qtype) {
      case RR_F32: return hess_blocked<float>(n, k, w, ldw, (float*)Q, ldq, piv, tol, r, ws, ws_bytes, s);
      case RR_BF16: return hess_blocked<__nv_bfloat16>(n, k, w, ldw, (__nv_bfloat16*)Q, ldq, piv, tol, r, ws, ws_bytes, s);
      case RR_E4M3: return hess_blocked<e4m3b_t>(n, k, w, ldw, (e4m3b_t*)Q, ldq, piv, tol, r, ws, ws_bytes, s);
      case RR_F64: return hess_blocked<double>(n, k, w, ldw, (double*)Q, ldq, piv, tol, r, ws, ws_bytes, s);
    }
    return RR_ERR_ARG;
  }
  if (arith == RR_F32) {
    float* w = (float*)W;
    switch (qtype) {
      case RR_F32: return hess_launch<float, float>(n, k, w, ldw, (float*)Q, ldq, piv, tol, ws, ws_bytes, s, max_grid);
      case RR_BF16: return hess_launch<float, __nv_bfloat16>(n, k, w, ldw, (__nv_bfloat16*)Q, ldq, piv, tol, ws, ws_bytes, s, max_grid);
      case RR_E4M3: return hess_launch<float, e4m3b_t>(n, k, w, ldw, (e4m3b_t*)Q, ldq, piv, tol, ws, ws_bytes, s, max_grid);
      case RR_F64: return hess_launch<float, double>(n, k, w, ldw, (double*)Q, ldq, piv, tol, ws, ws_bytes, s, max_grid);
    }
  } else if (arith == RR_F64) {
    double* w = (double*)W;
    switch (qtype) {
      case RR_F64: return hess_launch<double, double>(n, k, w, ldw, (double*)Q, ldq, piv, tol, ws, ws_bytes, s, max_grid);
      case RR_F32: return hess_launch<double, float>(n, k, w, ldw, (float*)Q, ldq, piv, tol, ws, ws_bytes, s, max_grid);
      case RR_BF16: return hess_launch<double, __nv_bfloat16>(n, k, w, ldw, (__nv_bfloat16*)Q, ldq, piv, tol, ws, ws_bytes, s, max_grid);
    }
  }
  return RR_ERR_ARG;
}

extern "C" rr_status rr_hessenberg_blocked(int64_t n, int64_t k, float* W, int64_t ldw, int32_t qtype, void* Q,
                                           int64_t ldq, int32_t* piv, double tol, int32_t panel, void* ws,
                                           size_t ws_bytes, void* stream) {
  if (n < 0 || k < 0 || k > 4096 || ldw < n || ldq < n || !W || !Q || !piv) return RR_ERR_ARG;
  if (n >= (int64_t)kNoRow || panel < 1 || panel > kPanelMax) return RR_ERR_ARG;
  if (k == 0) return RR_OK;
  cudaStream_t s = as_stream(stream);
  switch (qtype) {
    case RR_F32: return hess_blocked<float>(n, k, W, ldw, (float*)Q, ldq, piv, tol, panel, ws, ws_bytes, s);
    case RR_BF16: return hess_blocked<__nv_bfloat16>(n, k, W, ldw, (__nv_bfloat16*)Q, ldq, piv, tol, panel, ws, ws_bytes, s);
    case RR_F64: return hess_blocked<double>(n, k, W, ldw, (double*)Q, ldq, piv, tol, panel, ws, ws_bytes, s);
  }
  return RR_ERR_ARG;
}
