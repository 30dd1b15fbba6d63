// The basis builders the paper compares the Hessenberg process with (Sec. 4,
// Table 1; the timings of Table 3): modified Gram-Schmidt left-looking
// (MGS-L) and right-looking (MGS-R), classical Gram-Schmidt without (CGS) and
// with re-orthogonalisation (CGS-2), and the left-looking Hessenberg process
// (Hess-L); the right-looking Hessenberg process is Algorithm 8 itself
// (rr_hessenberg).  Storage FP64, FP32 or FP16 (FP16 storage computes in
// FP32, as the paper's FP16 runs do); compute FP64 for FP64 storage.
//
// GB300 form: row-parallel kernels over the n x k block in HBM, one launch per
// data-parallel step (the methods differ in how many global reductions a
// column needs, which is what Table 1's parallelism column counts):
//   dot partials  a warp per column, lanes over a CTA's rows (coalesced),
//                 one partial per (CTA, column), summed in a fixed order by
//                 a second kernel (deterministic);
//   row updates   a thread per row, the columns in order;
//   MGS-L         one launch per (column, earlier column) pair: finish the
//                 previous dot, subtract, start the next dot (fused).
#include <algorithm>
#include <cuda_fp16.h>

#include "rr_common.cuh"
#include "solver_kernels.cuh"

namespace rr {
namespace {

constexpr int kBT = 256;  // threads per CTA

template <typename S> struct Cmp { using type = float; };
template <> struct Cmp<double> { using type = double; };

template <typename S> __device__ __forceinline__ typename Cmp<S>::type ld_s(const S* p) { return (typename Cmp<S>::type)*p; }
template <> __device__ __forceinline__ float ld_s<__half>(const __half* p) { return __half2float(*p); }
template <typename S> __device__ __forceinline__ void st_s(S* p, typename Cmp<S>::type v) { *p = (S)v; }
template <> __device__ __forceinline__ void st_s<__half>(__half* p, float v) { *p = __float2half_rn(v); }

// rows [r0, r1) of CTA g for a grid of G CTAs
__device__ __forceinline__ void cta_rows(int64_t n, int64_t& r0, int64_t& r1) {
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  r0 = (int64_t)blockIdx.x * per;
  r1 = r0 + per < n ? r0 + per : n;
}

// parts[g * cnt + i] = sum over CTA g's rows of Q(r, i0 + i) x(r)
template <typename S>
__global__ void __launch_bounds__(kBT) k_dot_parts(int64_t n, const S* __restrict__ Q, int64_t ldq, int i0, int cnt,
                                                   const S* __restrict__ x, typename Cmp<S>::type* __restrict__ parts) {
  using C = typename Cmp<S>::type;
  int64_t r0, r1;
  cta_rows(n, r0, r1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < cnt; i += kBT / 32) {
    const S* q = Q + (int64_t)(i0 + i) * ldq;
    C acc = C(0);
    for (int64_t r = r0 + lane; r < r1; r += 32) acc += ld_s<S>(q + r) * ld_s<S>(x + r);
    acc = warp_sum(acc);
    if (lane == 0) parts[(size_t)blockIdx.x * cnt + i] = acc;
  }
}

// out[i] = sum_g parts[g * cnt + i] (fixed order); also R column entries
template <typename C>
__global__ void k_sum_parts(int G, int cnt, const C* __restrict__ parts, C* __restrict__ out, double* __restrict__ Rcol,
                            int mode) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  C s = C(0);
  for (int g = 0; g < G; ++g) s += parts[(size_t)g * cnt + i];
  if (mode == 1) s = sqrt(s);  // a norm
  out[i] = s;
  if (Rcol) Rcol[i] += (double)s;
}

// x(r) -= sum_i c_i Q(r, i0 + i), the columns in order
template <typename S>
__global__ void __launch_bounds__(kBT) k_sub_cols(int64_t n, const S* __restrict__ Q, int64_t ldq, int i0, int cnt,
                                                  const typename Cmp<S>::type* __restrict__ c, S* __restrict__ x) {
  using C = typename Cmp<S>::type;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    C t = ld_s<S>(x + r);
    for (int i = 0; i < cnt; ++i) t -= c[i] * ld_s<S>(Q + r + (int64_t)(i0 + i) * ldq);
    st_s<S>(x + r, t);
  }
}

// x <- x / *nrm
template <typename S>
__global__ void k_scale_col(int64_t n, const typename Cmp<S>::type* __restrict__ nrm, S* __restrict__ x) {
  using C = typename Cmp<S>::type;
  const C d = *nrm;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    st_s<S>(x + r, d > C(0) ? ld_s<S>(x + r) / d : C(0));
}

// R(j, j+1+c) = cc[c] (a row of R from the right-looking dots)
template <typename C>
__global__ void k_put_row(int64_t k, int64_t j, int cnt, const C* __restrict__ cc, double* __restrict__ R) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < cnt) R[j + (j + 1 + c) * k] = (double)cc[c];
}

// storage conversions for the Hessenberg comparators on FP16 blocks (FP16
// storage, FP32 arithmetic)
__global__ void k_h2f(int64_t n, int64_t k, const __half* __restrict__ W, int64_t ldw, float* __restrict__ F) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x)
    F[e] = __half2float(W[(e % n) + (e / n) * ldw]);
}
__global__ void k_f2h(int64_t n, int64_t k, const float* __restrict__ F, __half* __restrict__ W, int64_t ldw) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x)
    W[(e % n) + (e / n) * ldw] = __float2half_rn(F[e]);
}

// Q(:, c0 + c) -= q c_c for the trailing columns (rank-1 update, MGS-R)
template <typename S>
__global__ void __launch_bounds__(kBT) k_rank1(int64_t n, const S* __restrict__ q, const typename Cmp<S>::type* __restrict__ cc,
                                               S* __restrict__ Q, int64_t ldq, int c0, int cnt) {
  using C = typename Cmp<S>::type;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const C qv = ld_s<S>(q + r);
    for (int c = 0; c < cnt; ++c) {
      S* p = Q + r + (int64_t)(c0 + c) * ldq;
      st_s<S>(p, ld_s<S>(p) - qv * cc[c]);
    }
  }
}

// MGS-L fused step on column x against earlier column i:
//   (i >= 0) r_i = sum of parts_in; x -= r_i q_i on this CTA's rows; R(i) += r_i
//   (nxt >= 0) parts_out[g] = sum over the CTA's rows of q_nxt x  (the next dot,
//   or the squared norm when nxt is the column itself: q_nxt = x)
template <typename S>
__global__ void __launch_bounds__(kBT) k_mgs_step(int64_t n, const S* __restrict__ Q, int64_t ldq, int i,
                                                  S* __restrict__ x, const typename Cmp<S>::type* __restrict__ parts_in,
                                                  const S* __restrict__ qn, typename Cmp<S>::type* __restrict__ parts_out,
                                                  double* __restrict__ Rcol) {
  using C = typename Cmp<S>::type;
  __shared__ C red[kBT / 32];
  __shared__ C s_r;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  C ri = C(0);
  if (i >= 0) {
    if (warp == 0) {
      C s = C(0);
      for (int g = lane; g < (int)gridDim.x; g += 32) s += parts_in[g];
      s = warp_sum(s);
      if (lane == 0) {
        s_r = s;
        if (blockIdx.x == 0 && Rcol) Rcol[i] += (double)s;
      }
    }
    __syncthreads();
    ri = s_r;
  }
  int64_t r0, r1;
  cta_rows(n, r0, r1);
  const S* qi = i >= 0 ? Q + (int64_t)i * ldq : nullptr;
  C acc = C(0);
  for (int64_t r = r0 + threadIdx.x; r < r1; r += kBT) {
    C t = ld_s<S>(x + r);
    if (qi) {
      t -= ri * ld_s<S>(qi + r);
      st_s<S>(x + r, t);
      t = ld_s<S>(x + r);  // the stored (rounded) value, as the next pass reads it
    }
    if (qn) acc += ld_s<S>(qn == x ? x + r : qn + r) * t;
  }
  if (!parts_out) return;
  acc = warp_sum(acc);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    C s = C(0);
    for (int w = 0; w < kBT / 32; ++w) s += red[w];
    parts_out[blockIdx.x] = s;
  }
}

template <typename S>
size_t builder_ws_bytes(int64_t n, int64_t k, int G) {
  using C = typename Cmp<S>::type;
  return align_up((size_t)G * (k + 1) * sizeof(C)) * 2 + align_up((size_t)(k + 1) * sizeof(C)) * 2 + 256;
}

template <typename S>
rr_status run_builder(cudaStream_t s, int method, int64_t n, int64_t k, S* W, int64_t ldw, double* R, void* ws,
                      size_t ws_bytes) {
  using C = typename Cmp<S>::type;
  const int G = (int)std::max<int64_t>(1, std::min<int64_t>((n + kBT - 1) / kBT, 2 * (int64_t)num_sms()));
  if (ws_bytes < builder_ws_bytes<S>(n, k, G) || !ws) return RR_ERR_WORKSPACE;
  Arena ar(ws, ws_bytes);
  C* parts = ar.take<C>((size_t)G * (k + 1));
  C* parts2 = ar.take<C>((size_t)G * (k + 1));
  C* coef = ar.take<C>(k + 1);
  C* nrm = ar.take<C>(k + 1);
  if (R) RR_CUDA(cudaMemsetAsync(R, 0, (size_t)k * k * sizeof(double), s));
  const unsigned gu = (unsigned)G;
  auto col = [&](int64_t j) { return W + j * ldw; };
  auto Rc = [&](int64_t j) { return R ? R + j * k : nullptr; };
  auto normalise = [&](int64_t j) -> rr_status {
    k_dot_parts<S><<<gu, kBT, 0, s>>>(n, W, ldw, (int)j, 1, col(j), parts);
    k_sum_parts<C><<<1, 32, 0, s>>>(G, 1, parts, nrm, R ? Rc(j) + j : nullptr, 1);
    k_scale_col<S><<<gu, kBT, 0, s>>>(n, nrm, col(j));
    note_launches(3);
    return RR_OK;
  };
  for (int64_t j = 0; j < k; ++j) {
    switch (method) {
      case RR_CGS:
      case RR_CGS2:
        // classical: all dots against the earlier columns at once, then one
        // block subtraction (twice for CGS-2)
        for (int pass = 0; pass < (method == RR_CGS2 ? 2 : 1) && j > 0; ++pass) {
          k_dot_parts<S><<<gu, kBT, 0, s>>>(n, W, ldw, 0, (int)j, col(j), parts);
          k_sum_parts<C><<<(unsigned)((j + 127) / 128), 128, 0, s>>>(G, (int)j, parts, coef, Rc(j), 0);
          k_sub_cols<S><<<gu, kBT, 0, s>>>(n, W, ldw, 0, (int)j, coef, col(j));
          note_launches(3);
        }
        RR_TRY(normalise(j));
        break;
      case RR_MGS_L: {
        // modified, left-looking: one dot and one subtraction per earlier
        // column, in order; each launch finishes a dot and starts the next
        C* pin = parts;
        C* pout = parts2;
        k_mgs_step<S><<<gu, kBT, 0, s>>>(n, W, ldw, -1, col(j), nullptr, j > 0 ? col(0) : col(j), pout, nullptr);
        note_launches(1);
        for (int64_t i = 0; i < j; ++i) {
          std::swap(pin, pout);
          const S* qn = i + 1 < j ? col(i + 1) : col(j);
          k_mgs_step<S><<<gu, kBT, 0, s>>>(n, W, ldw, (int)i, col(j), pin, qn, pout, Rc(j));
          note_launches(1);
        }
        // pout holds the partial squared norms of the reduced column
        k_sum_parts<C><<<1, 32, 0, s>>>(G, 1, pout, nrm, R ? Rc(j) + j : nullptr, 1);
        k_scale_col<S><<<gu, kBT, 0, s>>>(n, nrm, col(j));
        note_launches(2);
        break;
      }
      case RR_MGS_R:
        // modified, right-looking: normalise column j, then remove it from
        // every later column at once (dots, rank-1 update)
        RR_TRY(normalise(j));
        if (j + 1 < k) {
          const int cnt = (int)(k - j - 1);
          k_dot_parts<S><<<gu, kBT, 0, s>>>(n, W, ldw, (int)j + 1, cnt, col(j), parts);
          k_sum_parts<C><<<(unsigned)((cnt + 127) / 128), 128, 0, s>>>(G, cnt, parts, coef, nullptr, 0);
          k_rank1<S><<<gu, kBT, 0, s>>>(n, col(j), coef, W, ldw, (int)j + 1, cnt);
          note_launches(3);
          if (R) {
            // R(j, j+1:k): the dots, one row of R
            k_put_row<C><<<(unsigned)((cnt + 127) / 128), 128, 0, s>>>(k, j, cnt, coef, R);
            note_launches(1);
          }
        }
        break;
      default:
        return RR_ERR_ARG;
    }
  }
  return check_launch("basis builder");
}

}  // namespace
}  // namespace rr

using namespace rr;

extern "C" size_t rr_basis_builder_workspace_size(int32_t method, int32_t storage, int64_t n, int64_t k) {
  (void)method;
  const int G = (int)std::max<int64_t>(1, std::min<int64_t>((n + kBT - 1) / kBT, 2 * (int64_t)num_sms()));
  size_t a = 0;
  switch (storage) {
    case RR_F64: a = builder_ws_bytes<double>(n, k, G); break;
    case RR_F32: a = builder_ws_bytes<float>(n, k, G); break;
    case RR_F16: a = builder_ws_bytes<__half>(n, k, G); break;
  }
  // Hess-L and Hess-R go through the Hessenberg kernels' workspaces (and an
  // FP32 copy of an FP16 block)
  const size_t h = std::max(rr_hessenberg_workspace_size(n, k, RR_F32), rr_hessenberg_workspace_size(n, k, RR_F64));
  const size_t hl = std::max(hess_left_ws_bytes(n, k, RR_F64), hess_left_ws_bytes(n, k, RR_F32));
  const size_t conv = storage == RR_F16 ? align_up((size_t)n * k * sizeof(float)) + 256 : 0;
  return std::max(a, std::max(h, hl) + conv) + 4096;
}

extern "C" rr_status rr_basis_builder(int32_t method, int32_t storage, int64_t n, int64_t k, void* W, int64_t ldw,
                                      double* R, int32_t* piv, void* ws, size_t ws_bytes, void* stream) {
  if (n <= 0 || k <= 0 || k > n || k > 4096 || ldw < n || !W || !ws) return RR_ERR_ARG;
  if (storage != RR_F64 && storage != RR_F32 && storage != RR_F16) return RR_ERR_ARG;
  if (ws_bytes < rr_basis_builder_workspace_size(method, storage, n, k)) return RR_ERR_WORKSPACE;
  cudaStream_t s = as_stream(stream);
  const int32_t arith = storage == RR_F64 ? RR_F64 : RR_F32;
  if (method == RR_HESS_R || method == RR_HESS_L) {
    if (!piv) return RR_ERR_ARG;
    // FP16 storage: the process in FP32 on a converted copy, converted back
    void* Wp = W;
    int64_t ldp = ldw;
    char* wsp = (char*)ws;
    size_t wsb = ws_bytes;
    if (storage == RR_F16) {
      const size_t fb = align_up((size_t)n * k * sizeof(float));
      if (wsb < fb + 256) return RR_ERR_WORKSPACE;
      Wp = wsp;
      ldp = n;
      wsp += fb;
      wsb -= fb;
      k_h2f<<<(unsigned)std::min<int64_t>((n * k + 255) / 256, 4096), 256, 0, s>>>(n, k, (const __half*)W, ldw,
                                                                                  (float*)Wp);
      RR_TRY(check_launch("basis builder convert"));
    }
    if (method == RR_HESS_R)
      RR_TRY(rr_hessenberg(arith, n, k, Wp, ldp, arith, Wp, ldp, piv, 0.0, wsp, wsb, stream));
    else
      RR_TRY(hess_left_run(s, arith, n, k, Wp, ldp, piv, wsp, wsb));
    if (storage == RR_F16) {
      k_f2h<<<(unsigned)std::min<int64_t>((n * k + 255) / 256, 4096), 256, 0, s>>>(n, k, (const float*)Wp,
                                                                                  (__half*)W, ldw);
      RR_TRY(check_launch("basis builder convert"));
    }
    return RR_OK;
  }
  switch (storage) {
    case RR_F64: return run_builder<double>(s, method, n, k, (double*)W, ldw, R, ws, ws_bytes);
    case RR_F32: return run_builder<float>(s, method, n, k, (float*)W, ldw, R, ws, ws_bytes);
    case RR_F16: return run_builder<__half>(s, method, n, k, (__half*)W, ldw, R, ws, ws_bytes);
  }
  return RR_ERR_ARG;
}
