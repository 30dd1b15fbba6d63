// Learned warm start: the start-block network's kernels.  The paper starts
// the iteration from a random block (Alg. 1, V drawn U(0,1)); here a small
// fully convolutional network of the operator's potential proposes it, and is
// trained on Ritz vectors the plain method produced.  FP32 storage and
// arithmetic, NCHW layout (an image with C channels and n pixels is the n x C
// column-major block whose column c is channel c in row-major pixel order).
//
//   conv3x3:   zero-padded 3x3 cross-correlation, weights (O, C, 3, 3), bias (O),
//              optional ReLU and optional added image (a skip connection)
//   backward:  data gradient (correlation with the flipped, transposed
//              weights) and weight / bias gradients (sums over pixels, one
//              atomic add per weight and CTA)
//   Procrustes-aligned loss gradient, Adam update, network output -> FP64 block.
#include "rr_common.cuh"

#include <algorithm>
#include <cmath>

namespace rr {

constexpr int kTile = 16;      // output tile side (one pixel per thread)
constexpr int kOC = 8;         // output channels per CTA
constexpr int kHalo = kTile + 2;
constexpr int kTS = 48;        // shared row stride: rows ty and ty + 1 fall in disjoint banks
constexpr int kWTiles = 4;     // pixel tiles per CTA in the weight-gradient kernel

// Stage one zero-padded (kTile + 2)^2 halo tile of plane `src` (H x Wd).
__device__ __forceinline__ void load_halo(float (*t)[kTS], const float* __restrict__ src, int H, int Wd, int i0,
                                          int j0) {
  for (int e = threadIdx.x; e < kHalo * kHalo; e += blockDim.x) {
    const int yy = e / kHalo, xx = e % kHalo;
    const int gi = i0 + yy - 1, gj = j0 + xx - 1;
    t[yy][xx] = (gi >= 0 && gi < H && gj >= 0 && gj < Wd) ? __ldg(src + (size_t)gi * Wd + gj) : 0.f;
  }
}

__device__ __forceinline__ void fma8(float (&acc)[8], const float4 wa, const float4 wb, float v) {
  acc[0] = fmaf(wa.x, v, acc[0]);
  acc[1] = fmaf(wa.y, v, acc[1]);
  acc[2] = fmaf(wa.z, v, acc[2]);
  acc[3] = fmaf(wa.w, v, acc[3]);
  acc[4] = fmaf(wb.x, v, acc[4]);
  acc[5] = fmaf(wb.y, v, acc[5]);
  acc[6] = fmaf(wb.z, v, acc[6]);
  acc[7] = fmaf(wb.w, v, acc[7]);
}

// y[n, o, i, j] = act(b[o] + add[n, o, i, j] + sum_{c, dy, dx} W[o, c, dy, dx] x[n, c, i + dy - 1, j + dx - 1])
// grid (tiles_x, tiles_y, N * ceil(O / 8)), 256 threads.
__global__ void __launch_bounds__(256) k_conv3x3_fwd(int N, int C, int H, int Wd, int O,
                                                     const float* __restrict__ x, const float* __restrict__ w,
                                                     const float* __restrict__ b, const float* __restrict__ add,
                                                     int64_t add_nstride, int relu, float* __restrict__ y) {
  __shared__ float xt[kHalo][kTS];
  __shared__ float4 wt[9][2];  // wt[tap] = weights of output channels o0 .. o0 + 7
  const int og = (O + kOC - 1) / kOC;
  const int n = blockIdx.z / og, o0 = (blockIdx.z % og) * kOC;
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
  float acc[kOC];
#pragma unroll
  for (int u = 0; u < kOC; ++u) acc[u] = 0.f;
  for (int c = 0; c < C; ++c) {
    load_halo(xt, x + ((size_t)n * C + c) * H * Wd, H, Wd, i0, j0);
    if (threadIdx.x < kOC * 9) {
      const int u = threadIdx.x / 9, t = threadIdx.x % 9;
      reinterpret_cast<float*>(wt)[t * kOC + u] = o0 + u < O ? w[(((size_t)(o0 + u)) * C + c) * 9 + t] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 9; ++t) fma8(acc, wt[t][0], wt[t][1], xt[ty + t / 3][tx + t % 3]);
    __syncthreads();
  }
  const int i = i0 + ty, j = j0 + tx;
  if (i < H && j < Wd)
#pragma unroll
    for (int u = 0; u < kOC; ++u)
      if (o0 + u < O) {
        const size_t pix = ((size_t)(o0 + u) * H + i) * Wd + j;
        float v = acc[u] + b[o0 + u];
        if (add) v += add[(size_t)n * add_nstride + pix];
        if (relu) v = fmaxf(v, 0.f);
        y[(size_t)n * O * H * Wd + pix] = v;
      }
}

// dx[n, c, i, j] = sum_{o, dy, dx} W[o, c, dy, dx] g[n, o, i - dy + 1, j - dx + 1]
// grid (tiles_x, tiles_y, N * ceil(C / 8)).
__global__ void __launch_bounds__(256) k_conv3x3_bwd_data(int N, int C, int H, int Wd, int O,
                                                          const float* __restrict__ g,
                                                          const float* __restrict__ w, float* __restrict__ dx) {
  __shared__ float gt[kHalo][kTS];
  __shared__ float4 wt[9][2];  // wt[tap] = W[o, c0 .. c0 + 7, tap]
  const int cgs = (C + kOC - 1) / kOC;
  const int n = blockIdx.z / cgs, c0 = (blockIdx.z % cgs) * kOC;
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
  float acc[kOC];
#pragma unroll
  for (int u = 0; u < kOC; ++u) acc[u] = 0.f;
  for (int o = 0; o < O; ++o) {
    load_halo(gt, g + ((size_t)n * O + o) * H * Wd, H, Wd, i0, j0);
    if (threadIdx.x < kOC * 9) {
      const int u = threadIdx.x / 9, t = threadIdx.x % 9;
      reinterpret_cast<float*>(wt)[t * kOC + u] = c0 + u < C ? w[(((size_t)o) * C + c0 + u) * 9 + t] : 0.f;
    }
    __syncthreads();
    // tap (dy, dx) = (t / 3, t % 3) reads g at (i - dy + 1, j - dx + 1): halo (ty - dy + 2, tx - dx + 2)
#pragma unroll
    for (int t = 0; t < 9; ++t) fma8(acc, wt[t][0], wt[t][1], gt[ty + 2 - t / 3][tx + 2 - t % 3]);
    __syncthreads();
  }
  const int i = i0 + ty, j = j0 + tx;
  if (i < H && j < Wd)
#pragma unroll
    for (int u = 0; u < kOC; ++u)
      if (c0 + u < C) dx[(((size_t)n * C + c0 + u) * H + i) * Wd + j] = acc[u];
}

// dW[o, c, ky, kx] += sum_{n, i, j} g[n, o, i, j] x[n, c, i + ky - 1, j + kx - 1],
// db[o] += sum g[n, o, i, j].  A CTA takes up to kWTiles consecutive 16 x 16
// pixel tiles of one image for 8 output x 8 input channels (576 weights, each
// summed by one thread in registers), then adds its partial sums atomically.
// grid (ceil(tiles / kWTiles), N, ceil(O / 8) * ceil(C / 8)).
__global__ void __launch_bounds__(256) k_conv3x3_bwd_w(int N, int C, int H, int Wd, int O,
                                                       const float* __restrict__ x, const float* __restrict__ g,
                                                       float* __restrict__ dw, float* __restrict__ db) {
  __shared__ float xt[kOC][kHalo][kHalo + 1];
  __shared__ float gt[kOC][kTile][kTile + 1];
  constexpr int kW = kOC * kOC * 9;   // 576 weights
  constexpr int kPer = (kW + 255) / 256;
  const int tiles_x = (Wd + kTile - 1) / kTile, tiles = tiles_x * ((H + kTile - 1) / kTile);
  const int n = blockIdx.y;
  const int cgs = (C + kOC - 1) / kOC;
  const int o0 = (blockIdx.z / cgs) * kOC, c0 = (blockIdx.z % cgs) * kOC;
  float acc[kPer];
#pragma unroll
  for (int r = 0; r < kPer; ++r) acc[r] = 0.f;
  float bacc = 0.f;
  for (int tt = 0; tt < kWTiles; ++tt) {
    const int tile = blockIdx.x * kWTiles + tt;
    if (tile >= tiles) break;
    const int i0 = (tile / tiles_x) * kTile, j0 = (tile % tiles_x) * kTile;
    for (int e = threadIdx.x; e < kOC * kHalo * kHalo; e += 256) {
      const int u = e / (kHalo * kHalo), r = e % (kHalo * kHalo);
      const int yy = r / kHalo, xx = r % kHalo;
      const int gi = i0 + yy - 1, gj = j0 + xx - 1;
      xt[u][yy][xx] = (c0 + u < C && gi >= 0 && gi < H && gj >= 0 && gj < Wd)
                          ? x[(((size_t)n * C + c0 + u) * H + gi) * Wd + gj]
                          : 0.f;
    }
    for (int e = threadIdx.x; e < kOC * kTile * kTile; e += 256) {
      const int u = e / (kTile * kTile), r = e % (kTile * kTile);
      const int yy = r / kTile, xx = r % kTile;
      const int gi = i0 + yy, gj = j0 + xx;
      gt[u][yy][xx] = (o0 + u < O && gi < H && gj < Wd) ? g[(((size_t)n * O + o0 + u) * H + gi) * Wd + gj] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int wi = threadIdx.x + r * 256;
      if (wi < kW) {
        const int ou = wi / (kOC * 9), rem = wi % (kOC * 9), cu = rem / 9, k = rem % 9, ky = k / 3, kx = k % 3;
        float s = 0.f;
        for (int yy = 0; yy < kTile; ++yy)
#pragma unroll
          for (int xx = 0; xx < kTile; ++xx) s = fmaf(gt[ou][yy][xx], xt[cu][yy + ky][xx + kx], s);
        acc[r] += s;
      }
    }
    if (c0 == 0 && threadIdx.x < kOC) {
      float s = 0.f;
      for (int yy = 0; yy < kTile; ++yy)
        for (int xx = 0; xx < kTile; ++xx) s += gt[threadIdx.x][yy][xx];
      bacc += s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const int wi = threadIdx.x + r * 256;
    if (wi < kW) {
      const int ou = wi / (kOC * 9), rem = wi % (kOC * 9), cu = rem / 9, k = rem % 9;
      if (o0 + ou < O && c0 + cu < C) atomicAdd(dw + (((size_t)(o0 + ou)) * C + c0 + cu) * 9 + k, acc[r]);
    }
  }
  if (c0 == 0 && threadIdx.x < kOC && o0 + (int)threadIdx.x < O) atomicAdd(db + o0 + threadIdx.x, bacc);
}

__global__ void k_relu_mask(int64_t count, float* __restrict__ g, const float* __restrict__ act) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    if (!(act[e] > 0.f)) g[e] = 0.f;
}

// V = scale * out (n x k, FP32, ld n), R = U W^T (k x k, from the SVD of
// V^T V*): r = V R - V*, grad = scale * 2 r R^T (the gradient with respect to
// `out`), loss += |r|^2.  One thread per row; K is k rounded up to 16/32/64.
constexpr int kProcMax = 64;
template <int K>
__global__ void __launch_bounds__(128) k_procrustes_grad(int64_t n, int k, const float* __restrict__ out,
                                                         const double* __restrict__ Vs, const double* __restrict__ U,
                                                         const double* __restrict__ Wm, float scale,
                                                         float* __restrict__ grad, double* __restrict__ loss) {
  __shared__ float R[K][K + 1];
  __shared__ double red[4];
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int a = e % K, c = e / K;
    double s = 0.0;
    if (a < k && c < k)
      for (int l = 0; l < k; ++l) s += U[a + (size_t)l * k] * Wm[c + (size_t)l * k];  // (U W^T)[a, c]
    R[a][c] = (float)s;
  }
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double part = 0.0;
  if (i < n) {
    float v[K], gr[K];
#pragma unroll
    for (int a = 0; a < K; ++a) {
      v[a] = a < k ? scale * out[i + (size_t)a * n] : 0.f;
      gr[a] = 0.f;
    }
#pragma unroll 1
    for (int c = 0; c < k; ++c) {
      float s = 0.f;
#pragma unroll
      for (int a = 0; a < K; ++a) s = fmaf(v[a], R[a][c], s);
      const float r = s - (float)Vs[i + (size_t)c * n];    // (V R - V*)[i, c]
      part += (double)r * r;
#pragma unroll
      for (int a = 0; a < K; ++a) gr[a] = fmaf(r, R[a][c], gr[a]);
    }
#pragma unroll
    for (int a = 0; a < K; ++a)
      if (a < k) grad[i + (size_t)a * n] = 2.f * scale * gr[a];
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(loss, red[0] + red[1] + red[2] + red[3]);
}

__global__ void k_adam(int64_t count, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const float ge = g[e];
    const float me = b1 * m[e] + (1.f - b1) * ge;
    const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    p[e] -= lr * (me / c1) / (sqrtf(ve / c2) + eps);
  }
}

__global__ void k_net_block(int64_t n, int k, const float* __restrict__ out, float scale, double* __restrict__ V,
                            int64_t ldv) {
  const int64_t total = n * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e % n;
    V[i + c * ldv] = (double)(scale * out[e]);
  }
}

inline unsigned grid_1d(int64_t count) { return (unsigned)std::min<int64_t>((count + 255) / 256, 152 * 16); }

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_conv3x3_forward(int32_t N, int32_t C, int32_t H, int32_t W, int32_t O, const float* x,
                                        const float* w, const float* b, const float* add, int64_t add_nstride,
                                        int32_t relu, float* y, void* stream) {
  if (N < 0 || C < 1 || H < 0 || W < 0 || O < 1 || !x || !w || !b || !y) return RR_ERR_ARG;
  if (add && N > 1 && add_nstride < (int64_t)O * H * W) return RR_ERR_ARG;
  if (N == 0 || H == 0 || W == 0) return RR_OK;
  dim3 g((unsigned)((W + kTile - 1) / kTile), (unsigned)((H + kTile - 1) / kTile),
         (unsigned)(N * ((O + kOC - 1) / kOC)));
  k_conv3x3_fwd<<<g, 256, 0, as_stream(stream)>>>(N, C, H, W, O, x, w, b, add, add_nstride, relu, y);
  return check_launch("rr_conv3x3_forward");
}

extern "C" rr_status rr_conv3x3_backward(int32_t N, int32_t C, int32_t H, int32_t W, int32_t O, const float* x,
                                         const float* w, const float* g, float* dx, float* dw, float* db,
                                         void* stream) {
  if (N < 0 || C < 1 || H < 0 || W < 0 || O < 1 || !x || !w || !g || !dw || !db) return RR_ERR_ARG;
  if (N == 0 || H == 0 || W == 0) return RR_OK;
  cudaStream_t s = as_stream(stream);
  const int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
  if (dx) {
    dim3 gd((unsigned)tx, (unsigned)ty, (unsigned)(N * ((C + kOC - 1) / kOC)));
    k_conv3x3_bwd_data<<<gd, 256, 0, s>>>(N, C, H, W, O, g, w, dx);
    note_launches(1);
  }
  dim3 gw((unsigned)((tx * ty + kWTiles - 1) / kWTiles), (unsigned)N,
          (unsigned)(((O + kOC - 1) / kOC) * ((C + kOC - 1) / kOC)));
  k_conv3x3_bwd_w<<<gw, 256, 0, s>>>(N, C, H, W, O, x, g, dw, db);
  return check_launch("rr_conv3x3_backward");
}

extern "C" rr_status rr_relu_mask(int64_t count, float* g, const float* act, void* stream) {
  if (count < 0 || !g || !act) return RR_ERR_ARG;
  if (count == 0) return RR_OK;
  k_relu_mask<<<grid_1d(count), 256, 0, as_stream(stream)>>>(count, g, act);
  return check_launch("rr_relu_mask");
}

extern "C" rr_status rr_procrustes_grad(int64_t n, int32_t k, const float* out, const double* Vstar,
                                        const double* U, const double* Wm, float scale, float* grad,
                                        double* loss, void* stream) {
  if (n < 0 || k < 1 || k > kProcMax || !out || !Vstar || !U || !Wm || !grad || !loss) return RR_ERR_ARG;
  if (n == 0) return RR_OK;
  const unsigned g = (unsigned)((n + 127) / 128);
  cudaStream_t s = as_stream(stream);
  if (k <= 16) k_procrustes_grad<16><<<g, 128, 0, s>>>(n, k, out, Vstar, U, Wm, scale, grad, loss);
  else if (k <= 32) k_procrustes_grad<32><<<g, 128, 0, s>>>(n, k, out, Vstar, U, Wm, scale, grad, loss);
  else k_procrustes_grad<64><<<g, 128, 0, s>>>(n, k, out, Vstar, U, Wm, scale, grad, loss);
  return check_launch("rr_procrustes_grad");
}

extern "C" rr_status rr_adam(int64_t count, float* p, const float* g, float* m, float* v, float lr, float b1,
                             float b2, float eps, int32_t t, void* stream) {
  if (count < 0 || t < 1 || !p || !g || !m || !v) return RR_ERR_ARG;
  if (count == 0) return RR_OK;
  const float c1 = (float)(1.0 - std::pow((double)b1, (double)t));
  const float c2 = (float)(1.0 - std::pow((double)b2, (double)t));
  k_adam<<<grid_1d(count), 256, 0, as_stream(stream)>>>(count, p, g, m, v, lr, b1, b2, eps, c1, c2);
  return check_launch("rr_adam");
}

extern "C" rr_status rr_net_block(int64_t n, int32_t k, const float* out, float scale, double* V, int64_t ldv,
                                  void* stream) {
  if (n < 0 || k < 0 || !out || !V || ldv < n) return RR_ERR_ARG;
  if (n == 0 || k == 0) return RR_OK;
  k_net_block<<<grid_1d(n * k), 256, 0, as_stream(stream)>>>(n, k, out, scale, V, ldv);
  return check_launch("rr_net_block");
}
