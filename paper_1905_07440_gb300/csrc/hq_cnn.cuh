// Periodic 3D convolutional action (device functions shared by the inner-move and the CNN
// kernels).
//
// Paper: "Global Updates" -- a convolutional network on the whole phonon field stands for
// the weight, so a move of a whole imaginary-time column is cheap to estimate.  Here the
// network is three 3x3x3 cross-correlations with periodic padding on the (x, y, tau) torus,
// 1 -> 16 -> 16 -> 1 channels, ReLU after the first two, and F_cnn(X) = sum of the last
// layer over every point; the input is z = X - x0 with x0 = -g/(M Omega^2).  Tap
// t = 9 (dl + 1) + 3 (dy + 1) + (dx + 1) reads (l + dl, y + dy, x + dx).  Weights are
// bfloat16, arithmetic FP32; every path computes a point through the same functions in the
// same order, so a value recomputed in a block-move window equals the cached one bit for bit.
#pragma once
#include "hq_device.cuh"
#include "hq_internal.h"

namespace hq {

constexpr int CN_T = 27, CN_C = kCnnC;
constexpr int CN_W1 = 0, CN_B1 = CN_T * CN_C, CN_W2 = CN_B1 + CN_C, CN_B2 = CN_W2 + CN_T * CN_C * CN_C,
              CN_W3 = CN_B2 + CN_C, CN_B3 = CN_W3 + CN_T * CN_C, CN_NP = CN_B3 + 1;
constexpr int CN_WPAD = (CN_NP + 3) & ~3;
constexpr int CN_WIN = 49;  // sites within torus distance 3

__device__ inline void cn_load_weights(const uint16_t* wb, float* w) {
  for (int k = threadIdx.x; k < CN_WPAD; k += blockDim.x) w[k] = (k < CN_NP) ? bf16_to_float(wb[k]) : 0.f;
  __syncthreads();
}

// site of (x + dx, y + dy) on the torus
__device__ __forceinline__ int cn_site(const Dev& d, int i, int dy, int dx) {
  const int x = i % d.nx, y = i / d.nx;
  return (x + dx + d.nx) % d.nx + d.nx * ((y + dy + d.ny) % d.ny);
}

// Layer-1 activations (after ReLU) at (l, i); site cs of every slice is shifted by cdx.
__device__ __forceinline__ void cn_layer1(const Dev& d, const float* w, const double* X, double x0, int l, int i,
                                          int cs, double cdx, float* out) {
  float a[CN_C];
#pragma unroll
  for (int c = 0; c < CN_C; ++c) a[c] = w[CN_B1 + c];
  for (int t = 0; t < CN_T; ++t) {
    const int ll = (l + t / 9 - 1 + d.L) % d.L, j = cn_site(d, i, (t / 3) % 3 - 1, t % 3 - 1);
    double v = X[(size_t)ll * d.n + j];
    if (j == cs) v = v + cdx;
    const float z = (float)(v - x0);
#pragma unroll
    for (int c = 0; c < CN_C; ++c) a[c] = fmaf(z, w[CN_W1 + t * CN_C + c], a[c]);
  }
  float4* o = reinterpret_cast<float4*>(out);
#pragma unroll
  for (int q = 0; q < CN_C / 4; ++q)
    o[q] = make_float4(fmaxf(a[4 * q], 0.f), fmaxf(a[4 * q + 1], 0.f), fmaxf(a[4 * q + 2], 0.f), fmaxf(a[4 * q + 3], 0.f));
}

__device__ __forceinline__ void cn_load16(const float* p, float* v) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < CN_C / 4; ++k) {
    const float4 f = q[k];
    v[4 * k] = f.x;
    v[4 * k + 1] = f.y;
    v[4 * k + 2] = f.z;
    v[4 * k + 3] = f.w;
  }
}

// Layer-2 activations (after ReLU) at (l, i); h1at(ll, j) gives the 16 layer-1 values there.
template <class H1>
__device__ __forceinline__ void cn_layer2(const Dev& d, const float* w, int l, int i, H1 h1at, float* out) {
  float a[CN_C];
#pragma unroll
  for (int c = 0; c < CN_C; ++c) a[c] = w[CN_B2 + c];
  for (int t = 0; t < CN_T; ++t) {
    const int ll = (l + t / 9 - 1 + d.L) % d.L, j = cn_site(d, i, (t / 3) % 3 - 1, t % 3 - 1);
    float h[CN_C];
    cn_load16(h1at(ll, j), h);
    const float* W = w + CN_W2 + t * CN_C * CN_C;
#pragma unroll
    for (int ci = 0; ci < CN_C; ++ci)
#pragma unroll
      for (int c = 0; c < CN_C; ++c) a[c] = fmaf(h[ci], W[ci * CN_C + c], a[c]);
  }
  float4* o = reinterpret_cast<float4*>(out);
#pragma unroll
  for (int q = 0; q < CN_C / 4; ++q)
    o[q] = make_float4(fmaxf(a[4 * q], 0.f), fmaxf(a[4 * q + 1], 0.f), fmaxf(a[4 * q + 2], 0.f), fmaxf(a[4 * q + 3], 0.f));
}

// Layer-3 output at (l, i); h2at(ll, j) gives the 16 layer-2 values there.
template <class H2>
__device__ __forceinline__ float cn_layer3(const Dev& d, const float* w, int l, int i, H2 h2at) {
  float o = w[CN_B3];
  for (int t = 0; t < CN_T; ++t) {
    const int ll = (l + t / 9 - 1 + d.L) % d.L, j = cn_site(d, i, (t / 3) % 3 - 1, t % 3 - 1);
    float h[CN_C];
    cn_load16(h2at(ll, j), h);
#pragma unroll
    for (int ci = 0; ci < CN_C; ++ci) o = fmaf(h[ci], w[CN_W3 + t * CN_C + ci], o);
  }
  return o;
}

// F_cnn of one field configuration by the whole CTA; layer outputs go to h1 [L N][16],
// h2 [L N][16] and (if o3 != nullptr) o3 [L N].  Returns F in every thread.
__device__ inline double cn_forward_all(const Dev& d, const float* w, const double* X, double x0, float* h1, float* h2,
                                        float* o3, double* red) {
  const int n = d.n, NL = d.n * d.L;
  for (int p = threadIdx.x; p < NL; p += blockDim.x) cn_layer1(d, w, X, x0, p / n, p % n, -1, 0.0, h1 + (size_t)p * CN_C);
  __syncthreads();
  auto h1at = [&](int ll, int j) { return h1 + ((size_t)ll * n + j) * CN_C; };
  for (int p = threadIdx.x; p < NL; p += blockDim.x) cn_layer2(d, w, p / n, p % n, h1at, h2 + (size_t)p * CN_C);
  __syncthreads();
  auto h2at = [&](int ll, int j) { return h2 + ((size_t)ll * n + j) * CN_C; };
  double part = 0.0;
  for (int p = threadIdx.x; p < NL; p += blockDim.x) {
    const float o = cn_layer3(d, w, p / n, p % n, h2at);
    if (o3) o3[p] = o;
    part += (double)o;
  }
  return block_sum(part, red);
}

// Sites within torus distance 1, 2, 3 of site i (each listed once, ascending) and the
// position of every site in the radius-1 and radius-2 lists (-1 outside).  Shared memory:
// cnt[4], lst [3][CN_WIN], pos [2][n].  Thread 0 builds; ends with a barrier.
struct CnWindow {
  int* cnt;
  int* lst;
  int* pos;
};

__device__ inline void cn_build_window(const Dev& d, int i, const CnWindow& wd) {
  if (threadIdx.x == 0) {
    const int xi = i % d.nx, yi = i / d.nx;
    int c1 = 0, c2 = 0, c3 = 0;
    for (int j = 0; j < d.n; ++j) {
      int ax = abs(j % d.nx - xi), ay = abs(j / d.nx - yi);
      ax = min(ax, d.nx - ax);
      ay = min(ay, d.ny - ay);
      const int r = max(ax, ay);
      wd.pos[j] = -1;
      wd.pos[d.n + j] = -1;
      if (r <= 1) { wd.pos[j] = c1; wd.lst[c1++] = j; }
      if (r <= 2) { wd.pos[d.n + j] = c2; wd.lst[CN_WIN + c2++] = j; }
      if (r <= 3) wd.lst[2 * CN_WIN + c3++] = j;
    }
    wd.cnt[0] = c1;
    wd.cnt[1] = c2;
    wd.cnt[2] = c3;
  }
  __syncthreads();
}

// F_cnn(X') - F_cnn(X) for X'(i, .) = X(i, .) + dx, from the cached activations of X: the
// proposal's layer-1 values in the radius-1 window, layer-2 in radius 2, outputs in radius 3
// (every slice) go to h1p / h2p / o3p.  Called by the whole CTA after cn_build_window;
// returns the difference in every thread.
__device__ inline double cn_block_delta(const Dev& d, const float* w, const CnWindow& wd, const double* X, double x0,
                                        int i, double dx, const float* h1c, const float* h2c, const float* o3c,
                                        float* h1p, float* h2p, float* o3p, double* red) {
  const int n = d.n, L = d.L;
  const int n1 = wd.cnt[0], n2 = wd.cnt[1], n3 = wd.cnt[2];
  const int* l1 = wd.lst;
  const int* l2 = wd.lst + CN_WIN;
  const int* l3 = wd.lst + 2 * CN_WIN;
  const int* pos1 = wd.pos;
  const int* pos2 = wd.pos + n;
  for (int q = threadIdx.x; q < n1 * L; q += blockDim.x) {
    const int l = q / n1, k = q % n1;
    cn_layer1(d, w, X, x0, l, l1[k], i, dx, h1p + (size_t)q * CN_C);
  }
  __syncthreads();
  auto h1at = [&](int ll, int j) {
    const int k = pos1[j];
    return k >= 0 ? h1p + ((size_t)ll * n1 + k) * CN_C : h1c + ((size_t)ll * n + j) * CN_C;
  };
  for (int q = threadIdx.x; q < n2 * L; q += blockDim.x) {
    const int l = q / n2, k = q % n2;
    cn_layer2(d, w, l, l2[k], h1at, h2p + (size_t)q * CN_C);
  }
  __syncthreads();
  auto h2at = [&](int ll, int j) {
    const int k = pos2[j];
    return k >= 0 ? h2p + ((size_t)ll * n2 + k) * CN_C : h2c + ((size_t)ll * n + j) * CN_C;
  };
  double part = 0.0;
  for (int q = threadIdx.x; q < n3 * L; q += blockDim.x) {
    const int l = q / n3, k = q % n3, j = l3[k];
    const float o = cn_layer3(d, w, l, j, h2at);
    o3p[q] = o;
    part += (double)o - (double)o3c[(size_t)l * n + j];
  }
  return block_sum(part, red);
}

// Accepted block move: the window values become the cached activations.
__device__ inline void cn_block_commit(const Dev& d, const CnWindow& wd, float* h1c, float* h2c, float* o3c,
                                       const float* h1p, const float* h2p, const float* o3p) {
  const int n = d.n, L = d.L;
  const int n1 = wd.cnt[0], n2 = wd.cnt[1], n3 = wd.cnt[2];
  for (int q = threadIdx.x; q < n1 * L * 4; q += blockDim.x) {
    const int pt = q / 4, v = q % 4, l = pt / n1, j = wd.lst[pt % n1];
    reinterpret_cast<float4*>(h1c + ((size_t)l * n + j) * CN_C)[v] = reinterpret_cast<const float4*>(h1p + (size_t)pt * CN_C)[v];
  }
  for (int q = threadIdx.x; q < n2 * L * 4; q += blockDim.x) {
    const int pt = q / 4, v = q % 4, l = pt / n2, j = wd.lst[CN_WIN + pt % n2];
    reinterpret_cast<float4*>(h2c + ((size_t)l * n + j) * CN_C)[v] = reinterpret_cast<const float4*>(h2p + (size_t)pt * CN_C)[v];
  }
  for (int q = threadIdx.x; q < n3 * L; q += blockDim.x) {
    const int l = q / n3, j = wd.lst[2 * CN_WIN + q % n3];
    o3c[(size_t)l * n + j] = o3p[q];
  }
  __syncthreads();
}

}  // namespace hq
