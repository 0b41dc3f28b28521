// Convolutional action for block moves: evaluation and training kernels.
//
// F_cnn(X) = sum over the (x, y, tau) torus of a three-layer periodic 3x3x3 network (see
// hq_cnn.cuh).  Training fits F_cnn(X_a) to log|det M(X_a)| minus the sample mean by mean
// squared error, as for the patch network.  Because F_cnn is a plain sum of the last layer,
// dF/d(layer-2 output at any point) is the same vector sum_t W3[t][.], which makes the first
// backward step a masked constant.  Every gradient entry is owned by one thread and summed
// over the CTA's samples in a fixed order; the per-CTA partials are summed in a fixed order by
// the Adam kernel, so training is deterministic.
#include "hq_cnn.cuh"
#include "../../include/holstein_dqmc.h"

namespace hq {

static_assert(CN_NP == HQ_CNN_PARAMS, "parameter count");

constexpr int CN_TILE = 32;  // points per staged tile in the weight-gradient passes

// ------------------------------------------------------------------------ evaluation
// F_cnn of every chain (grid = chains); refreshes the chain's cached activations.
__global__ void __launch_bounds__(HQ_THREADS) cnn_eval_kernel(Dev d, CnnState cn, const double* Xall, double* Fout,
                                                              double x0) {
  extern __shared__ __align__(16) char craw[];
  float* w = (float*)craw;
  double* red = (double*)(w + CN_WPAD);
  const int c = blockIdx.x, NL = d.n * d.L;
  cn_load_weights(cn.wbf, w);
  const double F = cn_forward_all(d, w, Xall + (size_t)c * NL, x0, cn.h1c + (size_t)c * NL * CN_C,
                                  cn.h2c + (size_t)c * NL * CN_C, cn.o3c + (size_t)c * NL, red);
  if (threadIdx.x == 0) Fout[c] = F;
}

// ------------------------------------------------------------------------ training
struct CnTrainSmem {
  float* w;      // [CN_WPAD]
  float* nbh;    // [CN_TILE][27][16] staged neighbourhoods (layer-1 values or inputs)
  float* dt;     // [CN_TILE][16] staged gradients at the tile's points
  float* hs;     // [HQ_THREADS][16] per-thread channel sums
  float* w3s;    // [16] sum over taps of W3
  double* red;   // [HQ_WARPS]
  double* scal;  // [2]
};

__host__ __device__ inline size_t cn_train_smem_bytes() {
  return sizeof(float) * (CN_WPAD + CN_TILE * CN_T * CN_C + CN_TILE * CN_C + HQ_THREADS * CN_C + CN_C) +
         sizeof(double) * (HQ_WARPS + 2);
}

// One minibatch: each CTA takes samples a = blockIdx.x, + gridDim.x, ...; forward with the
// activations kept in the CTA's slice of cn.tr, then the backward passes.  Writes F_a to Fb
// and the CTA's summed gradient to partials[blockIdx.x].
__global__ void __launch_bounds__(HQ_THREADS) cnn_train_kernel(Dev d, CnnState cn, const double* Xs,
                                                               const double* ys, const int* idx, int B, double x0,
                                                               double* Fb, float* partials) {
  extern __shared__ __align__(16) char craw[];
  CnTrainSmem s;
  float* f = (float*)craw;
  s.w = f; f += CN_WPAD;
  s.nbh = f; f += CN_TILE * CN_T * CN_C;
  s.dt = f; f += CN_TILE * CN_C;
  s.hs = f; f += HQ_THREADS * CN_C;
  s.w3s = f; f += CN_C;
  s.red = (double*)f;
  s.scal = s.red + HQ_WARPS;
  cn_load_weights(cn.wbf, s.w);
  const int n = d.n, NL = d.n * d.L, tid = threadIdx.x;
  if (tid < CN_C) {
    float a = 0.f;
    for (int t = 0; t < CN_T; ++t) a += s.w[CN_W3 + t * CN_C + tid];
    s.w3s[tid] = a;
  }
  float* A1 = cn.tr + (size_t)blockIdx.x * 3 * NL * CN_C;  // layer-1 activations
  float* A2 = A1 + (size_t)NL * CN_C;                      // layer-2 activations, then dL/da2
  float* D1 = A2 + (size_t)NL * CN_C;                      // dL/da1
  // owned entries: W2 pairs (tap, in) q0 = tid, q1 = tid + 256 (< 432), 16 outputs each;
  // W1 pairs (tap, out) the same indices; b2 / b1 channel (tid - 176) for 176 <= tid < 192;
  // W3 channel tid (< 16, same for every tap); b3 by thread 16.
  float g2a[CN_C], g2b[CN_C], g1a = 0.f, g1b = 0.f, gb = 0.f, gb1 = 0.f, g3 = 0.f;
#pragma unroll
  for (int c = 0; c < CN_C; ++c) g2a[c] = g2b[c] = 0.f;
  const int q0 = tid, q1 = tid + HQ_THREADS;
  const bool has1 = q1 < CN_T * CN_C;
  for (int a = blockIdx.x; a < B; a += gridDim.x) {
    const double* X = Xs + (size_t)idx[a] * NL;
    // forward
    const double F = cn_forward_all(d, s.w, X, x0, A1, A2, nullptr, s.red);
    if (tid == 0) Fb[a] = F;
    const float sg = (float)(2.0 * (F - ys[idx[a]]) / B);
    // layer 3: dF/dW3[t][ci] = sum_q h2(q)[ci] for every t; dF/db3 = L N
    float hs[CN_C];
#pragma unroll
    for (int c = 0; c < CN_C; ++c) hs[c] = 0.f;
    for (int p = tid; p < NL; p += HQ_THREADS) {
      float h[CN_C];
      cn_load16(A2 + (size_t)p * CN_C, h);
#pragma unroll
      for (int c = 0; c < CN_C; ++c) hs[c] += h[c];
    }
#pragma unroll
    for (int c = 0; c < CN_C; ++c) s.hs[tid * CN_C + c] = hs[c];
    __syncthreads();
    if (tid < CN_C) {
      float t3 = 0.f;
      for (int k = 0; k < HQ_THREADS; ++k) t3 += s.hs[k * CN_C + tid];
      g3 += sg * t3;
    } else if (tid == CN_C) {
      g3 += sg * (float)NL;
    }
    // dL/da2 = relu'(a2) sg sum_t W3[t]  (in place)
    for (int p = tid; p < NL; p += HQ_THREADS) {
      float* h = A2 + (size_t)p * CN_C;
#pragma unroll
      for (int c = 0; c < CN_C; ++c) h[c] = (h[c] > 0.f) ? sg * s.w3s[c] : 0.f;
    }
    __syncthreads();
    // W2, b2: sum_p d2(p)[co] h1(p + tap)[ci], tiles of CN_TILE points
    for (int p0 = 0; p0 < NL; p0 += CN_TILE) {
      for (int e = tid; e < CN_TILE * CN_T * 4; e += HQ_THREADS) {
        const int pt = e / (CN_T * 4), t = (e / 4) % CN_T, v = e % 4, p = p0 + pt;
        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < NL) {
          const int l = p / n, i = p % n;
          const int ll = (l + t / 9 - 1 + d.L) % d.L, j = cn_site(d, i, (t / 3) % 3 - 1, t % 3 - 1);
          val = reinterpret_cast<const float4*>(A1 + ((size_t)ll * n + j) * CN_C)[v];
        }
        reinterpret_cast<float4*>(s.nbh + ((size_t)pt * CN_T + t) * CN_C)[v] = val;
      }
      for (int e = tid; e < CN_TILE * CN_C; e += HQ_THREADS) {
        const int pt = e / CN_C, p = p0 + pt;
        s.dt[e] = (p < NL) ? A2[(size_t)p * CN_C + e % CN_C] : 0.f;
      }
      __syncthreads();
      for (int pt = 0; pt < CN_TILE; ++pt) {
        const float* dd = s.dt + pt * CN_C;
        const float ha = s.nbh[(size_t)pt * CN_T * CN_C + q0];
#pragma unroll
        for (int c = 0; c < CN_C; ++c) g2a[c] = fmaf(ha, dd[c], g2a[c]);
        if (has1) {
          const float hb = s.nbh[(size_t)pt * CN_T * CN_C + q1];
#pragma unroll
          for (int c = 0; c < CN_C; ++c) g2b[c] = fmaf(hb, dd[c], g2b[c]);
        }
        if (tid >= 176 && tid < 192) gb += dd[tid - 176];
      }
      __syncthreads();
    }
    // dL/da1(q)[ci] = relu'(a1(q)) sum_t sum_co W2[t][ci][co] d2(q - tap_t)[co]
    for (int p = tid; p < NL; p += HQ_THREADS) {
      const int l = p / n, i = p % n;
      float acc[CN_C];
#pragma unroll
      for (int c = 0; c < CN_C; ++c) acc[c] = 0.f;
      for (int t = 0; t < CN_T; ++t) {
        const int ll = (l - (t / 9 - 1) + d.L) % d.L, j = cn_site(d, i, -((t / 3) % 3 - 1), -(t % 3 - 1));
        float dd[CN_C];
        cn_load16(A2 + ((size_t)ll * n + j) * CN_C, dd);
        const float* W = s.w + CN_W2 + t * CN_C * CN_C;
#pragma unroll
        for (int ci = 0; ci < CN_C; ++ci) {
          float v = 0.f;
#pragma unroll
          for (int c = 0; c < CN_C; ++c) v = fmaf(W[ci * CN_C + c], dd[c], v);
          acc[ci] += v;
        }
      }
      float h[CN_C];
      cn_load16(A1 + (size_t)p * CN_C, h);
      float4* o = reinterpret_cast<float4*>(D1 + (size_t)p * CN_C);
#pragma unroll
      for (int q = 0; q < CN_C / 4; ++q)
        o[q] = make_float4(h[4 * q] > 0.f ? acc[4 * q] : 0.f, h[4 * q + 1] > 0.f ? acc[4 * q + 1] : 0.f,
                           h[4 * q + 2] > 0.f ? acc[4 * q + 2] : 0.f, h[4 * q + 3] > 0.f ? acc[4 * q + 3] : 0.f);
    }
    __syncthreads();
    // W1, b1: sum_p d1(p)[co] z(p + tap)
    for (int p0 = 0; p0 < NL; p0 += CN_TILE) {
      for (int e = tid; e < CN_TILE * CN_T; e += HQ_THREADS) {
        const int pt = e / CN_T, t = e % CN_T, p = p0 + pt;
        float z = 0.f;
        if (p < NL) {
          const int l = p / n, i = p % n;
          const int ll = (l + t / 9 - 1 + d.L) % d.L, j = cn_site(d, i, (t / 3) % 3 - 1, t % 3 - 1);
          z = (float)(X[(size_t)ll * n + j] - x0);
        }
        s.nbh[e] = z;
      }
      for (int e = tid; e < CN_TILE * CN_C; e += HQ_THREADS) {
        const int pt = e / CN_C, p = p0 + pt;
        s.dt[e] = (p < NL) ? D1[(size_t)p * CN_C + e % CN_C] : 0.f;
      }
      __syncthreads();
      for (int pt = 0; pt < CN_TILE; ++pt) {
        const float* dd = s.dt + pt * CN_C;
        g1a = fmaf(s.nbh[pt * CN_T + q0 / CN_C], dd[q0 % CN_C], g1a);
        if (has1) g1b = fmaf(s.nbh[pt * CN_T + q1 / CN_C], dd[q1 % CN_C], g1b);
        if (tid >= 176 && tid < 192) gb1 += dd[tid - 176];
      }
      __syncthreads();
    }
  }
  float* out = partials + (size_t)blockIdx.x * CN_WPAD;
#pragma unroll
  for (int c = 0; c < CN_C; ++c) out[CN_W2 + q0 * CN_C + c] = g2a[c];
  if (has1) {
#pragma unroll
    for (int c = 0; c < CN_C; ++c) out[CN_W2 + q1 * CN_C + c] = g2b[c];
  }
  out[CN_W1 + q0] = g1a;
  if (has1) out[CN_W1 + q1] = g1b;
  if (tid >= 176 && tid < 192) {
    out[CN_B2 + tid - 176] = gb;
    out[CN_B1 + tid - 176] = gb1;
  }
  if (tid < CN_C)
    for (int t = 0; t < CN_T; ++t) out[CN_W3 + t * CN_C + tid] = g3;
  else if (tid == CN_C)
    out[CN_B3] = g3;
}

// Sum of the per-CTA partials (fixed order) into grad; with lr > 0 an Adam step on the FP32
// master weights and a fresh bfloat16 copy.
__global__ void cnn_adam_kernel(CnnState cn, const float* partials, int nparts, float lr, int t_step) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= CN_NP) return;
  float g = 0.f;
  for (int p = 0; p < nparts; ++p) g += partials[(size_t)p * CN_WPAD + k];
  cn.grad[k] = g;
  if (lr > 0.f) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float m = b1 * cn.adam_m[k] + (1.f - b1) * g;
    const float v = b2 * cn.adam_v[k] + (1.f - b2) * g * g;
    cn.adam_m[k] = m;
    cn.adam_v[k] = v;
    const float mh = m / (1.f - powf(b1, (float)t_step)), vh = v / (1.f - powf(b2, (float)t_step));
    const float w = cn.master[k] - lr * mh / (sqrtf(vh) + eps);
    cn.master[k] = w;
    cn.wbf[k] = float_to_bf16(w);
  }
}

__global__ void cnn_set_kernel(CnnState cn, const float* src) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < CN_NP) {
    cn.master[k] = src[k];
    cn.wbf[k] = float_to_bf16(src[k]);
    cn.adam_m[k] = 0.f;
    cn.adam_v[k] = 0.f;
  }
}

__global__ void cnn_loss_kernel(CnnState cn, const double* ys, const int* idx, int B, double scale, double* loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double acc = 0.0;
    for (int a = 0; a < B; ++a) {
      const double r = cn.Fb[a] - ys[idx[a]];
      acc += r * r;
    }
    loss[0] += acc * scale;
  }
}

// ------------------------------------------------------------------------ launchers
static double mean_field_shift(const Dev& d) { return -d.g / (d.mass * d.omega * d.omega); }

cudaError_t cnn_launch_eval(const Dev& d, const CnnState& cn, const double* X, double* F, int /*write_cache*/,
                            cudaStream_t s) {
  const size_t sb = sizeof(float) * CN_WPAD + sizeof(double) * HQ_WARPS;
  opt_in_smem((const void*)cnn_eval_kernel, sb);
  cnn_eval_kernel<<<d.n_chains, HQ_THREADS, sb, s>>>(d, cn, X, F, mean_field_shift(d));
  return cudaGetLastError();
}

cudaError_t cnn_launch_set(const CnnState& cn, const float* src_device, cudaStream_t s) {
  cnn_set_kernel<<<(CN_NP + 255) / 256, 256, 0, s>>>(cn, src_device);
  return cudaGetLastError();
}

cudaError_t cnn_launch_batch(const Dev& d, const CnnState& cn, const double* Xs, const double* ys, const int* idx,
                             int B, float lr, int t_step, cudaStream_t s) {
  const int ctas = B < cn.train_ctas ? B : cn.train_ctas;
  const size_t sb = cn_train_smem_bytes();
  cudaError_t st = opt_in_smem((const void*)cnn_train_kernel, sb);
  if (st != cudaSuccess) return st;
  cnn_train_kernel<<<ctas, HQ_THREADS, sb, s>>>(d, cn, Xs, ys, idx, B, mean_field_shift(d), cn.Fb, cn.partials);
  cnn_adam_kernel<<<(CN_NP + 255) / 256, 256, 0, s>>>(cn, cn.partials, ctas, lr, t_step);
  return cudaGetLastError();
}

cudaError_t cnn_launch_loss(const CnnState& cn, const double* ys, const int* idx, int B, double scale, double* loss,
                            cudaStream_t s) {
  cnn_loss_kernel<<<1, 32, 0, s>>>(cn, ys, idx, B, scale, loss);
  return cudaGetLastError();
}

}  // namespace hq
