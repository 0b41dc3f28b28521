// Learned effective action and the cumulative (network-driven) sampler.
//
// Paper: "Local Updates" -- a fully connected network on the fields around a spacetime point
// predicts the weight change of a move -- and the cumulative update of the benchmark section:
// after network-driven sweeps the whole proposal X -> X' is accepted with min(1, p_c),
// p_c = [W(X')/W(X)] [exp(-beta E_NN[X]) / exp(-beta E_NN[X'])], so the chain stays exact.
//
// Here E_NN is one scalar function: F(X) = sum_{i,l} f(patch_{i,l}(X)), patch = X on the
// 5-site cross x 5 slices around (i, l) minus the mean field -g/(M Omega^2), f a 25-64-64-1
// ReLU network with bfloat16 weights and FP32 arithmetic.  Local moves are Metropolis moves on
// exp(-dtau S_ph + 2F) (exact phonon action); block moves on the same weight, or with the
// periodic convolutional action F_cnn in place of F (hq_cnn.cuh).  Each move is reversible for
// its own weight, so p_c = exp(2 dlog|det M| - 2 sum of the accepted moves' network changes)
// (the phonon action cancels; for one network the sum telescopes to F(X') - F(X)).
// Every kernel evaluates f through nn_patch_eval (one 8-lane group per patch, fixed order),
// so the inner chain and the acceptance see bit-identical values of f.
#include <cstdio>
#include "hq_cnn.cuh"
#include "hq_device.cuh"
#include "hq_internal.h"
#include "../../include/holstein_dqmc.h"

namespace hq {

// parameter layout: W1[25][64], b1[64], W2[64][64], b2[64], W3[64], b3
constexpr int NN_IN = 25, NN_H = 64;
constexpr int NN_HP = NN_H + 1;  // padded stride of the groups' hidden rows: the 4 groups of a
                                 // warp then read h1[v] from 4 different banks
constexpr int NN_W1 = 0, NN_B1 = NN_IN * NN_H, NN_W2 = NN_B1 + NN_H, NN_B2 = NN_W2 + NN_H * NN_H,
              NN_W3 = NN_B2 + NN_H, NN_B3 = NN_W3 + NN_H, NN_NP = NN_B3 + 1;
static_assert(NN_NP == HQ_NN_PARAMS, "parameter count");
constexpr int NN_WPAD = (NN_NP + 3) & ~3;
constexpr int NN_GROUPS = HQ_THREADS / 8;


__device__ inline void load_weights(const uint16_t* wb, float* w) {
  for (int k = threadIdx.x; k < NN_WPAD; k += HQ_THREADS) w[k] = (k < NN_NP) ? bf16_to_float(wb[k]) : 0.f;
  __syncthreads();
}

// f of one patch by the 8 lanes of a group (sub = lane in group): lane `sub` owns hidden units
// 8 sub .. 8 sub + 7.  z: the patch's 25 inputs, h1: 64 floats of group scratch.  All 32 lanes
// of the warp must call it together (group shuffles).  Returns f in every lane of the group.
__device__ __forceinline__ float nn_patch_eval(const float* w, const float* z, float* h1, int sub) {
  const float* W1 = w + NN_W1;
  const float* b1 = w + NN_B1;
  const float* W2 = w + NN_W2;
  const float* b2 = w + NN_B2;
  const float* W3 = w + NN_W3;
  const int u0 = sub * 8;
  float a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = b1[u0 + j];
  for (int k = 0; k < NN_IN; ++k) {
    const float zk = z[k];
    // the lane's 8 weights of this input as two 16-byte loads (fewer shared-memory requests)
    const float4 wa = *reinterpret_cast<const float4*>(W1 + k * NN_H + u0);
    const float4 wb = *reinterpret_cast<const float4*>(W1 + k * NN_H + u0 + 4);
    const float w8[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fmaf(zk, w8[j], a[j]);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) h1[u0 + j] = fmaxf(a[j], 0.f);
  __syncwarp();
  float c[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) c[j] = b2[u0 + j];
  for (int v = 0; v < NN_H; ++v) {
    const float hv = h1[v];
    const float4 wa = *reinterpret_cast<const float4*>(W2 + v * NN_H + u0);
    const float4 wb = *reinterpret_cast<const float4*>(W2 + v * NN_H + u0 + 4);
    const float w8[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j] = fmaf(hv, w8[j], c[j]);
  }
  float o = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) o = fmaf(fmaxf(c[j], 0.f), W3[u0 + j], o);
  o += __shfl_xor_sync(HQ_FULL, o, 4);
  o += __shfl_xor_sync(HQ_FULL, o, 2);
  o += __shfl_xor_sync(HQ_FULL, o, 1);
  __syncwarp();
  return o + w[NN_B3];
}

// Inputs of the patch centred at (l, i), with an optional change: points of site `cs` get
// +cdx on every slice (block move) or, if cl >= 0, only the point (cl, cs) is set to cx.
__device__ __forceinline__ void fill_patch(const Dev& d, const double* X, int l, int i, double x0, float* z,
                                           int sub, int cs, int cl, double cx, double cdx) {
  const int n = d.n, L = d.L, x = i % d.nx, y = i / d.nx;
  for (int k = sub; k < NN_IN; k += 8) {
    const int dl = k / 5 - 2, cidx = k % 5;
    const int cx_ = (cidx == 1) - (cidx == 2), cy_ = (cidx == 3) - (cidx == 4);
    const int ll = (l + dl + L) % L;
    const int j = (x + cx_ + d.nx) % d.nx + d.nx * ((y + cy_ + d.ny) % d.ny);
    double v = X[(size_t)ll * n + j];
    if (j == cs) {
      if (cl < 0) v = v + cdx;
      else if (ll == cl) v = cx;
    }
    z[k] = (float)(v - x0);
  }
  __syncwarp();
}

struct NNSmem {
  float* w;      // [NN_WPAD]
  float* z;      // [NN_GROUPS][NN_IN + 3]
  float* h1;     // [NN_GROUPS][NN_HP]
  double* red;   // [HQ_WARPS]
  double* pu2;   // [n] proposal uniforms (local)
  double* pxn;   // [n] proposed values
  double* pds;   // [n] dtau dS_ph
  double* gacc;  // [NN_GROUPS] per-group sums
  double* scal;  // [8]
  float* cw;     // [CN_WPAD] convolutional weights (with_cnn)
  CnWindow win;  // block-move window (with_cnn)
};

__host__ __device__ inline size_t nn_smem_bytes(int n, bool with_cnn = false) {
  size_t b = sizeof(double) * (HQ_WARPS + 3 * (size_t)n + NN_GROUPS + 8) +
             sizeof(float) * (NN_WPAD + NN_GROUPS * (NN_IN + 3) + NN_GROUPS * NN_HP);
  if (with_cnn) b += sizeof(float) * CN_WPAD + sizeof(int) * (4 + 3 * CN_WIN + 2 * (size_t)n);
  return b;
}

__device__ inline NNSmem nn_carve(int n, char* base, bool with_cnn = false) {
  NNSmem s;
  double* p = (double*)base;
  s.red = p; p += HQ_WARPS;
  s.pu2 = p; p += n;
  s.pxn = p; p += n;
  s.pds = p; p += n;
  s.gacc = p; p += NN_GROUPS;
  s.scal = p; p += 8;
  float* f = (float*)p;
  s.w = f; f += NN_WPAD;
  s.z = f; f += NN_GROUPS * (NN_IN + 3);
  s.h1 = f; f += NN_GROUPS * NN_HP;
  s.cw = nullptr;
  if (with_cnn) {
    s.cw = f; f += CN_WPAD;
    int* q = (int*)f;
    s.win.cnt = q; q += 4;
    s.win.lst = q; q += 3 * CN_WIN;
    s.win.pos = q;
  }
  return s;
}

// F of one configuration by the whole CTA (groups of 8 lanes per patch, fixed order); the
// patch values go to fc when fc != nullptr.  Returns F in every thread.
__device__ inline double fc_eval_all(const Dev& d, const NNSmem& s, const double* X, double x0, float* fc) {
  const int n = d.n, NL = d.n * d.L;
  const int g = threadIdx.x / 8, sub = threadIdx.x % 8;
  float* z = s.z + g * (NN_IN + 3);
  float* h1 = s.h1 + g * NN_HP;
  double part = 0.0;
  for (int base = 0; base < NL; base += NN_GROUPS) {
    const int row = base + g;
    const bool on = row < NL;
    fill_patch(d, X, on ? row / n : 0, on ? row % n : 0, x0, z, sub, -1, -1, 0.0, 0.0);
    const float f = nn_patch_eval(s.w, z, h1, sub);
    if (on && sub == 0) {
      if (fc) fc[row] = f;
      part += (double)f;
    }
  }
  if (sub == 0) s.gacc[g] = part;
  __syncthreads();
  double F = 0.0;
  for (int k = 0; k < NN_GROUPS; ++k) F += s.gacc[k];
  __syncthreads();
  return F;
}

// F(X) of every chain (grid = chains); also refreshes the patch cache fc.
__global__ void __launch_bounds__(HQ_THREADS) nn_eval_kernel(Dev d, NNState nn, const double* Xall, double* Fout,
                                                             int write_cache) {
  extern __shared__ __align__(16) char nraw[];
  const int c = blockIdx.x, n = d.n, NL = d.n * d.L;
  const NNSmem s = nn_carve(n, nraw);
  load_weights(nn.wbf, s.w);
  const double F = fc_eval_all(d, s, Xall + (size_t)c * NL, nn.x0, write_cache ? nn.fcache + (size_t)c * NL : nullptr);
  if (threadIdx.x == 0) Fout[c] = F;
}

// n_inner network-driven sweeps of every chain: local moves at every (l, i), then block
// moves at every site, each accepted on exp(2 dF - dtau dS_ph) with the exact phonon action
// (dF from the patch network, or for block moves with use_cnn from the convolutional action).
// A fixed visiting order of reversible moves is not reversible as a whole, and the
// cumulative accept needs a reversible proposal; so each step draws a direction (second
// uniform of the step's Philox block, tag 4): forward (l, i ascending, then block moves i
// ascending) or the exact reverse of that sequence, with probability 1/2 each.  The accepted
// moves' dF are summed (thread 0, fixed order) into nn.dFpath for the cumulative accept.
// The caches of the current fields (fc; with use_cnn also the convolutional activations) are
// valid on entry; with use_cnn each network's cache is rebuilt before its part when the other
// part has changed the fields.
__global__ void __launch_bounds__(HQ_THREADS) nn_inner_kernel(Dev d, NNState nn, CnnState cn, int n_inner,
                                                              int do_local, int do_block, int use_cnn, int window,
                                                              int site_window) {
  extern __shared__ __align__(16) char nraw[];
  const int c = blockIdx.x, n = d.n, L = d.L, NL = n * L;
  if (!d.active[c]) return;
  const NNSmem s = nn_carve(n, nraw, use_cnn != 0);
  load_weights(nn.wbf, s.w);
  if (use_cnn) cn_load_weights(cn.wbf, s.cw);
  double* X = d.X + (size_t)c * NL;
  float* fc = nn.fcache + (size_t)c * NL;
  float* fnew = nn.fnew + (size_t)c * 5 * L;
  float *h1c = nullptr, *h2c = nullptr, *o3c = nullptr, *h1p = nullptr, *h2p = nullptr, *o3p = nullptr;
  if (use_cnn) {
    h1c = cn.h1c + (size_t)c * NL * CN_C;
    h2c = cn.h2c + (size_t)c * NL * CN_C;
    o3c = cn.o3c + (size_t)c * NL;
    h1p = cn.h1p + (size_t)c * 9 * L * CN_C;
    h2p = cn.h2p + (size_t)c * 25 * L * CN_C;
    o3p = cn.o3p + (size_t)c * CN_WIN * L;
  }
  const int g = threadIdx.x / 8, sub = threadIdx.x % 8;
  float* z = s.z + g * (NN_IN + 3);
  float* h1 = s.h1 + g * NN_HP;
  const uint32_t* id = d.cid + 4 * (size_t)c;
  const uint32_t key0 = id[0], key1 = id[1], chain = id[2], step = id[3];
  long long nl_acc = 0, nb_acc = 0;
  double path = 0.0;                   // thread 0
  bool fc_stale = false, cn_stale = false;  // uniform over the CTA
  const double kfac = d.mass / (2.0 * d.dtau), pfac = 0.5 * d.dtau * d.mass * (d.omega * d.omega);
  double du1, du2;
  proposal_uniforms(key0, key1, 0u, step, chain, 4u, du1, du2);
  const bool fwd = du2 < 0.5;
  // local moves on W consecutive slices from a random start l0, block moves on Wb consecutive
  // sites (in index order, periodic) from a random start j0: the two uniforms of event 1 of
  // the step's tag-4 stream, independent of the fields, so each window's move sequence stays
  // reversible
  const int W = (window > 0 && window < L) ? window : L;
  const int Wb = (site_window > 0 && site_window < n) ? site_window : n;
  int l0 = 0, j0 = 0;
  if (W < L || Wb < n) {
    double wu1, wu2;
    proposal_uniforms(key0, key1, 1u, step, chain, 4u, wu1, wu2);
    l0 = (int)(wu1 * (double)L);
    if (l0 > L - 1) l0 = L - 1;
    j0 = (int)(wu2 * (double)n);
    if (j0 > n - 1) j0 = n - 1;
    if (W == L) l0 = 0;
    if (Wb == n) j0 = 0;
  }
  for (int u = 0; u < n_inner; ++u) {
    const uint32_t isw = step * (uint32_t)n_inner + (uint32_t)u;
    for (int part = 0; part < 2; ++part) {
    const bool local_part = (part == 0) == fwd;
    if (local_part && do_local) {
      if (fc_stale) {
        fc_eval_all(d, s, X, nn.x0, fc);
        fc_stale = false;
      }
      for (int sl0 = 0; sl0 < W; ++sl0) {
        const int sl = (l0 + (fwd ? sl0 : W - 1 - sl0)) % L;
        for (int i = threadIdx.x; i < n; i += HQ_THREADS) {
          double u1, u2;
          proposal_uniforms(key0, key1, (uint32_t)(sl * n + i), isw, chain, 2u, u1, u2);
          const double dx = d.dx_local * (2.0 * u1 - 1.0);
          const double xo = X[(size_t)sl * n + i], xn = xo + dx;
          const double xp = X[(size_t)((sl + 1) % L) * n + i], xm = X[(size_t)((sl - 1 + L) % L) * n + i];
          const double kin = (xp - xn) * (xp - xn) + (xn - xm) * (xn - xm) - (xp - xo) * (xp - xo) - (xo - xm) * (xo - xm);
          s.pu2[i] = u2;
          s.pxn[i] = xn;
          s.pds[i] = kfac * kin + pfac * (xn * xn - xo * xo);
        }
        __syncthreads();
        for (int i0 = 0; i0 < n; ++i0) {
          const int i = fwd ? i0 : n - 1 - i0;
          // the 25 patches containing (sl, i): centres (sl - dl, i - c), one per group
          float f = 0.f;
          int row = -1;
          if (g < 25) {
            const int dl = g / 5 - 2, cidx = g % 5;
            const int cx_ = (cidx == 1) - (cidx == 2), cy_ = (cidx == 3) - (cidx == 4);
            const int x = i % d.nx, y = i / d.nx;
            const int j = (x - cx_ + d.nx) % d.nx + d.nx * ((y - cy_ + d.ny) % d.ny);
            row = ((sl - dl + L) % L) * n + j;
          }
          fill_patch(d, X, row >= 0 ? row / n : 0, row >= 0 ? row % n : 0, nn.x0, z, sub, i, sl, s.pxn[i], 0.0);
          f = nn_patch_eval(s.w, z, h1, sub);
          if (sub == 0) s.gacc[g] = (row >= 0) ? (double)f - (double)fc[row] : 0.0;
          __syncthreads();
          if (threadIdx.x == 0) {
            double dF = 0.0;
            for (int k = 0; k < 25; ++k) dF += s.gacc[k];
            const double prob = exp(fmin(2.0 * dF - s.pds[i], 709.0));
            const int acc = s.pu2[i] < prob;
            s.scal[0] = acc;
            if (acc) {
              X[(size_t)sl * n + i] = s.pxn[i];
              path += dF;
            }
            nl_acc += acc;
          }
          __syncthreads();
          if (s.scal[0] != 0.0) {
            if (row >= 0 && sub == 0) fc[row] = f;
            cn_stale = true;
          }
          __syncthreads();
        }
      }
    }
    if (!local_part && do_block) {
      if (use_cnn && cn_stale) {
        cn_forward_all(d, s.cw, X, nn.x0, h1c, h2c, o3c, s.red);
        cn_stale = false;
      }
      for (int i0 = 0; i0 < Wb; ++i0) {
        const int i = (j0 + (fwd ? i0 : Wb - 1 - i0)) % n;
        if (threadIdx.x == 0) {
          double u1, u2;
          proposal_uniforms(key0, key1, (uint32_t)i, isw, chain, 3u, u1, u2);
          s.scal[1] = d.dx_global * (2.0 * u1 - 1.0);
          s.scal[2] = u2;
        }
        __syncthreads();
        const double dx = s.scal[1];
        double a = 0.0;
        for (int sl = threadIdx.x; sl < L; sl += HQ_THREADS) {
          const double x = X[(size_t)sl * n + i];
          a += (x + dx) * (x + dx) - x * x;
        }
        a = block_sum(a, s.red);
        const double dS = pfac * a;
        const int x = i % d.nx, y = i / d.nx;
        double dF;
        if (use_cnn) {
          cn_build_window(d, i, s.win);
          dF = cn_block_delta(d, s.cw, s.win, X, nn.x0, i, dx, h1c, h2c, o3c, h1p, h2p, o3p, s.red);
        } else {
          // the 5 L patches containing site i: centres (l, i - c)
          double pt = 0.0;
          for (int base = 0; base < 5 * L; base += NN_GROUPS) {
            const int q = base + g;
            const bool on = q < 5 * L;
            int row = 0;
            if (on) {
              const int cidx = q % 5, sl = q / 5;
              const int cx_ = (cidx == 1) - (cidx == 2), cy_ = (cidx == 3) - (cidx == 4);
              const int j = (x - cx_ + d.nx) % d.nx + d.nx * ((y - cy_ + d.ny) % d.ny);
              row = sl * n + j;
            }
            fill_patch(d, X, row / n, row % n, nn.x0, z, sub, i, -1, 0.0, dx);
            const float f = nn_patch_eval(s.w, z, h1, sub);
            if (on && sub == 0) {
              fnew[q] = f;
              pt += (double)f - (double)fc[row];
            }
          }
          if (sub == 0) s.gacc[g] = pt;
          __syncthreads();
          dF = 0.0;
          for (int k = 0; k < NN_GROUPS; ++k) dF += s.gacc[k];
        }
        if (threadIdx.x == 0) {
          const double prob = exp(fmin(2.0 * dF - dS, 709.0));
          const int acc = s.scal[2] < prob;
          s.scal[0] = acc;
          if (acc) path += dF;
          nb_acc += acc;
        }
        __syncthreads();
        if (s.scal[0] != 0.0) {
          for (int sl = threadIdx.x; sl < L; sl += HQ_THREADS) X[(size_t)sl * n + i] = X[(size_t)sl * n + i] + dx;
          if (use_cnn) {
            cn_block_commit(d, s.win, h1c, h2c, o3c, h1p, h2p, o3p);
            fc_stale = true;
          } else {
            for (int q = threadIdx.x; q < 5 * L; q += HQ_THREADS) {
              const int cidx = q % 5, sl = q / 5;
              const int cx_ = (cidx == 1) - (cidx == 2), cy_ = (cidx == 3) - (cidx == 4);
              const int j = (x - cx_ + d.nx) % d.nx + d.nx * ((y - cy_ + d.ny) % d.ny);
              fc[(size_t)sl * n + j] = fnew[q];
            }
          }
        }
        __syncthreads();
      }
    }
    }
  }
  if (threadIdx.x == 0) {
    long long* cnt = nn.counters + (size_t)c * kNNCounters;
    cnt[0] += (long long)n_inner * (do_local ? W * n : 0);
    cnt[1] += nl_acc;
    cnt[2] += (long long)n_inner * (do_block ? Wb : 0);
    cnt[3] += nb_acc;
    nn.dFpath[c] = path;
  }
}

// Cumulative accept of X' (fields now in d.X, log|det M(X')| in d.logdet after the stack
// build) against X (saved in nn.X0 with nn.ld0): p_c = exp(2 dlog|det M| - 2 nn.dFpath).
// With restore_g, a rejected chain also gets back G_0 of X (saved in nn.G0 before the inner
// sweep), so every chain's G holds G_0 of its final fields without another stack build.
__global__ void __launch_bounds__(HQ_THREADS) nn_decide_kernel(Dev d, NNState nn, int restore_g) {
  const int c = blockIdx.x, NL = d.n * d.L;
  if (!d.active[c]) return;
  __shared__ int acc;
  if (threadIdx.x == 0) {
    double u1, u2;
    const uint32_t* id = d.cid + 4 * (size_t)c;
    proposal_uniforms(id[0], id[1], 0u, id[3], id[2], 4u, u1, u2);
    const double ld1 = d.logdet[c], ld0 = nn.ld0[c];
    const double arg = 2.0 * (ld1 - ld0) - 2.0 * nn.dFpath[c];
    const double pc = exp(fmin(arg, 709.0));
    acc = u1 < pc;
    nn.last_pc[c] = pc;
    long long* cnt = nn.counters + (size_t)c * kNNCounters;
    cnt[4] += 1;
    cnt[5] += acc;
    if (!acc) d.logdet[c] = ld0;
    if (!isfinite(arg)) d.status[c] = HQ_ENAN;
  }
  __syncthreads();
  if (!acc) {
    double* X = d.X + (size_t)c * NL;
    const double* X0 = nn.X0 + (size_t)c * NL;
    for (int k = threadIdx.x; k < NL; k += HQ_THREADS) X[k] = X0[k];
    if (restore_g) {
      const size_t nn2 = (size_t)d.n * d.n;
      double* G = d.G + (size_t)c * nn2;
      const double* G0 = nn.G0 + (size_t)c * nn2;
      for (size_t k = threadIdx.x; k < nn2; k += HQ_THREADS) G[k] = G0[k];
    }
  }
}

// ------------------------------------------------------------------------ training
// Mean squared error (1/B) sum_a (F(X_a) - y_a)^2 over a minibatch.  Forward: F_a per sample.
// Backward: each CTA takes a fixed share of (sample, 32-patch tile) pairs; per tile the groups
// store inputs, hidden activations and output gradients in shared memory, then every thread
// accumulates the gradient entries it owns over the tile (fixed order: deterministic).  The
// per-CTA partial gradients are summed in a fixed order by the Adam kernel.
struct TrainSmem {
  float* w;
  float* z;    // [32][28]
  float* h1;   // [32][64]
  float* d1;   // [32][64] dL/da1
  float* d2;   // [32][64] dL/da2
  float* h2;   // [32][64]
  float* dout; // [32]
};

__host__ __device__ inline size_t train_smem_bytes() {
  return sizeof(float) * (NN_WPAD + NN_GROUPS * (NN_IN + 3) + 4 * NN_GROUPS * NN_H + NN_GROUPS);
}

__global__ void __launch_bounds__(HQ_THREADS) nn_batch_forward_kernel(Dev d, NNState nn, const double* Xs,
                                                                      const int* idx, double* Fb) {
  extern __shared__ __align__(16) char nraw[];
  const int a = blockIdx.x, n = d.n, NL = d.n * d.L;
  const NNSmem s = nn_carve(n, nraw);
  load_weights(nn.wbf, s.w);
  const double* X = Xs + (size_t)idx[a] * NL;
  const int g = threadIdx.x / 8, sub = threadIdx.x % 8;
  float* z = s.z + g * (NN_IN + 3);
  float* h1 = s.h1 + g * NN_HP;
  double part = 0.0;
  for (int base = 0; base < NL; base += NN_GROUPS) {
    const int row = base + g;
    const bool on = row < NL;
    fill_patch(d, X, on ? row / n : 0, on ? row % n : 0, nn.x0, z, sub, -1, -1, 0.0, 0.0);
    const float f = nn_patch_eval(s.w, z, h1, sub);
    if (on && sub == 0) part += (double)f;
  }
  if (sub == 0) s.gacc[g] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double F = 0.0;
    for (int k = 0; k < NN_GROUPS; ++k) F += s.gacc[k];
    Fb[a] = F;
  }
}

__global__ void __launch_bounds__(HQ_THREADS) nn_batch_backward_kernel(Dev d, NNState nn, const double* Xs,
                                                                       const double* ys, const int* idx, int B,
                                                                       const double* Fb, float* partials) {
  extern __shared__ __align__(16) char nraw[];
  const int n = d.n, NL = d.n * d.L;
  float* f0 = (float*)nraw;
  TrainSmem s;
  s.w = f0; f0 += NN_WPAD;
  s.z = f0; f0 += NN_GROUPS * (NN_IN + 3);
  s.h1 = f0; f0 += NN_GROUPS * NN_H;
  s.d1 = f0; f0 += NN_GROUPS * NN_H;
  s.d2 = f0; f0 += NN_GROUPS * NN_H;
  s.h2 = f0; f0 += NN_GROUPS * NN_H;
  s.dout = f0;
  load_weights(nn.wbf, s.w);
  const float* W1 = s.w + NN_W1;
  const float* b1 = s.w + NN_B1;
  const float* W2 = s.w + NN_W2;
  const float* b2 = s.w + NN_B2;
  const float* W3 = s.w + NN_W3;
  const int g = threadIdx.x / 8, sub = threadIdx.x % 8, u0 = sub * 8;
  float* z = s.z + g * (NN_IN + 3);
  float* h1 = s.h1 + g * NN_H;
  // gradient entries owned by this thread: W2 (16), W1 (<= 7), one of b1/b2/W3/b3
  float gW2[16], gW1[7], gX = 0.f;
#pragma unroll
  for (int k = 0; k < 16; ++k) gW2[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 7; ++k) gW1[k] = 0.f;
  const int tiles_per_sample = (NL + NN_GROUPS - 1) / NN_GROUPS;
  const int ntile = B * tiles_per_sample;
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int a = tile / tiles_per_sample, row = (tile % tiles_per_sample) * NN_GROUPS + g;
    const bool on = row < NL;
    const double* X = Xs + (size_t)idx[a] * NL;
    const float dF = (float)(2.0 * (Fb[a] - ys[idx[a]]) / B);
    fill_patch(d, X, on ? row / n : 0, on ? row % n : 0, nn.x0, z, sub, -1, -1, 0.0, 0.0);
    // forward, keeping a1 / a2 signs, h1, h2
    float a1[8], c2[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a1[j] = b1[u0 + j];
    for (int k = 0; k < NN_IN; ++k) {
      const float zk = z[k];
#pragma unroll
      for (int j = 0; j < 8; ++j) a1[j] = fmaf(zk, W1[k * NN_H + u0 + j], a1[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) h1[u0 + j] = fmaxf(a1[j], 0.f);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 8; ++j) c2[j] = b2[u0 + j];
    for (int v = 0; v < NN_H; ++v) {
      const float hv = h1[v];
#pragma unroll
      for (int j = 0; j < 8; ++j) c2[j] = fmaf(hv, W2[v * NN_H + u0 + j], c2[j]);
    }
    const float dout = on ? dF : 0.f;
    float* d2 = s.d2 + g * NN_H;
    float* h2 = s.h2 + g * NN_H;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      h2[u0 + j] = fmaxf(c2[j], 0.f);
      d2[u0 + j] = (c2[j] > 0.f) ? dout * W3[u0 + j] : 0.f;
    }
    if (sub == 0) s.dout[g] = dout;
    __syncwarp();
    // dL/da1 for this lane's 8 units: relu'(a1) sum_u W2[v][u] d2[u]
    float* d1 = s.d1 + g * NN_H;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int v = u0 + j;
      float acc = 0.f;
      for (int uu = 0; uu < NN_H; ++uu) acc = fmaf(W2[v * NN_H + uu], d2[uu], acc);
      d1[v] = (a1[j] > 0.f) ? acc : 0.f;
    }
    __syncthreads();
    // accumulate owned gradient entries over the tile's 32 patches
    for (int p = 0; p < NN_GROUPS; ++p) {
      const float* h1p = s.h1 + p * NN_H;
      const float* d2p = s.d2 + p * NN_H;
      const float* d1p = s.d1 + p * NN_H;
      const float* zp = s.z + p * (NN_IN + 3);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int e = threadIdx.x + k * HQ_THREADS;  // W2 entry e = v * 64 + u
        gW2[k] = fmaf(h1p[e / NN_H], d2p[e % NN_H], gW2[k]);
      }
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const int e = threadIdx.x + k * HQ_THREADS;  // W1 entry e = k_in * 64 + v
        if (e < NN_IN * NN_H) gW1[k] = fmaf(zp[e / NN_H], d1p[e % NN_H], gW1[k]);
      }
      const int t = threadIdx.x;
      if (t < NN_H) gX += d1p[t];                       // b1
      else if (t < 2 * NN_H) gX += d2p[t - NN_H];       // b2
      else if (t < 3 * NN_H) gX += s.h2[p * NN_H + t - 2 * NN_H] * s.dout[p];  // W3
      else if (t == 3 * NN_H) gX += s.dout[p];          // b3
    }
    __syncthreads();
  }
  float* out = partials + (size_t)blockIdx.x * NN_WPAD;
#pragma unroll
  for (int k = 0; k < 16; ++k) out[NN_W2 + threadIdx.x + k * HQ_THREADS] = gW2[k];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const int e = threadIdx.x + k * HQ_THREADS;
    if (e < NN_IN * NN_H) out[NN_W1 + e] = gW1[k];
  }
  const int t = threadIdx.x;
  if (t < NN_H) out[NN_B1 + t] = gX;
  else if (t < 2 * NN_H) out[NN_B2 + t - NN_H] = gX;
  else if (t < 3 * NN_H) out[NN_W3 + t - 2 * NN_H] = gX;
  else if (t == 3 * NN_H) out[NN_B3] = gX;
}

// Sum of the per-CTA partials (fixed order) into grad; with lr > 0 an Adam step on the FP32
// master weights and a fresh bfloat16 copy.
__global__ void nn_adam_kernel(NNState nn, const float* partials, int nparts, float lr, int t_step) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NN_NP) return;
  float g = 0.f;
  for (int p = 0; p < nparts; ++p) g += partials[(size_t)p * NN_WPAD + k];
  nn.grad[k] = g;
  if (lr > 0.f) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float m = b1 * nn.adam_m[k] + (1.f - b1) * g;
    const float v = b2 * nn.adam_v[k] + (1.f - b2) * g * g;
    nn.adam_m[k] = m;
    nn.adam_v[k] = v;
    const float mh = m / (1.f - powf(b1, (float)t_step)), vh = v / (1.f - powf(b2, (float)t_step));
    const float w = nn.master[k] - lr * mh / (sqrtf(vh) + eps);
    nn.master[k] = w;
    nn.wbf[k] = float_to_bf16(w);
  }
}

__global__ void nn_loss_kernel(NNState nn, const double* ys, const int* idx, int B, double scale) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double acc = 0.0;
    for (int a = 0; a < B; ++a) {
      const double r = nn.Fb[a] - ys[idx[a]];
      acc += r * r;
    }
    nn.loss[0] += acc * scale;
  }
}

__global__ void nn_set_kernel(NNState nn, const float* src) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < NN_NP) {
    nn.master[k] = src[k];
    nn.wbf[k] = float_to_bf16(src[k]);
    nn.adam_m[k] = 0.f;
    nn.adam_v[k] = 0.f;
  }
}

// ------------------------------------------------------------------------ launchers
static inline cudaError_t smem_opt_in(const void* k, size_t bytes) { return opt_in_smem(k, bytes); }

cudaError_t nn_launch_eval(const Dev& d, const NNState& nn, const double* X, double* F, int write_cache,
                           cudaStream_t s) {
  const size_t sb = nn_smem_bytes(d.n);
  smem_opt_in((const void*)nn_eval_kernel, sb);
  nn_eval_kernel<<<d.n_chains, HQ_THREADS, sb, s>>>(d, nn, X, F, write_cache);
  return cudaGetLastError();
}

cudaError_t nn_launch_inner(const Dev& d, const NNState& nn, const CnnState& cn, int n_inner, int do_local,
                            int do_block, int use_cnn, int window, int site_window, cudaStream_t s) {
  const size_t sb = nn_smem_bytes(d.n, use_cnn != 0);
  smem_opt_in((const void*)nn_inner_kernel, sb);
  nn_inner_kernel<<<d.n_chains, HQ_THREADS, sb, s>>>(d, nn, cn, n_inner, do_local, do_block, use_cnn, window,
                                                      site_window);
  return cudaGetLastError();
}

cudaError_t nn_launch_decide(const Dev& d, const NNState& nn, int restore_g, cudaStream_t s) {
  nn_decide_kernel<<<d.n_chains, HQ_THREADS, 0, s>>>(d, nn, restore_g);
  return cudaGetLastError();
}

cudaError_t nn_launch_loss(const NNState& nn, const double* ys, const int* idx, int B, double scale, cudaStream_t s) {
  nn_loss_kernel<<<1, 32, 0, s>>>(nn, ys, idx, B, scale);
  return cudaGetLastError();
}

cudaError_t nn_launch_set(const NNState& nn, const float* src_device, cudaStream_t s) {
  nn_set_kernel<<<(NN_NP + 255) / 256, 256, 0, s>>>(nn, src_device);
  return cudaGetLastError();
}

// One minibatch: forward, backward partials, reduction (+ Adam step when lr > 0).
cudaError_t nn_launch_batch(const Dev& d, const NNState& nn, const double* Xs, const double* ys, const int* idx,
                            int B, float lr, int t_step, cudaStream_t s) {
  const size_t sf = nn_smem_bytes(d.n);
  smem_opt_in((const void*)nn_batch_forward_kernel, sf);
  nn_batch_forward_kernel<<<B, HQ_THREADS, sf, s>>>(d, nn, Xs, idx, nn.Fb);
  const size_t sbk = train_smem_bytes();
  smem_opt_in((const void*)nn_batch_backward_kernel, sbk);
  nn_batch_backward_kernel<<<kNNTrainCtas, HQ_THREADS, sbk, s>>>(d, nn, Xs, ys, idx, B, nn.Fb, nn.partials);
  nn_adam_kernel<<<(NN_NP + 255) / 256, 256, 0, s>>>(nn, nn.partials, kNNTrainCtas, lr, t_step);
  return cudaGetLastError();
}

}  // namespace hq
