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
// Every kernel evaluates f through nn_tile_f (hq_nn_tc.cuh: 16 patches per warp on the tensor
// cores, bfloat16 operands, FP32 accumulation), so the inner chain and the acceptance see
// bit-identical values of f.
#include <cstdio>
#include "hq_cnn.cuh"
#include "hq_device.cuh"
#include "hq_nn_tc.cuh"
#include "hq_internal.h"
#include "../../include/holstein_dqmc.h"

namespace hq {

// parameter layout: W1[25][64], b1[64], W2[64][64], b2[64], W3[64], b3
constexpr int NN_IN = 25, NN_H = 64;
constexpr int NN_W1 = 0, NN_B1 = NN_IN * NN_H, NN_W2 = NN_B1 + NN_H, NN_B2 = NN_W2 + NN_H * NN_H,
              NN_W3 = NN_B2 + NN_H, NN_B3 = NN_W3 + NN_H, NN_NP = NN_B3 + 1;
static_assert(NN_NP == HQ_NN_PARAMS, "parameter count");
constexpr int NN_WPAD = (NN_NP + 3) & ~3;
constexpr int NN_GROUPS = HQ_THREADS / 8;


struct NNSmem {
  uint2* frag;   // [TC_FRAGS] weight fragments of the tensor-core layers
  float* tcf;    // [TC_FLOATS] b1, b2, W3, b3
  float* f25;    // [32] f of the patches of a local move
  float* pxf;    // [n] network inputs of the proposed values (local moves)
  int* nbr;      // [n][5] cross neighbours of every site: self, +x, -x, +y, -y
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
  size_t b = sizeof(uint2) * TC_FRAGS + sizeof(double) * (HQ_WARPS + 3 * (size_t)n + NN_GROUPS + 8) +
             sizeof(float) * (TC_FLOATS + 32 + (size_t)n) + sizeof(int) * 5 * (size_t)n;
  if (with_cnn) b += sizeof(float) * CN_WPAD + sizeof(int) * (4 + 3 * CN_WIN + 2 * (size_t)n);
  return b;
}

__device__ inline NNSmem nn_carve(int n, char* base, bool with_cnn = false) {
  NNSmem s;
  s.frag = (uint2*)base;
  double* p = (double*)(s.frag + TC_FRAGS);
  s.red = p; p += HQ_WARPS;
  s.pu2 = p; p += n;
  s.pxn = p; p += n;
  s.pds = p; p += n;
  s.gacc = p; p += NN_GROUPS;
  s.scal = p; p += 8;
  float* f = (float*)p;
  s.tcf = f; f += TC_FLOATS;
  s.f25 = f; f += 32;
  s.pxf = f; f += n;
  s.nbr = (int*)f; f += 5 * n;
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

// Position ll * n + j of input k of the patch centred at (l, i): slice ll = l + dl, site j =
// cross point c of i (k = 5 (dl + 2) + c; c = 0 the site itself, then +x, -x, +y, -y).
__device__ __forceinline__ int patch_pos(const Dev& d, int l, int i, int k) {
  const int L = d.L, x = i % d.nx, y = i / d.nx;
  const int dl = k / 5 - 2, cidx = k % 5;
  const int cx_ = (cidx == 1) - (cidx == 2), cy_ = (cidx == 3) - (cidx == 4);
  const int ll = (l + dl + L) % L;
  const int j = (x + cx_ + d.nx) % d.nx + d.nx * ((y + cy_ + d.ny) % d.ny);
  return ll * d.n + j;
}

// Network input of a field value: the value minus the mean field x0, rounded to float.  Every
// kernel forms inputs through this one expression, so a value gives the same input bits
// wherever it is formed.
__device__ __forceinline__ float net_input(double v, double x0) { return (float)(v - x0); }

// xf[k] = net_input(X[k]) for the L N values of a configuration (all threads; ends with a
// barrier).  Each value enters 25 patches: converting it once keeps the FP64 pipe (which does
// the subtraction and the rounding) out of the patch loops.
__device__ inline void to_inputs(const double* X, double x0, float* xf, int NL) {
  for (int k = threadIdx.x; k < NL; k += HQ_THREADS) xf[k] = net_input(X[k], x0);
  __syncthreads();
}

// Warp sum in a fixed order (every lane gets the same bits).
__device__ __forceinline__ double warp_sum_fixed(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(HQ_FULL, v, o);
  return v;
}

// F of one configuration by the whole CTA: warp w takes the tiles of 16 patch rows w, w + 8, ...
// (fixed order); the patch values go to fc when fc != nullptr.  Returns F in every thread.
__device__ inline double fc_eval_all(const Dev& d, const NNSmem& s, const NNFrags& w, const float* xf, float* fc) {
  const int n = d.n, NL = d.n * d.L;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, g = lane >> 2, t = lane & 3;
  double part = 0.0;
  for (int base = warp * 16; base < NL; base += HQ_WARPS * 16) {
    float f0, f1;
    nn_tile_f(w, [&](int row, int k) {
      const int r = base + row < NL ? base + row : NL - 1;
      return xf[patch_pos(d, r / n, r % n, k)];
    }, f0, f1);
    if (t == 0) {
      if (base + g < NL) {
        part += (double)f0;
        if (fc) fc[base + g] = f0;
      }
      if (base + g + 8 < NL) {
        part += (double)f1;
        if (fc) fc[base + g + 8] = f1;
      }
    }
  }
  part = warp_sum_fixed(part);
  if (lane == 0) s.gacc[warp] = part;
  __syncthreads();
  double F = 0.0;
  for (int k = 0; k < HQ_WARPS; ++k) F += s.gacc[k];
  __syncthreads();
  return F;
}

// F(X) of every chain (grid = chains); also refreshes the patch cache fc.
__global__ void __launch_bounds__(HQ_THREADS) nn_eval_kernel(Dev d, NNState nn, const double* Xall, double* Fout,
                                                             int write_cache) {
  extern __shared__ __align__(16) char nraw[];
  const int c = blockIdx.x, n = d.n, NL = d.n * d.L;
  const NNSmem s = nn_carve(n, nraw);
  const NNFrags w = nn_build_frags(nn.wbf, s.frag, s.tcf);
  float* xf = nn.xf + (size_t)c * NL;
  to_inputs(Xall + (size_t)c * NL, nn.x0, xf, NL);
  const double F = fc_eval_all(d, s, w, xf, write_cache ? nn.fcache + (size_t)c * NL : nullptr);
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
  for (int r = threadIdx.x; r < n; r += HQ_THREADS) {
    const int x = r % d.nx, y = r / d.nx;
    s.nbr[5 * r + 0] = r;
    s.nbr[5 * r + 1] = (x + 1) % d.nx + d.nx * y;
    s.nbr[5 * r + 2] = (x - 1 + d.nx) % d.nx + d.nx * y;
    s.nbr[5 * r + 3] = x + d.nx * ((y + 1) % d.ny);
    s.nbr[5 * r + 4] = x + d.nx * ((y - 1 + d.ny) % d.ny);
  }
  const NNFrags w = nn_build_frags(nn.wbf, s.frag, s.tcf);  // (ends with a barrier)
  if (use_cnn) cn_load_weights(cn.wbf, s.cw);
  double* X = d.X + (size_t)c * NL;
  float* xf = nn.xf + (size_t)c * NL;  // inputs of the current fields, kept with X below
  to_inputs(X, nn.x0, xf, NL);
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
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, g = lane >> 2, t = lane & 3;
  const uint32_t* id = d.cid + 4 * (size_t)c;
  const uint32_t key0 = id[0], key1 = id[1], chain = id[2], step = id[3];
  long long nl_acc = 0, nb_acc = 0;
  double path = 0.0;                   // thread 0
  int any_local = 0;                   // thread 0: a local move was accepted in this part
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
      any_local = 0;
      if (fc_stale) {
        fc_eval_all(d, s, w, xf, fc);
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
          s.pxf[i] = net_input(xn, nn.x0);
          s.pds[i] = kfac * kin + pfac * (xn * xn - xo * xo);
        }
        __syncthreads();
        // The moves of the slice run in warp 0 alone: a move's 25 patches are two tensor-core
        // tiles, its change of F a fixed-order warp sum, and the decision, the field and the
        // patch cache are updated without a CTA barrier (the other warps wait for the slice).
        if (warp == 0) {
          for (int i0 = 0; i0 < n; ++i0) {
            const int i = fwd ? i0 : n - 1 - i0;
            const double xn = s.pxn[i];
            // patch q = 5 (dl + 2) + c contains (sl, i): centre slice sl - dl, centre site the
            // neighbour of i opposite to c (q >= 25: padding rows)
            auto cslice = [&](int q) {
              const int v = sl - (q / 5 - 2);
              return v < 0 ? v + L : (v >= L ? v - L : v);
            };
            auto csite = [&](int q) {
              const int c = q % 5;
              return s.nbr[5 * i + (c == 0 ? 0 : (c & 1) ? c + 1 : c - 1)];
            };
            auto zv = [&](int q, int k) -> float {
              q = q < 25 ? q : 24;
              int ll = sl - (q / 5 - 2) + (k / 5 - 2);
              ll = ll < 0 ? ll + L : (ll >= L ? ll - L : ll);
              const int site = s.nbr[5 * csite(q) + k % 5];
              return (ll == sl && site == i) ? s.pxf[i] : xf[(size_t)ll * n + site];
            };
            float fv[4];
            nn_tile_f(w, [&](int row, int k) { return zv(row, k); }, fv[0], fv[1]);
            nn_tile_f(w, [&](int row, int k) { return zv(16 + row, k); }, fv[2], fv[3]);
            const int qs[4] = {g, g + 8, 16 + g, 24 + g};
            double part = 0.0;
            if (t == 0)
              for (int a = 0; a < 4; ++a)
                if (qs[a] < 25) part += (double)fv[a] - (double)fc[(size_t)cslice(qs[a]) * n + csite(qs[a])];
            const double dF = warp_sum_fixed(part);
            int acc = 0;
            if (lane == 0) {
              const double prob = exp(fmin(2.0 * dF - s.pds[i], 709.0));
              acc = s.pu2[i] < prob;
              if (acc) {
                X[(size_t)sl * n + i] = xn;
                xf[(size_t)sl * n + i] = s.pxf[i];
                path += dF;
                any_local = 1;
              }
              nl_acc += acc;
            }
            acc = __shfl_sync(HQ_FULL, acc, 0);
            if (acc && t == 0)
              for (int a = 0; a < 4; ++a)
                if (qs[a] < 25) fc[(size_t)cslice(qs[a]) * n + csite(qs[a])] = fv[a];
            __syncwarp();
          }
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) s.scal[3] = any_local;
      __syncthreads();
      if (s.scal[3] != 0.0) cn_stale = true;
      __syncthreads();
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
          // the 5 L patches containing site i: patch q has centre (q / 5, i - c), c = q % 5; warp
          // w takes the tiles w, w + 8, ... of 16 patches
          auto centre = [&](int q) {
            const int cidx = q % 5, sl = q / 5;
            const int cx_ = (cidx == 1) - (cidx == 2), cy_ = (cidx == 3) - (cidx == 4);
            const int j = (x - cx_ + d.nx) % d.nx + d.nx * ((y - cy_ + d.ny) % d.ny);
            return sl * n + j;
          };
          double pt = 0.0;
          for (int base = warp * 16; base < 5 * L; base += HQ_WARPS * 16) {
            float f0, f1;
            nn_tile_f(w, [&](int row, int k) {
              const int q = base + row < 5 * L ? base + row : 5 * L - 1;
              const int r = centre(q);
              const int pos = patch_pos(d, r / n, r % n, k);
              return pos % n == i ? net_input(X[pos] + dx, nn.x0) : xf[pos];
            }, f0, f1);
            if (t == 0) {
              const int q0 = base + g, q1 = q0 + 8;
              if (q0 < 5 * L) {
                fnew[q0] = f0;
                pt += (double)f0 - (double)fc[centre(q0)];
              }
              if (q1 < 5 * L) {
                fnew[q1] = f1;
                pt += (double)f1 - (double)fc[centre(q1)];
              }
            }
          }
          pt = warp_sum_fixed(pt);
          if (lane == 0) s.gacc[warp] = pt;
          __syncthreads();
          dF = 0.0;
          for (int k = 0; k < HQ_WARPS; ++k) dF += s.gacc[k];
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
          for (int sl = threadIdx.x; sl < L; sl += HQ_THREADS) {
            const double v = X[(size_t)sl * n + i] + dx;
            X[(size_t)sl * n + i] = v;
            xf[(size_t)sl * n + i] = net_input(v, nn.x0);
          }
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
// Mean squared error (1/B) sum_a (F(X_a) - y_a)^2 over a minibatch.  Forward: F_a per sample
// (nn_batch_forward_kernel, the same tensor-core tiles as every other evaluation).  Backward:
// nn_batch_backward_tc_kernel, per-CTA partial gradients summed in a fixed order by the Adam
// kernel.

__global__ void __launch_bounds__(HQ_THREADS) nn_batch_forward_kernel(Dev d, NNState nn, const double* Xs,
                                                                      const int* idx, double* Fb) {
  extern __shared__ __align__(16) char nraw[];
  const int a = blockIdx.x, n = d.n, NL = d.n * d.L;
  const NNSmem s = nn_carve(n, nraw);
  const NNFrags w = nn_build_frags(nn.wbf, s.frag, s.tcf);
  float* xa = nn.xb + (size_t)a * NL;  // read again by the backward pass
  to_inputs(Xs + (size_t)idx[a] * NL, nn.x0, xa, NL);
  const double F = fc_eval_all(d, s, w, xa, nullptr);
  if (threadIdx.x == 0) Fb[a] = F;
}

// Backward pass on the tensor cores (see hq_nn_tc.cuh): CTA k takes the 128-row chunks k, k +
// grid, ... of the minibatch's rows (row R = sample a * L N + patch), warp w rows 16 w .. 16 w + 15
// of a chunk.  Inputs come from nn.xb, written by the forward kernel.  partials[k] receives the
// CTA's gradient (every entry written once).
__global__ void __launch_bounds__(HQ_THREADS) nn_batch_backward_tc_kernel(Dev d, NNState nn,
                                                                          const double* ys, const int* idx, int B,
                                                                          const double* Fb, float* partials) {
  extern __shared__ __align__(16) char nraw[];
  const int n = d.n, NL = d.n * d.L, rows = B * NL;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, g = lane >> 2, t = lane & 3;
  uint2* frag = (uint2*)nraw;
  float* tcf = (float*)(frag + TR_FRAGS);
  float* colp = tcf + TC_FLOATS;              // [3][8 warps][64] column partials, then gb3 [8]
  uint16_t* h1h = (uint16_t*)(colp + 3 * 8 * TC_H + 8);
  uint16_t* h1l = h1h + TC_H * TR_LD;
  uint16_t* d2h = h1l + TC_H * TR_LD;
  uint16_t* d2l = d2h + TC_H * TR_LD;
  uint16_t* zh = d2l + TC_H * TR_LD;
  uint16_t* zl = zh + TC_K1 * TR_LD;
  uint16_t* d1h = zl + TC_K1 * TR_LD;
  uint16_t* d1l = d1h + TC_H * TR_LD;
  const NNFrags w = nn_build_frags(nn.wbf, frag, tcf);
  // W2^T fragments for d1 = d2 W2^T: B[k = u][n = v] = W2[v][u]
  uint2* w2t = frag + TC_FRAGS;
  for (int e = threadIdx.x; e < 4 * 8 * 32; e += HQ_THREADS) {
    const int ln = e % 32, j = (e / 32) % 8, st = e / 256;
    const int gg = ln >> 2, tt = ln & 3, v = 8 * j + gg, u = 16 * st + 2 * tt;
    const uint16_t* row = nn.wbf + NN_W2 + v * NN_H;
    w2t[e] = make_uint2(pack_bf16(row[u], row[u + 1]), pack_bf16(row[u + 8], row[u + 9]));
  }
  __syncthreads();
  // owned accumulators: gW2 block (m-tile warp/2, n-tiles 4 (warp%2) ..), gW1 block (m-tile
  // warp/4, n-tiles 2 (warp%4) ..), column partials of this lane's 16 columns
  float gw2[4][4], gw1[2][4], cw3[16], cb2[16], cb1[16], cb3 = 0.f;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int e = 0; e < 4; ++e) gw2[a][e] = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int e = 0; e < 4; ++e) gw1[a][e] = 0.f;
#pragma unroll
  for (int c = 0; c < 16; ++c) cw3[c] = cb2[c] = cb1[c] = 0.f;
  const int nchunk = (rows + TR_ROWS - 1) / TR_ROWS;
  for (int chunk = blockIdx.x; chunk < nchunk; chunk += gridDim.x) {
    const int r0 = chunk * TR_ROWS + 16 * warp;
    auto rowpos = [&](int row, int& a, int& pr) {
      const int R = r0 + row < rows ? r0 + row : rows - 1;
      a = R / NL;
      pr = R % NL;
    };
    // forward of the warp's 16 rows, keeping what the backward pass needs
    float acc1[8][4], acc2[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc1[j][e] = acc2[j][e] = 0.f;
#pragma unroll
    for (int st = 0; st < 2; ++st) {
      uint32_t ahi[4], alo[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = g + 8 * (q & 1);
        const int k = 16 * st + 2 * t + 8 * (q >> 1);
        int a, pr;
        rowpos(row, a, pr);
        const float* xa = nn.xb + (size_t)a * NL;  // the minibatch inputs of the forward kernel
        const float v0 = k < TC_IN ? xa[patch_pos(d, pr / n, pr % n, k)] : 0.f;
        const float v1 = k + 1 < TC_IN ? xa[patch_pos(d, pr / n, pr % n, k + 1)] : 0.f;
        split2(v0, v1, ahi[q], alo[q]);
        // z^T staging (rows k >= 25 are zero)
        zh[k * TR_LD + 16 * warp + row] = (uint16_t)(ahi[q] & 0xffffu);
        zl[k * TR_LD + 16 * warp + row] = (uint16_t)(alo[q] & 0xffffu);
        zh[(k + 1) * TR_LD + 16 * warp + row] = (uint16_t)(ahi[q] >> 16);
        zl[(k + 1) * TR_LD + 16 * warp + row] = (uint16_t)(alo[q] >> 16);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint2 b = w.w1[(st * 8 + j) * 32 + lane];
        mma_bf16(acc1[j], ahi, b);
        mma_bf16(acc1[j], alo, b);
      }
    }
    // a1 -> h1 (kept as hi/lo A fragments and staged transposed), masks in acc1's sign
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int v = 8 * j + 2 * t;
      acc1[j][0] += w.b1[v];
      acc1[j][1] += w.b1[v + 1];
      acc1[j][2] += w.b1[v];
      acc1[j][3] += w.b1[v + 1];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        uint16_t hh, hl;
        split1(fmaxf(acc1[j][e], 0.f), hh, hl);
        const int col = v + (e & 1), row = g + 8 * (e >> 1);
        h1h[col * TR_LD + 16 * warp + row] = hh;
        h1l[col * TR_LD + 16 * warp + row] = hl;
      }
    }
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      uint32_t ahi[4], alo[4];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int j = 2 * st + half;
        split2(fmaxf(acc1[j][0], 0.f), fmaxf(acc1[j][1], 0.f), ahi[2 * half], alo[2 * half]);
        split2(fmaxf(acc1[j][2], 0.f), fmaxf(acc1[j][3], 0.f), ahi[2 * half + 1], alo[2 * half + 1]);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint2 b = w.w2[(st * 8 + j) * 32 + lane];
        mma_bf16(acc2[j], ahi, b);
        mma_bf16(acc2[j], alo, b);
      }
    }
    // output gradients of the two rows of this lane
    float dout[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int a, pr;
      rowpos(g + 8 * h, a, pr);
      dout[h] = (r0 + g + 8 * h < rows) ? (float)(2.0 * (Fb[a] - ys[idx[a]]) / B) : 0.f;
    }
    if (t == 0) cb3 += dout[0] + dout[1];
    // d2 = relu'(a2) dout W3 (in acc2), gW3 and gb2 column sums, d2 staged transposed
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int u = 8 * j + 2 * t + (e & 1), row = g + 8 * (e >> 1);
        const float a2 = acc2[j][e] + w.b2[u];
        const float dv = a2 > 0.f ? dout[e >> 1] * w.w3[u] : 0.f;
        cw3[2 * j + (e & 1)] = fmaf(fmaxf(a2, 0.f), dout[e >> 1], cw3[2 * j + (e & 1)]);
        cb2[2 * j + (e & 1)] += dv;
        acc2[j][e] = dv;
        uint16_t hh, hl;
        split1(dv, hh, hl);
        d2h[u * TR_LD + 16 * warp + row] = hh;
        d2l[u * TR_LD + 16 * warp + row] = hl;
      }
    }
    // d1 = relu'(a1) (d2 W2^T)
    float acc3[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc3[j][e] = 0.f;
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      uint32_t ahi[4], alo[4];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int j = 2 * st + half;
        split2(acc2[j][0], acc2[j][1], ahi[2 * half], alo[2 * half]);
        split2(acc2[j][2], acc2[j][3], ahi[2 * half + 1], alo[2 * half + 1]);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint2 b = w2t[(st * 8 + j) * 32 + lane];
        mma_bf16(acc3[j], ahi, b);
        mma_bf16(acc3[j], alo, b);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int v = 8 * j + 2 * t + (e & 1), row = g + 8 * (e >> 1);
        const float dv = acc1[j][e] > 0.f ? acc3[j][e] : 0.f;
        cb1[2 * j + (e & 1)] += dv;
        uint16_t hh, hl;
        split1(dv, hh, hl);
        d1h[v * TR_LD + 16 * warp + row] = hh;
        d1l[v * TR_LD + 16 * warp + row] = hl;
      }
    }
    __syncthreads();
    // gW2 = h1^T d2 and gW1 = z^T d1 over the chunk's 128 rows
#pragma unroll
    for (int ks = 0; ks < TR_ROWS / 16; ++ks) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
        mma_tiles3(gw2[a], h1h, h1l, d2h, d2l, 16 * (warp / 2), 8 * (4 * (warp % 2) + a), 16 * ks);
#pragma unroll
      for (int a = 0; a < 2; ++a)
        mma_tiles3(gw1[a], zh, zl, d1h, d1l, 16 * (warp / 4), 8 * (2 * (warp % 4) + a), 16 * ks);
    }
    __syncthreads();
  }
  // column sums: over the 8 row groups of the warp, then over the warps (fixed order)
#pragma unroll
  for (int c = 0; c < 16; ++c) {
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      cw3[c] += __shfl_xor_sync(HQ_FULL, cw3[c], o);
      cb2[c] += __shfl_xor_sync(HQ_FULL, cb2[c], o);
      cb1[c] += __shfl_xor_sync(HQ_FULL, cb1[c], o);
    }
  }
#pragma unroll
  for (int o = 4; o < 32; o <<= 1) cb3 += __shfl_xor_sync(HQ_FULL, cb3, o);
  if (g == 0) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int u = 8 * j + 2 * t + e;
        colp[(0 * 8 + warp) * TC_H + u] = cw3[2 * j + e];
        colp[(1 * 8 + warp) * TC_H + u] = cb2[2 * j + e];
        colp[(2 * 8 + warp) * TC_H + u] = cb1[2 * j + e];
      }
    if (t == 0) colp[3 * 8 * TC_H + warp] = cb3;
  }
  __syncthreads();
  float* out = partials + (size_t)blockIdx.x * NN_WPAD;
  // gW2 [v][u] at NN_W2 + v * 64 + u: C rows = v (m-tile warp / 2), cols = u
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int v0 = 16 * (warp / 2) + g, u0 = 8 * (4 * (warp % 2) + a) + 2 * t;
    out[NN_W2 + v0 * NN_H + u0] = gw2[a][0];
    out[NN_W2 + v0 * NN_H + u0 + 1] = gw2[a][1];
    out[NN_W2 + (v0 + 8) * NN_H + u0] = gw2[a][2];
    out[NN_W2 + (v0 + 8) * NN_H + u0 + 1] = gw2[a][3];
  }
  // gW1 [k][v] at NN_W1 + k * 64 + v for k < 25
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int k0 = 16 * (warp / 4) + g, v0 = 8 * (2 * (warp % 4) + a) + 2 * t;
    if (k0 < NN_IN) {
      out[NN_W1 + k0 * NN_H + v0] = gw1[a][0];
      out[NN_W1 + k0 * NN_H + v0 + 1] = gw1[a][1];
    }
    if (k0 + 8 < NN_IN) {
      out[NN_W1 + (k0 + 8) * NN_H + v0] = gw1[a][2];
      out[NN_W1 + (k0 + 8) * NN_H + v0 + 1] = gw1[a][3];
    }
  }
  for (int e = threadIdx.x; e < 3 * TC_H + 1; e += HQ_THREADS) {
    float acc = 0.f;
    if (e < 3 * TC_H) {
      const int which = e / TC_H, u = e % TC_H;
      for (int ww = 0; ww < 8; ++ww) acc += colp[(which * 8 + ww) * TC_H + u];
      out[(which == 0 ? NN_W3 : which == 1 ? NN_B2 : NN_B1) + u] = acc;
    } else {
      for (int ww = 0; ww < 8; ++ww) acc += colp[3 * 8 * TC_H + ww];
      out[NN_B3] = acc;
    }
  }
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
  const size_t sbk = nn_train_tc_smem_bytes();
  smem_opt_in((const void*)nn_batch_backward_tc_kernel, sbk);
  // one wave: one CTA per SM (the kernel takes a whole SM's registers), at most kNNTrainCtas
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = kNNTrainCtas;
  }
  const int grid = sms < kNNTrainCtas ? sms : kNNTrainCtas;
  nn_batch_backward_tc_kernel<<<grid, HQ_THREADS, sbk, s>>>(d, nn, ys, idx, B, nn.Fb, nn.partials);
  nn_adam_kernel<<<(NN_NP + 255) / 256, 256, 0, s>>>(nn, nn.partials, grid, lr, t_step);
  return cudaGetLastError();
}

}  // namespace hq
