// Kernels of the Holstein DQMC engine: one CTA per Markov chain, FP64 throughout.
//
//   stack_build   fields -> left UDV stack of B_L..B_{b+1} at every restabilisation
//                 boundary b, fresh G_0 and log|det M|           (DQMC section: M = I + B_L..B_1)
//   local_phase   n_wrap-slice chunks of local Metropolis moves with delayed rank-k updates of
//                 G and the wrap G <- B_l G B_l^-1, then the right UDV update and a fresh
//                 G_l from the right factors and the left stack  (local updates at each
//                 spacetime point, fast update of the paper's ref. WhitePRB1989)
//   global_move   one block move X(i, .) += dX per chain with the full stabilised
//                 determinant ratio                              (block updates)
//   sweep_end     per-sweep observable records
#include <cstdio>
#include <mutex>
#include <utility>
#include <vector>
#include "hq_device.cuh"
#include "hq_internal.h"
#include "../../include/holstein_dqmc.h"

namespace hq {

int section_cycles(unsigned long long* out, int n) {
#ifdef HQ_SECTION_TIMING
  if (n > SEC_COUNT) n = SEC_COUNT;
  if (cudaMemcpyFromSymbol(out, g_section_cycles, sizeof(unsigned long long) * n) != cudaSuccess) return -1;
  unsigned long long zero[SEC_COUNT] = {0};
  cudaMemcpyToSymbol(g_section_cycles, zero, sizeof(zero));
  return n;
#else
  (void)out;
  (void)n;
  return 0;
#endif
}

struct Smem {
  double *ex, *exi, *ey, *eyi;
  double *dl, *u2, *xn, *dlt, *es, *dcorr, *tau, *norm2, *rinv, *vs, *dv, *rd;
  double *red, *scal;
  double *wv, *ws;  // blocked QR scratch (16-wide class only, else nullptr)
  int *perm, *piv, *sint;
};

static constexpr int kSmemVecs = 13;  // vs takes two

// Kernel template class of a lattice: the largest side rounded up to 2, 4, 8 or 16.
static inline int lmax_of(int nx, int ny) {
  const int m = nx > ny ? nx : ny;
  return m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : 16;
}

// doubles of the blocked QR scratch: the panel copy (n rows of kQbLd) and S (kQb x kQb)
__host__ __device__ inline size_t smem_qr_doubles(bool blocked, int n) {
  return blocked ? (size_t)n * kQbLd + kQb * kQb : 0;
}

// Shared memory of one chain's CTA in a kernel instantiated for class LMAX (`blocked` =
// qr_blocked_class(LMAX)): the layout of carve<LMAX>.
__host__ __device__ inline size_t smem_layout_bytes(int nx, int ny, int n, bool blocked) {
  return (size_t)(2 * nx * nx + 2 * ny * ny + kSmemVecs * n + 32 + 16) * sizeof(double) +
         smem_qr_doubles(blocked, n) * sizeof(double) + (size_t)(2 * n + 8) * sizeof(int);
}

size_t smem_bytes(const Dev& d) {
  return smem_layout_bytes(d.nx, d.ny, d.n, qr_blocked_class(lmax_of(d.nx, d.ny)));
}

size_t smem_bytes_class(const Dev& d, int lmax) { return smem_layout_bytes(d.nx, d.ny, d.n, qr_blocked_class(lmax)); }

template <int LMAX>
__device__ inline Smem carve(const Dev& d, double* base) {
  Smem s;
  double* p = base;
  const int n = d.n;
  s.ex = p; p += d.nx * d.nx;
  s.exi = p; p += d.nx * d.nx;
  s.ey = p; p += d.ny * d.ny;
  s.eyi = p; p += d.ny * d.ny;
  s.dl = p; p += n;
  s.u2 = p; p += n;
  s.xn = p; p += n;
  s.dlt = p; p += n;
  s.es = p; p += n;
  s.dcorr = p; p += n;
  s.tau = p; p += n;
  s.norm2 = p; p += n;
  s.rinv = p; p += n;
  s.vs = p; p += 2 * n;
  s.dv = p; p += n;
  s.rd = p; p += n;
  s.red = p; p += 32;
  s.scal = p; p += 16;
  // 16-byte aligned: every count above is even (nx, ny and n are even)
  s.wv = nullptr;
  s.ws = nullptr;
  if (qr_blocked_class(LMAX)) {
    s.wv = p; p += (size_t)n * kQbLd;
    s.ws = p; p += kQb * kQb;
  }
  int* q = reinterpret_cast<int*>(p);
  s.perm = q; q += n;
  s.piv = q; q += n;
  s.sint = q;
  return s;
}

__device__ inline void load_kinetic(const Dev& d, const Smem& s) {
  const int a = d.nx * d.nx, b = d.ny * d.ny;
  for (int i = threadIdx.x; i < 2 * a + 2 * b; i += HQ_THREADS) s.ex[i] = d.kin[i];  // contiguous
  __syncthreads();
}

__device__ inline double* chain_work(const Dev& d, int c, int slot) {
  return d.work + ((size_t)c * kWorkMats + slot) * (size_t)d.n * d.n;
}

__device__ inline void flag_nonfinite(const Dev& d, int c, double v) {
  if (!isfinite(v)) d.status[c] = HQ_ENAN;
}

// log|det(I + U D T)| from the last UDV factors (D in sm.dv):
// I + U D T = U Db (Db^-1 U^T + Ds T), so log|det| = sum log Db + log|det A|.  With G0,
// also G_0 = (I + (B_L..B_1)^T)^-T = Y^T with Y = A^-1 Db^-1 U^T.
__device__ double finish_logdet(const Dev& d, int c, const Smem& sm, const double* U, const double* Tc, double* G0) {
  const int n = d.n;
  HQ_TIC(ld);
  double* A = chain_work(d, c, WK_M1);
  double* Y = chain_work(d, c, WK_M2);
  for (int i = threadIdx.x; i < n; i += HQ_THREADS) sm.rinv[i] = 1.0 / fmax(sm.dv[i], 1.0);
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
    const int i = idx % n, col = idx / n;
    const double ds = fmin(sm.dv[i], 1.0);
    const double ut = U[(size_t)i * n + col] * sm.rinv[i];
    A[(size_t)col * n + i] = fma(ds, Tc[(size_t)col * n + i], ut);
    if (G0) Y[(size_t)col * n + i] = ut;
  }
  double lsum = 0.0;
  for (int i = threadIdx.x; i < n; i += HQ_THREADS) lsum += log(fmax(sm.dv[i], 1.0));
  const double lb = block_sum(lsum, sm.red);
  const double la = lu_logdet_blocked(A, n, n, sm.piv, sm.sint, sm.red);
  if (G0) {
    lu_diag_recip(A, n, n, sm.rd);
    lu_solve_blocked(A, n, n, sm.piv, sm.rd, Y);
    for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
      const int r = idx % n, col = idx / n;
      G0[(size_t)col * n + r] = Y[(size_t)r * n + col];
    }
    __syncthreads();
  }
  HQ_TOC(ld, SEC_LOGDET);
  return lb + la;
}

// UDV factors of the transposed top-down product (B_L .. B_1)^T = B_1^T .. B_L^T, built
// by left-multiplying B_s^T = exp(-dtau V_s) exp(-dtau K) for s = L-1 .. 0 and refactoring
// by pivoted QR after every chunk that ends on a restabilisation boundary.  The field at
// `site` (if >= 0) is shifted by dx in every slice (block-move proposal).  With `store`
// the factors at each boundary b > 0 go to the left stack.  Returns log|det M|; with
// G0 != nullptr also writes G_0 = (I + B_L..B_1)^-1.  With stop > 0 (a boundary) only the
// slices above it are taken: the factors end in the stack slot of `stop` and 0 is returned.
template <int LMAX>
__device__ double udv_top_down(const Dev& d, int c, const Smem& sm, const double* X, int site, double dx,
                               bool store, double* G0, int stop = 0) {
  const int n = d.n, L = d.L, nw = d.n_wrap;
  double* P = chain_work(d, c, WK_P);
  double* U = chain_work(d, c, WK_U);
  double* Tc = chain_work(d, c, WK_T);
  double* Tn = chain_work(d, c, WK_T2);
  double* Q = chain_work(d, c, WK_M1);
  const QrScratch qs{sm.tau, sm.vs, sm.rinv, sm.perm, sm.sint, sm.wv, sm.ws};
  int hi = L, lo = ((L - 1) / nw) * nw;
  bool first = true;
  while (true) {
    if (first) set_identity(P, n, n);
    else copy_scale_cols(P, U, n, n, sm.dv);
    __syncthreads();
    for (int s = hi - 1; s >= lo; --s) {
      HQ_TIC(dl);
      for (int r = threadIdx.x; r < n; r += HQ_THREADS) {
        double x = X[(size_t)s * n + r];
        if (r == site) x = x + dx;
        sm.dl[r] = exp(-d.dtau * (d.g * x - d.mu));
      }
      HQ_TOC(dl, SEC_DL);
      HQ_TIC(kin);
      // B_s^T P = exp(-dtau V_s) exp(-dtau K) P (the scaling reads dl after kin_rows' barrier)
      kin_rows<LMAX, KIN_SCALE_AFTER>(P, n, n, sm.ex, sm.ey, d.nx, d.ny, sm.dl);
      HQ_TOC(kin, SEC_KIN);
    }
    HQ_TIC(pp);
    prepivot<qr_group<LMAX>()>(P, Q, n, n, qs, sm.norm2);
    HQ_TOC(pp, SEC_PREPIVOT);
    HQ_TIC(qr);
    qr_factor<LMAX>(Q, n, n, qs);
    HQ_TOC(qr, SEC_QR);
    HQ_TIC(fq);
    qr_form_q<LMAX>(Q, n, n, U, qs);
    HQ_TOC(fq, SEC_FORMQ);
    HQ_TIC(tu);
    t_update(Q, n, n, qs, sm.dv, first ? nullptr : Tc, Tn, P);
    HQ_TOC(tu, SEC_TUPD);
    double* t = Tc; Tc = Tn; Tn = t;
    if (store && lo > 0) {
      const size_t b = (size_t)c * d.n_bound + (lo / nw - 1);
      copy_mat(d.stU + b * n * n, U, n, n);
      copy_mat(d.stT + b * n * n, Tc, n, n);
      for (int r = threadIdx.x; r < n; r += HQ_THREADS) d.stD[b * n + r] = sm.dv[r];
      __syncthreads();
    }
    first = false;
    if (lo <= stop) break;
    hi = lo;
    lo -= nw;
  }
  // with stop > 0 the factors of (B_L .. B_{stop+1})^T are in the stack slot of boundary stop
  return stop > 0 ? 0.0 : finish_logdet(d, c, sm, U, Tc, G0);
}

template <int LMAX>
__device__ void stack_build_body(const Dev& d, int c, double* smraw) {
  if (!d.active[c]) return;
  const Smem sm = carve<LMAX>(d, smraw);
  load_kinetic(d, sm);
  const double* X = d.X + (size_t)c * d.L * d.n;
  double* G = d.G + (size_t)c * d.n * d.n;
  const double ld = udv_top_down<LMAX>(d, c, sm, X, -1, 0.0, true, G);
  if (threadIdx.x == 0) {
    d.logdet[c] = ld;
    flag_nonfinite(d, c, ld);
  }
}

template <int LMAX>
__global__ void __launch_bounds__(HQ_THREADS) stack_build_kernel(Dev d) {
  extern __shared__ __align__(16) double smraw[];
  stack_build_body<LMAX>(d, blockIdx.x, smraw);
}

// ---------------------------------------------- log|det M| from two halves at once
// For few chains (2 C <= SMs) the stabilised product is built by two CTAs per chain: one takes
// the slices above the split boundary m (left factors (B_L..B_{m+1})^T into the stack slot of
// m, exactly as the stack build), the other the slices below it (right factors
// B_m..B_1 = UR DR TR, as the local phase's restabilisation).  A second launch joins them with
// the two-sided formula (green_two_sided): log|det M| and G_m.  The per-chain work matrices are
// shared out so that the halves never touch the same buffer: the top half uses P, U, T, T2,
// M1; the bottom half M2, M3 and the chain's G (overwritten by the join anyway).
template <int LMAX>
__device__ void udv_bottom_half(const Dev& d, int c, const Smem& sm, int m) {
  const int n = d.n, nw = d.n_wrap;
  const double* X = d.X + (size_t)c * d.L * n;
  double* UR = d.UR + (size_t)c * n * n;
  double* TR = d.TR + (size_t)c * n * n;
  double* DR = d.DR + (size_t)c * n;
  double* P = chain_work(d, c, WK_M2);
  double* Q = chain_work(d, c, WK_M3);
  double* T2 = d.G + (size_t)c * n * n;
  const QrScratch qs{sm.tau, sm.vs, sm.rinv, sm.perm, sm.sint, sm.wv, sm.ws};
  for (int s0 = 0; s0 < m; s0 += nw) {
    const int s1 = s0 + nw < m ? s0 + nw : m;
    const bool first = (s0 == 0);
    if (first) set_identity(P, n, n);
    else copy_scale_cols(P, UR, n, n, DR);
    __syncthreads();
    for (int s = s0; s < s1; ++s) {
      for (int r = threadIdx.x; r < n; r += HQ_THREADS) sm.dl[r] = exp(-d.dtau * (d.g * X[(size_t)s * n + r] - d.mu));
      __syncthreads();
      // B_s P = exp(-dtau K) exp(-dtau V_s) P
      kin_rows<LMAX, KIN_SCALE_BEFORE>(P, n, n, sm.ex, sm.ey, d.nx, d.ny, sm.dl);
    }
    prepivot<qr_group<LMAX>()>(P, Q, n, n, qs, sm.norm2);
    qr_factor<LMAX>(Q, n, n, qs);
    qr_form_q<LMAX>(Q, n, n, UR, qs);
    t_update(Q, n, n, qs, DR, first ? nullptr : TR, T2, P);
    copy_mat(TR, T2, n, n);
    __syncthreads();
  }
}

template <int LMAX>
__global__ void __launch_bounds__(HQ_THREADS) split_halves_kernel(Dev d, int m) {
  extern __shared__ __align__(16) double smraw[];
  const int C = d.n_chains;
  const int c = blockIdx.x % C;
  if (!d.active[c]) return;
  const Smem sm = carve<LMAX>(d, smraw);
  load_kinetic(d, sm);
  if (blockIdx.x < C) {
    udv_top_down<LMAX>(d, c, sm, d.X + (size_t)c * d.L * d.n, -1, 0.0, true, nullptr, m);
  } else {
    udv_bottom_half<LMAX>(d, c, sm, m);
  }
}

__device__ double green_two_sided(const Dev& d, int c, const Smem& sm, int l, double* Gf);

template <int LMAX>
__global__ void __launch_bounds__(HQ_THREADS) split_join_kernel(Dev d, int m) {
  extern __shared__ __align__(16) double smraw[];
  const int c = blockIdx.x;
  if (!d.active[c]) return;
  const Smem sm = carve<LMAX>(d, smraw);
  const double ld = green_two_sided(d, c, sm, m, d.G + (size_t)c * d.n * d.n);
  if (threadIdx.x == 0) {
    d.logdet[c] = ld;
    flag_nonfinite(d, c, ld);
  }
}

// Fresh G_l at boundary l from the right factors (B_l..B_1 = UR DR TR) and, if l < L,
// the left stack ((B_L..B_{l+1})^T = UL DL TL):
//   G_l = UL DLb^-1 [DRb^-1 UR^T UL DLb^-1 + DRs TR TL^T DLs]^-1 DRb^-1 UR^T.
// Returns log|det M|; G_l goes to Gf.
__device__ double green_two_sided(const Dev& d, int c, const Smem& sm, int l, double* Gf) {
  const int n = d.n;
  const double* UR = d.UR + (size_t)c * n * n;
  const double* TR = d.TR + (size_t)c * n * n;
  const double* DR = d.DR + (size_t)c * n;
  double* M1 = chain_work(d, c, WK_M1);
  double* M2 = chain_work(d, c, WK_M2);
  double* M3 = chain_work(d, c, WK_M3);
  double lsum = 0.0;
  double la;
  if (l < d.L) {
    const size_t b = (size_t)c * d.n_bound + (l / d.n_wrap - 1);
    const double* UL = d.stU + b * n * n;
    const double* TL = d.stT + b * n * n;
    const double* DL = d.stD + b * n;
    // reciprocals of the large parts DRb = max(DR, 1), DLb = max(DL, 1) (one division each)
    double* rdr = sm.rinv;
    double* rdl = sm.norm2;
    for (int i = threadIdx.x; i < n; i += HQ_THREADS) {
      rdr[i] = 1.0 / fmax(DR[i], 1.0);
      rdl[i] = 1.0 / fmax(DL[i], 1.0);
    }
    gemm_nn<true, false>(n, UR, UL, M1, n);   // UR^T UL (ends with a barrier)
    gemm_nn<false, true>(n, TR, TL, M2, n);   // TR TL^T
    for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
      const int i = idx % n, j = idx / n;
      const double drs = fmin(DR[i], 1.0), dls = fmin(DL[j], 1.0);
      const size_t o = (size_t)j * n + i;
      M2[o] = fma(M1[o] * rdr[i], rdl[j], drs * M2[o] * dls);
      M3[o] = UR[(size_t)i * n + j] * rdr[i];
    }
    for (int i = threadIdx.x; i < n; i += HQ_THREADS) lsum += log(fmax(DR[i], 1.0)) + log(fmax(DL[i], 1.0));
    __syncthreads();
    la = lu_logdet_blocked(M2, n, n, sm.piv, sm.sint, sm.red);
    lu_diag_recip(M2, n, n, sm.rd);
    lu_solve_blocked(M2, n, n, sm.piv, sm.rd, M3);
    // M1 <- UL DLb^-1, Gf = M1 M3
    for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
      const int j = idx / n;
      M1[idx] = UL[idx] * rdl[j];
    }
    __syncthreads();
    gemm_nn<false, false>(n, M1, M3, Gf, n);
  } else {
    double* rdr = sm.rinv;
    for (int i = threadIdx.x; i < n; i += HQ_THREADS) rdr[i] = 1.0 / fmax(DR[i], 1.0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
      const int i = idx % n, j = idx / n;
      const double drs = fmin(DR[i], 1.0);
      const double ut = UR[(size_t)i * n + j] * rdr[i];
      M2[(size_t)j * n + i] = fma(drs, TR[(size_t)j * n + i], ut);
      Gf[(size_t)j * n + i] = ut;
    }
    for (int i = threadIdx.x; i < n; i += HQ_THREADS) lsum += log(fmax(DR[i], 1.0));
    __syncthreads();
    la = lu_logdet_blocked(M2, n, n, sm.piv, sm.sint, sm.red);
    lu_diag_recip(M2, n, n, sm.rd);
    lu_solve_blocked(M2, n, n, sm.piv, sm.rd, Gf);
  }
  return block_sum(lsum, sm.red) + la;
}

// Electronic observables from a fresh G (Wick; both spins share G), added to the chain's
// per-sweep accumulators.
__device__ void measure_green(const Dev& d, int c, const Smem& sm, const double* G) {
  const int n = d.n;
  double sm_m = 0.0, sm_m2 = 0.0, sm_sm = 0.0, sm_g = 0.0, conn = 0.0;
  for (int r = threadIdx.x; r < n; r += HQ_THREADS) {
    const double g = G[(size_t)r * n + r];
    const double m = 1.0 - g;
    const double sg = (((r % d.nx) + (r / d.nx)) & 1) ? -1.0 : 1.0;
    sm_m += m;
    sm_m2 += m * m;
    sm_sm += sg * m;
    sm_g += g;
  }
  for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
    const int r = idx % n, col = idx / n;
    const double sr = (((r % d.nx) + (r / d.nx)) & 1) ? -1.0 : 1.0;
    const double sc = (((col % d.nx) + (col / d.nx)) & 1) ? -1.0 : 1.0;
    conn += sr * sc * G[(size_t)col * n + r] * G[(size_t)r * n + col];
  }
  sm_m = block_sum(sm_m, sm.red);
  sm_m2 = block_sum(sm_m2, sm.red);
  sm_sm = block_sum(sm_sm, sm.red);
  sm_g = block_sum(sm_g, sm.red);
  conn = block_sum(conn, sm.red);
  if (threadIdx.x == 0) {
    double* acc = d.acc + (size_t)c * kAccSlots;
    acc[ACC_DENSITY] += 2.0 * sm_m / n;
    acc[ACC_DOCC] += sm_m2 / n;
    acc[ACC_SCDW] += (4.0 * sm_sm * sm_sm + 2.0 * sm_g - 2.0 * conn) / n;
    acc[ACC_COUNT] += 1.0;
  }
}

// Flush of the delayed updates: G += A B^T (n x n, rank kk; A, B [kk][n]) as a register-tiled
// contraction, 4 x 4 entries of G per thread (8 loads per 16 FMAs instead of 2 per FMA); every
// entry still accumulates its kk products in order m = 0 .. kk-1 onto G, so the result does not
// depend on the tiling.
__device__ inline void flush_delayed(double* G, const double* A, const double* B, int n, int kk) {
  const int tiles = n >> 2;  // n is a multiple of 4
  for (int t = threadIdx.x; t < tiles * tiles; t += HQ_THREADS) {
    const int r0 = (t % tiles) * 4, c0 = (t / tiles) * 4;
    double acc[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int a = 0; a < 4; ++a) acc[a][b] = G[(size_t)(c0 + b) * n + r0 + a];
    for (int m = 0; m < kk; ++m) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = A[m * n + r0 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = B[m * n + c0 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int a = 0; a < 4; ++a) G[(size_t)(c0 + b) * n + r0 + a] = acc[a][b];
  }
}

template <int LMAX>
__device__ void local_chunk_body(const Dev& d, int c, int s0, int s1, int measure, double* smraw) {
  if (!d.active[c]) return;
  const int n = d.n, L = d.L, k = d.k;
  const Smem sm = carve<LMAX>(d, smraw);
  load_kinetic(d, sm);
  double* X = d.X + (size_t)c * L * n;
  double* G = d.G + (size_t)c * n * n;
  double* A = d.Adl + (size_t)c * k * n;
  double* B = d.Bdl + (size_t)c * k * n;
  const uint32_t* id = d.cid + 4 * (size_t)c;
  const uint32_t key0 = id[0], key1 = id[1], chain = id[2], sweep = id[3];
  long long n_acc = 0;

  for (int s = s0; s < s1; ++s) {
    HQ_TIC(pp);
    // Every proposal of this slice depends only on its own site's field and on the
    // neighbouring slices, so the random numbers, dX, delta = exp(-dtau g dX) - 1 and
    // exp(-dtau dS_ph) are prepared in parallel; only the ratio needs the running G.
    for (int i = threadIdx.x; i < n; i += HQ_THREADS) {
      double u1, u2;
      proposal_uniforms(key0, key1, (uint32_t)(s * n + i), sweep, chain, 0u, u1, u2);
      const double dx = d.dx_local * (2.0 * u1 - 1.0);
      const double xo = X[(size_t)s * n + i];
      const double xnew = xo + dx;
      const double xp = X[(size_t)((s + 1) % L) * n + i];
      const double xm = X[(size_t)((s - 1 + L) % L) * n + i];
      const double kin = (xp - xnew) * (xp - xnew) + (xnew - xm) * (xnew - xm) - (xp - xo) * (xp - xo) -
                         (xo - xm) * (xo - xm);
      const double pot = xnew * xnew - xo * xo;
      const double dS = d.mass / (2.0 * d.dtau) * kin + 0.5 * d.dtau * d.mass * (d.omega * d.omega) * pot;
      sm.u2[i] = u2;
      sm.xn[i] = xnew;
      sm.dlt[i] = exp(-d.dtau * d.g * dx) - 1.0;
      sm.es[i] = exp(-dS);
      sm.dcorr[i] = 0.0;
    }
    __syncthreads();
    HQ_TOC(pp, SEC_PROP_PREP);
    HQ_TIC(seq);
    int kk = 0;
    // Thread 0 runs the decisions in site order; a rejected proposal changes nothing, so it
    // walks on to the next accepted site before the CTA meets (one barrier per accepted move
    // instead of one per proposal).  sm.sint[2 + slot] = the accepted site, n when none is left.
    for (int i0 = 0, it = 0; i0 < n; ++it) {
      const int slot = it & 1;
      if (threadIdx.x == 0) {
        int next = n;
        for (int i = i0; i < n; ++i) {
          // ratio of one spin: R1 = 1 + delta (1 - G_ii), G_ii including pending updates
          const double gii = G[(size_t)i * n + i] + sm.dcorr[i];
          const double delta = sm.dlt[i];
          const double R1 = 1.0 + delta * (1.0 - gii);
          const double prob = R1 * R1 * sm.es[i];
          if (!isfinite(R1)) d.status[c] = HQ_ENAN;
          if (sm.u2[i] < prob) {
            X[(size_t)s * n + i] = sm.xn[i];
            ++n_acc;
            sm.scal[slot] = delta / R1;
            next = i;
            break;
          }
        }
        sm.sint[2 + slot] = next;
      }
      __syncthreads();
      const int i = sm.sint[2 + slot];
      i0 = i + 1;
      if (i < n) {
        // G' = Gc + a b^T with a = (delta/R1)(Gc[:, i] - e_i), b = Gc[i, :],
        // Gc = G + sum_m A[:, m] B[:, m]^T (updates not yet flushed).
        const double f = sm.scal[slot];
        // entry r of both new vectors in one thread, so the diagonal correction needs no
        // barrier of its own
        for (int r = threadIdx.x; r < n; r += HQ_THREADS) {
          double va = G[(size_t)i * n + r], vb = G[(size_t)r * n + i];
          for (int m = 0; m < kk; ++m) {
            va = fma(A[m * n + r], B[m * n + i], va);
            vb = fma(A[m * n + i], B[m * n + r], vb);
          }
          if (r == i) va -= 1.0;
          const double a = f * va;
          A[kk * n + r] = a;
          B[kk * n + r] = vb;
          sm.dcorr[r] = fma(a, vb, sm.dcorr[r]);
        }
        ++kk;
        if (kk == k) {
          __syncthreads();
          HQ_TIC(fl);
          flush_delayed(G, A, B, n, kk);
          HQ_TOC(fl, SEC_FLUSH);
          __syncthreads();
          for (int r = threadIdx.x; r < n; r += HQ_THREADS) sm.dcorr[r] = 0.0;
          kk = 0;
        }
        __syncthreads();
      }
    }
    if (kk > 0) {
      HQ_TIC(fl);
      flush_delayed(G, A, B, n, kk);
      HQ_TOC(fl, SEC_FLUSH);
    }
    HQ_TOC(seq, SEC_PROP_SEQ);
    HQ_TIC(wr);
    // wrap: G_l = exp(-dtau K) D_l G_{l-1} D_l^-1 exp(dtau K), D_l = exp(-dtau V_l)
    // (the proposal buffer u2 is free once the slice's moves are done: it takes 1 / D_l)
    for (int r = threadIdx.x; r < n; r += HQ_THREADS) {
      const double e = exp(-d.dtau * (d.g * X[(size_t)s * n + r] - d.mu));
      sm.dl[r] = e;
      sm.u2[r] = 1.0 / e;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
      const int r = idx % n, col = idx / n;
      G[(size_t)col * n + r] = (sm.dl[r] * G[(size_t)col * n + r]) * sm.u2[col];
    }
    __syncthreads();
    kin_rows<LMAX, KIN_PLAIN>(G, n, n, sm.ex, sm.ey, d.nx, d.ny);
    kin_cols<LMAX>(G, n, n, sm.exi, sm.eyi, d.nx, d.ny);
    HQ_TOC(wr, SEC_WRAP);
  }
  if (threadIdx.x == 0) {
    long long* cnt = d.counters + (size_t)c * kCounters;
    cnt[0] += (long long)(s1 - s0) * n;
    cnt[1] += n_acc;
  }

  // ---- restabilisation at l = s1: right factors B_{s1}..B_1 = UR DR TR
  double* UR = d.UR + (size_t)c * n * n;
  double* TR = d.TR + (size_t)c * n * n;
  double* DR = d.DR + (size_t)c * n;
  double* P = chain_work(d, c, WK_P);
  double* T2 = chain_work(d, c, WK_T2);
  double* Gf = chain_work(d, c, WK_U);
  HQ_TIC(rp);
  const bool first = (s0 == 0);
  if (first) set_identity(P, n, n);
  else copy_scale_cols(P, UR, n, n, DR);
  __syncthreads();
  for (int s = s0; s < s1; ++s) {
    for (int r = threadIdx.x; r < n; r += HQ_THREADS) sm.dl[r] = exp(-d.dtau * (d.g * X[(size_t)s * n + r] - d.mu));
    __syncthreads();
    // B_s P = exp(-dtau K) exp(-dtau V_s) P
    kin_rows<LMAX, KIN_SCALE_BEFORE>(P, n, n, sm.ex, sm.ey, d.nx, d.ny, sm.dl);
  }
  HQ_TOC(rp, SEC_RESTAB_PROD);
  HQ_TIC(rq);
  double* Q = chain_work(d, c, WK_M1);
  const QrScratch qs{sm.tau, sm.vs, sm.rinv, sm.perm, sm.sint, sm.wv, sm.ws};
  prepivot<qr_group<LMAX>()>(P, Q, n, n, qs, sm.norm2);
  qr_factor<LMAX>(Q, n, n, qs);
  qr_form_q<LMAX>(Q, n, n, UR, qs);
  t_update(Q, n, n, qs, DR, first ? nullptr : TR, T2, P);
  copy_mat(TR, T2, n, n);
  __syncthreads();
  HQ_TOC(rq, SEC_RESTAB_QR);
  HQ_TIC(rg);
  const double ld = green_two_sided(d, c, sm, s1, Gf);
  double err = 0.0, bad = 0.0;
  for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
    const double gf = Gf[idx];
    if (!isfinite(gf)) bad = 1.0;
    err = fmax(err, fabs(G[idx] - gf));
  }
  err = block_max(err, sm.red);
  bad = block_max(bad, sm.red);
  copy_mat(G, Gf, n, n);
  if (threadIdx.x == 0) {
    double* acc = d.acc + (size_t)c * kAccSlots;
    acc[ACC_WRAP] = fmax(acc[ACC_WRAP], err);
    if (s1 == L) d.logdet[c] = ld;
    flag_nonfinite(d, c, ld);
    if (bad != 0.0) d.status[c] = HQ_ENAN;
  }
  __syncthreads();
  HQ_TOC(rg, SEC_RESTAB_GREEN);
  HQ_TIC(ms);
  if (measure) measure_green(d, c, sm, G);
  HQ_TOC(ms, SEC_MEASURE);
}


// The local phase of a sweep as one persistent launch, like the block-move phase: task
// t = q * C + chain is chunk q (slices [q n_wrap, min((q + 1) n_wrap, L))) of that chain;
// workers take tasks from an atomic counter and a task waits (bounded) until its chain
// finished chunk q - 1, so an SM that runs one chain alone takes more chunks than an SM
// shared by two.  sched = [counter, abort, ..., progress[C] at kSchedHeader], zeroed first.
template <int LMAX>
__global__ void __launch_bounds__(HQ_THREADS) local_phase_kernel(Dev d, int measure) {
  extern __shared__ __align__(16) double smraw[];
  __shared__ int s_task;
  const int C = d.n_chains, Q = (d.L + d.n_wrap - 1) / d.n_wrap, ntask = Q * C;
  int* counter = d.sched;
  volatile int* abort_flag = d.sched + 1;
  volatile int* progress = d.sched + kSchedHeader;
  for (;;) {
    if (threadIdx.x == 0) {
      int t = -1;
      if (*abort_flag == 0) {
        t = atomicAdd(counter, 1);
        if (t < ntask && !bounded_wait_geq(&progress[t % C], t / C, abort_flag, kWaitLimitNs)) {
          if (atomicExch((int*)abort_flag, 1) == 0)
            for (int q = 0; q < C; ++q) d.status[q] = HQ_ETIMEOUT;
          t = -1;
        }
      }
      s_task = t;
    }
    __syncthreads();
    const int t = s_task;
    if (t < 0 || t >= ntask) break;
    __threadfence();  // acquire: the previous chunk of this chain (possibly on another SM)
    const int q = t / C, c = t % C;
    const int s0 = q * d.n_wrap, s1 = s0 + d.n_wrap < d.L ? s0 + d.n_wrap : d.L;
    local_chunk_body<LMAX>(d, c, s0, s1, measure, smraw);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // release the chunk before publishing it
      atomicExch((int*)&progress[c], q + 1);
    }
  }
}

// -------------------------------------------- block moves with chunk propagators
// For block moves the n_wrap-slice products M_q = B_lo^T .. B_{hi-1}^T (chunk q covers
// slices [q n_wrap, min((q+1) n_wrap, L))) are formed once per block-move phase.  A move
// X(i, .) += dX multiplies every exp(-dtau V_s) by (1 + delta e_i e_i^T),
// delta = exp(-dtau g dX) - 1, so with A_s = B_s^T and A'_s its shifted version
//   M'_q = A'_lo .. A'_{hi-1} = M_q + delta sum_s (A'_lo .. A'_{s-1} e_i)(e_i^T A_s .. A_{hi-1})
// (telescoping; rank <= n_wrap), and the UDV chain needs one dense GEMM per chunk instead
// of n_wrap slice applications.  The shifted M'_q go to the second buffer, which becomes
// current when the move is accepted.

__device__ inline double* chunk_mat(const Dev& d, int c, int buf, int q) {
  return d.cmat + (((size_t)c * 2 + buf) * d.n_chunks + q) * (size_t)d.n * d.n;
}

// per chain: V (n x L), R (n x L), shifted diagonal entry per slice (L)
__device__ inline double* chain_corr(const Dev& d, int c) {
  return d.corr + (size_t)c * (2 * (size_t)d.n * d.L + d.L);
}

// exp(-dtau V) of every slice and the chunk products M_q of chain c (current buffer).
template <int LMAX>
__device__ void build_chunks(const Dev& d, const Smem& sm, int c) {
  const int n = d.n, L = d.L, nw = d.n_wrap;
  const double* X = d.X + (size_t)c * L * n;
  double* ev = d.expV + (size_t)c * L * n;
  for (int idx = threadIdx.x; idx < L * n; idx += HQ_THREADS) ev[idx] = exp(-d.dtau * (d.g * X[idx] - d.mu));
  __syncthreads();
  const int cur = d.cbuf[c];
  for (int q = 0; q < d.n_chunks; ++q) {
    const int lo = q * nw, hi = min(lo + nw, L);
    double* M = chunk_mat(d, c, cur, q);
    set_identity(M, n, n);
    __syncthreads();
    for (int s = hi - 1; s >= lo; --s)
      kin_rows<LMAX, KIN_SCALE_AFTER>(M, n, n, sm.ex, sm.ey, d.nx, d.ny, ev + (size_t)s * n);
  }
}

// log|det M(X')| for X' = X + dx e_site (all slices) from the chunk propagators.
// One step of the correction-vector chains of every chunk at once.  Column s of V (or R)
// belongs to chunk q = s / n_wrap, position k = s - q n_wrap in a chunk of length m_q.
//   V step (1 <= step < n_wrap): columns with k >= m_q - step get A'_t = D'_t E, t = hi_q - 1 - step
//   R step (0 <= step < n_wrap): columns with k <= step get A_t^T = E D_t,      t = lo_q + step
// D_t = exp(-dtau V_t) from the cache ev, D'_t the same with entry `site` replaced by xs[t].
template <int LMAX, bool RCHAIN>
__device__ void corr_step(const Dev& d, const Smem& sm, double* W, int step, int site, const double* ev,
                          const double* xs) {
  const int n = d.n, L = d.L, nw = d.n_wrap, nx = d.nx, ny = d.ny;
  for (int line = threadIdx.x; line < ny * L; line += HQ_THREADS) {
    const int y = line % ny, col = line / ny;
    const int q = col / nw, k = col - q * nw, lo = q * nw, m = min(nw, L - lo);
    const bool on = (step < m) && (RCHAIN ? (k <= step) : (k >= m - step));
    if (!on) continue;
    const int t = RCHAIN ? lo + step : lo + m - 1 - step;
    double* base = W + (size_t)col * n + nx * y;
    double v[LMAX];
#pragma unroll
    for (int b = 0; b < LMAX; ++b) {
      v[b] = (b < nx) ? base[b] : 0.0;
      if (RCHAIN && b < nx) v[b] *= ev[(size_t)t * n + nx * y + b];
    }
#pragma unroll
    for (int a = 0; a < LMAX; ++a) {
      if (a < nx) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < LMAX; ++b)
          if (b < nx) acc = fma(sm.ex[a * nx + b], v[b], acc);
        base[a] = acc;
      }
    }
  }
  __syncthreads();
  for (int line = threadIdx.x; line < nx * L; line += HQ_THREADS) {
    const int x = line % nx, col = line / nx;
    const int q = col / nw, k = col - q * nw, lo = q * nw, m = min(nw, L - lo);
    const bool on = (step < m) && (RCHAIN ? (k <= step) : (k >= m - step));
    if (!on) continue;
    const int t = RCHAIN ? lo + step : lo + m - 1 - step;
    double* base = W + (size_t)col * n + x;
    double v[LMAX];
#pragma unroll
    for (int b = 0; b < LMAX; ++b) v[b] = (b < ny) ? base[b * nx] : 0.0;
#pragma unroll
    for (int a = 0; a < LMAX; ++a) {
      if (a < ny) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < LMAX; ++b)
          if (b < ny) acc = fma(sm.ey[a * ny + b], v[b], acc);
        if (!RCHAIN) {
          const int r = x + nx * a;
          acc *= (r == site) ? xs[t] : ev[(size_t)t * n + r];
        }
        base[a * nx] = acc;
      }
    }
  }
  __syncthreads();
}

template <int LMAX>
__device__ double udv_top_down_cm(const Dev& d, int c, const Smem& sm, int site, double dx) {
  const int n = d.n, L = d.L, nw = d.n_wrap;
  const double* X = d.X + (size_t)c * L * n;
  const double* ev = d.expV + (size_t)c * L * n;
  double* Vc = chain_corr(d, c);   // [L][n]: column s for slice s
  double* Rc = Vc + (size_t)n * L;
  double* xs = Rc + (size_t)n * L;
  const int cur = d.cbuf[c];
  double* P = chain_work(d, c, WK_P);
  double* U = chain_work(d, c, WK_U);
  double* Tc = chain_work(d, c, WK_T);
  double* Tn = chain_work(d, c, WK_T2);
  double* Q = chain_work(d, c, WK_M1);
  double* Y = chain_work(d, c, WK_M2);
  const QrScratch qs{sm.tau, sm.vs, sm.rinv, sm.perm, sm.sint, sm.wv, sm.ws};
  const double delta = expm1(-d.dtau * d.g * dx);
  HQ_TIC(cv);
  for (int s = threadIdx.x; s < L; s += HQ_THREADS) xs[s] = exp(-d.dtau * (d.g * (X[(size_t)s * n + site] + dx) - d.mu));
  for (int idx = threadIdx.x; idx < n * L; idx += HQ_THREADS) {
    const double e = (idx % n == site) ? 1.0 : 0.0;
    Vc[idx] = e;
    Rc[idx] = e;
  }
  __syncthreads();
  // column s of V: A'_lo .. A'_{s-1} e_site; of R: A_{hi-1}^T .. A_s^T e_site (chunk [lo, hi))
  for (int step = 1; step < nw; ++step) corr_step<LMAX, false>(d, sm, Vc, step, site, ev, xs);
  for (int step = 0; step < nw; ++step) corr_step<LMAX, true>(d, sm, Rc, step, site, ev, xs);
  // M'_q = M_q + delta sum_{s in q} V_s R_s^T for every chunk (four outputs per thread)
  const int nn4 = (n * n) >> 2;
  for (int idx = threadIdx.x; idx < d.n_chunks * nn4; idx += HQ_THREADS) {
    const int q = idx / nn4, e0 = (idx - q * nn4) * 4;
    const int lo = q * nw, m = min(nw, L - lo);
    const double* M = chunk_mat(d, c, cur, q);
    double* Mn = chunk_mat(d, c, 1 - cur, q);
    const int col = e0 / n, r0 = e0 - col * n;  // four consecutive rows of one column (n % 4 == 0)
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int k = 0; k < m; ++k) {
      const double* vk = Vc + (size_t)(lo + k) * n + r0;
      const double rk = Rc[(size_t)(lo + k) * n + col];
      a0 = fma(vk[0], rk, a0);
      a1 = fma(vk[1], rk, a1);
      a2 = fma(vk[2], rk, a2);
      a3 = fma(vk[3], rk, a3);
    }
    Mn[e0] = fma(delta, a0, M[e0]);
    Mn[e0 + 1] = fma(delta, a1, M[e0 + 1]);
    Mn[e0 + 2] = fma(delta, a2, M[e0 + 2]);
    Mn[e0 + 3] = fma(delta, a3, M[e0 + 3]);
  }
  __syncthreads();
  HQ_TOC(cv, SEC_DL);
  bool first = true;
  for (int q = d.n_chunks - 1; q >= 0; --q) {
    double* Mn = chunk_mat(d, c, 1 - cur, q);
    HQ_TIC(gm);
    if (first) {
      copy_mat(P, Mn, n, n);
    } else {
      copy_scale_cols(Y, U, n, n, sm.dv);
      __syncthreads();
      gemm_nn<false, false>(n, Mn, Y, P, n);
    }
    __syncthreads();
    HQ_TOC(gm, SEC_KIN);
    HQ_TIC(pp);
    prepivot<qr_group<LMAX>()>(P, Q, n, n, qs, sm.norm2);
    HQ_TOC(pp, SEC_PREPIVOT);
    HQ_TIC(qr);
    qr_factor<LMAX>(Q, n, n, qs);
    HQ_TOC(qr, SEC_QR);
    HQ_TIC(fq);
    qr_form_q<LMAX>(Q, n, n, U, qs);
    HQ_TOC(fq, SEC_FORMQ);
    HQ_TIC(tu);
    t_update(Q, n, n, qs, sm.dv, first ? nullptr : Tc, Tn, P);
    HQ_TOC(tu, SEC_TUPD);
    double* t = Tc; Tc = Tn; Tn = t;
    first = false;
  }
  return finish_logdet(d, c, sm, U, Tc, nullptr);
}

// Sites visited by a sweep's block moves: all N in index order, or with d.block_sites = S
// (0 < S < N) a run of S consecutive sites (index order, periodic) from j0 = floor(u N), u the
// first uniform of event N of the chain's block-move (tag 1) Philox block of this sweep -- a
// start independent of the fields, drawn afresh each sweep.
__device__ inline int block_move_count(const Dev& d) {
  return (d.block_sites > 0 && d.block_sites < d.n) ? d.block_sites : d.n;
}

__device__ inline int block_move_site(const Dev& d, int c, int k) {
  if (!(d.block_sites > 0 && d.block_sites < d.n)) return k;
  const uint32_t* id = d.cid + 4 * (size_t)c;
  double u1, u2;
  proposal_uniforms(id[0], id[1], (uint32_t)d.n, id[3], id[2], 1u, u1, u2);
  int j0 = (int)(u1 * (double)d.n);
  if (j0 > d.n - 1) j0 = d.n - 1;
  return (j0 + k) % d.n;
}

// One block move X(site, .) += dX of chain c: Philox draw, dtau dS_ph, the full stabilised
// log|det M(X')| and the Metropolis decision (all threads of the CTA).
template <int LMAX>
__device__ void block_move(const Dev& d, const Smem& sm, int c, int site) {
  const int n = d.n, L = d.L;
  double* X = d.X + (size_t)c * L * n;
  HQ_TIC(mv);
  if (threadIdx.x == 0) {
    double u1, u2;
    const uint32_t* id = d.cid + 4 * (size_t)c;
    proposal_uniforms(id[0], id[1], (uint32_t)site, id[3], id[2], 1u, u1, u2);
    sm.scal[0] = d.dx_global * (2.0 * u1 - 1.0);
    sm.scal[1] = u2;
  }
  __syncthreads();
  const double dx = sm.scal[0];
  double a = 0.0;
  for (int s = threadIdx.x; s < L; s += HQ_THREADS) {
    const double x = X[(size_t)s * n + site];
    a += (x + dx) * (x + dx) - x * x;
  }
  a = block_sum(a, sm.red);
  const double dS = 0.5 * d.dtau * d.mass * (d.omega * d.omega) * a;
  HQ_TOC(mv, SEC_MOVE);
  const double ld_new = d.use_cm ? udv_top_down_cm<LMAX>(d, c, sm, site, dx)
                                 : udv_top_down<LMAX>(d, c, sm, X, site, dx, false, nullptr);
  if (threadIdx.x == 0) {
    const double arg = 2.0 * (ld_new - d.logdet[c]) - dS;
    const double prob = exp(fmin(arg, 709.0));
    const int accept = sm.scal[1] < prob;
    long long* cnt = d.counters + (size_t)c * kCounters;
    cnt[2] += 1;
    if (accept) {
      cnt[3] += 1;
      d.logdet[c] = ld_new;
    }
    flag_nonfinite(d, c, ld_new);
    sm.sint[4] = accept;
  }
  __syncthreads();
  if (sm.sint[4]) {
    for (int s = threadIdx.x; s < L; s += HQ_THREADS) X[(size_t)s * n + site] = X[(size_t)s * n + site] + dx;
    if (d.use_cm) {
      // the shifted chunk propagators and diagonal become current
      const double* xs = chain_corr(d, c) + 2 * (size_t)n * L;
      double* ev = d.expV + (size_t)c * L * n;
      for (int s = threadIdx.x; s < L; s += HQ_THREADS) ev[(size_t)s * n + site] = xs[s];
      if (threadIdx.x == 0) d.cbuf[c] = 1 - d.cbuf[c];
    }
  }
}


// The block-move phase of a sweep as one persistent launch.  Task t = step * C + chain;
// a chain's steps are its N moves in site order, preceded (with chunk propagators) by the
// build of its propagators.  Workers take tasks from an atomic counter; a task
// waits until its chain has finished the previous site (progress flag written with a
// release fence after the move, read before the move with an acquire fence).  Faster SMs
// take more tasks, so the load balances across SMs whatever C is.  The wait is bounded:
// after kWaitLimitNs the worker raises the abort flag, marks the chain HQ_ETIMEOUT and
// every worker stops taking tasks.  sched = [counter, abort, ..., progress[C] at
// kSchedHeader], zeroed before the launch.
template <int LMAX>
__global__ void __launch_bounds__(HQ_THREADS, 2) global_phase_kernel(Dev d) {
  extern __shared__ __align__(16) double smraw[];
  __shared__ int s_task;
  const Smem sm = carve<LMAX>(d, smraw);
  load_kinetic(d, sm);
  const int C = d.n_chains, ntask = (block_move_count(d) + (d.use_cm ? 1 : 0)) * C;
  int* counter = d.sched;
  volatile int* abort_flag = d.sched + 1;
  volatile int* progress = d.sched + kSchedHeader;
  for (;;) {
    HQ_TIC(wait);
    if (threadIdx.x == 0) {
      int t = -1;
      if (*abort_flag == 0) {
        t = atomicAdd(counter, 1);
        if (t < ntask) {
          const int site = t / C, c = t % C;
          if (!bounded_wait_geq(&progress[c], site, abort_flag, kWaitLimitNs)) {
            // the phase did not complete: every chain's state is suspect
            if (atomicExch((int*)abort_flag, 1) == 0)
              for (int q = 0; q < C; ++q) d.status[q] = HQ_ETIMEOUT;
            t = -1;
          }
        }
      }
      s_task = t;
    }
    __syncthreads();
    HQ_TOC(wait, SEC_WAIT);
    const int t = s_task;
    if (t < 0 || t >= ntask) break;
    __threadfence();  // acquire: the previous step of this chain (possibly on another SM)
    const int step = t / C;
    if (d.active[t % C]) {
      if (d.use_cm) {
        if (step == 0) build_chunks<LMAX>(d, sm, t % C);
        else block_move<LMAX>(d, sm, t % C, block_move_site(d, t % C, step - 1));
      } else {
        block_move<LMAX>(d, sm, t % C, block_move_site(d, t % C, step));
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // release the move before publishing it
      atomicExch((int*)&progress[t % C], t / C + 1);
    }
  }
}

__device__ void sweep_end_body(const Dev& d, int c, int measured, double* red) {
  if (!d.active[c]) return;
  const int n = d.n, L = d.L;
  const double* X = d.X + (size_t)c * L * n;
  double s1 = 0.0, s2 = 0.0;
  for (int idx = threadIdx.x; idx < L * n; idx += HQ_THREADS) {
    const double x = X[idx];
    s1 += x;
    s2 += x * x;
  }
  s1 = block_sum(s1, red);
  s2 = block_sum(s2, red);
  if (threadIdx.x == 0) {
    double* acc = d.acc + (size_t)c * kAccSlots;
    double* tot = d.tot + (size_t)c * kTotSlots;
    const double xm = s1 / ((double)L * n), x2 = s2 / ((double)L * n);
    double vals[HQ_N_OBS];
    const bool has = measured && acc[ACC_COUNT] > 0.0;
    const double nanv = __longlong_as_double(0x7ff8000000000000LL);
    vals[HQ_OBS_DENSITY] = has ? acc[ACC_DENSITY] / acc[ACC_COUNT] : nanv;
    vals[HQ_OBS_DOUBLE_OCC] = has ? acc[ACC_DOCC] / acc[ACC_COUNT] : nanv;
    vals[HQ_OBS_SCDW] = has ? acc[ACC_SCDW] / acc[ACC_COUNT] : nanv;
    vals[HQ_OBS_X_MEAN] = xm;
    vals[HQ_OBS_X2] = x2;
    vals[HQ_OBS_WRAP_ERR] = acc[ACC_WRAP];
    const int slot = d.slen[c];
    if (slot < d.max_series) {
      for (int o = 0; o < HQ_N_OBS; ++o) d.series[((size_t)c * HQ_N_OBS + o) * d.max_series + slot] = vals[o];
      d.slen[c] = slot + 1;
    }
    d.cid[4 * (size_t)c + 3] += 1u;  // the chain's sweep (or cumulative step) counter
    if (d.wrap_tol > 0.0 && acc[ACC_WRAP] > d.wrap_tol) {
      // stabilisation back-off: the host halves n_wrap before the next sweep, or at the floor
      // reports the chain
      d.counters[(size_t)c * kCounters + 4] += 1;
      atomicOr(d.wrap_flag, 1);
      if (d.n_wrap <= d.n_wrap_min) d.status[c] = HQ_EUNSTABLE;
    }
    if (has) {
      tot[TOT_DENSITY] += vals[HQ_OBS_DENSITY];
      tot[TOT_DOCC] += vals[HQ_OBS_DOUBLE_OCC];
      tot[TOT_SCDW] += vals[HQ_OBS_SCDW];
      tot[TOT_MEASURED] += 1.0;
    }
    tot[TOT_XMEAN] += xm;
    tot[TOT_X2] += x2;
    tot[TOT_SWEEPS] += 1.0;
    tot[TOT_WRAP] = fmax(tot[TOT_WRAP], acc[ACC_WRAP]);
    for (int o = 0; o < kAccSlots; ++o) acc[o] = 0.0;
  }
}

__global__ void __launch_bounds__(HQ_THREADS) sweep_end_kernel(Dev d, int measured) {
  __shared__ double red[HQ_WARPS];
  sweep_end_body(d, blockIdx.x, measured, red);
}

// ------------------------------------------------ heterogeneous groups of engines
// Engines of different lattices, temperatures and couplings swept together by ONE persistent
// launch.  A chain's sweep is sequential (stack build, local chunks, block moves, records),
// so the unit of work is a whole chain-sweep: workers take chains from the group's table --
// sorted by estimated cost, longest first, so the long chains start at once and the short
// ones fill in around them -- and run every step of the chain.  No worker ever waits for
// another.  Kernels are instantiated for the largest lattice side of the group (the separable
// propagator's arithmetic does not depend on it) and take the largest shared-memory carve.
template <int LMAX>
__global__ void __launch_bounds__(HQ_THREADS) group_sweep_kernel(GroupDev g, int flags, int stack) {
  extern __shared__ __align__(16) double smraw[];
  __shared__ int s_task;
  __shared__ Dev sd;
  const bool do_local = flags & HQ_LOCAL, do_global = flags & HQ_GLOBAL, meas = flags & HQ_MEASURE;
  int cur = -1;
  Smem sm{};
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(g.sched, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();  // every thread has read s_task before the next iteration overwrites it
    if (t >= g.n_tasks) break;
    const uint32_t w = g.tasks[t];
    const int e = (int)(w >> 26), c = (int)(w & 0xffffu);
    if (e != cur) {
      if (threadIdx.x == 0) sd = g.devs[e];
      __syncthreads();
      sm = carve<LMAX>(sd, smraw);
      load_kinetic(sd, sm);
      cur = e;
    }
    if (!sd.active[c]) continue;
    if (stack) stack_build_body<LMAX>(sd, c, smraw);
    if (do_local)
      for (int s0 = 0; s0 < sd.L; s0 += sd.n_wrap) {
        const int s1 = s0 + sd.n_wrap < sd.L ? s0 + sd.n_wrap : sd.L;
        local_chunk_body<LMAX>(sd, c, s0, s1, meas ? 1 : 0, smraw);
      }
    if (do_global) {
      if (sd.use_cm) build_chunks<LMAX>(sd, sm, c);
      for (int k = 0, nb = block_move_count(sd); k < nb; ++k) block_move<LMAX>(sd, sm, c, block_move_site(sd, c, k));
    }
    sweep_end_body(sd, c, (meas && do_local) ? 1 : 0, sm.red);
    __syncthreads();
  }
}

// Electronic observables from G_0 of every chain (after a stack build).
template <int LMAX>
__global__ void __launch_bounds__(HQ_THREADS) measure_g0_kernel(Dev d) {
  extern __shared__ __align__(16) double smraw[];
  const Smem sm = carve<LMAX>(d, smraw);
  const int c = blockIdx.x;
  if (!d.active[c]) return;
  measure_green(d, c, sm, d.G + (size_t)c * d.n * d.n);
}

// Slot control without host memory: a copy from pageable host memory can wait for kernels
// running on other streams, so identity, activity and the per-slot reset are written by a
// kernel from its arguments.  slot < 0: every chain c gets chain word first + c (creation).
__global__ void slot_control_kernel(Dev d, int slot, uint32_t key0, uint32_t key1, uint32_t chain, uint32_t sweep,
                                    int active, int reset) {
  const int c = slot < 0 ? blockIdx.x : slot;
  const uint32_t word = slot < 0 ? chain + (uint32_t)blockIdx.x : chain;
  if (threadIdx.x == 0) {
    d.active[c] = active;
    if (reset) {
      uint32_t* id = d.cid + 4 * (size_t)c;
      id[0] = key0;
      id[1] = key1;
      id[2] = word;
      id[3] = sweep;
      d.slen[c] = 0;
      d.status[c] = 0;
      if (d.use_cm) d.cbuf[c] = 0;
    }
  }
  if (!reset) return;
  for (int o = threadIdx.x; o < kAccSlots; o += blockDim.x) d.acc[(size_t)c * kAccSlots + o] = 0.0;
  for (int o = threadIdx.x; o < kTotSlots; o += blockDim.x) d.tot[(size_t)c * kTotSlots + o] = 0.0;
  for (int o = threadIdx.x; o < kCounters; o += blockDim.x) d.counters[(size_t)c * kCounters + o] = 0;
}

__global__ void reset_acc_kernel(Dev d) {
  const int c = blockIdx.x;
  for (int o = threadIdx.x; o < kAccSlots; o += blockDim.x) d.acc[(size_t)c * kAccSlots + o] = 0.0;
}

// log W = 2 log|det M| - dtau S_ph per chain.
__global__ void __launch_bounds__(HQ_THREADS) log_weight_kernel(Dev d, double* out) {
  __shared__ double red[HQ_WARPS];
  const int c = blockIdx.x;
  const int n = d.n, L = d.L;
  const double* X = d.X + (size_t)c * L * n;
  double kin = 0.0, pot = 0.0;
  for (int idx = threadIdx.x; idx < L * n; idx += HQ_THREADS) {
    const int s = idx / n, i = idx % n;
    const double x = X[idx];
    const double xp = X[(size_t)((s + 1) % L) * n + i];
    kin += (xp - x) * (xp - x);
    pot += x * x;
  }
  kin = block_sum(kin, red);
  pot = block_sum(pot, red);
  if (threadIdx.x == 0) {
    const double act = d.mass / (2.0 * d.dtau) * kin + 0.5 * d.dtau * d.mass * (d.omega * d.omega) * pot;
    out[c] = 2.0 * d.logdet[c] - act;
  }
}

__global__ void proposals_kernel(uint32_t key0, uint32_t key1, uint32_t chain, uint32_t sweep, uint32_t tag,
                                 const uint32_t* events, int n, double* u1, double* u2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double a, b;
    proposal_uniforms(key0, key1, events[i], sweep, chain, tag, a, b);
    u1[i] = a;
    u2[i] = b;
  }
}

// ---------------------------------------------------------------- launchers

// Dynamic shared memory above the default 48 KB needs an opt-in per kernel.  The opt-in is
// set once per kernel and device, to the device maximum: engines of different shapes share
// kernel instantiations and run concurrently on their own streams, and changing the
// attribute between their launches would make a launch wait for the running ones.
cudaError_t opt_in_smem(const void* kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;
  int dev = 0, cap = 0;
  cudaError_t st = cudaGetDevice(&dev);
  if (st == cudaSuccess) st = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (st != cudaSuccess) return st;
  // the opt-in limit covers the kernel's static shared memory too
  cudaFuncAttributes fa;
  st = cudaFuncGetAttributes(&fa, kernel);
  if (st != cudaSuccess) return st;
  const int dyn_cap = cap - (int)fa.sharedSizeBytes;
  if (bytes > (size_t)dyn_cap) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& kd : done)
    if (kd.first == kernel && kd.second == dev) return cudaSuccess;
  st = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_cap);
  if (st == cudaSuccess) done.emplace_back(kernel, dev);
  return st;
}

template <typename K>
static inline void allow_smem(K kernel, size_t bytes) {
  opt_in_smem((const void*)kernel, bytes);
}

#define HQ_DISPATCH(KERNEL, d, stream, ...)                                                  \
  do {                                                                                      \
    const size_t sb = smem_bytes(d);                                                        \
    switch (lmax_of((d).nx, (d).ny)) {                                                      \
      case 2: allow_smem(KERNEL<2>, sb); KERNEL<2><<<(d).n_chains, HQ_THREADS, sb, stream>>>(__VA_ARGS__); break;   \
      case 4: allow_smem(KERNEL<4>, sb); KERNEL<4><<<(d).n_chains, HQ_THREADS, sb, stream>>>(__VA_ARGS__); break;   \
      case 8: allow_smem(KERNEL<8>, sb); KERNEL<8><<<(d).n_chains, HQ_THREADS, sb, stream>>>(__VA_ARGS__); break;   \
      default: allow_smem(KERNEL<16>, sb); KERNEL<16><<<(d).n_chains, HQ_THREADS, sb, stream>>>(__VA_ARGS__); break; \
    }                                                                                       \
  } while (0)

// ------------------------------------------------- log|det M| without allocation
// File-scope scratch for hq_logdet_noalloc: kWorkMats N x N work matrices per chain live here
// instead of in a caller arena.  Every GPU that loads the library holds it until the process
// exits.  All calls share it, so calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// exp(-sgn dtau K_ring) of a ring of m sites (K_ab = -t per displacement +-1) straight into
// shared memory: the ring is diagonal in plane waves with eigenvalues -2t cos(2 pi q/m), so
// E_ab = (1/m) sum_q cos(2 pi q (a-b)/m) exp(sgn 2 t dtau cos(2 pi q/m)).
__device__ inline void ring_propagators_smem(const Dev& d, const Smem& s) {
  const double two_pi = 6.283185307179586476925286766559;
  const int a2 = d.nx * d.nx, b2 = d.ny * d.ny;
  for (int idx = threadIdx.x; idx < 2 * a2 + 2 * b2; idx += HQ_THREADS) {
    int m, e;
    double sgn;
    if (idx < 2 * a2) { m = d.nx; e = idx % a2; sgn = idx < a2 ? 1.0 : -1.0; }
    else { m = d.ny; e = (idx - 2 * a2) % b2; sgn = idx - 2 * a2 < b2 ? 1.0 : -1.0; }
    const int a = e / m, b = e % m;
    double acc = 0.0;
    for (int q = 0; q < m; ++q)
      acc += cos(two_pi * q * (a - b) / m) * exp(sgn * 2.0 * d.t * d.dtau * cos(two_pi * q / m));
    s.ex[idx] = acc / m;  // ex, exi, ey, eyi are contiguous
  }
  __syncthreads();
}

template <int LMAX>
__global__ void __launch_bounds__(HQ_THREADS) logdet_noalloc_kernel(Dev d, double* out) {
  extern __shared__ __align__(16) double smraw[];
  const int c = blockIdx.x;
  const Smem sm = carve<LMAX>(d, smraw);
  ring_propagators_smem(d, sm);
  const double* X = d.X + (size_t)c * d.L * d.n;
  const double ld = udv_top_down<LMAX>(d, c, sm, X, -1, 0.0, false, nullptr);
  if (threadIdx.x == 0) out[c] = ld;
}

size_t noalloc_scratch_needed(int nx, int ny, int n_chains) {
  const size_t n = (size_t)nx * ny;
  return sizeof(double) * (size_t)n_chains * kWorkMats * n * n;
}

// Device address of the scratch on the current device, looked up once per device (the
// host-side name of a __device__ array is not a device address).
static cudaError_t noalloc_scratch_address(void** out) {
  static std::mutex mu;
  static void* addr[kMaxDevices] = {nullptr};
  int dev = 0;
  cudaError_t st = cudaGetDevice(&dev);
  if (st != cudaSuccess) return st;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    st = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (st != cudaSuccess) return st;
    addr[dev] = p;
  }
  *out = addr[dev];
  return cudaSuccess;
}

cudaError_t launch_logdet_noalloc(Dev d, double* out, cudaStream_t s) {
  void* base = nullptr;
  cudaError_t st = noalloc_scratch_address(&base);
  if (st != cudaSuccess) return st;
  // the kernel builds the kinetic factors in shared memory and needs no status word
  d.kin = nullptr;
  d.status = nullptr;
  d.work = (double*)base;
  HQ_DISPATCH(logdet_noalloc_kernel, d, s, d, out);
  return cudaGetLastError();
}

cudaError_t launch_stack_build(const Dev& d, cudaStream_t s) {
  HQ_DISPATCH(stack_build_kernel, d, s, d);
  return cudaGetLastError();
}

int split_point(const Dev& d) {
  const int q = (d.L + d.n_wrap - 1) / d.n_wrap;
  return q >= 2 ? (q / 2) * d.n_wrap : 0;
}

template <int LMAX>
static cudaError_t launch_split_t(const Dev& d, int m, int part, cudaStream_t s) {
  const size_t sb = smem_bytes(d);
  if (part == 0) {
    allow_smem(split_halves_kernel<LMAX>, sb);
    split_halves_kernel<LMAX><<<2 * d.n_chains, HQ_THREADS, sb, s>>>(d, m);
  } else {
    allow_smem(split_join_kernel<LMAX>, sb);
    split_join_kernel<LMAX><<<d.n_chains, HQ_THREADS, sb, s>>>(d, m);
  }
  return cudaGetLastError();
}

cudaError_t launch_split_logdet(const Dev& d, int m, int part, cudaStream_t s) {
  if (m <= 0 || m >= d.L || m % d.n_wrap != 0) return cudaErrorInvalidValue;
  switch (lmax_of(d.nx, d.ny)) {
    case 2: return launch_split_t<2>(d, m, part, s);
    case 4: return launch_split_t<4>(d, m, part, s);
    case 8: return launch_split_t<8>(d, m, part, s);
    default: return launch_split_t<16>(d, m, part, s);
  }
}


template <int LMAX>
static cudaError_t launch_local_phase_t(const Dev& d, int measure, cudaStream_t s) {
  const size_t sb = smem_bytes(d);
  allow_smem(local_phase_kernel<LMAX>, sb);
  int dev = 0, sms = 0, occ = 0;
  cudaError_t st = cudaGetDevice(&dev);
  if (st == cudaSuccess) st = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (st == cudaSuccess)
    st = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, local_phase_kernel<LMAX>, HQ_THREADS, sb);
  if (st != cudaSuccess) return st;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  // as in the block-move phase: one wave at most, at most one worker per active chain
  int workers = sms * (occ < kWorkersPerSm ? occ : kWorkersPerSm);
  if (workers > d.n_active) workers = d.n_active;
  if (workers < 1) workers = 1;
  st = cudaMemsetAsync(d.sched, 0, sizeof(int) * (kSchedHeader + d.n_chains), s);
  if (st != cudaSuccess) return st;
  local_phase_kernel<LMAX><<<workers, HQ_THREADS, sb, s>>>(d, measure);
  return cudaGetLastError();
}

cudaError_t launch_local_phase(const Dev& d, int measure, cudaStream_t s) {
  switch (lmax_of(d.nx, d.ny)) {
    case 2: return launch_local_phase_t<2>(d, measure, s);
    case 4: return launch_local_phase_t<4>(d, measure, s);
    case 8: return launch_local_phase_t<8>(d, measure, s);
    default: return launch_local_phase_t<16>(d, measure, s);
  }
}

template <int LMAX>
static cudaError_t launch_phase(const Dev& d, cudaStream_t s) {
  const size_t sb = smem_bytes(d);
  allow_smem(global_phase_kernel<LMAX>, sb);
  int dev = 0, sms = 0, occ = 0;
  cudaError_t st = cudaGetDevice(&dev);
  if (st == cudaSuccess) st = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (st == cudaSuccess)
    st = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, global_phase_kernel<LMAX>, HQ_THREADS, sb);
  if (st != cudaSuccess) return st;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  // One wave at most.  A worker only waits for a task that an earlier, running worker has
  // taken, so progress never depends on a block that is not resident (other streams may hold
  // SMs).  The steps of one chain are sequential, so at most one task per active chain runs
  // at once: more workers than active chains would only wait, holding SMs that concurrent
  // launches could use (idle slots' tasks are skipped by whichever worker takes them).
  int workers = sms * (occ < kWorkersPerSm ? occ : kWorkersPerSm);
  if (workers > d.n_active) workers = d.n_active;
  if (workers < 1) workers = 1;
  st = cudaMemsetAsync(d.sched, 0, sizeof(int) * (kSchedHeader + d.n_chains), s);
  if (st != cudaSuccess) return st;
  global_phase_kernel<LMAX><<<workers, HQ_THREADS, sb, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_global_phase(const Dev& d, cudaStream_t s) {
  switch (lmax_of(d.nx, d.ny)) {
    case 2: return launch_phase<2>(d, s);
    case 4: return launch_phase<4>(d, s);
    case 8: return launch_phase<8>(d, s);
    default: return launch_phase<16>(d, s);
  }
}

// ---- group launcher (lmax: largest lattice side class of the group; sb: largest carve).
// The caller zeroes the group's task counter first.
int lmax_class(int nx, int ny) { return lmax_of(nx, ny); }

template <int LMAX>
static cudaError_t launch_group_t(const GroupDev& g, size_t sb, int n_active, int flags, int stack, cudaStream_t s) {
  allow_smem(group_sweep_kernel<LMAX>, sb);
  int dev = 0, sms = 0, occ = 0;
  cudaError_t st = cudaGetDevice(&dev);
  if (st == cudaSuccess) st = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (st == cudaSuccess)
    st = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, group_sweep_kernel<LMAX>, HQ_THREADS, sb);
  if (st != cudaSuccess) return st;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  int workers = sms * (occ < kWorkersPerSm ? occ : kWorkersPerSm);
  if (workers > n_active) workers = n_active;
  if (workers < 1) workers = 1;
  group_sweep_kernel<LMAX><<<workers, HQ_THREADS, sb, s>>>(g, flags, stack);
  return cudaGetLastError();
}

cudaError_t launch_group_sweep(const GroupDev& g, int lmax, size_t sb, int n_active, int flags, int stack,
                               cudaStream_t s) {
  switch (lmax) {
    case 2: return launch_group_t<2>(g, sb, n_active, flags, stack, s);
    case 4: return launch_group_t<4>(g, sb, n_active, flags, stack, s);
    case 8: return launch_group_t<8>(g, sb, n_active, flags, stack, s);
    default: return launch_group_t<16>(g, sb, n_active, flags, stack, s);
  }
}

cudaError_t launch_measure_g0(const Dev& d, cudaStream_t s) {
  HQ_DISPATCH(measure_g0_kernel, d, s, d);
  return cudaGetLastError();
}

cudaError_t launch_sweep_end(const Dev& d, int measured, cudaStream_t s) {
  sweep_end_kernel<<<d.n_chains, HQ_THREADS, 0, s>>>(d, measured);
  return cudaGetLastError();
}

cudaError_t launch_slot_control(const Dev& d, int slot, uint32_t key0, uint32_t key1, uint32_t chain, uint32_t sweep,
                                int active, int reset, cudaStream_t s) {
  slot_control_kernel<<<slot < 0 ? d.n_chains : 1, 32, 0, s>>>(d, slot, key0, key1, chain, sweep, active, reset);
  return cudaGetLastError();
}

cudaError_t launch_reset_acc(const Dev& d, cudaStream_t s) {
  reset_acc_kernel<<<d.n_chains, 32, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_log_weight(const Dev& d, double* out, cudaStream_t s) {
  log_weight_kernel<<<d.n_chains, HQ_THREADS, 0, s>>>(d, out);
  return cudaGetLastError();
}

cudaError_t launch_proposals(uint32_t key0, uint32_t key1, uint32_t chain, uint32_t sweep, uint32_t tag,
                             const uint32_t* events, int n, double* u1, double* u2, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  proposals_kernel<<<(n + 255) / 256, 256, 0, s>>>(key0, key1, chain, sweep, tag, events, n, u1, u2);
  return cudaGetLastError();
}

// ------------------------------------------------------------ FP64 pipe probe
#define HQ_PROBE_ITERS 4096
// Wait probe: the bounded wait of the block-move phase on a flag that nothing sets, so the
// wait runs out after limit_ns and the kernel reports HQ_ETIMEOUT instead of hanging.
static __device__ int g_wait_probe_flag;   // nothing sets it
static __device__ int g_wait_probe_abort;  // nothing sets it
static __device__ int g_wait_probe_status;

__global__ void wait_probe_kernel(unsigned long long limit_ns) {
  if (threadIdx.x == 0)
    g_wait_probe_status =
        bounded_wait_geq(&g_wait_probe_flag, 1, &g_wait_probe_abort, limit_ns) ? HQ_OK : HQ_ETIMEOUT;
}

cudaError_t wait_probe(double limit_s, cudaStream_t s, int* status) {
  const unsigned long long ns = (unsigned long long)(limit_s * 1e9);
  wait_probe_kernel<<<1, 32, 0, s>>>(ns);
  cudaError_t st = cudaGetLastError();
  if (st == cudaSuccess) st = cudaMemcpyFromSymbolAsync(status, g_wait_probe_status, sizeof(int), 0,
                                                        cudaMemcpyDeviceToHost, s);
  if (st == cudaSuccess) st = cudaStreamSynchronize(s);
  return st;
}

__global__ void fp64_probe_kernel(double* out, double b, double c) {
  double a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int it = 0; it < HQ_PROBE_ITERS; ++it) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
    a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

__global__ void dmma_probe_kernel(double* out, double av, double bv) {
  double c[4][2];
  for (int j = 0; j < 4; ++j) {
    c[j][0] = threadIdx.x;
    c[j][1] = j;
  }
  const double a = av + threadIdx.x * 1e-3, b = bv;
  for (int it = 0; it < HQ_PROBE_ITERS / 2; ++it) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(c[j][0]), "+d"(c[j][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
  for (int j = 0; j < 4; ++j) s += c[j][0] + c[j][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

double fp64_probe_tflops(int kind, int reps, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1.0;
  const int grid = sms * 4, block = 256;
  double* out = nullptr;
  if (cudaMallocAsync(&out, sizeof(double) * grid * block, s) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&]() {
    if (kind == 1) dmma_probe_kernel<<<grid, block, 0, s>>>(out, 0.5, 0.25);
    else fp64_probe_kernel<<<grid, block, 0, s>>>(out, 0.999, 1e-3);
  };
  launch();
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  cudaStreamSynchronize(s);
  if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return -1.0;
  // DFMA: 8 FMAs per thread per iteration; DMMA: 4 m8n8k4 MMAs (512 flops) per warp per
  // iteration over HQ_PROBE_ITERS / 2 iterations.
  const double flops = kind == 1 ? (double)reps * grid * (block / 32) * (HQ_PROBE_ITERS / 2) * 4 * 512.0
                                 : (double)reps * grid * block * HQ_PROBE_ITERS * 8 * 2;
  return flops / (ms * 1e-3) / 1e12;
}

}  // namespace hq
