// Device building blocks of the Holstein DQMC engine (FP64, one CTA per Markov chain).
//
// Every routine is called by all HQ_THREADS threads of a CTA and works on column-major
// n x n matrices (element (r, c) at c*ld + r) that live in global memory (L1/L2 cached).
// The FP64 pipe is the bound on GB300 (about 1/74 of the FP32 rate), so the routines
// aim at keeping DFMAs in flight and at cutting FP64 work (separable kinetic propagator),
// not at staging: operand traffic per DFMA is far below L1 bandwidth.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define HQ_THREADS 256
#define HQ_WARPS (HQ_THREADS / 32)
#define HQ_FULL 0xffffffffu

namespace hq {

// Optional per-section cycle counters (compile with -DHQ_SECTION_TIMING): thread 0 of each
// CTA adds the clock64() span of a code section to a device array that
// hq_get_section_cycles() returns.  Off by default; no effect on results.
enum {
  SEC_DL = 0, SEC_KIN, SEC_PREPIVOT, SEC_QR, SEC_FORMQ, SEC_TUPD, SEC_LOGDET, SEC_MOVE, SEC_WAIT,
  SEC_PROP_PREP, SEC_PROP_SEQ, SEC_WRAP, SEC_RESTAB_PROD, SEC_RESTAB_QR, SEC_RESTAB_GREEN, SEC_MEASURE,
  SEC_FLUSH, SEC_COUNT
};
#ifdef HQ_SECTION_TIMING
static __device__ unsigned long long g_section_cycles[SEC_COUNT];  // per translation unit
#define HQ_TIC(name) const long long hq_tic_##name = clock64()
#define HQ_TOC(name, slot)                                                              \
  do {                                                                                \
    if (threadIdx.x == 0) atomicAdd(&g_section_cycles[slot], (unsigned long long)(clock64() - hq_tic_##name)); \
  } while (0)
#else
#define HQ_TIC(name) (void)0
#define HQ_TOC(name, slot) (void)0
#endif

struct Lattice {
  int nx, ny, n;
  const double* ex;   // exp(-dtau K_x), nx x nx row-major (shared memory)
  const double* exi;  // exp(+dtau K_x)
  const double* ey;   // exp(-dtau K_y), ny x ny
  const double* eyi;  // exp(+dtau K_y)
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(HQ_FULL, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(HQ_FULL, v, o));
  return v;
}

// Sum over the CTA in a fixed order (deterministic); every thread gets the result.
// red: HQ_WARPS doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < HQ_WARPS; ++w) s += red[w];
  return s;
}

__device__ __forceinline__ double block_max(double v, double* red) {
  v = warp_max(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = red[0];
#pragma unroll
  for (int w = 1; w < HQ_WARPS; ++w) s = fmax(s, red[w]);
  return s;
}

// ---------------------------------------------------------------- bounded waits
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Spin (with growing sleeps) until *v >= target.  Gives up -- returns false -- when *abort_flag
// becomes non-zero or after limit_ns of global time, so a wait never hangs the GPU.
__device__ inline bool bounded_wait_geq(volatile int* v, int target, volatile int* abort_flag,
                                        unsigned long long limit_ns) {
  if (*v >= target) return true;
  const unsigned long long t0 = global_timer_ns();
  unsigned ns = 32;
  while (*v < target) {
    if (*abort_flag != 0 || global_timer_ns() - t0 > limit_ns) return false;
    __nanosleep(ns);
    if (ns < 2048) ns *= 2;
  }
  return true;
}

// ---------------------------------------------------------------- bfloat16
__device__ __forceinline__ float bf16_to_float(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// round to nearest even (finite inputs)
__device__ __forceinline__ uint16_t float_to_bf16(float f) {
  const uint32_t u = __float_as_uint(f);
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of two 32x32->64 multiplies with the
// round constants, key bumped by the Weyl constants between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
}

// 53-bit uniform in [0,1) from the 27 high bits of a and the 26 high bits of b.
__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ void proposal_uniforms(uint32_t key0, uint32_t key1, uint32_t event,
                                                  uint32_t sweep, uint32_t chain, uint32_t tag,
                                                  double& u1, double& u2) {
  uint32_t c0 = event, c1 = sweep, c2 = chain, c3 = tag;
  philox4x32_10(c0, c1, c2, c3, key0, key1);
  u1 = uniform53(c0, c1);
  u2 = uniform53(c2, c3);
}

// ------------------------------------------------------- separable kinetic propagator
// exp(-dtau K) = E_x (x) E_y exactly, because K = K_x (x) 1 + 1 (x) K_y and the two terms
// commute on the periodic lattice.  Applying it to an n x n matrix costs 2 n^2 (nx + ny)
// flops instead of 2 n^3 for the dense product.

enum { KIN_PLAIN = 0, KIN_SCALE_BEFORE = 1, KIN_SCALE_AFTER = 2 };

// P <- (E_x (x) E_y) P (acts on the row = site index of every column).  With
// KIN_SCALE_BEFORE the rows are first multiplied by d (P <- E diag(d) P, a slice matrix
// B = exp(-dtau K) exp(-dtau V)); with KIN_SCALE_AFTER afterwards (P <- diag(d) E P = B^T P).
template <int LMAX, int MODE>
__device__ inline void kin_rows(double* P, int ld, int ncols, const double* ex, const double* ey, int nx, int ny,
                         const double* d = nullptr) {
  for (int line = threadIdx.x; line < ny * ncols; line += HQ_THREADS) {
    const int y = line % ny, j = line / ny;
    double* base = P + (size_t)j * ld + nx * y;
    double v[LMAX];
#pragma unroll
    for (int b = 0; b < LMAX; ++b) {
      v[b] = (b < nx) ? base[b] : 0.0;
      if (MODE == KIN_SCALE_BEFORE && b < nx) v[b] *= d[nx * y + b];
    }
#pragma unroll
    for (int a = 0; a < LMAX; ++a) {
      if (a < nx) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < LMAX; ++b)
          if (b < nx) acc = fma(ex[a * nx + b], v[b], acc);
        base[a] = acc;
      }
    }
  }
  __syncthreads();
  for (int line = threadIdx.x; line < nx * ncols; line += HQ_THREADS) {
    const int x = line % nx, j = line / nx;
    double* base = P + (size_t)j * ld + x;
    double v[LMAX];
#pragma unroll
    for (int b = 0; b < LMAX; ++b) v[b] = (b < ny) ? base[b * nx] : 0.0;
#pragma unroll
    for (int a = 0; a < LMAX; ++a) {
      if (a < ny) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < LMAX; ++b)
          if (b < ny) acc = fma(ey[a * ny + b], v[b], acc);
        if (MODE == KIN_SCALE_AFTER) acc *= d[x + nx * a];
        base[a * nx] = acc;
      }
    }
  }
  __syncthreads();
}

// P <- P (F_x (x) F_y)  (acts on the column index of every row); F given row-major.
template <int LMAX>
__device__ inline void kin_cols(double* P, int ld, int nrows, const double* fx, const double* fy, int nx, int ny) {
  for (int line = threadIdx.x; line < nrows * ny; line += HQ_THREADS) {
    const int r = line % nrows, y = line / nrows;
    double* base = P + (size_t)(nx * y) * ld + r;
    double v[LMAX];
#pragma unroll
    for (int b = 0; b < LMAX; ++b) v[b] = (b < nx) ? base[(size_t)b * ld] : 0.0;
#pragma unroll
    for (int a = 0; a < LMAX; ++a) {
      if (a < nx) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < LMAX; ++b)
          if (b < nx) acc = fma(v[b], fx[b * nx + a], acc);
        base[(size_t)a * ld] = acc;
      }
    }
  }
  __syncthreads();
  for (int line = threadIdx.x; line < nrows * nx; line += HQ_THREADS) {
    const int r = line % nrows, x = line / nrows;
    double* base = P + (size_t)x * ld + r;
    const size_t step = (size_t)nx * ld;
    double v[LMAX];
#pragma unroll
    for (int b = 0; b < LMAX; ++b) v[b] = (b < ny) ? base[b * step] : 0.0;
#pragma unroll
    for (int a = 0; a < LMAX; ++a) {
      if (a < ny) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < LMAX; ++b)
          if (b < ny) acc = fma(v[b], fy[b * ny + a], acc);
        base[a * step] = acc;
      }
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------- small helpers

__device__ __forceinline__ void set_identity(double* A, int ld, int n) {
  for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
    const int r = idx % n, c = idx / n;
    A[(size_t)c * ld + r] = (r == c) ? 1.0 : 0.0;
  }
}

// A <- diag(d) A  (row scaling)
__device__ __forceinline__ void scale_rows(double* A, int ld, int n, const double* d) {
  for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
    const int r = idx % n, c = idx / n;
    A[(size_t)c * ld + r] *= d[r];
  }
}

// B <- A diag(d)  (column scaling into another buffer)
__device__ __forceinline__ void copy_scale_cols(double* B, const double* A, int ld, int n, const double* d) {
  for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
    const int r = idx % n, c = idx / n;
    B[(size_t)c * ld + r] = A[(size_t)c * ld + r] * d[c];
  }
}

__device__ __forceinline__ void copy_mat(double* B, const double* A, int ld, int n) {
  for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
    const int r = idx % n, c = idx / n;
    B[(size_t)c * ld + r] = A[(size_t)c * ld + r];
  }
}

// ------------------------------------------- Householder QR with column pre-pivoting
// Column-pivoted QR in the form used for DQMC stabilisation by Bauer (SciPost Phys. Core 2,
// 011 (2020)): the columns are ordered once by decreasing Euclidean norm, then factored by
// unpivoted Householder QR.  The product being factored is column-graded (B..B U D), so the
// one-time ordering gives the graded R that the UDV decomposition needs, without per-step
// pivot searches and norm downdates.
//
constexpr int kQb = 16;         // panel width of the blocked QR and Q formation
constexpr int kQbLd = kQb + 2;  // row stride (doubles) of a panel's copy in shared memory: rows
                                // stay 16-byte aligned and consecutive rows start 4 banks apart

// Column work is spread over groups of kGroup lanes (qr_group below: 4 or 8 lanes, 64 or 32
// groups per CTA): each group reduces a column's dot product with log2(kGroup) shuffles, and
// every warp runs the same number of passes so the shuffles always see all 32 lanes.
struct QrScratch {
  double* tau;   // [n] reflector scalars
  double* vs;    // [2n] Householder vectors (current and next)
  double* rinv;  // [n] 1 / D
  int* perm;     // [n] perm[j] = original column placed at position j
  int* sint;     // >= 1
  double* wv;    // [n][kQbLd] panel of reflector vectors (blocked variants only)
  double* ws;    // [kQb][kQb] strict upper part of V^T V (blocked variants only)
};

// Lanes per column in the QR and Q-formation column updates (template parameter G).  Fewer lanes
// per column means fewer shuffle-and-add steps (FP64 instructions that do no algorithmic work)
// per column and longer FMA runs per lane, which pays for small matrices held in L1 (N <= 64);
// at N = 256 (512 KB per matrix, streamed through L2) 8 lanes per column, 64-byte column
// segments per load, are faster.  qr_group<LMAX>() picks it per lattice class.
template <int LMAX>
__host__ __device__ constexpr int qr_group() { return LMAX <= 8 ? 4 : 8; }

template <int G>
__device__ __forceinline__ double group_sum(double v) {
  static_assert(G == 2 || G == 4 || G == 8, "QR group size");
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(HQ_FULL, v, o);
  return v;
}

// Q <- columns of P ordered by decreasing norm (stable: ties keep index order); perm
// records the order.  Norms are compared through their IEEE bit patterns, which order
// non-negative doubles exactly like their values.  `norm2` is n doubles of scratch.
template <int kGroup>
__device__ inline void prepivot(const double* P, double* Q, int ld, int n, const QrScratch& s, double* norm2) {
  constexpr int kGroups = HQ_THREADS / kGroup;
  const int g = threadIdx.x / kGroup, sub = threadIdx.x % kGroup;
  for (int base = 0; base < n; base += kGroups) {
    const int c = base + g;
    double a = 0.0;
    if (c < n) {
      const double* col = P + (size_t)c * ld;
      for (int r = sub; r < n; r += kGroup) a = fma(col[r], col[r], a);
    }
    a = group_sum<kGroup>(a);
    if (c < n && sub == 0) norm2[c] = a;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += HQ_THREADS) {
    const long long mine = __double_as_longlong(norm2[c]);
    int rank = 0;
    for (int o = 0; o < n; ++o) {
      const long long other = __double_as_longlong(norm2[o]);
      rank += (other > mine) || (other == mine && o < c);
    }
    s.perm[rank] = c;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
    const int r = idx % n, j = idx / n;
    Q[(size_t)j * ld + r] = P[(size_t)s.perm[j] * ld + r];
  }
  __syncthreads();
}

// Householder vector for column j of P (warp 0 only): v has a unit leading entry, its
// tail overwrites P(j+1:, j), P(j, j) <- beta, tau[j] set (LAPACK xLARFG convention).
__device__ __forceinline__ void house_gen(double* P, int ld, int n, int j, double* vs, double* tau) {
  const int lane = threadIdx.x & 31;
  double* cj = P + (size_t)j * ld;
  double a = 0.0;
  for (int r = j + 1 + lane; r < n; r += 32) a = fma(cj[r], cj[r], a);
  a = warp_sum(a);
  const double alpha = cj[j];
  double tj = 0.0, beta = alpha, scal = 0.0;
  if (a != 0.0) {
    // beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta = 1 + |alpha| / ||x||,
    // v = x / (alpha - beta) below the unit leading entry
    const double s2 = fma(alpha, alpha, a);
    const double rs = rsqrt(s2);
    const double nrm = s2 * rs;
    beta = (alpha >= 0.0) ? -nrm : nrm;
    tj = fma(fabs(alpha), rs, 1.0);
    scal = 1.0 / (alpha - beta);
  }
  for (int r = j + 1 + lane; r < n; r += 32) {
    const double v = cj[r] * scal;
    cj[r] = v;
    vs[r] = v;
  }
  __syncwarp();
  if (lane == 0) {
    cj[j] = beta;
    vs[j] = 1.0;
    tau[j] = tj;
  }
  __syncwarp();
}

// In place unpivoted Householder QR: R in the upper triangle, reflector vectors (unit
// leading entry implied) below it, tau[j] the reflector scalars (LAPACK xGEQR2 result).
// One barrier per column with look-ahead: during step j, warp 0 applies reflector j to
// column j+1 and builds reflector j+1 while warps 1.. apply reflector j to columns j+2..
// (two vector buffers in `vs`, 2n doubles).
template <int kGroup>
__device__ inline void qr_householder(double* P, int ld, int n, const QrScratch& s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = (tid - 32) / kGroup, sub = tid % kGroup;  // groups of warps 1..
  constexpr int kTailGroups = (HQ_THREADS - 32) / kGroup;
  if (warp == 0) house_gen(P, ld, n, 0, s.vs, s.tau);
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const double* vc = s.vs + (j & 1) * n;
    double* vn = s.vs + ((j + 1) & 1) * n;
    const double tj = s.tau[j];
    if (warp == 0) {
      if (j + 1 < n) {
        double* cc = P + (size_t)(j + 1) * ld;
        if (tj != 0.0) {
          double w = 0.0;
          for (int r = j + lane; r < n; r += 32) w = fma(vc[r], cc[r], w);
          w = warp_sum(w) * tj;
          for (int r = j + lane; r < n; r += 32) cc[r] = fma(-w, vc[r], cc[r]);
          __syncwarp();
        }
        house_gen(P, ld, n, j + 1, vn, s.tau);
      }
    } else if (tj != 0.0) {
      for (int base = j + 2; base < n; base += kTailGroups) {
        const int c = base + g;
        double* cc = P + (size_t)c * ld;
        double w = 0.0;
        if (c < n)
          for (int r = j + sub; r < n; r += kGroup) w = fma(vc[r], cc[r], w);
        w = group_sum<kGroup>(w) * tj;
        if (c < n)
          for (int r = j + sub; r < n; r += kGroup) cc[r] = fma(-w, vc[r], cc[r]);
      }
    }
    __syncthreads();
  }
}

// U <- Q = H_0 H_1 ... H_{n-1} (explicit), from the reflectors stored in P and tau.
// One barrier per reflector: the next reflector's vector is staged into the other half of
// `vs` while the current one is applied.  (A compact-WY blocked variant was measured slower
// here: its serial T-factor build per block outweighs the barriers it saves.)
template <int kGroup>
__device__ inline void form_q(const double* P, int ld, int n, double* U, const QrScratch& s) {
  constexpr int kGroups = HQ_THREADS / kGroup;
  const int g = threadIdx.x / kGroup, sub = threadIdx.x % kGroup;
  set_identity(U, ld, n);
  const int jl = n - 1;
  for (int r = jl + threadIdx.x; r < n; r += HQ_THREADS) s.vs[(jl & 1) * n + r] = 1.0;
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    const double* vc = s.vs + (j & 1) * n;
    if (j > 0) {
      double* vn = s.vs + ((j - 1) & 1) * n;
      for (int r = j - 1 + threadIdx.x; r < n; r += HQ_THREADS) vn[r] = (r == j - 1) ? 1.0 : P[(size_t)(j - 1) * ld + r];
    }
    const double tj = s.tau[j];
    if (tj != 0.0) {
      for (int base = j; base < n; base += kGroups) {
        const int c = base + g;
        double* uc = U + (size_t)c * ld;
        double w = 0.0;
        if (c < n)
          for (int r = j + sub; r < n; r += kGroup) w = fma(vc[r], uc[r], w);
        w = group_sum<kGroup>(w) * tj;
        if (c < n)
          for (int r = j + sub; r < n; r += kGroup) uc[r] = fma(-w, vc[r], uc[r]);
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------ blocked QR and Q formation (16-wide class)
// At N up to 256 a column-by-column QR or Q formation sweeps a matrix of up to 512 KB once per
// column, and those sweeps run out of L1 and L2.  The blocked variants take the columns in panels
// of kQb.  A panel is factored column by column (qr_panel: the look-ahead scheme of
// qr_householder restricted to the panel), and its kQb reflectors then reach the rest of the
// matrix at once in the compact WY form H_j0 ... H_j1-1 = I - V T V^T (Schreiber and Van Loan,
// SIAM J. Sci. Stat. Comput. 10 (1989)).  T is never formed.  Its inverse is diag(1/tau) + S,
// with S the strict upper part of V^T V (the "UT transform": Joffrain, Low, Quintana-Orti, van
// de Geijn and Van Zee, ACM TOMS 32 (2006)), so each column's small triangular product becomes
// a substitution without divisions.  The factorisation is the unblocked one up to rounding:
// R above the diagonal, the unit-lower reflector vectors below it, and tau.  So the T update
// and every other reader of the QR see the same layout.

// Smallest lattice class (largest side rounded up to 2, 4, 8, 16) that takes the blocked
// variants; a build may lower it (-DHQ_QR_BLOCKED_MIN=8) to compare the two forms.
#ifndef HQ_QR_BLOCKED_MIN
#define HQ_QR_BLOCKED_MIN 16
#endif
__host__ __device__ constexpr bool qr_blocked_class(int lmax) { return lmax >= HQ_QR_BLOCKED_MIN; }

// Panel factorisation of columns j0 .. j1 - 1 (rows j .. n - 1 for column j).  Columns from
// j1 on are not touched.
template <int kGroup>
__device__ inline void qr_panel(double* P, int ld, int n, int j0, int j1, const QrScratch& s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = (tid - 32) / kGroup, sub = tid % kGroup;
  constexpr int kTailGroups = (HQ_THREADS - 32) / kGroup;
  if (warp == 0) house_gen(P, ld, n, j0, s.vs + (j0 & 1) * n, s.tau);
  __syncthreads();
  for (int j = j0; j < j1; ++j) {
    const double* vc = s.vs + (j & 1) * n;
    double* vn = s.vs + ((j + 1) & 1) * n;
    const double tj = s.tau[j];
    if (warp == 0) {
      if (j + 1 < j1) {
        double* cc = P + (size_t)(j + 1) * ld;
        if (tj != 0.0) {
          double w = 0.0;
          for (int r = j + lane; r < n; r += 32) w = fma(vc[r], cc[r], w);
          w = warp_sum(w) * tj;
          for (int r = j + lane; r < n; r += 32) cc[r] = fma(-w, vc[r], cc[r]);
          __syncwarp();
        }
        house_gen(P, ld, n, j + 1, vn, s.tau);
      }
    } else if (tj != 0.0) {
      for (int base = j + 2; base < j1; base += kTailGroups) {
        const int c = base + g;
        double* cc = P + (size_t)c * ld;
        double w = 0.0;
        if (c < j1)
          for (int r = j + sub; r < n; r += kGroup) w = fma(vc[r], cc[r], w);
        w = group_sum<kGroup>(w) * tj;
        if (c < j1)
          for (int r = j + sub; r < n; r += kGroup) cc[r] = fma(-w, vc[r], cc[r]);
      }
    }
    __syncthreads();
  }
}

// The reflectors of columns j0 .. j1 - 1 of P (j1 - j0 <= kQb; unit leading entries implied,
// tau[j0 ..]) applied at once to columns c0 .. n - 1, rows j0 .. n - 1, of A (A may be P when
// c0 >= j1):
//   kTrans:  A <- (H_j0 ... H_j1-1)^T A = A - V T^T (V^T A)   (trailing update of the QR)
//   !kTrans: A <- H_j0 ... H_j1-1 A     = A - V T (V^T A)     (Q formation)
// With W = V^T A, Z = T^T W is the forward substitution Z_k = tau_k (W_k - sum_{m<k} S_mk Z_m)
// and Z = T W the backward one Z_k = tau_k (W_k - sum_{m>k} S_km Z_m).  A column of A belongs to
// a group of 4 lanes (64 groups, more columns in further passes): each lane takes every fourth
// row, keeps kQb partial sums, and the group adds them with two shuffle steps.  V is copied to
// shared memory (s.wv, zero-padded to kQb columns) and read as 16-byte pairs.
template <bool kTrans>
__device__ __noinline__ void wy_apply(const double* P, int ld, int n, int j0, int j1, const QrScratch& s, double* A,
                                int c0) {
  const int kb = j1 - j0, nr = n - j0;
  double* V = s.wv;
  double* S = s.ws;
  for (int idx = threadIdx.x; idx < nr * kQb; idx += HQ_THREADS) {
    const int rr = idx / kQb, k = idx % kQb;
    double v = 0.0;
    if (k < kb) v = rr > k ? P[(size_t)(j0 + k) * ld + j0 + rr] : (rr == k ? 1.0 : 0.0);
    V[rr * kQbLd + k] = v;
  }
  __syncthreads();
  // S_ab = v_a . v_b for a < b: pair q = b (b - 1) / 2 + a per group of 8 lanes and pass
  {
    constexpr int kPairs = kQb * (kQb - 1) / 2;
    const int g8 = threadIdx.x >> 3, sub8 = threadIdx.x & 7;
    for (int base = 0; base < kPairs; base += HQ_THREADS / 8) {
      const int q = base + g8;
      int b = 1;
      while (b * (b + 1) / 2 <= q) ++b;
      const int a = q - b * (b - 1) / 2;
      double acc = 0.0;
      if (q < kPairs && b < kb)
        for (int rr = b + sub8; rr < nr; rr += 8) acc = fma(V[rr * kQbLd + a], V[rr * kQbLd + b], acc);
      acc = group_sum<8>(acc);
      if (q < kPairs && sub8 == 0) S[a * kQb + b] = acc;
    }
  }
  __syncthreads();
  const int g4 = threadIdx.x >> 2, sub = threadIdx.x & 3;
  const int ncols = n - c0;
  for (int base = 0; base < ncols; base += HQ_THREADS / 4) {
    const bool on = base + g4 < ncols;
    double* ac = A + (size_t)(c0 + (on ? base + g4 : 0)) * ld + j0;
    double w[kQb];
#pragma unroll
    for (int k = 0; k < kQb; ++k) w[k] = 0.0;
    if (on)
      for (int rr = sub; rr < nr; rr += 4) {
        const double a = ac[rr];
        const double2* vr = reinterpret_cast<const double2*>(V + rr * kQbLd);
#pragma unroll
        for (int k2 = 0; k2 < kQb / 2; ++k2) {
          const double2 v = vr[k2];
          w[2 * k2] = fma(v.x, a, w[2 * k2]);
          w[2 * k2 + 1] = fma(v.y, a, w[2 * k2 + 1]);
        }
      }
#pragma unroll
    for (int k = 0; k < kQb; ++k) w[k] = group_sum<4>(w[k]);
    if (kTrans) {
#pragma unroll
      for (int k = 0; k < kQb; ++k) {
        double z = w[k];
#pragma unroll
        for (int m = 0; m < k; ++m) z = fma(-S[m * kQb + k], w[m], z);
        w[k] = (k < kb ? s.tau[j0 + k] : 0.0) * z;
      }
    } else {
#pragma unroll
      for (int k = kQb - 1; k >= 0; --k) {
        double z = w[k];
#pragma unroll
        for (int m = k + 1; m < kQb; ++m) z = fma(-S[k * kQb + m], w[m], z);
        w[k] = (k < kb ? s.tau[j0 + k] : 0.0) * z;
      }
    }
    if (on)
      for (int rr = sub; rr < nr; rr += 4) {
        const double2* vr = reinterpret_cast<const double2*>(V + rr * kQbLd);
        double a = ac[rr];
#pragma unroll
        for (int k2 = 0; k2 < kQb / 2; ++k2) {
          const double2 v = vr[k2];
          a = fma(-v.x, w[2 * k2], a);
          a = fma(-v.y, w[2 * k2 + 1], a);
        }
        ac[rr] = a;
      }
  }
  __syncthreads();
}

template <int kGroup>
__device__ inline void qr_blocked(double* P, int ld, int n, const QrScratch& s) {
  for (int j0 = 0; j0 < n; j0 += kQb) {
    const int j1 = j0 + kQb < n ? j0 + kQb : n;
    qr_panel<kGroup>(P, ld, n, j0, j1, s);
    if (j1 < n) wy_apply<true>(P, ld, n, j0, j1, s, P, j1);
  }
}

// U <- H_0 ... H_{n-1}: the panels' block reflectors applied to the identity, last panel first
// (columns below a panel's first are still unit vectors there and need no update).
__device__ inline void form_q_blocked(const double* P, int ld, int n, double* U, const QrScratch& s) {
  set_identity(U, ld, n);
  __syncthreads();
  for (int j0 = ((n - 1) / kQb) * kQb; j0 >= 0; j0 -= kQb) {
    const int j1 = j0 + kQb < n ? j0 + kQb : n;
    wy_apply<false>(P, ld, n, j0, j1, s, U, j0);
  }
}

// The QR and the Q formation of a lattice class: blocked for the 16-wide class, column by
// column (with qr_group<LMAX>() lanes per column) below it.
template <int LMAX>
__device__ inline void qr_factor(double* P, int ld, int n, const QrScratch& s) {
  if constexpr (qr_blocked_class(LMAX)) qr_blocked<qr_group<LMAX>()>(P, ld, n, s);
  else qr_householder<qr_group<LMAX>()>(P, ld, n, s);
}

template <int LMAX>
__device__ inline void qr_form_q(const double* P, int ld, int n, double* U, const QrScratch& s) {
  if constexpr (qr_blocked_class(LMAX)) form_q_blocked(P, ld, n, U, s);
  else form_q<qr_group<LMAX>()>(P, ld, n, U, s);
}

// D[j] = |R_jj| and Tout = T' Tprev with T'(j, perm[c]) = R(j, c) / D[j] for c >= j
// (T' = D^-1 R Pi^T).  With Tprev == nullptr, Tout = T'.  Otherwise Tprev's rows are first
// gathered into Bs in pivot order (Bs(c, k) = Tprev(perm[c], k); Bs is scratch, e.g. the
// product that was just factored), so that Tout = D^-1 R Bs: upper triangular times dense, in
// 4 x 4 register tiles.  A warp takes 8 x 4 tiles (32 rows x 16 columns) and runs its k loop
// from its first row: R is read only at k >= row (below the diagonal P holds the reflectors).
// Blocks go to warps round-robin in row-block-major order, which spreads the long (top) and
// short (bottom) k ranges over the warps.
__device__ inline void t_update(const double* P, int ld, int n, const QrScratch& s, double* D,
                                const double* Tprev, double* Tout, double* Bs) {
  for (int j = threadIdx.x; j < n; j += HQ_THREADS) {
    const double dj = fabs(P[(size_t)j * ld + j]);
    D[j] = dj;
    s.rinv[j] = 1.0 / dj;
  }
  if (Tprev == nullptr) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
      const int j = idx % n, c = idx / n;
      Tout[(size_t)s.perm[c] * ld + j] = (c >= j) ? P[(size_t)c * ld + j] * s.rinv[j] : 0.0;
    }
  } else {
    for (int idx = threadIdx.x; idx < n * n; idx += HQ_THREADS) {
      const int c = idx % n, k = idx / n;
      Bs[(size_t)k * ld + c] = Tprev[(size_t)k * ld + s.perm[c]];
    }
    __syncthreads();
    const int tiles = n >> 2;  // n is a multiple of 4
    const int nrb = (tiles + 7) >> 3, ncb = (tiles + 3) >> 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rt = lane & 7, ct = lane >> 3;
    for (int blk = warp; blk < nrb * ncb; blk += HQ_WARPS) {
      const int R0 = (blk / ncb) * 32;
      const int r0 = R0 + 4 * rt, c0 = (blk % ncb) * 16 + 4 * ct;
      if (r0 >= n || c0 >= n) continue;
      double acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
      for (int k = R0; k < n; ++k) {
        double av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = (k >= r0 + a) ? P[(size_t)k * ld + r0 + a] : 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bs[(size_t)(c0 + b) * ld + k];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const double ri = s.rinv[r0 + a];
#pragma unroll
        for (int b = 0; b < 4; ++b) Tout[(size_t)(c0 + b) * ld + r0 + a] = acc[a][b] * ri;
      }
    }
  }
  __syncthreads();
}

// rd[j] = 1 / U_jj of the LU factors (one division per diagonal entry, not per use).
__device__ __forceinline__ void lu_diag_recip(const double* A, int ld, int n, double* rd) {
  for (int j = threadIdx.x; j < n; j += HQ_THREADS) rd[j] = 1.0 / A[(size_t)j * ld + j];
  __syncthreads();
}

// ------------------------------------------------------- blocked LU and triangular solves
// Right-looking LU with partial pivoting in panels of kLb columns (the LAPACK getrf scheme): a
// panel is factored column by column (pivot search over the whole column, swaps and updates
// inside the panel), its row swaps are then applied to the other columns, U12 = L11^-1 A12 is a
// small triangular solve per column, and the trailing block takes A22 -= L21 U12 as one rank-kLb
// update in 4 x 4 register tiles.  The column-by-column form swept the whole trailing matrix
// once per column with three loads per multiply-add.  Layout: L unit lower, U upper, piv[j]
// the row swapped with j at step j.
constexpr int kLb = 16;

// C(r0:r1, c0:c1) -= A(r0:r1, k0:k0+kb) B(k0:k0+kb, c0:c1), all column-major with stride ld;
// r1 - r0 and c1 - c0 multiples of 4, kb <= kLb.  The read and written regions must not overlap.
// No barrier at the end.
__device__ inline void rank_update(double* C, const double* A, const double* B, int ld, int r0, int r1, int c0, int c1,
                                   int k0, int kb) {
  const int tr = (r1 - r0) >> 2, tc = (c1 - c0) >> 2;
  for (int t = threadIdx.x; t < tr * tc; t += HQ_THREADS) {
    const int r = r0 + (t % tr) * 4, c = c0 + (t / tr) * 4;
    double acc[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int a = 0; a < 4; ++a) acc[a][b] = C[(size_t)(c + b) * ld + r + a];
    for (int k = k0; k < k0 + kb; ++k) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = A[(size_t)k * ld + r + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = B[(size_t)(c + b) * ld + k];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(-av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int a = 0; a < 4; ++a) C[(size_t)(c + b) * ld + r + a] = acc[a][b];
  }
}

// In-place blocked LU with partial pivoting; returns sum_j log|U_jj| (same value in every thread).
__device__ inline double lu_logdet_blocked(double* A, int ld, int n, int* piv, int* sint, double* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int p0 = 0; p0 < n; p0 += kLb) {
    const int p1 = p0 + kLb < n ? p0 + kLb : n, kb = p1 - p0;
    // panel: columns p0 .. p1 - 1
    for (int j = p0; j < p1; ++j) {
      double* aj = A + (size_t)j * ld;
      if (warp == 0) {
        double best = -1.0;
        int bi = j;
        for (int r = j + lane; r < n; r += 32) {
          const double v = fabs(aj[r]);
          if (v > best) { best = v; bi = r; }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const double ob = __shfl_xor_sync(HQ_FULL, best, o);
          const int oi = __shfl_xor_sync(HQ_FULL, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) {
          sint[0] = bi;
          piv[j] = bi;
          red[0] = 1.0 / aj[bi];
        }
      }
      __syncthreads();
      const int p = sint[0];
      if (p != j) {
        if (tid < kb) {
          double* ac = A + (size_t)(p0 + tid) * ld;
          const double a = ac[j];
          ac[j] = ac[p];
          ac[p] = a;
        }
        __syncthreads();
      }
      const double rp = red[0];
      for (int r = j + 1 + tid; r < n; r += HQ_THREADS) aj[r] *= rp;
      __syncthreads();
      const int m = n - j - 1, w = p1 - j - 1;
      for (int idx = tid; idx < m * w; idx += HQ_THREADS) {
        const int r = j + 1 + idx % m, c = j + 1 + idx / m;
        A[(size_t)c * ld + r] = fma(-aj[r], A[(size_t)c * ld + j], A[(size_t)c * ld + r]);
      }
      __syncthreads();
    }
    // the panel's swaps on the other columns, then U12 = L11^-1 A12 (one column per thread)
    for (int c = tid; c < n; c += HQ_THREADS) {
      if (c >= p0 && c < p1) continue;
      double* ac = A + (size_t)c * ld;
      for (int j = p0; j < p1; ++j) {
        const int p = piv[j];
        if (p != j) { const double a = ac[j]; ac[j] = ac[p]; ac[p] = a; }
      }
      if (c >= p1) {
        double x[kLb];
#pragma unroll
        for (int i = 0; i < kLb; ++i) x[i] = i < kb ? ac[p0 + i] : 0.0;
#pragma unroll
        for (int i = 0; i < kLb; ++i) {
          if (i < kb) {
            const double* li = A + (size_t)(p0 + i) * ld + p0;
#pragma unroll
            for (int r = i + 1; r < kLb; ++r)
              if (r < kb) x[r] = fma(-li[r], x[i], x[r]);
          }
        }
#pragma unroll
        for (int i = 0; i < kLb; ++i)
          if (i < kb) ac[p0 + i] = x[i];
      }
    }
    __syncthreads();
    if (p1 < n) {
      rank_update(A, A, A, ld, p1, n, p1, n, p0, kb);
      __syncthreads();
    }
  }
  double a = 0.0;
  for (int j = tid; j < n; j += HQ_THREADS) a += log(fabs(A[(size_t)j * ld + j]));
  return block_sum(a, red);
}

// Y <- A^-1 Y (n right-hand sides) for the factors of lu_logdet_blocked; rd: reciprocals of U's
// diagonal (lu_diag_recip).  The row swaps, then L and U by blocks of kLb rows: a kLb x kLb
// triangular solve per column (one column per thread, in registers) and a rank-kLb update of
// the rows still to solve.
__device__ inline void lu_solve_blocked(const double* A, int ld, int n, const int* piv, const double* rd, double* Y) {
  const int tid = threadIdx.x;
  for (int c = tid; c < n; c += HQ_THREADS) {
    double* y = Y + (size_t)c * ld;
    for (int j = 0; j < n; ++j) {
      const int p = piv[j];
      if (p != j) { const double a = y[j]; y[j] = y[p]; y[p] = a; }
    }
  }
  __syncthreads();
  for (int p0 = 0; p0 < n; p0 += kLb) {
    const int p1 = p0 + kLb < n ? p0 + kLb : n, kb = p1 - p0;
    for (int c = tid; c < n; c += HQ_THREADS) {
      double* y = Y + (size_t)c * ld + p0;
      double x[kLb];
#pragma unroll
      for (int i = 0; i < kLb; ++i) x[i] = i < kb ? y[i] : 0.0;
#pragma unroll
      for (int i = 0; i < kLb; ++i) {
        if (i < kb) {
          const double* li = A + (size_t)(p0 + i) * ld + p0;
#pragma unroll
          for (int r = i + 1; r < kLb; ++r)
            if (r < kb) x[r] = fma(-li[r], x[i], x[r]);
        }
      }
#pragma unroll
      for (int i = 0; i < kLb; ++i)
        if (i < kb) y[i] = x[i];
    }
    __syncthreads();
    if (p1 < n) {
      rank_update(Y, A, Y, ld, p1, n, 0, n, p0, kb);
      __syncthreads();
    }
  }
  for (int p0 = ((n - 1) / kLb) * kLb; p0 >= 0; p0 -= kLb) {
    const int p1 = p0 + kLb < n ? p0 + kLb : n, kb = p1 - p0;
    for (int c = tid; c < n; c += HQ_THREADS) {
      double* y = Y + (size_t)c * ld + p0;
      double x[kLb];
#pragma unroll
      for (int i = 0; i < kLb; ++i) x[i] = i < kb ? y[i] : 0.0;
#pragma unroll
      for (int i = kLb - 1; i >= 0; --i) {
        if (i < kb) {
          x[i] *= rd[p0 + i];
          const double* ui = A + (size_t)(p0 + i) * ld + p0;
#pragma unroll
          for (int r = 0; r < i; ++r) x[r] = fma(-ui[r], x[i], x[r]);
        }
      }
#pragma unroll
      for (int i = 0; i < kLb; ++i)
        if (i < kb) y[i] = x[i];
    }
    __syncthreads();
    if (p0 > 0) {
      rank_update(Y, A, Y, ld, 0, p0, 0, n, p0, kb);
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------- CTA GEMM
// C = op(A) op(B) for n x n column-major operands (n a multiple of 4: n = nx*ny with
// even sides); each thread accumulates 4x4 tiles.
template <bool TA, bool TB>
__device__ inline void gemm_nn(int n, const double* A, const double* B, double* C, int ld) {
  const int tiles = n >> 2;
  for (int t = threadIdx.x; t < tiles * tiles; t += HQ_THREADS) {
    const int r0 = (t % tiles) * 4, c0 = (t / tiles) * 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int k = 0; k < n; ++k) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = TA ? A[(size_t)(r0 + a) * ld + k] : A[(size_t)k * ld + r0 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = TB ? B[(size_t)k * ld + c0 + b] : B[(size_t)(c0 + b) * ld + k];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) C[(size_t)(c0 + b) * ld + r0 + a] = acc[a][b];
  }
  __syncthreads();
}

}  // namespace hq
