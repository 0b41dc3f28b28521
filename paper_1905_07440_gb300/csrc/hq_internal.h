// Internal interface between the C-ABI host code and the kernels (not exported).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace hq {

constexpr int kMaxSide = 16;
constexpr int kMaxN = 256;
constexpr int kMaxK = 32;
constexpr int kWorkMats = 7;   // per-chain N x N work matrices
constexpr int kAccSlots = 8;   // per-chain per-sweep accumulators
constexpr int kTotSlots = 16;  // per-chain running totals
constexpr int kCounters = 5;   // local proposed / accepted, global proposed / accepted, wrap_tol exceeded
constexpr int kSchedHeader = 32;  // block-move task queue: counter, abort flag, then progress[C]
constexpr int kWorkersPerSm = 2;
constexpr int kMaxDevices = 64;
constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;  // static scratch of hq_logdet_noalloc
constexpr unsigned long long kWaitLimitNs = 30ull * 1000000000ull;  // bounded wait of a task

// accumulator slots (per sweep)
enum { ACC_DENSITY = 0, ACC_DOCC = 1, ACC_SCDW = 2, ACC_COUNT = 3, ACC_WRAP = 4 };
// running-total slots
enum { TOT_DENSITY = 0, TOT_DOCC = 1, TOT_SCDW = 2, TOT_MEASURED = 3, TOT_XMEAN = 4, TOT_X2 = 5,
       TOT_SWEEPS = 6, TOT_WRAP = 7 };
// work matrix slots
enum { WK_P = 0, WK_U = 1, WK_T = 2, WK_T2 = 3, WK_M1 = 4, WK_M2 = 5, WK_M3 = 6 };

struct Dev {
  // model and run shape
  int nx, ny, n, L, n_wrap, k, n_chains, first_chain, n_bound, max_series;
  double t, mu, omega, mass, g, dtau, dx_local, dx_global;
  uint32_t key0, key1;
  // device buffers (bases over all chains)
  const double* kin;  // ex[nx*nx], exi[nx*nx], ey[ny*ny], eyi[ny*ny]
  double* X;          // [C][L][N]
  double* G;          // [C][N*N] column-major
  double* logdet;     // [C]
  double* UR;         // [C][N*N] right UDV (product B_l..B_1)
  double* TR;         // [C][N*N]
  double* DR;         // [C][N]
  double* work;       // [C][kWorkMats][N*N]
  double* stU;        // [C][n_bound][N*N] left stack (transposed product B_L..B_{b+1})
  double* stT;        // [C][n_bound][N*N]
  double* stD;        // [C][n_bound][N]
  double* Adl;        // [C][k][N] delayed-update columns
  double* Bdl;        // [C][k][N] delayed-update rows
  double* acc;        // [C][kAccSlots]
  double* tot;        // [C][kTotSlots]
  double* series;     // [C][HQ_N_OBS][max_series]
  long long* counters;  // [C][kCounters]
  int* status;        // [C]
  int* sched;         // [kSchedHeader + C] block-move task queue
  uint32_t* cid;      // [C][4] per chain: Philox key (2 words), chain word, sweep/step counter
  int* active;        // [C] 0: the slot takes no work
  int* slen;          // [C] per-sweep records kept for the chain
  double wrap_tol;    // stabilisation back-off threshold (0: off)
  int n_wrap_min;     // back-off floor
  int* wrap_flag;     // [1] set by a chain whose sweep exceeded wrap_tol
  int n_active;       // host count of active slots (sizes the persistent launch)
  int block_sites;    // block moves per sweep: 0 every site, else a run of this many sites
  // chunk propagators for block moves (used when use_cm != 0)
  int use_cm, n_chunks;
  double* expV;       // [C][L][N] exp(-dtau V) of the current fields
  double* cmat;       // [C][2][n_chunks][N*N] chunk products, current and proposed
  int* cbuf;          // [C] index of the current buffer
  double* corr;       // [C][2 N L + L] correction vectors of every chunk, shifted diagonal
};

// A heterogeneous group of engines swept together (device copy of each engine's
// descriptor; task table of chain-sweeps, entry = engine << 26 | chain, longest first).
constexpr int kGroupMaxEngines = 64;
struct GroupDev {
  const Dev* devs;        // [n_eng]
  const uint32_t* tasks;  // [n_tasks]
  int* sched;             // [kSchedHeader] task counter
  int n_eng, n_tasks;
};

// FP64 flop model of one chunk of a block move: n_wrap separable slice applications versus
// the chunk-propagator update (rank-m correction vectors, rank-m update, one GEMM).
inline bool chunk_propagators_pay(int nx, int ny, int L, int n_wrap) {
  const double n = (double)nx * ny;
  const int chunks = (L + n_wrap - 1) / n_wrap;
  const double m = (double)L / chunks;
  const double slice = 2.0 * n * n * (nx + ny) + n * n;
  const double vec = 2.0 * n * (nx + ny) + n;
  const double sep = m * slice;
  const double cm = 2.0 * n * n * n + 2.0 * m * n * n + m * m * vec + n * n;
  return cm < 0.9 * sep;
}

// State of the learned effective action and the cumulative sampler (separate device arena).
constexpr int kNNCounters = 6;   // inner local prop/acc, inner block prop/acc, cumulative prop/acc
constexpr int kNNTrainCtas = 256;
struct NNState {
  uint16_t* wbf;        // bfloat16 weights used by every kernel
  float* master;        // FP32 master weights (training)
  float* grad;          // last gradient
  float* adam_m;
  float* adam_v;
  float* partials;      // [kNNTrainCtas][padded params] per-CTA gradient partials
  float* fcache;        // [C][L N] f of every patch of the current fields
  float* fnew;          // [C][5 L] block-move scratch
  double* X0;           // [C][L N] fields at the start of a cumulative step
  double* ld0;          // [C]
  double* F0;           // [C]
  double* F1;           // [C]
  double* last_pc;      // [C]
  double* Fb;           // [max batch] minibatch F
  double* loss;         // [1] epoch loss accumulator
  int* idx;             // [max samples] minibatch order
  long long* counters;  // [C][kNNCounters]
  double* dFpath;       // [C] sum of the accepted inner moves' network changes (cumulative step)
  double* G0;           // [C][N*N] G_0 of the step's starting fields (measured steps)
  float* xf;            // [C][L N] network inputs (float)(X - x0) of the current fields
  float* xb;            // [max batch][L N] network inputs of a training minibatch
  double x0;            // input shift -g/(M Omega^2)
};

// Periodic 3D convolutional action for block moves: three 3x3x3 layers 1 -> 16 -> 16 -> 1
// on the (x, y, tau) torus, summed over every point.  Activations are stored after the ReLU,
// 16 floats per point (point-major).  Window buffers hold the block-move proposal around the
// moved site: radius 1 (layer 1), 2 (layer 2), 3 (layer 3) in the lattice, every slice.
constexpr int kCnnC = 16;
constexpr int kCnnTrainCtas = 152;
struct CnnState {
  int on;               // parameters have been set
  uint16_t* wbf;        // bfloat16 weights used by every kernel
  float* master;        // FP32 master weights (training)
  float* grad;
  float* adam_m;
  float* adam_v;
  float* partials;      // [train_ctas][padded params]
  int train_ctas;
  float* h1c;           // [C][L N][16] layer-1 activations of the current fields
  float* h2c;           // [C][L N][16]
  float* o3c;           // [C][L N] layer-3 outputs
  float* h1p;           // [C][9 L][16] proposal, window radius 1
  float* h2p;           // [C][25 L][16] radius 2
  float* o3p;           // [C][49 L] radius 3
  float* tr;            // [train_ctas][3][L N][16] training activations and gradients
  double* Fb;           // [max batch] minibatch F
  double* F;            // [C]
};

size_t smem_bytes(const Dev& d);
// shared memory of a chain of d in a kernel of class lmax (group launches: the group's class)
size_t smem_bytes_class(const Dev& d, int lmax);

// Raise a kernel's dynamic shared memory limit to the device maximum (once per kernel and
// device) when it needs more than the default 48 KB.
cudaError_t opt_in_smem(const void* kernel, size_t bytes);

// Launchers (asynchronous on the stream).  Return cudaGetLastError().
cudaError_t launch_stack_build(const Dev& d, cudaStream_t s);
// The whole local phase (every chunk of every chain) as one persistent launch.
cudaError_t launch_local_phase(const Dev& d, int measure, cudaStream_t s);
cudaError_t launch_global_phase(const Dev& d, cudaStream_t s);
cudaError_t launch_sweep_end(const Dev& d, int measured, cudaStream_t s);
cudaError_t launch_reset_acc(const Dev& d, cudaStream_t s);
// Slot identity/activity: slot >= 0 sets that slot (reset: key, chain word, sweep counter,
// series length, accumulators, counters, status); slot < 0 sets every chain c with chain
// word chain + c.
cudaError_t launch_slot_control(const Dev& d, int slot, uint32_t key0, uint32_t key1, uint32_t chain, uint32_t sweep,
                                int active, int reset, cudaStream_t s);
cudaError_t launch_log_weight(const Dev& d, double* out_logw, cudaStream_t s);
cudaError_t launch_proposals(uint32_t key0, uint32_t key1, uint32_t chain, uint32_t sweep, uint32_t tag,
                             const uint32_t* events, int n, double* u1, double* u2, cudaStream_t s);
double fp64_probe_tflops(int kind, int reps, cudaStream_t s);
cudaError_t launch_measure_g0(const Dev& d, cudaStream_t s);
cudaError_t nn_launch_eval(const Dev& d, const NNState& nn, const double* X, double* F, int write_cache,
                           cudaStream_t s);

cudaError_t nn_launch_decide(const Dev& d, const NNState& nn, int restore_g, cudaStream_t s);
cudaError_t nn_launch_set(const NNState& nn, const float* src_device, cudaStream_t s);
cudaError_t nn_launch_batch(const Dev& d, const NNState& nn, const double* Xs, const double* ys, const int* idx,
                            int B, float lr, int t_step, cudaStream_t s);
cudaError_t nn_launch_loss(const NNState& nn, const double* ys, const int* idx, int B, double scale, cudaStream_t s);
// Inner network sweeps; window > 0 limits local moves to `window` consecutive slices and
// site_window > 0 block moves to `site_window` consecutive sites, from random starts per step.
cudaError_t nn_launch_inner(const Dev& d, const NNState& nn, const CnnState& cn, int n_inner, int do_local,
                            int do_block, int use_cnn, int window, int site_window, cudaStream_t s);
cudaError_t cnn_launch_eval(const Dev& d, const CnnState& cn, const double* X, double* F, int write_cache,
                            cudaStream_t s);
cudaError_t cnn_launch_set(const CnnState& cn, const float* src_device, cudaStream_t s);
cudaError_t cnn_launch_batch(const Dev& d, const CnnState& cn, const double* Xs, const double* ys, const int* idx,
                             int B, float lr, int t_step, cudaStream_t s);
cudaError_t cnn_launch_loss(const CnnState& cn, const double* ys, const int* idx, int B, double scale,
                            double* loss, cudaStream_t s);
int section_cycles(unsigned long long* out, int n);
// Bounded-wait probe (limit_s of waiting on a flag nothing sets); writes the kernel's status.
cudaError_t wait_probe(double limit_s, cudaStream_t s, int* status);
int lmax_class(int nx, int ny);
// One persistent launch sweeping every chain of a group (flags as hq_sweep; stack != 0 runs
// the stack build first).
cudaError_t launch_group_sweep(const GroupDev& g, int lmax, size_t sb, int n_active, int flags, int stack,
                               cudaStream_t s);
// Split boundary of the two-half log|det M| (a restabilisation boundary near L/2), 0 if the
// product has fewer than two chunks.
int split_point(const Dev& d);
// log|det M| and G_m of every chain's fields by two CTAs per chain (slices above and below the
// boundary m; part 0) joined by the two-sided formula (part 1, after part 0); writes the stack
// slot of boundary m and the right factors UR, DR, TR (part 0), d.logdet and d.G = G_m (part 1).
cudaError_t launch_split_logdet(const Dev& d, int m, int part, cudaStream_t s);
size_t noalloc_scratch_needed(int nx, int ny, int n_chains);
// log|det M| per chain with all scratch in the library's static device array (no allocation).
cudaError_t launch_logdet_noalloc(Dev d, double* out, cudaStream_t s);

}  // namespace hq
