/*
 * holstein_dqmc.h -- C ABI of the GB300 DQMC fermion-weight engine for the 2D Holstein model.
 *
 * Model and method: Li, Dee, Khatami, Johnston, arXiv:1905.07440.
 *   "Model": H = H0 + H_lat + H_e-ph on an N = nx*ny periodic square lattice, hopping t,
 *            chemical potential mu, ion mass M, phonon frequency Omega, coupling g X_i n_i.
 *   "Determinant quantum Monte Carlo": L = beta/dtau imaginary-time slices; the phonon
 *            field X(i,l) is sampled with weight W(X) = exp(-dtau S_ph) det(M_up) det(M_dn),
 *            M = I + B_L ... B_1, S_ph = M/(2 dtau^2) sum (X_{i,l+1}-X_{i,l})^2
 *            + M Omega^2/2 sum X_{i,l}^2; local moves X(i,l) += dX and block moves
 *            X(i,.) += dX_i are accepted with p = W(X')/W(X).
 *
 * Conventions (all FP64):
 *   B_l = exp(-dtau K) exp(-dtau V_l), K_ij = -t per nearest-neighbour displacement,
 *   V_l = diag(g X(.,l) - mu).  G_l = (I + B_l..B_1 B_L..B_{l+1})^{-1}, G_ij = <c_i c_j^+>.
 *   Site index i = x + nx*y.  Fields are laid out X[chain][l][i] (l = 0..L-1 is slice l+1).
 *   A sweep = local moves at every (l, i) (l ascending, i ascending) with delayed rank-k
 *   updates of G and a wrap G <- B_l G B_l^{-1} after each slice, restabilisation every
 *   n_wrap slices (column-pivoted QR, UDV), then one block move per site (i ascending),
 *   each accepted on the full stabilised determinant ratio.
 *   Proposals come from Philox4x32-10 (Salmon et al., SC'11): key = seed, counter =
 *   (event, sweep, chain, tag), event = l*N + i (tag 0, local) or i (tag 1, block);
 *   u = ((w0>>5)*2^26 + (w1>>6)) 2^-53, dX = dx*(2 u1 - 1); accept iff u2 < p.
 *
 * Memory: the caller owns every host buffer; the API copies in and out.  The engine
 * never allocates device memory: the caller passes one device arena of at least
 * hq_arena_bytes() bytes (256-byte aligned), which holds all device state, and keeps it
 * alive until hq_destroy().  Work is issued on the caller's CUDA stream (borrowed); calls
 * that return data to the host synchronise that stream, other calls do not.
 *
 * Errors: functions return HQ_OK (0) or a negative HQ_E* code; hq_last_error() gives a
 * message.  Nothing is thrown across the ABI.
 */
#ifndef HOLSTEIN_DQMC_H
#define HOLSTEIN_DQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HQ_OK 0
#define HQ_EINVAL (-1)     /* bad argument or parameter set */
#define HQ_ENOMEM (-2)     /* arena too small / misaligned */
#define HQ_ECUDA (-3)      /* a CUDA runtime call failed */
#define HQ_EUNSTABLE (-4)  /* wrap error above wrap_tol at the n_wrap floor (reported, chain kept) */
#define HQ_ENAN (-5)       /* non-finite G, ratio or log-determinant */
#define HQ_ETIMEOUT (-6)   /* a bounded device wait expired (chain state incomplete) */

/* hq_sweep flags */
#define HQ_LOCAL 1u
#define HQ_GLOBAL 2u
#define HQ_MEASURE 4u

/* observable ids for hq_get_series */
#define HQ_OBS_DENSITY 0    /* <n> = (2/N) sum_i (1 - G_ii), averaged over restabilised slices */
#define HQ_OBS_DOUBLE_OCC 1 /* (1/N) sum_i (1 - G_ii)^2 */
#define HQ_OBS_SCDW 2       /* S_CDW(pi,pi) = (1/N) sum_ij (-1)^(i+j) <n_i n_j> (Wick) */
#define HQ_OBS_X_MEAN 3     /* (1/NL) sum X at the end of the sweep */
#define HQ_OBS_X2 4         /* (1/NL) sum X^2 at the end of the sweep */
#define HQ_OBS_WRAP_ERR 5   /* max |G_wrapped - G_fresh| over the sweep's restabilisations */
#define HQ_N_OBS 6

typedef struct hq_params {
  int nx, ny;       /* lattice sides: even, 2..16 each (N = nx*ny <= 256) */
  double t;         /* nearest-neighbour hopping */
  double mu;        /* chemical potential (half filling: -g^2/(M Omega^2)) */
  double omega;     /* phonon frequency Omega > 0 */
  double mass;      /* ion mass M > 0 */
  double g;         /* electron-phonon coupling */
  double beta;      /* inverse temperature; beta/dtau must be an integer L >= 2 */
  double dtau;      /* Trotter step > 0 */
  int n_wrap;       /* restabilise every n_wrap slices, >= 1 */
  int delay_k;      /* delayed-update rank, 1..32 */
  double dx_local;  /* local proposal dX ~ U[-dx_local, dx_local) */
  double dx_global; /* block proposal dX ~ U[-dx_global, dx_global) */
  uint64_t seed;    /* Philox key */
  int block_method; /* block-move algorithm: 0 chosen by the FP64 flop model, 1 every slice
                       through the separable exp(-dtau K), 2 chunk propagators (same results
                       up to rounding; hq_autotune measures them) */
  int n_wrap_min;   /* stabilisation back-off floor (with wrap_tol > 0): 1..n_wrap, 0 = 1 */
  double wrap_tol;  /* stabilisation back-off: 0 off; > 0, after every sweep with local moves
                       hq_sweep reads whether a chain's largest |G_wrapped - G_fresh| of that
                       sweep exceeded wrap_tol (one device-to-host read and a stream
                       synchronisation per sweep), and if so halves n_wrap for the whole engine
                       (restabilising twice as often; its chains share one chunk structure) down
                       to n_wrap_min; at the floor the chains concerned get status HQ_EUNSTABLE
                       and hq_sweep returns HQ_EUNSTABLE (the sweeps are done, the chains kept).
                       The arena is sized for n_wrap_min. */
} hq_params;

typedef struct hq_obs {   /* per chain, accumulated since hq_create / hq_restore */
  int64_t sweeps;          /* sweeps run */
  int64_t measured;        /* sweeps with electronic measurements */
  int64_t local_proposed, local_accepted;
  int64_t global_proposed, global_accepted;
  double density, double_occ, s_cdw;  /* means over measured sweeps */
  double x_mean, x2;                  /* means over sweeps */
  double max_wrap_error;              /* max over all restabilisations */
  double logdet;                      /* log|det M| of the current fields */
  int32_t status;                     /* 0, or HQ_ENAN / HQ_ETIMEOUT / HQ_EUNSTABLE */
  int32_t n_wrap;                     /* the engine's current restabilisation interval */
  int64_t wrap_exceeded;              /* sweeps whose largest wrap error exceeded wrap_tol */
} hq_obs;

typedef struct hq_engine hq_engine;

/* Bytes of device arena needed for n_chains chains keeping up to max_series per-sweep
 * records of each observable.  Returns 0 if the parameters are invalid. */
size_t hq_arena_bytes(const hq_params* p, int n_chains, int max_series);

/* Create an engine for n_chains independent chains (Philox chain ids first_chain ..
 * first_chain+n_chains-1).  device_arena: device pointer, 256-byte aligned, >= arena_bytes
 * from hq_arena_bytes(); owned by the caller.  stream: a cudaStream_t (NULL = legacy
 * default stream), borrowed.  Fields start at zero; call hq_set_fields(). */
int hq_create(const hq_params* p, int n_chains, int first_chain, int max_series,
              void* device_arena, size_t arena_bytes, void* stream, hq_engine** out);

/* Copy fields in from the host, X_host[chain][l][i] (n_chains*L*N doubles); G, the UDV
 * stack and log|det M| are recomputed before the next use.  Resets no counters.
 * Paper, "Model": the phonon field X_{i,l} on the space-time lattice. */
int hq_set_fields(hq_engine* e, const double* X_host);
/* Same from a device buffer of the same layout (copied on the engine's stream). */
int hq_set_fields_device(hq_engine* e, const double* X_device);
/* Copy the current fields out to the host (synchronises the stream). */
int hq_get_fields(hq_engine* e, double* X_host);

/* Run n_sweeps sweeps of every chain.  flags: HQ_LOCAL | HQ_GLOBAL | HQ_MEASURE.
 * Paper, "Determinant quantum Monte Carlo": local Metropolis moves of X_{i,l} with the
 * determinant ratio and the fast update of G, wraps and periodic restabilisation, then one
 * block move per site accepted on the full determinant ratio.  Asynchronous on the engine's stream; returns HQ_EINVAL for bad flags, HQ_ENOMEM if
 * more than max_series measured sweeps would be recorded. */
int hq_sweep(hq_engine* e, int n_sweeps, unsigned flags);

/* log W = 2 log|det M| - dtau S_ph and log|det M| of the current fields, one per chain
 * (host arrays of n_chains doubles; either may be NULL).  Synchronises.
 * Paper, "Determinant quantum Monte Carlo": the weight e^{-dtau S_ph} (det M)^2. */
int hq_log_weight(hq_engine* e, double* logw_host, double* logdet_host);

/* G_0 = G_L of one chain for the current fields, row-major G[i*N+j] = G_ij = <c_i c_j^+>
 * (host, N*N doubles); *slice = 0.  Synchronises.  Paper, "Determinant quantum Monte
 * Carlo": the equal-time Green's function (I + B_L ... B_1)^-1. */
int hq_get_green(hq_engine* e, int chain, double* G_host, int* slice);

/* Per-chain accumulated observables (host array of n_chains hq_obs).  Synchronises.
 * Paper, "Benchmarks": <X^2>, double occupancy and the CDW structure factor S(pi, pi). */
int hq_get_observables(hq_engine* e, hq_obs* out);

/* Per-sweep series of one observable: out[chain][s] for s < *n_out (host, n_chains *
 * max_series doubles; *n_out = the longest chain record).  NaN where the sweep had no
 * electronic measurement or beyond a chain's own record. */
int hq_get_series(hq_engine* e, int obs_id, double* out, int* n_out);

/* Serialise the chain state (fields, sweep counter, counters, accumulators, series).
 * With buf == NULL only *len is set.  Synchronises. */
int hq_checkpoint(hq_engine* e, void* buf, size_t* len);
/* Restore a state written by hq_checkpoint for the same parameters and chain count. */
int hq_restore(hq_engine* e, const void* buf, size_t len);

/* Block moves of a plain sweep on a run of sites (the reduced protocol for large lattices,
 * where a block move costs a whole stabilised determinant): with sites > 0 (and < N) each
 * sweep's block moves visit `sites` consecutive sites j0, j0 + 1, ... (mod N, index order) with
 * j0 = floor(u N), u the first uniform of event N of the chain's tag-1 Philox block of that
 * sweep; the moves themselves draw from their site's event as in a full sweep.  0 (default) or
 * sites >= N: every site.  Applies to hq_sweep and hq_group_sweep.  Errors: HQ_EINVAL for a
 * null engine or sites < 0. */
int hq_set_block_sites(hq_engine* e, int sites);

/* Block-move algorithm in use: 0 = every slice applied through the separable exp(-dtau K)
 * per move, 1 = chunk propagators (the n_wrap-slice products kept per chain, updated by a
 * rank-n_wrap correction per move and applied with one GEMM per chunk).  Chosen by
 * hq_params.block_method, or when that is 0 by an FP64 flop model.  Both give the same
 * determinants up to rounding. */
int hq_block_move_method(const hq_engine* e);

/* Heterogeneous groups.  Engines of different lattices, temperatures and couplings (each
 * with its own chains, fields and arena) swept together by one persistent launch per sweep:
 * a chain's sweep (stack build, local chunks, block moves, records) is sequential, so workers
 * take whole chain-sweeps from the group's table, longest estimated first, and short chains
 * fill in around long ones; small engines fill the GPU together instead of one after another.
 * Each chain computes exactly what its own engine's hq_sweep computes.  The group borrows the
 * engines: do not destroy them while the group exists (hq_group_sweep orders itself after the
 * engines' streams, and the engines' later calls after itself).  The group's device arena
 * (hq_group_arena_bytes, 256-byte aligned) holds the engine descriptors and the task table,
 * uploaded once, so an engine's chain count must not change afterwards (slots may be idled
 * and reloaded).
 * Errors: HQ_EINVAL for 0 or more than 64 engines, a repeated or null engine, an engine with
 * more than 65535 chains; HQ_ENOMEM for a missing or small arena. */
typedef struct hq_group hq_group;
size_t hq_group_arena_bytes(hq_engine* const* engines, int n_engines);
int hq_group_create(hq_engine* const* engines, int n_engines, void* device_arena, size_t arena_bytes,
                    void* cuda_stream, hq_group** out);
/* n_sweeps sweeps of every chain of every engine (flags as hq_sweep).  Asynchronous. */
int hq_group_sweep(hq_group* g, int n_sweeps, unsigned flags);
void hq_group_destroy(hq_group* g);

/* Autotuner for the runtime choices that change speed but not results (beyond rounding): the
 * delayed-update rank k and the block-move algorithm.  For every pair (ks[a], methods[b])
 * (methods: 1 per-slice, 2 chunk propagators) it builds an engine of n_chains chains with
 * parameters p in the caller's device arena (at least hq_autotune_arena_bytes bytes, 256-byte
 * aligned; the engine is destroyed before the next pair), copies the fields X_device
 * [n_chains][L][N] in, runs `warmup` sweeps with `flags`, then times `reps` sweeps with CUDA
 * events on the stream.  ms_out[a * n_methods + b] receives milliseconds per sweep; best_k
 * and best_method the fastest pair.  Synchronises.  The paper has no counterpart: it fixes
 * neither k nor the block-move algorithm.
 * Errors: HQ_EINVAL for bad arguments or a candidate outside 1..32 / 1..2; HQ_ENOMEM if the
 * arena is too small; CUDA errors as HQ_ECUDA. */
size_t hq_autotune_arena_bytes(const hq_params* p, int n_chains, const int* ks, int n_k);
int hq_autotune(const hq_params* p, int n_chains, const double* X_device, void* device_arena, size_t arena_bytes,
                void* stream, const int* ks, int n_k, const int* methods, int n_methods, unsigned flags, int warmup,
                int reps, double* ms_out, int* best_k, int* best_method);

/* Slots.  Every chain slot carries its own Philox key, chain word and sweep counter (set by
 * hq_create to seed, first_chain + slot, 0; the counter advances by one per sweep or
 * cumulative step of that chain), so a chain's trajectory depends only on its own fields and
 * identity, not on which slot it occupies or what else runs in the engine.
 * hq_set_chain loads one slot (fields X_host [L][N], key `seed`, chain word, counter), clears
 * its counters, totals and series, and makes it active; it synchronises the stream, so the
 * caller may reuse X_host on return.  X_host in page-locked memory keeps the copy from
 * waiting for kernels of other streams.  hq_set_active(e, slot, 0) idles a slot (it takes no
 * work until reactivated or reloaded); it is stream-ordered and does not synchronise.
 * Errors: HQ_EINVAL for a null engine or pointer or a slot outside [0, n_chains). */
int hq_set_chain(hq_engine* e, int slot, const double* X_host, uint64_t seed, uint32_t chain_id, uint32_t sweep);
int hq_set_active(hq_engine* e, int slot, int active);

/* Number of chains, sites N, slices L and sweeps run. */
int hq_shape(const hq_engine* e, int* n_chains, int* n_sites, int* n_slices, int64_t* sweeps);

/* Message of the engine's last error; with e == NULL, that of the calling thread's last
 * failing call that takes no engine (hq_logdet_noalloc). */
const char* hq_last_error(const hq_engine* e);
void hq_destroy(hq_engine* e);

/* Proposal stream check: the Philox uniforms (u1, u2) the sampler draws for the given
 * events of (chain, sweep, tag), computed on the device.  u1_host, u2_host: n doubles.
 * Synchronises the given stream. */
int hq_proposal_uniforms(uint64_t seed, uint32_t chain, uint32_t sweep, uint32_t tag,
                         const uint32_t* events_host, int n, double* u1_host,
                         double* u2_host, void* stream);

/* Integrated autocorrelation time of a series (host code): tau = 1/2 + sum_{t=1}^{W}
 * rho(t) with the smallest window W >= c*tau (Madras-Sokal; c = 6 is usual).  Returns
 * tau, stores W in *window if non-NULL.  n < 2 gives 0.5. */
double hq_tau_int(const double* series, int n, double c, int* window);

/* Kernel timing of hq_sweep and hq_cumulative_sweep: when enabled, CUDA events on the
 * engine's stream bracket every launch group -- phase 0: stack build (1 launch), 1: local phase
 * (1 persistent launch), 2: block moves (1 persistent launch: N x n_chains moves, or the run of
 * sites set by hq_set_block_sites), 3: sweep end (with a measured cumulative step also the
 * measurement launch), 4: the two-half log|det M| of cumulative steps (1 launch, two CTAs per
 * chain), 5: its join (1 launch), 6: network evaluation of the current fields (patch network,
 * and the convolutional action when used), 7: the inner network-driven sweep (1 launch).  The
 * cumulative decide launch is not timed.  hq_get_timing synchronises, returns the milliseconds
 * and launches per phase accumulated since the last call (ms[HQ_N_PHASES],
 * launches[HQ_N_PHASES]) and clears them. */
#define HQ_N_PHASES 8
int hq_set_timing(hq_engine* e, int enable);

/* CUDA-graph replay of sweeps (no counterpart in the paper; it trims the host's launch cost,
 * which matters for small lattices whose sweeps take a few milliseconds).  With enable != 0,
 * hq_sweep runs the first sweep of each shape eagerly, captures the next one on the engine's
 * stream and replays the captured graph for later sweeps of the same shape (flags, whether the
 * state must be rebuilt first, number of active slots).  Results are identical to eager
 * sweeps.  Needs a stream created by the caller (not stream 0); per-phase timing
 * (hq_set_timing) runs sweeps eagerly.  Errors: HQ_EINVAL for a null engine or stream 0. */
int hq_set_graphs(hq_engine* e, int enable);
int hq_get_timing(hq_engine* e, double* ms, int64_t* launches);

/* log|det M| of every chain's fields, with no device allocation of any kind.
 *
 * The paper has no counterpart: this is a service of this library.  It is for callers that
 * cannot allocate device memory themselves -- code that only receives buffers from a host
 * framework whose own memory pool owns the device (and forbids cudaMalloc/cudaFree next
 * to it), or code that must not allocate once it is running, such as a latency-bound
 * serving loop.  Such a caller passes only its inputs and outputs:
 *   p          model and run shape (as for hq_create; delay_k is not used but must still be
 *              valid, 1..32),
 *   n_chains   number of chains, >= 1,
 *   X_device   device pointer, fields X[chain][l][i] (n_chains * L * N doubles, read only),
 *   logdet_device  device pointer, n_chains doubles written with log|det(I + B_L..B_1)|,
 *   stream     cudaStream_t (NULL = legacy default stream); the call is asynchronous.
 * The kernel builds the kinetic factors exp(-+dtau K) in shared memory from their closed form,
 * so the call reads no host memory.  Its scratch (7 N x N FP64 matrices per chain) comes from a
 * file-scope static device array of HQ_NOALLOC_SCRATCH_BYTES = 64 MiB, which every GPU that
 * loads the library holds until the process exits.  Calls needing more (more than 292 chains of
 * N = 64, or 18 of N = 256) are rejected with HQ_ENOMEM and a message in hq_last_error(NULL);
 * invalid parameters give HQ_EINVAL.  The first call on a device looks up the array's device
 * address once for that device; make that first call before any stream capture.  Every call
 * shares the one array, so calls that overlap on the GPU (other streams, other host threads)
 * race on it: serialise them.  Non-finite results show up as NaN/Inf in logdet_device.  The
 * result equals hq_log_weight's log|det M| for the same fields. */
#define HQ_NOALLOC_SCRATCH_BYTES (64u << 20)
int hq_logdet_noalloc(const hq_params* p, int n_chains, const double* X_device, double* logdet_device,
                      void* stream);

/* ------------------------------------------------------------------------------------
 * Learned effective action and cumulative (network-driven) moves.
 *
 * Paper, "Local Updates" and the cumulative update of the benchmark section: a network
 * trained on configurations of the conventional sampler drives many moves, and the whole
 * proposal X -> X' is then accepted with min(1, p_c),
 *   p_c = [W(X')/W(X)] [exp(-beta E_NN[X]) / exp(-beta E_NN[X'])],
 * so the chain samples the exact weight.  Here E_NN is the scalar
 *   F(X) = sum_{i,l} f(patch_{i,l}(X)),  patch = X on the 5-site cross x 5 slices around
 *   (i, l) minus the mean field -g/(M Omega^2),  f: 25 -> 64 -> 64 -> 1, ReLU, linear out,
 * with bfloat16 weights and FP32 arithmetic.  Local moves are Metropolis moves on
 * exp(-dtau S_ph + 2F) with the exact phonon action; block moves on the same weight, or
 * (HQ_CNN_BLOCK) with the convolutional action F_cnn below in place of F.  Every move is
 * reversible for its own weight, so the cumulative accept is
 *   p_c = exp(2 [log|det M(X')| - log|det M(X)|] - 2 sum over accepted inner moves of dF)
 * (the phonon action cancels; with one network the sum is F(X') - F(X)).
 * Parameters are a flat float vector: W1[25][64] (input k, unit u at k*64+u), b1[64],
 * W2[64][64] (v*64+u), b2[64], W3[64], b3.  Inputs are ordered (slice offset -2..2) x
 * (cross site: centre, +x, -x, +y, -y).  Requires nx, ny >= 4 and L >= 5.
 * Random numbers: Philox tags 2 (inner local, event l*N+i), 3 (inner block, event i) with
 * counter word 1 = step * n_inner + inner sweep, and 4 (cumulative accept, event 0, word 1 =
 * step, u = the first uniform).
 * ------------------------------------------------------------------------------------ */
#define HQ_NN_PARAMS 5889

typedef struct hq_learned_stats {   /* per chain, since the network state was attached */
  int64_t inner_local_proposed, inner_local_accepted;
  int64_t inner_block_proposed, inner_block_accepted;
  int64_t cumulative_proposed, cumulative_accepted;
  double last_pc;                    /* p_c of the last cumulative step */
} hq_learned_stats;

/* Device bytes of the network state for training minibatches of up to max_batch samples out
 * of sets of up to max_samples (0 if the engine's lattice is too small for the patches). */
size_t hq_nn_arena_bytes(const hq_engine* e, int max_batch, int max_samples);
/* Attach a caller-owned, 256-byte aligned device arena of hq_nn_arena_bytes() bytes. */
int hq_nn_attach(hq_engine* e, void* device_arena, size_t bytes, int max_batch, int max_samples);
/* Set the parameters from HQ_NN_PARAMS host floats (rounded to bfloat16 for use; the FP32
 * values are kept as the training master copy; the optimiser state is reset). */
int hq_nn_set_params(hq_engine* e, const float* theta_host);
/* FP32 master parameters, or with bf16 != 0 the bfloat16 values the kernels use. */
int hq_nn_get_params(hq_engine* e, float* theta_host, int bf16);
/* F(X) of every chain's current fields (host, n_chains doubles).  Synchronises.  Paper,
 * "Local Updates": the network's effective action on local space-time patches of X. */
int hq_nn_eval(hq_engine* e, double* F_host);
/* Paper, "Global Updates" (training of both networks): fit to (X, exact log-weight) pairs
 * from the plain sampler.
 * Adam training (lr, beta1 0.9, beta2 0.999) of F towards targets y on samples X:
 * X_device [n_samples][L][N] doubles and y_device [n_samples] doubles, device pointers of the
 * engine's lattice; loss (1/B) sum (F(X_a) - y_a)^2 per minibatch of `batch` samples; epoch
 * order from `seed`.  loss_host (optional): mean loss of each epoch.  Synchronises. */
int hq_nn_train(hq_engine* e, const double* X_device, const double* y_device, int n_samples, int epochs,
                int batch, float lr, uint64_t seed, double* loss_host);
/* Gradient of (1/n) sum_a (F(X_a) - y_a)^2 over all n_samples (<= max_batch), no update:
 * grad_host HQ_NN_PARAMS floats, loss_host one double.  Synchronises. */
int hq_nn_gradient(hq_engine* e, const double* X_device, const double* y_device, int n_samples, float* grad_host,
                   double* loss_host);
/* Paper, "Benchmarks": the cumulative update, accepted with p_c = [W(X')/W(X)] times the
 * ratio of the network weights, so the chain samples the exact weight.
 * n_steps cumulative steps of every chain: n_inner network-driven sweeps (flags HQ_LOCAL:
 * a local move at every (l, i); HQ_GLOBAL: a block move at every site, with HQ_CNN_BLOCK on
 * F_cnn), then the exact accept of the cumulative move; HQ_MEASURE also records electronic
 * observables of G_0 after each step (G_0 of the starting fields is kept, so a rejected chain
 * needs no second stabilised determinant).  Asynchronous.
 * Errors: HQ_EINVAL for bad arguments, HQ_CNN_BLOCK without convolutional parameters, or no
 * attached network state. */
int hq_cumulative_sweep(hq_engine* e, int n_steps, int n_inner, unsigned flags);
int hq_get_learned_stats(hq_engine* e, hq_learned_stats* out);
/* Size of a cumulative proposal: with slices > 0 (and < L) the local moves of each inner sweep
 * visit only `slices` consecutive slices, l0, l0 + 1, ... (mod L), with l0 = floor(u L) from
 * event 1 of the step's tag-4 Philox block (first uniform); block moves are unchanged (turn
 * them off with the flags).  Fewer moves per proposal mean a smaller accumulated network error
 * and a higher cumulative acceptance at the same exact-weight cost per step.  0 (default) or
 * slices >= L: every slice.  Errors: HQ_EINVAL for a null engine or slices < 0. */
int hq_set_inner_window(hq_engine* e, int slices);
/* How a cumulative step computes the exact log|det M(X')| (no counterpart in the paper, which
 * gives no implementation): mode 1, one CTA per chain builds the whole stabilised product (the
 * stack build; measured steps record the observables of G_0); mode 2, two CTAs per chain build
 * the slices above and below a restabilisation boundary m near L/2 at the same time, and a
 * second launch joins the halves with the two-sided formula of the local sweep's
 * restabilisation (measured steps record the observables of G_m, an equally valid equal-time
 * estimator); mode 0 (default) takes mode 2 when two CTAs per chain fit the device's SMs
 * (2 n_chains <= SMs) and the product has at least two chunks, else mode 1.  Both give the same
 * log|det M| up to rounding.  Returns the boundary m in use (0 for mode 1) or a negative error:
 * HQ_EINVAL for a null engine, a mode outside 0..2, or mode 2 with fewer than two chunks. */
int hq_set_logdet_split(hq_engine* e, int mode);
/* The same for block moves: with sites > 0 (and < N) each inner sweep's block moves visit only
 * `sites` consecutive sites j0, j0 + 1, ... (mod N, site index order), j0 = floor(u N) with u
 * the second uniform of event 1 of the step's tag-4 block.  0 (default) or sites >= N: every
 * site.  Errors: HQ_EINVAL for a null engine or sites < 0. */
int hq_set_inner_sites(hq_engine* e, int sites);

/* ------------------------------------------------------------------------------------
 * Convolutional action for block moves (paper, "Global Updates": a convolutional network on
 * the whole field predicts the weight, so a move of a whole imaginary-time column is cheap
 * to estimate).  F_cnn(X) = sum over the (x, y, tau) torus of three 3x3x3 cross-correlations
 * with periodic padding, 1 -> 16 -> 16 -> 1 channels, ReLU after the first two, on
 * z = X + g/(M Omega^2); tap t = 9 (dl + 1) + 3 (dy + 1) + (dx + 1) reads (l + dl, y + dy,
 * x + dx).  Parameters, one flat float vector: W1[27][16] (tap, out), b1[16],
 * W2[27][16][16] (tap, in, out), b2[16], W3[27][16] (tap, in), b3; bfloat16 weights, FP32
 * arithmetic.  Its state lives in the hq_nn_attach arena (activations of every chain's
 * current fields, 33 floats per point).  A block move's change of F_cnn is computed from the
 * cached activations in the window of lattice distance <= 3 around the moved site.
 * ------------------------------------------------------------------------------------ */
#define HQ_CNN_PARAMS 7809
#define HQ_CNN_BLOCK 8u   /* hq_cumulative_sweep flag: block moves use F_cnn */

/* Set the convolutional parameters from HQ_CNN_PARAMS host floats (bfloat16 for use, FP32
 * master copy kept, optimiser state reset); enables HQ_CNN_BLOCK.  Synchronises.
 * Errors: HQ_EINVAL without an attached network state or with a null pointer. */
int hq_cnn_set_params(hq_engine* e, const float* theta_host);
/* FP32 master parameters, or with bf16 != 0 the bfloat16 values the kernels use. */
int hq_cnn_get_params(hq_engine* e, float* theta_host, int bf16);
/* F_cnn of every chain's current fields (host, n_chains doubles); refreshes the cached
 * activations.  Synchronises.  Paper, "Global Updates": the convolutional network on the
 * (x, y, tau) field that drives block moves. */
int hq_cnn_eval(hq_engine* e, double* F_host);
/* Training and gradient of F_cnn, with the arguments and semantics of hq_nn_train and
 * hq_nn_gradient (targets y, minibatch loss (1/B) sum (F_cnn(X_a) - y_a)^2, Adam). */
int hq_cnn_train(hq_engine* e, const double* X_device, const double* y_device, int n_samples, int epochs,
                 int batch, float lr, uint64_t seed, double* loss_host);
int hq_cnn_gradient(hq_engine* e, const double* X_device, const double* y_device, int n_samples, float* grad_host,
                    double* loss_host);

/* Failure-detection probe (no counterpart in the paper).  Every device-side wait of the
 * library (a block-move task waiting for its chain's previous step) is bounded: after its
 * limit it gives up, marks the chains HQ_ETIMEOUT and the kernel returns, so a stuck phase
 * leaves a usable context.  This entry point runs that same wait on a device flag that nothing
 * sets, with a limit of limit_seconds (0 < limit <= 2), on the stream, synchronises, and writes
 * the kernel's result to *status_out: HQ_ETIMEOUT when the wait ran out (the expected
 * result).  Returns HQ_OK, HQ_EINVAL for a bad limit or pointer, HQ_ECUDA on a CUDA error. */
int hq_wait_probe(double limit_seconds, void* stream, int* status_out);

/* Per-section device cycle counters (profiling builds compiled with -DHQ_SECTION_TIMING):
 * copies up to n counters (sum over CTAs of thread 0's clock64 spans; ids in
 * csrc/hq_device.cuh) to out and clears them.  Returns the number copied; 0 in normal
 * builds. */
int hq_get_section_cycles(uint64_t* out, int n);

/* FP64 pipe probe: runs a throughput kernel on the stream (reps launches of about 10 ms)
 * and returns achieved TFLOP/s, or <= 0 on error.  kind 0: DFMA (fma on doubles, the
 * engine's arithmetic); kind 1: DMMA (mma.sync m8n8k4 f64, the FP64 tensor path).  Used to
 * state the FP64 roofline; allocates and frees its own small buffer. */
#define HQ_PROBE_DFMA 0
#define HQ_PROBE_DMMA 1
double hq_fp64_peak_tflops(int kind, int reps, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HOLSTEIN_DQMC_H */
