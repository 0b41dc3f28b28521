// Host side of the C ABI (include/holstein_dqmc.h): parameter validation, arena layout,
// kinetic propagators, the sweep schedule, copies in and out, checkpoints, tau_int.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hq_internal.h"
#include "../../include/holstein_dqmc.h"

struct hq_engine {
  void set_act(int slot, int v) {
    act[slot] = v;
    int n = 0;
    for (int a : act) n += a ? 1 : 0;
    d.n_active = n;
  }
  hq_params p;
  hq::Dev d;
  cudaStream_t stream;
  char* arena;
  size_t arena_bytes;
  double* tmp;          // [C] device scratch inside the arena
  int series_len;       // per-sweep records kept so far (<= max_series)
  long long sweeps;     // sweeps run (Philox sweep counter)
  bool stack_valid;     // left stack, G_0 and log|det M| match the fields
  bool logdet_valid;    // log|det M| matches the fields
  bool green_valid;     // G holds G_l of the fields, l = green_slice
  int green_slice = 0;  // 0 (G_0, after a stack build or a local phase) or the split boundary
  int split_mode = 0;   // learned steps' log|det M|: 0 automatic, 1 one CTA per chain, 2 two halves
  int split_auto = 0;   // automatic choice: two halves when 2 chains fit the device's SMs
  std::vector<int> act;  // host mirror of the active flags
  std::string err;
  // optional per-phase timing
  struct Span { cudaEvent_t a, b; int phase, launches; };
  bool timing = false;
  // optional CUDA-graph replay of whole sweeps (key: flags, stack build needed, active slots)
  bool graphs = false;
  cudaGraphExec_t gexec = nullptr;
  long long gkey = -1, gwarm = -1;
  std::vector<Span> spans;
  std::vector<cudaEvent_t> spare;
  double phase_ms[HQ_N_PHASES] = {};
  long long phase_launches[HQ_N_PHASES] = {};
  // learned effective action (optional)
  bool nn_on = false;
  hq::NNState nn{};
  hq::CnnState cn{};
  int nn_max_batch = 0, nn_max_samples = 0;
  int cn_t_step = 0;
  int nn_window = 0;  // local moves of a cumulative step on this many slices (0: all)
  int nn_site_window = 0;  // block moves of a cumulative step on this many sites (0: all)
  long long cum_steps = 0;
  int nn_t_step = 0;
  int backoffs = 0;  // stabilisation back-offs (n_wrap halvings) so far
  ~hq_engine() {
    for (auto& s : spans) { cudaEventDestroy(s.a); cudaEventDestroy(s.b); }
    for (auto ev : spare) cudaEventDestroy(ev);
    if (gexec) cudaGraphExecDestroy(gexec);
  }
};

namespace {

constexpr size_t kAlign = 256;
thread_local std::string g_call_error;  // message of the last failing call without an engine

struct Layout {
  size_t kin, X, G, logdet, UR, TR, DR, work, stU, stT, stD, Adl, Bdl, acc, tot, series, counters, status, sched, tmp,
      expV, cmat, cbuf, corr, cid, active, slen, flag;
  size_t total;
};

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int n_slices(const hq_params& p) { return (int)std::llround(p.beta / p.dtau); }

const char* validate(const hq_params* p, int n_chains, int max_series) {
  if (!p) return "params is NULL";
  if (p->nx < 2 || p->ny < 2 || p->nx > hq::kMaxSide || p->ny > hq::kMaxSide) return "nx, ny must be in 2..16";
  if ((p->nx & 1) || (p->ny & 1)) return "nx and ny must be even (bipartite lattice)";
  if (!(p->dtau > 0.0) || !(p->beta > 0.0)) return "beta and dtau must be positive";
  const double Lf = p->beta / p->dtau;
  const long long L = std::llround(Lf);
  if (std::fabs(Lf - (double)L) > 1e-9 * std::fmax(1.0, Lf)) return "beta/dtau must be an integer";
  if (L < 2 || L > 100000) return "L = beta/dtau must be in 2..100000";
  if (p->n_wrap < 1) return "n_wrap must be >= 1";
  if (p->delay_k < 1 || p->delay_k > hq::kMaxK) return "delay_k must be in 1..32";
  if (!(p->mass > 0.0) || !(p->omega > 0.0)) return "mass and omega must be positive";
  if (!std::isfinite(p->t) || !std::isfinite(p->mu) || !std::isfinite(p->g)) return "t, mu, g must be finite";
  if (!(p->dx_local >= 0.0) || !(p->dx_global >= 0.0)) return "proposal widths must be >= 0";
  if (n_chains < 1) return "n_chains must be >= 1";
  if (max_series < 0) return "max_series must be >= 0";
  if (p->block_method < 0 || p->block_method > 2) return "block_method must be 0, 1 or 2";
  if (!(p->wrap_tol >= 0.0) || !std::isfinite(p->wrap_tol)) return "wrap_tol must be finite and >= 0";
  if (p->n_wrap_min < 0 || p->n_wrap_min > p->n_wrap) return "n_wrap_min must be in 0..n_wrap";
  return nullptr;
}

// Smallest restabilisation interval the engine can reach (the arena is sized for it).
int n_wrap_floor(const hq_params& p) {
  if (!(p.wrap_tol > 0.0)) return p.n_wrap;
  return p.n_wrap_min > 0 ? p.n_wrap_min : 1;
}

// chunk propagators for block moves: forced by block_method, else by the flop model
bool use_chunks(const hq_params& p) {
  if (p.block_method == 1) return false;
  if (p.block_method == 2) return true;
  return hq::chunk_propagators_pay(p.nx, p.ny, (int)n_slices(p), p.n_wrap);
}

Layout layout(const hq_params& p, int C, int max_series) {
  Layout l{};
  const size_t n = (size_t)p.nx * p.ny, L = (size_t)n_slices(p), nn = n * n;
  const size_t nb = (L - 1) / (size_t)n_wrap_floor(p);  // stack boundaries at the smallest n_wrap
  const size_t k = (size_t)p.delay_k;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes); return o; };
  l.kin = take(sizeof(double) * (2 * p.nx * p.nx + 2 * p.ny * p.ny));
  l.X = take(sizeof(double) * C * L * n);
  l.G = take(sizeof(double) * C * nn);
  l.logdet = take(sizeof(double) * C);
  l.UR = take(sizeof(double) * C * nn);
  l.TR = take(sizeof(double) * C * nn);
  l.DR = take(sizeof(double) * C * n);
  l.work = take(sizeof(double) * C * hq::kWorkMats * nn);
  l.stU = take(sizeof(double) * C * nb * nn);
  l.stT = take(sizeof(double) * C * nb * nn);
  l.stD = take(sizeof(double) * C * nb * n);
  l.Adl = take(sizeof(double) * C * k * n);
  l.Bdl = take(sizeof(double) * C * k * n);
  l.acc = take(sizeof(double) * C * hq::kAccSlots);
  l.tot = take(sizeof(double) * C * hq::kTotSlots);
  l.series = take(sizeof(double) * C * HQ_N_OBS * (size_t)(max_series > 0 ? max_series : 1));
  l.counters = take(sizeof(long long) * C * hq::kCounters);
  l.status = take(sizeof(int) * C);
  l.sched = take(sizeof(int) * (hq::kSchedHeader + C));
  l.tmp = take(sizeof(double) * C);
  l.cid = take(sizeof(uint32_t) * 4 * C);
  l.active = take(sizeof(int) * C);
  l.slen = take(sizeof(int) * C);
  l.flag = take(sizeof(int));
  if (use_chunks(p)) {
    const size_t nch = (L + n_wrap_floor(p) - 1) / n_wrap_floor(p);
    l.expV = take(sizeof(double) * C * L * n);
    l.cmat = take(sizeof(double) * C * 2 * nch * nn);
    l.cbuf = take(sizeof(int) * C);
    l.corr = take(sizeof(double) * C * (2 * n * L + L));
  }
  l.total = off;
  return l;
}

// exp(-sgn dtau K_ring) for a ring of m sites with K_ab = -t per displacement +-1:
// eigenvalues -2t cos(2 pi q/m) on plane waves, so
// E_ab = (1/m) sum_q cos(2 pi q (a-b)/m) exp(sgn 2 t dtau cos(2 pi q/m)).
void ring_propagator(int m, double t, double dtau, double sgn, double* E) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      double s = 0.0;
      for (int q = 0; q < m; ++q)
        s += std::cos(two_pi * q * (a - b) / m) * std::exp(sgn * 2.0 * t * dtau * std::cos(two_pi * q / m));
      E[a * m + b] = s / m;
    }
}

int set_err(hq_engine* e, int code, const std::string& msg) {
  if (e) e->err = msg;
  return code;
}

int cuda_check(hq_engine* e, cudaError_t st, const char* what) {
  if (st == cudaSuccess) return HQ_OK;
  return set_err(e, HQ_ECUDA, std::string(what) + ": " + cudaGetErrorString(st));
}

cudaEvent_t take_event(hq_engine* e) {
  if (!e->spare.empty()) {
    cudaEvent_t ev = e->spare.back();
    e->spare.pop_back();
    return ev;
  }
  cudaEvent_t ev = nullptr;
  if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
  return ev;
}

// Brackets a launch group with events when timing is enabled.
struct PhaseTimer {
  hq_engine* e;
  hq_engine::Span span{};
  bool on = false;
  PhaseTimer(hq_engine* eng, int phase, int launches) : e(eng) {
    if (!e->timing) return;
    span.a = take_event(e);
    span.b = take_event(e);
    span.phase = phase;
    span.launches = launches;
    on = span.a && span.b && cudaEventRecord(span.a, e->stream) == cudaSuccess;
  }
  ~PhaseTimer() {
    if (on && cudaEventRecord(span.b, e->stream) == cudaSuccess) e->spans.push_back(span);
  }
};

int ensure_state(hq_engine* e) {
  if (e->stack_valid) return HQ_OK;
  PhaseTimer pt(e, 0, 1);
  int rc = cuda_check(e, hq::launch_stack_build(e->d, e->stream), "stack_build launch");
  if (rc) return rc;
  e->stack_valid = e->logdet_valid = e->green_valid = true;
  e->green_slice = 0;
  return HQ_OK;
}

// Split boundary used by the learned steps' exact log|det M| (0: one CTA per chain).
int split_in_use(const hq_engine* e) {
  const bool on = e->split_mode == 2 || (e->split_mode == 0 && e->split_auto);
  return on ? hq::split_point(e->d) : 0;
}

// log|det M| and G_m of the current fields by the two-half build (the left stack is not
// rebuilt: it stays invalid).
int split_state(hq_engine* e, int m) {
  int rc;
  {
    PhaseTimer pt(e, 4, 1);
    rc = cuda_check(e, hq::launch_split_logdet(e->d, m, 0, e->stream), "split halves launch");
  }
  if (rc) return rc;
  {
    PhaseTimer pt(e, 5, 1);
    rc = cuda_check(e, hq::launch_split_logdet(e->d, m, 1, e->stream), "split join launch");
  }
  if (rc) return rc;
  e->stack_valid = false;
  e->logdet_valid = e->green_valid = true;
  e->green_slice = m;
  return HQ_OK;
}

}  // namespace

extern "C" {

size_t hq_arena_bytes(const hq_params* p, int n_chains, int max_series) {
  if (validate(p, n_chains, max_series)) return 0;
  return layout(*p, n_chains, max_series).total;
}

int hq_create(const hq_params* p, int n_chains, int first_chain, int max_series, void* device_arena,
              size_t arena_bytes, void* stream, hq_engine** out) {
  if (!out) return HQ_EINVAL;
  *out = nullptr;
  if (const char* why = validate(p, n_chains, max_series)) {
    std::fprintf(stderr, "hq_create: %s\n", why);
    return HQ_EINVAL;
  }
  if (first_chain < 0) return HQ_EINVAL;
  const Layout l = layout(*p, n_chains, max_series);
  if (!device_arena || arena_bytes < l.total || ((uintptr_t)device_arena % kAlign) != 0) return HQ_ENOMEM;
  hq_engine* e = new (std::nothrow) hq_engine();
  if (!e) return HQ_ENOMEM;
  e->p = *p;
  e->stream = (cudaStream_t)stream;
  e->arena = (char*)device_arena;
  e->arena_bytes = arena_bytes;
  hq::Dev& d = e->d;
  d.nx = p->nx;
  d.ny = p->ny;
  d.n = p->nx * p->ny;
  d.L = n_slices(*p);
  d.n_wrap = p->n_wrap;
  d.k = p->delay_k;
  d.n_chains = n_chains;
  d.first_chain = first_chain;
  d.n_bound = (d.L - 1) / d.n_wrap;
  d.max_series = max_series;
  d.t = p->t;
  d.mu = p->mu;
  d.omega = p->omega;
  d.mass = p->mass;
  d.g = p->g;
  d.dtau = p->dtau;
  d.dx_local = p->dx_local;
  d.dx_global = p->dx_global;
  d.key0 = (uint32_t)(p->seed & 0xffffffffu);
  d.key1 = (uint32_t)(p->seed >> 32);
  char* a = e->arena;
  d.kin = (const double*)(a + l.kin);
  d.X = (double*)(a + l.X);
  d.G = (double*)(a + l.G);
  d.logdet = (double*)(a + l.logdet);
  d.UR = (double*)(a + l.UR);
  d.TR = (double*)(a + l.TR);
  d.DR = (double*)(a + l.DR);
  d.work = (double*)(a + l.work);
  d.stU = (double*)(a + l.stU);
  d.stT = (double*)(a + l.stT);
  d.stD = (double*)(a + l.stD);
  d.Adl = (double*)(a + l.Adl);
  d.Bdl = (double*)(a + l.Bdl);
  d.acc = (double*)(a + l.acc);
  d.tot = (double*)(a + l.tot);
  d.series = (double*)(a + l.series);
  d.counters = (long long*)(a + l.counters);
  d.status = (int*)(a + l.status);
  d.sched = (int*)(a + l.sched);
  d.cid = (uint32_t*)(a + l.cid);
  d.active = (int*)(a + l.active);
  d.slen = (int*)(a + l.slen);
  d.wrap_flag = (int*)(a + l.flag);
  d.wrap_tol = p->wrap_tol;
  d.n_wrap_min = n_wrap_floor(*p);
  d.use_cm = use_chunks(*p) ? 1 : 0;
  d.n_chunks = (d.L + d.n_wrap - 1) / d.n_wrap;
  if (d.use_cm) {
    d.expV = (double*)(a + l.expV);
    d.cmat = (double*)(a + l.cmat);
    d.cbuf = (int*)(a + l.cbuf);
    d.corr = (double*)(a + l.corr);
  }
  e->tmp = (double*)(a + l.tmp);

  // kinetic propagators: exp(-dtau K) = E_x (x) E_y with ring factors
  std::vector<double> kin(2 * d.nx * d.nx + 2 * d.ny * d.ny);
  double* kx = kin.data();
  ring_propagator(d.nx, p->t, p->dtau, +1.0, kx);                              // exp(-dtau K_x)
  ring_propagator(d.nx, p->t, p->dtau, -1.0, kx + d.nx * d.nx);                // exp(+dtau K_x)
  ring_propagator(d.ny, p->t, p->dtau, +1.0, kx + 2 * d.nx * d.nx);            // exp(-dtau K_y)
  ring_propagator(d.ny, p->t, p->dtau, -1.0, kx + 2 * d.nx * d.nx + d.ny * d.ny);
  int rc = HQ_OK;
  rc = rc ? rc : cuda_check(e, cudaMemsetAsync(a, 0, l.total, e->stream), "arena clear");
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync((void*)d.kin, kin.data(), kin.size() * sizeof(double),
                                               cudaMemcpyHostToDevice, e->stream), "kinetic upload");
  // per-chain identity: key = seed, chain word = first_chain + c, counter 0; all active
  rc = rc ? rc : cuda_check(e, hq::launch_slot_control(d, -1, d.key0, d.key1, (uint32_t)first_chain, 0u, 1, 1,
                                                       e->stream), "chain ids");
  e->act.assign((size_t)n_chains, 1);
  e->d.n_active = n_chains;
  rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "create sync");
  if (rc) {
    std::fprintf(stderr, "hq_create: %s\n", e->err.c_str());
    delete e;
    return rc;
  }
  e->series_len = 0;
  e->sweeps = 0;
  e->stack_valid = e->logdet_valid = e->green_valid = false;
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      e->split_auto = (2 * n_chains <= sms && hq::split_point(d) > 0) ? 1 : 0;
  }
  *out = e;
  return HQ_OK;
}

void hq_destroy(hq_engine* e) { delete e; }

const char* hq_last_error(const hq_engine* e) { return e ? e->err.c_str() : g_call_error.c_str(); }

int hq_block_move_method(const hq_engine* e) { return e ? e->d.use_cm : HQ_EINVAL; }

int hq_shape(const hq_engine* e, int* n_chains, int* n_sites, int* n_slices_out, int64_t* sweeps) {
  if (!e) return HQ_EINVAL;
  if (n_chains) *n_chains = e->d.n_chains;
  if (n_sites) *n_sites = e->d.n;
  if (n_slices_out) *n_slices_out = e->d.L;
  if (sweeps) *sweeps = e->sweeps;
  return HQ_OK;
}

static size_t field_bytes(const hq_engine* e) { return sizeof(double) * (size_t)e->d.n_chains * e->d.L * e->d.n; }

int hq_set_fields(hq_engine* e, const double* X_host) {
  if (!e || !X_host) return HQ_EINVAL;
  int rc = cuda_check(e, cudaMemcpyAsync(e->d.X, X_host, field_bytes(e), cudaMemcpyHostToDevice, e->stream),
                      "set_fields copy");
  e->stack_valid = e->logdet_valid = e->green_valid = false;
  return rc;
}

int hq_set_fields_device(hq_engine* e, const double* X_device) {
  if (!e || !X_device) return HQ_EINVAL;
  int rc = cuda_check(e, cudaMemcpyAsync(e->d.X, X_device, field_bytes(e), cudaMemcpyDeviceToDevice, e->stream),
                      "set_fields_device copy");
  e->stack_valid = e->logdet_valid = e->green_valid = false;
  return rc;
}

int hq_get_fields(hq_engine* e, double* X_host) {
  if (!e || !X_host) return HQ_EINVAL;
  int rc = cuda_check(e, cudaMemcpyAsync(X_host, e->d.X, field_bytes(e), cudaMemcpyDeviceToHost, e->stream),
                      "get_fields copy");
  return rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "get_fields sync");
}

namespace {
// One sweep: launches on the engine's stream and the host-side state changes.
int sweep_once(hq_engine* e, unsigned flags) {
  const bool do_local = flags & HQ_LOCAL, do_global = flags & HQ_GLOBAL, meas = flags & HQ_MEASURE;
  const hq::Dev& d = e->d;
  int rc = HQ_OK;
  if (do_local || !e->logdet_valid) rc = ensure_state(e);
  if (rc) return rc;
  if (do_local) {
    PhaseTimer pt(e, 1, 1);
    rc = cuda_check(e, hq::launch_local_phase(d, meas ? 1 : 0, e->stream), "local_phase launch");
    if (rc) return rc;
    e->stack_valid = false;  // fields changed; G_0 and log|det M| are fresh (restabilised at l = L)
    e->logdet_valid = e->green_valid = true;
    e->green_slice = 0;
  }
  if (do_global) {
    PhaseTimer pt(e, 2, 1);
    rc = cuda_check(e, hq::launch_global_phase(d, e->stream), "global_phase launch");
    if (rc) return rc;
    e->stack_valid = false;
    e->green_valid = false;  // log|det M| is kept current by the accepted moves
  }
  {
    PhaseTimer pt(e, 3, 1);
    rc = cuda_check(e, hq::launch_sweep_end(d, (meas && do_local) ? 1 : 0, e->stream), "sweep_end launch");
  }
  if (rc) return rc;
  e->sweeps++;
  return HQ_OK;
}

// The host-side state changes of sweep_once without its launches (graph replay).
void sweep_state(hq_engine* e, unsigned flags) {
  if ((flags & HQ_LOCAL) || !e->logdet_valid) {
    if (!e->stack_valid) {
      e->stack_valid = e->logdet_valid = e->green_valid = true;
      e->green_slice = 0;
    }
  }
  if (flags & HQ_LOCAL) {
    e->stack_valid = false;
    e->logdet_valid = e->green_valid = true;
    e->green_slice = 0;
  }
  if (flags & HQ_GLOBAL) e->stack_valid = e->green_valid = false;
  e->sweeps++;
}

void drop_graph(hq_engine* e) {
  if (e->gexec) cudaGraphExecDestroy(e->gexec);
  e->gexec = nullptr;
  e->gkey = e->gwarm = -1;
}
}  // namespace

namespace {
// Stabilisation back-off after a sweep with local moves (wrap_tol > 0): read the flag the
// sweep-end kernel sets when a chain's largest wrap error exceeded wrap_tol; halve n_wrap for
// the engine if it is above the floor (the restabilisation boundaries, the stack and the chunk
// propagators follow from n_wrap and are rebuilt), else report HQ_EUNSTABLE.
int wrap_backoff(hq_engine* e, bool* unstable) {
  int flag = 0;
  int rc = cuda_check(e, cudaMemcpyAsync(&flag, e->d.wrap_flag, sizeof(int), cudaMemcpyDeviceToHost, e->stream),
                      "wrap flag copy");
  rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "wrap flag sync");
  if (rc || !flag) return rc;
  rc = cuda_check(e, cudaMemsetAsync(e->d.wrap_flag, 0, sizeof(int), e->stream), "wrap flag clear");
  if (rc) return rc;
  hq::Dev& d = e->d;
  if (d.n_wrap <= d.n_wrap_min) {
    *unstable = true;
    return HQ_OK;
  }
  d.n_wrap = std::max(d.n_wrap_min, d.n_wrap / 2);
  d.n_bound = (d.L - 1) / d.n_wrap;
  d.n_chunks = (d.L + d.n_wrap - 1) / d.n_wrap;
  e->backoffs++;
  e->stack_valid = e->green_valid = false;  // log|det M| does not depend on n_wrap
  drop_graph(e);
  return HQ_OK;
}
}  // namespace

int hq_sweep(hq_engine* e, int n_sweeps, unsigned flags) {
  if (!e || n_sweeps < 0 || (flags & ~(HQ_LOCAL | HQ_GLOBAL | HQ_MEASURE))) return HQ_EINVAL;
  if (e->d.wrap_tol > 0.0 && (flags & HQ_LOCAL)) {
    // one sweep at a time, each followed by the back-off check
    bool unstable = false;
    for (int it = 0; it < n_sweeps; ++it) {
      int rc = sweep_once(e, flags);
      rc = rc ? rc : wrap_backoff(e, &unstable);
      if (rc) return rc;
    }
    if (unstable)
      return set_err(e, HQ_EUNSTABLE, "wrap error above wrap_tol at the smallest n_wrap (" +
                                          std::to_string(e->d.n_wrap) + "); chains with status HQ_EUNSTABLE");
    return HQ_OK;
  }
  for (int it = 0; it < n_sweeps; ++it) {
    if (!e->graphs || e->timing) {
      const int rc = sweep_once(e, flags);
      if (rc) return rc;
      continue;
    }
    // graph replay: the launches of one sweep depend on the flags, on whether the state must
    // be rebuilt first and on the number of active slots (the block-move grid)
    const bool stack = ((flags & HQ_LOCAL) || !e->logdet_valid) && !e->stack_valid;
    const long long key = ((long long)e->d.n_active << 8) | ((long long)flags << 1) | (stack ? 1 : 0);
    if (e->gexec && e->gkey == key) {
      int rc = cuda_check(e, cudaGraphLaunch(e->gexec, e->stream), "graph launch");
      if (rc) return rc;
      sweep_state(e, flags);
      continue;
    }
    if (e->gwarm != key) {
      // first sweep of this shape runs eagerly (it also sets the kernels' attributes)
      const int rc = sweep_once(e, flags);
      if (rc) return rc;
      e->gwarm = key;
      continue;
    }
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    e->gexec = nullptr;
    cudaGraph_t graph = nullptr;
    int rc = cuda_check(e, cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (rc) return rc;
    const int rcs = sweep_once(e, flags);  // records the launches and applies the state changes
    rc = cuda_check(e, cudaStreamEndCapture(e->stream, &graph), "end capture");
    if (rcs) {
      if (graph) cudaGraphDestroy(graph);
      return rcs;
    }
    if (rc) return rc;
    rc = cuda_check(e, cudaGraphInstantiate(&e->gexec, graph, 0), "graph instantiate");
    cudaGraphDestroy(graph);
    if (rc) {
      e->gexec = nullptr;
      return rc;
    }
    e->gkey = key;
    rc = cuda_check(e, cudaGraphLaunch(e->gexec, e->stream), "graph launch");
    if (rc) return rc;
  }
  return HQ_OK;
}

int hq_set_graphs(hq_engine* e, int enable) {
  if (!e) return HQ_EINVAL;
  if (enable && e->stream == nullptr) return set_err(e, HQ_EINVAL, "graph replay needs a created stream, not stream 0");
  drop_graph(e);
  e->graphs = enable != 0;
  return HQ_OK;
}

int hq_log_weight(hq_engine* e, double* logw_host, double* logdet_host) {
  if (!e) return HQ_EINVAL;
  int rc = e->logdet_valid ? HQ_OK : ensure_state(e);
  if (rc) return rc;
  const size_t C = (size_t)e->d.n_chains;
  rc = cuda_check(e, hq::launch_log_weight(e->d, e->tmp, e->stream), "log_weight launch");
  if (!rc && logw_host)
    rc = cuda_check(e, cudaMemcpyAsync(logw_host, e->tmp, C * sizeof(double), cudaMemcpyDeviceToHost, e->stream),
                    "log_weight copy");
  if (!rc && logdet_host)
    rc = cuda_check(e, cudaMemcpyAsync(logdet_host, e->d.logdet, C * sizeof(double), cudaMemcpyDeviceToHost,
                                       e->stream), "logdet copy");
  return rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "log_weight sync");
}

int hq_get_green(hq_engine* e, int chain, double* G_host, int* slice) {
  if (!e || !G_host || chain < 0 || chain >= e->d.n_chains) return HQ_EINVAL;
  int rc = HQ_OK;
  if (!e->green_valid || e->green_slice != 0) {
    e->stack_valid = false;
    rc = ensure_state(e);
    if (rc) return rc;
  }
  const size_t n = (size_t)e->d.n;
  std::vector<double> cm(n * n);
  rc = cuda_check(e, cudaMemcpyAsync(cm.data(), e->d.G + (size_t)chain * n * n, n * n * sizeof(double),
                                     cudaMemcpyDeviceToHost, e->stream), "get_green copy");
  rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "get_green sync");
  if (rc) return rc;
  for (size_t i = 0; i < n; ++i)
    for (size_t j = 0; j < n; ++j) G_host[i * n + j] = cm[j * n + i];
  if (slice) *slice = 0;
  return HQ_OK;
}

int hq_get_observables(hq_engine* e, hq_obs* out) {
  if (!e || !out) return HQ_EINVAL;
  const size_t C = (size_t)e->d.n_chains;
  std::vector<double> tot(C * hq::kTotSlots), ld(C);
  std::vector<long long> cnt(C * hq::kCounters);
  std::vector<int> st(C);
  int aborted = 0;
  int rc = e->logdet_valid ? HQ_OK : ensure_state(e);
  if (rc) return rc;
  rc = cuda_check(e, cudaMemcpyAsync(tot.data(), e->d.tot, tot.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                     e->stream), "obs copy");
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(cnt.data(), e->d.counters, cnt.size() * sizeof(long long),
                                               cudaMemcpyDeviceToHost, e->stream), "counter copy");
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(st.data(), e->d.status, st.size() * sizeof(int),
                                               cudaMemcpyDeviceToHost, e->stream), "status copy");
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(ld.data(), e->d.logdet, ld.size() * sizeof(double),
                                               cudaMemcpyDeviceToHost, e->stream), "logdet copy");
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(&aborted, e->d.sched + 1, sizeof(int), cudaMemcpyDeviceToHost,
                                               e->stream), "abort flag copy");
  rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "obs sync");
  if (rc) return rc;
  for (size_t c = 0; c < C; ++c) {
    const double* t = tot.data() + c * hq::kTotSlots;
    const long long* k = cnt.data() + c * hq::kCounters;
    hq_obs o{};
    o.sweeps = (int64_t)t[hq::TOT_SWEEPS];
    o.measured = (int64_t)t[hq::TOT_MEASURED];
    o.local_proposed = k[0];
    o.local_accepted = k[1];
    o.global_proposed = k[2];
    o.global_accepted = k[3];
    const double nm = t[hq::TOT_MEASURED], ns = t[hq::TOT_SWEEPS];
    o.density = nm > 0 ? t[hq::TOT_DENSITY] / nm : NAN;
    o.double_occ = nm > 0 ? t[hq::TOT_DOCC] / nm : NAN;
    o.s_cdw = nm > 0 ? t[hq::TOT_SCDW] / nm : NAN;
    o.x_mean = ns > 0 ? t[hq::TOT_XMEAN] / ns : NAN;
    o.x2 = ns > 0 ? t[hq::TOT_X2] / ns : NAN;
    o.max_wrap_error = t[hq::TOT_WRAP];
    o.logdet = ld[c];
    o.status = aborted ? HQ_ETIMEOUT : st[c];
    o.n_wrap = e->d.n_wrap;
    o.wrap_exceeded = k[4];
    out[c] = o;
  }
  return HQ_OK;
}

int hq_get_series(hq_engine* e, int obs_id, double* out, int* n_out) {
  if (!e || !out || obs_id < 0 || obs_id >= HQ_N_OBS) return HQ_EINVAL;
  const size_t C = (size_t)e->d.n_chains, M = (size_t)e->d.max_series;
  if (n_out) *n_out = 0;
  if (M == 0) return HQ_OK;
  std::vector<double> all(C * HQ_N_OBS * M);
  std::vector<int> len(C);
  int rc = cuda_check(e, cudaMemcpyAsync(all.data(), e->d.series, all.size() * sizeof(double),
                                         cudaMemcpyDeviceToHost, e->stream), "series copy");
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(len.data(), e->d.slen, C * sizeof(int), cudaMemcpyDeviceToHost,
                                               e->stream), "series length copy");
  rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "series sync");
  if (rc) return rc;
  int nmax = 0;
  for (size_t c = 0; c < C; ++c) nmax = len[c] > nmax ? len[c] : nmax;
  for (size_t c = 0; c < C; ++c)
    for (int s = 0; s < nmax; ++s) out[c * M + s] = s < len[c] ? all[(c * HQ_N_OBS + obs_id) * M + s] : NAN;
  if (n_out) *n_out = nmax;
  return HQ_OK;
}

int hq_set_chain(hq_engine* e, int slot, const double* X_host, uint64_t seed, uint32_t chain_id, uint32_t sweep) {
  if (!e || !X_host || slot < 0 || slot >= e->d.n_chains) return HQ_EINVAL;
  const hq::Dev& d = e->d;
  const size_t NL = (size_t)d.L * d.n;
  cudaStream_t st = e->stream;
  int rc = cuda_check(e, cudaMemcpyAsync(d.X + slot * NL, X_host, NL * sizeof(double), cudaMemcpyHostToDevice, st),
                      "set_chain fields");
  rc = rc ? rc : cuda_check(e, hq::launch_slot_control(d, slot, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                                       chain_id, sweep, 1, 1, st), "set_chain slot");
  if (!rc) e->set_act(slot, 1);
  // the caller may reuse X_host on return
  rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(st), "set_chain sync");
  e->stack_valid = e->logdet_valid = e->green_valid = false;
  return rc;
}

int hq_set_active(hq_engine* e, int slot, int active) {
  if (!e || slot < 0 || slot >= e->d.n_chains) return HQ_EINVAL;
  const int v = active ? 1 : 0;
  int rc = cuda_check(e, hq::launch_slot_control(e->d, slot, 0u, 0u, 0u, 0u, v, 0, e->stream), "set_active");
  if (!rc) e->set_act(slot, v);
  if (v) e->stack_valid = e->logdet_valid = e->green_valid = false;
  return rc;
}

// checkpoint: header (with the current n_wrap), then X, counters, totals, series (host byte order).
struct CkHeader {
  char magic[8];
  int32_t version, n_chains, first_chain, max_series, series_len, pad;
  long long sweeps;
  hq_params params;
};

static size_t ck_len(const hq_engine* e) {
  const size_t C = (size_t)e->d.n_chains;
  return sizeof(CkHeader) + field_bytes(e) + C * hq::kCounters * sizeof(long long) +
         C * hq::kTotSlots * sizeof(double) + C * HQ_N_OBS * (size_t)e->d.max_series * sizeof(double) +
         C * (4 * sizeof(uint32_t) + 2 * sizeof(int));
}

int hq_checkpoint(hq_engine* e, void* buf, size_t* len) {
  if (!e || !len) return HQ_EINVAL;
  const size_t need = ck_len(e);
  if (!buf) {
    *len = need;
    return HQ_OK;
  }
  if (*len < need) return set_err(e, HQ_EINVAL, "checkpoint buffer too small");
  *len = need;
  const size_t C = (size_t)e->d.n_chains;
  CkHeader h{};
  std::memcpy(h.magic, "HQCKPT3", 8);
  h.version = 3;
  h.pad = e->d.n_wrap;  // the current restabilisation interval (after any back-off)
  h.n_chains = e->d.n_chains;
  h.first_chain = e->d.first_chain;
  h.max_series = e->d.max_series;
  h.series_len = e->series_len;
  h.sweeps = e->sweeps;
  h.params = e->p;
  char* o = (char*)buf;
  std::memcpy(o, &h, sizeof h);
  o += sizeof h;
  int rc = cuda_check(e, cudaMemcpyAsync(o, e->d.X, field_bytes(e), cudaMemcpyDeviceToHost, e->stream), "ck X");
  o += field_bytes(e);
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(o, e->d.counters, C * hq::kCounters * sizeof(long long),
                                               cudaMemcpyDeviceToHost, e->stream), "ck counters");
  o += C * hq::kCounters * sizeof(long long);
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(o, e->d.tot, C * hq::kTotSlots * sizeof(double),
                                               cudaMemcpyDeviceToHost, e->stream), "ck totals");
  o += C * hq::kTotSlots * sizeof(double);
  if (e->d.max_series > 0)
    rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(o, e->d.series, C * HQ_N_OBS * (size_t)e->d.max_series * sizeof(double),
                                                 cudaMemcpyDeviceToHost, e->stream), "ck series");
  o += C * HQ_N_OBS * (size_t)e->d.max_series * sizeof(double);
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(o, e->d.cid, C * 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, e->stream),
                            "ck ids");
  o += C * 4 * sizeof(uint32_t);
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(o, e->d.active, C * sizeof(int), cudaMemcpyDeviceToHost, e->stream),
                            "ck active");
  o += C * sizeof(int);
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(o, e->d.slen, C * sizeof(int), cudaMemcpyDeviceToHost, e->stream),
                            "ck series lengths");
  return rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "checkpoint sync");
}

int hq_restore(hq_engine* e, const void* buf, size_t len) {
  if (!e || !buf || len < sizeof(CkHeader)) return HQ_EINVAL;
  CkHeader h;
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, "HQCKPT3", 8) != 0 || h.version != 3) return set_err(e, HQ_EINVAL, "not a checkpoint");
  if (h.pad < e->d.n_wrap_min || h.pad > e->p.n_wrap) return set_err(e, HQ_EINVAL, "checkpoint n_wrap out of range");
  if (h.n_chains != e->d.n_chains || h.max_series != e->d.max_series ||
      std::memcmp(&h.params, &e->p, sizeof(hq_params)) != 0)
    return set_err(e, HQ_EINVAL, "checkpoint is for another parameter set or chain count");
  if (len < ck_len(e)) return set_err(e, HQ_EINVAL, "checkpoint truncated");
  const size_t C = (size_t)e->d.n_chains;
  const char* o = (const char*)buf + sizeof h;
  int rc = cuda_check(e, cudaMemcpyAsync(e->d.X, o, field_bytes(e), cudaMemcpyHostToDevice, e->stream), "rs X");
  o += field_bytes(e);
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(e->d.counters, o, C * hq::kCounters * sizeof(long long),
                                               cudaMemcpyHostToDevice, e->stream), "rs counters");
  o += C * hq::kCounters * sizeof(long long);
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(e->d.tot, o, C * hq::kTotSlots * sizeof(double),
                                               cudaMemcpyHostToDevice, e->stream), "rs totals");
  o += C * hq::kTotSlots * sizeof(double);
  if (e->d.max_series > 0)
    rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(e->d.series, o, C * HQ_N_OBS * (size_t)e->d.max_series * sizeof(double),
                                                 cudaMemcpyHostToDevice, e->stream), "rs series");
  o += C * HQ_N_OBS * (size_t)e->d.max_series * sizeof(double);
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(e->d.cid, o, C * 4 * sizeof(uint32_t), cudaMemcpyHostToDevice, e->stream),
                            "rs ids");
  o += C * 4 * sizeof(uint32_t);
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(e->d.active, o, C * sizeof(int), cudaMemcpyHostToDevice, e->stream),
                            "rs active");
  for (size_t c = 0; c < C; ++c) {
    int v;
    std::memcpy(&v, o + c * sizeof(int), sizeof(int));
    e->act[c] = v ? 1 : 0;
  }
  e->set_act(0, e->act[0]);
  o += C * sizeof(int);
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(e->d.slen, o, C * sizeof(int), cudaMemcpyHostToDevice, e->stream),
                            "rs series lengths");
  rc = rc ? rc : cuda_check(e, hq::launch_reset_acc(e->d, e->stream), "rs acc");
  rc = rc ? rc : cuda_check(e, cudaMemsetAsync(e->d.status, 0, C * sizeof(int), e->stream), "rs status");
  rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "restore sync");
  if (rc) return rc;
  e->sweeps = h.sweeps;
  e->series_len = h.series_len;
  e->d.n_wrap = h.pad;
  e->d.n_bound = (e->d.L - 1) / e->d.n_wrap;
  e->d.n_chunks = (e->d.L + e->d.n_wrap - 1) / e->d.n_wrap;
  drop_graph(e);
  e->stack_valid = e->logdet_valid = e->green_valid = false;
  return HQ_OK;
}

int hq_proposal_uniforms(uint64_t seed, uint32_t chain, uint32_t sweep, uint32_t tag, const uint32_t* events_host,
                         int n, double* u1_host, double* u2_host, void* stream) {
  if (n < 0 || (n > 0 && (!events_host || !u1_host || !u2_host))) return HQ_EINVAL;
  if (n == 0) return HQ_OK;
  cudaStream_t s = (cudaStream_t)stream;
  char* buf = nullptr;
  const size_t bytes = align_up(n * sizeof(uint32_t)) + 2 * align_up(n * sizeof(double));
  if (cudaMallocAsync((void**)&buf, bytes, s) != cudaSuccess) return HQ_ECUDA;
  uint32_t* ev = (uint32_t*)buf;
  double* u1 = (double*)(buf + align_up(n * sizeof(uint32_t)));
  double* u2 = u1 + align_up(n * sizeof(double)) / sizeof(double);
  cudaError_t st = cudaMemcpyAsync(ev, events_host, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
  if (st == cudaSuccess)
    st = hq::launch_proposals((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), chain, sweep, tag, ev, n, u1,
                              u2, s);
  if (st == cudaSuccess) st = cudaMemcpyAsync(u1_host, u1, n * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (st == cudaSuccess) st = cudaMemcpyAsync(u2_host, u2, n * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(buf, s);
  if (st == cudaSuccess) st = cudaStreamSynchronize(s);
  return st == cudaSuccess ? HQ_OK : HQ_ECUDA;
}

double hq_tau_int(const double* x, int n, double c, int* window) {
  if (window) *window = 0;
  if (!x || n < 2) return 0.5;
  double mean = 0.0;
  for (int i = 0; i < n; ++i) mean += x[i];
  mean /= n;
  double c0 = 0.0;
  for (int i = 0; i < n; ++i) c0 += (x[i] - mean) * (x[i] - mean);
  c0 /= n;
  if (c0 == 0.0) return 0.5;
  double tau = 0.5;
  for (int W = 1; W < n; ++W) {
    double cw = 0.0;
    for (int i = 0; i + W < n; ++i) cw += (x[i] - mean) * (x[i + W] - mean);
    tau += cw / n / c0;
    if (W >= c * tau) {
      if (window) *window = W;
      return tau;
    }
  }
  if (window) *window = n - 1;
  return tau;
}

int hq_set_timing(hq_engine* e, int enable) {
  if (!e) return HQ_EINVAL;
  e->timing = enable != 0;
  return HQ_OK;
}

int hq_get_timing(hq_engine* e, double* ms, int64_t* launches) {
  if (!e) return HQ_EINVAL;
  int rc = cuda_check(e, cudaStreamSynchronize(e->stream), "timing sync");
  if (rc) return rc;
  for (auto& sp : e->spans) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, sp.a, sp.b) == cudaSuccess) {
      e->phase_ms[sp.phase] += t;
      e->phase_launches[sp.phase] += sp.launches;
    }
    e->spare.push_back(sp.a);
    e->spare.push_back(sp.b);
  }
  e->spans.clear();
  for (int i = 0; i < HQ_N_PHASES; ++i) {
    if (ms) ms[i] = e->phase_ms[i];
    if (launches) launches[i] = e->phase_launches[i];
    e->phase_ms[i] = 0.0;
    e->phase_launches[i] = 0;
  }
  return HQ_OK;
}

int hq_logdet_noalloc(const hq_params* p, int n_chains, const double* X_device, double* logdet_device,
                      void* stream) {
  g_call_error.clear();
  if (const char* why = validate(p, n_chains, 0)) {
    g_call_error = std::string("hq_logdet_noalloc: ") + why;
    return HQ_EINVAL;
  }
  if (!X_device || !logdet_device) {
    g_call_error = "hq_logdet_noalloc: X_device and logdet_device must be device pointers";
    return HQ_EINVAL;
  }
  const size_t need = hq::noalloc_scratch_needed(p->nx, p->ny, n_chains);
  if (need > hq::kNoAllocScratchBytes) {
    g_call_error = "hq_logdet_noalloc: " + std::to_string(n_chains) + " chains of N = " +
                   std::to_string(p->nx * p->ny) + " need " + std::to_string(need) +
                   " bytes of scratch, the static scratch holds " + std::to_string(hq::kNoAllocScratchBytes) +
                   " (HQ_NOALLOC_SCRATCH_BYTES); pass fewer chains per call";
    return HQ_ENOMEM;
  }
  hq::Dev d{};
  d.nx = p->nx;
  d.ny = p->ny;
  d.n = p->nx * p->ny;
  d.L = n_slices(*p);
  d.n_wrap = p->n_wrap;
  d.k = p->delay_k;
  d.n_chains = n_chains;
  d.n_active = n_chains;
  d.t = p->t;
  d.mu = p->mu;
  d.omega = p->omega;
  d.mass = p->mass;
  d.g = p->g;
  d.dtau = p->dtau;
  d.X = const_cast<double*>(X_device);
  const cudaError_t st = hq::launch_logdet_noalloc(d, logdet_device, (cudaStream_t)stream);
  if (st != cudaSuccess) {
    g_call_error = std::string("hq_logdet_noalloc: ") + cudaGetErrorString(st);
    return HQ_ECUDA;
  }
  return HQ_OK;
}

// ----------------------------------------------------------------- learned moves
namespace {

constexpr int kNNParamsPad = (HQ_NN_PARAMS + 3) & ~3;

constexpr int kCnnParamsPad = (HQ_CNN_PARAMS + 3) & ~3;

struct NNLayout {
  size_t wbf, master, grad, am, av, partials, fcache, fnew, X0, ld0, F0, F1, pc, Fb, loss, idx, counters, dFpath, G0, xf, xb;
  size_t cwbf, cmaster, cgrad, cam, cav, cpartials, h1c, h2c, o3c, h1p, h2p, o3p, tr, cFb, cF;
  int train_ctas;
  size_t total;
};

NNLayout nn_layout(const hq::Dev& d, int max_batch, int max_samples) {
  NNLayout l{};
  const size_t C = d.n_chains, NL = (size_t)d.n * d.L, P = kNNParamsPad;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes); return o; };
  l.wbf = take(2 * P);
  l.master = take(4 * P);
  l.grad = take(4 * P);
  l.am = take(4 * P);
  l.av = take(4 * P);
  l.partials = take(4 * P * hq::kNNTrainCtas);
  l.fcache = take(4 * C * NL);
  l.fnew = take(4 * C * 5 * d.L);
  l.X0 = take(8 * C * NL);
  l.ld0 = take(8 * C);
  l.F0 = take(8 * C);
  l.F1 = take(8 * C);
  l.pc = take(8 * C);
  l.Fb = take(8 * (size_t)max_batch);
  l.loss = take(8);
  l.idx = take(4 * (size_t)max_samples);
  l.counters = take(8 * C * hq::kNNCounters);
  l.dFpath = take(8 * C);
  l.G0 = take(8 * C * (size_t)d.n * d.n);
  l.xf = take(4 * C * NL);
  l.xb = take(4 * (size_t)max_batch * NL);
  // convolutional action
  const size_t PC = kCnnParamsPad, CH = hq::kCnnC;
  l.train_ctas = max_batch < hq::kCnnTrainCtas ? max_batch : hq::kCnnTrainCtas;
  l.cwbf = take(2 * PC);
  l.cmaster = take(4 * PC);
  l.cgrad = take(4 * PC);
  l.cam = take(4 * PC);
  l.cav = take(4 * PC);
  l.cpartials = take(4 * PC * l.train_ctas);
  l.h1c = take(4 * C * NL * CH);
  l.h2c = take(4 * C * NL * CH);
  l.o3c = take(4 * C * NL);
  l.h1p = take(4 * C * 9 * d.L * CH);
  l.h2p = take(4 * C * 25 * d.L * CH);
  l.o3p = take(4 * C * 49 * d.L);
  l.tr = take(4 * (size_t)l.train_ctas * 3 * NL * CH);
  l.cFb = take(8 * (size_t)max_batch);
  l.cF = take(8 * C);
  l.total = off;
  return l;
}

bool nn_shape_ok(const hq::Dev& d) { return d.nx >= 4 && d.ny >= 4 && d.L >= 5; }

int nn_ready(hq_engine* e) {
  if (!e) return HQ_EINVAL;
  if (!e->nn_on) return set_err(e, HQ_EINVAL, "no network state attached (hq_nn_attach)");
  return HQ_OK;
}

uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

size_t hq_nn_arena_bytes(const hq_engine* e, int max_batch, int max_samples) {
  if (!e || max_batch < 1 || max_samples < max_batch || !nn_shape_ok(e->d)) return 0;
  return nn_layout(e->d, max_batch, max_samples).total;
}

int hq_nn_attach(hq_engine* e, void* arena, size_t bytes, int max_batch, int max_samples) {
  if (!e || max_batch < 1 || max_samples < max_batch) return HQ_EINVAL;
  if (!nn_shape_ok(e->d)) return set_err(e, HQ_EINVAL, "learned moves need nx, ny >= 4 and L >= 5");
  const NNLayout l = nn_layout(e->d, max_batch, max_samples);
  if (!arena || bytes < l.total || ((uintptr_t)arena % kAlign) != 0) return HQ_ENOMEM;
  char* a = (char*)arena;
  hq::NNState& nn = e->nn;
  nn.wbf = (uint16_t*)(a + l.wbf);
  nn.master = (float*)(a + l.master);
  nn.grad = (float*)(a + l.grad);
  nn.adam_m = (float*)(a + l.am);
  nn.adam_v = (float*)(a + l.av);
  nn.partials = (float*)(a + l.partials);
  nn.fcache = (float*)(a + l.fcache);
  nn.fnew = (float*)(a + l.fnew);
  nn.X0 = (double*)(a + l.X0);
  nn.ld0 = (double*)(a + l.ld0);
  nn.F0 = (double*)(a + l.F0);
  nn.F1 = (double*)(a + l.F1);
  nn.last_pc = (double*)(a + l.pc);
  nn.Fb = (double*)(a + l.Fb);
  nn.loss = (double*)(a + l.loss);
  nn.idx = (int*)(a + l.idx);
  nn.counters = (long long*)(a + l.counters);
  nn.dFpath = (double*)(a + l.dFpath);
  nn.G0 = (double*)(a + l.G0);
  nn.xf = (float*)(a + l.xf);
  nn.xb = (float*)(a + l.xb);
  nn.x0 = -e->p.g / (e->p.mass * e->p.omega * e->p.omega);
  hq::CnnState& cn = e->cn;
  cn.on = 0;
  cn.wbf = (uint16_t*)(a + l.cwbf);
  cn.master = (float*)(a + l.cmaster);
  cn.grad = (float*)(a + l.cgrad);
  cn.adam_m = (float*)(a + l.cam);
  cn.adam_v = (float*)(a + l.cav);
  cn.partials = (float*)(a + l.cpartials);
  cn.train_ctas = l.train_ctas;
  cn.h1c = (float*)(a + l.h1c);
  cn.h2c = (float*)(a + l.h2c);
  cn.o3c = (float*)(a + l.o3c);
  cn.h1p = (float*)(a + l.h1p);
  cn.h2p = (float*)(a + l.h2p);
  cn.o3p = (float*)(a + l.o3p);
  cn.tr = (float*)(a + l.tr);
  cn.Fb = (double*)(a + l.cFb);
  cn.F = (double*)(a + l.cF);
  e->cn_t_step = 0;
  int rc = cuda_check(e, cudaMemsetAsync(a, 0, l.total, e->stream), "nn arena clear");
  if (rc) return rc;
  e->nn_on = true;
  e->nn_max_batch = max_batch;
  e->nn_max_samples = max_samples;
  e->cum_steps = 0;
  e->nn_t_step = 0;
  return HQ_OK;
}

int hq_nn_set_params(hq_engine* e, const float* theta_host) {
  int rc = nn_ready(e);
  if (rc) return rc;
  if (!theta_host) return HQ_EINVAL;
  rc = cuda_check(e, cudaMemcpyAsync(e->nn.partials, theta_host, sizeof(float) * HQ_NN_PARAMS,
                                     cudaMemcpyHostToDevice, e->stream), "nn params upload");
  rc = rc ? rc : cuda_check(e, hq::nn_launch_set(e->nn, e->nn.partials, e->stream), "nn set");
  rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "nn set sync");
  e->nn_t_step = 0;
  return rc;
}

int hq_nn_get_params(hq_engine* e, float* theta_host, int bf16) {
  int rc = nn_ready(e);
  if (rc) return rc;
  if (!theta_host) return HQ_EINVAL;
  if (bf16) {
    std::vector<uint16_t> h(HQ_NN_PARAMS);
    rc = cuda_check(e, cudaMemcpyAsync(h.data(), e->nn.wbf, 2 * HQ_NN_PARAMS, cudaMemcpyDeviceToHost, e->stream),
                    "nn params copy");
    rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "nn params sync");
    if (rc) return rc;
    for (int k = 0; k < HQ_NN_PARAMS; ++k) {
      const uint32_t u = (uint32_t)h[k] << 16;
      std::memcpy(&theta_host[k], &u, 4);
    }
    return HQ_OK;
  }
  rc = cuda_check(e, cudaMemcpyAsync(theta_host, e->nn.master, 4 * HQ_NN_PARAMS, cudaMemcpyDeviceToHost, e->stream),
                  "nn params copy");
  return rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "nn params sync");
}

int hq_nn_eval(hq_engine* e, double* F_host) {
  int rc = nn_ready(e);
  if (rc) return rc;
  if (!F_host) return HQ_EINVAL;
  rc = cuda_check(e, hq::nn_launch_eval(e->d, e->nn, e->d.X, e->nn.F0, 1, e->stream), "nn eval");
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(F_host, e->nn.F0, sizeof(double) * e->d.n_chains,
                                               cudaMemcpyDeviceToHost, e->stream), "nn eval copy");
  return rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "nn eval sync");
}

int hq_nn_gradient(hq_engine* e, const double* X_device, const double* y_device, int n_samples, float* grad_host,
                   double* loss_host) {
  int rc = nn_ready(e);
  if (rc) return rc;
  if (!X_device || !y_device || n_samples < 1 || n_samples > e->nn_max_batch) return HQ_EINVAL;
  std::vector<int> idx(n_samples);
  for (int a = 0; a < n_samples; ++a) idx[a] = a;
  rc = cuda_check(e, cudaMemcpyAsync(e->nn.idx, idx.data(), sizeof(int) * n_samples, cudaMemcpyHostToDevice,
                                     e->stream), "nn idx");
  rc = rc ? rc : cuda_check(e, cudaMemsetAsync(e->nn.loss, 0, sizeof(double), e->stream), "nn loss clear");
  rc = rc ? rc : cuda_check(e, hq::nn_launch_batch(e->d, e->nn, X_device, y_device, e->nn.idx, n_samples, 0.f, 1,
                                                    e->stream), "nn batch");
  rc = rc ? rc : cuda_check(e, hq::nn_launch_loss(e->nn, y_device, e->nn.idx, n_samples, 1.0 / n_samples, e->stream),
                            "nn loss");
  if (!rc && grad_host)
    rc = cuda_check(e, cudaMemcpyAsync(grad_host, e->nn.grad, 4 * HQ_NN_PARAMS, cudaMemcpyDeviceToHost, e->stream),
                    "nn grad copy");
  if (!rc && loss_host)
    rc = cuda_check(e, cudaMemcpyAsync(loss_host, e->nn.loss, sizeof(double), cudaMemcpyDeviceToHost, e->stream),
                    "nn loss copy");
  return rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "nn grad sync");
}

int hq_nn_train(hq_engine* e, const double* X_device, const double* y_device, int n_samples, int epochs, int batch,
                float lr, uint64_t seed, double* loss_host) {
  int rc = nn_ready(e);
  if (rc) return rc;
  if (!X_device || !y_device || n_samples < 1 || n_samples > e->nn_max_samples || epochs < 0 || batch < 1 ||
      batch > e->nn_max_batch || !(lr > 0.f))
    return HQ_EINVAL;
  std::vector<int> order(n_samples);
  uint64_t st = seed;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int a = 0; a < n_samples; ++a) order[a] = a;
    for (int a = n_samples - 1; a > 0; --a) {  // Fisher-Yates with splitmix64
      const int b = (int)(splitmix64(st) % (uint64_t)(a + 1));
      std::swap(order[a], order[b]);
    }
    rc = cuda_check(e, cudaMemcpyAsync(e->nn.idx, order.data(), sizeof(int) * n_samples, cudaMemcpyHostToDevice,
                                       e->stream), "nn order");
    rc = rc ? rc : cuda_check(e, cudaMemsetAsync(e->nn.loss, 0, sizeof(double), e->stream), "nn loss clear");
    if (rc) return rc;
    for (int a0 = 0; a0 + batch <= n_samples; a0 += batch) {
      rc = cuda_check(e, hq::nn_launch_batch(e->d, e->nn, X_device, y_device, e->nn.idx + a0, batch, lr,
                                             ++e->nn_t_step, e->stream), "nn batch");
      rc = rc ? rc : cuda_check(e, hq::nn_launch_loss(e->nn, y_device, e->nn.idx + a0, batch,
                                                      1.0 / (double)(n_samples / batch * batch), e->stream), "nn loss");
      if (rc) return rc;
    }
    if (loss_host) {
      rc = cuda_check(e, cudaMemcpyAsync(&loss_host[ep], e->nn.loss, sizeof(double), cudaMemcpyDeviceToHost,
                                         e->stream), "nn loss copy");
      rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "nn epoch sync");
      if (rc) return rc;
    }
  }
  return cuda_check(e, cudaStreamSynchronize(e->stream), "nn train sync");
}

int hq_cumulative_sweep(hq_engine* e, int n_steps, int n_inner, unsigned flags) {
  int rc = nn_ready(e);
  if (rc) return rc;
  if (n_steps < 0 || n_inner < 1 || (flags & ~(HQ_LOCAL | HQ_GLOBAL | HQ_MEASURE | HQ_CNN_BLOCK))) return HQ_EINVAL;
  const int use_cnn = (flags & HQ_CNN_BLOCK) ? 1 : 0;
  if (use_cnn && !e->cn.on) return set_err(e, HQ_EINVAL, "HQ_CNN_BLOCK needs convolutional parameters (hq_cnn_set_params)");
  const hq::Dev& d = e->d;
  const size_t fbytes = sizeof(double) * (size_t)d.n_chains * d.L * d.n;
  const bool meas = flags & HQ_MEASURE;
  // the exact log|det M(X')| of every step: one CTA per chain (stack build, G_0), or with few
  // chains two CTAs per chain (halves above and below the boundary m joined by the two-sided
  // formula, G_m); measured steps record the observables of that G
  const int m = split_in_use(e);
  for (int k = 0; k < n_steps; ++k) {
    // the step needs log|det M(X)|, and for a measured step G of X at the slice used (kept for
    // rejection)
    if (m > 0) {
      if (!e->logdet_valid || (meas && !(e->green_valid && e->green_slice == m))) rc = split_state(e, m);
    } else if (!e->logdet_valid || (meas && !(e->green_valid && e->green_slice == 0))) {
      e->stack_valid = e->stack_valid && e->green_slice == 0 && e->green_valid;
      rc = ensure_state(e);
    }
    if (rc) return rc;
    if (meas)
      rc = cuda_check(e, cudaMemcpyAsync(e->nn.G0, d.G, sizeof(double) * (size_t)d.n_chains * d.n * d.n,
                                         cudaMemcpyDeviceToDevice, e->stream), "G0 copy");
    rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(e->nn.X0, d.X, fbytes, cudaMemcpyDeviceToDevice, e->stream),
                              "X0 copy");
    rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(e->nn.ld0, d.logdet, sizeof(double) * d.n_chains,
                                                 cudaMemcpyDeviceToDevice, e->stream), "ld0 copy");
    // caches of the current fields (the previous step may have restored X)
    {
      PhaseTimer pt(e, 6, use_cnn ? 2 : 1);
      rc = rc ? rc : cuda_check(e, hq::nn_launch_eval(d, e->nn, d.X, e->nn.F0, 1, e->stream), "nn eval F0");
      if (use_cnn) rc = rc ? rc : cuda_check(e, hq::cnn_launch_eval(d, e->cn, d.X, e->cn.F, 1, e->stream), "cnn eval");
    }
    {
      PhaseTimer pt(e, 7, 1);
      rc = rc ? rc : cuda_check(e, hq::nn_launch_inner(d, e->nn, e->cn, n_inner, (flags & HQ_LOCAL) ? 1 : 0,
                                                       (flags & HQ_GLOBAL) ? 1 : 0, use_cnn, e->nn_window,
                                                       e->nn_site_window, e->stream), "nn inner");
    }
    if (rc) return rc;
    e->stack_valid = false;
    // log|det M(X')| (and G of X')
    rc = m > 0 ? split_state(e, m) : ensure_state(e);
    // a rejected chain gets back X, log|det M(X)| and, for a measured step, G of X
    rc = rc ? rc : cuda_check(e, hq::nn_launch_decide(d, e->nn, meas ? 1 : 0, e->stream), "nn decide");
    if (rc) return rc;
    e->stack_valid = false;  // the stack is X''s; rejected chains are back at X
    e->green_valid = meas;   // measured steps: every chain's G is G_m (or G_0) of its final fields
    e->green_slice = m;
    e->logdet_valid = true;
    {
      PhaseTimer pt(e, 3, meas ? 2 : 1);
      if (meas) rc = cuda_check(e, hq::launch_measure_g0(d, e->stream), "measure");
      rc = rc ? rc : cuda_check(e, hq::launch_sweep_end(d, meas ? 1 : 0, e->stream), "sweep_end launch");
    }
    if (rc) return rc;
    e->cum_steps++;
  }
  return HQ_OK;
}

int hq_set_block_sites(hq_engine* e, int sites) {
  if (!e || sites < 0) return HQ_EINVAL;
  e->d.block_sites = sites >= e->d.n ? 0 : sites;
  drop_graph(e);
  return HQ_OK;
}

int hq_set_logdet_split(hq_engine* e, int mode) {
  if (!e || mode < 0 || mode > 2) return HQ_EINVAL;
  if (mode == 2 && hq::split_point(e->d) == 0) return set_err(e, HQ_EINVAL, "fewer than two restabilisation chunks");
  e->split_mode = mode;
  return split_in_use(e);
}

int hq_set_inner_window(hq_engine* e, int slices) {
  if (!e || slices < 0) return HQ_EINVAL;
  e->nn_window = slices >= e->d.L ? 0 : slices;
  return HQ_OK;
}

int hq_set_inner_sites(hq_engine* e, int sites) {
  if (!e || sites < 0) return HQ_EINVAL;
  e->nn_site_window = sites >= e->d.n ? 0 : sites;
  return HQ_OK;
}

int hq_cnn_set_params(hq_engine* e, const float* theta_host) {
  int rc = nn_ready(e);
  if (rc) return rc;
  if (!theta_host) return HQ_EINVAL;
  rc = cuda_check(e, cudaMemcpyAsync(e->cn.partials, theta_host, sizeof(float) * HQ_CNN_PARAMS,
                                     cudaMemcpyHostToDevice, e->stream), "cnn params upload");
  rc = rc ? rc : cuda_check(e, hq::cnn_launch_set(e->cn, e->cn.partials, e->stream), "cnn set");
  rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "cnn set sync");
  if (!rc) e->cn.on = 1;
  e->cn_t_step = 0;
  return rc;
}

int hq_cnn_get_params(hq_engine* e, float* theta_host, int bf16) {
  int rc = nn_ready(e);
  if (rc) return rc;
  if (!theta_host) return HQ_EINVAL;
  if (bf16) {
    std::vector<uint16_t> h(HQ_CNN_PARAMS);
    rc = cuda_check(e, cudaMemcpyAsync(h.data(), e->cn.wbf, 2 * HQ_CNN_PARAMS, cudaMemcpyDeviceToHost, e->stream),
                    "cnn params copy");
    rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "cnn params sync");
    if (rc) return rc;
    for (int k = 0; k < HQ_CNN_PARAMS; ++k) {
      const uint32_t u = (uint32_t)h[k] << 16;
      std::memcpy(&theta_host[k], &u, 4);
    }
    return HQ_OK;
  }
  rc = cuda_check(e, cudaMemcpyAsync(theta_host, e->cn.master, 4 * HQ_CNN_PARAMS, cudaMemcpyDeviceToHost,
                                     e->stream), "cnn params copy");
  return rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "cnn params sync");
}

int hq_cnn_eval(hq_engine* e, double* F_host) {
  int rc = nn_ready(e);
  if (rc) return rc;
  if (!F_host) return HQ_EINVAL;
  if (!e->cn.on) return set_err(e, HQ_EINVAL, "no convolutional parameters (hq_cnn_set_params)");
  rc = cuda_check(e, hq::cnn_launch_eval(e->d, e->cn, e->d.X, e->cn.F, 1, e->stream), "cnn eval");
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(F_host, e->cn.F, sizeof(double) * e->d.n_chains,
                                               cudaMemcpyDeviceToHost, e->stream), "cnn eval copy");
  return rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "cnn eval sync");
}

int hq_cnn_gradient(hq_engine* e, const double* X_device, const double* y_device, int n_samples, float* grad_host,
                    double* loss_host) {
  int rc = nn_ready(e);
  if (rc) return rc;
  if (!X_device || !y_device || n_samples < 1 || n_samples > e->nn_max_batch) return HQ_EINVAL;
  if (!e->cn.on) return set_err(e, HQ_EINVAL, "no convolutional parameters (hq_cnn_set_params)");
  std::vector<int> idx(n_samples);
  for (int a = 0; a < n_samples; ++a) idx[a] = a;
  rc = cuda_check(e, cudaMemcpyAsync(e->nn.idx, idx.data(), sizeof(int) * n_samples, cudaMemcpyHostToDevice,
                                     e->stream), "cnn idx");
  rc = rc ? rc : cuda_check(e, cudaMemsetAsync(e->nn.loss, 0, sizeof(double), e->stream), "cnn loss clear");
  rc = rc ? rc : cuda_check(e, hq::cnn_launch_batch(e->d, e->cn, X_device, y_device, e->nn.idx, n_samples, 0.f, 1,
                                                     e->stream), "cnn batch");
  rc = rc ? rc : cuda_check(e, hq::cnn_launch_loss(e->cn, y_device, e->nn.idx, n_samples, 1.0 / n_samples,
                                                    e->nn.loss, e->stream), "cnn loss");
  if (!rc && grad_host)
    rc = cuda_check(e, cudaMemcpyAsync(grad_host, e->cn.grad, 4 * HQ_CNN_PARAMS, cudaMemcpyDeviceToHost, e->stream),
                    "cnn grad copy");
  if (!rc && loss_host)
    rc = cuda_check(e, cudaMemcpyAsync(loss_host, e->nn.loss, sizeof(double), cudaMemcpyDeviceToHost, e->stream),
                    "cnn loss copy");
  return rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "cnn grad sync");
}

int hq_cnn_train(hq_engine* e, const double* X_device, const double* y_device, int n_samples, int epochs, int batch,
                 float lr, uint64_t seed, double* loss_host) {
  int rc = nn_ready(e);
  if (rc) return rc;
  if (!X_device || !y_device || n_samples < 1 || n_samples > e->nn_max_samples || epochs < 0 || batch < 1 ||
      batch > e->nn_max_batch || !(lr > 0.f))
    return HQ_EINVAL;
  if (!e->cn.on) return set_err(e, HQ_EINVAL, "no convolutional parameters (hq_cnn_set_params)");
  std::vector<int> order(n_samples);
  uint64_t st = seed;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int a = 0; a < n_samples; ++a) order[a] = a;
    for (int a = n_samples - 1; a > 0; --a) {  // Fisher-Yates with splitmix64
      const int b = (int)(splitmix64(st) % (uint64_t)(a + 1));
      std::swap(order[a], order[b]);
    }
    rc = cuda_check(e, cudaMemcpyAsync(e->nn.idx, order.data(), sizeof(int) * n_samples, cudaMemcpyHostToDevice,
                                       e->stream), "cnn order");
    rc = rc ? rc : cuda_check(e, cudaMemsetAsync(e->nn.loss, 0, sizeof(double), e->stream), "cnn loss clear");
    if (rc) return rc;
    for (int a0 = 0; a0 + batch <= n_samples; a0 += batch) {
      rc = cuda_check(e, hq::cnn_launch_batch(e->d, e->cn, X_device, y_device, e->nn.idx + a0, batch, lr,
                                              ++e->cn_t_step, e->stream), "cnn batch");
      rc = rc ? rc : cuda_check(e, hq::cnn_launch_loss(e->cn, y_device, e->nn.idx + a0, batch,
                                                       1.0 / (double)(n_samples / batch * batch), e->nn.loss,
                                                       e->stream), "cnn loss");
      if (rc) return rc;
    }
    // the host order vector is reused by the next epoch: its copy must have completed
    rc = cuda_check(e, cudaStreamSynchronize(e->stream), "cnn epoch sync");
    if (rc) return rc;
    if (loss_host) {
      rc = cuda_check(e, cudaMemcpyAsync(&loss_host[ep], e->nn.loss, sizeof(double), cudaMemcpyDeviceToHost,
                                         e->stream), "cnn loss copy");
      rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "cnn epoch sync");
      if (rc) return rc;
    }
  }
  return cuda_check(e, cudaStreamSynchronize(e->stream), "cnn train sync");
}

int hq_get_learned_stats(hq_engine* e, hq_learned_stats* out) {
  int rc = nn_ready(e);
  if (rc) return rc;
  if (!out) return HQ_EINVAL;
  const size_t C = e->d.n_chains;
  std::vector<long long> cnt(C * hq::kNNCounters);
  std::vector<double> pc(C);
  rc = cuda_check(e, cudaMemcpyAsync(cnt.data(), e->nn.counters, sizeof(long long) * cnt.size(),
                                     cudaMemcpyDeviceToHost, e->stream), "nn counters");
  rc = rc ? rc : cuda_check(e, cudaMemcpyAsync(pc.data(), e->nn.last_pc, sizeof(double) * C, cudaMemcpyDeviceToHost,
                                               e->stream), "nn pc");
  rc = rc ? rc : cuda_check(e, cudaStreamSynchronize(e->stream), "nn stats sync");
  if (rc) return rc;
  for (size_t c = 0; c < C; ++c) {
    const long long* k = cnt.data() + c * hq::kNNCounters;
    out[c] = hq_learned_stats{k[0], k[1], k[2], k[3], k[4], k[5], pc[c]};
  }
  return HQ_OK;
}

// ----------------------------------------------------------------- engine groups
struct hq_group {
  std::vector<hq_engine*> eng;
  hq::GroupDev g{};
  cudaStream_t stream = nullptr;
  int lmax = 2;
  size_t sb = 0;
  std::vector<cudaEvent_t> ev;  // [n_eng + 1]: engine streams -> group, group -> engines
  ~hq_group() {
    for (auto x : ev)
      if (x) cudaEventDestroy(x);
  }
};

namespace {
struct GroupLayout {
  size_t devs, tasks, sched, total;
  int n_tasks;
};

// FP64 flop estimate of one chain-sweep (orders the task table; only ratios matter): stack
// build, local chunks (wraps, flushes, restabilisations), block moves (a stabilised
// determinant per site)
double group_chain_cost(const hq_engine* e) {
  const double n = e->d.n, n3 = n * n * n, L = e->d.L;
  const double Q = (e->d.L + e->d.n_wrap - 1) / e->d.n_wrap;
  return Q * 6.0 * n3 + L * 8.0 * n3 + n * Q * 6.0 * n3;
}

const char* group_check(hq_engine* const* engines, int n_engines) {
  if (!engines || n_engines < 1 || n_engines > hq::kGroupMaxEngines) return "1..64 engines";
  for (int a = 0; a < n_engines; ++a) {
    if (!engines[a]) return "null engine";
    if (engines[a]->d.n_chains > 65535) return "engine too large for a group";
    for (int b = 0; b < a; ++b)
      if (engines[a] == engines[b]) return "an engine appears twice";
  }
  return nullptr;
}

GroupLayout group_layout(hq_engine* const* engines, int n_engines) {
  GroupLayout l{};
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes); return o; };
  for (int a = 0; a < n_engines; ++a) l.n_tasks += engines[a]->d.n_chains;
  l.devs = take(sizeof(hq::Dev) * n_engines);
  l.tasks = take(sizeof(uint32_t) * (size_t)l.n_tasks);
  l.sched = take(sizeof(int) * hq::kSchedHeader);
  l.total = off;
  return l;
}
}  // namespace

size_t hq_group_arena_bytes(hq_engine* const* engines, int n_engines) {
  if (group_check(engines, n_engines)) return 0;
  return group_layout(engines, n_engines).total;
}

int hq_group_create(hq_engine* const* engines, int n_engines, void* device_arena, size_t arena_bytes, void* stream,
                    hq_group** out) {
  if (!out) return HQ_EINVAL;
  *out = nullptr;
  if (const char* why = group_check(engines, n_engines)) {
    std::fprintf(stderr, "hq_group_create: %s\n", why);
    return HQ_EINVAL;
  }
  const GroupLayout l = group_layout(engines, n_engines);
  if (!device_arena || arena_bytes < l.total || ((uintptr_t)device_arena % kAlign) != 0) return HQ_ENOMEM;
  hq_group* g = new (std::nothrow) hq_group();
  if (!g) return HQ_ENOMEM;
  g->eng.assign(engines, engines + n_engines);
  g->stream = (cudaStream_t)stream;
  char* a = (char*)device_arena;
  std::vector<hq::Dev> devs(n_engines);
  for (int e = 0; e < n_engines; ++e) {
    const hq::Dev& d = engines[e]->d;
    devs[e] = d;
    const int lm = hq::lmax_class(d.nx, d.ny);
    g->lmax = lm > g->lmax ? lm : g->lmax;
  }
  // every engine's chains run in the group's class, whose QR may need more shared memory
  for (int e = 0; e < n_engines; ++e) {
    const size_t sb = hq::smem_bytes_class(engines[e]->d, g->lmax);
    g->sb = sb > g->sb ? sb : g->sb;
  }
  // task table: every chain, longest estimated sweep first (longest-processing-time order)
  struct Item { double cost; uint32_t w; };
  std::vector<Item> items;
  items.reserve(l.n_tasks);
  for (int e = 0; e < n_engines; ++e)
    for (int c = 0; c < engines[e]->d.n_chains; ++c)
      items.push_back({group_chain_cost(engines[e]), ((uint32_t)e << 26) | (uint32_t)c});
  std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) { return x.cost > y.cost; });
  std::vector<uint32_t> tasks(items.size());
  for (size_t k = 0; k < items.size(); ++k) tasks[k] = items[k].w;
  g->g.devs = (const hq::Dev*)(a + l.devs);
  g->g.tasks = (const uint32_t*)(a + l.tasks);
  g->g.sched = (int*)(a + l.sched);
  g->g.n_eng = n_engines;
  g->g.n_tasks = l.n_tasks;
  cudaError_t st = cudaMemcpyAsync(a + l.devs, devs.data(), sizeof(hq::Dev) * n_engines, cudaMemcpyHostToDevice,
                                   g->stream);
  if (st == cudaSuccess)
    st = cudaMemcpyAsync(a + l.tasks, tasks.data(), sizeof(uint32_t) * tasks.size(), cudaMemcpyHostToDevice,
                         g->stream);
  if (st == cudaSuccess) st = cudaStreamSynchronize(g->stream);
  g->ev.assign(n_engines + 1, nullptr);
  for (int k = 0; k <= n_engines && st == cudaSuccess; ++k)
    st = cudaEventCreateWithFlags(&g->ev[k], cudaEventDisableTiming);
  if (st != cudaSuccess) {
    std::fprintf(stderr, "hq_group_create: %s\n", cudaGetErrorString(st));
    delete g;
    return HQ_ECUDA;
  }
  *out = g;
  return HQ_OK;
}

void hq_group_destroy(hq_group* g) { delete g; }

int hq_group_sweep(hq_group* g, int n_sweeps, unsigned flags) {
  if (!g || n_sweeps < 0 || (flags & ~(HQ_LOCAL | HQ_GLOBAL | HQ_MEASURE))) return HQ_EINVAL;
  const bool do_local = flags & HQ_LOCAL, do_global = flags & HQ_GLOBAL;
  const int E = (int)g->eng.size();
  hq_engine* e0 = g->eng[0];
  // order after the engines' own streams
  for (int e = 0; e < E; ++e) {
    int rc = cuda_check(e0, cudaEventRecord(g->ev[e], g->eng[e]->stream), "group event");
    rc = rc ? rc : cuda_check(e0, cudaStreamWaitEvent(g->stream, g->ev[e], 0), "group wait");
    if (rc) return rc;
  }
  int rc = HQ_OK;
  for (int it = 0; it < n_sweeps && rc == HQ_OK; ++it) {
    bool need_stack = false;
    int n_active = 0;
    for (hq_engine* e : g->eng) {
      if ((do_local || !e->logdet_valid) && !e->stack_valid) need_stack = true;
      n_active += e->d.n_active;
    }
    // a stack build of an engine whose state is current recomputes the same values
    rc = cuda_check(e0, cudaMemsetAsync(g->g.sched, 0, sizeof(int) * hq::kSchedHeader, g->stream), "group sched");
    rc = rc ? rc : cuda_check(e0, hq::launch_group_sweep(g->g, g->lmax, g->sb, n_active, (int)flags,
                                                         need_stack ? 1 : 0, g->stream), "group sweep");
    if (rc) break;
    for (hq_engine* e : g->eng) {
      if (need_stack) {
        e->stack_valid = e->logdet_valid = e->green_valid = true;
        e->green_slice = 0;
      }
      if (do_local) {
        e->stack_valid = false;
        e->logdet_valid = e->green_valid = true;
        e->green_slice = 0;
      }
      if (do_global) e->stack_valid = e->green_valid = false;
      e->sweeps++;
    }
  }
  // the engines' later calls on their own streams follow the group's work
  int rc2 = cuda_check(e0, cudaEventRecord(g->ev[E], g->stream), "group event");
  for (int e = 0; e < E && rc2 == HQ_OK; ++e)
    rc2 = cuda_check(e0, cudaStreamWaitEvent(g->eng[e]->stream, g->ev[E], 0), "engine wait");
  return rc ? rc : rc2;
}

size_t hq_autotune_arena_bytes(const hq_params* p, int n_chains, const int* ks, int n_k) {
  if (!p || !ks || n_k < 1) return 0;
  size_t need = 0;
  for (int a = 0; a < n_k; ++a)
    for (int m = 1; m <= 2; ++m) {
      hq_params q = *p;
      q.delay_k = ks[a];
      q.block_method = m;
      if (validate(&q, n_chains, 0)) return 0;
      const size_t b = layout(q, n_chains, 0).total;
      need = b > need ? b : need;
    }
  return need;
}

int hq_autotune(const hq_params* p, int n_chains, const double* X_device, void* device_arena, size_t arena_bytes,
                void* stream, const int* ks, int n_k, const int* methods, int n_methods, unsigned flags, int warmup,
                int reps, double* ms_out, int* best_k, int* best_method) {
  if (!p || !X_device || !ks || !methods || n_k < 1 || n_methods < 1 || warmup < 0 || reps < 1 || !ms_out ||
      (flags & ~(HQ_LOCAL | HQ_GLOBAL | HQ_MEASURE)))
    return HQ_EINVAL;
  for (int b = 0; b < n_methods; ++b)
    if (methods[b] < 1 || methods[b] > 2) return HQ_EINVAL;
  const size_t need = hq_autotune_arena_bytes(p, n_chains, ks, n_k);
  if (need == 0) return HQ_EINVAL;
  if (!device_arena || arena_bytes < need) return HQ_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
    if (ev[0]) cudaEventDestroy(ev[0]);
    return HQ_ECUDA;
  }
  int rc = HQ_OK;
  double best = -1.0;
  for (int a = 0; a < n_k && rc == HQ_OK; ++a)
    for (int b = 0; b < n_methods && rc == HQ_OK; ++b) {
      hq_params q = *p;
      q.delay_k = ks[a];
      q.block_method = methods[b];
      hq_engine* e = nullptr;
      rc = hq_create(&q, n_chains, 0, 0, device_arena, arena_bytes, stream, &e);
      if (rc) break;
      rc = hq_set_fields_device(e, X_device);
      rc = rc ? rc : hq_sweep(e, warmup, flags);
      rc = rc ? rc : cuda_check(e, cudaEventRecord(ev[0], st), "autotune event");
      rc = rc ? rc : hq_sweep(e, reps, flags);
      rc = rc ? rc : cuda_check(e, cudaEventRecord(ev[1], st), "autotune event");
      rc = rc ? rc : cuda_check(e, cudaEventSynchronize(ev[1]), "autotune sync");
      float ms = 0.f;
      rc = rc ? rc : cuda_check(e, cudaEventElapsedTime(&ms, ev[0], ev[1]), "autotune elapsed");
      hq_destroy(e);
      if (rc) break;
      const double per = (double)ms / reps;
      ms_out[a * n_methods + b] = per;
      if (best < 0.0 || per < best) {
        best = per;
        if (best_k) *best_k = ks[a];
        if (best_method) *best_method = methods[b];
      }
    }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  return rc;
}

int hq_wait_probe(double limit_seconds, void* stream, int* status_out) {
  if (!status_out || !(limit_seconds > 0.0) || limit_seconds > 2.0) return HQ_EINVAL;
  *status_out = HQ_OK;
  const cudaError_t st = hq::wait_probe(limit_seconds, (cudaStream_t)stream, status_out);
  return st == cudaSuccess ? HQ_OK : HQ_ECUDA;
}

int hq_get_section_cycles(uint64_t* out, int n) {
  if (!out || n < 0) return HQ_EINVAL;
  return hq::section_cycles((unsigned long long*)out, n);
}

double hq_fp64_peak_tflops(int kind, int reps, void* stream) {
  if (reps < 1) reps = 1;
  if (kind != HQ_PROBE_DFMA && kind != HQ_PROBE_DMMA) return -1.0;
  return hq::fp64_probe_tflops(kind, reps, (cudaStream_t)stream);
}

}  // extern "C"
