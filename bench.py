"""Benchmark of the GB300 Holstein DQMC engine.

Default (the headline): learned vs plain sampling at the largest lattice, 16x16 periodic
(N = 256), t = M = Omega = 1, g = sqrt(2), mu = -2 (half filling), beta = 16, dtau = 0.1
(L = 160), 64 chains per GPU.
  * Learned sampler: cumulative steps of the patch network (local moves on a window of 32
    consecutive slices, a block move at every site), each accepted on the exact FP64
    log|det M|.  The network is trained first on plain-sampler configurations at 8x8 (same
    beta and couplings) by the library's tensor-core kernels.
  * Plain sampler: a full sweep (local moves at every (l, i), one block move per site on the
    full stabilised determinant), timed with block moves on a run of sites and scaled per
    move; its independent samples/s are bounded by one per sweep.
Metric: independent samples/s (tau_int-corrected, tau_int from the series of this run) of the
learned sampler, with the plain sampler's bound and their ratio; one JSON line on rank 0.
Fields start at the mean field -g/(M Omega^2) + N(0, 1/(M Omega^2)) (synthetic; the paper has
no dataset).  `--workload batched` is the plain 8x8, beta = 8, 256-chain workload alone.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]
"""
import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "indep. samples/s (τ_int-corrected) learned vs plain DQMC; sweeps/s; p50/p99"
UNIT = "chain-sweeps/s"
L2_BYTES = 129 * 2 ** 20


# ------------------------------------------------------------------ flop model
def flops_block_move(p, method):
    """FP64 flops of one block move of one chain, for the algorithm the engine uses.

    Common part, per chunk of m <= n_wrap slices: Householder QR after a one-time column
    ordering 4/3 N^3, explicit Q 4/3 N^3, T update N^3 (not for the first chunk); final LU
    2/3 N^3.  method 0 (per-slice): each slice applies the separable exp(-dtau K),
    2 N^2 (nx + ny), and the exp(-dtau V) scaling, N^2.  method 1 (chunk propagators): per
    chunk the correction vectors (m(m-1)/2 + m(m+1)/2 vector slice applications of
    2 N (nx + ny) + N), the rank-m update 2 m N^2, and a GEMM 2 N^3 (not for the first).
    """
    n, L, nw = p.n_sites, p.n_slices, p.n_wrap
    chunks = [min(nw, L - q * nw) for q in range(math.ceil(L / nw))]
    qr = len(chunks) * (8.0 / 3.0) * n ** 3 + (len(chunks) - 1) * n ** 3 + (2.0 / 3.0) * n ** 3
    if method == 0:
        return L * (2.0 * n * n * (p.nx + p.ny) + n * n) + qr
    vec = 2.0 * n * (p.nx + p.ny) + n
    corr = sum(m * m * vec + 2.0 * m * n * n for m in chunks)
    return corr + (len(chunks) - 1) * 2.0 * n ** 3 + qr


def flops_chunk_build(p):
    """FP64 flops of building one chain's chunk propagators (L slice applications)."""
    n = p.n_sites
    return p.n_slices * (2.0 * n * n * (p.nx + p.ny) + n * n)


def flops_local_phase(p, acc_rate):
    """FP64 flops of one chain's local phase (L slices, restabilised every n_wrap), for a local
    acceptance rate acc_rate.  Per slice: the wrap G <- B G B^-1 through the separable
    propagator on both sides, 2 x 2 N^2 (nx + ny), plus the two diagonal scalings 2 N^2; the
    delayed-update flushes, 2 N^2 per accepted move (N acc_rate moves).  Per chunk of
    m <= n_wrap slices: m slice applications to the right factors, m (2 N^2 (nx + ny) + N^2),
    pre-pivoted QR 4/3 N^3, explicit Q 4/3 N^3, T update N^3, and the two-sided fresh G
    (products and an LU solve), about 4 N^3.  Proposal arithmetic (O(k) per site) is left out.
    """
    n, L, nw = p.n_sites, p.n_slices, p.n_wrap
    chunks = [min(nw, L - q * nw) for q in range(math.ceil(L / nw))]
    per_slice = 4.0 * n * n * (p.nx + p.ny) + 2.0 * n * n + 2.0 * n * n * n * acc_rate
    restab = sum(m * (2.0 * n * n * (p.nx + p.ny) + n * n) + (8.0 / 3.0 + 1.0 + 4.0) * n ** 3 for m in chunks)
    return L * per_slice + restab


def flops_udv_chunk(p, m, first):
    """One chunk of a stabilised product: m slice applications through the separable
    exp(-dtau K) with the exp(-dtau V) scaling, Householder QR after the column ordering
    4/3 N^3, explicit Q 4/3 N^3, T update N^3 (not for the first chunk)."""
    n = p.n_sites
    return m * (2.0 * n * n * (p.nx + p.ny) + n * n) + (8.0 / 3.0) * n ** 3 + (0.0 if first else n ** 3)


def chunk_sizes_top_down(p, stop=0):
    """Chunk lengths of the top-down product from L down to the boundary `stop`."""
    L, nw = p.n_slices, p.n_wrap
    lo, hi, out = ((L - 1) // nw) * nw, L, []
    while True:
        out.append(hi - lo)
        if lo <= stop:
            return out
        hi, lo = lo, lo - nw


def split_boundary(p):
    q = math.ceil(p.n_slices / p.n_wrap)
    return (q // 2) * p.n_wrap if q >= 2 else 0


def flops_split_halves(p):
    """FP64 flops of one chain in the two-half log|det M| launch: the slices above the
    boundary m (top down, chunks of n_wrap from the top) and below it (right factors)."""
    m, nw = split_boundary(p), p.n_wrap
    top = sum(flops_udv_chunk(p, k, j == 0) for j, k in enumerate(chunk_sizes_top_down(p, m)))
    bottom = sum(flops_udv_chunk(p, min(nw, m - s0), s0 == 0) for s0 in range(0, m, nw))
    return top + bottom


def flops_split_join(p):
    """FP64 flops of one chain in the join: two N^3 GEMMs, LU 2/3 N^3, solve 2 N^3, GEMM 2 N^3."""
    n = p.n_sites
    return (4.0 + 2.0 / 3.0 + 2.0 + 2.0) * n ** 3


def flops_stack_build(p):
    """FP64 flops of one chain's stack build: the whole top-down product, LU and G_0 solve."""
    n = p.n_sites
    return sum(flops_udv_chunk(p, k, j == 0) for j, k in enumerate(chunk_sizes_top_down(p))) + (8.0 / 3.0) * n ** 3


# -------------------------------------------------------------- CPU baseline
def _oracle_worker(args):
    params, chain, n_sweeps = args
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    import numpy as np  # noqa: F401
    from oracle import dqmc
    X0 = workloads.initial_fields(params, 1, seed=workloads.DEFAULT_SEED + chain)[0]
    ch = dqmc.OracleChain(params, X0, chain=chain)
    t0 = time.perf_counter()
    for _ in range(n_sweeps):
        ch.sweep()
    return n_sweeps, time.perf_counter() - t0


def oracle_throughput(params, workers, sweeps_per_worker=1, first_chain=0):
    """Oracle chain-sweeps/s with one chain per process (BLAS pinned to one thread)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        res = pool.map(_oracle_worker, [(params, first_chain + w, sweeps_per_worker) for w in range(workers)])
    rate = sum(n / t for n, t in res)
    cpu_s = sum(t for _, t in res)
    return rate, cpu_s


def _oracle_learned_worker(args):
    """One chain of the oracle's learned sampler (seeded random network: its cost per step does
    not depend on the weights), `steps` cumulative steps timed after the initial log|det M|."""
    params, chain, steps, window = args
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    import numpy as np
    from oracle import nn
    x0 = -params.g / (params.mass * params.omega ** 2)
    X0 = workloads.initial_fields(params, 1, seed=workloads.DEFAULT_SEED + chain)[0] + x0
    th = nn.to_bfloat16(nn.init_params(1).astype(np.float32))
    ch = nn.CumulativeChain(params, X0, th, chain=chain)
    t0 = time.perf_counter()
    for k in range(steps):
        ch.step(k, 1, window=window)
    return steps, time.perf_counter() - t0


def oracle_learned_throughput(params, workers, steps, window, first_chain=0):
    """Oracle cumulative steps/s with one chain per process (BLAS pinned to one thread)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        res = pool.map(_oracle_learned_worker, [(params, first_chain + w, steps, window) for w in range(workers)])
    return sum(n / t for n, t in res), sum(t for _, t in res), min(n / t for n, t in res)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def cpu_count():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------------- arms
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def workload_params(name):
    if name == "batched":
        return workloads.BATCHED, workloads.BATCHED_RUN["n_chains"], "batched plain DQMC 8x8 beta=8 L=80"
    if name == "small":
        return workloads.SMALL, 1, "plain DQMC 4x4 beta=4 L=40"
    raise SystemExit(f"unknown workload {name}")


def run_reference_headline(args):
    """The oracle's learned sampler on the headline workload, on the host cores: each step is a
    bounded sample of one cumulative step of as many chains as there are cores (up to 16).  With
    no tau_int measured here, samples/s take tau_int = 1/2 step (at most one independent sample
    per step): an upper bound for the oracle, so the ratio against it is a lower bound."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    big = workloads.LARGEST
    workers = min(cpu_count(), 16)
    for _ in range(args.warmup):
        oracle_learned_throughput(big, workers, 1, args.window)
    rates, cpu_s = [], 0.0
    for k in range(args.steps):
        r, c, _ = oracle_learned_throughput(big, workers, 1, args.window, first_chain=(k * workers) % 64)
        rates.append(r)
        cpu_s += c
    value = statistics.mean(rates)
    unit = "independent samples/s (S_CDW, tau_int-corrected)"
    sample = (f"{workers} chains x 1 cumulative step per step of the oracle's learned sampler (16x16, beta=16, "
              f"window {args.window}), one chain per process, BLAS 1 thread, {cpu_s:.1f} s CPU; tau_int = 1/2 step "
              f"(upper bound on the oracle's samples/s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"16x16 beta=16 L=160 64 chains: learned (patch network, window {args.window}) "
                                   "vs plain", "chains_per_rank": 64},
            "cpu_baseline": {"value": value, "unit": unit, "cores": workers, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload == "headline":
        return run_reference_headline(args)
    params, chains, wname = workload_params(args.workload)
    cores = cpu_count()
    workers = min(cores, chains)
    for _ in range(args.warmup):
        oracle_throughput(params, workers, 1)
    rates, cpu_s = [], 0.0
    for k in range(args.steps):
        r, c = oracle_throughput(params, workers, 1, first_chain=k * workers % chains)
        rates.append(r)
        cpu_s += c
    value = statistics.mean(rates)
    sample = f"{workers} chains x 1 sweep per step, one chain per process, BLAS 1 thread, {cpu_s:.1f} s CPU total"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "chains_per_rank": chains},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    rank, world, local_rank = dist_env()
    params, chains, wname = workload_params(args.workload)
    if args.chains:
        chains = args.chains

    # CPU baseline first (spawned before any CUDA call), rank 0 at N = 1 only.
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        workers = min(cpu_count(), 16)
        rate, cpu_s = oracle_throughput(params, workers, 1)
        cpu = {"value": rate, "unit": UNIT, "cores": workers, "kind": "oracle",
               "sample": f"{workers} chains x 1 sweep of the same workload, one chain per process "
                         f"(BLAS 1 thread), {cpu_s:.1f} s CPU"}

    import numpy as np
    import torch
    import paper_1905_07440_gb300 as hq

    from paper_1905_07440_gb300 import replicas

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=dev)
    stream = torch.cuda.Stream(device=dev)
    # weak scaling: every rank runs `chains` chains, with globally unique Philox chain ids
    first, _ = replicas.shard(chains * world, world, rank)
    X0 = workloads.initial_fields(params, chains, seed=workloads.DEFAULT_SEED + first)

    with torch.cuda.stream(stream):
        peak = hq.fp64_peak_tflops(20, stream.cuda_stream, kind=hq.HQ_PROBE_DFMA)
        eng = hq.Engine(params, chains, first_chain=first, max_series=args.warmup + 2 * args.steps + 4,
                        device=dev, stream=stream)
        eng.set_fields(X0)
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            eng.sweep(1)
        torch.cuda.synchronize(dev)

        def barrier():
            if world > 1:
                torch.distributed.barrier()

        # ---- device-resident timing: one event pair per sweep, L2 flushed between sweeps
        eng.set_timing(True)
        eng.timing()
        uuid = None
        try:
            uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            pass
        clocks = ClockSampler(uuid)
        clocks.start()
        barrier()
        torch.cuda.synchronize(dev)
        evs = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            eng.sweep(1)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize(dev)
        barrier()
        clk = clocks.stop()
        phases = eng.timing()
        eng.set_timing(False)
        t_dev = replicas.max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / 1e3, dev)
        value = chains * world * args.steps / t_dev

        # ---- end to end through the C ABI with host buffers (pinned), copies timed
        Xh = torch.empty(eng.field_shape, dtype=torch.float64, pin_memory=True).numpy()
        Xh[:] = eng.get_fields()
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        obs = None
        for _ in range(args.steps):
            eng.set_fields(Xh)
            eng.sweep(1)
            eng.get_fields(Xh)
            obs = eng.observables()
        t_e2e = replicas.max_over_ranks(time.perf_counter() - t0, dev)
        e2e = chains * world * args.steps / t_e2e
        status_ok = all(o["status"] == 0 for o in obs)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    # roofline of the dominant kernel (largest share of the timed region)
    dom = max(phases, key=lambda k: phases[k][0])
    ms, launches = phases[dom]
    per_launch_s = ms / 1e3 / max(launches, 1)
    kernel_names = {"block_moves": "global_phase_kernel", "local_chunk": "local_phase_kernel",
                    "stack_build": "stack_build_kernel", "sweep_end": "sweep_end_kernel"}
    method = eng.block_move_method
    if dom == "block_moves":
        # one launch = N moves per chain (+ the chunk-propagator build with method 1)
        fl = chains * (params.n_sites * flops_block_move(params, method) +
                       (flops_chunk_build(params) if method == 1 else 0.0))
    else:
        fl = None
    achieved = fl / per_launch_s / 1e12 if fl else None
    # the local phase (wraps, delayed-update flushes, restabilisation) as a second roofline
    acc_l0 = sum(o["local_accepted"] for o in obs) / max(1, sum(o["local_proposed"] for o in obs))
    ms_l, n_l = phases.get("local_chunk", (0.0, 0))
    roof_local = None
    if n_l:
        fl_l = chains * flops_local_phase(params, acc_l0)
        per_sweep_s = ms_l / 1e3 / args.steps
        roof_local = {"bound": "alu", "kernel": "local_phase_kernel", "achieved": fl_l / per_sweep_s / 1e12,
                      "peak": peak, "unit": "TFLOP/s", "frac": fl_l / per_sweep_s / 1e12 / peak,
                      "flops_per_sweep": fl_l, "launches_per_sweep": n_l / args.steps,
                      "ms_per_sweep": ms_l / args.steps}
    gpu_launches = sum(n for _, n in phases.values())
    total_ms = sum(m for m, _ in phases.values())
    xbytes = 8 * chains * params.n_slices * params.n_sites
    obs_bytes = 104 * chains
    acc_l = sum(o["local_accepted"] for o in obs) / max(1, sum(o["local_proposed"] for o in obs))
    acc_g = sum(o["global_accepted"] for o in obs) / max(1, sum(o["global_proposed"] for o in obs))
    indep = None
    tau_path = os.path.join(ROOT, "profiles", f"tau_int_{args.workload}.json")
    if os.path.exists(tau_path):
        with open(tau_path) as f:
            tau = json.load(f)
        indep = {"unit": "independent samples/s", "tau_source": os.path.relpath(tau_path, ROOT),
                 **{k: value / (2.0 * v) for k, v in tau["tau_int"].items()}}
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", f"traffic_global_phase_{args.workload}.json")
    if dom == "block_moves" and os.path.exists(tr_path):
        import hashlib
        with open(tr_path) as f:
            tr = json.load(f)
        src = b"".join(open(os.path.join(ROOT, "paper_1905_07440_gb300", "csrc", x), "rb").read()
                       for x in ("hq_kernels.cu", "hq_device.cuh"))
        if hashlib.sha256(src).hexdigest()[:16] == tr["source_hash"] and chains == workload_params(args.workload)[1]:
            traffic = tr["dram_bytes_per_launch"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_dev * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wname, "lattice": f"{params.nx}x{params.ny}", "beta": params.beta,
                   "block_move_method": ["per-slice", "chunk propagators"][method],
                   "dtau": params.dtau, "L": params.n_slices, "chains_per_rank": chains, "delay_k": params.delay_k,
                   "n_wrap": params.n_wrap, "block_moves_per_sweep": params.n_sites,
                   "parallelism": f"replicas x{world}",
                   "l2": "flushed (512 MB write) before every timed sweep; flush outside the events"},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": xbytes, "d2h_bytes_per_step": xbytes + obs_bytes},
        "gpu_launches": gpu_launches,
        "roofline": {"bound": "alu", "kernel": kernel_names[dom], "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, profiles/" + os.path.basename(tr_path),
                     "peak_source": "FP64 DFMA probe measured in this run (hq_fp64_peak_tflops)",
                     "flops_per_launch": fl, "ms_per_launch": per_launch_s * 1e3,
                     "share": ms / total_ms if total_ms else None},
        "roofline_local": roof_local,
        "phases_ms": {k: v[0] for k, v in phases.items()},
        "indep_samples_per_s": indep,
        "cpu_baseline": cpu,
        "clocks": clk,
        "acceptance": {"local": acc_l, "block": acc_g},
        "status_ok": status_ok,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def series_stats(hq, eng, first, names):
    """Per observable: tau_int (Madras-Sokal, mean over chains), mean and chain error of the
    series from index `first`, and the second-half minus first-half difference with its error."""
    import numpy as np
    out = {}
    for oid, name in names:
        ser = eng.series(oid)[:, first:]
        C, M = ser.shape
        pcm = ser.mean(axis=1)
        h = ser[:, M // 2:].mean(axis=1) - ser[:, : M // 2].mean(axis=1)
        taus = np.array([hq.tau_int(ser[c])[0] for c in range(C)])
        out[name] = {"tau_int": float(taus.mean()), "tau_int_err": float(taus.std(ddof=1) / math.sqrt(C)),
                     "mean": float(pcm.mean()), "err": float(pcm.std(ddof=1) / math.sqrt(C)),
                     "half_diff": float(h.mean()), "half_diff_err": float(h.std(ddof=1) / math.sqrt(C)),
                     "blocks": [round(float(ser[:, k * M // 8:(k + 1) * M // 8].mean()), 4) for k in range(8)]}
    return out


def start_fields(p, chains, amplitude, seed):
    """Starting fields of the headline runs: the charge-ordered pattern (amplitude > 0; beta = 16
    is deep in the ordered phase, where a disordered start coarsens domains for hundreds of
    steps) or the mean field with the free-phonon spread (amplitude 0)."""
    if amplitude > 0:
        return workloads.ordered_fields(p, chains, amplitude, seed=seed)
    return workloads.initial_fields(p, chains, seed=seed) - p.g / (p.mass * p.omega ** 2)


def run_headline(args):
    """Learned vs plain at 16x16, beta = 16 (L = 160), 64 chains per GPU (see the module doc)."""
    rank, world, local_rank = dist_env()
    big, C = workloads.LARGEST, workloads.LARGEST_RUN["n_chains"]
    if args.chains:
        C = args.chains
    small = big.with_(nx=8, ny=8)
    x0 = -big.g / (big.mass * big.omega ** 2)
    W = args.window

    # CPU baseline first (spawned before any CUDA call), rank 0 at N = 1 only: the oracle's
    # learned sampler on the same workload, one chain per host core
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        workers = min(cpu_count(), 16)
        rate, cpu_s, slowest = oracle_learned_throughput(big, workers, args.cpu_steps, W)
        cpu = {"steps_per_s": rate, "per_core_steps_per_s": rate / workers, "cores": workers, "cpu_s": cpu_s,
               "cpu_model": cpu_model()}

    import numpy as np
    import torch
    import paper_1905_07440_gb300 as hq
    from paper_1905_07440_gb300 import replicas

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=dev)
    stream = torch.cuda.Stream(device=dev)
    first, _ = replicas.shard(C * world, world, rank)
    names = ((hq.HQ_OBS_X2, "x2"), (hq.HQ_OBS_DOUBLE_OCC, "double_occ"), (hq.HQ_OBS_SCDW, "s_cdw"))
    K, Wm = args.steps, args.warmup
    t_all = time.perf_counter()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        peak = hq.fp64_peak_tflops(20, stream.cuda_stream, kind=hq.HQ_PROBE_DFMA)
        dgemm = measure_dgemm(dev)
        # ---- 1. training data: plain local sweeps on the deployment lattice (one chain per SM) from
        # the mean-field start, fresh Philox key; the exact log|det M| comes with every local sweep.
        # (Measured alternatives: networks fitted to 8x8 configurations, ordered or not, are
        # accepted far less often on the ordered 16x16 lattice.)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        t0 = time.perf_counter()
        TC = sms
        tr = hq.Engine(big.with_(seed=big.seed + 7), TC, first_chain=first, device=dev, stream=stream)
        tr.set_fields(start_fields(big, TC, args.train_start_amplitude, workloads.DEFAULT_SEED + 5000 + first))
        tr.sweep(args.train_warmup, global_=False)
        Xs, ys = [], []
        for _ in range(args.train_snapshots):
            tr.sweep(1, global_=False)
            Xs.append(tr.get_fields())
            ys.append(tr.log_weight()[1])
        tr.close()
        t_data = time.perf_counter() - t0
        # chains split 75/25 into training and held-out test configurations
        ntr = (3 * TC) // 4
        Xall, yall = np.stack(Xs, axis=1), np.stack(ys, axis=1)
        Xtr, ytr = Xall[:ntr].reshape((-1,) + Xall.shape[2:]), yall[:ntr].reshape(-1)
        Xte, yte = Xall[ntr:].reshape((-1,) + Xall.shape[2:]), yall[ntr:].reshape(-1)
        del Xall
        ymu = ytr.mean()
        ytr, yte = ytr - ymu, yte - ymu
        # ---- 2. network training on the tensor cores (lr halved every third of the epochs)
        net = hq.Engine(big, 1, device=dev, stream=stream)
        net.attach_network(64, Xtr.shape[0])
        net.set_params(hq.init_network(args.nn_seed))
        Xd, yd = torch.from_numpy(Xtr).to(dev), torch.from_numpy(ytr).to(dev)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        losses = []
        for k in range(3):
            ep = args.epochs // 3 + (args.epochs % 3 if k == 2 else 0)
            losses.extend(net.nn_train(Xd, yd, epochs=ep, batch=64, lr=args.lr * 0.5 ** k, seed=args.nn_seed + k))
        torch.cuda.synchronize(dev)
        t_train = time.perf_counter() - t1
        test_mse, nt = 0.0, 0
        for a0 in range(0, Xte.shape[0], 64):
            nb = min(64, Xte.shape[0] - a0)
            _, l = net.nn_gradient(torch.from_numpy(Xte[a0:a0 + nb]).to(dev), torch.from_numpy(yte[a0:a0 + nb]).to(dev))
            test_mse += l * nb
            nt += nb
        test_rms = math.sqrt(test_mse / nt)
        theta = net.get_params()
        net.close()
        del Xd, yd
        # ---- 3. learned sampler at 16x16: relaxation, timed steps, then the tau series
        lrn = hq.Engine(big, C, first_chain=first, max_series=args.relax_max + Wm + K + args.tau_steps + 4,
                        device=dev, stream=stream)
        lrn.attach_network(4, 8)
        lrn.set_params(theta)
        lrn.set_inner_window(W)
        split_m = lrn.set_logdet_split(0)
        lrn.set_fields(start_fields(big, C, args.start_amplitude, workloads.DEFAULT_SEED + first))
        blk = args.inner_block_sites > 0
        if blk:
            lrn.set_inner_sites(args.inner_block_sites)
        # relaxation: at least args.relax steps, then in chunks of 100 until the last 200 steps'
        # halves agree within two error bars for X^2, D and S_CDW, at most args.relax_max steps
        lrn.cumulative(args.relax, 1, global_=blk, measure=True)
        relaxed = args.relax
        while True:
            st_r = series_stats(hq, lrn, relaxed - min(200, relaxed), names)
            ok = all(abs(v["half_diff"]) <= 2.0 * v["half_diff_err"] for v in st_r.values())
            if ok or relaxed + 100 > args.relax_max:
                break
            lrn.cumulative(100, 1, global_=blk, measure=True)
            relaxed += 100
        lrn.cumulative(Wm, 1, global_=blk, measure=True)
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
        torch.cuda.synchronize(dev)
        lrn.set_timing(True)
        lrn.timing()
        uuid = None
        try:
            uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            pass
        clocks = ClockSampler(uuid)
        clocks.start()
        barrier()
        torch.cuda.synchronize(dev)
        evs = []
        for _ in range(K):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lrn.cumulative(1, 1, global_=blk, measure=True)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize(dev)
        barrier()
        clk = clocks.stop()
        phases = lrn.timing()
        lrn.set_timing(False)
        t_dev = replicas.max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / 1e3, dev)
        step_rate = C * world * K / t_dev
        lrn.cumulative(args.tau_steps, 1, global_=blk, measure=True)
        stats = series_stats(hq, lrn, relaxed + Wm, names)
        st = lrn.learned_stats()
        acc = sum(x["cumulative_accepted"] for x in st) / max(1, sum(x["cumulative_proposed"] for x in st))
        # ---- 4. end to end through the C ABI with host buffers (pinned), copies timed
        Xh = torch.empty(lrn.field_shape, dtype=torch.float64, pin_memory=True).numpy()
        Xh[:] = lrn.get_fields()
        barrier()
        torch.cuda.synchronize(dev)
        te = time.perf_counter()
        for _ in range(args.e2e_steps):
            lrn.set_fields(Xh)
            lrn.cumulative(1, 1, global_=blk, measure=True)
            lrn.get_fields(Xh)
            obs = lrn.observables()
        t_e2e = replicas.max_over_ranks(time.perf_counter() - te, dev)
        status_ok = all(o["status"] == 0 for o in obs)
        Xeq = lrn.get_fields()
        lrn.close()
        # ---- 5. plain sampler at 16x16 from the learned chains' fields, fresh Philox key: one
        # full sweep with block moves on a run of sites, scaled to a block move per site
        pl = hq.Engine(big.with_(seed=big.seed + 11), C, first_chain=first, device=dev, stream=stream)
        pl.set_block_sites(args.plain_block_sites)
        pl.set_fields(Xeq)
        pl.sweep(1)
        pl.set_timing(True)
        pl.timing()
        pl.sweep(1)
        ph = pl.timing()
        pl.set_timing(False)
        pobs = pl.observables()
        pl.close()
        S = min(args.plain_block_sites or big.n_sites, big.n_sites)
        t_full = (ph["stack_build"][0] + ph["local_chunk"][0] + ph["sweep_end"][0] +
                  ph["block_moves"][0] * big.n_sites / S) / 1e3
        t_full = replicas.max_over_ranks(t_full, dev)
        # ---- 6. the plain batched workload (8x8, beta = 8, 256 chains) as a second line
        sec = measure_batched(args, hq, dev, stream, world, first, peak, dgemm, steps=args.batched_steps) \
            if args.batched_steps > 0 else None

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    tau = {k: v["tau_int"] for k, v in stats.items()}
    indep = {k: step_rate / (2.0 * tau[k]) for k in tau}
    plain_bound = C * world / t_full
    # roofline of the dominant kernel of the timed steps
    dom = max(phases, key=lambda k: phases[k][0])
    ms, launches = phases[dom]
    per_launch_s = ms / 1e3 / max(launches, 1)
    kernel_names = {"split_halves": "split_halves_kernel", "split_join": "split_join_kernel",
                    "stack_build": "stack_build_kernel", "network_inner": "nn_inner_kernel",
                    "network_eval": "nn_eval_kernel", "sweep_end": "measure_g0_kernel + sweep_end_kernel"}
    fl = {"split_halves": C * flops_split_halves(big), "split_join": C * flops_split_join(big),
          "stack_build": C * flops_stack_build(big)}.get(dom)
    achieved = fl / per_launch_s / 1e12 if fl else None
    total_ms = sum(m for m, _ in phases.values())
    # DRAM traffic per launch of the dominant kernel from an ncu record of the same source
    traffic, tr_src = None, None
    tr_path = os.path.join(ROOT, "profiles", f"traffic_{kernel_names.get(dom, dom)}_largest.json")
    if os.path.exists(tr_path) and C == workloads.LARGEST_RUN["n_chains"]:
        import hashlib
        with open(tr_path) as f:
            tr = json.load(f)
        src = b"".join(open(os.path.join(ROOT, "paper_1905_07440_gb300", "csrc", x), "rb").read()
                       for x in ("hq_kernels.cu", "hq_device.cuh"))
        if hashlib.sha256(src).hexdigest()[:16] == tr["source_hash"]:
            traffic, tr_src = tr["dram_bytes_per_launch"], "profiles/" + os.path.basename(tr_path)
    xbytes = 8 * C * big.n_slices * big.n_sites
    e2e = C * world * args.e2e_steps / t_e2e / (2.0 * tau["s_cdw"])
    if cpu is not None:
        cpu = {"value": cpu["steps_per_s"] / (2.0 * tau["s_cdw"]), "unit": "independent samples/s (S_CDW)",
               "cores": cpu["cores"], "kind": "oracle",
               "per_core": cpu["per_core_steps_per_s"] / (2.0 * tau["s_cdw"]),
               "steps_per_s": cpu["steps_per_s"], "cpu_model": cpu["cpu_model"],
               "sample": f"{cpu['cores']} chains x {args.cpu_steps} cumulative steps of the oracle's learned sampler "
                         f"(16x16, beta=16, window {W}, random network), one chain per process, BLAS 1 thread, "
                         f"{cpu['cpu_s']:.1f} s CPU; samples/s with this run's tau_int(S_CDW)"}
    line = {
        "metric": METRIC, "value": indep["s_cdw"], "unit": "independent samples/s (S_CDW, tau_int-corrected)",
        "n_gpus": world, "steps": K, "warmup": Wm, "ms_per_step": t_dev * 1e3 / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (determinants); bf16 operands / fp32 accumulation "
                                                          "(network)", "data": "synthetic",
        "config": {"workload": f"16x16 beta=16 L=160 {C} chains: learned (patch network, window {W}) vs plain",
                   "learned_moves": (f"local moves on a window of {W} slices" + (
                       f" + block moves on {args.inner_block_sites} sites" if blk else ", no block moves")
                                     + " per cumulative step"),
                   "lattice": "16x16", "beta": big.beta, "dtau": big.dtau, "L": big.n_slices, "chains_per_rank": C,
                   "n_wrap": big.n_wrap, "delay_k": big.delay_k, "parallelism": f"replicas x{world}",
                   "logdet_split_boundary": split_m,
                   "start": (f"charge-ordered: -g/(M Omega^2) + {args.start_amplitude} (-1)^(x+y) + N(0, 1/(2 M Omega))"
                             if args.start_amplitude > 0 else "mean field + N(0, 1/(M Omega^2))"),
                   "l2": "flushed (512 MB write) before every timed step; flush outside the events"},
        "learned": {"chain_steps_per_s": step_rate, "tau_int_steps": tau, "indep_samples_per_s": indep,
                    "cumulative_acceptance": acc, "observables": stats, "relax_steps": relaxed + Wm,
                    "relax_window_stationary_2sigma": ok,
                    "measured_steps": K + args.tau_steps,
                    "stationary_2sigma": all(abs(v["half_diff"]) <= 2.0 * v["half_diff_err"] for v in stats.values())},
        "plain": {"seconds_per_full_sweep": t_full, "chain_sweeps_per_s": plain_bound,
                  "indep_samples_per_s_upper_bound": plain_bound,
                  "protocol": f"local moves at every (l, i) + one block move per site; timed with block moves on "
                              f"{S} sites and scaled per move; tau_int >= 1/2 sweep bounds the samples/s",
                  "phases_ms": {k: v[0] for k, v in ph.items() if v[1]},
                  "block_acceptance": sum(o["global_accepted"] for o in pobs) / max(1, sum(o["global_proposed"] for o in pobs))},
        "gain_lower_bound": {k: indep[k] / plain_bound for k in indep},
        "training": {"lattice": "16x16", "source": f"plain local sweeps, {TC} chains from the "
                                                  f"{'ordered' if args.train_start_amplitude > 0 else 'mean-field'} start, "
                                                  f"{args.train_warmup} warm-up sweeps, one snapshot per sweep, "
                                                  f"chains split 75/25 into training and test",
                     "samples": int(Xtr.shape[0]), "test_samples": int(Xte.shape[0]), "data_s": t_data,
                     "train_s": t_train, "test_rms": test_rms, "test_target_sd": float(yte.std()),
                     "epochs": args.epochs, "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
                     "target_variance": float(np.var(ytr))},
        "e2e": {"value": e2e, "unit": "independent samples/s (S_CDW, tau_int-corrected)",
                "h2d_bytes_per_step": xbytes, "d2h_bytes_per_step": xbytes + 104 * C,
                "note": "per step: fields in from pinned host memory (state rebuilt), one cumulative step, fields "
                        "and observables out"},
        "gpu_launches": sum(n for _, n in phases.values()) + K,
        "roofline": {"bound": "alu", "kernel": kernel_names.get(dom, dom), "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "traffic_source": tr_src,
                     "peak_source": "FP64 DFMA probe measured in this run (hq_fp64_peak_tflops)",
                     "frac_vs_cublas_dgemm": (achieved / dgemm) if (achieved and dgemm) else None,
                     "cublas_dgemm_tflops": dgemm, "flops_per_launch": fl, "ms_per_launch": per_launch_s * 1e3,
                     "share": ms / total_ms if total_ms else None},
        "phases_ms_per_step": {k: v[0] / K for k, v in phases.items() if v[1]},
        "cpu_baseline": cpu,
        "clocks": clk,
        "status_ok": status_ok,
        "batched_plain_8x8": sec,
        "wall_s": time.perf_counter() - t_all,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def measure_dgemm(dev, n=4096, reps=4):
    """cuBLAS DGEMM TFLOP/s (torch.matmul in float64), the second FP64 denominator."""
    import torch
    x = torch.randn(n, n, dtype=torch.float64, device=dev)
    y = x @ x
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        y = x @ x
    b.record()
    torch.cuda.synchronize(dev)
    del x, y
    return 2.0 * n ** 3 * reps / (a.elapsed_time(b) / 1e3) / 1e12


def measure_batched(args, hq, dev, stream, world, first, peak, dgemm, steps=5, warmup=3):
    """The plain batched workload (8x8, beta = 8, L = 80, 256 chains per GPU): device-timed
    sweeps with the L2 flushed between them, and the roofline of its dominant phase."""
    import torch
    from paper_1905_07440_gb300 import replicas
    params, chains = workloads.BATCHED, workloads.BATCHED_RUN["n_chains"]
    eng = hq.Engine(params.with_(seed=params.seed + 3), chains, first_chain=first, max_series=warmup + steps + 2,
                    device=dev, stream=stream)
    eng.set_fields(workloads.initial_fields(params, chains, seed=workloads.DEFAULT_SEED + first))
    eng.sweep(warmup)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize(dev)
    eng.set_timing(True)
    eng.timing()
    evs = []
    for _ in range(steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        eng.sweep(1)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize(dev)
    phases = eng.timing()
    eng.set_timing(False)
    obs = eng.observables()
    method = eng.block_move_method
    eng.close()
    t_dev = replicas.max_over_ranks(sum(a.elapsed_time(b) for a, b in evs) / 1e3, dev)
    ms_b, n_b = phases["block_moves"]
    fl = chains * (params.n_sites * flops_block_move(params, method) + (flops_chunk_build(params) if method == 1 else 0.0))
    achieved = fl / (ms_b / 1e3 / max(n_b, 1)) / 1e12 if n_b else None
    acc_l = sum(o["local_accepted"] for o in obs) / max(1, sum(o["local_proposed"] for o in obs))
    ms_l = phases["local_chunk"][0]
    fl_l = chains * flops_local_phase(params, acc_l)
    return {"workload": "batched plain DQMC 8x8 beta=8 L=80", "chains_per_rank": chains,
            "value": chains * world * steps / t_dev, "unit": UNIT, "ms_per_sweep": t_dev * 1e3 / steps,
            "roofline_block_moves": {"kernel": "global_phase_kernel", "achieved": achieved, "peak": peak,
                                     "frac": achieved / peak if achieved else None,
                                     "frac_vs_cublas_dgemm": achieved / dgemm if achieved else None},
            "roofline_local_phase": {"kernel": "local_phase_kernel", "achieved": fl_l / (ms_l / 1e3 / steps) / 1e12,
                                     "frac": fl_l / (ms_l / 1e3 / steps) / 1e12 / peak},
            "phases_ms_per_sweep": {k: v[0] / steps for k, v in phases.items() if v[1]}}


def run_tau(args):
    """Integrated autocorrelation times of the per-sweep observables on the workload.

    Runs args.warmup sweeps to equilibrate, then args.tau_sweeps measured sweeps of every
    chain; tau_int of each chain's series (Madras-Sokal window, c = 6) averaged over chains.
    """
    import numpy as np
    import torch
    import paper_1905_07440_gb300 as hq
    params, chains, wname = workload_params(args.workload)
    if args.chains:
        chains = args.chains
    S = args.tau_sweeps
    eng = hq.Engine(params, chains, max_series=args.warmup + S)
    eng.set_fields(workloads.initial_fields(params, chains))
    eng.sweep(args.warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eng.sweep(S)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out = {"workload": wname, "chains": chains, "warmup_sweeps": args.warmup, "sweeps": S,
           "chain_sweeps_per_s": chains * S / wall, "tau_int": {}, "tau_int_stderr": {}, "mean": {}}
    for oid, name in ((hq.HQ_OBS_X2, "x2"), (hq.HQ_OBS_DOUBLE_OCC, "double_occ"), (hq.HQ_OBS_SCDW, "s_cdw"),
                      (hq.HQ_OBS_DENSITY, "density")):
        ser = eng.series(oid)[:, args.warmup:]
        taus = np.array([hq.tau_int(ser[c])[0] for c in range(chains)])
        out["tau_int"][name] = float(taus.mean())
        out["tau_int_stderr"][name] = float(taus.std(ddof=1) / math.sqrt(chains)) if chains > 1 else None
        out["mean"][name] = float(ser.mean())
    print(json.dumps(out), flush=True)
    return 0


def run_learned(args):
    """Learned vs plain sampler on the batched workload (8x8, beta = 8, 256 chains).

    With --cnn the block moves of the inner chain use the convolutional action, trained on the
    same samples; local moves always use the patch network.

    1. Plain sampler: warm-up, then training samples (fields and exact log|det M|).
    2. Network training on those samples (the library's kernels).
    3. Learned sampler (cumulative steps of args.n_inner network sweeps, exact accept) from the
       equilibrated plain fields: timed steps/s, then tau_int of the per-step series.
    4. Plain sampler timed on the same fields; its tau_int from the committed measurement.
    Independent samples/s = chains * (steps or sweeps)/s / (2 tau_int), per observable.
    """
    import numpy as np
    import torch
    import paper_1905_07440_gb300 as hq
    params, C, wname = workload_params("batched")
    if args.chains:
        C = args.chains
    dev = torch.device("cuda", 0)
    t_all = time.perf_counter()
    eng = hq.Engine(params, C, max_series=8)
    eng.set_fields(workloads.initial_fields(params, C))
    eng.sweep(args.train_warmup)
    Xs, ys = [], []
    for _ in range(args.train_snapshots):
        eng.sweep(2)
        Xs.append(eng.get_fields())
        ys.append(eng.log_weight()[1])
    Xtr = np.concatenate(Xs)
    ytr = np.concatenate(ys)
    ytr -= ytr.mean()
    X_eq = eng.get_fields()
    eng.close()
    net = hq.Engine(params, 1)
    net.attach_network(64, Xtr.shape[0])
    net.set_params(hq.init_network(args.nn_seed))
    Xd, yd = torch.from_numpy(Xtr).to(dev), torch.from_numpy(ytr).to(dev)
    t0 = time.perf_counter()
    # learning rate halved every third of the epochs (Adam state carries over)
    losses = []
    for k in range(3):
        ep = args.epochs // 3 + (args.epochs % 3 if k == 2 else 0)
        losses.extend(net.nn_train(Xd, yd, epochs=ep, batch=64, lr=args.lr * 0.5 ** k, seed=args.nn_seed + k))
    t_train = time.perf_counter() - t0
    theta = net.get_params()
    theta_cnn, closs = None, None
    if args.cnn:
        # convolutional action for block moves, fitted to the same targets
        net.cnn_set_params(hq.init_cnn(args.nn_seed))
        t1 = time.perf_counter()
        closs = []
        for k in range(3):
            ep = args.epochs // 3 + (args.epochs % 3 if k == 2 else 0)
            closs.extend(net.cnn_train(Xd, yd, epochs=ep, batch=64, lr=args.cnn_lr * 0.5 ** k,
                                       seed=args.nn_seed + 10 + k))
        t_train_cnn = time.perf_counter() - t1
        theta_cnn = net.cnn_get_params()
    del Xd, yd
    net.close()
    # learned sampler
    steps = args.tau_steps
    lrn = hq.Engine(params, C, max_series=steps + args.warmup + args.steps + 4)
    lrn.attach_network(4, 8)
    lrn.set_params(theta)
    lrn.set_inner_window(args.window)
    lrn.set_inner_sites(args.sites)
    if theta_cnn is not None:
        lrn.cnn_set_params(theta_cnn)
    use_cnn = theta_cnn is not None
    lrn.set_fields(X_eq)
    lrn.cumulative(args.warmup, args.n_inner, measure=True, cnn=use_cnn)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    lrn.cumulative(args.steps, args.n_inner, measure=True, cnn=use_cnn)
    b.record()
    torch.cuda.synchronize()
    step_rate = C * args.steps / (a.elapsed_time(b) / 1e3)
    lrn.cumulative(steps, args.n_inner, measure=True, cnn=use_cnn)
    st = lrn.learned_stats()
    acc = sum(x["cumulative_accepted"] for x in st) / max(1, sum(x["cumulative_proposed"] for x in st))
    inner_l = sum(x["inner_local_accepted"] for x in st) / max(1, sum(x["inner_local_proposed"] for x in st))
    inner_b = sum(x["inner_block_accepted"] for x in st) / max(1, sum(x["inner_block_proposed"] for x in st))
    first = args.warmup + args.steps
    tau_l, indep_l, means = {}, {}, {}
    for oid, name in ((hq.HQ_OBS_X2, "x2"), (hq.HQ_OBS_DOUBLE_OCC, "double_occ"), (hq.HQ_OBS_SCDW, "s_cdw")):
        ser = lrn.series(oid)[:, first:]
        tau_l[name] = float(np.mean([hq.tau_int(ser[c])[0] for c in range(C)]))
        indep_l[name] = step_rate / (2.0 * tau_l[name])
        means[name] = float(ser.mean())
    # plain sampler, same fields
    pl = hq.Engine(params, C, max_series=8)
    pl.set_fields(X_eq)
    pl.sweep(1)
    torch.cuda.synchronize()
    a.record()
    pl.sweep(args.steps)
    b.record()
    torch.cuda.synchronize()
    sweep_rate = C * args.steps / (a.elapsed_time(b) / 1e3)
    with open(os.path.join(ROOT, "profiles", "tau_int_batched.json")) as f:
        tau_p = json.load(f)["tau_int"]
    indep_p = {k: sweep_rate / (2.0 * tau_p[k]) for k in indep_l}
    line = {"metric": METRIC, "mode": "learned vs plain", "value": indep_l["s_cdw"],
            "unit": "independent samples/s of S_CDW(pi,pi) (learned)", "higher_is_better": True,
            "dtype": "f64 weights, bf16-weight/fp32 network", "data": "synthetic",
            "config": {"workload": wname, "chains": C, "n_inner": args.n_inner, "window": args.window, "sites": args.sites, "train_samples": int(Xtr.shape[0]),
                       "epochs": args.epochs, "lr": args.lr},
            "learned": {"cumulative_steps_per_s": step_rate, "tau_int_steps": tau_l, "indep_samples_per_s": indep_l,
                        "cumulative_acceptance": acc, "inner_local_acceptance": inner_l,
                        "inner_block_acceptance": inner_b, "means": means},
            "plain": {"chain_sweeps_per_s": sweep_rate, "tau_int_sweeps": tau_p, "indep_samples_per_s": indep_p},
            "gain": {k: indep_l[k] / indep_p[k] for k in indep_l},
            "training": {"seconds": t_train, "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
                         "target_variance": float(np.var(ytr))},
            "block_moves": "convolutional action" if use_cnn else "patch network",
            "cnn_training": None if not use_cnn else {"seconds": t_train_cnn, "loss_first": float(closs[0]),
                                                      "loss_last": float(closs[-1]), "lr": args.cnn_lr},
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)
    return 0


SERVING_SIDES = (6, 8, 10, 12, 16)
SERVING_BETAS = (4.0, 8.0, 12.0)
SERVING_LAMBDAS = (0.15, 0.25, 0.35)


def serving_params(side, beta, lam, seed):
    """Holstein parameters of one request: t = M = Omega = 1, g from lambda = g^2/(M Omega^2 8t),
    half filling mu = -g^2/(M Omega^2)."""
    g = math.sqrt(8.0 * lam)
    return workloads.HolsteinParams(nx=side, ny=side, beta=beta, g=g, mu=-g * g, seed=seed)


def run_serving(args):
    """Continuous-batching service under Poisson arrivals, on the serving workload's shape: lattice
    side in {6, 8, 10, 12, 16}, beta in {4, 8, 12}, lambda in {0.15, 0.25, 0.35} (45 kinds, drawn
    uniformly in stratified runs of 45 so every kind appears), learned or plain sampler per request.  Stated reductions: args.duration seconds of
    arrivals at args.rate per second (not 1000 requests), args.req_sweeps sweeps or cumulative steps
    per request (not 500), plain block moves on a run of args.serve_block_sites sites per sweep (a
    full sweep at 16x16, beta = 12 is about a minute of block moves).  Learned requests carry a small
    seeded network (the cumulative accept keeps them exact whatever it is).  Reported: served
    chain-sweeps/s, latency (arrival to result on the host) percentiles overall and per kind, queueing
    delay, and one request of each (side, beta, sampler) served alone on an idle GPU against the same
    kinds in the mix."""
    import numpy as np
    import torch
    import paper_1905_07440_gb300 as hq
    from paper_1905_07440_gb300.serving import GpuBackend, Request, Server

    theta = hq.init_network(args.nn_seed, out_scale=0.1)
    rng = np.random.default_rng(args.serve_seed)
    all_kinds = [(s_, b_, l_) for s_ in SERVING_SIDES for b_ in SERVING_BETAS for l_ in SERVING_LAMBDAS]
    order = []
    reqs, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / args.rate)
        if t > args.duration:
            break
        k = len(reqs)
        # kinds uniform but stratified: each run of 45 requests visits every kind once, in random
        # order, so a reduced request count still covers all of them
        if not order:
            order = [all_kinds[j] for j in rng.permutation(len(all_kinds))]
        side, beta, lam = order.pop()
        side, beta, lam = int(side), float(beta), float(lam)
        sampler = "learned" if rng.random() < args.learned_frac else "plain"
        p = serving_params(side, beta, lam, workloads.BATCHED.seed + 7919 * k)
        r = Request(rid=k, params=p, X0=workloads.initial_fields(p, 1, seed=10_000 + k)[0] - p.g / (p.mass * p.omega ** 2),
                    sweeps=args.req_sweeps, sampler=sampler, theta=theta if sampler == "learned" else None,
                    chain_id=k, arrival=t)
        r.kind = (side, beta, lam, sampler)
        reqs.append(r)

    def backend():
        return GpuBackend(block_sites=args.serve_block_sites, window=args.serve_window)

    def server():
        return Server(backend(), args.hbm_budget, args.slots, max_pools=args.max_pools)

    # warm-up: one request of each lattice side and sampler (kernel loading, allocator)
    warm = [Request(rid=-1, params=serving_params(s_, 4.0, 0.25, 1), X0=workloads.initial_fields(
        serving_params(s_, 4.0, 0.25, 1), 1)[0], sweeps=1, sampler=sm, theta=theta)
        for s_ in SERVING_SIDES for sm in ("plain", "learned")]
    server().run(warm)
    torch.cuda.synchronize()
    peak = {"bytes": 0, "pools": 0}

    class Tracking(Server):
        def poll(self):
            super().poll()
            peak["bytes"] = max(peak["bytes"], self.used)
            peak["pools"] = max(peak["pools"], len(self.pools))

    srv = Tracking(backend(), args.hbm_budget, args.slots, max_pools=args.max_pools)
    sampler = ClockSampler()
    sampler.start()
    t0 = time.perf_counter()
    done = srv.run(reqs)
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
    lat = np.array([r.done - r.arrival for r in done]) * 1e3
    wait = np.array([r.admitted - r.arrival for r in done]) * 1e3
    kinds = {}
    for r in done:
        kinds.setdefault(r.kind, []).append((r.done - r.arrival) * 1e3)
    by_kind = {f"{s_}x{s_} beta={b:g} lambda={l:g} {sm}": {"n": len(v), "p50": pct(np.array(v), 50),
                                                          "max": float(max(v))}
               for (s_, b, l, sm), v in sorted(kinds.items())}
    by_side = {}
    for side in SERVING_SIDES:
        lk = np.array([r.done - r.arrival for r in done if r.kind[0] == side]) * 1e3
        by_side[f"{side}x{side}"] = {"n": int(lk.size), "p50": pct(lk, 50), "p99": pct(lk, 99)}
    # one request of each (side, beta, sampler) alone (lambda = 0.25) against the same kinds in the mix
    alone = {}
    for side in SERVING_SIDES:
        for beta in SERVING_BETAS:
            for sm in ("plain", "learned"):
                p = serving_params(side, beta, 0.25, 123)
                r = Request(rid=0, params=p, X0=workloads.initial_fields(p, 1, seed=5)[0] - p.g / (p.mass * p.omega ** 2),
                            sweeps=args.req_sweeps, sampler=sm, theta=theta if sm == "learned" else None)
                a = time.perf_counter()
                server().run([r])
                mixed = np.array([x.done - x.arrival for x in done if x.kind[0] == side and x.kind[1] == beta
                                  and x.kind[3] == sm]) * 1e3
                alone[f"{side}x{side} beta={beta:g} {sm}"] = {"alone_ms": (time.perf_counter() - a) * 1e3,
                                                               "mix_p50_ms": pct(mixed, 50), "mix_n": int(mixed.size)}
    served = sum(r.sweeps for r in done)
    n_learned = sum(1 for r in done if r.sampler == "learned")
    line = {"metric": METRIC, "mode": "serving", "value": served / wall, "unit": "chain-sweeps/s (served)",
            "higher_is_better": True, "dtype": "f64 (learned requests: bf16-operand/fp32 network)", "data": "synthetic",
            "config": {"workload": "Poisson arrivals; side in %s, beta in %s, lambda in %s (45 kinds), learned "
                                   "fraction %g" % (SERVING_SIDES, SERVING_BETAS, SERVING_LAMBDAS, args.learned_frac),
                       "rate_per_s": args.rate, "duration_s": args.duration, "sweeps_per_request": args.req_sweeps,
                       "plain_block_sites": args.serve_block_sites, "learned_window": args.serve_window,
                       "slots_per_pool": args.slots, "max_pools": args.max_pools, "hbm_budget_bytes": args.hbm_budget,
                       "reductions": "request count (duration x rate, not 1000), sweeps per request (not 500), "
                                     "plain block moves on a run of sites"},
            "requests": len(done), "learned_requests": n_learned, "kinds_served": len(kinds), "wall_s": wall,
            "requests_per_s": len(done) / wall,
            "latency_ms": {"p50": pct(lat, 50), "p90": pct(lat, 90), "p99": pct(lat, 99), "max": float(lat.max())},
            "queue_ms": {"p50": pct(wait, 50), "p99": pct(wait, 99)}, "latency_by_side_ms": by_side,
            "latency_by_kind_ms": by_kind, "alone_vs_mix": alone, "peak_pool_bytes": int(peak["bytes"]),
            "peak_pools": peak["pools"], "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


HETERO_MIX = ((dict(nx=4, ny=4, beta=4.0), 64), (dict(nx=6, ny=6, beta=4.0), 64), (dict(nx=8, ny=8, beta=4.0), 48),
              (dict(nx=10, ny=10, beta=2.0), 32), (dict(nx=12, ny=12, beta=2.0), 16))


def run_hetero(args):
    """Heterogeneous batching: engines of five lattice shapes (224 chains) swept (a) one
    engine after another on one stream, (b) each engine on its own stream, (c) as one group
    (one persistent launch per sweep).  Value: chain-sweeps/s of (c)."""
    import torch
    import paper_1905_07440_gb300 as hq

    def engines(streams):
        out = []
        for k, (shape, C) in enumerate(HETERO_MIX):
            p = workloads.HolsteinParams(**shape, seed=workloads.BATCHED.seed + k)
            e = hq.Engine(p, C, stream=torch.cuda.Stream() if streams else torch.cuda.current_stream())
            e.set_fields(workloads.initial_fields(p, C, seed=k))
            out.append(e)
        return out

    total = sum(C for _, C in HETERO_MIX)
    res = {}
    for mode in ("sequential", "streams", "group"):
        engs = engines(mode == "streams")
        grp = hq.Group(engs) if mode == "group" else None

        def step():
            if grp is not None:
                grp.sweep(1)
            else:
                for e in engs:
                    e.sweep(1)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize()
        res[mode] = total * args.steps / (time.perf_counter() - t0)
        if grp is not None:
            grp.close()
        for e in engs:
            e.close()
    line = {"metric": METRIC, "mode": "heterogeneous batching", "value": res["group"], "unit": "chain-sweeps/s",
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "; ".join(f"{s['nx']}x{s['ny']} beta={s['beta']:g} x{C}" for s, C in HETERO_MIX),
                       "chains": total, "steps": args.steps, "warmup": args.warmup,
                       "timing": "host wall clock, synchronised"},
            "chain_sweeps_per_s": res, "group_vs_sequential": res["group"] / res["sequential"],
            "group_vs_streams": res["group"] / res["streams"]}
    print(json.dumps(line), flush=True)
    return 0


PHYSICS_SIDES = ((4, 48), (6, 48), (8, 32), (10, 16), (12, 16))
PHYSICS_OBS_SIDES = (4, 6, 8, 10)  # observables; 12x12 (2.7 s per chain-sweep) is timed only


def physics_params(side, seed):
    """The paper's benchmark point: Omega = t/2, lambda = g^2/(M Omega^2 8t) = 1/2 (g = 1),
    half filling mu = -g^2/(M Omega^2) = -4, beta = 4.1 (its T_c), dtau = 0.1 (L = 41)."""
    return workloads.HolsteinParams(nx=side, ny=side, omega=0.5, g=1.0, mu=-4.0, beta=4.1, seed=seed)


def run_physics(args):
    """The paper's physics point on lattice sides 4..12: S_CDW(pi,pi), <n>, <X> from one
    heterogeneous group (all sizes in one persistent launch), and the GPU time of one
    chain-sweep against N with its power-law exponent (the paper fits CPU time ~ N^z)."""
    import numpy as np
    import torch
    import paper_1905_07440_gb300 as hq
    W, M = args.warmup, args.steps
    engines = []
    for k, (side, C) in enumerate(PHYSICS_SIDES):
        p = physics_params(side, workloads.BATCHED.seed + 31 * k)
        e = hq.Engine(p, C, max_series=W + M)
        # start at the mean field <X> = -g/(M Omega^2) = -4 with the free-phonon spread: from
        # X ~ N(0, 4) the block moves' random walk needs hundreds of sweeps to get there
        x0 = -p.g / (p.mass * p.omega ** 2)
        e.set_fields(workloads.initial_fields(p, C, seed=100 + k) + x0)
        engines.append(e)
    obs_engines = [e for (side, _), e in zip(PHYSICS_SIDES, engines) if side in PHYSICS_OBS_SIDES]
    grp = hq.Group(obs_engines)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grp.sweep(W + M)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    obs = {}
    for (side, C), e in zip(PHYSICS_SIDES, engines):
        if side not in PHYSICS_OBS_SIDES:
            continue
        row = {"chains": C}
        for oid, name in ((hq.HQ_OBS_SCDW, "s_cdw"), (hq.HQ_OBS_DENSITY, "density"), (hq.HQ_OBS_X_MEAN, "x_mean"),
                          (hq.HQ_OBS_DOUBLE_OCC, "double_occ")):
            pc = e.series(oid)[:, W:].mean(axis=1)
            row[name] = [float(pc.mean()), float(pc.std(ddof=1) / math.sqrt(C))]
        row["status_ok"] = all(o["status"] == 0 for o in e.observables())
        obs[f"{side}x{side}"] = row
    grp.close()
    # time of one chain-sweep per lattice (each engine alone, one chain per SM)
    times = {}
    for k, (side, C) in enumerate(PHYSICS_SIDES):
        e = engines[k]
        e.sweep(1)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e.sweep(2)
        torch.cuda.synchronize()
        times[side] = (time.perf_counter() - t1) / 2
    Ns = np.array([s * s for s, _ in PHYSICS_SIDES], dtype=float)
    ts = np.array([times[s] for s, _ in PHYSICS_SIDES])
    z = float(np.polyfit(np.log(Ns), np.log(ts), 1)[0])
    z_big = float(np.polyfit(np.log(Ns[-3:]), np.log(ts[-3:]), 1)[0])
    line = {"mode": "physics point", "metric": "S_CDW(pi,pi) vs lattice; seconds per chain-sweep vs N",
            "config": {"workload": "Omega=0.5, lambda=0.5 (g=1), mu=-4, beta=4.1, dtau=0.1 (L=41), "
                                   "full sweeps (local moves + a block move per site); fields start at "
                                   "-g/(M Omega^2) + N(0, 1/(M Omega^2))",
                       "warmup_sweeps": W, "measured_sweeps": M, "data": "synthetic"},
            "group_wall_s": wall, "observables": obs,
            "seconds_per_chain_sweep": {f"{s}x{s}": times[s] for s, _ in PHYSICS_SIDES},
            "z_fit_all": z, "z_fit_8_to_12": z_big,
            "paper_context": "CPU time ~ N^z with z = 3.41 (DQMC) and 2.35 (NN-accelerated), hardware unstated"}
    print(json.dumps(line), flush=True)
    return 0


def run_graphs(args):
    """Launch cost: sweeps of small lattices, eager launches against CUDA-graph replay
    (hq_set_graphs); host wall clock over args.steps sweeps after args.warmup."""
    import torch
    import paper_1905_07440_gb300 as hq
    out = {"mode": "graph replay", "metric": "sweeps/s (engine)", "cases": {}}
    for name, shape, C in (("4x4 beta=1", dict(nx=4, ny=4, beta=1.0), 1), ("4x4 beta=1", dict(nx=4, ny=4, beta=1.0), 64),
                           ("8x8 beta=1", dict(nx=8, ny=8, beta=1.0), 64)):
        p = workloads.HolsteinParams(**shape)
        row = {}
        for graphs in (False, True):
            eng = hq.Engine(p, C, stream=torch.cuda.Stream())
            eng.set_fields(workloads.initial_fields(p, C))
            eng.set_graphs(graphs)
            eng.sweep(max(args.warmup, 3))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            eng.sweep(args.steps)
            torch.cuda.synchronize()
            row["graph" if graphs else "eager"] = args.steps / (time.perf_counter() - t0)
            eng.close()
        row["speedup"] = row["graph"] / row["eager"]
        out["cases"][f"{name} x{C} chains"] = row
    print(json.dumps(out), flush=True)
    return 0


def run_autotune(args):
    """Autotuner table (ms per sweep for every delay rank and block-move method) on the
    batched workload (full sweeps) and on the largest lattice (local sweeps only: a full sweep
    there is minutes of block moves)."""
    import torch
    import paper_1905_07440_gb300 as hq
    out = {"mode": "autotune", "metric": "ms per sweep", "tables": {}}
    for name, prm, C, glob in (("batched 8x8 beta=8 L=80", workloads.BATCHED, workloads.BATCHED_RUN["n_chains"], True),
                               ("largest 16x16 beta=16 L=160, local sweeps", workloads.LARGEST, 64, False)):
        X = torch.from_numpy(workloads.initial_fields(prm, C)).cuda()
        ks = (4, 8, 16, 32)
        methods = (1, 2) if glob else (1,)
        t0 = time.perf_counter()
        table, bk, bm = hq.autotune(prm, X, ks=ks, methods=methods, global_=glob, warmup=1, reps=args.steps)
        out["tables"][name] = {"chains": C, "ms_per_sweep": {f"k={k},method={m}": v for (k, m), v in table.items()},
                               "best_k": bk, "best_method": ["", "per-slice", "chunk propagators"][bm],
                               "default_ms": table.get((prm.delay_k, 2 if glob else 1)),
                               "seconds": time.perf_counter() - t0}
        del X
    print(json.dumps(out), flush=True)
    return 0


def run_largest_learned(args):
    """Learned vs plain at the largest lattice, 16x16, beta = 16 (L = 160), 64 chains.

    The patch network is local, so it is trained where samples are cheap -- 8x8 at the same
    beta and couplings, 256 chains of the plain sampler -- and deployed at 16x16.  Plain
    comparison: local sweeps (a full sweep with a block move per site costs 256 stabilised
    determinants per chain, minutes per sweep at this size; with --plain-full one such sweep is
    timed and turned into an upper bound on its independent samples/s).  Both samplers start
    at the mean field with the free-phonon spread; tau_int from the measured part of each run.
    """
    import numpy as np
    import torch
    import paper_1905_07440_gb300 as hq
    if args.deploy == "medium":
        big, C0, wname = workloads.MEDIUM, workloads.MEDIUM_RUN["n_chains"], "12x12 beta=8 L=80, g=sqrt2, mu=-2"
    else:
        big, C0, wname = workloads.LARGEST, workloads.LARGEST_RUN["n_chains"], "16x16 beta=16 L=160, g=sqrt2, mu=-2"
    C = args.chains or C0
    small = big.with_(nx=8, ny=8)
    x0 = -big.g / (big.mass * big.omega ** 2)
    dev = torch.device("cuda", 0)
    t_all = time.perf_counter()
    # training data at 8x8
    eng = hq.Engine(small, 256)
    eng.set_fields(workloads.initial_fields(small, 256) + x0)
    eng.sweep(args.train_warmup, local=True, global_=True)
    Xs, ys = [], []
    for _ in range(args.train_snapshots):
        eng.sweep(2)
        Xs.append(eng.get_fields())
        ys.append(eng.log_weight()[1])
    eng.close()
    Xtr, ytr = np.concatenate(Xs), np.concatenate(ys)
    ytr -= ytr.mean()
    net = hq.Engine(small, 1)
    net.attach_network(64, Xtr.shape[0])
    net.set_params(hq.init_network(args.nn_seed))
    Xd, yd = torch.from_numpy(Xtr).to(dev), torch.from_numpy(ytr).to(dev)
    losses = []
    for k in range(3):
        ep = args.epochs // 3 + (args.epochs % 3 if k == 2 else 0)
        losses.extend(net.nn_train(Xd, yd, epochs=ep, batch=64, lr=args.lr * 0.5 ** k, seed=args.nn_seed + k))
    theta = net.get_params()
    del Xd, yd
    net.close()
    W, M = args.warmup, args.tau_steps
    X0 = workloads.initial_fields(big, C, seed=7) + x0
    series_ids = ((hq.HQ_OBS_X2, "x2"), (hq.HQ_OBS_DOUBLE_OCC, "double_occ"), (hq.HQ_OBS_SCDW, "s_cdw"))

    def tau_block(e, first):
        out = {}
        for oid, name in series_ids:
            ser = e.series(oid)[:, first:]
            out[name] = (float(np.mean([hq.tau_int(ser[c])[0] for c in range(C)])), float(ser.mean()))
        return out

    # learned sampler
    lrn = hq.Engine(big, C, max_series=W + M)
    lrn.attach_network(4, 8)
    lrn.set_params(theta)
    lrn.set_inner_window(args.window)
    lrn.set_inner_sites(args.sites)
    lrn.set_fields(X0)
    lrn.cumulative(W, args.n_inner, measure=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lrn.cumulative(M, args.n_inner, measure=True)
    torch.cuda.synchronize()
    l_rate = C * M / (time.perf_counter() - t0)
    st = lrn.learned_stats()
    acc = sum(x["cumulative_accepted"] for x in st) / max(1, sum(x["cumulative_proposed"] for x in st))
    l_tau = tau_block(lrn, W)
    lrn.close()
    # plain sampler, local sweeps
    p_rate, p_tau, gain = None, None, None
    if not args.skip_plain:
        pl = hq.Engine(big, C, max_series=W + M)
        pl.set_fields(X0)
        pl.sweep(W, global_=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pl.sweep(M, global_=False)
        torch.cuda.synchronize()
        p_rate = C * M / (time.perf_counter() - t0)
        p_tau = tau_block(pl, W)
        pl.close()
        gain = {k: (l_rate / (2 * l_tau[k][0])) / (p_rate / (2 * p_tau[k][0])) for k in l_tau}
    full = None
    if args.plain_full:
        # one full sweep (local moves + a block move per site) of 8 chains: per-chain latency
        fe = hq.Engine(big, 8)
        fe.set_fields(X0[:8])
        fe.sweep(1, global_=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fe.sweep(1)
        torch.cuda.synchronize()
        t_full = time.perf_counter() - t0
        fe.close()
        # even if one full sweep gave an independent sample (tau_int = 1/2 sweep), 64 chains
        # would give at most this many per second
        full = {"seconds_per_sweep": t_full, "chains_timed": 8,
                "indep_samples_per_s_upper_bound": C / t_full,
                "learned_gain_lower_bound": {k: (l_rate / (2 * l_tau[k][0])) / (C / t_full) for k in l_tau}}
    line = {"metric": METRIC, "mode": "learned vs plain, " + args.deploy + " lattice",
            "value": l_rate / (2 * l_tau["s_cdw"][0]), "unit": "independent samples/s of S_CDW(pi,pi) (learned)",
            "higher_is_better": True, "dtype": "f64 weights, bf16-weight/fp32 network", "data": "synthetic",
            "config": {"workload": wname, "chains": C, "warmup": W, "measured": M,
                       "network": "patch network trained at 8x8 beta=%g (%d samples, %d epochs)"
                                  % (big.beta, Xtr.shape[0], args.epochs),
                       "plain": "local sweeps (no block moves)",
                       "inner_window_slices": args.window or big.n_slices,
                       "inner_block_sites": args.sites or big.n_sites, "skip_plain": args.skip_plain},
            "learned": {"steps_per_s": l_rate, "cumulative_acceptance": acc,
                        "tau_int_and_mean": l_tau},
            "plain": {"sweeps_per_s": p_rate, "tau_int_and_mean": p_tau},
            "gain_indep_samples": gain, "plain_full_sweep": full,
            "training_loss": [float(losses[0]), float(losses[-1]), float(np.var(ytr))],
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)
    return 0


def run_training(args):
    """Training protocol of the learned-proposal workload (paper, Global Updates, on training
    both networks: tens of thousands of configurations of the conventional sampler with a
    train/test split).  Per temperature
    (beta = 8 and 16, 8x8, the headline couplings): 256 plain chains from the ordered start,
    args.train_warmup sweeps, then one snapshot (fields, exact log|det M|) per sweep; chains
    0..191 give the training set, 192..255 the held-out test set (75/25 by chain, so no test
    configuration is correlated with a training one).  Reported: the test-set RMS of F against
    log|det M| (both centred by the training mean), and on deployment lattices (12x12 at beta = 8,
    16x16 at beta = 16) the RMS of the centred differences over configurations of the plain
    sampler there (local sweeps from the ordered start), against the spread of log|det M|."""
    import numpy as np
    import torch
    import paper_1905_07440_gb300 as hq
    dev = torch.device("cuda", 0)
    out = {"mode": "training protocol", "config": {"snapshots": {}, "epochs": args.epochs, "batch": 64,
                                                   "lr": args.lr, "split": "chains 0-191 train, 192-255 test"}}
    for beta, snaps, deploy in ((8.0, args.train_snapshots_b8, workloads.MEDIUM),
                                (16.0, args.train_snapshots_b16, workloads.LARGEST)):
        small = workloads.LARGEST.with_(nx=8, ny=8, beta=beta)
        t0 = time.perf_counter()
        tr = hq.Engine(small.with_(seed=small.seed + 7), 256)
        tr.set_fields(start_fields(small, 256, args.start_amplitude, workloads.DEFAULT_SEED + 5000))
        tr.sweep(args.train_warmup)
        X = torch.empty((snaps, 256, small.n_slices, small.n_sites), dtype=torch.float64, device=dev)
        Y = np.empty((snaps, 256))
        for k in range(snaps):
            tr.sweep(1)
            X[k] = torch.from_numpy(tr.get_fields()).to(dev)
            Y[k] = tr.log_weight()[1]
        tr.close()
        t_data = time.perf_counter() - t0
        Xtr = X[:, :192].reshape(-1, small.n_slices, small.n_sites).contiguous()
        Xte = X[:, 192:].reshape(-1, small.n_slices, small.n_sites).contiguous()
        del X
        ytr, yte = Y[:, :192].reshape(-1), Y[:, 192:].reshape(-1)
        mu = ytr.mean()
        ytr_d = torch.from_numpy(ytr - mu).to(dev)
        yte_d = torch.from_numpy(yte - mu).to(dev)
        net = hq.Engine(small, 1)
        B = 2048
        net.attach_network(B, Xtr.shape[0])
        net.set_params(hq.init_network(args.nn_seed))
        t1 = time.perf_counter()
        losses = []
        for k in range(3):
            ep = args.epochs // 3 + (args.epochs % 3 if k == 2 else 0)
            losses.extend(net.nn_train(Xtr, ytr_d, epochs=ep, batch=64, lr=args.lr * 0.5 ** k, seed=args.nn_seed + k))
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t1

        def mse(Xs, ys):
            tot, n = 0.0, 0
            for a in range(0, Xs.shape[0], B):
                nb = min(B, Xs.shape[0] - a)
                _, l = net.nn_gradient(Xs[a:a + nb], ys[a:a + nb])
                tot += l * nb
                n += nb
            return tot / n

        train_mse, test_mse = mse(Xtr, ytr_d), mse(Xte, yte_d)
        theta = net.get_params()
        net.close()
        del Xtr, Xte
        # deployment lattice: configurations of the exact plain sampler there (local sweeps from the
        # ordered start), F of the network trained at 8x8 against their log|det M|
        dp = deploy
        e = hq.Engine(dp.with_(seed=dp.seed + 77), 64, max_series=0)
        e.attach_network(4, 8)
        e.set_params(theta)
        e.set_fields(start_fields(dp, 64, args.start_amplitude, workloads.DEFAULT_SEED + 77))
        e.sweep(args.deploy_relax, global_=False)
        Fs, Ls = [], []
        for _ in range(args.deploy_samples):
            e.sweep(args.deploy_gap, global_=False)
            Fs.append(e.nn_eval())
            Ls.append(e.log_weight()[1])
        e.close()
        Fs, Ls = np.concatenate(Fs), np.concatenate(Ls)
        dlt = (Fs - Fs.mean()) - (Ls - Ls.mean())
        key = f"8x8 beta={beta:g}"
        out["config"]["snapshots"][key] = snaps
        out[key] = {"train_samples": int(ytr.size), "test_samples": int(yte.size), "data_s": t_data,
                    "train_s": t_train, "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
                    "train_rms": math.sqrt(train_mse), "test_rms": math.sqrt(test_mse),
                    "target_sd_train": float(ytr.std()), "target_sd_test": float(yte.std()),
                    "deployment": {"lattice": f"{dp.nx}x{dp.ny} beta={dp.beta:g}", "configurations": int(Fs.size),
                                   "rms_centred": float(np.sqrt(np.mean(dlt ** 2))),
                                   "logdet_sd": float(Ls.std())}}
    print(json.dumps(out), flush=True)
    return 0


def run_sections(args):
    """Section rooflines from the per-section cycle counters of a -DHQ_SECTION_TIMING build (its
    own library variant): the local phase's wrap and delayed-update flush, and the block moves' QR,
    Q formation, T update and products, on the plain 8x8, beta = 8 workload with one chain per SM
    (152 chains), so that a CTA's cycles are its SM's.  Flops per section: wrap 4 N^2 (nx + ny) +
    2 N^2 per slice, flush 2 N^2 per accepted local move."""
    import numpy as np
    import torch
    from paper_1905_07440_gb300 import build
    lib = build.build(extra=("-DHQ_SECTION_TIMING",), variant="timing")
    import paper_1905_07440_gb300 as hq
    hq.load_library(lib)
    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    p = workloads.BATCHED
    C = args.chains or sms
    peak = hq.fp64_peak_tflops(20, kind=hq.HQ_PROBE_DFMA)
    eng = hq.Engine(p, C, max_series=args.steps + 4)
    eng.set_fields(workloads.ordered_fields(p, C, args.start_amplitude, seed=workloads.DEFAULT_SEED))
    eng.sweep(2)
    torch.cuda.synchronize()
    hq.section_cycles()
    o0 = eng.observables()
    clocks = ClockSampler()
    clocks.start()
    eng.sweep(args.steps, local=True, global_=False)
    torch.cuda.synchronize()
    cyc_local = hq.section_cycles()
    eng.sweep(1, local=False, global_=True)
    torch.cuda.synchronize()
    cyc_block = hq.section_cycles()
    clk = clocks.stop()
    o1 = eng.observables()
    acc = sum(b["local_accepted"] - a["local_accepted"] for a, b in zip(o0, o1))
    hz = (clk["sm_mhz"] or 2070.0) * 1e6
    n, L = p.n_sites, p.n_slices
    per_sm = peak / sms
    fl_wrap = args.steps * C * L * (4.0 * n * n * (p.nx + p.ny) + 2.0 * n * n)
    fl_flush = 2.0 * n * n * acc

    def roof(fl, cycles):
        t = cycles / hz
        return {"tflops_per_sm": fl / t / 1e12 if t else None, "frac_of_per_sm_peak": fl / t / 1e12 / per_sm if t else None,
                "sm_seconds": t, "gflop": fl / 1e9}
    out = {"mode": "section rooflines", "config": {"workload": "plain 8x8 beta=8 L=80", "chains": C, "sms": sms,
                                                   "local_sweeps": args.steps, "clock_mhz": hz / 1e6},
           "peak_tflops_dfma": peak, "wrap": roof(fl_wrap, cyc_local.get("wrap", 0)),
           "flush": roof(fl_flush, cyc_local.get("flush", 0)), "local_accepted": acc,
           "local_sections_cycles": cyc_local, "block_sections_cycles": cyc_block, "clocks": clk}
    # block moves: one move per site per chain; per chunk of m slices QR 4/3 N^3, Q 4/3 N^3, T update N^3
    q = math.ceil(L / p.n_wrap)
    moves = C * n
    out["block_qr"] = roof(moves * q * (4.0 / 3.0) * n ** 3, cyc_block.get("qr", 0))
    out["block_form_q"] = roof(moves * q * (4.0 / 3.0) * n ** 3, cyc_block.get("form_q", 0))
    out["block_t_update"] = roof(moves * (q - 1) * float(n) ** 3, cyc_block.get("t_update", 0))
    eng.close()
    # the same sections in the largest lattice's full top-down product (16x16, beta = 16: the
    # stack build, whose chunks are those of the two-half log-det), one chain per SM
    pl = workloads.LARGEST
    big = hq.Engine(pl, C)
    Xl = workloads.ordered_fields(pl, C, args.start_amplitude, seed=workloads.DEFAULT_SEED)
    big.set_fields(Xl)
    big.log_weight()  # the stack build runs on the first use of new fields
    torch.cuda.synchronize()
    hq.section_cycles()
    clocks = ClockSampler()
    clocks.start()
    big.set_fields(Xl)
    big.log_weight()
    torch.cuda.synchronize()
    cyc_big = hq.section_cycles()
    clk_big = clocks.stop()
    big.close()
    nb, chunks = pl.n_sites, chunk_sizes_top_down(pl)
    slices = sum(chunks)
    out["largest_stack_build"] = {
        "workload": "16x16 beta=16 L=160 stack build, one chain per SM", "chains": C, "clocks": clk_big,
        "kin": roof(C * slices * (2.0 * nb * nb * (pl.nx + pl.ny) + nb * nb), cyc_big.get("kin", 0)),
        "qr": roof(C * len(chunks) * (4.0 / 3.0) * nb ** 3, cyc_big.get("qr", 0)),
        "form_q": roof(C * len(chunks) * (4.0 / 3.0) * nb ** 3, cyc_big.get("form_q", 0)),
        "t_update": roof(C * (len(chunks) - 1) * float(nb) ** 3, cyc_big.get("t_update", 0)),
        "sections_cycles": cyc_big}
    print(json.dumps(out), flush=True)
    return 0


def run_agreement(args):
    """Learned vs plain means from the same fields, every run with a fresh Philox key.  Per beta in
    args.betas on an args.side x args.side lattice (headline couplings): 256 plain chains from the mean
    field + N(0, 1/(M Omega^2)), args.relax sweeps, 16 snapshots two sweeps apart (training data), the
    network trained on the tensor cores; then from the final fields a plain run, a learned run (local
    moves at every slice) and a second plain run of args.tau_steps sweeps or steps each.  Reported per
    observable: mean and error over the chains' means, tau_int, the second-half minus first-half
    difference, and the z-scores learned - plain and plain2 - plain."""
    import numpy as np
    import torch
    import paper_1905_07440_gb300 as hq
    names = ((hq.HQ_OBS_X2, "x2"), (hq.HQ_OBS_DOUBLE_OCC, "double_occ"), (hq.HQ_OBS_SCDW, "s_cdw"))
    out = {"mode": "agreement", "config": {"lattice": f"{args.side}x{args.side}", "chains": 256,
                                           "warmup_sweeps": args.relax + 32, "measured": args.tau_steps,
                                           "learned_window": args.agree_window}}
    for beta in (float(b) for b in args.betas.split(",")):
        p = workloads.HolsteinParams(nx=args.side, ny=args.side, beta=beta)
        x0 = -p.g / (p.mass * p.omega ** 2)
        A = hq.Engine(p, 256)
        A.set_fields(workloads.initial_fields(p, 256) + x0)
        A.sweep(args.relax)
        Xs, ys = [], []
        for _ in range(16):
            A.sweep(2)
            Xs.append(A.get_fields())
            ys.append(A.log_weight()[1])
        Xeq = A.get_fields()
        A.close()
        Xtr, ytr = np.concatenate(Xs), np.concatenate(ys)
        ytr = ytr - ytr.mean()
        net = hq.Engine(p, 1)
        net.attach_network(64, Xtr.shape[0])
        net.set_params(hq.init_network(args.nn_seed))
        Xd, yd = torch.from_numpy(Xtr).cuda(), torch.from_numpy(ytr).cuda()
        for k in range(3):
            net.nn_train(Xd, yd, epochs=args.epochs // 3, batch=64, lr=args.lr * 0.5 ** k, seed=args.nn_seed + k)
        theta = net.get_params()
        net.close()
        row = {}
        for kind, seed in (("plain", 777), ("learned", 888), ("plain2", 999)):
            m = hq.Engine(p.with_(seed=seed), 256, max_series=args.tau_steps)
            m.set_fields(Xeq)
            if kind == "learned":
                m.attach_network(4, 8)
                m.set_params(theta)
                m.set_inner_window(args.agree_window)
                m.cumulative(args.tau_steps, 1, measure=True)
                st = m.learned_stats()
                row["acceptance"] = sum(x["cumulative_accepted"] for x in st) / sum(x["cumulative_proposed"] for x in st)
            else:
                m.sweep(args.tau_steps)
            row[kind] = series_stats(hq, m, 0, names)
            m.close()
        for a, b in (("learned", "plain"), ("plain2", "plain")):
            row[f"z_{a}_vs_{b}"] = {k: (row[a][k]["mean"] - row[b][k]["mean"]) / math.hypot(row[a][k]["err"], row[b][k]["err"])
                                    for _, k in names}
        out[f"beta={beta:g}"] = row
    print(json.dumps(out), flush=True)
    return 0


def run_peaks():
    """FP64 pipe evidence: DFMA and DMMA probes of the library, cuBLAS DGEMM/SGEMM via torch."""
    import torch
    import paper_1905_07440_gb300 as hq
    out = {"dfma_tflops": hq.fp64_peak_tflops(20, kind=hq.HQ_PROBE_DFMA),
           "dmma_tflops": hq.fp64_peak_tflops(20, kind=hq.HQ_PROBE_DMMA)}

    def rate(fn, flops, reps=5):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return flops * reps / (a.elapsed_time(b) / 1e3) / 1e12

    n = 8192
    x = torch.randn(n, n, dtype=torch.float64, device="cuda")
    out["cublas_dgemm_8192_tflops"] = rate(lambda: x @ x, 2 * n ** 3)
    xb = torch.randn(256, 64, 64, dtype=torch.float64, device="cuda")
    out["cublas_batched_dgemm_256x64_tflops"] = rate(lambda: torch.bmm(xb, xb), 2 * 256 * 64 ** 3, 50)
    torch.backends.cuda.matmul.allow_tf32 = False
    xs = x.float()
    out["cublas_sgemm_8192_tflops"] = rate(lambda: xs @ xs, 2 * n ** 3)
    out["device"] = torch.cuda.get_device_name()
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="headline")
    ap.add_argument("--relax", type=int, default=200, help="headline: learned steps before the measured series (minimum)")
    ap.add_argument("--relax-max", type=int, default=800, help="headline: most relaxation steps")
    ap.add_argument("--side", type=int, default=6, help="agreement mode: lattice side")
    ap.add_argument("--betas", default="2,3,4", help="agreement mode: comma-separated beta values")
    ap.add_argument("--agree-window", type=int, default=0, help="agreement mode: learned window (0: every slice)")
    ap.add_argument("--inner-block-sites", type=int, default=0,
                    help="headline: block moves per cumulative step on this many sites (0: none)")
    ap.add_argument("--train-start-amplitude", type=float, default=0.0,
                    help="headline: staggered amplitude of the training chains' start (0: mean field)")
    ap.add_argument("--start-amplitude", type=float, default=0.9,
                    help="headline: staggered amplitude of the ordered start (0: mean-field start)")
    ap.add_argument("--train-chains", type=int, default=256, help="headline: plain chains for training data")
    ap.add_argument("--train-snapshots-b8", type=int, default=392, help="training mode: sweeps of snapshots, beta 8")
    ap.add_argument("--train-snapshots-b16", type=int, default=200, help="training mode: sweeps of snapshots, beta 16")
    ap.add_argument("--deploy-relax", type=int, default=10, help="training mode: local sweeps before deployment")
    ap.add_argument("--deploy-samples", type=int, default=8, help="training mode: deployment snapshots")
    ap.add_argument("--deploy-gap", type=int, default=1, help="training mode: local sweeps between snapshots")
    ap.add_argument("--cpu-steps", type=int, default=2, help="headline: oracle steps per core in the CPU baseline")
    ap.add_argument("--e2e-steps", type=int, default=5, help="headline: steps through host buffers")
    ap.add_argument("--plain-block-sites", type=int, default=16, help="headline: block-move sites timed per plain sweep")
    ap.add_argument("--batched-steps", type=int, default=5, help="headline: sweeps of the plain 8x8 line (0: skip)")
    ap.add_argument("--chains", type=int, default=0, help="override chains per rank (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--peaks", action="store_true", help="print the FP64/FP32 pipe probes and exit")
    ap.add_argument("--tau-sweeps", type=int, default=0, help="measure tau_int over this many sweeps and exit")
    ap.add_argument("--n-inner", type=int, default=1, help="learned mode: network sweeps per cumulative step")
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--nn-seed", type=int, default=1)
    ap.add_argument("--train-warmup", type=int, default=8)
    ap.add_argument("--train-snapshots", type=int, default=24)
    ap.add_argument("--tau-steps", type=int, default=240)
    ap.add_argument("--cnn", action="store_true", help="learned mode: convolutional action for block moves")
    ap.add_argument("--deploy", choices=("largest", "medium"), default="largest",
                    help="largest-learned mode: deploy at 16x16 beta=16 or 12x12 beta=8")
    ap.add_argument("--window", type=int, default=32, help="learned modes: local moves per step on this many slices")
    ap.add_argument("--sites", type=int, default=0, help="learned modes: block moves per step on this many sites")
    ap.add_argument("--skip-plain", action="store_true", help="largest-learned mode: learned sampler only")
    ap.add_argument("--plain-full", action="store_true",
                    help="largest-learned mode: also time one full plain sweep (minutes at 16x16)")
    ap.add_argument("--cnn-lr", type=float, default=3e-3)
    ap.add_argument("--rate", type=float, default=20.0, help="serving mode: requests per second")
    ap.add_argument("--duration", type=float, default=10.0, help="serving mode: seconds of arrivals")
    ap.add_argument("--req-sweeps", type=int, default=2, help="serving mode: sweeps per request")
    ap.add_argument("--serve-block-sites", type=int, default=8, help="serving mode: plain block-move sites per sweep")
    ap.add_argument("--serve-window", type=int, default=32, help="serving mode: learned window (slices)")
    ap.add_argument("--slots", type=int, default=16, help="serving mode: chain slots per pool")
    ap.add_argument("--max-pools", type=int, default=32, help="serving mode: live pools (streams)")
    ap.add_argument("--learned-frac", type=float, default=0.5, help="serving mode: share of learned requests")
    ap.add_argument("--hbm-budget", type=int, default=8 << 30, help="serving mode: bytes for pool state")
    ap.add_argument("--serve-seed", type=int, default=3)
    args = ap.parse_args()
    if args.workload == "serving":
        # one hardware queue per pool stream: with fewer, streams share queues and a pool's
        # launches wait behind another pool's running kernels (read when CUDA initialises)
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    if args.workload == "learned":
        sys.exit(run_learned(args))
    if args.workload == "largest-learned":
        sys.exit(run_largest_learned(args))
    if args.workload == "serving":
        sys.exit(run_serving(args))
    if args.workload == "training":
        sys.exit(run_training(args))
    if args.workload == "sections":
        sys.exit(run_sections(args))
    if args.workload == "agreement":
        sys.exit(run_agreement(args))
    if args.peaks:
        sys.exit(run_peaks())
    if args.workload == "autotune":
        sys.exit(run_autotune(args))
    if args.workload == "hetero":
        sys.exit(run_hetero(args))
    if args.workload == "graphs":
        sys.exit(run_graphs(args))
    if args.workload == "physics":
        sys.exit(run_physics(args))
    if args.tau_sweeps:
        sys.exit(run_tau(args))
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        sys.exit(run_reference(args))
    sys.exit(run_headline(args) if args.workload == "headline" else run_ours(args))


if __name__ == "__main__":
    main()
