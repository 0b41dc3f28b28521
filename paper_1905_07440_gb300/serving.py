"""Continuous-batching service for DQMC requests (host scheduler over the C ABI).

A request asks for `sweeps` sweeps (plain) or cumulative steps (learned) of one chain with
its own parameters, fields, Philox key and chain word.  Requests with the same model and
lattice parameters share a pool: one engine whose chain slots run in lockstep on the pool's
own CUDA stream.  A request that arrives while others run is admitted at the next sweep
boundary of a pool with a free slot; new pools are created only while the device arenas of
all live pools stay inside the HBM budget, and empty pools are released.  Pools run
concurrently on their streams, so their work overlaps on the device.  Because every chain
carries its own key, chain word and sweep counter, a request's result is the same alone and
in any mix.

Each live pool needs a hardware work queue of its own: CUDA maps streams onto
CUDA_DEVICE_MAX_CONNECTIONS queues (8 unless set before CUDA initialises), and streams that
share a queue run their launches in submission order, so a pool's short launch would wait
behind another pool's long block-move phase.  Set it to at least max_pools (32 at most).
"""
import collections
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    params: object            # workloads.HolsteinParams (its seed is the chain's Philox key)
    X0: np.ndarray            # [L][N] initial fields
    sweeps: int
    sampler: str = "plain"    # "plain" or "learned"
    chain_id: int = 0
    theta: object = None      # network parameters for "learned"
    arrival: float = 0.0
    admitted: float = None
    done: float = None
    X: np.ndarray = None      # final fields
    obs: dict = None          # the chain's accumulated observables


def pool_key(req):
    p = req.params
    theta_key = None if req.sampler == "plain" else hash(np.asarray(req.theta, dtype=np.float32).tobytes())
    return (p.nx, p.ny, p.t, p.mu, p.omega, p.mass, p.g, p.beta, p.dtau, p.n_wrap, p.delay_k, p.dx_local,
            p.dx_global, req.sampler, theta_key)


class Pool:
    def __init__(self, backend, req, slots):
        self.key = pool_key(req)
        self.sampler = req.sampler
        self.engine, self.bytes = backend.new_engine(req.params, slots, req.sampler, req.theta)
        self.slots = [None] * slots
        self.left = [0] * slots
        self.busy = False
        self.idle_since = None    # clock time at which the pool last became empty

    def free_slot(self):
        for k, r in enumerate(self.slots):
            if r is None:
                return k
        return -1

    def active(self):
        return [k for k, r in enumerate(self.slots) if r is not None]


class Server:
    """Admission, continuous batching and completion of requests on one GPU."""

    def __init__(self, backend, hbm_budget, slots_per_pool=32, keep_idle_s=2.0, max_pools=32,
                 clock=time.perf_counter):
        self.backend = backend
        self.budget = hbm_budget
        self.slots_per_pool = slots_per_pool
        self.max_pools = max_pools      # live pools (one CUDA stream each)
        self.keep_idle_s = keep_idle_s  # empty pools stay (warm) this long unless memory is needed
        self.clock = clock
        self.queue = collections.deque()
        self.pools = []
        self.finished = []

    @property
    def used(self):
        return sum(p.bytes for p in self.pools)

    def submit(self, req):
        self.queue.append(req)

    def _release(self, pool):
        self.backend.release(pool.engine)
        self.pools.remove(pool)

    def _fits(self, need):
        return self.used + need <= self.budget and len(self.pools) < self.max_pools

    def _make_room(self, need):
        """Release empty pools, longest idle first, until a pool of `need` more bytes fits the
        budget and the pool limit."""
        for pool in sorted((p for p in self.pools if not p.active() and not p.busy), key=lambda p: p.idle_since):
            if self._fits(need):
                break
            self._release(pool)
        return self._fits(need)

    def _admit(self):
        """Place queued requests, in arrival order, at sweep boundaries: into an idle pool of the
        same key with a free slot; if every pool of that key is full, into a new pool when the
        HBM budget allows one (after releasing empty pools); otherwise (a matching pool is
        mid-sweep, or no room) they wait."""
        waiting = collections.deque()
        while self.queue:
            req = self.queue.popleft()
            key = pool_key(req)
            same = [p for p in self.pools if p.key == key and p.free_slot() >= 0]
            pool = next((p for p in same if not p.busy), None)
            if pool is None and not same:
                need = self.backend.engine_bytes(req.params, self.slots_per_pool, req.sampler)
                if self._make_room(need):
                    pool = Pool(self.backend, req, self.slots_per_pool)
                    self.pools.append(pool)
            if pool is None:
                waiting.append(req)
                continue
            k = pool.free_slot()
            self.backend.load(pool.engine, k, req)
            pool.slots[k] = req
            pool.left[k] = req.sweeps
            pool.idle_since = None
            req.admitted = self.clock()
        self.queue = waiting

    def _launch(self):
        for pool in self.pools:
            if not pool.busy and pool.active():
                self.backend.advance(pool.engine, pool.sampler)
                pool.busy = True

    def _collect(self):
        for pool in self.pools:
            if pool.busy and self.backend.ready(pool.engine):
                pool.busy = False
                done = []
                for k in pool.active():
                    pool.left[k] -= 1
                    if pool.left[k] == 0:
                        done.append(k)
                if done:
                    X, obs = self.backend.results(pool.engine)
                    now = self.clock()
                    for k in done:
                        req = pool.slots[k]
                        req.X, req.obs, req.done = X[k].copy(), obs[k], now
                        self.backend.idle(pool.engine, k)
                        pool.slots[k] = None
                        self.finished.append(req)
                    if not pool.active():
                        pool.idle_since = now
        now = self.clock()
        for pool in [p for p in self.pools if not p.active() and not p.busy]:
            if pool.idle_since is None:
                pool.idle_since = now
            elif now - pool.idle_since > self.keep_idle_s:
                self._release(pool)

    def poll(self):
        """One scheduling round: collect finished sweeps, admit, launch the next sweeps."""
        self._collect()
        self._admit()
        self._launch()

    def pending(self):
        return bool(self.queue) or any(p.active() or p.busy for p in self.pools)

    def close(self):
        """Release every pool (call when no request is pending)."""
        for pool in list(self.pools):
            self._release(pool)

    def run(self, requests, sleep=1e-4):
        """Serve requests arriving at their `arrival` times (seconds from the start)."""
        queued = sorted(requests, key=lambda r: r.arrival)
        t0 = self.clock()
        k = 0
        while k < len(queued) or self.pending():
            now = self.clock() - t0
            while k < len(queued) and queued[k].arrival <= now:
                queued[k].arrival = t0 + queued[k].arrival
                self.submit(queued[k])
                k += 1
            self.poll()
            if k < len(queued) and not self.pending():
                time.sleep(min(sleep, max(0.0, queued[k].arrival - (self.clock() - t0))))
        self.close()
        return self.finished


class GpuBackend:
    """Engines of the C ABI, each pool on a CUDA stream of its own."""

    def __init__(self, device=0, nn_batch=4, block_sites=0, window=0):
        """block_sites > 0: plain pools take their block moves on a run of that many sites per
        sweep (hq_set_block_sites); window > 0: learned pools take their local moves on that
        many slices per step (hq_set_inner_window)."""
        import torch
        import paper_1905_07440_gb300 as hq
        self.torch, self.hq, self.device = torch, hq, torch.device("cuda", device)
        self.nn_batch = nn_batch
        self.block_sites, self.window = block_sites, window
        self._free_streams = []
        self._in_use = set()

    def _stream(self):
        """A stream no live pool uses.  PyTorch hands out streams round-robin from a small
        pool, so a fresh one can be a stream a busy pool still holds; two pools on one stream
        would run one after the other."""
        st = self._free_streams.pop() if self._free_streams else None
        for prio in (0, -1):
            for _ in range(64 if st is None else 0):
                cand = self.torch.cuda.Stream(device=self.device, priority=prio)
                if cand.cuda_stream not in self._in_use:
                    st = cand
                    break
        if st is None:
            raise RuntimeError("no CUDA stream free for another pool")
        self._in_use.add(st.cuda_stream)
        return st

    def engine_bytes(self, params, slots, sampler):
        nb = self.hq.arena_bytes(params, slots, 0)
        return nb * (2 if sampler == "learned" else 1)

    def new_engine(self, params, slots, sampler, theta):
        stream = self._stream()
        eng = self.hq.Engine(params, slots, max_series=0, device=self.device, stream=stream)
        nbytes = eng.arena.numel()
        if sampler == "learned":
            eng.attach_network(self.nn_batch, self.nn_batch)
            eng.set_params(theta)
            eng.set_inner_window(self.window)
            nbytes += eng.nn_arena.numel()
        else:
            eng.set_block_sites(self.block_sites)
        for k in range(slots):
            eng.set_active(k, False)
        eng._done_event = None
        return eng, nbytes

    def load(self, eng, slot, req):
        eng.set_chain(slot, req.X0, req.params.seed, req.chain_id, 0)

    def advance(self, eng, sampler):
        """Enqueue one sweep (or cumulative step) of every active slot on the pool's stream."""
        if sampler == "learned":
            eng.cumulative(1, 1)
        else:
            eng.sweep(1)
        ev = self.torch.cuda.Event()
        ev.record(eng.stream)
        eng._done_event = ev

    def ready(self, eng):
        return eng._done_event is None or eng._done_event.query()

    def results(self, eng):
        obs = eng.observables()
        if getattr(eng, "nn_arena", None) is not None:
            for o, st in zip(obs, eng.learned_stats()):
                o.update(st)
        return eng.get_fields(), obs

    def idle(self, eng, slot):
        eng.set_active(slot, False)

    def release(self, eng):
        st = eng.stream
        eng.close()
        self._in_use.discard(st.cuda_stream)
        self._free_streams.append(st)
