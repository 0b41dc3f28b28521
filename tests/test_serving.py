"""Serving scheduler: admission by HBM budget, continuous batching, release of empty pools
(CPU, with a fake backend whose 'sweeps' are counters), and on the GPU the same results for
a request alone and in a mix, and a served request's chain against the CPU oracle."""
import numpy as np
import pytest

from paper_1905_07440_gb300.serving import Request, Server
from workloads import HolsteinParams, initial_fields


class FakeEngine:
    def __init__(self, slots):
        self.fields = [None] * slots
        self.sweeps = [0] * slots
        self.active = [False] * slots
        self.pending = 0


class FakeBackend:
    """Each advance() is one sweep of every active slot, finished after `lag` polls."""

    def __init__(self, bytes_per_engine=100, lag=1):
        self.bytes, self.lag, self.created, self.released = bytes_per_engine, lag, 0, 0

    def engine_bytes(self, params, slots, sampler):
        return self.bytes

    def new_engine(self, params, slots, sampler, theta):
        self.created += 1
        return FakeEngine(slots), self.bytes

    def load(self, eng, slot, req):
        eng.fields[slot] = np.array(req.X0, copy=True)
        eng.sweeps[slot] = 0
        eng.active[slot] = True

    def advance(self, eng, sampler):
        for k, a in enumerate(eng.active):
            if a:
                eng.fields[k] = eng.fields[k] + 1.0
                eng.sweeps[k] += 1
        eng.pending = self.lag

    def ready(self, eng):
        eng.pending -= 1
        return eng.pending <= 0

    def results(self, eng):
        return eng.fields, [{"sweeps": s} for s in eng.sweeps]

    def idle(self, eng, slot):
        eng.active[slot] = False

    def release(self, eng):
        self.released += 1


def make(rid, nx, sweeps, arrival=0.0):
    p = HolsteinParams(nx=nx, ny=nx, beta=0.5, seed=rid)
    return Request(rid=rid, params=p, X0=np.zeros((p.n_slices, p.n_sites)), sweeps=sweeps, arrival=arrival)


def test_every_request_gets_exactly_its_sweeps():
    be = FakeBackend()
    srv = Server(be, hbm_budget=1000, slots_per_pool=3)
    reqs = [make(k, 4 + 2 * (k % 3), 1 + k % 5) for k in range(20)]
    for r in reqs:
        srv.submit(r)
    while srv.pending():
        srv.poll()
    srv.close()
    assert len(srv.finished) == 20
    for r in srv.finished:
        assert r.obs["sweeps"] == r.sweeps
        assert np.all(r.X == r.sweeps)
    assert be.released == be.created


def test_budget_limits_live_pools_and_queues_the_rest():
    be = FakeBackend(bytes_per_engine=100)
    srv = Server(be, hbm_budget=250, slots_per_pool=2)
    for k in range(6):  # 3 shapes -> 3 pools wanted, budget allows 2
        srv.submit(make(k, 4 + 2 * (k % 3), 3))
    srv.poll()
    assert len(srv.pools) == 2 and srv.used <= 250
    assert len(srv.queue) == 2
    peak = 0
    while srv.pending():
        srv.poll()
        peak = max(peak, srv.used)
    assert peak <= 250 and len(srv.finished) == 6


def test_empty_pools_stay_warm_then_release():
    t = [0.0]
    be = FakeBackend()
    srv = Server(be, hbm_budget=1000, slots_per_pool=2, keep_idle_s=5.0, clock=lambda: t[0])
    srv.submit(make(1, 4, 1))
    while srv.pending():
        srv.poll()
    assert len(srv.pools) == 1 and be.released == 0      # empty but kept
    t[0] = 1.0
    srv.submit(make(2, 4, 1))                             # reuses the warm pool
    while srv.pending():
        srv.poll()
    assert be.created == 1
    t[0] = 10.0
    srv.poll()
    assert not srv.pools and be.released == 1             # idle past keep_idle_s


def test_idle_pools_are_released_for_budget():
    be = FakeBackend(bytes_per_engine=100)
    srv = Server(be, hbm_budget=150, slots_per_pool=2, keep_idle_s=1e9)
    srv.submit(make(1, 4, 1))
    while srv.pending():
        srv.poll()
    srv.submit(make(2, 6, 1))                             # other shape: needs the idle pool's memory
    while srv.pending():
        srv.poll()
    assert be.created == 2 and be.released == 1 and len(srv.finished) == 2


def test_late_arrivals_join_a_running_pool():
    be = FakeBackend()
    srv = Server(be, hbm_budget=1000, slots_per_pool=4)
    a = make(1, 4, 6)
    srv.submit(a)
    srv.poll()
    srv.poll()
    b = make(2, 4, 2)
    srv.submit(b)
    while srv.pending():
        srv.poll()
    assert be.created == 1                     # same shape: admitted into the running pool
    assert b.done <= a.done and b.admitted > a.admitted


@pytest.mark.gpu
def test_results_alone_equal_results_in_the_mix():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07440_gb300.serving import GpuBackend
    shapes = [HolsteinParams(nx=4, ny=4, beta=1.0, seed=11), HolsteinParams(nx=6, ny=6, beta=0.5, seed=12),
              HolsteinParams(nx=4, ny=4, beta=1.0, g=1.0, mu=-1.0, seed=13)]
    reqs = []
    for k in range(12):
        p = shapes[k % 3].with_(seed=1000 + k)
        reqs.append(Request(rid=k, params=p, X0=initial_fields(p, 1, seed=50 + k)[0], sweeps=2 + k % 3,
                            chain_id=k, arrival=0.002 * k))
    mix = Server(GpuBackend(), hbm_budget=8 << 30, slots_per_pool=4).run(reqs)
    assert len(mix) == 12
    for r in mix:
        alone = Server(GpuBackend(), hbm_budget=8 << 30, slots_per_pool=1).run(
            [Request(rid=r.rid, params=r.params, X0=initial_fields(r.params, 1, seed=50 + r.rid)[0],
                     sweeps=r.sweeps, chain_id=r.chain_id)])
        assert np.array_equal(alone[0].X, r.X), r.rid
        assert alone[0].obs["local_accepted"] == r.obs["local_accepted"]


@pytest.mark.gpu
def test_learned_requests_alone_equal_in_the_mix():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import nn
    from paper_1905_07440_gb300.serving import GpuBackend
    th = nn.init_params(4)
    th[-nn.N_H - 1:] *= 2.0
    base = HolsteinParams(nx=4, ny=4, beta=1.0)
    reqs = []
    for k in range(6):
        p = base.with_(seed=500 + k)
        kind = "learned" if k % 2 == 0 else "plain"
        reqs.append(Request(rid=k, params=p, X0=initial_fields(p, 1, seed=70 + k)[0], sweeps=2 + k % 2,
                            sampler=kind, theta=th if kind == "learned" else None, chain_id=k))
    mix = Server(GpuBackend(), hbm_budget=8 << 30, slots_per_pool=4).run(reqs)
    assert len(mix) == 6
    for r in mix:
        solo = Request(rid=r.rid, params=r.params, X0=initial_fields(r.params, 1, seed=70 + r.rid)[0],
                       sweeps=r.sweeps, sampler=r.sampler, theta=r.theta, chain_id=r.chain_id)
        alone = Server(GpuBackend(), hbm_budget=8 << 30, slots_per_pool=1).run([solo])
        assert np.array_equal(alone[0].X, r.X), r.rid
        if r.sampler == "learned":
            assert alone[0].obs["cumulative_accepted"] == r.obs["cumulative_accepted"]


@pytest.mark.gpu
def test_served_requests_match_the_oracle():
    """A plain and a learned request served in a mix with other requests end on the oracle
    chain with the request's identity (key = its seed, chain word = chain_id, counter from 0):
    plain fields bit for bit; learned fields bit for bit unless a decision was closer than the
    FP32 network can resolve (|u - p|/p < 1e-4)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import dqmc, nn
    from paper_1905_07440_gb300.serving import GpuBackend
    th = nn.init_params(4)
    th[-nn.N_H - 1:] *= 2.0
    shapes = [HolsteinParams(nx=4, ny=4, beta=1.0), HolsteinParams(nx=6, ny=4, beta=0.8, g=1.0, mu=-1.0)]
    reqs = []
    for k in range(8):
        p = shapes[k % 2].with_(seed=700 + k)
        kind = "learned" if (k % 4 == 0 and p.nx >= 4 and p.ny >= 4) else "plain"
        reqs.append(Request(rid=k, params=p, X0=initial_fields(p, 1, seed=90 + k)[0], sweeps=2 + k % 2,
                            sampler=kind, theta=th if kind == "learned" else None, chain_id=40 + k,
                            arrival=0.001 * k))
    done = {r.rid: r for r in Server(GpuBackend(), hbm_budget=8 << 30, slots_per_pool=3).run(reqs)}
    assert len(done) == 8
    thb = nn.to_bfloat16(th.astype(np.float32))
    checked = {"plain": 0, "learned": 0}
    for k in (0, 1, 3, 4):
        r = done[k]
        X0 = initial_fields(r.params, 1, seed=90 + k)[0]
        if r.sampler == "plain":
            ch = dqmc.OracleChain(r.params, X0, chain=r.chain_id)
            recs = [ch.sweep() for _ in range(r.sweeps)]
            assert np.array_equal(r.X, ch.X), k
            assert r.obs["local_accepted"] == sum(x["local_accepted"] for x in recs)
            checked["plain"] += 1
        else:
            ch = nn.CumulativeChain(r.params, X0, thb, chain=r.chain_id)
            acc = sum(ch.step(j, 1)[1] for j in range(r.sweeps))
            if np.array_equal(r.X, ch.X):
                assert r.obs["cumulative_accepted"] == acc
                checked["learned"] += 1
            else:
                assert ch.min_margin < 1e-4, ch.min_margin
    assert checked["plain"] >= 2 and checked["learned"] >= 1, checked
