"""Heterogeneous engine groups: engines of different lattices, temperatures and couplings
swept together by one persistent launch compute exactly what each engine computes alone."""
import numpy as np
import pytest

from workloads import HolsteinParams, initial_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1905_07440_gb300 as mod
    mod.load_library()
    return mod


SHAPES = [
    (HolsteinParams(nx=4, ny=4, beta=1.0, n_wrap=3, delay_k=4, seed=101), 3),
    (HolsteinParams(nx=6, ny=6, beta=0.8, g=1.0, mu=-1.0, seed=102), 2),
    (HolsteinParams(nx=8, ny=8, beta=0.5, delay_k=8, seed=103), 4),
    (HolsteinParams(nx=10, ny=6, beta=0.6, n_wrap=4, seed=104, block_method=1), 2),
]


def make(hq, p, C, idle=()):
    eng = hq.Engine(p, C, max_series=4)
    eng.set_fields(initial_fields(p, C, seed=p.seed))
    for k in idle:
        eng.set_active(k, False)
    return eng


@pytest.mark.parametrize("idle", [False, True])
def test_group_equals_each_engine_alone(hq, idle):
    idles = [((1,) if idle and k == 0 else ()) for k in range(len(SHAPES))]
    group_engines = [make(hq, p, C, idles[k]) for k, (p, C) in enumerate(SHAPES)]
    grp = hq.Group(group_engines)
    grp.sweep(2)
    for k, (p, C) in enumerate(SHAPES):
        alone = make(hq, p, C, idles[k])
        alone.sweep(2)
        Xg, Xa = group_engines[k].get_fields(), alone.get_fields()
        assert np.array_equal(Xg, Xa), k
        _, ldg = group_engines[k].log_weight()
        _, lda = alone.log_weight()
        for c in range(C):
            if c in idles[k]:
                assert np.array_equal(Xg[c], initial_fields(p, C, seed=p.seed)[c])
                continue
            assert abs(ldg[c] - lda[c]) <= 1e-12 * abs(lda[c]), (k, c)
        og, oa = group_engines[k].observables(), alone.observables()
        for c in range(C):
            for key in ("local_accepted", "global_accepted", "status"):
                assert og[c][key] == oa[c][key], (k, c, key)
        for oid in (hq.HQ_OBS_DENSITY, hq.HQ_OBS_X2, hq.HQ_OBS_SCDW):
            sg, sa = group_engines[k].series(oid), alone.series(oid)
            assert np.array_equal(np.isnan(sg), np.isnan(sa))
            assert np.allclose(sg[~np.isnan(sg)], sa[~np.isnan(sa)], rtol=1e-12, atol=0)
    grp.close()


def test_group_chains_match_the_oracle(hq):
    """One chain of every engine of a group against the CPU oracle chain with that chain's
    identity (Philox key = the engine's seed, chain word = its index, sweep counter from 0):
    fields bit for bit, log|det M| and G to 1e-10, acceptance counts exact."""
    from oracle import dqmc
    engines = [make(hq, p, C) for p, C in SHAPES]
    grp = hq.Group(engines)
    grp.sweep(2)
    for k, (p, C) in enumerate(SHAPES):
        c = C - 1
        X0 = initial_fields(p, C, seed=p.seed)[c]
        ch = dqmc.OracleChain(p, X0, chain=c)
        recs = [ch.sweep() for _ in range(2)]
        eng = engines[k]
        assert np.array_equal(eng.get_fields()[c], ch.X), k
        _, ld = eng.log_weight()
        assert abs(ld[c] - ch.logdet) <= 1e-10 * abs(ch.logdet), k
        assert np.max(np.abs(eng.green(c) - ch.G)) < 1e-10, k
        o = eng.observables()[c]
        assert o["local_accepted"] == sum(r["local_accepted"] for r in recs), k
        assert o["global_accepted"] == sum(r["global_accepted"] for r in recs), k
        s = eng.series(hq.HQ_OBS_SCDW)[c]
        assert np.max(np.abs(s - np.array([r["s_cdw"] for r in recs]))) < 1e-9, k
    grp.close()


def test_group_then_engine_calls_are_ordered(hq):
    """After a group sweep an engine's own sweep continues from the group's result."""
    engines = [make(hq, p, C) for p, C in SHAPES[:2]]
    grp = hq.Group(engines)
    grp.sweep(1)
    for e in engines:
        e.sweep(1)
    grp.sweep(1)
    for k, (p, C) in enumerate(SHAPES[:2]):
        alone = make(hq, p, C)
        alone.sweep(3)
        assert np.array_equal(engines[k].get_fields(), alone.get_fields()), k


def test_group_rejects_bad_sets(hq):
    import ctypes
    lib = hq.load_library()
    e = make(hq, *SHAPES[0])
    arr = (ctypes.c_void_p * 2)(e._h.value, e._h.value)
    assert lib.hq_group_arena_bytes(arr, 2) == 0          # repeated engine
    assert lib.hq_group_arena_bytes(arr, 0) == 0
    with pytest.raises(hq.HQError):
        hq.Group([e, e])
