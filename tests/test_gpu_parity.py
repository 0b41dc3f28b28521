"""GPU parity: the CUDA engine (through the C ABI) against the CPU oracle.

Tolerances (FP64 steps): log|det M| and log W to 1e-10 relative, G to 1e-10 absolute
(|G_ij| <= 1), per-sweep electronic observables to 1e-9.  Decisions are identical under
the shared Philox stream, so fields X must match bit for bit and acceptance counts
exactly.
"""
import math

import numpy as np
import pytest

from workloads import HolsteinParams, SMALL, BATCHED, LARGEST, initial_fields, random_fields, uniform_fields

pytestmark = pytest.mark.gpu

LD_RTOL = 1e-10
G_ATOL = 1e-10
OBS_ATOL = 1e-9


@pytest.fixture(scope="module")
def hq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1905_07440_gb300 as mod
    mod.load_library()
    return mod


def oracle_chains(p, X0, n_sweeps, flags=(True, True), block_sites=0):
    from oracle import dqmc
    out = []
    for c in range(X0.shape[0]):
        ch = dqmc.OracleChain(p, X0[c], chain=c)
        recs = [ch.sweep(do_local=flags[0], do_global=flags[1], block_sites=block_sites) for _ in range(n_sweeps)]
        out.append((ch, recs))
    return out


def check_against_oracle(hq, p, X0, n_sweeps, local=True, global_=True, max_series=8, block_sites=0):
    eng = hq.Engine(p, X0.shape[0], max_series=max_series)
    eng.set_block_sites(block_sites)
    eng.set_fields(X0)
    eng.sweep(n_sweeps, local=local, global_=global_, measure=True)
    Xg = eng.get_fields()
    lw, ld = eng.log_weight()
    obs = eng.observables()
    series = {k: eng.series(k) for k in range(hq.HQ_N_OBS)}
    ref = oracle_chains(p, X0, n_sweeps, (local, global_), block_sites)
    for c, (ch, recs) in enumerate(ref):
        assert np.array_equal(Xg[c], ch.X), f"chain {c}: fields differ"
        assert abs(ld[c] - ch.logdet) <= LD_RTOL * max(1.0, abs(ch.logdet))
        assert abs(lw[c] - ch.log_weight()) <= LD_RTOL * max(1.0, abs(ch.log_weight()))
        G = eng.green(c)
        assert np.max(np.abs(G - ch.G)) < G_ATOL
        if local:
            assert obs[c]["local_accepted"] == sum(r["local_accepted"] for r in recs)
        if global_:
            assert obs[c]["global_accepted"] == sum(r["global_accepted"] for r in recs)
            assert obs[c]["global_proposed"] == n_sweeps * (block_sites or p.n_sites)
        for s, r in enumerate(recs):
            for k, name in ((hq.HQ_OBS_X_MEAN, "x_mean"), (hq.HQ_OBS_X2, "x2")):
                assert abs(series[k][c, s] - r[name]) < OBS_ATOL
            if local:
                for k, name in ((hq.HQ_OBS_DENSITY, "density"), (hq.HQ_OBS_DOUBLE_OCC, "double_occ"),
                                (hq.HQ_OBS_SCDW, "s_cdw")):
                    assert abs(series[k][c, s] - r[name]) < OBS_ATOL, name
                assert series[hq.HQ_OBS_WRAP_ERR][c, s] < 1e-9
        assert obs[c]["status"] == 0
    eng.close()


# ------------------------------------------------------------ proposal stream

def test_proposal_stream_matches_oracle_and_known_answers(hq):
    from oracle import philox
    # published Philox4x32-10 known answer: counter 0, key 0
    u1, u2 = hq.proposal_uniforms(0, 0, 0, [0], 0)
    assert u1[0] == philox.words_to_uniform(0x6627E8D5, 0xE169C58D)
    assert u2[0] == philox.words_to_uniform(0xBC57AC4C, 0x9B00DBD8)
    ev = np.arange(0, 100000, 7)
    for seed, chain, sweep, tag in ((20190517, 3, 11, 0), (2 ** 40 + 5, 255, 999, 1)):
        g1, g2 = hq.proposal_uniforms(seed, chain, sweep, ev, tag)
        o1, o2 = philox.proposal_uniforms(seed, chain, sweep, ev, tag)
        assert np.array_equal(g1, o1) and np.array_equal(g2, o2)


# ------------------------------------------------------ weights from the fields

@pytest.mark.parametrize("nx,beta,n_wrap,chains", [(2, 1.0, 3, 3), (4, 4.0, 10, 4), (6, 2.5, 4, 2),
                                                   (8, 8.0, 10, 3), (12, 2.0, 10, 2)])
def test_log_weight_and_green_from_fields(hq, nx, beta, n_wrap, chains):
    from oracle import dqmc
    p = HolsteinParams(nx=nx, ny=nx, beta=beta, n_wrap=n_wrap)
    X = random_fields(p, chains, seed=100 + nx, scale=1.0, offset=-1.2)
    eng = hq.Engine(p, chains)
    eng.set_fields(X)
    lw, ld = eng.log_weight()
    expK, _ = dqmc.kinetic_propagators(p)
    for c in range(chains):
        G_ref, ld_ref = dqmc.green_at(p, expK, X[c], 0)
        assert abs(ld[c] - ld_ref) <= LD_RTOL * abs(ld_ref)
        lw_ref = 2 * ld_ref - dqmc.phonon_action(p, X[c])
        assert abs(lw[c] - lw_ref) <= LD_RTOL * abs(lw_ref)
        assert np.max(np.abs(eng.green(c) - G_ref)) < G_ATOL


def test_uniform_field_closed_form_on_largest_lattice(hq):
    """log det M = sum_k log(1 + exp(-beta (eps_k + g x0 - mu))) at 16x16, beta = 16."""
    from tests import closed_forms as cf
    p = LARGEST
    x0 = (-0.9, 0.3)
    X = np.concatenate([uniform_fields(p, 1, v) for v in x0])
    eng = hq.Engine(p, 2)
    eng.set_fields(X)
    _, ld = eng.log_weight()
    for c, v in enumerate(x0):
        ref = cf.free_logdet(16, 16, p.t, p.mu, p.beta, shift=p.g * v)
        assert abs(ld[c] - ref) <= LD_RTOL * abs(ref)
        assert np.max(np.abs(eng.green(c) - cf.free_green(16, 16, p.t, p.mu, p.beta, shift=p.g * v))) < G_ATOL


def test_particle_hole_symmetry_on_gpu(hq):
    p = HolsteinParams(nx=8, ny=8, beta=8.0)
    X = random_fields(p, 2, seed=4, offset=-1.0)
    c = -2.0 * p.g / (p.mass * p.omega ** 2)
    eng = hq.Engine(p, 4)
    eng.set_fields(np.concatenate([X, c - X]))
    lw, _ = eng.log_weight()
    for k in range(2):
        assert abs(lw[k] - lw[k + 2]) <= 1e-10 * abs(lw[k])


# ---------------------------------------------------------------- full sweeps

def test_sweeps_small_workload(hq):
    """4x4, beta = 4 (L = 40), k = 16: the small workload's shape, two chains, three sweeps."""
    X0 = initial_fields(SMALL, 2)
    check_against_oracle(hq, SMALL, X0, 3)


@pytest.mark.parametrize("nx,beta,n_wrap,k", [(2, 1.0, 3, 1), (2, 0.2, 10, 4), (4, 2.0, 7, 3),
                                              (6, 2.0, 5, 32), (8, 1.5, 4, 16)])
def test_sweeps_ragged_and_edge_shapes(hq, nx, beta, n_wrap, k):
    p = HolsteinParams(nx=nx, ny=nx, beta=beta, n_wrap=n_wrap, delay_k=k, seed=77 + nx)
    X0 = initial_fields(p, 2, seed=5)
    check_against_oracle(hq, p, X0, 2)


@pytest.mark.parametrize("nx,beta,n_wrap,method", [(6, 1.0, 2, 0), (6, 1.0, 5, 1), (8, 2.0, 10, 1), (4, 1.0, 3, 0)])
def test_block_move_methods_against_oracle(hq, nx, beta, n_wrap, method):
    """Both block-move algorithms (separable slices per move / chunk propagators) agree with
    the oracle; the flop model picks the one named for each shape."""
    p = HolsteinParams(nx=nx, ny=nx, beta=beta, n_wrap=n_wrap, delay_k=8, seed=11)
    eng = hq.Engine(p, 1)
    assert eng.block_move_method == method
    eng.close()
    X0 = initial_fields(p, 2, seed=21)
    check_against_oracle(hq, p, X0, 2, local=True, global_=True)


@pytest.mark.parametrize("nx,beta,n_wrap", [(4, 1.0, 3), (8, 1.0, 10), (6, 2.0, 7)])
@pytest.mark.parametrize("forced", [1, 2])
def test_forced_block_move_method_against_oracle(hq, nx, beta, n_wrap, forced):
    """block_method forces either algorithm whatever the flop model says; both agree with the
    oracle (fields bit for bit, log-determinants and G to rounding)."""
    p = HolsteinParams(nx=nx, ny=nx, beta=beta, n_wrap=n_wrap, delay_k=8, seed=13, block_method=forced)
    eng = hq.Engine(p, 1)
    assert eng.block_move_method == forced - 1
    eng.close()
    X0 = initial_fields(p, 2, seed=23)
    check_against_oracle(hq, p, X0, 1, local=False, global_=True)


def test_autotune_times_every_pair(hq):
    import torch
    p = HolsteinParams(nx=6, ny=6, beta=1.0, seed=3)
    X = torch.from_numpy(initial_fields(p, 8, seed=1)).cuda()
    table, bk, bm = hq.autotune(p, X, ks=(4, 16), methods=(1, 2), warmup=1, reps=1)
    assert set(table) == {(4, 1), (4, 2), (16, 1), (16, 2)}
    assert all(v > 0 for v in table.values())
    assert table[(bk, bm)] == min(table.values())
    # the fields given to the autotuner are not modified
    assert np.array_equal(X.cpu().numpy(), initial_fields(p, 8, seed=1))


def test_local_only_and_global_only(hq):
    p = HolsteinParams(nx=4, ny=4, beta=2.0, delay_k=5)
    X0 = initial_fields(p, 2, seed=9)
    check_against_oracle(hq, p, X0, 2, local=True, global_=False)
    check_against_oracle(hq, p, X0, 2, local=False, global_=True)


def test_delay_rank_does_not_change_the_chain(hq):
    base = HolsteinParams(nx=6, ny=6, beta=3.0, n_wrap=10)
    X0 = initial_fields(base, 3, seed=2)
    res = []
    for k in (1, 2, 16, 32):
        eng = hq.Engine(base.with_(delay_k=k), 3)
        eng.set_fields(X0)
        eng.sweep(2)
        res.append((eng.get_fields(), eng.log_weight()[1], [eng.green(c) for c in range(3)]))
    for X, ld, Gs in res[1:]:
        assert np.array_equal(X, res[0][0])
        assert np.max(np.abs(ld - res[0][1]) / np.abs(res[0][1])) < LD_RTOL
        for a, b in zip(Gs, res[0][2]):
            assert np.max(np.abs(a - b)) < G_ATOL


def test_zero_width_moves_accept_everything(hq):
    p = HolsteinParams(nx=4, ny=4, beta=1.0, dx_local=0.0, dx_global=0.0)
    X0 = initial_fields(p, 1)
    eng = hq.Engine(p, 1)
    eng.set_fields(X0)
    eng.sweep(1)
    o = eng.observables()[0]
    assert o["local_accepted"] == o["local_proposed"] == p.n_sites * p.n_slices
    assert o["global_accepted"] == o["global_proposed"] == p.n_sites
    assert np.array_equal(eng.get_fields(), X0)


def test_checkpoint_resume_equals_straight_run(hq):
    p = HolsteinParams(nx=4, ny=4, beta=2.0, delay_k=8)
    X0 = initial_fields(p, 2, seed=13)
    a = hq.Engine(p, 2, max_series=8)
    a.set_fields(X0)
    a.sweep(4)
    b = hq.Engine(p, 2, max_series=8)
    b.set_fields(X0)
    b.sweep(2)
    blob = b.checkpoint()
    c = hq.Engine(p, 2, max_series=8)
    c.restore(blob)
    c.sweep(2)
    assert np.array_equal(a.get_fields(), c.get_fields())
    assert c.sweeps_done == 4
    for k in range(hq.HQ_N_OBS):
        assert np.allclose(a.series(k), c.series(k), rtol=0, atol=1e-12, equal_nan=True)
    oa, oc = a.observables(), c.observables()
    for x, y in zip(oa, oc):
        assert x["local_accepted"] == y["local_accepted"] and x["global_accepted"] == y["global_accepted"]
    assert np.max(np.abs(a.green(1) - c.green(1))) < G_ATOL


def test_batched_workload_sampled_chains(hq):
    """8x8, beta = 8 (L = 80), 256 chains, k = 16, local + one block move per site: the
    batched launch as timed by the benchmark; chains 0, 97 and 255 checked against the
    oracle after one sweep, all chains for status and a finite weight."""
    C = 256
    X0 = initial_fields(BATCHED, C)
    eng = hq.Engine(BATCHED, C, max_series=4)
    eng.set_fields(X0)
    eng.sweep(1)
    Xg = eng.get_fields()
    lw, ld = eng.log_weight()
    obs = eng.observables()
    assert all(o["status"] == 0 for o in obs)
    assert np.all(np.isfinite(lw))
    from oracle import dqmc
    for c in (0, 97, 255):
        ch = dqmc.OracleChain(BATCHED, X0[c], chain=c)
        r = ch.sweep()
        assert np.array_equal(Xg[c], ch.X)
        assert abs(ld[c] - ch.logdet) <= LD_RTOL * abs(ch.logdet)
        assert np.max(np.abs(eng.green(c) - ch.G)) < G_ATOL
        assert obs[c]["local_accepted"] == r["local_accepted"]
        assert obs[c]["global_accepted"] == r["global_accepted"]
        assert abs(eng.series(hq.HQ_OBS_SCDW)[c, 0] - r["s_cdw"]) < OBS_ATOL


def test_largest_lattice_local_sweep_sampled(hq):
    """16x16, beta = 16 (L = 160): a local sweep of 4 chains, chain 2 against the oracle."""
    C = 4
    X0 = initial_fields(LARGEST, C)
    eng = hq.Engine(LARGEST, C, max_series=2)
    eng.set_fields(X0)
    eng.sweep(1, local=True, global_=False)
    from oracle import dqmc
    ch = dqmc.OracleChain(LARGEST, X0[2], chain=2)
    r = ch.sweep(do_local=True, do_global=False)
    assert np.array_equal(eng.get_fields()[2], ch.X)
    assert abs(eng.log_weight()[1][2] - ch.logdet) <= LD_RTOL * abs(ch.logdet)
    assert np.max(np.abs(eng.green(2) - ch.G)) < G_ATOL
    assert abs(eng.series(hq.HQ_OBS_DENSITY)[2, 0] - r["density"]) < OBS_ATOL


def test_invalid_arguments_are_rejected(hq):
    import ctypes
    lib = hq.load_library()
    p = SMALL
    eng = hq.Engine(p, 1)
    with pytest.raises(hq.HQError):
        eng._check(lib.hq_sweep(eng._h, 1, 64), "hq_sweep")
    with pytest.raises(hq.HQError):
        eng.green(5)
    out = ctypes.c_void_p()
    assert lib.hq_create(ctypes.byref(hq.make_params(p)), 1, 0, 0, None, 0, None, ctypes.byref(out)) == hq.HQ_ENOMEM


def test_slot_identity_matches_oracle_and_is_position_independent(hq):
    """A chain loaded into slot 2 of a mixed engine (own key, chain word, sweep counter; other
    slots busy or idle) follows the oracle chain with that identity, bit for bit."""
    from oracle import dqmc
    p = HolsteinParams(nx=4, ny=4, beta=1.5, delay_k=4)
    X = initial_fields(p, 4, seed=12)
    eng = hq.Engine(p, 4, max_series=4)
    eng.set_fields(X)
    eng.set_chain(2, X[3], seed=987654321, chain_id=77, sweep=5)
    eng.set_active(1, False)
    eng.sweep(2)
    Xg = eng.get_fields()
    assert np.array_equal(Xg[1], X[1])  # idle slot untouched
    ch = dqmc.OracleChain(p.with_(seed=987654321), X[3], chain=77, sweep=5)
    ch.sweep()
    ch.sweep()
    assert np.array_equal(Xg[2], ch.X)
    alone = hq.Engine(p, 1)
    alone.set_chain(0, X[3], seed=987654321, chain_id=77, sweep=5)
    alone.sweep(2)
    assert np.array_equal(alone.get_fields()[0], Xg[2])


def test_graph_replay_equals_eager_sweeps(hq):
    """Sweeps replayed from a captured CUDA graph give bit-identical fields, log-determinants
    and counts to eager sweeps, across changes of flags and of the active slots."""
    import torch
    p = HolsteinParams(nx=6, ny=6, beta=1.2, n_wrap=5, seed=17)
    X0 = initial_fields(p, 4, seed=3)
    runs = []
    for graphs in (False, True):
        eng = hq.Engine(p, 4, max_series=16, stream=torch.cuda.Stream())
        eng.set_fields(X0)
        eng.set_graphs(graphs)
        eng.sweep(3)
        eng.sweep(3, local=False)
        eng.set_active(2, False)
        eng.sweep(3)
        _, ld = eng.log_weight()
        runs.append((eng.get_fields(), ld, eng.observables(), eng.series(hq.HQ_OBS_X2)))
    (Xa, lda, oa, sa), (Xb, ldb, ob, sb) = runs
    assert np.array_equal(Xa, Xb)
    assert np.array_equal(lda, ldb)
    assert np.array_equal(sa, sb, equal_nan=True)
    for c in range(4):
        assert oa[c]["local_accepted"] == ob[c]["local_accepted"]
        assert oa[c]["global_accepted"] == ob[c]["global_accepted"]
    eng = hq.Engine(p, 1)
    if eng.stream.cuda_stream == 0:
        with pytest.raises(hq.HQError):
            eng.set_graphs(True)


def test_bounded_wait_runs_out_and_context_stays_usable(hq):
    """The library's device wait on a flag that nothing sets gives up after its limit and
    reports HQ_ETIMEOUT; the context is still usable: a sweep afterwards matches the oracle."""
    import time
    t0 = time.perf_counter()
    assert hq.wait_probe(0.05) == hq.HQ_ETIMEOUT
    assert hq.wait_probe(0.02) == hq.HQ_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    p = HolsteinParams(nx=4, ny=4, beta=1.0, seed=5)
    check_against_oracle(hq, p, initial_fields(p, 2, seed=4), 1)
