"""GPU parity of the learned effective action and the cumulative sampler against the oracle.

Network outputs use bfloat16 weights (the same rounded values on both sides) and FP32
arithmetic on the GPU, FP64 in the oracle: F and its gradient must agree to 2e-3 relative.
The cumulative accept uses the exact FP64 log-determinants, so the chain samples the exact
weight whatever the network: a run with a random network must reproduce the free-phonon
closed form at g = 0, and plain and learned samplers must agree on observables at g != 0.
"""
import math

import numpy as np
import pytest

from workloads import HolsteinParams, initial_fields, random_fields

pytestmark = pytest.mark.gpu

NN_RTOL = 2e-3


@pytest.fixture(scope="module")
def hq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1905_07440_gb300 as mod
    mod.load_library()
    return mod


def scaled_params(seed, scale):
    from oracle import nn
    th = nn.init_params(seed)
    th[-nn.N_H - 1:] *= scale  # output layer
    return th


def test_effective_action_matches_oracle(hq):
    from oracle import nn
    for nx, beta, seed in ((4, 1.0, 1), (6, 0.8, 2)):
        p = HolsteinParams(nx=nx, ny=nx, beta=beta)
        X = random_fields(p, 3, seed=seed, offset=-1.4)
        th = scaled_params(seed, 5.0)
        eng = hq.Engine(p, 3)
        eng.attach_network(4, 8)
        eng.set_params(th)
        assert np.array_equal(eng.get_params(bf16=True).astype(np.float64), nn.to_bfloat16(th.astype(np.float32)))
        eng.set_fields(X)
        F = eng.nn_eval()
        act = nn.EffectiveAction(p, nn.to_bfloat16(th.astype(np.float32)))
        for c in range(3):
            ref = act.F(X[c])
            assert abs(F[c] - ref) <= NN_RTOL * max(1.0, abs(ref)), (F[c], ref)


def test_gradient_matches_oracle(hq):
    import torch
    from oracle import nn
    p = HolsteinParams(nx=4, ny=4, beta=0.6)
    X = random_fields(p, 6, seed=7, offset=-1.4)
    y = np.linspace(-2.0, 3.0, 6)
    th = scaled_params(3, 3.0)
    eng = hq.Engine(p, 1)
    eng.attach_network(8, 8)
    eng.set_params(th)
    g, loss = eng.nn_gradient(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    lref, gref = nn.loss_and_grad(p, nn.to_bfloat16(th.astype(np.float32)), X, y)
    assert abs(loss - lref) <= NN_RTOL * lref
    assert np.max(np.abs(g - gref)) <= NN_RTOL * np.max(np.abs(gref))


def test_training_lowers_the_loss(hq):
    import torch
    from oracle import nn
    p = HolsteinParams(nx=4, ny=4, beta=0.6)
    rng = np.random.default_rng(0)
    X = random_fields(p, 64, seed=11, offset=-1.4)
    target = nn.EffectiveAction(p, nn.to_bfloat16(scaled_params(9, 20.0).astype(np.float32)))
    y = np.array([target.F(x) for x in X])
    y -= y.mean()
    eng = hq.Engine(p, 1)
    eng.attach_network(16, 64)
    eng.set_params(scaled_params(1, 1.0))
    losses = eng.nn_train(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), epochs=30, batch=16, lr=3e-3, seed=5)
    assert losses[-1] < 0.2 * losses[0], losses


@pytest.mark.parametrize("split", [1, 2])
def test_cumulative_step_matches_oracle(hq, split):
    """Cumulative steps with the exact log|det M(X')| from one CTA per chain (split 1) or from
    two halves joined by the two-sided formula (split 2) follow the oracle chain."""
    from oracle import nn
    p = HolsteinParams(nx=4, ny=4, beta=1.0, n_wrap=3, seed=31)
    C = 3
    X0 = initial_fields(p, C, seed=3)
    th = scaled_params(4, 2.0)
    eng = hq.Engine(p, C)
    m = eng.set_logdet_split(split)
    assert (m > 0) == (split == 2) and m % p.n_wrap == 0 and m < p.n_slices
    eng.attach_network(4, 8)
    eng.set_params(th)
    eng.set_fields(X0)
    eng.cumulative(n_steps=2, n_inner=1)
    Xg = eng.get_fields()
    stats = eng.learned_stats()
    _, ld = eng.log_weight()
    thb = nn.to_bfloat16(th.astype(np.float32))
    for c in range(C):
        ch = nn.CumulativeChain(p, X0[c], thb, chain=c)
        acc = 0
        for k in range(2):
            pc, a = ch.step(k, 1)
            acc += a
        if np.array_equal(Xg[c], ch.X):
            assert stats[c]["cumulative_accepted"] == acc
            assert abs(stats[c]["last_pc"] - pc) <= 1e-3 * max(pc, 1e-12) or (pc > 1 and stats[c]["last_pc"] > 1)
            assert abs(ld[c] - ch.logdet) <= 1e-10 * abs(ch.logdet)
        else:
            # divergence only through a decision the FP32 network could not resolve
            assert ch.min_margin < 1e-4, ch.min_margin


def equilibrated(hq, p, C, sweeps, seed):
    """Fields of C chains after `sweeps` plain sweeps (exact sampler), and their log|det M|."""
    eng = hq.Engine(p, C)
    eng.set_fields(initial_fields(p, C, seed=seed))
    eng.sweep(sweeps)
    X = eng.get_fields()
    _, ld = eng.log_weight()
    return X, ld


@pytest.mark.slow
def test_cumulative_sampler_is_exact_for_free_phonons(hq):
    """g = 0: log|det M| does not depend on X, so whatever the network the chain must sample
    exp(-dtau S_ph); <X^2> must match the Gaussian closed form.  Chains start equilibrated."""
    from tests import closed_forms as cf
    p = HolsteinParams(nx=4, ny=4, beta=2.0, g=0.0, mu=0.0, seed=5)
    C, steps, burn = 64, 80, 10
    X, _ = equilibrated(hq, p, C, 40, seed=8)
    eng = hq.Engine(p, C, max_series=steps)
    eng.attach_network(4, 8)
    eng.set_params(scaled_params(2, 0.3))
    eng.set_fields(X)
    eng.cumulative(n_steps=steps, n_inner=1)
    s = eng.series(hq.HQ_OBS_X2)[:, burn:]
    per_chain = s.mean(axis=1)
    mean, err = per_chain.mean(), per_chain.std(ddof=1) / math.sqrt(C)
    ref = cf.free_phonon_x2(p.n_slices, p.dtau, p.mass, p.omega)
    st = eng.learned_stats()
    rate = sum(x["cumulative_accepted"] for x in st) / sum(x["cumulative_proposed"] for x in st)
    assert rate > 0.2, rate
    assert abs(mean - ref) < 4 * err, (mean, ref, err, rate)


@pytest.mark.slow
def test_trained_network_sampler_agrees_with_plain_within_two_error_bars(hq):
    """g != 0 at half filling, 6x6, beta = 4: train the network on plain-sampler configurations,
    then run the plain sampler and the cumulative sampler (exact accept) from the same
    equilibrated fields, each with a fresh Philox key, for at least 20 tau_int.  <X^2>, the
    double occupancy and S_CDW(pi,pi) must agree within two error bars (errors from the spread
    of the 256 independent chains' means), both series must be stationary (second half minus
    first half within three error bars), and the trained network must be accepted far more
    often than an untrained one."""
    import torch
    p = HolsteinParams(nx=6, ny=6, beta=4.0, seed=17)
    C, warm, meas = 256, 200, 300
    x0 = -p.g / (p.mass * p.omega ** 2)
    eng = hq.Engine(p, C)
    eng.set_fields(initial_fields(p, C, seed=2) + x0)
    eng.sweep(warm)
    Xs, ys = [], []
    for _ in range(16):
        eng.sweep(2)
        Xs.append(eng.get_fields())
        ys.append(eng.log_weight()[1])
    Xtr = np.concatenate(Xs)
    ytr = np.concatenate(ys)
    ytr = ytr - ytr.mean()
    net = hq.Engine(p, 1)
    net.attach_network(64, Xtr.shape[0])
    net.set_params(scaled_params(1, 1.0))
    Xd, yd = torch.from_numpy(Xtr).cuda(), torch.from_numpy(ytr).cuda()
    losses = []
    for k in range(3):
        losses.extend(net.nn_train(Xd, yd, epochs=20, batch=64, lr=3e-3 * 0.5 ** k, seed=3 + k))
    assert losses[-1] < 0.05 * np.var(ytr), (losses[-1], np.var(ytr))
    theta = net.get_params()
    X0 = eng.get_fields()
    res, rates, taus = {}, {}, {}
    names = ((hq.HQ_OBS_X2, "x2"), (hq.HQ_OBS_DOUBLE_OCC, "d"), (hq.HQ_OBS_SCDW, "s"))
    for k, (kind, th, steps) in enumerate((("plain", None, meas), ("trained", theta, meas),
                                           ("untrained", scaled_params(6, 1.0), 40))):
        # a fresh Philox key per run: the training engine's key with counters from 0 again
        # would replay the noise that produced X0 and couple the run to that trajectory
        e = hq.Engine(p.with_(seed=p.seed + 101 * (k + 1)), C, max_series=steps)
        e.set_fields(X0)
        if th is None:
            e.sweep(steps)
        else:
            e.attach_network(4, 8)
            e.set_params(th)
            e.cumulative(n_steps=steps, n_inner=1, measure=True)
            st = e.learned_stats()
            rates[kind] = sum(x["cumulative_accepted"] for x in st) / sum(x["cumulative_proposed"] for x in st)
        if kind == "untrained":
            continue
        res[kind] = {}
        for oid, name in names:
            ser = e.series(oid)
            pc = ser.mean(axis=1)
            half = ser[:, steps // 2:].mean(axis=1) - ser[:, : steps // 2].mean(axis=1)
            res[kind][name] = (pc.mean(), pc.std(ddof=1) / math.sqrt(C), half.mean(), half.std(ddof=1) / math.sqrt(C))
            taus[(kind, name)] = np.mean([hq.tau_int(ser[c])[0] for c in range(C)])
    assert rates["trained"] > 0.3 and rates["trained"] > 2 * rates["untrained"], rates
    for key, tau in taus.items():
        assert meas >= 20 * tau, (key, tau)
    for _, name in names:
        (a, ea, ha, hea), (b, eb, hb, heb) = res["plain"][name], res["trained"][name]
        assert abs(a - b) < 2.0 * math.hypot(ea, eb), (name, a, b, ea, eb, rates)
        assert abs(ha) < 3.0 * hea and abs(hb) < 3.0 * heb, (name, ha, hea, hb, heb)


@pytest.mark.parametrize("window,sites", [(3, 0), (7, 0), (0, 5), (4, 6)])
def test_cumulative_window_matches_oracle(hq, window, sites):
    """Cumulative steps whose local moves visit a random window of slices and whose block
    moves visit a random run of sites follow the oracle."""
    from oracle import nn
    p = HolsteinParams(nx=4, ny=4, beta=1.0, seed=37)
    C = 3
    X0 = initial_fields(p, C, seed=6)
    th = scaled_params(5, 2.0)
    eng = hq.Engine(p, C)
    eng.attach_network(4, 8)
    eng.set_params(th)
    eng.set_inner_window(window)
    eng.set_inner_sites(sites)
    eng.set_fields(X0)
    eng.cumulative(n_steps=3, n_inner=1)
    Xg = eng.get_fields()
    stats = eng.learned_stats()
    thb = nn.to_bfloat16(th.astype(np.float32))
    for c in range(C):
        assert stats[c]["inner_local_proposed"] == 3 * (window or p.n_slices) * p.n_sites
        assert stats[c]["inner_block_proposed"] == 3 * (sites or p.n_sites)
        ch = nn.CumulativeChain(p, X0[c], thb, chain=c)
        acc = sum(ch.step(k, 1, window=window, site_window=sites)[1] for k in range(3))
        if np.array_equal(Xg[c], ch.X):
            assert stats[c]["cumulative_accepted"] == acc
        else:
            assert ch.min_margin < 1e-4, ch.min_margin
        # slices outside every window visited keep their values unless a block move shifted them
        d = Xg[c] - X0[c]
        assert np.all(np.isfinite(d))


@pytest.mark.parametrize("split", [1, 2])
def test_measured_cumulative_steps_match_oracle_measurements(hq, split):
    """Measured cumulative steps: the recorded density, double occupancy and S_CDW(pi,pi) of
    each step are those of G_m of the chain's fields after the step (the oracle's fresh G_m;
    m = 0 with one CTA per chain, the split boundary with two halves), for accepted and
    rejected steps alike (a rejected step restores the saved G_m)."""
    from oracle import dqmc, nn
    p = HolsteinParams(nx=4, ny=4, beta=1.0, n_wrap=4, seed=43)
    C, steps = 3, 4
    X0 = initial_fields(p, C, seed=8)
    th = scaled_params(7, 2.0)
    eng = hq.Engine(p, C, max_series=steps)
    m = eng.set_logdet_split(split)
    eng.attach_network(4, 8)
    eng.set_params(th)
    eng.set_fields(X0)
    eng.cumulative(n_steps=steps, n_inner=1, measure=True)
    Xg = eng.get_fields()
    ser = {k: eng.series(k) for k in (hq.HQ_OBS_DENSITY, hq.HQ_OBS_DOUBLE_OCC, hq.HQ_OBS_SCDW)}
    thb = nn.to_bfloat16(th.astype(np.float32))
    expK, _ = dqmc.kinetic_propagators(p)
    checked = 0
    for c in range(C):
        ch = nn.CumulativeChain(p, X0[c], thb, chain=c)
        recs = []
        for k in range(steps):
            ch.step(k, 1)
            recs.append(dqmc.measure_green(p, dqmc.green_at(p, expK, ch.X, m)[0]))
        if not np.array_equal(Xg[c], ch.X):
            assert ch.min_margin < 1e-4, ch.min_margin
            continue
        checked += 1
        for k in range(steps):
            for oid, name in ((hq.HQ_OBS_DENSITY, "density"), (hq.HQ_OBS_DOUBLE_OCC, "double_occ"),
                              (hq.HQ_OBS_SCDW, "s_cdw")):
                assert abs(ser[oid][c, k] - recs[k][name]) < 1e-9, (c, k, name)
    assert checked >= 2
