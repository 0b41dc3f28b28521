"""GPU parity of the convolutional action (block moves) against the oracle.

F_cnn, its training gradient and the cumulative sampler with convolutional block moves are
compared with oracle/cnn.py and oracle/nn.py's CumulativeChain (bfloat16-rounded weights on
both sides; FP32 arithmetic on the GPU, FP64 in the oracle: 2e-3 relative).  The window
update of a block move is checked on lattices narrower and wider than the 7-site window,
and the sampler's exactness on the free-phonon closed form.
"""
import math

import numpy as np
import pytest

from workloads import HolsteinParams, initial_fields, random_fields

pytestmark = pytest.mark.gpu

RTOL = 2e-3


@pytest.fixture(scope="module")
def hq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1905_07440_gb300 as mod
    mod.load_library()
    return mod


def bf(theta):
    from oracle import nn
    return nn.to_bfloat16(np.asarray(theta, dtype=np.float32))


def engine(hq, p, C, th_fc, th_cnn, max_series=0):
    eng = hq.Engine(p, C, max_series=max_series)
    eng.attach_network(8, 8)
    eng.set_params(th_fc)
    eng.cnn_set_params(th_cnn)
    return eng


@pytest.mark.parametrize("nx,ny,beta", [(4, 4, 0.6), (6, 4, 0.8), (8, 8, 0.5), (10, 8, 0.5)])
def test_cnn_eval_matches_oracle(hq, nx, ny, beta):
    from oracle import cnn, nn
    p = HolsteinParams(nx=nx, ny=ny, beta=beta)
    X = random_fields(p, 3, seed=nx, offset=-1.4)
    th = cnn.init_params(nx, out_scale=40.0)
    th[cnn.N_PARAMS - 1] = 0.05
    eng = engine(hq, p, 3, nn.init_params(1), th)
    assert np.array_equal(eng.cnn_get_params(bf16=True).astype(np.float64), bf(th))
    eng.set_fields(X)
    F = eng.cnn_eval()
    act = cnn.CnnAction(p, bf(th))
    for c in range(3):
        ref = act.F(X[c])
        assert abs(F[c] - ref) <= RTOL * max(1.0, abs(ref)), (c, F[c], ref)


def test_cnn_gradient_matches_oracle(hq):
    import torch
    from oracle import cnn, nn
    p = HolsteinParams(nx=4, ny=4, beta=0.6)
    X = random_fields(p, 5, seed=7, offset=-1.4)
    y = np.linspace(-3.0, 2.0, 5)
    th = cnn.init_params(3, out_scale=30.0)
    eng = engine(hq, p, 1, nn.init_params(1), th)
    g, loss = eng.cnn_gradient(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    lref, gref = cnn.loss_and_grad(p, bf(th), X, y)
    assert abs(loss - lref) <= RTOL * lref
    scale = np.max(np.abs(gref))
    assert np.max(np.abs(g - gref)) <= RTOL * scale, np.argmax(np.abs(g - gref))


def test_cnn_training_lowers_the_loss(hq):
    import torch
    from oracle import cnn, nn
    p = HolsteinParams(nx=4, ny=4, beta=0.6)
    X = random_fields(p, 64, seed=11, offset=-1.4)
    target = cnn.CnnAction(p, bf(cnn.init_params(9, out_scale=20.0)))
    y = np.array([target.F(x) for x in X])
    y -= y.mean()
    eng = engine(hq, p, 1, nn.init_params(1), cnn.init_params(1))
    eng.attach_network(16, 64)
    eng.set_params(nn.init_params(1))
    eng.cnn_set_params(cnn.init_params(1))
    losses = eng.cnn_train(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), epochs=30, batch=16, lr=1e-2,
                           seed=5)
    assert losses[-1] < 0.2 * losses[0], losses


@pytest.mark.parametrize("nx,beta", [(4, 1.0), (8, 0.5)])
def test_cumulative_with_cnn_block_moves_matches_oracle(hq, nx, beta):
    from oracle import cnn, nn
    p = HolsteinParams(nx=nx, ny=nx, beta=beta, seed=41)
    C = 3
    X0 = initial_fields(p, C, seed=5)
    th = nn.init_params(4)
    th[-nn.N_H - 1:] *= 2.0
    thc = cnn.init_params(6, out_scale=3.0)
    eng = engine(hq, p, C, th, thc)
    eng.set_fields(X0)
    eng.cumulative(n_steps=2, n_inner=1, cnn=True)
    Xg = eng.get_fields()
    stats = eng.learned_stats()
    _, ld = eng.log_weight()
    for c in range(C):
        ch = nn.CumulativeChain(p, X0[c], bf(th), chain=c, cnn_theta=bf(thc))
        acc = 0
        for k in range(2):
            pc, a = ch.step(k, 1)
            acc += a
        if np.array_equal(Xg[c], ch.X):
            assert stats[c]["cumulative_accepted"] == acc
            assert abs(stats[c]["last_pc"] - pc) <= 1e-3 * max(pc, 1e-12) or (pc > 1 and stats[c]["last_pc"] > 1)
            assert abs(ld[c] - ch.logdet) <= 1e-10 * abs(ch.logdet)
        else:
            # divergence only through a decision the FP32 networks could not resolve
            assert ch.min_margin < 1e-4, ch.min_margin


def test_cnn_block_moves_only_touch_block_counters(hq):
    """Block moves alone (no local moves) with the convolutional action: acceptance counted,
    fields change by whole columns only."""
    from oracle import cnn, nn
    p = HolsteinParams(nx=4, ny=4, beta=1.0, seed=3)
    X0 = initial_fields(p, 4, seed=9)
    eng = engine(hq, p, 4, nn.init_params(2), cnn.init_params(2, out_scale=0.5))
    eng.set_fields(X0)
    eng.cumulative(n_steps=3, n_inner=2, local=False, cnn=True)
    st = eng.learned_stats()
    X = eng.get_fields()
    for c in range(4):
        assert st[c]["inner_local_proposed"] == 0 and st[c]["inner_block_proposed"] == 3 * 2 * p.n_sites
        d = X[c] - X0[c]
        assert np.allclose(d, d[0:1, :], atol=1e-12)  # every slice of a site moved together


@pytest.mark.slow
def test_cnn_sampler_is_exact_for_free_phonons(hq):
    """g = 0: whatever the networks, the cumulative chain with convolutional block moves must
    sample exp(-dtau S_ph): <X^2> against the Gaussian closed form."""
    from oracle import cnn, nn
    from tests import closed_forms as cf
    p = HolsteinParams(nx=4, ny=4, beta=2.0, g=0.0, mu=0.0, seed=15)
    C, steps, burn = 64, 80, 10
    pl = hq.Engine(p, C)
    pl.set_fields(initial_fields(p, C, seed=8))
    pl.sweep(40)
    X = pl.get_fields()
    th = nn.init_params(2)
    th[-nn.N_H - 1:] *= 0.3  # output layer: small network changes keep p_c near 1
    eng = engine(hq, p, C, th, cnn.init_params(5, out_scale=0.05), max_series=steps)
    eng.set_fields(X)
    eng.cumulative(n_steps=steps, n_inner=1, cnn=True)
    s = eng.series(hq.HQ_OBS_X2)[:, burn:]
    per_chain = s.mean(axis=1)
    mean, err = per_chain.mean(), per_chain.std(ddof=1) / math.sqrt(C)
    ref = cf.free_phonon_x2(p.n_slices, p.dtau, p.mass, p.omega)
    st = eng.learned_stats()
    rate = sum(x["cumulative_accepted"] for x in st) / sum(x["cumulative_proposed"] for x in st)
    assert rate > 0.1, rate
    assert abs(mean - ref) < 4 * err, (mean, ref, err, rate)
