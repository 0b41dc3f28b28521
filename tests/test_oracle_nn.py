"""Pins of the effective-action oracle (oracle/nn.py): bfloat16 rounding against torch,
backpropagation against central finite differences, incremental move deltas against
from-scratch differences, symmetry of the patch sum, and a linear closed form."""
import numpy as np
import pytest

from oracle import nn
from workloads import HolsteinParams, random_fields


def test_bfloat16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 0.0, 65504.0]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(nn.to_bfloat16(x), ref)


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = nn.init_params(3)
    theta[-1] = 0.3
    Z = rng.standard_normal((7, nn.N_IN))
    dout = rng.standard_normal(7)
    out, cache = nn.mlp(theta, Z)
    g = nn.mlp_backward(theta, cache, dout)
    for k in rng.choice(nn.N_PARAMS, 60, replace=False):
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (dout @ nn.mlp(tp, Z)[0] - dout @ nn.mlp(tm, Z)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), k


def test_loss_gradient_matches_finite_differences():
    p = HolsteinParams(nx=4, ny=4, beta=0.5)
    Xs = random_fields(p, 3, seed=2, offset=-1.4)
    ys = np.array([3.0, -1.0, 0.5])
    theta = nn.init_params(5)
    loss, g = nn.loss_and_grad(p, theta, Xs, ys)
    rng = np.random.default_rng(4)
    for k in rng.choice(nn.N_PARAMS, 20, replace=False):
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (nn.loss_and_grad(p, tp, Xs, ys)[0] - nn.loss_and_grad(p, tm, Xs, ys)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(fd)), k


@pytest.mark.parametrize("nx,beta", [(2, 0.3), (4, 0.8), (6, 1.0)])
def test_move_deltas_against_from_scratch(nx, beta):
    p = HolsteinParams(nx=nx, ny=nx, beta=beta)
    act = nn.EffectiveAction(p, nn.init_params(nx))
    X = random_fields(p, 1, seed=nx, offset=-1.4)[0]
    L, N = X.shape
    for l, i, xn in ((0, 0, 0.3), (L - 1, N - 1, -2.0), (L // 2, N // 3, 1.1)):
        Xn = X.copy()
        Xn[l, i] = xn
        assert abs(act.delta_local(X, l, i, xn) - (act.F(Xn) - act.F(X))) < 1e-10
    for i, dx in ((0, 0.7), (N - 1, -0.4)):
        Xn = X.copy()
        Xn[:, i] += dx
        assert abs(act.delta_block(X, i, dx) - (act.F(Xn) - act.F(X))) < 1e-10


def test_patch_sum_is_translation_invariant():
    p = HolsteinParams(nx=4, ny=4, beta=0.8)
    act = nn.EffectiveAction(p, nn.init_params(9))
    X = random_fields(p, 1, seed=9)[0]
    F = act.F(X)
    assert abs(act.F(np.roll(X, 3, axis=0)) - F) < 1e-10 * abs(F)
    Xs = X.reshape(p.n_slices, p.ny, p.nx)
    assert abs(act.F(np.roll(Xs, 1, axis=2).reshape(X.shape)) - F) < 1e-10 * abs(F)
    assert abs(act.F(np.roll(Xs, -1, axis=1).reshape(X.shape)) - F) < 1e-10 * abs(F)


def test_linear_closed_form():
    """Equal non-negative first-layer columns, W2 = I, zero biases and non-negative inputs
    make f linear: F = sum(W3) * sum(w) * sum over all points of z."""
    p = HolsteinParams(nx=4, ny=4, beta=0.6)
    rng = np.random.default_rng(3)
    w = rng.random(nn.N_IN)
    prm = {"W1": np.repeat(w[:, None], nn.N_H, axis=1), "b1": np.zeros(nn.N_H), "W2": np.eye(nn.N_H),
           "b2": np.zeros(nn.N_H), "W3": rng.standard_normal(nn.N_H), "b3": 0.0}
    act = nn.EffectiveAction(p, nn.flatten(prm))
    X = act.x0 + np.abs(random_fields(p, 1, seed=3)[0])
    ref = prm["W3"].sum() * w.sum() * np.sum(X - act.x0)
    assert abs(act.F(X) - ref) < 1e-10 * abs(ref)


def test_full_windows_equal_the_full_sweep():
    """A slice window of L and a site window of N are the full inner sweep: same fields, same
    p_c, same decisions; a smaller window only moves points inside it."""
    p = HolsteinParams(nx=4, ny=4, beta=0.6, seed=19)
    th = nn.init_params(3)
    th[-nn.N_H - 1:] *= 10.0
    X0 = random_fields(p, 1, seed=5, offset=-1.4)[0]
    a = nn.CumulativeChain(p, X0, th, chain=2)
    b = nn.CumulativeChain(p, X0, th, chain=2)
    for k in range(2):
        ra = a.step(k, 1)
        rb = b.step(k, 1, window=p.n_slices, site_window=p.n_sites)
        assert ra == rb
        assert np.array_equal(a.X, b.X)
    c = nn.CumulativeChain(p, X0, th, chain=2)
    c.step(0, 1, local=True, block=False, window=2)
    moved = np.any(c.X != X0, axis=1)
    assert moved.sum() <= 2   # only the two slices of the window can change
