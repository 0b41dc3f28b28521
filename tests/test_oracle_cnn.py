"""Pins of the convolutional effective action (oracle/cnn.py): the first layer against
scipy's periodic correlation, backpropagation against central finite differences, translation
invariance on the (x, y, tau) torus, a linear closed form, and the path-sum form of the
cumulative accept for a single network."""
import math

import numpy as np
import pytest

from oracle import cnn, nn
from workloads import HolsteinParams, random_fields


def test_first_layer_matches_scipy_periodic_correlation():
    ndimage = pytest.importorskip("scipy.ndimage")
    p = HolsteinParams(nx=4, ny=6, beta=0.5)
    rng = np.random.default_rng(0)
    theta = cnn.init_params(1)
    P = cnn.unflatten(theta)
    z = cnn.field(p, random_fields(p, 1, seed=1)[0])
    a1 = cnn.conv(z, P["W1"][:, None, :], P["b1"])
    for co in rng.choice(cnn.C_H, 4, replace=False):
        kern = np.zeros((3, 3, 3))
        for t, (dl, dy, dx) in enumerate(cnn.TAPS):
            kern[dl + 1, dy + 1, dx + 1] = P["W1"][t, co]
        ref = ndimage.correlate(z[0], kern, mode="wrap") + P["b1"][co]
        assert np.max(np.abs(a1[co] - ref)) < 1e-12


def test_backprop_matches_finite_differences():
    p = HolsteinParams(nx=4, ny=4, beta=0.5)
    Xs = random_fields(p, 2, seed=3, offset=-1.4)
    ys = np.array([1.5, -0.5])
    theta = cnn.init_params(2, out_scale=30.0)
    theta[cnn.N_PARAMS - 1] = 0.2
    loss, g = cnn.loss_and_grad(p, theta, Xs, ys)
    rng = np.random.default_rng(5)
    for k in np.concatenate([rng.choice(cnn.N_PARAMS, 40, replace=False), [0, cnn.N_PARAMS - 1]]):
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (cnn.loss_and_grad(p, tp, Xs, ys)[0] - cnn.loss_and_grad(p, tm, Xs, ys)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(fd)), (k, fd, g[k])


def test_translation_invariance_on_the_torus():
    p = HolsteinParams(nx=4, ny=6, beta=0.8)
    act = cnn.CnnAction(p, cnn.init_params(4, out_scale=50.0))
    X = random_fields(p, 1, seed=4)[0]
    F = act.F(X)
    assert abs(act.F(np.roll(X, 3, axis=0)) - F) < 1e-10 * abs(F)
    Xs = X.reshape(p.n_slices, p.ny, p.nx)
    assert abs(act.F(np.roll(Xs, 1, axis=2).reshape(X.shape)) - F) < 1e-10 * abs(F)
    assert abs(act.F(np.roll(Xs, -2, axis=1).reshape(X.shape)) - F) < 1e-10 * abs(F)


def test_linear_closed_form():
    """Non-negative weights, zero biases and non-negative inputs make every layer linear; the
    sum over a torus of a correlation is (sum of the kernel) x (sum of the input), so
    F = sum_c2 w3[c2] sum_c1 w2[c1][c2] w1[c1] sum z with w = kernel sums over taps."""
    p = HolsteinParams(nx=4, ny=4, beta=0.6)
    rng = np.random.default_rng(3)
    prm = {"W1": rng.random((27, cnn.C_H)), "b1": np.zeros(cnn.C_H), "W2": rng.random((27, cnn.C_H, cnn.C_H)) * 0.1,
           "b2": np.zeros(cnn.C_H), "W3": rng.random((27, cnn.C_H)), "b3": 0.0}
    act = cnn.CnnAction(p, cnn.flatten(prm))
    X = nn.x_shift(p) + np.abs(random_fields(p, 1, seed=3)[0])
    w1, w2, w3 = prm["W1"].sum(axis=0), prm["W2"].sum(axis=0), prm["W3"].sum(axis=0)
    ref = w3 @ (w2.T @ w1) * np.sum(X - nn.x_shift(p))
    assert abs(act.F(X) - ref) < 1e-10 * abs(ref)


def test_single_network_path_sum_equals_endpoint_difference():
    """With one network for both move kinds the accepted changes telescope: the path sum used
    in p_c equals F(X') - F(X)."""
    p = HolsteinParams(nx=4, ny=4, beta=0.5, seed=9)
    th = nn.init_params(2)
    th[-nn.N_H - 1:] *= 40.0
    X0 = random_fields(p, 1, seed=2, offset=-1.4)[0]
    ch = nn.CumulativeChain(p, X0, th, chain=1)
    act = nn.EffectiveAction(p, th)
    for k in range(2):
        Xb = ch.X.copy()
        pc, acc = ch.step(k, 1)
        ref = act.F(ch.X if acc else Xb) - act.F(Xb) if acc else None
        if acc:
            assert abs(ch.dF_path - ref) < 1e-9 * max(1.0, abs(ref))
        # the proposal's endpoint difference (accepted or not) is what p_c used
        assert math.isfinite(pc)
