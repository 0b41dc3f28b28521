"""Periodic 3D convolutional effective action for block moves (CPU oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/dqmc.py): imported by tests/ and bench.py's CPU legs.

Paper: "Global Updates" -- a convolutional network on the whole phonon field predicts the
weight of a configuration, which makes the change under a move of a whole imaginary-time
column cheap to estimate -- and the cumulative update of the benchmark section.

Readings (also in the design notes):
  * The network acts on the (x, y, tau) torus: input z = X + g/(M Omega^2) (mean-field
    shift), three 3x3x3 convolutions with periodic padding, 1 -> 16 -> 16 -> 1 channels, ReLU
    after the first two, and F_cnn(X) = the sum of the last layer over every point.  As for
    the patch network, W_eff = exp(-dtau S_ph + 2 F_cnn): F_cnn stands for log|det M|.
  * Tap t = 9 (dl + 1) + 3 (dy + 1) + (dx + 1) reads the input at (l + dl, y + dy, x + dx)
    (cross-correlation, as in the usual convolution layers).
  * Parameters, one flat vector: W1[27][16] (tap, out), b1[16], W2[27][16][16] (tap, in,
    out), b2[16], W3[27][16] (tap, in), b3; weights stored in bfloat16 like the patch network.
  * A block move shifts X(i, .) at every slice; its change of F_cnn is F_cnn(X') - F_cnn(X),
    written here from scratch.
"""
import numpy as np

from .nn import x_shift

C_H = 16
TAPS = tuple((dl, dy, dx) for dl in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1))
SHAPES = (("W1", (27, C_H)), ("b1", (C_H,)), ("W2", (27, C_H, C_H)), ("b2", (C_H,)), ("W3", (27, C_H)), ("b3", ()))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape) if shape else theta[o]
        o += k
    return out


def flatten(params):
    return np.concatenate([np.atleast_1d(np.asarray(params[name], dtype=np.float64)).ravel() for name, _ in SHAPES])


def init_params(seed, out_scale=1.0):
    """He-style random initialisation (seeded); the last layer is scaled by 0.01 * out_scale."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.standard_normal((27, C_H)) * np.sqrt(2.0 / 27), "b1": np.zeros(C_H),
         "W2": rng.standard_normal((27, C_H, C_H)) * np.sqrt(2.0 / (27 * C_H)), "b2": np.zeros(C_H),
         "W3": rng.standard_normal((27, C_H)) * 0.01 * out_scale, "b3": 0.0}
    return flatten(p)


def shifted(a, dl, dy, dx):
    """b[..., l, y, x] = a[..., l + dl, y + dy, x + dx] (periodic in the last three axes)."""
    return np.roll(a, shift=(-dl, -dy, -dx), axis=(-3, -2, -1))


def conv(inp, W, b):
    """Periodic 3x3x3 cross-correlation: inp [Cin][L][ny][nx], W [27][Cin][Cout], b [Cout]."""
    out = np.zeros((W.shape[2],) + inp.shape[1:]) + np.asarray(b).reshape(-1, 1, 1, 1)
    for t, (dl, dy, dx) in enumerate(TAPS):
        out += np.einsum("c...,co->o...", shifted(inp, dl, dy, dx), W[t])
    return out


def conv_backward(inp, W, dout):
    """Gradients of sum(dout * conv(inp, W, b)): (d inp, d W, d b)."""
    dW = np.zeros_like(W)
    dinp = np.zeros_like(inp)
    for t, (dl, dy, dx) in enumerate(TAPS):
        dW[t] = shifted(inp, dl, dy, dx).reshape(inp.shape[0], -1) @ dout.reshape(dout.shape[0], -1).T
        # inp at q feeds output q - tap through W[t]
        dinp += shifted(np.einsum("co,o...->c...", W[t], dout), -dl, -dy, -dx)
    return dinp, dW, dout.sum(axis=(1, 2, 3))


def field(p, X):
    """z = X - x0 as a 1-channel [1][L][ny][nx] array (site i = x + nx y)."""
    return (np.asarray(X, dtype=np.float64) - x_shift(p)).reshape(1, p.n_slices, p.ny, p.nx)


def forward(theta, z):
    """Layer outputs for input z [1][L][ny][nx]: (out3 [1][L][ny][nx], cache)."""
    P = unflatten(theta)
    a1 = conv(z, P["W1"][:, None, :], P["b1"])
    h1 = np.maximum(a1, 0.0)
    a2 = conv(h1, P["W2"], P["b2"])
    h2 = np.maximum(a2, 0.0)
    out = conv(h2, P["W3"][:, :, None], np.array([P["b3"]]))
    return out, (z, a1, h1, a2, h2)


def backward(theta, cache, dF):
    """Gradient of dF * F_cnn with respect to the flat parameters."""
    P = unflatten(theta)
    z, a1, h1, a2, h2 = cache
    dout = np.full((1,) + z.shape[1:], float(dF))
    dh2, dW3, db3 = conv_backward(h2, P["W3"][:, :, None], dout)
    da2 = dh2 * (a2 > 0)
    dh1, dW2, db2 = conv_backward(h1, P["W2"], da2)
    da1 = dh1 * (a1 > 0)
    _, dW1, db1 = conv_backward(z, P["W1"][:, None, :], da1)
    return flatten({"W1": dW1[:, 0, :], "b1": db1, "W2": dW2, "b2": db2, "W3": dW3[:, :, 0], "b3": db3[0]})


class CnnAction:
    """F_cnn(X) for one lattice shape and parameter vector."""

    def __init__(self, p, theta):
        self.p = p
        self.theta = np.asarray(theta, dtype=np.float64)

    def F(self, X):
        return float(np.sum(forward(self.theta, field(self.p, X))[0]))

    def delta_block(self, X, i, dx):
        """F_cnn(X') - F_cnn(X) for X'(i, .) = X(i, .) + dx."""
        Xn = np.array(X, dtype=np.float64, copy=True)
        Xn[:, i] += dx
        return self.F(Xn) - self.F(X)


def loss_and_grad(p, theta, Xs, ys):
    """Mean squared error (1/B) sum_a (F_cnn(X_a) - y_a)^2 and its gradient."""
    B = len(Xs)
    loss = 0.0
    grad = np.zeros(N_PARAMS)
    for X, y in zip(Xs, ys):
        out, cache = forward(theta, field(p, X))
        r = float(np.sum(out)) - y
        loss += r * r / B
        grad += backward(theta, cache, 2.0 * r / B)
    return loss, grad
