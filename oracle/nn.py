"""Learned effective action for network-driven moves (CPU oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/dqmc.py): imported by tests/ and bench.py's CPU legs.

Paper: "Local Updates" (a fully connected network fed the change of the field and the fields
at nearby spacetime points predicts the weight change of a move) and the cumulative update of
the benchmark section: after a number of network-driven sweeps the whole proposal X -> X' is
accepted with min(1, p_c), p_c = [W(X')/W(X)] [exp(-beta E_NN[X]) / exp(-beta E_NN[X'])].

Readings (also in the design notes):
  * p_c needs E_NN to be one scalar function of the configuration, so the network does not
    predict a weight change directly: it defines F(X) = sum_{i,l} f(patch_{i,l}(X)), and the
    learned weight is W_eff(X) = exp(-dtau S_ph(X) + 2 F(X)) -- the phonon action is exact, F
    stands for log|det M(X)| (one spin species; both species give the factor 2).  The change
    of F under any move is exact: only patches that contain a changed field contribute.
  * patch_{i,l}: X at the 5-site cross {i, i+x, i-x, i+y, i-y} on the 5 slices l-2..l+2
    (periodic in space and imaginary time), 25 inputs ordered (slice offset, cross site),
    shifted by the mean field: z = X + g / (M Omega^2).
  * f: 25 -> 64 -> 64 -> 1 with ReLU hidden layers and a linear output; weights are stored in
    bfloat16 (round to nearest even from float32), arithmetic here is FP64.
  * Training fits F(X_a) to log|det M(X_a)| minus its sample mean, by mean squared error.
"""
import math

import numpy as np

from . import dqmc
from .philox import proposal_uniforms

TAG_NN_LOCAL = 2
TAG_NN_BLOCK = 3
TAG_CUMULATIVE = 4

N_IN = 25
N_H = 64
CROSS = ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1))
DT = (-2, -1, 0, 1, 2)

# parameter layout (flat float vector): W1[25][64], b1[64], W2[64][64], b2[64], W3[64], b3
SHAPES = (("W1", (N_IN, N_H)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_H,)), ("b3", ()))
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


def to_bfloat16(x):
    """Round float values to bfloat16 (round to nearest, ties to even) and back to float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64).reshape(np.shape(x))


def init_params(seed):
    """He-style random initialisation (seeded), output layer small."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.standard_normal((N_IN, N_H)) * math.sqrt(2.0 / N_IN), "b1": np.zeros(N_H),
         "W2": rng.standard_normal((N_H, N_H)) * math.sqrt(2.0 / N_H), "b2": np.zeros(N_H),
         "W3": rng.standard_normal(N_H) * 0.01, "b3": 0.0}
    return flatten(p)


def x_shift(p):
    """Mean-field shift of the inputs, z = X - x0 with x0 = -g / (M Omega^2)."""
    return -p.g / (p.mass * p.omega ** 2)


def patch_index(nx, ny, L):
    """Flat indices into X[L][N] of every patch: array [L*N][25], row l*N + i."""
    N = nx * ny
    idx = np.empty((L * N, N_IN), dtype=np.int64)
    for l in range(L):
        for i in range(N):
            x, y = i % nx, i // nx
            k = 0
            for dl in DT:
                ll = (l + dl) % L
                for cx, cy in CROSS:
                    j = (x + cx) % nx + nx * ((y + cy) % ny)
                    idx[l * N + i, k] = ll * N + j
                    k += 1
    return idx


def mlp(theta, Z):
    """f for a batch of inputs Z [B][25]; returns (out [B], cache for backprop)."""
    P = unflatten(theta)
    a1 = Z @ P["W1"] + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"] + P["b2"]
    h2 = np.maximum(a2, 0.0)
    out = h2 @ P["W3"] + P["b3"]
    return out, (Z, a1, h1, a2, h2)


def mlp_backward(theta, cache, dout):
    """Gradient of sum_b dout[b] f(Z_b) with respect to the flat parameters."""
    P = unflatten(theta)
    Z, a1, h1, a2, h2 = cache
    g = {"W3": h2.T @ dout, "b3": float(np.sum(dout))}
    d2 = np.outer(dout, P["W3"]) * (a2 > 0)
    g["W2"] = h1.T @ d2
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ P["W2"].T) * (a1 > 0)
    g["W1"] = Z.T @ d1
    g["b1"] = d1.sum(axis=0)
    return flatten(g)


class EffectiveAction:
    """F(X) = sum of f over all patches, for one lattice shape and parameter vector."""

    def __init__(self, p, theta):
        self.p = p
        self.theta = np.asarray(theta, dtype=np.float64)
        self.idx = patch_index(p.nx, p.ny, p.n_slices)
        self.x0 = x_shift(p)

    def inputs(self, X, rows=None):
        Xf = np.asarray(X, dtype=np.float64).reshape(-1) - self.x0
        ix = self.idx if rows is None else self.idx[rows]
        return Xf[ix]

    def patch_values(self, X):
        return mlp(self.theta, self.inputs(X))[0]

    def F(self, X):
        return float(np.sum(self.patch_values(X)))

    def rows_touching(self, sites_slices):
        """Patch rows whose 25 inputs include any of the given (slice, site) points."""
        pts = {l * self.p.n_sites + i for l, i in sites_slices}
        return np.array([r for r in range(self.idx.shape[0]) if pts.intersection(self.idx[r])], dtype=np.int64)

    def delta_local(self, X, l, i, x_new):
        """F(X') - F(X) for X'(i, l) = x_new, from the 25 patches that contain (i, l)."""
        rows = self._local_rows(l, i)
        Xn = np.array(X, dtype=np.float64, copy=True)
        Xn[l, i] = x_new
        return float(np.sum(mlp(self.theta, self.inputs(Xn, rows))[0] - mlp(self.theta, self.inputs(X, rows))[0]))

    def delta_block(self, X, i, dx):
        """F(X') - F(X) for X'(i, .) = X(i, .) + dx, from the 5 L patches that contain site i."""
        rows = self._block_rows(i)
        Xn = np.array(X, dtype=np.float64, copy=True)
        Xn[:, i] += dx
        return float(np.sum(mlp(self.theta, self.inputs(Xn, rows))[0] - mlp(self.theta, self.inputs(X, rows))[0]))

    def _local_rows(self, l, i):
        p = self.p
        x, y = i % p.nx, i // p.nx
        rows = []
        for dl in DT:
            ll = (l - dl) % p.n_slices
            for cx, cy in CROSS:
                j = (x - cx) % p.nx + p.nx * ((y - cy) % p.ny)
                rows.append(ll * p.n_sites + j)
        return np.array(sorted(set(rows)), dtype=np.int64)

    def _block_rows(self, i):
        p = self.p
        x, y = i % p.nx, i // p.nx
        centers = sorted({(x - cx) % p.nx + p.nx * ((y - cy) % p.ny) for cx, cy in CROSS})
        return np.array([l * p.n_sites + j for l in range(p.n_slices) for j in centers], dtype=np.int64)


def loss_and_grad(p, theta, Xs, ys):
    """Mean squared error (1/B) sum_a (F(X_a) - y_a)^2 and its gradient."""
    act = EffectiveAction(p, theta)
    B = len(Xs)
    loss = 0.0
    grad = np.zeros(N_PARAMS)
    for X, y in zip(Xs, ys):
        Z = act.inputs(X)
        out, cache = mlp(theta, Z)
        r = float(np.sum(out)) - y
        loss += r * r / B
        grad += mlp_backward(theta, cache, np.full(out.shape, 2.0 * r / B))
    return loss, grad


class CumulativeChain:
    """The network-driven sampler with the exact cumulative accept (paper, NNMC section).

    Inner moves are Metropolis moves, each on its own learned weight: local moves on
    exp(-dtau S_ph + 2F) (patch network F), block moves on exp(-dtau S_ph + 2F_b) with F_b the
    convolutional action when `cnn_theta` is given, else F as well.  After n_inner inner
    sweeps the proposal X -> X' is accepted with min(1, p_c).

    Reading of p_c: reversing the realised sequence of moves has probability ratio
    prod over accepted moves of pi_j(before) / pi_j(after) (detailed balance of each move), so
    p_c = [W(X')/W(X)] prod_j pi_j(before)/pi_j(after) = exp(2 dlog|det M| - 2 sum_acc dF_j):
    the phonon action cancels and the accepted network changes enter as a path sum (for a
    single network the sum is F(X') - F(X)).  The smallest relative distance |u - p| / p of
    any decision is kept in min_margin (for parity checks).
    """

    def __init__(self, p, X, theta, chain=0, cnn_theta=None, record=False):
        self.p = p
        self.record = record
        self.moves = []   # with record: every inner move of the last step (state before, proposal, u, decision)
        self.X = np.array(X, dtype=np.float64, copy=True)
        self.chain = int(chain)
        self.act = EffectiveAction(p, theta)
        self.cnn = None
        if cnn_theta is not None:
            from .cnn import CnnAction
            self.cnn = CnnAction(p, cnn_theta)
        self.expK, _ = dqmc.kinetic_propagators(p)
        self.logdet = dqmc.log_det_M(p, self.expK, self.X)
        self.min_margin = math.inf
        self.dF_path = 0.0

    def _decide(self, u, prob):
        self.min_margin = min(self.min_margin, abs(u - prob) / max(prob, 1e-300))
        return bool(u < prob)

    def _log(self, kind, X, where, value, u, dF, accepted):
        if self.record:
            self.moves.append(dict(kind=kind, before=X.copy(), where=where, value=value, u=float(u), dF=dF,
                                   accepted=accepted))

    def step(self, k, n_inner, local=True, block=True, window=0, site_window=0):
        """One cumulative step.  The inner moves run forward (local moves l, i ascending, then
        block moves i ascending) or as the exact reverse of that sequence, each with
        probability 1/2 (second uniform of the step's tag-4 Philox block): a fixed order of
        reversible moves is not reversible, and p_c relies on a reversible proposal.

        window > 0 (and < L): the local moves visit only `window` consecutive slices starting at
        l0 = floor(u L), u the first uniform of event 1 of the step's tag-4 block (chosen
        independently of the fields, so each window's sequence is reversible on its own).
        site_window > 0 (and < N): the block moves visit only `site_window` consecutive sites
        (index order, periodic) from j0 = floor(v N), v the second uniform of that block."""
        p, X = self.p, self.X
        L, N = X.shape
        W = window if 0 < window < L else L
        Wb = site_window if 0 < site_window < N else N
        l0 = j0 = 0
        if W < L or Wb < N:
            wu, wv = proposal_uniforms(p.seed, self.chain, k, [1], TAG_CUMULATIVE)
            if W < L:
                l0 = min(int(float(wu[0]) * L), L - 1)
            if Wb < N:
                j0 = min(int(float(wv[0]) * N), N - 1)
        slices = [(l0 + j) % L for j in range(W)]
        sites = [(j0 + j) % N for j in range(Wb)]
        X0 = X.copy()
        ld0 = self.logdet
        path = 0.0
        self.moves = []
        uc, ud = proposal_uniforms(p.seed, self.chain, k, [0], TAG_CUMULATIVE)
        fwd = bool(ud[0] < 0.5)
        self.last_forward = fwd
        order = (lambda m: range(m)) if fwd else (lambda m: range(m - 1, -1, -1))
        for u in range(n_inner):
            isw = k * n_inner + u
            parts = ("local", "block") if fwd else ("block", "local")
            for part in parts:
                if part == "local" and local:
                    for j in order(W):
                        s = slices[j]
                        u1, u2 = proposal_uniforms(p.seed, self.chain, isw, s * N + np.arange(N), TAG_NN_LOCAL)
                        for i in order(N):
                            xn = X[s, i] + p.dx_local * (2.0 * u1[i] - 1.0)
                            dS = dqmc.local_action_change(p, X, s, i, xn)
                            dF = self.act.delta_local(X, s, i, xn)
                            ok = self._decide(u2[i], math.exp(min(2.0 * dF - dS, 709.0)))
                            self._log("local", X, (s, i), xn, u2[i], dF, ok)
                            if ok:
                                X[s, i] = xn
                                path += dF
                if part == "block" and block:
                    u1, u2 = proposal_uniforms(p.seed, self.chain, isw, np.arange(N), TAG_NN_BLOCK)
                    for jb in order(Wb):
                        i = sites[jb]
                        dx = p.dx_global * (2.0 * u1[i] - 1.0)
                        dS = dqmc.global_action_change(p, X, i, dx)
                        dF = self.cnn.delta_block(X, i, dx) if self.cnn is not None else self.act.delta_block(X, i, dx)
                        ok = self._decide(u2[i], math.exp(min(2.0 * dF - dS, 709.0)))
                        self._log("block", X, i, dx, u2[i], dF, ok)
                        if ok:
                            X[:, i] += dx
                            path += dF
        ld1 = dqmc.log_det_M(p, self.expK, X)
        self.dF_path = path
        pc = math.exp(min(2.0 * (ld1 - ld0) - 2.0 * path, 709.0))
        accepted = self._decide(float(uc[0]), pc)
        if accepted:
            self.logdet = ld1
        else:
            X[:] = X0
            self.logdet = ld0
        return pc, accepted
