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


# ------------------------------------------------------------- cumulative accept pins

def _path_log_ratio(ch, X_start, log_pi):
    """Replays the recorded inner moves of the last step and returns (X', log of the reverse
    path's probability over the forward path's).  Each move is a Metropolis move with a
    symmetric proposal on its own weight pi_j (log_pi(kind, X)); a rejected move contributes
    the same rejection factor to both paths, an accepted move a -> b contributes
    min(1, pi(a)/pi(b)) / min(1, pi(b)/pi(a)).  Also checks every recorded decision against
    u < min(1, pi(b)/pi(a)) computed from the full weights."""
    X = X_start.copy()
    lr = 0.0
    for m in ch.moves:
        assert np.array_equal(m["before"], X)
        b = X.copy()
        if m["kind"] == "local":
            b[m["where"]] = m["value"]
        else:
            b[:, m["where"]] += m["value"]
        d = log_pi(m["kind"], b) - log_pi(m["kind"], X)
        fwd, rev = min(1.0, np.exp(d)), min(1.0, np.exp(-d))
        if abs(m["u"] - fwd) > 1e-9 * max(fwd, 1e-300):
            assert (m["u"] < fwd) == m["accepted"], (m["kind"], m["u"], fwd)
        if m["accepted"]:
            lr += np.log(rev) - np.log(fwd)
            X = b
    return X, lr


@pytest.mark.parametrize("with_cnn", [False, True])
def test_cumulative_accept_equals_the_explicit_path_probability_ratio(with_cnn):
    """Paper, cumulative update: p_c = [W(X')/W(X)] [P(X' -> X) / P(X -> X')] for the
    proposal made of network-driven moves.  On a 2x2, L = 4 lattice, for each recorded step
    (forward and reverse visiting orders) the oracle's p_c must equal W(X')/W(X) from fresh
    determinants and the phonon action, times the ratio of the reverse path's to the forward
    path's acceptance probabilities, each computed from the full learned weights
    exp(-dtau S_ph + 2 F) (not the incremental changes the sampler uses), to 1e-12 in log."""
    import math
    from oracle import cnn, dqmc
    p = HolsteinParams(nx=2, ny=2, beta=0.4, seed=123)
    th = nn.init_params(8)
    th[-nn.N_H - 1:] *= 30.0
    th = nn.to_bfloat16(th.astype(np.float32))
    act = nn.EffectiveAction(p, th)
    cth = cnn_act = None
    if with_cnn:
        cth = nn.to_bfloat16(cnn.init_params(3, out_scale=30.0).astype(np.float32))
        cnn_act = cnn.CnnAction(p, cth)
    expK, _ = dqmc.kinetic_propagators(p)

    def log_pi(kind, X):
        F = cnn_act.F(X) if (kind == "block" and cnn_act is not None) else act.F(X)
        return -dqmc.phonon_action(p, X) + 2.0 * F

    def log_w(X):
        return 2.0 * dqmc.log_det_M(p, expK, X) - dqmc.phonon_action(p, X)

    X0 = random_fields(p, 1, seed=4, offset=-1.4)[0]
    ch = nn.CumulativeChain(p, X0, th, chain=3, cnn_theta=cth, record=True)
    dirs = set()
    n_acc_moves = 0
    for k in range(8):
        Xs = ch.X.copy()
        pc, accepted = ch.step(k, 1)
        dirs.add(ch.last_forward)
        Xp, lr = _path_log_ratio(ch, Xs, log_pi)
        n_acc_moves += sum(m["accepted"] for m in ch.moves)
        expected = log_w(Xp) - log_w(Xs) + lr
        assert abs(math.log(pc) - expected) < 1e-12 * max(1.0, abs(expected)), (k, math.log(pc), expected)
        assert np.array_equal(ch.X, Xp if accepted else Xs)
    assert dirs == {True, False}
    assert n_acc_moves > 20


def _free_phonon_sampler(p, L, N):
    """Exact samples of X at g = 0: each site's time column is Gaussian with the circulant
    precision of dtau S_ph."""
    A = np.zeros((L, L))
    for l in range(L):
        A[l, l] = 2.0 * p.mass / p.dtau + p.dtau * p.mass * p.omega ** 2
        A[l, (l + 1) % L] -= p.mass / p.dtau
        A[l, (l - 1) % L] -= p.mass / p.dtau
    chol = np.linalg.cholesky(np.linalg.inv(A))
    return lambda rng, n: np.einsum("ab,nbi->nai", chol, rng.standard_normal((n, L, N)))


def test_cumulative_sampler_reproduces_the_free_phonon_closed_form():
    """g = 0: log|det M| does not depend on X, so the cumulative sampler with any network must
    sample exp(-dtau S_ph), whose <X^2> is the closed form (1/L) sum_q 1/[(2M/dtau)(1 - cos
    2 pi q/L) + dtau M Omega^2].  The network chosen here biases the inner moves strongly: the
    inner chain alone would sample exp(-dtau S_ph + 2F), whose <X^2> (importance-reweighted
    exact samples) lies many error bars away, so only a correct cumulative accept passes."""
    import math
    from oracle import autocorr
    from tests import closed_forms as cf
    p = HolsteinParams(nx=2, ny=2, beta=0.8, g=0.0, mu=0.0, seed=5)
    L, N = p.n_slices, p.n_sites
    ref = cf.free_phonon_x2(L, p.dtau, p.mass, p.omega)
    th = nn.to_bfloat16(nn.init_params(2).astype(np.float32))
    draw = _free_phonon_sampler(p, L, N)
    series, acc, steps = [], 0, 450
    for c in range(4):
        ch = nn.CumulativeChain(p, draw(np.random.default_rng(100 + c), 1)[0], th, chain=c)
        s = []
        for k in range(steps):
            acc += ch.step(k, 1)[1]
            s.append(float(np.mean(ch.X ** 2)))
        series.append(np.array(s))
    tau = float(np.mean([autocorr.tau_int(x)[0] for x in series]))
    allx = np.concatenate(series)
    err = float(np.std(allx)) / math.sqrt(allx.size / (2.0 * tau))
    assert 0.3 < acc / (4 * steps) < 0.9
    assert abs(allx.mean() - ref) < 3.0 * err, (allx.mean(), ref, err, tau)
    # the inner chain's own distribution is far from the closed form
    act = nn.EffectiveAction(p, th)
    S = draw(np.random.default_rng(0), 20000)
    F = np.array([act.F(x) for x in S])
    w = np.exp(2.0 * (F - F.max()))
    biased = float(np.sum(w * np.mean(S ** 2, axis=(1, 2))) / np.sum(w))
    assert abs(biased - ref) > 10.0 * err, (biased, ref, err)
