"""Pins of the CPU oracle against closed forms, brute force and invariants.

None of these retypes the oracle's formulas: each compares it with something the
model or mathematics fixes independently (plane-wave closed forms, Fock-space traces,
plain unstabilised determinants, mpmath, symmetry, detailed balance, a Gaussian
closed form for the free phonons, published Philox known answers).
"""
import math
import os

import numpy as np
import pytest

from oracle import dqmc, philox, autocorr
from workloads import HolsteinParams, initial_fields, random_fields, uniform_fields
from tests import closed_forms as cf
from tests import fock

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small(nx=4, beta=1.0, **kw):
    return HolsteinParams(nx=nx, ny=nx, beta=beta, **kw)


# ------------------------------------------------------------------------ Philox

def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    for r in rows:
        out = philox.philox4x32_10(np.array(r[:4]), (r[4], r[5]))
        assert [int(w) for w in out] == r[6:]


def test_philox_uniform_grid_and_moments():
    u1, u2 = philox.proposal_uniforms(12345, 3, 7, np.arange(200000), philox.TAG_LOCAL)
    for u in (u1, u2):
        assert np.all(u >= 0.0) and np.all(u < 1.0)
        assert np.all(np.floor(u * 2.0 ** 53) == u * 2.0 ** 53)
        assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
        assert abs((u * u).mean() - 1 / 3) < 5 * math.sqrt(4 / 45 / u.size)
    assert abs(np.corrcoef(u1, u2)[0, 1]) < 0.02
    # distinct streams for a different tag / chain / sweep
    v1, _ = philox.proposal_uniforms(12345, 3, 7, np.arange(1000), philox.TAG_GLOBAL)
    w1, _ = philox.proposal_uniforms(12345, 4, 7, np.arange(1000), philox.TAG_LOCAL)
    assert not np.array_equal(v1, u1[:1000]) and not np.array_equal(w1, u1[:1000])


# ------------------------------------------------------------------ free fermions

@pytest.mark.parametrize("nx,beta,l", [(2, 2.0, 0), (4, 4.0, 13), (8, 8.0, 80), (8, 16.0, 37)])
def test_free_fermion_green_and_logdet(nx, beta, l):
    p = small(nx, beta, g=0.0, mu=-0.7)
    expK, _ = dqmc.kinetic_propagators(p)
    X = random_fields(p, 1, seed=nx)[0]       # irrelevant at g = 0
    G, ld = dqmc.green_at(p, expK, X, l)
    ref_ld = cf.free_logdet(nx, nx, p.t, p.mu, beta)
    assert abs(ld - ref_ld) <= 1e-11 * max(1.0, abs(ref_ld))
    assert np.max(np.abs(G - cf.free_green(nx, nx, p.t, p.mu, beta))) < 1e-11


def test_free_fermion_largest_lattice():
    p = HolsteinParams(nx=16, ny=16, beta=16.0, g=0.0, mu=-2.0)
    expK, _ = dqmc.kinetic_propagators(p)
    X = np.zeros((p.n_slices, p.n_sites))
    G, ld = dqmc.green_at(p, expK, X, 0)
    ref = cf.free_logdet(16, 16, p.t, p.mu, p.beta)
    assert abs(ld - ref) <= 1e-11 * abs(ref)
    assert np.max(np.abs(G - cf.free_green(16, 16, p.t, p.mu, p.beta))) < 1e-10


@pytest.mark.parametrize("nx,beta,x0", [(4, 4.0, -1.3), (8, 16.0, 0.4), (16, 16.0, -0.9)])
def test_uniform_field_logdet(nx, beta, x0):
    p = small(nx, beta)
    expK, _ = dqmc.kinetic_propagators(p)
    X = uniform_fields(p, 1, x0)[0]
    G, ld = dqmc.green_at(p, expK, X, 0)
    ref = cf.free_logdet(nx, nx, p.t, p.mu, beta, shift=p.g * x0)
    assert abs(ld - ref) <= 1e-11 * max(1.0, abs(ref))
    assert np.max(np.abs(G - cf.free_green(nx, nx, p.t, p.mu, beta, shift=p.g * x0))) < 1e-10


def test_atomic_limit():
    p = small(4, 3.0, t=0.0)
    expK, _ = dqmc.kinetic_propagators(p)
    X = random_fields(p, 1, seed=5, scale=2.0)[0]
    a = p.dtau * np.sum(p.g * X - p.mu, axis=0)         # dtau sum_l V_il
    for l in (0, 7, 29):
        G, ld = dqmc.green_at(p, expK, X, l)
        assert np.max(np.abs(G - np.diag(1.0 / (1.0 + np.exp(-a))))) < 1e-13
        assert abs(ld - np.sum(np.log1p(np.exp(-a)))) < 1e-11 * abs(ld)


# -------------------------------------------------------------- particle-hole symmetry

@pytest.mark.parametrize("nx,beta,seed", [(2, 2.0, 1), (4, 4.0, 2), (6, 3.0, 3), (8, 8.0, 4)])
def test_particle_hole_symmetry(nx, beta, seed):
    """At mu = -g^2/(M Omega^2): log W(c - X) = log W(X) with c = -2g/(M Omega^2)."""
    p = small(nx, beta)
    expK, _ = dqmc.kinetic_propagators(p)
    X = random_fields(p, 1, seed=seed, scale=1.0, offset=-1.0)[0]
    c = -2.0 * p.g / (p.mass * p.omega ** 2)
    lw, lw2 = dqmc.log_weight(p, expK, X), dqmc.log_weight(p, expK, c - X)
    assert abs(lw - lw2) <= 1e-11 * abs(lw)
    ld, ld2 = dqmc.log_det_M(p, expK, X), dqmc.log_det_M(p, expK, c - X)
    shift = p.dtau * np.sum(p.g * X - p.mu)
    assert abs(ld2 - (ld + shift)) <= 1e-11 * max(abs(ld), abs(shift))


# -------------------------------------------------------------------- brute force

def _plain_product(p, expK, X, l):
    L = X.shape[0]
    P = np.eye(p.n_sites)
    for s in dqmc.slice_order(L, l):
        P = dqmc.slice_matrix(p, expK, X[s]) @ P
    return P


@pytest.mark.parametrize("nx,beta,l", [(2, 1.0, 0), (2, 1.0, 4), (4, 1.0, 0), (4, 1.0, 7)])
def test_brute_force_small_beta(nx, beta, l):
    p = small(nx, beta, n_wrap=3)
    expK, _ = dqmc.kinetic_propagators(p)
    X = random_fields(p, 1, seed=11 + nx)[0]
    P = _plain_product(p, expK, X, l)
    G, ld = dqmc.green_at(p, expK, X, l)
    assert abs(ld - np.linalg.slogdet(np.eye(p.n_sites) + P)[1]) < 1e-12 * max(1, abs(ld))
    assert np.max(np.abs(G - np.linalg.inv(np.eye(p.n_sites) + P))) < 1e-12


def test_mpmath_determinant():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    p = small(2, 1.0)
    K = dqmc.hopping_matrix(p)
    X = random_fields(p, 1, seed=3)[0]
    # exp(-dtau K) by its Taylor series in 50-digit arithmetic, independent of eigh
    Km = mp.matrix(K.tolist()) * (-p.dtau)
    E = mp.eye(p.n_sites)
    term = mp.eye(p.n_sites)
    for n in range(1, 60):
        term = term * Km / n
        E = E + term
    P = mp.eye(p.n_sites)
    for s in range(p.n_slices):
        D = mp.diag([mp.exp(-p.dtau * (p.g * mp.mpf(float(x)) - p.mu)) for x in X[s]])
        P = E * D * P
    ref = mp.log(abs(mp.det(mp.eye(p.n_sites) + P)))
    expK, _ = dqmc.kinetic_propagators(p)
    assert abs(dqmc.log_det_M(p, expK, X) - float(ref)) < 1e-13 * abs(float(ref))


# ------------------------------------------------------------- Fock-space pins

@pytest.mark.parametrize("l", [0, 3, 10])
def test_green_and_observables_against_fock_space(l):
    p = small(2, 1.0, n_wrap=4)
    expK, _ = dqmc.kinetic_propagators(p)
    X = random_fields(p, 1, seed=21, scale=0.7)[0]
    cs = fock.annihilators(p.n_sites)
    K = dqmc.hopping_matrix(p)
    ops = fock.slice_operators(K, [p.g * X[s] - p.mu for s in range(p.n_slices)], p.dtau, cs)
    rho = fock.rho_at(ops, l)
    G, ld = dqmc.green_at(p, expK, X, l)
    assert np.max(np.abs(G - fock.green_fock(rho, cs))) < 1e-12
    assert abs(ld - math.log(abs(np.trace(rho)))) < 1e-12 * max(1, abs(ld))
    ref = fock.spinful_observables(rho, cs, dqmc.staggered_signs(p))
    got = dqmc.measure_green(p, G)
    for k in ref:
        assert abs(got[k] - ref[k]) < 1e-11, k


# ------------------------------------------------------- update formulas vs fresh

def test_local_ratio_update_and_wrap_against_fresh():
    p = small(4, 2.0)
    expK, expKinv = dqmc.kinetic_propagators(p)
    X = random_fields(p, 1, seed=8)[0]
    L, N = X.shape
    s, i, dx = 6, 5, 0.37
    G_prev, ld = dqmc.green_at(p, expK, X, s)       # G_{l-1} for slice l = s+1
    Xn = X.copy()
    Xn[s, i] += dx
    Gn_prev, ldn = dqmc.green_at(p, expK, Xn, s)
    delta = math.exp(-p.dtau * p.g * dx) - 1.0
    R1 = 1.0 + delta * (1.0 - G_prev[i, i])
    assert abs(2 * math.log(R1) - 2 * (ldn - ld)) < 1e-12
    col = G_prev[:, i].copy()
    col[i] -= 1.0
    G_upd = G_prev + (delta / R1) * np.outer(col, G_prev[i, :])
    assert np.max(np.abs(G_upd - Gn_prev)) < 1e-13
    d = dqmc.slice_diagonal(p, Xn[s])
    G_wrap = expK @ ((d[:, None] * G_upd) / d[None, :]) @ expKinv
    assert np.max(np.abs(G_wrap - dqmc.green_at(p, expK, Xn, s + 1)[0])) < 1e-12


def test_global_action_and_local_action_against_full_action():
    p = small(4, 2.0)
    X = random_fields(p, 1, seed=9)[0]
    Xn = X.copy()
    Xn[3, 2] += 0.21
    assert abs(dqmc.local_action_change(p, X, 3, 2, Xn[3, 2]) -
               (dqmc.phonon_action(p, Xn) - dqmc.phonon_action(p, X))) < 1e-11
    Xn = X.copy()
    Xn[:, 7] -= 0.6
    assert abs(dqmc.global_action_change(p, X, 7, -0.6) -
               (dqmc.phonon_action(p, Xn) - dqmc.phonon_action(p, X))) < 1e-11


def test_detailed_balance_every_accepted_move():
    """For every accepted move: fresh log W(X') - log W(X) = log R - dS used."""
    p = small(4, 2.0, n_wrap=5)
    expK, _ = dqmc.kinetic_propagators(p)
    X = random_fields(p, 1, seed=33, scale=0.8, offset=-1.4)[0]
    ch = dqmc.OracleChain(p, X, chain=2, record=True)
    ch.sweep()
    moves = [m for m in ch.moves if m["accepted"]]
    assert len([m for m in moves if m["kind"] == "local"]) > 50
    assert len([m for m in moves if m["kind"] == "global"]) > 0
    # X after each accepted move is the next accepted move's X_before (or the final X)
    afters = [m["X_before"] for m in moves[1:]] + [ch.X]
    for m, Xa in zip(moves, afters):
        lw_b = dqmc.log_weight(p, expK, m["X_before"])
        lw_a = dqmc.log_weight(p, expK, Xa)
        assert abs((lw_a - lw_b) - (m["log_ratio"] - m["dS"])) < 1e-9, m["kind"]


def test_sweep_keeps_green_consistent():
    p = small(4, 4.0)
    expK, _ = dqmc.kinetic_propagators(p)
    X = random_fields(p, 1, seed=4)[0]
    ch = dqmc.OracleChain(p, X)
    for _ in range(2):
        r = ch.sweep()
        assert r["max_wrap_error"] < 1e-10
    G, ld = dqmc.green_at(p, expK, ch.X, 0)
    assert np.max(np.abs(ch.G - G)) < 1e-13 and abs(ch.logdet - ld) < 1e-10


# --------------------------------------------------------------- free phonons

@pytest.mark.slow
def test_free_phonon_x2_statistics():
    p = HolsteinParams(nx=2, ny=2, beta=4.0, g=0.0, mu=0.0)
    X = random_fields(p, 1, seed=99, scale=0.7)[0]
    ch = dqmc.OracleChain(p, X, chain=0)
    series = []
    for _ in range(1200):
        series.append(ch.sweep(measure=True)["x2"])
    series = np.array(series[200:])
    tau, _ = autocorr.tau_int(series)
    err = series.std() * math.sqrt(2 * tau / series.size)
    ref = cf.free_phonon_x2(p.n_slices, p.dtau, p.mass, p.omega)
    assert abs(ref - 0.518042) < 1e-6
    assert abs(series.mean() - ref) < 3 * err, (series.mean(), ref, err, tau)


# ------------------------------------------------------------------- tau_int

def test_tau_int_white_noise_and_ar1():
    rng = np.random.default_rng(1)
    w = rng.standard_normal(20000)
    assert abs(autocorr.tau_int(w)[0] - 0.5) < 0.05
    for rho in (0.5, 0.9):
        x = np.empty(100000)
        x[0] = 0
        e = rng.standard_normal(x.size)
        for k in range(1, x.size):
            x[k] = rho * x[k - 1] + e[k]
        ref = 0.5 * (1 + rho) / (1 - rho)
        assert abs(autocorr.tau_int(x)[0] - ref) < 0.1 * ref


def test_stabilisation_backoff_halves_n_wrap_down_to_the_floor():
    """Back-off reading: a sweep whose largest wrap error exceeds wrap_tol halves n_wrap for the
    next sweeps, down to n_wrap_min, where the chain is reported unstable; a tolerance above the
    rounding-level wrap error changes nothing.  Every sweep stays consistent: G after the sweep
    equals a fresh G at the current n_wrap."""
    p = HolsteinParams(nx=4, ny=4, beta=1.6, n_wrap=8, n_wrap_min=2, wrap_tol=1e-300, seed=7)  # L = 16
    X0 = initial_fields(p, 1, seed=3)[0]
    ch = dqmc.OracleChain(p, X0)
    seq = []
    for _ in range(4):
        r = ch.sweep()
        assert r["max_wrap_error"] > 0.0
        seq.append(ch.n_wrap)
    assert seq == [4, 2, 2, 2]
    assert ch.wrap_exceeded == 4 and ch.unstable
    expK, _ = dqmc.kinetic_propagators(p)
    G, ld = dqmc.green_at(p, expK, ch.X, 0, ch.n_wrap)
    assert np.max(np.abs(G - ch.G)) < 1e-10 and abs(ld - ch.logdet) < 1e-10 * abs(ld)
    loose = dqmc.OracleChain(p.with_(wrap_tol=1e-6), X0)
    for _ in range(3):
        loose.sweep()
    assert loose.n_wrap == 8 and loose.wrap_exceeded == 0 and not loose.unstable
