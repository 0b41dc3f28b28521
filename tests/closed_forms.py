"""Closed forms that pin the oracle (derived from the model, not from the oracle's code).

* Free fermions (g = 0): on the periodic Nx x Ny lattice the hopping matrix is diagonal
  in plane waves with eps_k = -2t (cos kx + cos ky), k = 2 pi (mx/Nx, my/Ny).  Then
  M = I + exp(-beta (K - mu)) exactly for any Trotter step (all slices commute), so
  log det M = sum_k log(1 + exp(-beta (eps_k - mu))) and
  G_ij = (1/N) sum_k cos(k . (r_i - r_j)) / (1 + exp(-beta (eps_k - mu))).
* A uniform field X = x0 only shifts mu -> mu - g x0.
* The atomic limit t = 0 makes every B_l diagonal:
  det M = prod_i (1 + exp(-dtau sum_l V_il)), G_ii = 1 / (1 + exp(-dtau sum_l V_il)).
* Free phonons (g = 0): dtau S_ph = X^T A X / 2 per site with A circulant in imaginary
  time, eigenvalues (2M/dtau)(1 - cos(2 pi q / L)) + dtau M Omega^2, so
  <X_il^2> = (1/L) sum_q 1 / [(2M/dtau)(1 - cos(2 pi q/L)) + dtau M Omega^2].
"""
import math

import numpy as np


def dispersion(nx, ny, t):
    eps = []
    for my in range(ny):
        for mx in range(nx):
            kx, ky = 2 * math.pi * mx / nx, 2 * math.pi * my / ny
            eps.append((kx, ky, -2.0 * t * (math.cos(kx) + math.cos(ky))))
    return eps


def _log1pexp(z):
    return z + math.log1p(math.exp(-z)) if z > 0 else math.log1p(math.exp(z))


def free_logdet(nx, ny, t, mu, beta, shift=0.0):
    """sum_k log(1 + exp(-beta (eps_k + shift - mu)))."""
    return sum(_log1pexp(-beta * (e + shift - mu)) for _, _, e in dispersion(nx, ny, t))


def free_green(nx, ny, t, mu, beta, shift=0.0):
    N = nx * ny
    G = np.zeros((N, N))
    xs = np.array([i % nx for i in range(N)])
    ys = np.array([i // nx for i in range(N)])
    dxm = xs[:, None] - xs[None, :]
    dym = ys[:, None] - ys[None, :]
    for kx, ky, e in dispersion(nx, ny, t):
        z = -beta * (e + shift - mu)
        f = 1.0 / (1.0 + math.exp(z)) if z < 700 else 0.0
        G += np.cos(kx * dxm + ky * dym) * f
    return G / N


def free_phonon_x2(L, dtau, mass, omega):
    return sum(1.0 / ((2 * mass / dtau) * (1 - math.cos(2 * math.pi * q / L)) + dtau * mass * omega ** 2)
               for q in range(L)) / L
