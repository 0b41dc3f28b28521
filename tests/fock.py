"""Brute-force many-body (Fock-space) evaluation for tiny lattices.

Used only to pin the oracle: it never goes through single-particle matrices, UDV
factors or Wick's theorem.  Spinless modes 0..n-1 are built by a Jordan-Wigner string;
a bilinear sum_ij c_i^dagger h_ij c_j becomes a 2^n x 2^n matrix and its exponential is
taken with scipy.linalg.expm.  For the spinful Holstein problem both spins see the same
single-particle operators, so the two-spin density operator is rho_up (x) rho_dn.
"""
import numpy as np
import scipy.linalg


def annihilators(n):
    """c_0..c_{n-1} as dense 2^n x 2^n matrices (mode i is bit i of the basis index)."""
    dim = 1 << n
    cs = []
    for i in range(n):
        c = np.zeros((dim, dim))
        for s in range(dim):
            if s >> i & 1:
                sign = -1.0 if bin(s & ((1 << i) - 1)).count("1") % 2 else 1.0
                c[s ^ (1 << i), s] = sign
        cs.append(c)
    return cs


def bilinear(cs, h):
    n = len(cs)
    out = np.zeros_like(cs[0])
    for i in range(n):
        for j in range(n):
            if h[i, j] != 0.0:
                out += h[i, j] * cs[i].T @ cs[j]
    return out


def slice_operators(K, V_list, dtau, cs):
    """Fock-space exp(-dtau K^) exp(-dtau V^_l) for each slice l."""
    eK = scipy.linalg.expm(-dtau * bilinear(cs, K))
    return [eK @ scipy.linalg.expm(-dtau * bilinear(cs, np.diag(v))) for v in V_list]


def rho_at(ops, l):
    """B^_l ... B^_1 B^_L ... B^_{l+1} (ops[s] is slice s+1)."""
    L = len(ops)
    order = list(range(l, L)) + list(range(0, l))
    rho = np.eye(ops[0].shape[0])
    for s in order:
        rho = ops[s] @ rho
    return rho


def green_fock(rho, cs):
    """G_ij = Tr(rho c_i c_j^dagger) / Tr(rho)."""
    z = np.trace(rho)
    n = len(cs)
    G = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            G[i, j] = np.trace(rho @ cs[i] @ cs[j].T) / z
    return G


def spinful_observables(rho, cs, signs):
    """density, double occupancy and S_CDW(pi, pi) for rho_up (x) rho_dn = rho (x) rho."""
    n = len(cs)
    dim = rho.shape[0]
    eye = np.eye(dim)
    rho2 = np.kron(rho, rho)
    z = np.trace(rho2)
    nup = [np.kron(cs[i].T @ cs[i], eye) for i in range(n)]
    ndn = [np.kron(eye, cs[i].T @ cs[i]) for i in range(n)]
    ntot = [nup[i] + ndn[i] for i in range(n)]
    dens = sum(np.trace(rho2 @ ntot[i]) for i in range(n)) / z / n
    docc = sum(np.trace(rho2 @ nup[i] @ ndn[i]) for i in range(n)) / z / n
    s = 0.0
    for i in range(n):
        for j in range(n):
            s += signs[i] * signs[j] * np.trace(rho2 @ ntot[i] @ ntot[j]) / z
    return dict(density=float(dens), double_occ=float(docc), s_cdw=float(s / n))
