"""Seeded synthetic inputs for the Holstein DQMC engine.

This module holds the workload definitions (model parameters and run shapes) and the
seeded generators of the initial phonon field.  It contains none of the method's
arithmetic, and both the CPU oracle and the CUDA path draw their inputs from it.

The paper has no public dataset: its workloads are its own DQMC chains on N = Nx^2
periodic square lattices with dtau = 0.1.  The runs below use the paper's model with
t = M = Omega = 1, lambda = g^2 / (M Omega^2 8 t) = 0.25 (g = sqrt(2)) and half filling
mu = -g^2 / (M Omega^2) = -2, at the lattice sizes, temperatures and chain counts named.
"""
import math
from dataclasses import dataclass, asdict, replace

import numpy as np

DEFAULT_SEED = 20190517


@dataclass(frozen=True)
class HolsteinParams:
    nx: int
    ny: int
    t: float = 1.0
    mu: float = -2.0
    omega: float = 1.0
    mass: float = 1.0
    g: float = math.sqrt(2.0)
    beta: float = 4.0
    dtau: float = 0.1
    n_wrap: int = 10
    delay_k: int = 16
    dx_local: float = 0.5
    dx_global: float = 1.0
    seed: int = DEFAULT_SEED
    block_method: int = 0  # engine's block-move algorithm (0 flop model, 1 per slice, 2 chunks)
    n_wrap_min: int = 0    # stabilisation back-off floor (0: 1)
    wrap_tol: float = 0.0  # stabilisation back-off threshold on |G_wrapped - G_fresh| (0: off)

    @property
    def n_sites(self) -> int:
        return self.nx * self.ny

    @property
    def n_slices(self) -> int:
        return int(round(self.beta / self.dtau))

    def as_dict(self):
        return asdict(self)

    def with_(self, **kw):
        return replace(self, **kw)


def half_filling_mu(g, mass=1.0, omega=1.0):
    """Chemical potential of the particle-hole symmetric point for the coupling g X n."""
    return -g * g / (mass * omega * omega)


def coupling_from_lambda(lam, t=1.0, mass=1.0, omega=1.0):
    """g from the dimensionless coupling lambda = g^2 / (M Omega^2 8 t)."""
    return math.sqrt(lam * mass * omega * omega * 8.0 * t)


# 4x4, beta = 4 (L = 40), one chain, 100 warm-up + 200 measured sweeps: the small case.
SMALL = HolsteinParams(nx=4, ny=4, beta=4.0, delay_k=16)
SMALL_RUN = dict(n_chains=1, warmup_sweeps=100, sweeps=200)

# 8x8, beta = 8 (L = 80), 256 chains, delay rank 16, one global move per site per sweep.
BATCHED = HolsteinParams(nx=8, ny=8, beta=8.0, delay_k=16)
BATCHED_RUN = dict(n_chains=256, sweeps=1000)

# 12x12, beta = 8 (L = 80), 128 chains (plain part of the learned-proposal workload).
MEDIUM = HolsteinParams(nx=12, ny=12, beta=8.0, delay_k=16)
MEDIUM_RUN = dict(n_chains=128)

# 16x16, beta = 16 (L = 160), 64 chains: the largest lattice.
LARGEST = HolsteinParams(nx=16, ny=16, beta=16.0, delay_k=16)
LARGEST_RUN = dict(n_chains=64, sweeps=2000)


def initial_fields(params: HolsteinParams, n_chains: int, seed: int = DEFAULT_SEED):
    """X[chain][l][i] drawn i.i.d. from N(0, 1/(M Omega^2)); chain c uses seed + c."""
    L, N = params.n_slices, params.n_sites
    sd = 1.0 / math.sqrt(params.mass * params.omega ** 2)
    X = np.empty((n_chains, L, N), dtype=np.float64)
    for c in range(n_chains):
        X[c] = np.random.default_rng(seed + c).normal(0.0, sd, size=(L, N))
    return X


def ordered_fields(params: HolsteinParams, n_chains: int, amplitude: float, seed: int = DEFAULT_SEED):
    """Charge-ordered start for low temperatures: X(i, l) = -g/(M Omega^2) + amplitude (-1)^(x+y)
    plus i.i.d. N(0, 1/(2 M Omega)) (the oscillator's zero-point spread); chain c uses seed + c."""
    L, N = params.n_slices, params.n_sites
    x0 = -params.g / (params.mass * params.omega ** 2)
    stag = np.array([1.0 if ((i % params.nx) + (i // params.nx)) % 2 == 0 else -1.0 for i in range(N)])
    sd = 1.0 / math.sqrt(2.0 * params.mass * params.omega)
    X = np.empty((n_chains, L, N), dtype=np.float64)
    for c in range(n_chains):
        X[c] = x0 + amplitude * stag[None, :] + np.random.default_rng(seed + c).normal(0.0, sd, size=(L, N))
    return X


def random_fields(params: HolsteinParams, n_chains: int, seed: int, scale: float = 1.0,
                  offset: float = 0.0):
    """Generic seeded test fields: offset + scale * N(0, 1) of shape [chain][L][N]."""
    rng = np.random.default_rng(seed)
    return offset + scale * rng.standard_normal((n_chains, params.n_slices, params.n_sites))


def uniform_fields(params: HolsteinParams, n_chains: int, x0: float):
    """Every X(i, l) equal to x0."""
    return np.full((n_chains, params.n_slices, params.n_sites), float(x0))
