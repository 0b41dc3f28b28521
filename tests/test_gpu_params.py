"""GPU parity at the model's other parameters (paper, "Model": hopping t, ion mass M, phonon
frequency Omega, coupling g, chemical potential mu) and on the 16-wide kernel template that the
12x12 and 16x16 lattices use.

Every other parity file runs t = M = Omega = 1; here the kernels' t, M and Omega arithmetic
(the kinetic factors, the phonon action of local and block moves) is compared with the oracle at
t = 0.8, M = 1.3, Omega = 0.5, and at the paper's own benchmark point (Omega = t/2,
lambda = g^2/(M Omega^2 8t) = 1/2, half filling mu = -g^2/(M Omega^2) = -4, beta = 4.1).
Tolerances as in test_gpu_parity: fields bit for bit, log|det M| to 1e-10 relative, G to 1e-10.
"""
import numpy as np
import pytest

from workloads import HolsteinParams, initial_fields, half_filling_mu
from tests.test_gpu_parity import check_against_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1905_07440_gb300 as mod
    mod.load_library()
    return mod


def off_unit(nx, ny, beta, **kw):
    """t = 0.8, M = 1.3, Omega = 0.5, g = 1 at half filling."""
    base = dict(t=0.8, mass=1.3, omega=0.5, g=1.0)
    base.update(kw)
    return HolsteinParams(nx=nx, ny=ny, beta=beta, mu=half_filling_mu(base["g"], base["mass"], base["omega"]), **base)


@pytest.mark.parametrize("nx,ny,n_wrap,k", [(4, 4, 10, 16), (6, 6, 4, 5), (10, 6, 3, 8)])
def test_full_sweeps_at_non_unit_t_mass_omega(hq, nx, ny, n_wrap, k):
    """Local moves (delayed updates, wraps, restabilisation) and a block move per site with
    t, M, Omega all different from 1; 10x6 runs on the 16-wide template."""
    p = off_unit(nx, ny, 1.0, n_wrap=n_wrap, delay_k=k, seed=2024 + nx)
    X0 = initial_fields(p, 2, seed=31)
    check_against_oracle(hq, p, X0, 2)


@pytest.mark.parametrize("forced", [1, 2])
@pytest.mark.parametrize("nx,beta,n_wrap,unit", [(12, 0.5, 10, False), (16, 0.3, 10, True), (16, 0.4, 2, False)])
def test_block_moves_on_the_largest_lattices(hq, nx, beta, n_wrap, unit, forced):
    """Global-only sweeps at 12x12 and 16x16 (the 16-wide template), both block-move
    algorithms, one or two chunks per product; fields bit for bit against the oracle."""
    if unit:
        p = HolsteinParams(nx=nx, ny=nx, beta=beta, n_wrap=n_wrap, seed=91, block_method=forced)
    else:
        p = off_unit(nx, nx, beta, n_wrap=n_wrap, seed=92, block_method=forced)
    eng = hq.Engine(p, 1)
    assert eng.block_move_method == forced - 1
    eng.close()
    X0 = initial_fields(p, 1, seed=17)
    check_against_oracle(hq, p, X0, 1, local=False, global_=True)


def test_local_sweep_at_non_unit_parameters_on_the_largest_template(hq):
    """12x12 local sweep (16-wide template) with t, M, Omega != 1 and a ragged last chunk."""
    p = off_unit(12, 12, 0.7, n_wrap=3, delay_k=16, seed=93)
    X0 = initial_fields(p, 1, seed=19)
    check_against_oracle(hq, p, X0, 1, local=True, global_=False)


@pytest.mark.parametrize("nx,chains", [(4, 2), (6, 1)])
def test_paper_benchmark_point(hq, nx, chains):
    """Omega = 0.5, g = 1 (lambda = 1/2), mu = -4, beta = 4.1 (L = 41: a ragged last chunk of
    one slice), fields started at the mean field -g/(M Omega^2) with the free-phonon spread, as
    the physics-point benchmark does; one full sweep."""
    p = HolsteinParams(nx=nx, ny=nx, omega=0.5, g=1.0, mu=-4.0, beta=4.1, seed=95)
    X0 = initial_fields(p, chains, seed=23) - p.g / (p.mass * p.omega ** 2)
    check_against_oracle(hq, p, X0, 1)


@pytest.mark.parametrize("nx,beta,sites,local,method", [(4, 1.0, 3, False, 1), (6, 0.8, 5, True, 2),
                                                        (12, 0.4, 7, False, 2)])
def test_block_moves_on_a_run_of_sites(hq, nx, beta, sites, local, method):
    """The reduced protocol for large lattices: each sweep's block moves on a run of `sites`
    consecutive sites from a Philox-drawn start (event N of the sweep's block-move stream);
    fields, counts and weights against the oracle over two sweeps (two different starts)."""
    p = HolsteinParams(nx=nx, ny=nx, beta=beta, seed=97, block_method=method, delay_k=8)
    X0 = initial_fields(p, 2, seed=29)
    check_against_oracle(hq, p, X0, 2, local=local, global_=True, block_sites=sites)


def test_stabilisation_backoff_matches_the_oracle(hq):
    """wrap_tol below the rounding-level wrap error: every sweep halves n_wrap (8 -> 4 -> 2), the
    third sweep at the floor returns HQ_EUNSTABLE with the chains' status set, and the chains
    still follow the oracle with the same back-off bit for bit; a loose tolerance does nothing."""
    from oracle import dqmc
    p = HolsteinParams(nx=4, ny=4, beta=1.6, n_wrap=8, n_wrap_min=2, wrap_tol=1e-300, delay_k=4, seed=61)
    X0 = initial_fields(p, 2, seed=5)
    eng = hq.Engine(p, 2, max_series=8)
    eng.set_fields(X0)
    eng.sweep(2)
    assert all(o["n_wrap"] == 2 and o["wrap_exceeded"] == 2 and o["status"] == 0 for o in eng.observables())
    with pytest.raises(hq.HQError, match=r"\(-4\)"):
        eng.sweep(1)
    obs = eng.observables()
    Xg = eng.get_fields()
    _, ld = eng.log_weight()
    for c in range(2):
        assert obs[c]["n_wrap"] == 2 and obs[c]["wrap_exceeded"] == 3 and obs[c]["status"] == hq.HQ_EUNSTABLE
        ch = dqmc.OracleChain(p, X0[c], chain=c)
        for _ in range(3):
            ch.sweep()
        assert ch.n_wrap == 2 and ch.unstable
        assert np.array_equal(Xg[c], ch.X)
        assert abs(ld[c] - ch.logdet) <= 1e-10 * abs(ch.logdet)
        assert np.max(np.abs(eng.green(c) - ch.G)) < 1e-10
    loose = hq.Engine(p.with_(wrap_tol=1e-6), 2)
    loose.set_fields(X0)
    loose.sweep(3)
    assert all(o["n_wrap"] == 8 and o["wrap_exceeded"] == 0 and o["status"] == 0 for o in loose.observables())
