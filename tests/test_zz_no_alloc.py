"""hq_logdet_noalloc: log|det M| with no device allocation by the library.

Some callers cannot allocate device memory -- they only hold buffers handed over by a host
framework whose memory pool owns the GPU, or they must not allocate once running (a
serving loop).  This entry point takes only their input and output buffers and keeps its
scratch in a static device array inside the library.  The test drives it through the C ABI
on caller-owned tensors and compares it with the engine's log|det M| (hq_log_weight) on the
same fields, on two calls in a row (the second reuses the scratch the first left behind), and
with the CPU oracle's log|det M| directly.
The file sorts last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from workloads import BATCHED, HolsteinParams, initial_fields, random_fields

pytestmark = pytest.mark.gpu

LD_RTOL = 1e-10


@pytest.fixture(scope="module")
def hq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1905_07440_gb300 as mod
    mod.load_library()
    return mod


def engine_logdet(hq, p, X):
    eng = hq.Engine(p, X.shape[0])
    eng.set_fields(X)
    _, ld = eng.log_weight()
    eng.close()
    return ld


def test_noalloc_logdet_matches_engine_on_two_calls(hq):
    import torch
    calls = [(BATCHED, initial_fields(BATCHED, 24)),
             (HolsteinParams(nx=6, ny=6, beta=3.0, n_wrap=7), random_fields(
                 HolsteinParams(nx=6, ny=6, beta=3.0, n_wrap=7), 40, seed=3, offset=-1.0))]
    stream = torch.cuda.current_stream()
    for p, X in calls:
        Xd = torch.from_numpy(X).cuda()
        out = torch.full((X.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        hq.logdet_noalloc(p, Xd, out, stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = engine_logdet(hq, p, X)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / np.abs(ref)) < LD_RTOL


def test_noalloc_logdet_matches_the_oracle(hq):
    """Small lattices against the oracle's stabilised log|det M| (scipy pivoted QR), including
    a ragged n_wrap and non-unit t, M, Omega; two calls in a row on the shared scratch."""
    import torch
    from oracle import dqmc
    cases = [HolsteinParams(nx=4, ny=4, beta=1.0), HolsteinParams(nx=6, ny=4, beta=1.3, n_wrap=4, t=0.8,
                                                                   mass=1.3, omega=0.5, g=1.0, mu=-3.0)]
    for p in cases:
        X = random_fields(p, 3, seed=41, offset=-1.0)
        Xd = torch.from_numpy(X).cuda()
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        hq.logdet_noalloc(p, Xd, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        expK, _ = dqmc.kinetic_propagators(p)
        for c in range(3):
            ref = dqmc.log_det_M(p, expK, X[c])
            assert abs(got[c] - ref) <= LD_RTOL * abs(ref), (p, c, got[c], ref)


def test_noalloc_rejects_sizes_beyond_the_scratch(hq):
    import torch
    p = HolsteinParams(nx=16, ny=16, beta=1.0)
    X = torch.zeros((64, p.n_slices, p.n_sites), dtype=torch.float64, device="cuda")
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(hq.HQError, match="scratch"):
        hq.logdet_noalloc(p, X, out)
