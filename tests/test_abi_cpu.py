"""C-ABI checks that need no GPU: the library loads, exports every declared symbol,
validates parameters on the host and computes tau_int like the oracle."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

from workloads import HolsteinParams

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "holstein_dqmc.h")


def _lib():
    import paper_1905_07440_gb300 as hq
    if not os.path.exists(hq.LIB_PATH):
        from paper_1905_07440_gb300 import build
        build.build()
    return hq, hq.load_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hq_[a-z0-9_]+)\s*\(", src)))


def test_header_declarations_match_binding():
    hq, _ = _lib()
    assert declared_functions() == sorted(hq.EXPORTED)


def test_library_exports_every_declared_symbol():
    hq, lib = _lib()
    out = subprocess.run(["nm", "-D", "--defined-only", hq.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hq_[a-z0-9_]+)\b", out))
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_arena_bytes_validates_parameters():
    hq, _ = _lib()
    from workloads import SMALL, BATCHED
    assert hq.arena_bytes(SMALL, 1) > 0
    assert hq.arena_bytes(BATCHED, 256, 1000) > hq.arena_bytes(BATCHED, 128, 1000)
    bad = [SMALL.with_(nx=3, ny=3), SMALL.with_(nx=18, ny=18), SMALL.with_(beta=4.05), SMALL.with_(dtau=0.0),
           SMALL.with_(delay_k=0), SMALL.with_(delay_k=33), SMALL.with_(n_wrap=0), SMALL.with_(mass=0.0),
           SMALL.with_(beta=0.1)]
    for p in bad:
        assert hq.arena_bytes(p, 1) == 0, p
    assert hq.arena_bytes(SMALL, 0) == 0


def test_arena_holds_the_largest_lattice():
    hq, _ = _lib()
    from workloads import LARGEST
    nb = hq.arena_bytes(LARGEST, 64, 2000)
    # fields, G, UDV stack (15 boundaries x 2 N^2), 7 work matrices, right factors
    n, L = 256, 160
    assert nb >= 8 * 64 * (L * n + (15 * 2 + 10) * n * n)
    assert nb < 4 * 2 ** 30


def test_tau_int_matches_oracle():
    hq, _ = _lib()
    from oracle import autocorr
    rng = np.random.default_rng(7)
    x = np.empty(5000)
    x[0] = 0.0
    for k in range(1, x.size):
        x[k] = 0.8 * x[k - 1] + rng.standard_normal()
    t_c, w_c = hq.tau_int(x)
    t_o, w_o = autocorr.tau_int(x)
    assert w_c == w_o
    assert abs(t_c - t_o) < 1e-10 * t_o
    assert hq.tau_int(np.ones(10))[0] == 0.5


def test_autotune_arena_is_the_largest_candidate():
    import paper_1905_07440_gb300 as hq
    lib = hq.load_library()
    p = HolsteinParams(nx=8, ny=8, beta=2.0)

    def need(ks):
        arr = (ctypes.c_int * len(ks))(*ks)
        return int(lib.hq_autotune_arena_bytes(ctypes.byref(hq.make_params(p)), 16, arr, len(ks)))

    one = {k: need([k]) for k in (1, 8, 32)}
    assert 0 < one[1] <= one[8] <= one[32]
    assert need([8, 1, 32]) == one[32]
    # the chunk-propagator layout is the larger one and is always included
    for m in (1, 2):
        assert hq.arena_bytes(p.with_(delay_k=32, block_method=m), 16) <= one[32]
    assert need([0]) == 0 and need([33]) == 0


def test_wait_probe_rejects_bad_limits():
    import paper_1905_07440_gb300 as hq
    lib = hq.load_library()
    st = ctypes.c_int()
    for bad in (0.0, -1.0, 3.0):
        assert lib.hq_wait_probe(bad, None, ctypes.byref(st)) == hq.HQ_EINVAL
    assert lib.hq_wait_probe(0.1, None, None) == hq.HQ_EINVAL


def test_group_arena_rejects_empty_sets():
    import paper_1905_07440_gb300 as hq
    lib = hq.load_library()
    assert lib.hq_group_arena_bytes(None, 0) == 0
    assert lib.hq_group_arena_bytes(None, 3) == 0
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.hq_group_arena_bytes(arr, 1) == 0          # null engine


def test_noalloc_binding_rejects_bad_tensors_before_the_library():
    """The no-allocation entry point trusts the sizes it is given, so the binding checks dtype,
    shape, length and device on the host; none of these calls reaches the library."""
    import torch
    import paper_1905_07440_gb300 as hq
    p = HolsteinParams(nx=4, ny=4, beta=1.0)
    good = torch.zeros((3, p.n_slices, p.n_sites), dtype=torch.float64)
    out = torch.zeros(3, dtype=torch.float64)
    with pytest.raises(TypeError):
        hq.logdet_noalloc(p, good.float(), out)
    with pytest.raises(TypeError):
        hq.logdet_noalloc(p, good, out.float())
    with pytest.raises(ValueError, match="shape"):
        hq.logdet_noalloc(p, torch.zeros((3, p.n_slices + 1, p.n_sites), dtype=torch.float64), out)
    with pytest.raises(ValueError, match="shape"):
        hq.logdet_noalloc(p, torch.zeros((p.n_slices, p.n_sites), dtype=torch.float64), out)
    with pytest.raises(ValueError, match="chains"):
        hq.logdet_noalloc(p, good, torch.zeros(2, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA"):
        hq.logdet_noalloc(p, good, out)


def test_backoff_parameters_are_validated_and_size_the_arena():
    hq, _ = _lib()
    p = HolsteinParams(nx=6, ny=6, beta=2.0, n_wrap=10)
    assert hq.arena_bytes(p.with_(wrap_tol=-1.0), 1) == 0
    assert hq.arena_bytes(p.with_(wrap_tol=float("inf")), 1) == 0
    assert hq.arena_bytes(p.with_(n_wrap_min=11, wrap_tol=1e-8), 1) == 0
    base = hq.arena_bytes(p, 4)
    # the stack is sized for the smallest n_wrap the back-off can reach
    assert hq.arena_bytes(p.with_(wrap_tol=1e-8, n_wrap_min=10), 4) == base
    assert hq.arena_bytes(p.with_(wrap_tol=1e-8, n_wrap_min=2), 4) > base
    assert hq.arena_bytes(p.with_(wrap_tol=1e-8), 4) >= hq.arena_bytes(p.with_(wrap_tol=1e-8, n_wrap_min=2), 4)
