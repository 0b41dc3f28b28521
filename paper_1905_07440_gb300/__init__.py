"""Python binding of the GB300 Holstein DQMC engine (C ABI in include/holstein_dqmc.h).

Argument marshalling only: every step of a sweep runs in the CUDA library
libholstein_dqmc.so built in this directory (see build.py).  PyTorch provides the
device arena and the stream; there is no CPU fallback -- importing the binding fails
loudly when the library has not been built.
"""
import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libholstein_dqmc.so")

HQ_OK = 0
HQ_EINVAL = -1
HQ_ENOMEM = -2
HQ_ECUDA = -3
HQ_EUNSTABLE = -4
HQ_ENAN = -5
HQ_ETIMEOUT = -6

HQ_LOCAL = 1
HQ_GLOBAL = 2
HQ_MEASURE = 4

HQ_OBS_DENSITY = 0
HQ_OBS_DOUBLE_OCC = 1
HQ_OBS_SCDW = 2
HQ_OBS_X_MEAN = 3
HQ_OBS_X2 = 4
HQ_OBS_WRAP_ERR = 5
HQ_N_OBS = 6
OBS_NAMES = ("density", "double_occ", "s_cdw", "x_mean", "x2", "wrap_error")


class hq_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("t", ctypes.c_double), ("mu", ctypes.c_double),
                ("omega", ctypes.c_double), ("mass", ctypes.c_double), ("g", ctypes.c_double),
                ("beta", ctypes.c_double), ("dtau", ctypes.c_double), ("n_wrap", ctypes.c_int),
                ("delay_k", ctypes.c_int), ("dx_local", ctypes.c_double), ("dx_global", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("block_method", ctypes.c_int), ("n_wrap_min", ctypes.c_int),
                ("wrap_tol", ctypes.c_double)]


class hq_obs(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("measured", ctypes.c_int64),
                ("local_proposed", ctypes.c_int64), ("local_accepted", ctypes.c_int64),
                ("global_proposed", ctypes.c_int64), ("global_accepted", ctypes.c_int64),
                ("density", ctypes.c_double), ("double_occ", ctypes.c_double), ("s_cdw", ctypes.c_double),
                ("x_mean", ctypes.c_double), ("x2", ctypes.c_double), ("max_wrap_error", ctypes.c_double),
                ("logdet", ctypes.c_double), ("status", ctypes.c_int32), ("n_wrap", ctypes.c_int32),
                ("wrap_exceeded", ctypes.c_int64)]


class hq_learned_stats(ctypes.Structure):
    _fields_ = [("inner_local_proposed", ctypes.c_int64), ("inner_local_accepted", ctypes.c_int64),
                ("inner_block_proposed", ctypes.c_int64), ("inner_block_accepted", ctypes.c_int64),
                ("cumulative_proposed", ctypes.c_int64), ("cumulative_accepted", ctypes.c_int64),
                ("last_pc", ctypes.c_double)]


HQ_NN_PARAMS = 5889
HQ_CNN_PARAMS = 7809
HQ_CNN_BLOCK = 8

_P = ctypes.POINTER
_dp = _P(ctypes.c_double)
_vp = ctypes.c_void_p
_SIGNATURES = {
    "hq_arena_bytes": (ctypes.c_size_t, [_P(hq_params), ctypes.c_int, ctypes.c_int]),
    "hq_create": (ctypes.c_int, [_P(hq_params), ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t,
                                 _vp, _P(_vp)]),
    "hq_set_fields": (ctypes.c_int, [_vp, _dp]),
    "hq_set_fields_device": (ctypes.c_int, [_vp, _vp]),
    "hq_get_fields": (ctypes.c_int, [_vp, _dp]),
    "hq_sweep": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_uint]),
    "hq_log_weight": (ctypes.c_int, [_vp, _dp, _dp]),
    "hq_get_green": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _P(ctypes.c_int)]),
    "hq_get_observables": (ctypes.c_int, [_vp, _P(hq_obs)]),
    "hq_get_series": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _P(ctypes.c_int)]),
    "hq_checkpoint": (ctypes.c_int, [_vp, _vp, _P(ctypes.c_size_t)]),
    "hq_restore": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "hq_block_move_method": (ctypes.c_int, [_vp]),
    "hq_set_chain": (ctypes.c_int, [_vp, ctypes.c_int, _dp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]),
    "hq_set_active": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "hq_shape": (ctypes.c_int, [_vp, _P(ctypes.c_int), _P(ctypes.c_int), _P(ctypes.c_int), _P(ctypes.c_int64)]),
    "hq_last_error": (ctypes.c_char_p, [_vp]),
    "hq_destroy": (None, [_vp]),
    "hq_proposal_uniforms": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                            _P(ctypes.c_uint32), ctypes.c_int, _dp, _dp, _vp]),
    "hq_tau_int": (ctypes.c_double, [_dp, ctypes.c_int, ctypes.c_double, _P(ctypes.c_int)]),
    "hq_fp64_peak_tflops": (ctypes.c_double, [ctypes.c_int, ctypes.c_int, _vp]),
    "hq_set_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "hq_set_graphs": (ctypes.c_int, [_vp, ctypes.c_int]),
    "hq_wait_probe": (ctypes.c_int, [ctypes.c_double, _vp, _P(ctypes.c_int)]),
    "hq_logdet_noalloc": (ctypes.c_int, [_P(hq_params), ctypes.c_int, _vp, _vp, _vp]),
    "hq_nn_arena_bytes": (ctypes.c_size_t, [_vp, ctypes.c_int, ctypes.c_int]),
    "hq_nn_attach": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_int]),
    "hq_nn_set_params": (ctypes.c_int, [_vp, _P(ctypes.c_float)]),
    "hq_nn_get_params": (ctypes.c_int, [_vp, _P(ctypes.c_float), ctypes.c_int]),
    "hq_nn_eval": (ctypes.c_int, [_vp, _dp]),
    "hq_nn_train": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                   ctypes.c_uint64, _dp]),
    "hq_nn_gradient": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _P(ctypes.c_float), _dp]),
    "hq_cumulative_sweep": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint]),
    "hq_set_inner_window": (ctypes.c_int, [_vp, ctypes.c_int]),
    "hq_set_inner_sites": (ctypes.c_int, [_vp, ctypes.c_int]),
    "hq_set_logdet_split": (ctypes.c_int, [_vp, ctypes.c_int]),
    "hq_set_block_sites": (ctypes.c_int, [_vp, ctypes.c_int]),
    "hq_cnn_set_params": (ctypes.c_int, [_vp, _P(ctypes.c_float)]),
    "hq_cnn_get_params": (ctypes.c_int, [_vp, _P(ctypes.c_float), ctypes.c_int]),
    "hq_cnn_eval": (ctypes.c_int, [_vp, _dp]),
    "hq_cnn_train": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                    ctypes.c_uint64, _dp]),
    "hq_cnn_gradient": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _P(ctypes.c_float), _dp]),
    "hq_get_learned_stats": (ctypes.c_int, [_vp, _P(hq_learned_stats)]),
    "hq_get_section_cycles": (ctypes.c_int, [_P(ctypes.c_uint64), ctypes.c_int]),
    "hq_group_arena_bytes": (ctypes.c_size_t, [_P(_vp), ctypes.c_int]),
    "hq_group_create": (ctypes.c_int, [_P(_vp), ctypes.c_int, _vp, ctypes.c_size_t, _vp, _P(_vp)]),
    "hq_group_sweep": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_uint]),
    "hq_group_destroy": (None, [_vp]),
    "hq_autotune_arena_bytes": (ctypes.c_size_t, [_P(hq_params), ctypes.c_int, _P(ctypes.c_int), ctypes.c_int]),
    "hq_autotune": (ctypes.c_int, [_P(hq_params), ctypes.c_int, _vp, _vp, ctypes.c_size_t, _vp, _P(ctypes.c_int),
                                   ctypes.c_int, _P(ctypes.c_int), ctypes.c_int, ctypes.c_uint, ctypes.c_int,
                                   ctypes.c_int, _dp, _P(ctypes.c_int), _P(ctypes.c_int)]),
    "hq_get_timing": (ctypes.c_int, [_vp, _dp, _P(ctypes.c_int64)]),
}
HQ_N_PHASES = 8
PHASES = ("stack_build", "local_chunk", "block_moves", "sweep_end", "split_halves", "split_join", "network_eval",
          "network_inner")
EXPORTED = tuple(_SIGNATURES)

_lib = None


def load_library(path=LIB_PATH):
    """Load libholstein_dqmc.so and declare every exported symbol.  Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1905_07440_gb300.build.build() "
                          "(the engine has no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(_dp)


class HQError(RuntimeError):
    pass


def make_params(p):
    """hq_params from any object with the workloads.HolsteinParams attributes."""
    return hq_params(p.nx, p.ny, p.t, p.mu, p.omega, p.mass, p.g, p.beta, p.dtau, p.n_wrap, p.delay_k,
                     p.dx_local, p.dx_global, p.seed, int(getattr(p, "block_method", 0)),
                     int(getattr(p, "n_wrap_min", 0)), float(getattr(p, "wrap_tol", 0.0)))


def arena_bytes(params, n_chains, max_series=0):
    lib = load_library()
    return int(lib.hq_arena_bytes(ctypes.byref(make_params(params)), n_chains, max_series))


class Engine:
    """n_chains independent Holstein DQMC chains on one GPU (thin wrapper of hq_*)."""

    def __init__(self, params, n_chains, first_chain=0, max_series=0, device=None, stream=None):
        import torch
        self.lib = load_library()
        self.params = params
        self.n_chains = int(n_chains)
        self.max_series = int(max_series)
        self._p = make_params(params)
        nbytes = self.lib.hq_arena_bytes(ctypes.byref(self._p), self.n_chains, self.max_series)
        if nbytes == 0:
            raise HQError("invalid parameters")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.arena.data_ptr()
        aligned = (base + 255) // 256 * 256
        self._h = ctypes.c_void_p()
        rc = self.lib.hq_create(ctypes.byref(self._p), self.n_chains, int(first_chain), self.max_series,
                                ctypes.c_void_p(aligned), nbytes, ctypes.c_void_p(self.stream.cuda_stream),
                                ctypes.byref(self._h))
        if rc != HQ_OK:
            raise HQError(f"hq_create failed ({rc})")
        n_c, n_s, n_l = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.lib.hq_shape(self._h, ctypes.byref(n_c), ctypes.byref(n_s), ctypes.byref(n_l), None)
        self.n_sites, self.n_slices = n_s.value, n_l.value

    def _check(self, rc, what):
        if rc != HQ_OK:
            msg = self.lib.hq_last_error(self._h)
            raise HQError(f"{what} failed ({rc}): {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.hq_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def field_shape(self):
        return (self.n_chains, self.n_slices, self.n_sites)

    def set_fields(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64)
        if X.shape != self.field_shape:
            raise ValueError(f"fields must have shape {self.field_shape}")
        self._check(self.lib.hq_set_fields(self._h, _dptr(X)), "hq_set_fields")

    def set_fields_device(self, X):
        """X: contiguous float64 CUDA tensor of field_shape."""
        assert X.is_cuda and X.dtype.is_floating_point and X.element_size() == 8 and X.is_contiguous()
        assert tuple(X.shape) == self.field_shape
        self._check(self.lib.hq_set_fields_device(self._h, ctypes.c_void_p(X.data_ptr())), "hq_set_fields_device")

    def get_fields(self, out=None):
        out = np.empty(self.field_shape) if out is None else out
        self._check(self.lib.hq_get_fields(self._h, _dptr(out)), "hq_get_fields")
        return out

    def sweep(self, n=1, local=True, global_=True, measure=True):
        """Raises HQError (code HQ_EUNSTABLE = -4) when the stabilisation back-off reached its floor;
        the sweeps have run and the chains are kept."""
        flags = (HQ_LOCAL if local else 0) | (HQ_GLOBAL if global_ else 0) | (HQ_MEASURE if measure else 0)
        self._check(self.lib.hq_sweep(self._h, int(n), flags), "hq_sweep")

    def log_weight(self):
        lw = np.empty(self.n_chains)
        ld = np.empty(self.n_chains)
        self._check(self.lib.hq_log_weight(self._h, _dptr(lw), _dptr(ld)), "hq_log_weight")
        return lw, ld

    def green(self, chain):
        G = np.empty((self.n_sites, self.n_sites))
        sl = ctypes.c_int()
        self._check(self.lib.hq_get_green(self._h, int(chain), _dptr(G), ctypes.byref(sl)), "hq_get_green")
        return G

    def observables(self):
        arr = (hq_obs * self.n_chains)()
        self._check(self.lib.hq_get_observables(self._h, arr), "hq_get_observables")
        return [{f: getattr(o, f) for f, _ in hq_obs._fields_} for o in arr]

    def series(self, obs_id):
        out = np.full((self.n_chains, max(self.max_series, 1)), np.nan)
        n = ctypes.c_int()
        self._check(self.lib.hq_get_series(self._h, int(obs_id), _dptr(out), ctypes.byref(n)), "hq_get_series")
        return out[:, :n.value]

    def checkpoint(self):
        n = ctypes.c_size_t()
        self._check(self.lib.hq_checkpoint(self._h, None, ctypes.byref(n)), "hq_checkpoint")
        buf = ctypes.create_string_buffer(n.value)
        self._check(self.lib.hq_checkpoint(self._h, buf, ctypes.byref(n)), "hq_checkpoint")
        return buf.raw[: n.value]

    def restore(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._check(self.lib.hq_restore(self._h, buf, len(blob)), "hq_restore")

    def set_graphs(self, enable=True):
        """Replay sweeps from a captured CUDA graph (needs a non-default stream)."""
        self._check(self.lib.hq_set_graphs(self._h, 1 if enable else 0), "hq_set_graphs")

    def set_timing(self, enable=True):
        self._check(self.lib.hq_set_timing(self._h, 1 if enable else 0), "hq_set_timing")

    def timing(self):
        """{phase: (milliseconds, launches)} accumulated since the last call."""
        ms = np.zeros(HQ_N_PHASES)
        n = (ctypes.c_int64 * HQ_N_PHASES)()
        self._check(self.lib.hq_get_timing(self._h, _dptr(ms), n), "hq_get_timing")
        return {PHASES[i]: (float(ms[i]), int(n[i])) for i in range(HQ_N_PHASES)}

    def set_chain(self, slot, X, seed, chain_id, sweep=0):
        """Load one slot: fields X [L][N], Philox key `seed`, chain word, sweep counter.  The
        fields go through a page-locked staging buffer so that the copy does not wait for
        kernels that other engines run on other streams."""
        import torch
        X = np.asarray(X, dtype=np.float64)
        if X.shape != self.field_shape[1:]:
            raise ValueError(f"fields must have shape {self.field_shape[1:]}")
        if getattr(self, "_stage", None) is None:
            self._stage = torch.empty(self.field_shape[1:], dtype=torch.float64, pin_memory=True)
        self._stage.numpy()[...] = X
        self._check(self.lib.hq_set_chain(self._h, int(slot), ctypes.cast(self._stage.data_ptr(), _dp), int(seed),
                                          int(chain_id), int(sweep)), "hq_set_chain")

    def set_active(self, slot, active):
        self._check(self.lib.hq_set_active(self._h, int(slot), 1 if active else 0), "hq_set_active")

    # ------------------------------------------------------------ learned moves
    def attach_network(self, max_batch=64, max_samples=4096):
        """Allocate (PyTorch) and attach the network state for training and cumulative moves."""
        import torch
        nb = self.lib.hq_nn_arena_bytes(self._h, int(max_batch), int(max_samples))
        if nb == 0:
            raise HQError("learned moves need nx, ny >= 4 and L >= 5")
        self.nn_arena = torch.empty(nb + 256, dtype=torch.uint8, device=self.arena.device)
        base = (self.nn_arena.data_ptr() + 255) // 256 * 256
        self._check(self.lib.hq_nn_attach(self._h, ctypes.c_void_p(base), nb, int(max_batch), int(max_samples)),
                    "hq_nn_attach")

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.size == HQ_NN_PARAMS
        self._check(self.lib.hq_nn_set_params(self._h, t.ctypes.data_as(_P(ctypes.c_float))), "hq_nn_set_params")

    def get_params(self, bf16=False):
        t = np.empty(HQ_NN_PARAMS, dtype=np.float32)
        self._check(self.lib.hq_nn_get_params(self._h, t.ctypes.data_as(_P(ctypes.c_float)), 1 if bf16 else 0),
                    "hq_nn_get_params")
        return t

    def nn_eval(self):
        F = np.empty(self.n_chains)
        self._check(self.lib.hq_nn_eval(self._h, _dptr(F)), "hq_nn_eval")
        return F

    def nn_gradient(self, X, y):
        """X: CUDA float64 [n][L][N], y: CUDA float64 [n]; returns (grad, loss)."""
        g = np.empty(HQ_NN_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self.lib.hq_nn_gradient(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                            int(X.shape[0]), g.ctypes.data_as(_P(ctypes.c_float)),
                                            ctypes.byref(loss)), "hq_nn_gradient")
        return g, loss.value

    def nn_train(self, X, y, epochs, batch, lr, seed=1):
        losses = np.empty(max(int(epochs), 1))
        self._check(self.lib.hq_nn_train(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                         int(X.shape[0]), int(epochs), int(batch), float(lr), int(seed),
                                         _dptr(losses)), "hq_nn_train")
        return losses[: int(epochs)]

    def cumulative(self, n_steps=1, n_inner=1, local=True, global_=True, measure=False, cnn=False):
        """Cumulative steps; cnn=True drives block moves by the convolutional action."""
        flags = ((HQ_LOCAL if local else 0) | (HQ_GLOBAL if global_ else 0) | (HQ_MEASURE if measure else 0)
                 | (HQ_CNN_BLOCK if cnn else 0))
        self._check(self.lib.hq_cumulative_sweep(self._h, int(n_steps), int(n_inner), flags), "hq_cumulative_sweep")

    def set_inner_window(self, slices):
        """Local moves of each cumulative step on `slices` consecutive slices (0: all)."""
        self._check(self.lib.hq_set_inner_window(self._h, int(slices)), "hq_set_inner_window")

    def set_block_sites(self, sites):
        """Block moves of each plain sweep on a run of `sites` consecutive sites (0: all)."""
        self._check(self.lib.hq_set_block_sites(self._h, int(sites)), "hq_set_block_sites")

    def set_logdet_split(self, mode):
        """Exact log|det M| of cumulative steps: 0 automatic, 1 one CTA per chain (G_0), 2 two
        halves joined at a boundary m (G_m).  Returns m (0 when not split)."""
        rc = self.lib.hq_set_logdet_split(self._h, int(mode))
        if rc < 0:
            self._check(rc, "hq_set_logdet_split")
        return int(rc)

    def set_inner_sites(self, sites):
        """Block moves of each cumulative step on `sites` consecutive sites (0: all)."""
        self._check(self.lib.hq_set_inner_sites(self._h, int(sites)), "hq_set_inner_sites")

    # convolutional action (block moves)
    def cnn_set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.size == HQ_CNN_PARAMS
        self._check(self.lib.hq_cnn_set_params(self._h, t.ctypes.data_as(_P(ctypes.c_float))), "hq_cnn_set_params")

    def cnn_get_params(self, bf16=False):
        t = np.empty(HQ_CNN_PARAMS, dtype=np.float32)
        self._check(self.lib.hq_cnn_get_params(self._h, t.ctypes.data_as(_P(ctypes.c_float)), 1 if bf16 else 0),
                    "hq_cnn_get_params")
        return t

    def cnn_eval(self):
        F = np.empty(self.n_chains)
        self._check(self.lib.hq_cnn_eval(self._h, _dptr(F)), "hq_cnn_eval")
        return F

    def cnn_gradient(self, X, y):
        """X: CUDA float64 [n][L][N], y: CUDA float64 [n]; returns (grad, loss)."""
        g = np.empty(HQ_CNN_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self.lib.hq_cnn_gradient(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                             int(X.shape[0]), g.ctypes.data_as(_P(ctypes.c_float)),
                                             ctypes.byref(loss)), "hq_cnn_gradient")
        return g, loss.value

    def cnn_train(self, X, y, epochs, batch, lr, seed=1):
        losses = np.empty(max(int(epochs), 1))
        self._check(self.lib.hq_cnn_train(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                          int(X.shape[0]), int(epochs), int(batch), float(lr), int(seed),
                                          _dptr(losses)), "hq_cnn_train")
        return losses[: int(epochs)]

    def learned_stats(self):
        arr = (hq_learned_stats * self.n_chains)()
        self._check(self.lib.hq_get_learned_stats(self._h, arr), "hq_get_learned_stats")
        return [{f: getattr(o, f) for f, _ in hq_learned_stats._fields_} for o in arr]

    @property
    def block_move_method(self):
        """0: separable slice applications per move; 1: chunk propagators."""
        return int(self.lib.hq_block_move_method(self._h))

    @property
    def sweeps_done(self):
        s = ctypes.c_int64()
        self.lib.hq_shape(self._h, None, None, None, ctypes.byref(s))
        return s.value


class Group:
    """Engines of different shapes swept together by one persistent launch per sweep; thin
    wrapper of hq_group_*."""

    def __init__(self, engines, stream=None):
        import torch
        self.lib = load_library()
        self.engines = list(engines)
        self._arr = (_vp * len(self.engines))(*[e._h.value for e in self.engines])
        nb = int(self.lib.hq_group_arena_bytes(self._arr, len(self.engines)))
        if nb == 0:
            raise HQError("invalid engine group")
        dev = self.engines[0].arena.device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self.arena = torch.empty(nb + 256, dtype=torch.uint8, device=dev)
        base = (self.arena.data_ptr() + 255) // 256 * 256
        self._h = ctypes.c_void_p()
        rc = self.lib.hq_group_create(self._arr, len(self.engines), ctypes.c_void_p(base), nb,
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._h))
        if rc != HQ_OK:
            raise HQError(f"hq_group_create failed ({rc})")

    def sweep(self, n=1, local=True, global_=True, measure=True):
        flags = (HQ_LOCAL if local else 0) | (HQ_GLOBAL if global_ else 0) | (HQ_MEASURE if measure else 0)
        rc = self.lib.hq_group_sweep(self._h, int(n), flags)
        if rc != HQ_OK:
            raise HQError(f"hq_group_sweep failed ({rc})")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.hq_group_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_SCRATCH_BYTES = 64 << 20


def logdet_noalloc(params, X, out, stream=None):
    """hq_logdet_noalloc on caller-owned CUDA tensors: X float64 [chains][L][N], out float64
    [chains].  The library allocates nothing; its static scratch is shared by all calls.
    The tensors are checked here (dtype, shape, device, layout) before the library sees their
    addresses, since the kernel trusts the sizes it is given."""
    import torch
    L, N = int(round(params.beta / params.dtau)), params.nx * params.ny
    if X.dtype != torch.float64 or out.dtype != torch.float64:
        raise TypeError("X and out must be float64 tensors")
    if X.dim() != 3 or tuple(X.shape[1:]) != (L, N) or X.shape[0] < 1:
        raise ValueError(f"X must have shape [chains][{L}][{N}] for these parameters, got {tuple(X.shape)}")
    if out.numel() < X.shape[0]:
        raise ValueError(f"out holds {out.numel()} values, {X.shape[0]} chains need as many")
    if not (X.is_cuda and out.is_cuda) or X.device != out.device:
        raise ValueError("X and out must be CUDA tensors on the same device")
    if not (X.is_contiguous() and out.is_contiguous()):
        raise ValueError("X and out must be contiguous")
    lib = load_library()
    rc = lib.hq_logdet_noalloc(ctypes.byref(make_params(params)), int(X.shape[0]), ctypes.c_void_p(X.data_ptr()),
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream or 0))
    if rc != HQ_OK:
        msg = lib.hq_last_error(None)
        raise HQError(f"hq_logdet_noalloc failed ({rc}): {msg.decode() if msg else ''}")


def proposal_uniforms(seed, chain, sweep, events, tag, stream=None):
    lib = load_library()
    ev = np.ascontiguousarray(events, dtype=np.uint32)
    u1 = np.empty(ev.size)
    u2 = np.empty(ev.size)
    rc = lib.hq_proposal_uniforms(int(seed), int(chain), int(sweep), int(tag), ev.ctypes.data_as(_P(ctypes.c_uint32)),
                                  ev.size, _dptr(u1), _dptr(u2), ctypes.c_void_p(stream or 0))
    if rc != HQ_OK:
        raise HQError(f"hq_proposal_uniforms failed ({rc})")
    return u1, u2


def autotune(params, X, ks=(4, 8, 16, 32), methods=(1, 2), local=True, global_=True, warmup=1, reps=2,
             stream=None):
    """Time every (delay rank, block-move method) pair on the fields X (CUDA float64
    [chains][L][N]); returns ({(k, method): ms per sweep}, best_k, best_method)."""
    import torch
    lib = load_library()
    prm = make_params(params)
    C = int(X.shape[0])
    karr = (ctypes.c_int * len(ks))(*ks)
    marr = (ctypes.c_int * len(methods))(*methods)
    nb = int(lib.hq_autotune_arena_bytes(ctypes.byref(prm), C, karr, len(ks)))
    if nb == 0:
        raise HQError("invalid autotune parameters")
    arena = torch.empty(nb + 256, dtype=torch.uint8, device=X.device)
    base = (arena.data_ptr() + 255) // 256 * 256
    st = stream if stream is not None else torch.cuda.current_stream(X.device)
    ms = np.zeros(len(ks) * len(methods))
    bk, bm = ctypes.c_int(), ctypes.c_int()
    flags = (HQ_LOCAL if local else 0) | (HQ_GLOBAL if global_ else 0)
    rc = lib.hq_autotune(ctypes.byref(prm), C, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(base), nb,
                         ctypes.c_void_p(st.cuda_stream), karr, len(ks), marr, len(methods), flags, int(warmup),
                         int(reps), _dptr(ms), ctypes.byref(bk), ctypes.byref(bm))
    if rc != HQ_OK:
        raise HQError(f"hq_autotune failed ({rc})")
    table = {(k, m): float(ms[a * len(methods) + b]) for a, k in enumerate(ks) for b, m in enumerate(methods)}
    return table, bk.value, bm.value


def init_network(seed, out_scale=1.0):
    """Seeded He initialisation of the patch network in the flat layout of hq_nn_set_params:
    W1[25][64], b1[64], W2[64][64], b2[64], W3[64], b3 (biases zero, W3 ~ 0.01 N(0,1) scaled
    by out_scale)."""
    rng = np.random.default_rng(seed)
    w1 = rng.standard_normal((25, 64)) * math.sqrt(2.0 / 25)
    w2 = rng.standard_normal((64, 64)) * math.sqrt(2.0 / 64)
    w3 = rng.standard_normal(64) * 0.01 * out_scale
    out = np.concatenate([w1.ravel(), np.zeros(64), w2.ravel(), np.zeros(64), w3, [0.0]]).astype(np.float32)
    assert out.size == HQ_NN_PARAMS
    return out


def init_cnn(seed, out_scale=1.0):
    """Seeded He initialisation of the convolutional action in the flat layout of
    hq_cnn_set_params: W1[27][16], b1[16], W2[27][16][16], b2[16], W3[27][16], b3 (biases
    zero, the last layer 0.01 N(0,1) scaled by out_scale)."""
    rng = np.random.default_rng(seed)
    w1 = rng.standard_normal((27, 16)) * math.sqrt(2.0 / 27)
    w2 = rng.standard_normal((27, 16, 16)) * math.sqrt(2.0 / (27 * 16))
    w3 = rng.standard_normal((27, 16)) * 0.01 * out_scale
    out = np.concatenate([w1.ravel(), np.zeros(16), w2.ravel(), np.zeros(16), w3.ravel(), [0.0]]).astype(np.float32)
    assert out.size == HQ_CNN_PARAMS
    return out


def tau_int(series, c=6.0):
    lib = load_library()
    x = np.ascontiguousarray(series, dtype=np.float64)
    w = ctypes.c_int()
    t = lib.hq_tau_int(_dptr(x), x.size, float(c), ctypes.byref(w))
    return float(t), w.value


SECTIONS = ("dl", "kin", "prepivot", "qr", "form_q", "t_update", "logdet", "move", "wait", "prop_prep",
            "prop_seq", "wrap", "restab_prod", "restab_qr", "restab_green", "measure", "flush")


def wait_probe(limit_seconds=0.05, stream=None):
    """Run the library's bounded device wait on a flag nothing sets; returns the kernel's
    status (HQ_ETIMEOUT when the wait ran out)."""
    lib = load_library()
    st = ctypes.c_int()
    rc = lib.hq_wait_probe(float(limit_seconds), ctypes.c_void_p(stream), ctypes.byref(st))
    if rc != HQ_OK:
        raise HQError(f"hq_wait_probe failed ({rc})")
    return st.value


def section_cycles():
    """{section: cycles} from a -DHQ_SECTION_TIMING build (empty otherwise); clears them."""
    out = (ctypes.c_uint64 * len(SECTIONS))()
    n = load_library().hq_get_section_cycles(out, len(SECTIONS))
    if n < 0:
        raise HQError(f"hq_get_section_cycles failed ({n})")
    return {SECTIONS[i]: int(out[i]) for i in range(n)}


HQ_PROBE_DFMA = 0
HQ_PROBE_DMMA = 1


def fp64_peak_tflops(reps=20, stream=None, kind=HQ_PROBE_DFMA):
    return float(load_library().hq_fp64_peak_tflops(int(kind), int(reps), ctypes.c_void_p(stream or 0)))
