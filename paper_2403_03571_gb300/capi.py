"""Thin ctypes binding of libapd.so (include/apd.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Functions keep the C names; array arguments are
torch CUDA tensors (device memory) and streams are torch CUDA streams.
Loading fails loudly when the library is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libapd.so")

APD_OK = 0
APD_NOT_CONVERGED = 1
APD_WARN_TOL_INFEASIBLE = 2
APD_ERR_ARG = -1
APD_ERR_NOT_SPD = -2
APD_ERR_CUDA = -3
APD_ERR_WORKSPACE = -4
APD_ERR_TIMEOUT = -5
APD_ERR_UNSUPPORTED = -6

APD_FP32 = 0
APD_TC_BF16 = 1
APD_TC_TF32 = 2

# every symbol include/apd.h declares
EXPORTED = (
    "apd_workspace_create", "apd_workspace_destroy", "apd_workspace_status", "apd_last_stats",
    "apd_assign", "apd_cell_moments", "apd_dual_value_grad", "apd_solve_opts_default",
    "apd_solve_weights", "apd_lloyd_step", "apd_lloyd", "apd_choose_resolution",
    "apd_status_string", "apd_version", "apd_profile_enable", "apd_profile_read",
    "apd_cell_moments_noalloc", "apd_tensor_core_check",
    "apd_batch_create", "apd_batch_destroy", "apd_batch_tile_info", "apd_batch_kernel_launches",
    "apd_batch_cell_moments", "apd_batch_solve_weights", "apd_batch_solve_weights_judged",
    "apd_warmstart_sizes", "apd_warmstart_create", "apd_warmstart_destroy", "apd_warmstart_get",
    "apd_warmstart_features", "apd_warmstart_fit_norm", "apd_warmstart_predict",
    "apd_warmstart_train_step", "apd_solve_weights_warm",
    "apd_multires_opts_default", "apd_solve_weights_multires", "apd_batch_solve_weights_multires",
    "apd_warmstart_train_step_pairs", "apd_workspace_set_pruning", "apd_batch_set_pruning",
    "apd_profile_read_scored", "apd_lloyd_multires", "apd_refine_opts_default", "apd_solve_weights_refine",
    "apd_points_moments", "apd_points_dual_value_grad", "apd_refine_next_grid",
    "apd_masked_moments", "apd_masked_dual_value_grad", "apd_workspace_set_wait_limit",
    "apd_shard_range", "apd_cell_moments_slab", "apd_workspace_set_shard", "apd_lbfgs_check",
    "apd_workspace_set_graphs",
    "apd_workspace_set_incremental",
)


class ApdGrid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("res", ctypes.c_int32 * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class ApdSeeds(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("x", ctypes.c_void_p), ("A", ctypes.c_void_p),
                ("w", ctypes.c_void_p)]


class ApdEvalStats(ctypes.Structure):
    _fields_ = [("pixels", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("rescored_fp64", ctypes.c_int64)]


class ApdSolveOpts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("max_evals", ctypes.c_int32),
                ("history", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("check_volumes", ctypes.c_int32)]


class ApdSolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("evaluations", ctypes.c_int32), ("solves", ctypes.c_int32),
                ("max_rel_err", ctypes.c_double), ("g", ctypes.c_double),
                ("rescored_fp64", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("coarse_evaluations", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# int (*)(void *ctx, int64_t *moments, int64_t words, const apd_seeds *seeds, cudaStream_t stream)
REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                             ctypes.POINTER(ApdSeeds), ctypes.c_void_p)


class ApdMultiresOpts(ctypes.Structure):
    _fields_ = [("factor", ctypes.c_int32), ("coarse_eps", ctypes.c_double),
                ("coarse_max_evals", ctypes.c_int32), ("carry_history", ctypes.c_int32),
                ("min_cell_span", ctypes.c_int32), ("coarse_stall_evals", ctypes.c_int32)]


class ApdRefineOpts(ctypes.Structure):
    _fields_ = [("growth", ctypes.c_double), ("max_res", ctypes.c_int32 * 3), ("max_rounds", ctypes.c_int32)]


class ApdPoints(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("count", ctypes.c_int64), ("y", ctypes.c_void_p),
                ("mass", ctypes.c_void_p)]


class ApdError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: status {code} ({status_string(code)})")


_lib = None
_P = ctypes.POINTER
_vp = ctypes.c_void_p


def load(path: Optional[str] = None):
    """Load libapd.so (built by ``paper_2403_03571_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libapd.so not found at {path}; run paper_2403_03571_gb300.build.build()")
    L = ctypes.CDLL(path)
    L.apd_workspace_create.argtypes = [_P(_vp), ctypes.c_int32, ctypes.c_int32, ctypes.c_int64]
    L.apd_workspace_destroy.argtypes = [_vp]
    L.apd_workspace_destroy.restype = None
    L.apd_workspace_status.argtypes = [_vp, _vp]
    L.apd_last_stats.argtypes = [_vp, _P(ApdEvalStats), _vp]
    L.apd_assign.argtypes = [_P(ApdGrid), _P(ApdSeeds), ctypes.c_int32, _vp, _vp, _vp, _vp]
    L.apd_workspace_set_wait_limit.argtypes = [_vp, ctypes.c_int64]
    L.apd_workspace_set_graphs.argtypes = [_vp, ctypes.c_int32]
    L.apd_workspace_set_incremental.argtypes = [_vp, ctypes.c_int32]
    L.apd_shard_range.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_int32),
                                  _P(ctypes.c_int32)]
    L.apd_cell_moments_slab.argtypes = [_P(ApdGrid), ctypes.c_int32, ctypes.c_int32, _P(ApdSeeds), ctypes.c_int32,
                                        _vp, _vp, _vp]
    L.apd_workspace_set_shard.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, REDUCE_FN, _vp]
    L.apd_cell_moments.argtypes = [_P(ApdGrid), _P(ApdSeeds), ctypes.c_int32, _vp, _vp, _vp]
    L.apd_dual_value_grad.argtypes = [_P(ApdGrid), _P(ApdSeeds), _vp, ctypes.c_int32, _vp, _vp, _vp,
                                      _vp, _vp]
    L.apd_solve_opts_default.argtypes = [_P(ApdSolveOpts)]
    L.apd_solve_opts_default.restype = None
    L.apd_solve_weights.argtypes = [_P(ApdGrid), _P(ApdSeeds), _vp, _vp, _P(ApdSolveOpts),
                                    _P(ApdSolveInfo), _vp, _vp]
    L.apd_lloyd_step.argtypes = [_P(ApdGrid), _P(ApdSeeds), _vp, _vp, _vp, _P(ApdSolveOpts),
                                 _P(ApdSolveInfo), _vp, _vp]
    L.apd_lloyd.argtypes = [_P(ApdGrid), _P(ApdSeeds), _vp, ctypes.c_int32, _vp, _vp,
                            _P(ApdSolveOpts), _P(ApdSolveInfo), _vp, _vp]
    L.apd_choose_resolution.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double]
    L.apd_choose_resolution.restype = ctypes.c_int64
    L.apd_status_string.argtypes = [ctypes.c_int]
    L.apd_status_string.restype = ctypes.c_char_p
    L.apd_version.restype = ctypes.c_int32
    L.apd_profile_enable.argtypes = [_vp, ctypes.c_int32]
    L.apd_cell_moments_noalloc.argtypes = [_P(ApdGrid), _P(ApdSeeds), _vp, _vp]
    L.apd_tensor_core_check.argtypes = [ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_int32),
                                        _P(ctypes.c_float)]
    L.apd_lbfgs_check.argtypes = [ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, ctypes.c_int32, _vp,
                                  _P(ctypes.c_double)]
    L.apd_profile_read.argtypes = [_vp, _P(ctypes.c_double), _P(ctypes.c_int64), _P(ctypes.c_int64),
                                   _P(ctypes.c_int64)]
    L.apd_batch_create.argtypes = [_P(_vp), ctypes.c_int32, ctypes.c_int32, _P(ApdGrid),
                                   _P(ctypes.c_int32), ctypes.c_int32]
    L.apd_batch_destroy.argtypes = [_vp]
    L.apd_batch_destroy.restype = None
    L.apd_batch_tile_info.argtypes = [_vp, _P(ctypes.c_int32), _P(ctypes.c_int32),
                                      _P(ctypes.c_double), _P(ctypes.c_int32)]
    L.apd_batch_kernel_launches.argtypes = [_vp]
    L.apd_batch_kernel_launches.restype = ctypes.c_int64
    L.apd_batch_cell_moments.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    L.apd_batch_solve_weights.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _P(ApdSolveOpts),
                                          _P(ApdSolveInfo), _vp]
    L.apd_batch_solve_weights_judged.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _P(ApdSolveOpts),
                                                 _P(ApdSolveInfo), _P(ctypes.c_int32), _vp]
    L.apd_warmstart_sizes.argtypes = [ctypes.c_int32, _P(ctypes.c_int32), _P(ctypes.c_int32)]
    L.apd_warmstart_create.argtypes = [_P(_vp), ctypes.c_int32, _P(ctypes.c_float), _P(ctypes.c_float)]
    L.apd_warmstart_destroy.argtypes = [_vp]
    L.apd_warmstart_destroy.restype = None
    L.apd_warmstart_get.argtypes = [_vp, _P(ctypes.c_float), _P(ctypes.c_float)]
    L.apd_warmstart_features.argtypes = [_vp, ctypes.c_int32, _P(ctypes.c_int64), _P(ctypes.c_double),
                                         _vp, _vp, _vp, _vp, _vp, _vp]
    L.apd_warmstart_train_step_pairs.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp,
                                                 ctypes.c_float, ctypes.c_float, _vp, _vp, _vp]
    L.apd_warmstart_fit_norm.argtypes = [_vp, ctypes.c_int64, _vp, _vp]
    L.apd_warmstart_predict.argtypes = [_vp, ctypes.c_int32, _P(ctypes.c_int64), _P(ctypes.c_double),
                                        _vp, _vp, _vp]
    L.apd_warmstart_train_step.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp, ctypes.c_float, _vp, _vp,
                                           _vp]
    L.apd_solve_weights_warm.argtypes = [_P(ApdGrid), _P(ApdSeeds), _vp, _vp, _P(ApdSolveOpts),
                                         _P(ApdSolveInfo), _vp, _vp, _P(ctypes.c_int32), _vp]
    L.apd_multires_opts_default.argtypes = [_P(ApdMultiresOpts)]
    L.apd_multires_opts_default.restype = None
    L.apd_solve_weights_multires.argtypes = [_P(ApdGrid), _P(ApdSeeds), _vp, _vp, _P(ApdSolveOpts),
                                             _P(ApdMultiresOpts), _P(ApdSolveInfo), _vp, _vp,
                                             _P(ctypes.c_int32), _vp]
    L.apd_batch_solve_weights_multires.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _P(ApdSolveOpts),
                                                   _P(ApdMultiresOpts), ctypes.c_int32, _P(ApdSolveInfo),
                                                   _P(ctypes.c_int32), _vp]
    L.apd_workspace_set_pruning.argtypes = [_vp, ctypes.c_int32]
    L.apd_profile_read_scored.argtypes = [_vp, _P(ctypes.c_int64)]
    L.apd_lloyd_multires.argtypes = [_P(ApdGrid), _P(ApdSeeds), _vp, ctypes.c_int32, _vp, _vp, _P(ApdSolveOpts),
                                     _P(ApdMultiresOpts), _P(ApdSolveInfo), _vp, _vp, _P(ctypes.c_int32), _vp]
    L.apd_batch_set_pruning.argtypes = [_vp, ctypes.c_int32]
    L.apd_points_moments.argtypes = [_P(ApdPoints), _P(ApdSeeds), _vp, _vp, _vp, _vp]
    L.apd_points_dual_value_grad.argtypes = [_P(ApdPoints), _P(ApdSeeds), _vp, _vp, _vp, _vp, _vp, _vp]
    L.apd_masked_moments.argtypes = [_P(ApdGrid), ctypes.c_int32, _P(ApdSeeds), _vp, _vp, _vp, _vp, _vp]
    L.apd_masked_dual_value_grad.argtypes = [_P(ApdGrid), ctypes.c_int32, _P(ApdSeeds), _vp, _vp, _vp, _vp, _vp,
                                             _vp, _vp]
    L.apd_refine_next_grid.argtypes = [_P(ApdGrid), ctypes.c_double, ctypes.c_double, _P(ApdRefineOpts),
                                       ctypes.c_int64, _P(ApdGrid)]
    L.apd_refine_opts_default.argtypes = [_P(ApdRefineOpts)]
    L.apd_refine_opts_default.restype = None
    L.apd_solve_weights_refine.argtypes = [_P(ApdGrid), _P(ApdSeeds), _vp, _vp, _P(ApdSolveOpts),
                                           _P(ApdRefineOpts), _P(ApdSolveInfo), _P(ApdGrid), _vp, _vp]
    _lib = L
    return L


def status_string(code: int) -> str:
    return load().apd_status_string(int(code)).decode()


def make_grid(grid) -> ApdGrid:
    """ApdGrid from an object with dim, res, lo, hi (e.g. synth.Grid)."""
    g = ApdGrid()
    g.dim = grid.dim
    for d in range(3):
        g.res[d] = grid.res[d] if d < grid.dim else 1
        g.lo[d] = grid.lo[d] if d < grid.dim else 0.0
        g.hi[d] = grid.hi[d] if d < grid.dim else 1.0
    return g


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("arrays must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def make_seeds(x, A, w) -> ApdSeeds:
    s = ApdSeeds()
    s.n = int(x.shape[0])
    s.x, s.A, s.w = _ptr(x).value, _ptr(A).value, _ptr(w).value
    return s


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc, what, ok=(APD_OK,)):
    if rc not in ok:
        raise ApdError(rc, what)
    return rc


class Workspace:
    """Owns an apd_workspace (device scratch for one stream)."""

    def __init__(self, dim: int, max_n: int, max_j: int):
        L = load()
        h = ctypes.c_void_p()
        _check(L.apd_workspace_create(ctypes.byref(h), dim, int(max_n), int(max_j)),
               "apd_workspace_create")
        self.handle = h
        self.dim, self.max_n, self.max_j = dim, max_n, max_j

    def close(self):
        if self.handle:
            load().apd_workspace_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None) -> int:
        return load().apd_workspace_status(self.handle, _stream(stream))

    def set_pruning(self, enable: bool = True):
        _check(load().apd_workspace_set_pruning(self.handle, int(bool(enable))), "apd_workspace_set_pruning")

    def set_shard(self, rank: int, world: int, hook=None):
        """Score only rank's slab of every grid and sum the moments with ``hook`` (a
        REDUCE_FN, kept alive here); world == 1 restores whole-grid passes."""
        self._hook = hook
        _check(load().apd_workspace_set_shard(self.handle, int(rank), int(world),
                                              hook if hook is not None else REDUCE_FN(), None),
               "apd_workspace_set_shard")

    def set_wait_limit(self, polls: int = -1):
        """Poll limit of the FP32 scoring kernel's bounded waits (-1: the default)."""
        _check(load().apd_workspace_set_wait_limit(self.handle, int(polls)), "apd_workspace_set_wait_limit")

    def set_graphs(self, enable: bool = True):
        """Replay the weight solves' evaluations from captured CUDA graphs (default on)."""
        _check(load().apd_workspace_set_graphs(self.handle, int(bool(enable))), "apd_workspace_set_graphs")

    def set_incremental(self, mode=1):
        """Incremental evaluations in weight solves: 0 (or False) off, 1 (or True,
        the default) on grids of at least 2^20 pixels, 2 on every grid."""
        _check(load().apd_workspace_set_incremental(self.handle, int(mode)),
               "apd_workspace_set_incremental")

    def profile(self, enable: bool = True):
        _check(load().apd_profile_enable(self.handle, int(bool(enable))), "apd_profile_enable")

    def profile_read(self):
        """(summed scoring-kernel ms, scoring launches, pairs, all kernel launches) since
        the last read."""
        ms, n, pairs, kl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().apd_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(n),
                                       ctypes.byref(pairs), ctypes.byref(kl)), "apd_profile_read")
        return ms.value, n.value, pairs.value, kl.value

    def pairs_scored(self) -> int:
        """Pairs the FP32 scoring evaluated since the last call (resets the count)."""
        v = ctypes.c_int64()
        _check(load().apd_profile_read_scored(self.handle, ctypes.byref(v)), "apd_profile_read_scored")
        return v.value

    def last_stats(self, stream=None) -> ApdEvalStats:
        st = ApdEvalStats()
        _check(load().apd_last_stats(self.handle, ctypes.byref(st), _stream(stream)), "apd_last_stats")
        return st


def apd_assign(grid, x, A, w, labels, ws: Workspace, precision=APD_FP32, stream=None, tie_gap=None):
    """Labels (int32 [J]) and, when ``tie_gap`` (float64 [J]) is given, the relative
    gap of the two smallest FP64 costs of every pixel."""
    g, s = make_grid(grid), make_seeds(x, A, w)
    return _check(load().apd_assign(ctypes.byref(g), ctypes.byref(s), precision, _ptr(labels),
                                    _ptr(tie_gap), ws.handle, _stream(stream)), "apd_assign")


def apd_cell_moments(grid, x, A, w, moments, ws: Workspace, precision=APD_FP32, stream=None):
    g, s = make_grid(grid), make_seeds(x, A, w)
    return _check(load().apd_cell_moments(ctypes.byref(g), ctypes.byref(s), precision, _ptr(moments),
                                          ws.handle, _stream(stream)), "apd_cell_moments")


def apd_shard_range(res: int, rank: int, world: int):
    """(k_begin, k_count) of rank's contiguous slab of an axis of ``res`` pixels."""
    kb, kc = ctypes.c_int32(), ctypes.c_int32()
    _check(load().apd_shard_range(int(res), int(rank), int(world), ctypes.byref(kb), ctypes.byref(kc)),
           "apd_shard_range")
    return kb.value, kc.value


def apd_cell_moments_slab(grid, k_begin, k_count, x, A, w, moments, ws: Workspace, precision=APD_FP32,
                          stream=None):
    g, s = make_grid(grid), make_seeds(x, A, w)
    return _check(load().apd_cell_moments_slab(ctypes.byref(g), int(k_begin), int(k_count), ctypes.byref(s),
                                               precision, _ptr(moments), ws.handle, _stream(stream)),
                  "apd_cell_moments_slab")


def apd_dual_value_grad(grid, x, A, w, v, g_out, grad, err_out, ws: Workspace, precision=APD_FP32,
                        stream=None):
    g, s = make_grid(grid), make_seeds(x, A, w)
    return _check(load().apd_dual_value_grad(ctypes.byref(g), ctypes.byref(s), _ptr(v), precision,
                                             _ptr(g_out), _ptr(grad), _ptr(err_out), ws.handle,
                                             _stream(stream)), "apd_dual_value_grad")


def apd_cell_moments_noalloc(grid, x, A, w, moments, stream=None):
    """Per-cell moments without a workspace (static device scratch; for callers that
    cannot allocate device memory).  Returns the C status code unchanged."""
    g, s = make_grid(grid), make_seeds(x, A, w)
    return load().apd_cell_moments_noalloc(ctypes.byref(g), ctypes.byref(s), _ptr(moments),
                                           _stream(stream))


def apd_tensor_core_check(kind: int, variant: int = 0):
    """(status, mismatching elements, max abs error) of the tcgen05 self-check."""
    mm, err = ctypes.c_int32(), ctypes.c_float()
    rc = load().apd_tensor_core_check(int(kind), int(variant), ctypes.byref(mm), ctypes.byref(err))
    return rc, mm.value, err.value


def apd_lbfgs_check(S, Y, g, fused=False):
    """(status, p, <g, p>) of the L-BFGS direction self-check: S, Y float64
    [hist, n] (row k = pair k, newest last), g float64 [n]; host arrays.  fused:
    the newest pair goes through the push kernel that also forms the direction
    (it then enters as y = g - (g - y), rounded on the device)."""
    import numpy as np
    S = np.ascontiguousarray(S, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    hist, n = S.shape
    p = np.empty(n, dtype=np.float64)
    gp = ctypes.c_double()
    rc = load().apd_lbfgs_check(int(n), int(hist), S.ctypes.data, Y.ctypes.data, g.ctypes.data, int(bool(fused)),
                                p.ctypes.data, ctypes.byref(gp))
    return rc, p, gp.value


def solve_opts(eps=0.01, max_evals=1000, history=10, precision=APD_FP32, check_volumes=1):
    o = ApdSolveOpts()
    load().apd_solve_opts_default(ctypes.byref(o))
    o.eps, o.max_evals, o.history, o.precision, o.check_volumes = (
        eps, max_evals, history, precision, check_volumes)
    return o


_SOLVE_OK = (APD_OK, APD_NOT_CONVERGED, APD_WARN_TOL_INFEASIBLE)


def apd_solve_weights(grid, x, A, w0, v, w_out, ws: Workspace, opts=None, stream=None):
    g, s = make_grid(grid), make_seeds(x, A, w0)
    info = ApdSolveInfo()
    opts = opts or solve_opts()
    rc = load().apd_solve_weights(ctypes.byref(g), ctypes.byref(s), _ptr(v), _ptr(w_out),
                                  ctypes.byref(opts), ctypes.byref(info), ws.handle, _stream(stream))
    _check(rc, "apd_solve_weights", _SOLVE_OK)
    return rc, info


def apd_lloyd_step(grid, x, A, w0, v, x_out, w_out, ws: Workspace, opts=None, stream=None):
    g, s = make_grid(grid), make_seeds(x, A, w0)
    info = ApdSolveInfo()
    opts = opts or solve_opts()
    rc = load().apd_lloyd_step(ctypes.byref(g), ctypes.byref(s), _ptr(v), _ptr(x_out), _ptr(w_out),
                               ctypes.byref(opts), ctypes.byref(info), ws.handle, _stream(stream))
    _check(rc, "apd_lloyd_step", _SOLVE_OK)
    return rc, info


def apd_lloyd(grid, x0, A, w0, v, rounds, x_out, w_out, ws: Workspace, opts=None, stream=None):
    g, s = make_grid(grid), make_seeds(x0, A, w0)
    info = ApdSolveInfo()
    opts = opts or solve_opts()
    rc = load().apd_lloyd(ctypes.byref(g), ctypes.byref(s), _ptr(v), int(rounds), _ptr(x_out),
                          _ptr(w_out), ctypes.byref(opts), ctypes.byref(info), ws.handle,
                          _stream(stream))
    _check(rc, "apd_lloyd", _SOLVE_OK)
    return rc, info


def apd_choose_resolution(dim, v_min, eps=0.01, domain_measure=1.0) -> int:
    return int(load().apd_choose_resolution(dim, v_min, eps, domain_measure))


class Batch:
    """Owns an apd_batch: `count` independent instances (grids[b], n[b] seeds) whose
    seed arrays are concatenated in instance order."""

    def __init__(self, dim: int, grids, n, tile: int = -1):
        L = load()
        self.dim = int(dim)
        self.count = len(grids)
        self.n = [int(k) for k in n]
        arr = (ApdGrid * self.count)(*[make_grid(g) for g in grids])
        nn = (ctypes.c_int32 * self.count)(*self.n)
        h = ctypes.c_void_p()
        _check(L.apd_batch_create(ctypes.byref(h), self.dim, self.count, arr, nn, int(tile)),
               "apd_batch_create")
        self.handle = h

    def close(self):
        if self.handle:
            load().apd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tile_info(self):
        """(chosen variant or -1, [ms per variant], [(P, TY, TZ) per variant])."""
        L = load()
        t, nv = ctypes.c_int32(), ctypes.c_int32()
        _check(L.apd_batch_tile_info(self.handle, ctypes.byref(t), ctypes.byref(nv), None, None),
               "apd_batch_tile_info")
        ms = (ctypes.c_double * nv.value)()
        sh = (ctypes.c_int32 * (3 * nv.value))()
        _check(L.apd_batch_tile_info(self.handle, ctypes.byref(t), ctypes.byref(nv), ms, sh),
               "apd_batch_tile_info")
        return t.value, list(ms), [tuple(sh[3 * k:3 * k + 3]) for k in range(nv.value)]

    def kernel_launches(self) -> int:
        return int(load().apd_batch_kernel_launches(self.handle))

    def set_pruning(self, enable: bool = True):
        _check(load().apd_batch_set_pruning(self.handle, int(bool(enable))), "apd_batch_set_pruning")


def apd_batch_cell_moments(batch: Batch, x, A, w, moments, stream=None):
    """Moments of every instance at weights w (concatenated); returns the C status."""
    return load().apd_batch_cell_moments(batch.handle, _ptr(x), _ptr(A), _ptr(w), _ptr(moments),
                                         _stream(stream))


def apd_batch_solve_weights(batch: Batch, x, A, w0, v, w_out, opts=None, stream=None):
    """Algorithm 2 for every instance; returns (C status, [ApdSolveInfo per instance]).
    The status is not raised: per-instance errors are in each info's status."""
    info = (ApdSolveInfo * batch.count)()
    opts = opts or solve_opts()
    rc = load().apd_batch_solve_weights(batch.handle, _ptr(x), _ptr(A), _ptr(w0), _ptr(v),
                                        _ptr(w_out), ctypes.byref(opts), info, _stream(stream))
    return rc, list(info)


def apd_batch_solve_weights_judged(batch: Batch, x, A, w_pred, v, w_out, opts=None, stream=None):
    """Batched solve from predicted weights, each instance judged against W = 0;
    returns (C status, [ApdSolveInfo], [1 where the prediction was kept])."""
    info = (ApdSolveInfo * batch.count)()
    used = (ctypes.c_int32 * batch.count)()
    opts = opts or solve_opts()
    rc = load().apd_batch_solve_weights_judged(batch.handle, _ptr(x), _ptr(A), _ptr(w_pred), _ptr(v),
                                               _ptr(w_out), ctypes.byref(opts), info, used,
                                               _stream(stream))
    return rc, list(info), list(used)


def warmstart_sizes(dim: int):
    """(features per seed, network parameters) for dimension dim."""
    f, p = ctypes.c_int32(), ctypes.c_int32()
    _check(load().apd_warmstart_sizes(int(dim), ctypes.byref(f), ctypes.byref(p)), "apd_warmstart_sizes")
    return f.value, p.value


def _boxes(grids):
    """[count][6] float64 boxes (lo[3], hi[3]) of synth.Grid-like objects."""
    import numpy as np
    out = np.zeros((len(grids), 6))
    out[:, 3:] = 1.0
    for b, g in enumerate(grids):
        gg = make_grid(g)
        for a in range(gg.dim):
            out[b, a], out[b, 3 + a] = gg.lo[a], gg.hi[a]
    return np.ascontiguousarray(out)


def _offsets(counts):
    import numpy as np
    offs = np.zeros(len(counts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(np.asarray(counts, dtype=np.int64))
    return offs


class WarmStart:
    """Owns an apd_mlp (the warm-start network on the device)."""

    def __init__(self, dim: int, params, norm=None):
        import numpy as np
        L = load()
        self.dim = int(dim)
        self.n_features, self.n_params = warmstart_sizes(dim)
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (self.n_params,):
            raise ValueError(f"expected {self.n_params} parameters, got {p.shape}")
        nz = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        if nz is not None and nz.shape != (2 * self.n_features,):
            raise ValueError("norm must hold mean and inverse std per feature")
        h = ctypes.c_void_p()
        fp = ctypes.POINTER(ctypes.c_float)
        _check(L.apd_warmstart_create(ctypes.byref(h), self.dim, p.ctypes.data_as(fp),
                                      None if nz is None else nz.ctypes.data_as(fp)), "apd_warmstart_create")
        self.handle = h

    def close(self):
        if self.handle:
            load().apd_warmstart_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self):
        """(params, norm) as float32 numpy arrays."""
        import numpy as np
        p = np.zeros(self.n_params, dtype=np.float32)
        nz = np.zeros(2 * self.n_features, dtype=np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        _check(load().apd_warmstart_get(self.handle, p.ctypes.data_as(fp), nz.ctypes.data_as(fp)),
               "apd_warmstart_get")
        return p, nz

    def features(self, counts, grids, x, A, v, out, knn=None, stream=None):
        """Features of every seed of the instances (counts[b] seeds on grids[b]'s box);
        knn (int32 [N][8], optional) receives the neighbour rows."""
        offs = _offsets(counts)
        m = _boxes(grids)
        return _check(load().apd_warmstart_features(
            self.handle, len(counts), offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(x), _ptr(A), _ptr(v), _ptr(out),
            _ptr(knn), _stream(stream)), "apd_warmstart_features")

    def fit_norm(self, features, stream=None):
        return _check(load().apd_warmstart_fit_norm(self.handle, int(features.shape[0]), _ptr(features),
                                                    _stream(stream)), "apd_warmstart_fit_norm")

    def predict(self, counts, grids, features, w_out, stream=None):
        offs = _offsets(counts)
        m = _boxes(grids)
        return _check(load().apd_warmstart_predict(
            self.handle, len(counts), offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(features), _ptr(w_out),
            _stream(stream)), "apd_warmstart_predict")

    def train_step_pairs(self, idx, features, targets, knn, y_buf, dy_buf, lr, mu=0.0, grad_out=None,
                         loss_out=None, stream=None):
        return _check(load().apd_warmstart_train_step_pairs(
            self.handle, int(idx.shape[0]), _ptr(idx), _ptr(features), _ptr(targets), _ptr(knn), _ptr(y_buf),
            _ptr(dy_buf), float(mu), float(lr), _ptr(grad_out), _ptr(loss_out), _stream(stream)),
            "apd_warmstart_train_step_pairs")

    def train_step(self, idx, features, targets, lr, grad_out=None, loss_out=None, stream=None):
        return _check(load().apd_warmstart_train_step(self.handle, int(idx.shape[0]), _ptr(idx), _ptr(features),
                                                      _ptr(targets), float(lr), _ptr(grad_out), _ptr(loss_out),
                                                      _stream(stream)), "apd_warmstart_train_step")


def apd_solve_weights_warm(grid, x, A, v, w_out, ws: Workspace, net: WarmStart, opts=None, stream=None):
    """Single-instance solve from the network's prediction judged against W = 0;
    returns (status, ApdSolveInfo, used_prediction)."""
    g, s = make_grid(grid), make_seeds(x, A, v)
    info = ApdSolveInfo()
    used = ctypes.c_int32()
    opts = opts or solve_opts()
    rc = load().apd_solve_weights_warm(ctypes.byref(g), ctypes.byref(s), _ptr(v), _ptr(w_out),
                                       ctypes.byref(opts), ctypes.byref(info), ws.handle, net.handle,
                                       ctypes.byref(used), _stream(stream))
    _check(rc, "apd_solve_weights_warm", _SOLVE_OK)
    return rc, info, used.value


def multires_opts(factor=2, coarse_eps=0.05, coarse_max_evals=60, carry_history=False, min_cell_span=None,
                  coarse_stall_evals=None):
    m = ApdMultiresOpts()
    load().apd_multires_opts_default(ctypes.byref(m))
    m.factor, m.coarse_eps, m.coarse_max_evals = int(factor), float(coarse_eps), int(coarse_max_evals)
    m.carry_history = int(bool(carry_history))
    if min_cell_span is not None:
        m.min_cell_span = int(min_cell_span)
    if coarse_stall_evals is not None:
        m.coarse_stall_evals = int(coarse_stall_evals)
    return m


def apd_solve_weights_multires(grid, x, A, w0, v, w_out, ws: Workspace, opts=None, mopts=None,
                               net: Optional[WarmStart] = None, stream=None):
    """Coarse-to-fine solve (optionally from the network's judged prediction);
    returns (status, ApdSolveInfo, used_prediction)."""
    g, s = make_grid(grid), make_seeds(x, A, w0)
    info = ApdSolveInfo()
    used = ctypes.c_int32()
    opts = opts or solve_opts()
    mopts = mopts or multires_opts()
    rc = load().apd_solve_weights_multires(ctypes.byref(g), ctypes.byref(s), _ptr(v), _ptr(w_out),
                                           ctypes.byref(opts), ctypes.byref(mopts), ctypes.byref(info),
                                           ws.handle, net.handle if net is not None else None,
                                           ctypes.byref(used), _stream(stream))
    _check(rc, "apd_solve_weights_multires", _SOLVE_OK)
    return rc, info, used.value


def make_points(y, mass) -> ApdPoints:
    """ApdPoints over device tensors y [count, dim] and mass [count] (FP64, contiguous)."""
    p = ApdPoints()
    p.dim = int(y.shape[1])
    p.count = int(y.shape[0])
    p.y = _ptr(y)
    p.mass = _ptr(mass)
    return p


def apd_points_moments(y, mass, x, A, w, moments, ws: Workspace, labels=None, stream=None):
    """Labels (optional) and FP64 measure-weighted moments of arbitrary elements."""
    p, s = make_points(y, mass), make_seeds(x, A, w)
    _check(load().apd_points_moments(ctypes.byref(p), ctypes.byref(s), _ptr(moments), _ptr(labels), ws.handle,
                                     _stream(stream)), "apd_points_moments")


def apd_points_dual_value_grad(y, mass, x, A, w, v, g_out, grad, err_out, ws: Workspace, stream=None):
    """Eqs. (2.7)-(2.8) on arbitrary elements (device outputs)."""
    p, s = make_points(y, mass), make_seeds(x, A, w)
    _check(load().apd_points_dual_value_grad(ctypes.byref(p), ctypes.byref(s), _ptr(v), _ptr(g_out), _ptr(grad),
                                             _ptr(err_out), ws.handle, _stream(stream)),
           "apd_points_dual_value_grad")


def apd_masked_moments(grid, refine, x, A, w, moments, coarse_labels, ws: Workspace, refined=None, stream=None):
    """Masked two-level discretisation: Algorithm 1 on `grid`, boundary coarse
    pixels refined by `refine` per axis; integer moments of the fine grid into
    `moments`, coarse labels into `coarse_labels`, the count of fine pixels
    scored into `refined` (optional, int64 [1])."""
    g, s = make_grid(grid), make_seeds(x, A, w)
    _check(load().apd_masked_moments(ctypes.byref(g), int(refine), ctypes.byref(s), _ptr(moments),
                                     _ptr(coarse_labels), _ptr(refined), ws.handle, _stream(stream)),
           "apd_masked_moments")


def apd_masked_dual_value_grad(grid, refine, x, A, w, v, g_out, grad, err_out, coarse_labels, ws: Workspace,
                               stream=None):
    """Eqs. (2.7)-(2.8) on the fine grid of the masked discretisation (device outputs)."""
    g, s = make_grid(grid), make_seeds(x, A, w)
    _check(load().apd_masked_dual_value_grad(ctypes.byref(g), int(refine), ctypes.byref(s), _ptr(v), _ptr(g_out),
                                             _ptr(grad), _ptr(err_out), _ptr(coarse_labels), ws.handle,
                                             _stream(stream)), "apd_masked_dual_value_grad")


def refine_opts(growth=1.5, max_res=(0, 0, 0), max_rounds=4) -> ApdRefineOpts:
    r = ApdRefineOpts()
    r.growth = growth
    for d in range(3):
        r.max_res[d] = int(max_res[d]) if d < len(max_res) else 0
    r.max_rounds = max_rounds
    return r


def apd_solve_weights_refine(grid, x, A, w0, v, w_out, ws: Workspace, opts=None, ropts=None, stream=None):
    """Weight solve that refines the grid while the tolerance is out of reach
    (Algorithm 2, step 4); returns (status, ApdSolveInfo, final grid as a
    synth.Grid)."""
    from paper_2403_03571_gb300 import synth
    g, s = make_grid(grid), make_seeds(x, A, w0)
    info = ApdSolveInfo()
    out = ApdGrid()
    opts = opts or solve_opts()
    ropts = ropts or refine_opts()
    rc = load().apd_solve_weights_refine(ctypes.byref(g), ctypes.byref(s), _ptr(v), _ptr(w_out),
                                         ctypes.byref(opts), ctypes.byref(ropts), ctypes.byref(info),
                                         ctypes.byref(out), ws.handle, _stream(stream))
    _check(rc, "apd_solve_weights_refine", _SOLVE_OK)
    final = synth.Grid(grid.dim, tuple(out.res[d] for d in range(grid.dim)),
                       lo=tuple(out.lo[d] for d in range(grid.dim)), hi=tuple(out.hi[d] for d in range(grid.dim)))
    return rc, info, final


def apd_batch_solve_weights_multires(batch: Batch, x, A, w0, v, w_out, opts=None, mopts=None, judge=False,
                                     stream=None):
    """Batched coarse-to-fine solve; returns (C status, [ApdSolveInfo], [used prediction])."""
    info = (ApdSolveInfo * batch.count)()
    used = (ctypes.c_int32 * batch.count)()
    opts = opts or solve_opts()
    mopts = mopts or multires_opts()
    rc = load().apd_batch_solve_weights_multires(batch.handle, _ptr(x), _ptr(A), _ptr(w0), _ptr(v), _ptr(w_out),
                                                 ctypes.byref(opts), ctypes.byref(mopts), int(bool(judge)), info,
                                                 used, _stream(stream))
    return rc, list(info), list(used)


def apd_lloyd_multires(grid, x0, A, w0, v, rounds, x_out, w_out, ws: Workspace, opts=None, mopts=None,
                       net: Optional[WarmStart] = None, stream=None):
    """Algorithm 3 with coarse-to-fine solves; returns (status, ApdSolveInfo, used_prediction)."""
    g, s = make_grid(grid), make_seeds(x0, A, w0)
    info = ApdSolveInfo()
    used = ctypes.c_int32()
    opts = opts or solve_opts()
    mopts = mopts or multires_opts()
    rc = load().apd_lloyd_multires(ctypes.byref(g), ctypes.byref(s), _ptr(v), int(rounds), _ptr(x_out),
                                   _ptr(w_out), ctypes.byref(opts), ctypes.byref(mopts), ctypes.byref(info),
                                   ws.handle, net.handle if net is not None else None, ctypes.byref(used),
                                   _stream(stream))
    _check(rc, "apd_lloyd_multires", _SOLVE_OK)
    return rc, info, used.value
