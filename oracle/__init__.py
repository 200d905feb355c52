"""FP64 CPU oracle for anisotropic power diagrams (APDs).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library path never does.
It shares no code with the CUDA path: the brute-force core is plain C
(``apd_oracle.c``, FP64, no FMA contraction) and the solvers here are scipy's
L-BFGS-B plus plain numpy.

Functions and the passages they follow (arXiv 2403.03571):

* ``pixel_centres``            -- eq. (2.6), Section 2.3 (regular grid);
* ``assign`` / ``assign_ids``  -- Algorithm 1 (cost matrix, argmin; lowest index on ties);
* ``moments``                  -- per-cell counts and integer coordinate moments;
* ``moments_ids``              -- the same over a listed subset of pixels (a slab of the grid);
* ``dual_from_moments``        -- eq. (2.7) written through those moments (the form a
                                  sharded evaluation exchanges);
* ``dual``                     -- eqs. (2.7), (2.8) and the stop rule of Algorithm 2;
* ``solve_weights``            -- Algorithm 2 with a library L-BFGS (scipy L-BFGS-B);
* ``lbfgs_direction``          -- the limited-memory BFGS direction of Algorithm 2's ascent
                                  (the two-loop recursion of Nocedal and Wright, Numerical
                                  Optimization, 2nd ed., Algorithm 7.4);
* ``lloyd``                    -- Algorithm 3 (discrete centroids, warm-started weights);
* ``resolution_lower_bound``   -- eq. (2.9) / Table 1;
* ``resolution_practical``     -- eq. (2.10).

Submodules: ``points`` (non-uniform discretisation, Section 2.3), ``masked``
(the masked two-level grid of the Section 4 outlook), ``warmstart`` (features,
network and losses of the learned warm start).

Parity unpinned: iteration counts of ``solve_weights`` (the paper leaves the
L-BFGS details open); only its end state (volumes within tolerance) is pinned.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np

from . import build as _build

_lib = None

_c_i32p = ctypes.POINTER(ctypes.c_int32)
_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_assign.argtypes = [ctypes.c_int32, _c_dp, _c_dp, _c_i32p, ctypes.c_int32, _c_dp,
                                    _c_dp, _c_dp, _c_i32p, _c_dp, ctypes.c_int32]
        L.oracle_assign_ids.argtypes = [ctypes.c_int32, _c_dp, _c_dp, _c_i32p, ctypes.c_int32, _c_dp,
                                        _c_dp, _c_dp, _c_i64p, ctypes.c_int64, _c_i32p, _c_dp,
                                        ctypes.c_int32]
        L.oracle_moments.argtypes = [ctypes.c_int32, _c_i32p, ctypes.c_int32, _c_i32p, _c_i64p,
                                     ctypes.c_int32]
        L.oracle_moments_ids.argtypes = [ctypes.c_int32, _c_i32p, ctypes.c_int32, _c_i64p, ctypes.c_int64,
                                         _c_i32p, _c_i64p, ctypes.c_int32]
        L.oracle_dual_from_labels.argtypes = [ctypes.c_int32, _c_dp, _c_dp, _c_i32p, ctypes.c_int32,
                                              _c_dp, _c_dp, _c_dp, _c_dp, _c_i32p, _c_dp, _c_dp,
                                              _c_dp, _c_i64p, _c_dp, ctypes.c_int32]
        L.oracle_centroids.argtypes = [ctypes.c_int32, _c_dp, _c_dp, _c_i32p, ctypes.c_int32, _c_dp,
                                       _c_i32p, _c_dp, ctypes.c_int32]
        L.oracle_cost.argtypes = [ctypes.c_int32, _c_dp, _c_dp, _c_dp, ctypes.c_double]
        L.oracle_cost.restype = ctypes.c_double
        L.oracle_max_threads.restype = ctypes.c_int
        for f in (L.oracle_assign, L.oracle_assign_ids, L.oracle_moments, L.oracle_moments_ids,
                  L.oracle_dual_from_labels, L.oracle_centroids):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _grid_args(grid):
    lo = np.ascontiguousarray(grid.lo, dtype=np.float64)
    hi = np.ascontiguousarray(grid.hi, dtype=np.float64)
    res = np.ascontiguousarray(grid.res, dtype=np.int32)
    return lo, hi, res


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def grid_steps(grid) -> np.ndarray:
    return np.array([(h - l) / r for l, h, r in zip(grid.lo, grid.hi, grid.res)])


def pixel_volume(grid) -> float:
    P = 1.0
    for h in grid_steps(grid):
        P *= h
    return P


def pixel_centres(grid, ids: Optional[np.ndarray] = None) -> np.ndarray:
    """Centres lo + (k + 1/2) h of the given linear pixel ids (all when None), [n, D]."""
    J = grid.num_pixels
    ids = np.arange(J, dtype=np.int64) if ids is None else np.asarray(ids, dtype=np.int64)
    h = grid_steps(grid)
    out = np.empty((ids.shape[0], grid.dim))
    r = ids.copy()
    for d in range(grid.dim):
        k = r % grid.res[d]
        r //= grid.res[d]
        out[:, d] = grid.lo[d] + (k.astype(np.float64) + 0.5) * h[d]
    return out


def assign(grid, x, A, w, with_gap: bool = False, nthreads: int = 0):
    """Algorithm 1 over every pixel: labels int32 [J] (and relative gaps [J])."""
    x, A, w = _f64(x), _f64(A), _f64(w)
    n = x.shape[0]
    lo, hi, res = _grid_args(grid)
    labels = np.empty(grid.num_pixels, dtype=np.int32)
    gap = np.empty(grid.num_pixels) if with_gap else None
    rc = lib().oracle_assign(grid.dim, _p(lo, _c_dp), _p(hi, _c_dp), _p(res, _c_i32p), n,
                             _p(x, _c_dp), _p(A, _c_dp), _p(w, _c_dp), _p(labels, _c_i32p),
                             _p(gap, _c_dp), nthreads)
    _check(rc, "assign")
    return (labels, gap) if with_gap else labels


def assign_ids(grid, x, A, w, ids, with_gap: bool = False, nthreads: int = 0):
    """Algorithm 1 for the listed pixel ids only."""
    x, A, w = _f64(x), _f64(A), _f64(w)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    lo, hi, res = _grid_args(grid)
    labels = np.empty(ids.shape[0], dtype=np.int32)
    gap = np.empty(ids.shape[0]) if with_gap else None
    rc = lib().oracle_assign_ids(grid.dim, _p(lo, _c_dp), _p(hi, _c_dp), _p(res, _c_i32p),
                                 x.shape[0], _p(x, _c_dp), _p(A, _c_dp), _p(w, _c_dp),
                                 _p(ids, _c_i64p), ids.shape[0], _p(labels, _c_i32p),
                                 _p(gap, _c_dp), nthreads)
    _check(rc, "assign_ids")
    return (labels, gap) if with_gap else labels


def moment_width(dim: int) -> int:
    return 1 + dim + dim * (dim + 1) // 2


def moments(grid, labels, n: int, nthreads: int = 0) -> np.ndarray:
    """int64 [n, K]: count, sum of u = 2k+1 per axis, upper triangle of sum u u^T."""
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    res = np.ascontiguousarray(grid.res, dtype=np.int32)
    out = np.empty((n, moment_width(grid.dim)), dtype=np.int64)
    rc = lib().oracle_moments(grid.dim, _p(res, _c_i32p), n, _p(labels, _c_i32p),
                              _p(out, _c_i64p), nthreads)
    _check(rc, "moments")
    return out


def moments_ids(grid, ids, labels, n: int, nthreads: int = 0) -> np.ndarray:
    """Integer moments (layout of ``moments``) of the listed pixels only: labels[t]
    belongs to full-grid pixel ids[t], and the odd coordinates u = 2k + 1 are the
    full grid's, so the moments of a partition of the grid sum to ``moments``."""
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    if ids.shape != labels.shape:
        raise ValueError("ids and labels differ in length")
    res = np.ascontiguousarray(grid.res, dtype=np.int32)
    out = np.empty((n, moment_width(grid.dim)), dtype=np.int64)
    rc = lib().oracle_moments_ids(grid.dim, _p(res, _c_i32p), n, _p(ids, _c_i64p), ids.shape[0],
                                  _p(labels, _c_i32p), _p(out, _c_i64p), nthreads)
    _check(rc, "moments_ids")
    return out


def slab_ids(grid, k_begin: int, k_count: int) -> np.ndarray:
    """Linear ids of the pixels whose last-axis index lies in [k_begin, k_begin + k_count)."""
    per = int(np.prod(grid.res[:-1], dtype=np.int64))
    return np.arange(k_begin * per, (k_begin + k_count) * per, dtype=np.int64)


def dual_from_moments(grid, x, A, w, v, mom):
    """Eqs. (2.7)-(2.8) from the integer moments alone: with y_j = lo + (h / 2) u_j,
    c_i = lo - x_i and D = diag(h / 2), the cost sum of cell i is
        Q_i = m_i c_i^T A_i c_i + 2 c_i^T A_i D S1_i + tr(D A_i D S2_i),
    so g~ = sum_i (v_i - m_i |P|) w_i + |P| Q_i and grad_i = v_i - m_i |P|.
    Returns (g~, grad, max_rel_err)."""
    x, A, w, v = _f64(x), _f64(A), _f64(w), _f64(v)
    mom = np.asarray(mom, dtype=np.int64)
    dim = grid.dim
    h = grid_steps(grid)
    P = pixel_volume(grid)
    m = mom[:, 0].astype(np.float64)
    S1 = mom[:, 1:1 + dim].astype(np.float64)
    S2 = np.zeros((x.shape[0], dim, dim))
    e = 1 + dim
    for a in range(dim):
        for b in range(a, dim):
            S2[:, a, b] = mom[:, e]
            S2[:, b, a] = mom[:, e]
            e += 1
    As = 0.5 * (A + np.transpose(A, (0, 2, 1)))
    c = np.asarray(grid.lo, dtype=np.float64)[None, :] - x
    Dh = 0.5 * h
    Ac = np.einsum("nab,nb->na", As, c)
    Q = m * np.einsum("na,na->n", c, Ac) + 2.0 * np.einsum("na,na->n", Ac * Dh[None, :], S1)
    Q += np.einsum("nab,nab->n", As * Dh[None, :, None] * Dh[None, None, :], S2)
    grad = v - m * P
    g = float(np.sum(grad * w + P * Q))
    return g, grad, float(np.max(np.abs(grad) / v))


def dual_from_labels(grid, x, A, w, v, labels, nthreads: int = 0):
    """(g~, grad [n], max_rel_err, counts m [n], per-cell cost sums [n]) for a labelling."""
    x, A, w, v = _f64(x), _f64(A), _f64(w), _f64(v)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    n = x.shape[0]
    lo, hi, res = _grid_args(grid)
    g = np.zeros(1)
    grad = np.empty(n)
    err = np.zeros(1)
    m = np.empty(n, dtype=np.int64)
    qs = np.empty(n)
    rc = lib().oracle_dual_from_labels(grid.dim, _p(lo, _c_dp), _p(hi, _c_dp), _p(res, _c_i32p), n,
                                       _p(x, _c_dp), _p(A, _c_dp), _p(w, _c_dp), _p(v, _c_dp),
                                       _p(labels, _c_i32p), _p(g, _c_dp), _p(grad, _c_dp),
                                       _p(err, _c_dp), _p(m, _c_i64p), _p(qs, _c_dp), nthreads)
    _check(rc, "dual")
    return float(g[0]), grad, float(err[0]), m, qs


def dual(grid, x, A, w, v, nthreads: int = 0):
    """Eqs. (2.7)-(2.8) at W: returns (g~, grad, max_rel_err)."""
    labels = assign(grid, x, A, w, nthreads=nthreads)
    g, grad, err, _, _ = dual_from_labels(grid, x, A, w, v, labels, nthreads)
    return g, grad, err


def centroids(grid, x, labels, nthreads: int = 0) -> np.ndarray:
    """Discrete centroids of Algorithm 3 (empty cells keep their seed)."""
    x = _f64(x)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    lo, hi, res = _grid_args(grid)
    out = np.empty_like(x)
    rc = lib().oracle_centroids(grid.dim, _p(lo, _c_dp), _p(hi, _c_dp), _p(res, _c_i32p),
                                x.shape[0], _p(x, _c_dp), _p(labels, _c_i32p), _p(out, _c_dp),
                                nthreads)
    _check(rc, "centroids")
    return out


def cost(y, xi, Ai, wi) -> float:
    """One entry of the cost matrix of Algorithm 1 (same arithmetic as the C core)."""
    y, xi, Ai = _f64(y), _f64(xi), _f64(Ai)
    return float(lib().oracle_cost(y.shape[0], _p(y, _c_dp), _p(xi, _c_dp), _p(Ai, _c_dp),
                                   float(wi)))


class _Converged(Exception):
    pass


def solve_weights(grid, x, A, v, w0=None, eps: float = 0.01, max_evals: int = 5000,
                  nthreads: int = 0):
    """Algorithm 2: maximise g~ with a library L-BFGS (scipy L-BFGS-B, no bounds) from W0
    (zero by default); stop at the first evaluation with max_i |v_i - m_i|P|| / v_i < eps.

    Returns (W, info) where info = {"converged", "evals", "max_rel_err", "g"}.
    L-BFGS-B may stop on a kink of the piecewise-linear g~ before the tolerance; it is
    then restarted from its best point until the evaluation budget is spent."""
    from scipy.optimize import minimize

    x, A, v = _f64(x), _f64(A), _f64(v)
    n = x.shape[0]
    W = np.zeros(n) if w0 is None else _f64(w0).copy()
    state = {"evals": 0, "best": None}

    def fun(Wc):
        state["evals"] += 1
        g, grad, err = dual(grid, x, A, Wc, v, nthreads)
        if state["best"] is None or err < state["best"][1]:
            state["best"] = (Wc.copy(), err, g)
        if err < eps:
            raise _Converged()
        if state["evals"] >= max_evals:
            raise _Converged()
        return -g, -grad

    converged = False
    try:
        while state["evals"] < max_evals:
            before = state["evals"]
            res = minimize(fun, W, jac=True, method="L-BFGS-B",
                           options={"maxiter": 100000, "maxfun": max_evals, "ftol": 0.0,
                                    "gtol": 0.0, "maxcor": 10})
            W = state["best"][0].copy() if state["best"] is not None else res.x
            if state["evals"] == before + 1:
                break
    except _Converged:
        pass
    Wb, err, g = state["best"]
    converged = err < eps
    return Wb, {"converged": converged, "evals": state["evals"], "max_rel_err": err, "g": g}


def lbfgs_direction(S, Y, g, gamma: float) -> np.ndarray:
    """p = -H g for the limited-memory BFGS matrix H built from H0 = gamma I and the
    pairs (s_k, y_k), rows of S and Y with the newest last: the two-loop recursion
    (Nocedal and Wright, Algorithm 7.4), in FP64.  Algorithm 2 ascends g~ with
    L-BFGS; in the minimisation of -g~ this is the search direction for gradient g."""
    S = np.asarray(S, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    q = np.array(g, dtype=np.float64)
    m = S.shape[0]
    rho = [1.0 / float(S[k] @ Y[k]) for k in range(m)]
    alpha = [0.0] * m
    for k in range(m - 1, -1, -1):        # newest to oldest
        alpha[k] = rho[k] * float(S[k] @ q)
        q = q - alpha[k] * Y[k]
    r = gamma * q
    for k in range(m):                    # oldest to newest
        beta = rho[k] * float(Y[k] @ r)
        r = r + (alpha[k] - beta) * S[k]
    return -r


def lloyd(grid, x, A, v, K: int = 5, eps: float = 0.01, w0=None, max_evals: int = 5000,
          nthreads: int = 0):
    """Algorithm 3: K rounds of {solve (Algorithm 2), move seeds to discrete centroids,
    warm-start the weights}, then a final solve.  Returns (X, W, infos)."""
    X = _f64(x).copy()
    W = np.zeros(X.shape[0]) if w0 is None else _f64(w0).copy()
    infos = []
    for _ in range(K):
        W, info = solve_weights(grid, X, A, v, W, eps, max_evals, nthreads)
        infos.append(info)
        labels = assign(grid, X, A, W, nthreads=nthreads)
        X = centroids(grid, X, labels, nthreads)
    W, info = solve_weights(grid, X, A, v, W, eps, max_evals, nthreads)
    infos.append(info)
    return X, W, infos


def resolution_lower_bound(n: int, dim: int, eps: float = 0.01) -> float:
    """Eq. (2.9): single phase on the unit box needs M > (N / eps)^(1/D)."""
    return (n / eps) ** (1.0 / dim)


def resolution_table_entry(n: int, dim: int, eps: float = 0.01) -> int:
    """Table 1 prints the bound of eq. (2.9) rounded to the nearest integer."""
    return int(math.floor(resolution_lower_bound(n, dim, eps) + 0.5))


def resolution_practical(dim: int, v_min: float, eps: float = 0.01, measure: float = 1.0) -> int:
    """Eq. (2.10): smallest M with |Omega| / M^D <= eps min_i v_i / 2^D (non-strict; the
    strict form would give 201 instead of the M = 200 the paper uses for D = 3,
    N = 10^4, single phase)."""
    t = (2.0 ** dim) * measure / (eps * v_min)
    m = int(math.ceil(t ** (1.0 / dim) - 1e-9))
    while measure / m ** dim > eps * v_min / 2.0 ** dim * (1 + 1e-12):
        m += 1
    while m > 1 and measure / (m - 1) ** dim <= eps * v_min / 2.0 ** dim * (1 + 1e-12):
        m -= 1
    return m
