"""FP64 CPU oracle of Algorithm 1 on a non-uniform discretisation.

TEST INFRASTRUCTURE ONLY: tests/ and ``bench.py`` may import it; the library
path never does.  Plain numpy; shares no code with the CUDA path.

Section 2.3 allows any discretisation of the domain into elements P_j with
sample points y_j and measures |P_j| (a triangulation, say); the regular grid
is the special case y_j = pixel centre, |P_j| = |P|.  With labels
H_j = argmin_i c_ij (lowest index on ties) and c_ij = (y_j - x_i)^T A_i
(y_j - x_i) - w_i (the cost matrix of Algorithm 1, same operation order as the
C core: d = y - x; q = sum_a sum_b (d_a A_ab) d_b, a outer, b inner, every
operation rounded on its own), the moments of cell i are the element-measure
weighted sums m_i = sum |P_j|, S1_i = sum |P_j| y_j, S2_i = sum |P_j| y_j y_j^T
(upper triangle), and eqs. (2.7)-(2.8) read
    g~(W) = sum_i v_i w_i + sum_j |P_j| c_{H_j j},   grad_i = v_i - m_i.

Pins (tests/test_oracle_points.py): on the pixel centres of a grid with
|P_j| = |P| the labels equal the C oracle's bit for bit and the moments and
dual equal the grid oracle's; with A_i = I and w = 0 the labels are the
nearest seeds of a k-d tree query.
"""
from __future__ import annotations

import numpy as np


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def moment_width(dim: int) -> int:
    return 1 + dim + dim * (dim + 1) // 2


def costs(y, x, A, w) -> np.ndarray:
    """Cost matrix [count, n] of Algorithm 1 (FP64, the C core's operation order)."""
    y, x, A, w = _f64(y), _f64(x), _f64(A), _f64(w)
    dim = y.shape[1]
    d = y[:, None, :] - x[None, :, :]  # [count, n, D]
    q = np.zeros(d.shape[:2])
    for a in range(dim):
        for b in range(dim):
            q = q + (d[:, :, a] * A[None, :, a, b]) * d[:, :, b]
    return q - w[None, :]


def assign(y, x, A, w, chunk: int = 4096) -> np.ndarray:
    """Labels int32 [count]: argmin over seeds, lowest index on ties."""
    y = _f64(y)
    out = np.empty(y.shape[0], dtype=np.int32)
    for s in range(0, y.shape[0], chunk):
        out[s:s + chunk] = np.argmin(costs(y[s:s + chunk], x, A, w), axis=1)
    return out


def moments(y, mass, labels, n: int) -> np.ndarray:
    """FP64 [n, K]: m_i, S1_i (D), upper triangle of S2_i (a <= b, row-major)."""
    y, mass = _f64(y), _f64(mass)
    dim = y.shape[1]
    out = np.zeros((n, moment_width(dim)))
    np.add.at(out[:, 0], labels, mass)
    for a in range(dim):
        np.add.at(out[:, 1 + a], labels, mass * y[:, a])
    k = 1 + dim
    for a in range(dim):
        for b in range(a, dim):
            np.add.at(out[:, k], labels, mass * y[:, a] * y[:, b])
            k += 1
    return out


def dual(y, mass, x, A, w, v, chunk: int = 4096):
    """(g~, grad [n], max_i |grad_i| / v_i) at W, summed over the elements."""
    y, mass, w, v = _f64(y), _f64(mass), _f64(w), _f64(v)
    n = w.shape[0]
    total = 0.0
    m = np.zeros(n)
    for s in range(0, y.shape[0], chunk):
        c = costs(y[s:s + chunk], x, A, w)
        lab = np.argmin(c, axis=1)
        cmin = c[np.arange(c.shape[0]), lab]
        total += float(np.sum(mass[s:s + chunk] * cmin))
        np.add.at(m, lab, mass[s:s + chunk])
    g = float(np.sum(v * w)) + total
    grad = v - m
    return g, grad, float(np.max(np.abs(grad) / v))
