"""The FP32 direct-form cost and its rounding bound, used by the non-uniform and
masked scoring kernels (pass 1: threshold min_k (C_k + E_k); pass 2: FP64 on
the seeds with C_k - E_k under it), restated in numpy with the kernel's FP32
operations and checked on the CPU against the exact rational cost:

  d_a = (yh_a - xh_a) + (yl_a - xl_a)          (FP32 high/low splits of FP64 y, x)
  q   = sum_a d_a (A d)_a                      (FMA chains, FP32 symmetric A)
  qa  = sum_a |d_a| (|A| |d|)_a
  wp  = (wh - wrh) + (wl - wrl),  C = q - wp   (weights relative to w_ref)
  E   = 16 u (qa + |wp| + |C|),   u = 2^-24.

|C - C_exact| <= E is what makes the FP64 argmin one of pass 2's candidates."""
from fractions import Fraction as Fr

import numpy as np
import pytest

U = 2.0 ** -24


def _f32(v):
    return np.float32(v)


def _fma32(a, b, c):
    # a * b is exact in float64; the sum is rounded to float64, then to float32
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _split(v):
    h = np.float32(v)
    return h, np.float32(np.float64(v) - np.float64(h))


def _spd(g, dim, cond):
    Q, _ = np.linalg.qr(g.standard_normal((dim, dim)))
    ev = np.exp(g.uniform(0.0, np.log(cond), dim))
    M = (Q * ev) @ Q.T
    return 0.5 * (M + M.T)


def cost32(y, x, A, w, wref):
    """(C, qa + |wp| + |C|) with the kernel's FP32 operations."""
    D = len(y)
    yh, yl = zip(*[_split(v) for v in y])
    xh, xl = zip(*[_split(v) for v in x])
    wh, wl = _split(w)
    wrh, wrl = _split(wref)
    d = [_f32(_f32(yh[a] - xh[a]) + _f32(yl[a] - xl[a])) for a in range(D)]
    a32 = [[_f32(A[i][j]) for j in range(D)] for i in range(D)]

    def chain(coef, vec):
        acc = _f32(coef[0] * vec[0])
        for j in range(1, D):
            acc = _fma32(coef[j], vec[j], acc)
        return acc

    t = [chain(a32[i], d) for i in range(D)]
    q = chain(d, t)
    e = [abs(v) for v in d]
    s = [chain([abs(v) for v in a32[i]], e) for i in range(D)]
    qa = chain(e, s)
    wp = _f32(_f32(wh - wrh) + _f32(wl - wrl))
    c = _f32(q - wp)
    return c, _f32(_f32(qa + abs(wp)) + abs(c))


def exact_cost(y, x, A, w, wref):
    D = len(y)
    d = [Fr(float(y[i])) - Fr(float(x[i])) for i in range(D)]
    q = sum(d[i] * Fr(float(A[i][j])) * d[j] for i in range(D) for j in range(D))
    return q - (Fr(float(w)) - Fr(float(wref)))


def _sample(g, dim, it):
    A = _spd(g, dim, [1.0, 10.0, 1e3][it % 3]) * 10 ** g.uniform(-1, 2)
    x = g.uniform(-0.2, 1.2, dim)
    y = x + 10 ** g.uniform(-4, 0) * g.standard_normal(dim) if it % 2 else g.uniform(0.0, 1.0, dim)
    w = g.standard_normal() * 10 ** g.uniform(-4, 0)
    wref = w + abs(g.standard_normal()) * 10 ** g.uniform(-6, 0)
    return y, x, A, w, wref


@pytest.mark.parametrize("dim", [2, 3])
def test_direct_cost_error_is_within_its_bound(dim):
    g = np.random.Generator(np.random.PCG64(40 + dim))
    worst = 0.0
    for it in range(1500):
        y, x, A, w, wref = _sample(g, dim, it)
        c, base = cost32(y, x, A, w, wref)
        err = abs(Fr(float(c)) - exact_cost(y, x, A, w, wref))
        bound = Fr(16) * Fr(U) * Fr(float(base))
        assert err <= bound, (it, float(err), float(bound))
        if base > 0:
            worst = max(worst, float(err / (Fr(U) * Fr(float(base)))))
    # planted mistake: the same bound with u in place of 16 u is violated
    assert worst > 1.0, worst


@pytest.mark.parametrize("dim", [2, 3])
def test_fp64_argmin_is_a_candidate(dim):
    # the two-pass rule of the kernels: the seed of the smallest exact cost has
    # C - E under min_k (C_k + E_k), for pixels among many near-equal seeds
    g = np.random.Generator(np.random.PCG64(50 + dim))
    for _ in range(60):
        n = 24
        y = g.uniform(0.0, 1.0, dim)
        xs = y + 1e-3 * g.standard_normal((n, dim))
        As = [_spd(g, dim, 10.0) for _ in range(n)]
        ws = 1e-7 * g.standard_normal(n)
        wref = float(ws.max())
        cs, Es, exact = [], [], []
        for i in range(n):
            c, base = cost32(y, xs[i], As[i], ws[i], wref)
            cs.append(float(c))
            Es.append(16 * U * float(base))
            exact.append(exact_cost(y, xs[i], As[i], ws[i], wref))
        thr = min(c + E for c, E in zip(cs, Es))
        best = min(range(n), key=lambda i: exact[i])
        assert cs[best] - Es[best] <= thr
