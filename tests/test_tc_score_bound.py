"""The tensor-core scorer's rounding bounds, checked on the CPU.

A tile of the tcgen05 kernel (8^3 voxels in 3D, 32 x 16 pixels in 2D) scores
pixel j against seed i as the dot product of pixel features
f = [y'_a y'_b (a <= b), y'_a, 1] (y' = pixel centre - tile centre, FP32) and
seed features phi = [A_ab (x2 off the diagonal), -2 (A x')_a, x'^T A x' - w']
(x' = x_i - tile centre from FP32 high/low splits, w' = w_i - w_ref), both
rounded to TF32 (round to nearest, ties away) or BF16 (round to nearest even),
products summed in FP32.  The kernel relies on two facts:
  1. |score - C_exact| <= err_unit * sum_k |f_k phi_k|,
     err_unit = 1.5 (2 e + e^2 + 100 u), e = 2^-11 (TF32) or 2^-9 (BF16);
  2. every seed outside a pixel's three best scores has an exact cost of at
     least s4 - psi, s4 the fourth-best score and psi the kernel's bound from
     max ||A||_F, min lambda_min and the tile radius R.
This file restates the scores in numpy (two summation orders) and checks both
facts against exact rational costs; an err_unit without the operand roundings
fails fact 1 (planted mistake)."""
from fractions import Fraction as Fr

import numpy as np
import pytest

U = 2.0 ** -24
GEOM = {3: (8, 8, 8), 2: (32, 16, 1)}


def f32(v):
    return np.float32(v)


def fma32(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def to_tf32(v):
    b = np.array([v], dtype=np.float32).view(np.uint32)[0]
    r = (np.uint64(b) + np.uint64(0x1000)) & np.uint64(0xFFFFE000)
    return np.array([np.uint32(r)], dtype=np.uint32).view(np.float32)[0]


def to_bf16(v):
    b = np.uint64(np.array([v], dtype=np.float32).view(np.uint32)[0])
    r = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return np.array([np.uint32(r)], dtype=np.uint32).view(np.float32)[0]


def split(v):
    h = np.float32(v)
    return h, np.float32(np.float64(v) - np.float64(h))


def spd(g, dim, cond):
    Q, _ = np.linalg.qr(g.standard_normal((dim, dim)))
    ev = np.exp(g.uniform(0.0, np.log(cond), dim))
    M = (Q * ev) @ Q.T
    return 0.5 * (M + M.T)


def pixel_features(D, yp):
    if D == 3:
        return [f32(yp[0] * yp[0]), f32(yp[0] * yp[1]), f32(yp[0] * yp[2]), f32(yp[1] * yp[1]),
                f32(yp[1] * yp[2]), f32(yp[2] * yp[2]), yp[0], yp[1], yp[2], f32(1.0)]
    return [f32(yp[0] * yp[0]), f32(yp[0] * yp[1]), f32(yp[1] * yp[1]), yp[0], yp[1], f32(1.0)]


def seed_features(D, x, A, w, cen, wref):
    xch, xcl = zip(*[split(c) for c in cen])
    rxh, rxl = zip(*[split(v) for v in x])
    xp = [f32(f32(rxh[a] - xch[a]) + f32(rxl[a] - xcl[a])) for a in range(D)]
    wh, wl = split(w)
    wrh, wrl = split(wref)
    wp = f32(f32(wh - wrh) + f32(wl - wrl))
    a = [[f32(A[i][j]) for j in range(D)] for i in range(D)]
    t = []
    for i in range(D):
        acc = f32(a[i][0] * xp[0])
        for j in range(1, D):
            acc = fma32(a[i][j], xp[j], acc)
        t.append(acc)
    q = f32(xp[0] * t[0])
    for i in range(1, D):
        q = fma32(xp[i], t[i], q)
    two = f32(2.0)
    if D == 3:
        return [a[0][0], two * a[0][1], two * a[0][2], a[1][1], two * a[1][2], a[2][2],
                -two * t[0], -two * t[1], -two * t[2], f32(q - wp)]
    return [a[0][0], two * a[0][1], a[1][1], -two * t[0], -two * t[1], f32(q - wp)]


def score(f, phi, rnd, order):
    prods = [np.float64(rnd(fk)) * np.float64(rnd(pk)) for fk, pk in zip(f, phi)]  # exact
    idx = range(len(prods)) if order == 0 else reversed(range(len(prods)))
    s = f32(0.0)
    for k in idx:
        s = f32(np.float64(s) + prods[k])
    return s


def exact_cost(y, x, A, w, wref):
    D = len(y)
    d = [y[i] - Fr(float(x[i])) for i in range(D)]
    q = sum(d[i] * Fr(float(A[i][j])) * d[j] for i in range(D) for j in range(D))
    return q - (Fr(float(w)) - Fr(float(wref)))


def err_unit(kind, with_operands=True):
    e = 2.0 ** -11 if kind == "tf32" else 2.0 ** -9
    return 1.5 * ((2 * e + e * e) if with_operands else 0.0) + 1.5 * 100 * U


def run_case(D, kind, seed, eu, order, n=48, pixels=12):
    """(violations of fact 1, violations of fact 2) for one random tile."""
    g = np.random.Generator(np.random.PCG64(seed))
    rnd = to_tf32 if kind == "tf32" else to_bf16
    res = (256, 256, 256) if D == 3 else (1024, 1024)
    h = 1.0 / np.asarray(res, dtype=np.float64)
    h32 = [f32(v) for v in h]
    td = GEOM[D]
    kb = [int(g.integers(0, res[a] // td[a])) * td[a] for a in range(D)]
    cen = [(kb[a] + td[a] // 2) * h[a] for a in range(D)]
    half = np.array([0.5 * td[a] * h[a] for a in range(D)])
    R = float(np.sqrt((half ** 2).sum()) * (1 + 1e-6))
    span = 3.0 * half.max()
    xs = np.array(cen) + g.uniform(-span, span, (n, D))
    As = [spd(g, D, [1.0, 10.0, 1e3][seed % 3]) * 10 ** g.uniform(-0.5, 0.5) for _ in range(n)]
    ws = g.uniform(0.0, 1.0, n) * span ** 2
    wref = float(ws.max())
    Lam = max(float(np.linalg.norm(A)) for A in As)
    lam = min(float(np.linalg.eigvalsh(A).min()) for A in As) * (1 - 1e-9)
    phis = [seed_features(D, xs[i], As[i], ws[i], cen, wref) for i in range(n)]
    bad1 = bad2 = 0
    for _ in range(pixels):
        lk = [int(g.integers(0, td[a])) for a in range(D)]
        yp = [f32(f32(f32(lk[a] - td[a] // 2) + f32(0.5)) * h32[a]) for a in range(D)]
        f = pixel_features(D, yp)
        y = [(Fr(kb[a] + lk[a]) + Fr(1, 2)) * Fr(float(h[a])) for a in range(D)]
        sc, ex = [], []
        for i in range(n):
            s = score(f, phis[i], rnd, order)
            c = exact_cost(y, xs[i], As[i], ws[i], wref)
            mag = sum(abs(float(fk) * float(pk)) for fk, pk in zip(f, phis[i]))
            bad1 += abs(Fr(float(s)) - c) > Fr(eu * mag)
            sc.append(float(s))
            ex.append(c)
        order_s = np.argsort(sc, kind="stable")
        s3 = sc[order_s[3]]
        eu0 = err_unit(kind)
        c_out = abs(s3)
        r1 = 2 * R + np.sqrt(c_out / lam)
        psi = eu0 * (Lam * r1 * r1 + c_out)
        c_out = abs(s3) + psi
        r1 = 2 * R + np.sqrt(c_out / lam)
        psi = 1.1 * eu0 * (Lam * r1 * r1 + c_out)
        for i in order_s[3:]:
            bad2 += ex[i] < Fr(s3 - psi)
    return bad1, bad2


@pytest.mark.parametrize("D", [3, 2])
@pytest.mark.parametrize("kind", ["tf32", "bf16"])
def test_tensor_core_scores_within_bounds(D, kind):
    for seed in range(6):
        for order in (0, 1):
            assert run_case(D, kind, seed, err_unit(kind), order) == (0, 0), (seed, order)


def test_err_unit_without_operand_rounding_is_violated():
    # planted mistake: only the FP32 part of err_unit
    assert run_case(3, "tf32", 0, err_unit("tf32", with_operands=False), 0)[0] > 0
