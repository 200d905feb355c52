"""The tensor-core scorer's rounding bounds and certificate, checked on the CPU.

A tile of the tcgen05 kernel (8^3 voxels in 3D, 32 x 16 pixels in 2D) scores
pixel j against seed i as the dot product of the pixel features
f = [y'_a y'_b (a <= b), y'_a, 1] (y' = pixel centre - tile centre, FP32) and the
seed features phi = [A_ab (x2 off the diagonal), -2 (A x')_a, x'^T A x' - w']
(x' = x_i - tile centre from FP32 high/low splits, w' = w_i - w_ref).  Each
FP32 feature v is split into operands vh = rnd(v), vl = rnd(v - vh) of the
tensor format (TF32: round to nearest, ties away; BF16: round to nearest even),
the contraction sums fh.phih + fl.phih + fh.phil in FP32, and the kernel keeps
the score with the step-local seed index in its five low mantissa bits.

This file restates that arithmetic in numpy and checks, against exact rational
costs C' = (y - x)^T A (y - x) + (w_ref - w):
  1. every packed score lies within err_unit * sum_k |f_k phi_k| of C';
  2. the candidate pre-pass's lower bound (lambda_min dist^2 + (w_ref - w),
     FP32 with its directed roundings and slacks, restated with exact
     rounding) never exceeds C' at a pixel of the tile; nor does its second,
     centre form (q - 2 sum |(A d)_a| r_a with d the box centre's offset), and
     the centre form's upper bound is never below C' (boxes of one tile and of
     a 2 x 2 (x 2) super-tile, conditioning up to 10^3);
  3. the certificate: whenever s1 + psi(s1) < min(s2 - psi(s2), T_excl), the
     best score's seed is the exact argmin over all seeds (those left out of
     the candidate list included).
Planted mistakes: operands that are not split, a lower bound built with the
largest eigenvalue in place of the smallest, and a centre form without its
linear term must fail."""
from fractions import Fraction as Fr

import numpy as np
import pytest

U = 2.0 ** -24
GEOM = {3: (8, 8, 8), 2: (32, 16, 1)}


def f32(v):
    return np.float32(v)


def fma32(a, b, c):
    return np.float32(Fr(float(a)) * Fr(float(b)) + Fr(float(c)))


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


def rd32(x):
    """Largest float32 <= the rational x (exact directed rounding)."""
    f = np.float32(float(x))
    while Fr(float(f)) > x:
        f = np.nextafter(f, np.float32(-np.inf))
    while Fr(float(np.nextafter(f, np.float32(np.inf)))) <= x:
        f = np.nextafter(f, np.float32(np.inf))
    return f


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
        feats = [a[0][0], two * a[0][1], two * a[0][2], a[1][1], two * a[1][2], a[2][2],
                 -two * t[0], -two * t[1], -two * t[2], f32(q - wp)]
    else:
        feats = [a[0][0], two * a[0][1], a[1][1], -two * t[0], -two * t[1], f32(q - wp)]
    return feats, xp, wp


def score(f, phi, rnd, order, split_ops=True):
    """Packed-free score: the split contraction summed in FP32 in one of two orders."""
    prods = []
    for fk, pk in zip(f, phi):
        fh, ph = rnd(fk), rnd(pk)
        if split_ops:
            fl, pl = rnd(f32(fk - fh)), rnd(f32(pk - ph))
            prods += [Fr(float(fh)) * Fr(float(ph)), Fr(float(fl)) * Fr(float(ph)), Fr(float(fh)) * Fr(float(pl))]
        else:
            prods.append(Fr(float(fh)) * Fr(float(ph)))
    idx = range(len(prods)) if order == 0 else reversed(range(len(prods)))
    s = f32(0.0)
    for k in idx:
        s = np.float32(Fr(float(s)) + prods[k])
    return s


def pack(s, idx):
    b = np.array([s], dtype=np.float32).view(np.uint32)[0]
    return np.array([(b & np.uint32(0xFFFFFFE0)) | np.uint32(idx)], dtype=np.uint32).view(np.float32)[0]


def exact_cost(y, x, A, w, wref):
    D = len(y)
    d = [y[i] - Fr(float(x[i])) for i in range(D)]
    q = sum(d[i] * Fr(float(A[i][j])) * d[j] for i in range(D) for j in range(D))
    return q - (Fr(float(w)) - Fr(float(wref)))


def err_unit(kind):
    e = 2.0 ** -11 if kind == "tf32" else 2.0 ** -8
    return 1.5 * (3.1 * e * e + 32 * 2.0 ** -22 + 100 * U + 2.0 ** -18)


def psi(s, eu, Lam, lam, R):
    """The kernel's bound, linear in |s|: Lambda (2R + sqrt(C/lambda))^2 + C <=
    8 Lambda R^2 + (2 Lambda / lambda + 1) C, at C <= |s| + eu (that sum at |s|)."""
    ps0, ps1 = 8 * Lam * R * R, 2 * Lam / lam + 1
    c = abs(s) + eu * (ps1 * abs(s) + ps0)
    return 1.1 * eu * (ps1 * c + ps0)


def lower_bound(D, xp, wp, lam_i, rlo, rhi, with_slack=True):
    """The pre-pass's FP32 lower bound of C' over the tile's pixel box, with the
    kernel's directed roundings done exactly."""
    d2 = f32(0.0)
    for a in range(D):
        xs = xp[a]
        slack = f32(f32(1e-6) * f32(f32(abs(rlo[a]) + abs(rhi[a])) + f32(2.0) * abs(xs))) + f32(1e-30)
        if not with_slack:
            slack = f32(0.0)
        dl = max(f32(max(f32(xs - rhi[a]), f32(rlo[a] - xs)) - slack), f32(0.0))
        d2 = rd32(Fr(float(dl)) * Fr(float(dl)) + Fr(float(d2)))
    wn = f32(-wp)
    wslack = f32(f32(1e-6) * abs(wn)) + f32(1e-30)
    t = rd32(Fr(float(rd32(Fr(float(lam_i)) * Fr(float(d2))))) * Fr(float(f32(1.0 - 1e-5))))
    return rd32(Fr(float(t)) + Fr(float(rd32(Fr(float(wn)) - Fr(float(wslack))))))


def make_tile(D, seed, n):
    g = np.random.Generator(np.random.PCG64(seed))
    res = (256, 256, 256) if D == 3 else (1024, 1024)
    h = 1.0 / np.asarray(res, dtype=np.float64)
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
    return g, h, td, kb, cen, R, xs, As, ws, wref


def run_case(D, kind, seed, order, n=40, pixels=10, split_ops=True, with_slack=True):
    """(violations of fact 1, of fact 2, of fact 3) on one random tile."""
    g, h, td, kb, cen, R, xs, As, ws, wref = make_tile(D, seed, n)
    rnd = to_tf32 if kind == "tf32" else to_bf16
    h32 = [f32(v) for v in h]
    eu = err_unit(kind)
    Lam = max(float(np.linalg.norm(A)) for A in As)
    lam_i = [f32(np.linalg.eigvalsh(A).min() * (1 - 1e-6)) for A in As]
    lam = min(float(v) for v in lam_i)
    feats = [seed_features(D, xs[i], As[i], ws[i], cen, wref) for i in range(n)]
    rlo = [f32(f32(f32(-(td[a] // 2)) + f32(0.5)) * h32[a]) for a in range(D)]
    rhi = [f32(f32(f32(td[a] - 1 - td[a] // 2) + f32(0.5)) * h32[a]) for a in range(D)]
    lbs = [lower_bound(D, feats[i][1], feats[i][2], lam_i[i], rlo, rhi, with_slack) for i in range(n)]
    # candidates: a random half of the seeds (the certificate must hold for any split)
    cand = g.random(n) < 0.5
    cand[int(np.argmin([float(v) for v in lbs]))] = True
    texcl = min([float(lbs[i]) for i in range(n) if not cand[i]], default=np.inf)
    bad1 = bad2 = bad3 = 0
    for _ in range(pixels):
        lk = [int(g.integers(0, td[a])) for a in range(D)]
        yp = [f32(f32(f32(lk[a] - td[a] // 2) + f32(0.5)) * h32[a]) for a in range(D)]
        f = pixel_features(D, yp)
        y = [(Fr(kb[a] + lk[a]) + Fr(1, 2)) * Fr(float(h[a])) for a in range(D)]
        ex = [exact_cost(y, xs[i], As[i], ws[i], wref) for i in range(n)]
        keys = []
        for i in range(n):
            k = pack(score(f, feats[i][0], rnd, order, split_ops), i % 32)
            mag = sum(abs(float(fk) * float(pk)) for fk, pk in zip(f, feats[i][0]))
            bad1 += abs(Fr(float(k)) - ex[i]) > Fr(eu * mag)
            bad2 += Fr(float(lbs[i])) > ex[i]
            keys.append(float(k) if cand[i] else np.inf)
        o = np.argsort(keys, kind="stable")
        s1, s2 = keys[o[0]], keys[o[1]]
        Ub = s1 + psi(s1, eu, Lam, lam, R)
        if Ub < s2 - psi(s2, eu, Lam, lam, R) and Ub < texcl:
            best = min(range(n), key=lambda i: (ex[i], i))
            bad3 += best != o[0]
    return bad1, bad2, bad3


@pytest.mark.parametrize("D", [3, 2])
@pytest.mark.parametrize("kind", ["tf32", "bf16"])
def test_tensor_core_scores_bounds_and_certificate(D, kind):
    for seed in range(4):
        for order in (0, 1):
            assert run_case(D, kind, seed, order) == (0, 0, 0), (seed, order)


def test_unsplit_operands_violate_the_bound():
    # planted mistake: plain BF16 operands with the split form's err_unit
    assert run_case(3, "bf16", 0, 0, split_ops=False)[0] > 0


def test_lower_bound_with_lambda_max_is_violated():
    # planted mistake: the largest eigenvalue in place of the smallest in the lower bound
    viol = 0
    for seed in range(3):
        g, h, td, kb, cen, R, xs, As, ws, wref = make_tile(3, seed, 30)
        h32 = [f32(v) for v in h]
        rlo = [f32(f32(f32(-(td[a] // 2)) + f32(0.5)) * h32[a]) for a in range(3)]
        rhi = [f32(f32(f32(td[a] - 1 - td[a] // 2) + f32(0.5)) * h32[a]) for a in range(3)]
        for i in range(30):
            feats, xp, wp = seed_features(3, xs[i], As[i], ws[i], cen, wref)
            lmax = f32(np.linalg.eigvalsh(As[i]).max())
            lb = lower_bound(3, xp, wp, lmax, rlo, rhi)
            for _ in range(4):
                lk = [int(g.integers(0, td[a])) for a in range(3)]
                y = [(Fr(kb[a] + lk[a]) + Fr(1, 2)) * Fr(float(h[a])) for a in range(3)]
                viol += Fr(float(lb)) > exact_cost(y, xs[i], As[i], ws[i], wref)
    assert viol > 0


def ru32(x):
    """Smallest float32 >= the rational x (exact directed rounding)."""
    return -rd32(-x)


def centre_bounds(D, xp, wp, A, lam_i, lmax_i, rlo, rhi, with_lin=True):
    """The pre-pass's bounds with both forms, restated: FP32 round-to-nearest
    where the kernel rounds to nearest, exact directed rounding where it rounds
    up or down.  Returns (lower, upper) = (max of the forms, min of the forms)."""
    a32 = [[f32(A[i][j]) for j in range(D)] for i in range(D)]
    d2lo, d2hi = f32(0.0), f32(0.0)
    dv, rr = [], []
    for a in range(D):
        xs = xp[a]
        slack = f32(f32(f32(1e-6) * f32(f32(abs(rlo[a]) + abs(rhi[a])) + f32(2.0) * abs(xs))) + f32(1e-30))
        dl = max(f32(max(f32(xs - rhi[a]), f32(rlo[a] - xs)) - slack), f32(0.0))
        dh = f32(max(abs(f32(xs - rlo[a])), abs(f32(xs - rhi[a]))) + slack)
        d2lo = rd32(Fr(float(dl)) * Fr(float(dl)) + Fr(float(d2lo)))
        d2hi = ru32(Fr(float(dh)) * Fr(float(dh)) + Fr(float(d2hi)))
        dv.append(f32(f32(f32(0.5) * f32(rlo[a] + rhi[a])) - xs))
        rr.append(f32(f32(f32(0.5) * f32(rhi[a] - rlo[a])) + slack))
    wn = f32(-wp)
    wslack = f32(f32(f32(1e-6) * abs(wn)) + f32(1e-30))
    lo_w, hi_w = rd32(Fr(float(wn)) - Fr(float(wslack))), ru32(Fr(float(wn)) + Fr(float(wslack)))
    lb1 = rd32(Fr(float(rd32(Fr(float(rd32(Fr(float(lam_i)) * Fr(float(d2lo))))) * Fr(float(f32(1.0 - 1e-5))))))
               + Fr(float(lo_w)))
    ub1 = ru32(Fr(float(ru32(Fr(float(ru32(Fr(float(lmax_i)) * Fr(float(d2hi))))) * Fr(float(f32(1.0 + 1e-5))))))
               + Fr(float(hi_w)))
    q = lin = quad = S = f32(0.0)
    for a in range(D):
        ga = qa = sa = f32(0.0)
        for b in range(D):
            ga = fma32(a32[a][b], dv[b], ga)
            qa = fma32(abs(a32[a][b]), rr[b], qa)
            sa = fma32(abs(a32[a][b]), f32(abs(dv[b]) + rr[b]), sa)
        q = fma32(dv[a], ga, q)
        lin = fma32(abs(ga), rr[a], lin)
        quad = fma32(qa, rr[a], quad)
        S = fma32(sa, f32(abs(dv[a]) + rr[a]), S)
    lin = f32(2.0) * lin if with_lin else f32(0.0)
    E = f32(f32(f32(1e-5) * S) + f32(1e-30))
    lb2 = rd32(Fr(float(rd32(Fr(float(rd32(Fr(float(q)) - Fr(float(lin))))) - Fr(float(E))))) + Fr(float(lo_w)))
    ub2 = ru32(Fr(float(ru32(Fr(float(ru32(Fr(float(q)) + Fr(float(lin))))) + Fr(float(ru32(Fr(float(quad)) + Fr(float(E)))))))) + Fr(float(hi_w)))
    return max(lb1, lb2), min(ub1, ub2), lb2 > lb1


def centre_case(D, seed, super_box, with_lin=True, n=30, pixels=12):
    """(lower-bound violations, upper-bound violations, seeds whose centre form is
    the tighter lower bound) over random seeds and pixels of one box."""
    g, h, td, kb, cen, R, xs, As, ws, wref = make_tile(D, seed, n)
    xs = np.array(cen) + (xs - np.array(cen)) * g.uniform(1.0, 4.0, (n, 1))  # near and farther seeds
    h32 = [f32(v) for v in h]
    span = [2 * td[a] if super_box else td[a] for a in range(D)]
    rlo = [f32(f32(f32(-(td[a] // 2)) + f32(0.5)) * h32[a]) for a in range(D)]
    rhi = [f32(f32(f32(span[a] - 1 - td[a] // 2) + f32(0.5)) * h32[a]) for a in range(D)]
    bad_lo = bad_hi = tighter = 0
    for i in range(n):
        A = As[i]
        ev = np.linalg.eigvalsh(A)
        lam_i = f32(ev.min() * (1 - 1e-6))
        lmax_i = f32(ev.max() * (1 + 1e-6))
        _, xp, wp = seed_features(D, xs[i], A, ws[i], cen, wref)
        lb, ub, t = centre_bounds(D, xp, wp, A, lam_i, lmax_i, rlo, rhi, with_lin)
        tighter += t
        for _ in range(pixels):
            lk = [int(g.integers(0, span[a])) for a in range(D)]
            y = [(Fr(kb[a] + lk[a]) + Fr(1, 2)) * Fr(float(h[a])) for a in range(D)]
            c = exact_cost(y, xs[i], A, ws[i], wref)
            bad_lo += Fr(float(lb)) > c
            bad_hi += Fr(float(ub)) < c
    return bad_lo, bad_hi, tighter


@pytest.mark.parametrize("D", [3, 2])
@pytest.mark.parametrize("super_box", [False, True])
def test_centre_form_bounds(D, super_box):
    tighter = 0
    for seed in range(6):  # conditioning 1, 10, 10^3 by seed
        lo, hi, t = centre_case(D, seed, super_box)
        assert (lo, hi) == (0, 0), seed
        tighter += t
    assert tighter > 0  # the centre form does improve on the eigenvalue form somewhere


def test_centre_form_without_its_linear_term_is_violated():
    # planted mistake: the lower bound q - E without -2 sum |(A d)_a| r_a
    assert sum(centre_case(3, seed, False, with_lin=False)[0] for seed in range(3)) > 0
