"""The exactness argument of the tile scorer, checked on the CPU.

The FP32 scoring kernel writes the cost of seed i at a pixel of a tile around
the tile's centre point c (FP64, rounded once to FP32 offsets):
    C = (A00 delta + b) delta + a,   delta = pixel offset along axis 0,
with per-(row, seed) coefficients a, b built from the seed's FP32 offsets
(d0 = c0 - x0, x1 - c1, x2 - c2), its FP32 symmetric A and w - w_ref.  A
pixel's two smallest keys b1 <= b2 (costs with the seed's 5-bit group index
in the low mantissa bits) decide its label unless
    b2 - b1 <= 2 E,   E = kappa u T,   T = Lambda (R + sqrt(|b1| / lambda))^2 + |b1|,
(kappa = 160, u = 2^-24, Lambda >= max ||A_i||_F, lambda <= min lambda_min(A_i),
R the tile half-diagonal), in which case the pixel is rescored in FP64.

This file restates that arithmetic in numpy (FP32 operations, FMAs through
float64) for the 3D 16^3 and 2D 64 x 64 tiles and checks, against exact
rational costs at the FP64 pixel centres: every seed whose exact cost is near
the best has a key within E of it, and a pixel that is not queued has the
exact argmin (lowest index on ties) as its FP32 label.  A bound with kappa = 1
fails the first check (planted mistake)."""
from fractions import Fraction as Fr

import numpy as np
import pytest

U = 2.0 ** -24
KAPPA = 160.0


def f32(v):
    return np.float32(v)


def fma32(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def pack(c, idx):
    bits = np.array([c], dtype=np.float32).view(np.uint32)[0]
    return np.array([(bits & ~np.uint32(31)) | np.uint32(idx)], dtype=np.uint32).view(np.float32)[0]


def spd(g, dim, cond):
    Q, _ = np.linalg.qr(g.standard_normal((dim, dim)))
    ev = np.exp(g.uniform(0.0, np.log(cond), dim))
    M = (Q * ev) @ Q.T
    return 0.5 * (M + M.T)


def lam_min(A):
    return float(np.linalg.eigvalsh(A).min())


def seed_coeffs(D, cref, wref, x, A, w, contract):
    """The chunk transform of one seed: FP32 row-form inputs (phi) of the kernel."""
    d0 = f32(cref[0] - x[0])
    x1p = f32(x[1] - cref[1])
    x2p = f32(x[2] - cref[2]) if D == 3 else f32(0.0)
    wp = f32(w - wref)
    a = {(i, j): f32(A[i][j]) for i in range(D) for j in range(D)}
    a00d0 = f32(a[0, 0] * d0)
    const = fma32(a00d0, d0, -wp) if contract else f32(f32(a00d0 * d0) - wp)
    return d0, x1p, x2p, a, const


def row_coeffs(D, phi, f1, f2):
    """seed_pair_coeffs for one seed: (q00, b, a) of the row (f1, f2)."""
    d0, x1p, x2p, a, const = phi
    d1 = f32(f1 - x1p)
    if D == 3:
        d2 = f32(f2 - x2p)
        e0 = fma32(a[0, 2], d2, f32(a[0, 1] * d1))
        bb = fma32(f32(2.0), e0, f32(f32(f32(2.0) * a[0, 0]) * d0))
        t = fma32(f32(f32(2.0) * a[1, 2]), d2, f32(a[1, 1] * d1))
        aa = fma32(d1, t, const)
        aa = fma32(f32(f32(2.0) * d0), e0, aa)
        av = fma32(f32(a[2, 2] * d2), d2, aa)
    else:
        u1 = fma32(a[1, 1], d1, f32(f32(f32(2.0) * a[0, 1]) * d0))
        av = fma32(d1, u1, const)
        bb = fma32(f32(f32(2.0) * a[0, 1]), d1, f32(f32(f32(2.0) * a[0, 0]) * d0))
    return a[0, 0], bb, av


def exact_cost(y, x, A, w, wref):
    D = len(y)
    d = [y[i] - Fr(float(x[i])) for i in range(D)]
    q = sum(d[i] * Fr(float(A[i][j])) * d[j] for i in range(D) for j in range(D))
    return q - (Fr(float(w)) - Fr(float(wref)))


# tile shapes of the kernel: (TX * P) x TY x TZ pixels
TILES = {3: (16, 16, 16), 2: (64, 64, 1)}


def run_case(D, seed, kappa, contract, n=32, pixels=24):
    """Returns (worst |key - exact| / (u T) over the near-best seeds, violations of
    the E bound, unqueued pixels whose label is not the exact argmin)."""
    g = np.random.Generator(np.random.PCG64(seed))
    res = (256, 256, 256) if D == 3 else (1024, 1024)
    lo, hi = np.zeros(D), np.ones(D)
    h = (hi - lo) / np.asarray(res, dtype=np.float64)
    h32 = [f32(v) for v in h]
    W0, TY, TZ = TILES[D]
    kt = [int(g.integers(0, res[0] // W0)) * W0, int(g.integers(0, res[1] // TY)) * TY]
    if D == 3:
        kt.append(int(g.integers(0, res[2] // TZ)) * TZ)
    kc = [kt[0] + W0 // 2, kt[1] + TY // 2] + ([kt[2] + TZ // 2] if D == 3 else [])
    cref = [lo[a] + kc[a] * h[a] for a in range(D)] + ([0.0] if D == 2 else [])
    half = np.array([0.5 * W0 * h[0], 0.5 * TY * h[1]] + ([0.5 * TZ * h[2]] if D == 3 else []))
    R = float(np.sqrt((half ** 2).sum()) * (1 + 1e-6))
    # seeds around the tile, competing weights
    centre = np.array(cref[:D])
    span = 3.0 * half.max()
    xs = centre + g.uniform(-span, span, (n, D))
    As = [spd(g, D, [1.0, 10.0, 1e3][seed % 3]) * 10 ** g.uniform(-0.5, 0.5) for _ in range(n)]
    ws = g.uniform(0.0, 1.0, n) * (span ** 2)
    wref = float(ws.max())
    Lam = max(float(np.linalg.norm(A)) for A in As)
    lam = min(lam_min(A) for A in As) * (1 - 1e-9)
    phis = [seed_coeffs(D, cref, wref, xs[i], As[i], ws[i], contract) for i in range(n)]
    worst, bad_bound, bad_label = 0.0, 0, 0
    for _ in range(pixels):
        off = [int(g.integers(0, W0)), int(g.integers(0, TY))] + ([int(g.integers(0, TZ))] if D == 3 else [])
        k = [kt[a] + off[a] for a in range(D)]
        delta = f32(f32(f32(off[0] - W0 // 2) + f32(0.5)) * h32[0])
        f1 = f32(f32(f32(off[1] - TY // 2) + f32(0.5)) * h32[1])
        f2 = f32(f32(f32(off[2] - TZ // 2) + f32(0.5)) * h32[2]) if D == 3 else f32(0.0)
        y = [Fr(float(lo[a])) + (Fr(k[a]) + Fr(1, 2)) * Fr(float(h[a])) for a in range(D)]
        keys, exact = [], []
        for i in range(n):
            q00, bb, av = row_coeffs(D, phis[i], f1, f2)
            c = fma32(fma32(q00, delta, bb), delta, av)
            keys.append(pack(c, i))
            exact.append(exact_cost(y, xs[i], As[i], ws[i], wref))
        order = np.argsort(np.array(keys, dtype=np.float32), kind="stable")
        gbest, b1, b2 = int(order[0]), float(keys[order[0]]), float(keys[order[1]])
        sbest = min(range(n), key=lambda i: (exact[i], i))
        cs = abs(b1) * 1.0078125 + 1e-30
        rr = R + np.sqrt(cs / lam)
        T = Lam * rr * rr + cs
        E = kappa * U * T
        for i in range(n):
            if exact[i] <= exact[sbest] + Fr(4.0 * E):
                err = abs(Fr(float(keys[i])) - exact[i])
                worst = max(worst, float(err) / (U * T))
                bad_bound += err > Fr(E)
        if b2 - b1 > 2.0 * E and gbest != sbest:
            bad_label += 1
    return worst, bad_bound, bad_label


@pytest.mark.parametrize("D", [3, 2])
@pytest.mark.parametrize("contract", [False, True])
def test_row_form_keys_are_within_the_bound_and_labels_exact(D, contract):
    worst_all = 0.0
    for seed in range(12):
        worst, bad_bound, bad_label = run_case(D, seed, KAPPA, contract)
        assert bad_bound == 0 and bad_label == 0, (seed, worst, bad_bound, bad_label)
        worst_all = max(worst_all, worst)
    assert worst_all < KAPPA


def test_a_bound_without_its_multiplier_is_violated():
    # planted mistake: kappa = 1 instead of 160
    assert any(run_case(3, seed, 1.0, False)[1] > 0 for seed in range(12))
