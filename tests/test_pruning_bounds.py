"""The lower bounds the pruned FP32 scoring skips seeds and seed groups with,
restated in numpy with the kernel's FP32 roundings, checked on the CPU to lie
below the exact costs of every pixel centre of the warp's box (the property
the exactness of the pruning rests on; the GPU parity tests check the labels).

Bounds (cost relative to w_ref = max w, so that all costs are >= 0):
  seed  i: lam_i * dist(box, x_i)^2 * (1 - 1e-5) + rd(w_ref - w_i), with x_i as
           its FP32 offset from the tile centre and the box relative to it;
  group g: lam_g * dist(box, group box)^2 * (1 - 1e-5) + rd(w_ref - max w),
           boxes in absolute FP32 coordinates rounded outwards;
each distance shrunk by a slack of 1e-6 (|lo| + |hi| + |a| + |b|) per axis."""
import numpy as np

F32 = np.float32


def rd32(v):
    """Largest float32 <= v (v float64)."""
    f = np.float32(v)
    return np.nextafter(f, np.float32(-np.inf)) if np.float64(f) > v else f


def ru32(v):
    f = np.float32(v)
    return np.nextafter(f, np.float32(np.inf)) if np.float64(f) < v else f


def mul_rd(a, b):
    return rd32(np.float64(a) * np.float64(b))  # the product of two float32 is exact in float64


def fma32(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def spd(g, dim, cond):
    Q, _ = np.linalg.qr(g.standard_normal((dim, dim)))
    ev = np.exp(g.uniform(0.0, np.log(cond), dim))
    return (Q * ev) @ Q.T


def lam_lower(A):
    return rd32(np.linalg.eigvalsh(0.5 * (A + A.T))[0] * (1 - 1e-12))


def axis_dist(lo, hi, a_lo, a_hi):
    slack = F32(1e-6) * (abs(lo) + abs(hi) + abs(a_lo) + abs(a_hi))
    return max(F32(max(a_lo - hi, lo - a_hi)) - slack, F32(0.0))


def exact_costs(y, x, A, w, wref):
    d = y - x
    return np.einsum("pa,ab,pb->p", d, A, d) - w + wref


def test_seed_and_group_bounds_are_below_the_exact_costs():
    g = np.random.Generator(np.random.PCG64(2024))
    for case in range(300):
        dim = 2 + case % 2
        res = int(g.choice([64, 256, 1024]))
        h = 1.0 / res
        # a tile (16 pixels per axis) and one warp's block of pixel rows inside it
        t0 = g.integers(0, res // 16, dim) * 16
        kc = t0 + 8  # tile centre pixel index
        c = kc * h
        klo = t0 + g.integers(0, 8, dim)
        khi = np.minimum(klo + g.integers(0, 8, dim), t0 + 15)
        ks = np.stack(np.meshgrid(*[np.arange(klo[a], khi[a] + 1) for a in range(dim)], indexing="ij"), -1)
        y = (ks.reshape(-1, dim) + 0.5) * h
        # a group of seeds near or far from the tile, conditioning up to 1e3
        n = 32
        centre = c + g.normal(0.0, float(g.choice([0.01, 0.05, 0.3])), dim)
        x = centre + g.normal(0.0, 0.02, (n, dim))
        A = np.stack([spd(g, dim, float(g.choice([1.5, 30.0, 1000.0]))) for _ in range(n)])
        w = g.normal(0.0, 1e-3, n)
        wref = w.max() + abs(g.normal(0.0, 1e-3))
        # relative warp box (the kernel's FP32 products of half-integer offsets and h)
        h32 = F32(h)
        rlo = [F32((F32(klo[a] - kc[a]) + F32(0.5)) * h32) for a in range(dim)]
        rhi = [F32((F32(khi[a] - kc[a]) + F32(0.5)) * h32) for a in range(dim)]
        # absolute warp box, rounded outwards
        alo = [rd32((klo[a] + 0.5) * h) for a in range(dim)]
        ahi = [ru32((khi[a] + 0.5) * h) for a in range(dim)]
        costs = [exact_costs(y, x[i], A[i], w[i], wref) for i in range(n)]
        for i in range(n):
            xs = [F32(x[i][a] - c[a]) for a in range(dim)]
            d2 = F32(0.0)
            for a in range(dim):
                t = axis_dist(rlo[a], rhi[a], xs[a], xs[a])
                d2 = fma32(t, t, d2)
            lb = F32(mul_rd(mul_rd(lam_lower(A[i]), d2), F32(1.0) - F32(1e-5)) + rd32(wref - w[i]))
            assert np.float64(lb) <= costs[i].min(), (case, i, lb, costs[i].min())
        # the group bound over all 32 seeds
        glo = [rd32(x[:, a].min()) for a in range(dim)]
        ghi = [ru32(x[:, a].max()) for a in range(dim)]
        lam_g = min(lam_lower(A[i]) for i in range(n))
        d2 = F32(0.0)
        for a in range(dim):
            t = axis_dist(alo[a], ahi[a], glo[a], ghi[a])
            d2 = fma32(t, t, d2)
        lb = F32(mul_rd(mul_rd(lam_g, d2), F32(1.0) - F32(1e-5)) + rd32(wref - w.max()))
        assert np.float64(lb) <= min(cst.min() for cst in costs), case


def test_a_planted_mistake_in_the_bound_is_caught():
    # the same check with lambda_max in place of the lambda_min lower bound (a
    # plausible slip) must be violated by some anisotropic seed near the box
    g = np.random.Generator(np.random.PCG64(7))
    dim, h = 3, 1.0 / 256
    y = (np.stack(np.meshgrid(*[np.arange(0, 8)] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5) * h
    lo, hi = y.min(0), y.max(0)
    violated = 0
    for _ in range(200):
        x = lo + g.uniform(-0.05, 0.08, 3)
        A = spd(g, dim, 50.0)
        cst = exact_costs(y, x, A, 0.0, 0.0)
        t = np.maximum(np.maximum(lo - x, x - hi), 0.0)
        assert np.linalg.eigvalsh(A)[0] * (t @ t) <= cst.min() * (1 + 1e-12)
        violated += np.linalg.eigvalsh(A)[-1] * (t @ t) > cst.min()
    assert violated > 0
