"""The incremental evaluation's decision rules, restated in numpy and checked
against exact costs on the CPU (no GPU).

The weights enter every cost of eq. (2.1) linearly: from weights w0 to w the
cost of seed k changes by -(w_k - w0_k), so C_k - C_a changes by exactly
-(D_k - D_a), D = w - w0.  The recording scorer keeps per pixel its label a,
its runner-up b and certified bounds gl <= C_b - C_a <= gu, g3 <= C_k - C_a
(every other k); the re-decision kernel then keeps a, picks a or b by the
sign of an interval, or leaves the pixel to a full re-decision.  These tests
restate, in FP32 with the kernels' directed roundings, (1) the scorer's
top-three tournament (sorted pairs, sorted triples merged by
m-th smallest = min over i + j = m of max(A_i, B_j)) and its tracking of the
runner-up's step, and (2) the re-decision rule, and check them against sorted
values and exact argmins; planted mistakes in each must fail."""
import numpy as np
import pytest

F32 = np.float32


def ru(x):
    """x (float64) rounded up to float32."""
    x = np.asarray(x, dtype=np.float64)
    f = x.astype(F32)
    return np.where(f.astype(np.float64) >= x, f, np.nextafter(f, F32(np.inf)))


def rd(x):
    x = np.asarray(x, dtype=np.float64)
    f = x.astype(F32)
    return np.where(f.astype(np.float64) <= x, f, np.nextafter(f, F32(-np.inf)))


# ---------------------------------------------------------------- tournament
def pack(v):
    """Scores with the slot index in the five low mantissa bits (as the scorer)."""
    bits = v.astype(F32).view(np.uint32)
    return ((bits & ~np.uint32(31)) | np.arange(32, dtype=np.uint32)).view(F32)


def step_top3(v, c3_quad=None):
    """Three smallest of 32 packed scores, as the scorer's tournament forms them."""
    v = list(v)
    for e in range(16):
        lo, hi = min(v[2 * e], v[2 * e + 1]), max(v[2 * e], v[2 * e + 1])
        v[2 * e], v[2 * e + 1] = lo, hi
    for e in range(0, 32, 4):
        a1, a2, b1, b2 = v[e], v[e + 1], v[e + 2], v[e + 3]
        v[e] = min(a1, b1)
        v[e + 1] = min(max(a1, b1), min(a2, b2))
        v[e + 2] = (c3_quad or (lambda a1, a2, b1, b2: min(max(a1, b2), max(a2, b1))))(a1, a2, b1, b2)
    w = 8
    while w <= 32:
        for e in range(0, 32, w):
            a1, a2, a3 = v[e], v[e + 1], v[e + 2]
            b1, b2, b3 = v[e + w // 2], v[e + w // 2 + 1], v[e + w // 2 + 2]
            v[e] = min(a1, b1)
            v[e + 1] = min(a2, b2, max(a1, b1))
            v[e + 2] = min(min(a3, b3, max(a2, b1)), max(a1, b2))
        w *= 2
    return v[0], v[1], v[2]


def run_tournament(steps, c3_quad=None):
    k1 = k2 = k3 = F32(np.finfo(F32).max)
    bstep = bstep2 = 0
    for k, s in enumerate(steps):
        v0, v1, v2 = step_top3(pack(s), c3_quad)
        o1, o2 = k1, k2
        better = v0 < o1
        k1 = min(o1, v0)
        k2 = min(o2, v1, max(o1, v0))
        k3 = min(min(k3, v2, max(o2, v0)), max(o1, v1))
        bstep2 = bstep if k2 == o1 else (bstep2 if k2 == o2 else k)
        bstep = k if better else bstep
    return (k1, k2, k3), (bstep, bstep2)


@pytest.mark.parametrize("seed", range(6))
def test_top3_tournament_matches_sorting(seed):
    g = np.random.default_rng(seed)
    for trial in range(40):
        nsteps = int(g.integers(1, 5))
        steps = [g.standard_normal(32).astype(F32) * F32(g.choice([1e-3, 1.0, 1e3])) for _ in range(nsteps)]
        if trial % 5 == 0:  # repeated values across and within steps
            steps = [np.round(s, 1).astype(F32) for s in steps]
        packed = [pack(s) for s in steps]
        allv = np.concatenate(packed)
        (k1, k2, k3), (bs, bs2) = run_tournament(steps)
        want = np.sort(allv)[:3]
        assert (k1, k2, k3) == tuple(want)
        # the recorded steps hold the first and second smallest packed scores
        assert packed[bs][int(k1.view(np.uint32) & 31)] == k1
        assert packed[bs2][int(k2.view(np.uint32) & 31)] == k2


def test_top3_tournament_planted_mistake_fails():
    # a quad merge that takes the smaller of the two pairs' maxima as the third;
    # the three smallest scores sit in one group of four (where it matters)
    g = np.random.default_rng(7)
    bad = lambda a1, a2, b1, b2: min(a2, b2)  # noqa: E731
    fails = 0
    for _ in range(50):
        s = (10.0 + g.random(32)).astype(F32)
        q = 4 * int(g.integers(0, 8))
        s[q:q + 4] = g.permutation(np.array([1.0, 2.0, 3.0, 4.0], dtype=F32))
        got, _ = run_tournament([s], c3_quad=bad)
        good, _ = run_tournament([s])
        assert good == tuple(np.sort(pack(s))[:3])
        fails += got != good
    assert fails > 0


# ---------------------------------------------------------------- re-decision
def make_case(g, n=40, m=3000, slack=1e-6):
    """Exact costs at w0 (float64, isotropic 2D), records with outward slack."""
    x = g.random((n, 2))
    y = g.random((m, 2))
    w0 = g.normal(0, 0.01, n)
    C0 = ((y[:, None, :] - x[None, :, :]) ** 2).sum(-1) - w0[None, :]
    order = np.argsort(C0, axis=1)
    a, b, c = order[:, 0], order[:, 1], order[:, 2]
    r = np.arange(m)
    s = slack * g.random(m)
    gl = rd(C0[r, b] - C0[r, a] - s)
    gu = ru(C0[r, b] - C0[r, a] + s)
    g3 = rd(C0[r, c] - C0[r, a] - s)
    return x, y, w0, C0, a, b, gl, gu, g3


def redecide(a, b, gl, gu, g3, dw, flip=False):
    """The re-decision kernel's rule: label, or -1 (interval holds 0: FP32/FP64),
    or -2 (full re-decision).  dw = w - w0 (float64)."""
    dlo, dhi = rd(dw), ru(dw)                     # per-seed float intervals
    Dband = ru(dw.max() - dw.min())
    drift_hi = ru(dw.max())
    gap0 = np.maximum(np.minimum(gl, g3), F32(0))
    out = np.full(a.shape, -2, dtype=np.int64)
    keep = gap0 > Dband
    out[keep] = a[keep]
    rest = ~keep
    thr = ru(drift_hi.astype(np.float64) - dlo[a].astype(np.float64))
    pairable = rest & (g3 > thr)
    sgn = -1.0 if flip else 1.0
    s_hi = ru(sgn * (dhi[b].astype(np.float64) - dlo[a].astype(np.float64)))
    s_lo = rd(sgn * (dlo[b].astype(np.float64) - dhi[a].astype(np.float64)))
    if flip:
        s_hi, s_lo = np.maximum(s_hi, s_lo), np.minimum(s_hi, s_lo)
    lo = rd(gl.astype(np.float64) - s_hi.astype(np.float64))
    hi = ru(gu.astype(np.float64) - s_lo.astype(np.float64))
    out[pairable & (lo > 0)] = a[pairable & (lo > 0)]
    out[pairable & (hi < 0)] = b[pairable & (hi < 0)]
    out[pairable & ~(lo > 0) & ~(hi < 0)] = -1
    return out, gap0, Dband, thr


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("scale", [1e-4, 1e-3, 1e-2])
def test_redecision_rule_gives_the_exact_argmin(seed, scale):
    g = np.random.default_rng(100 + seed)
    x, y, w0, C0, a, b, gl, gu, g3 = make_case(g)
    dw = g.normal(0, scale, len(w0))
    out, gap0, Dband, thr = redecide(a, b, gl, gu, g3, dw)
    exact = np.argmin(C0 - dw[None, :], axis=1)
    decided = out >= 0
    # (a drift comparable with the cost gaps leaves most pixels to a full re-decision)
    assert decided.mean() > (0.5 if scale <= 1e-3 else 0.1)
    assert np.array_equal(out[decided], exact[decided])
    # every pixel whose label changed was re-decided
    assert np.all(out[exact != a] != a[exact != a])
    # the histogram bound of the full re-decisions (bins up to D's) counts them all
    full = out == -2
    bins = lambda v: (v.astype(F32).view(np.uint32) >> 21).astype(np.int64)  # noqa: E731
    eD = int(bins(np.array([Dband]))[0])
    hist_count = np.count_nonzero((g3 > 0) & (bins(g3) <= eD))
    assert hist_count >= np.count_nonzero(full & (g3 > 0))


def test_redecision_planted_sign_mistake_fails():
    # the drift difference taken as D_a - D_b instead of D_b - D_a
    g = np.random.default_rng(5)
    wrong = 0
    for _ in range(5):
        x, y, w0, C0, a, b, gl, gu, g3 = make_case(g)
        dw = g.normal(0, 3e-3, len(w0))
        out, *_ = redecide(a, b, gl, gu, g3, dw, flip=True)
        exact = np.argmin(C0 - dw[None, :], axis=1)
        d = out >= 0
        wrong += np.count_nonzero(out[d] != exact[d])
    assert wrong > 0
