"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (Table 1, the M = 200 example of Section 3.2), special cases that
reduce to a library routine (Voronoi and power diagrams as nearest-neighbour
queries of scipy's cKDTree, eq. (2.1) cases (i)-(ii)), closed forms (bisector
of two seeds with equal A; the Apollonius sphere of the Moebius case (iv);
N = 1 sums over the grid), invariants (gauge, counts sum to J, concavity of
g~ giving an exact finite-difference sandwich around eq. (2.8)) and brute
force on tiny inputs.  Some tests plant a mistake in a copy of the oracle's
output and check that the pin rejects it.
"""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_2403_03571_gb300 import synth
from conftest import golden_rows


def _grid(dim, m):
    return synth.Grid.cube(dim, m)


def _identity(n, dim):
    return np.tile(np.eye(dim), (n, 1, 1))


# ----------------------------------------------------------------------------- resolution


def test_table1_reproduced():
    rows = golden_rows("table1_resolution.txt")
    assert len(rows) == 18
    for d, n, m in rows:
        assert oracle.resolution_table_entry(int(n), int(d), 0.01) == int(m), (d, n, m)


def test_table1_is_lower_bound_of_eq_2_9():
    # every printed M is within rounding of (N/eps)^(1/D)
    for d, n, m in golden_rows("table1_resolution.txt"):
        b = oracle.resolution_lower_bound(int(n), int(d), 0.01)
        assert abs(b - int(m)) <= 0.5


def test_choice_of_m_worked_example():
    for d, n, eps, m in golden_rows("choice_of_m_example.txt"):
        d, n, eps, m = int(d), int(n), float(eps), int(m)
        assert oracle.resolution_practical(d, 1.0 / n, eps) == m


def test_choice_of_m_is_smallest():
    for d in (2, 3):
        for vmin in (1e-3, 3.7e-4, 2e-5):
            m = oracle.resolution_practical(d, vmin, 0.01)
            assert 1.0 / m ** d <= 0.01 * vmin / 2 ** d * (1 + 1e-12)
            assert 1.0 / (m - 1) ** d > 0.01 * vmin / 2 ** d


# ----------------------------------------------------------------------------- grid


def test_pixel_centres_match_linspace():
    g = synth.Grid(3, (5, 7, 3), lo=(-1.0, 0.25, 2.0), hi=(1.0, 0.75, 5.0))
    y = oracle.pixel_centres(g)
    axes = [np.linspace(l + (h - l) / (2 * r), h - (h - l) / (2 * r), r)
            for l, h, r in zip(g.lo, g.hi, g.res)]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    ref = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-15)


# ----------------------------------------------------------------------------- Algorithm 1


@pytest.mark.parametrize("dim,m,n", [(2, 64, 37), (3, 20, 29)])
def test_voronoi_case_is_nearest_seed(dim, m, n):
    """eq. (2.1) case (i): A = I, w = 0 gives the Voronoi diagram."""
    g = _grid(dim, m)
    x = synth.rng(11).random((n, dim))
    lab, gap = oracle.assign(g, x, _identity(n, dim), np.zeros(n), with_gap=True)
    y = oracle.pixel_centres(g)
    dist, idx = cKDTree(x).query(y, k=2)
    clear = (dist[:, 1] ** 2 - dist[:, 0] ** 2) > 1e-12
    assert clear.mean() > 0.99
    np.testing.assert_array_equal(lab[clear], idx[clear, 0])


@pytest.mark.parametrize("dim,m,n", [(2, 64, 31), (3, 16, 23)])
def test_power_case_is_lifted_nearest_seed(dim, m, n):
    """eq. (2.1) case (ii): A = I is a power diagram; lifting each seed to
    (x_i, sqrt(wmax - w_i)) turns it into a nearest-neighbour query."""
    g = _grid(dim, m)
    r = synth.rng(12)
    x = r.random((n, dim))
    w = 0.02 * r.standard_normal(n)
    lab = oracle.assign(g, x, _identity(n, dim), w)
    lifted = np.concatenate([x, np.sqrt(w.max() - w)[:, None]], axis=1)
    y = oracle.pixel_centres(g)
    yl = np.concatenate([y, np.zeros((y.shape[0], 1))], axis=1)
    dist, idx = cKDTree(lifted).query(yl, k=2)
    clear = (dist[:, 1] ** 2 - dist[:, 0] ** 2) > 1e-12
    assert clear.mean() > 0.99
    np.testing.assert_array_equal(lab[clear], idx[clear, 0])
    # planted mistake: the weight entering with the wrong sign is caught
    bad = oracle.assign(g, x, _identity(n, dim), -w)
    assert np.any(bad[clear] != idx[clear, 0])


def _two_seed_case(dim, seed):
    r = synth.rng(seed)
    if dim == 2:
        A = synth.aniso_2d_lognormal(r, 1, 0.5)[0]
    else:
        A = synth.aniso_3d_lognormal(r, 1, 0.5)[0]
    x = r.random((2, dim))
    w = np.array([0.01, -0.02])
    return x, A, w


@pytest.mark.parametrize("dim,m", [(2, 128), (3, 24)])
def test_two_seeds_equal_A_bisector(dim, m):
    """Two seeds with the same A: cell 0 is the half-space
    2 y^T A (x1 - x0) <= x1^T A x1 - x0^T A x0 + w0 - w1."""
    g = _grid(dim, m)
    x, A, w = _two_seed_case(dim, 13)
    lab = oracle.assign(g, x, np.stack([A, A]), w)
    y = oracle.pixel_centres(g)
    lhs = 2 * y @ (A @ (x[1] - x[0]))
    rhs = x[1] @ A @ x[1] - x[0] @ A @ x[0] + w[0] - w[1]
    margin = rhs - lhs
    clear = np.abs(margin) > 1e-10
    np.testing.assert_array_equal(lab[clear], np.where(margin[clear] > 0, 0, 1))


def test_two_seeds_bisector_area_2d():
    """Area of cell 0 versus the exact clip of the unit square by the bisector
    half-plane; the discretisation error is at most perimeter * h."""
    m = 256
    g = _grid(2, m)
    x, A, w = _two_seed_case(2, 14)
    lab = oracle.assign(g, x, np.stack([A, A]), w)
    nvec = 2 * A @ (x[1] - x[0])
    c = x[1] @ A @ x[1] - x[0] @ A @ x[0] + w[0] - w[1]
    # clip polygon (unit square) by half-plane nvec . y <= c (Sutherland-Hodgman)
    poly = [(0.0, 0.0), (1.0, 0.0), (1.0, 1.0), (0.0, 1.0)]
    out = []
    for i in range(4):
        p, q = np.array(poly[i]), np.array(poly[(i + 1) % 4])
        fp, fq = nvec @ p - c, nvec @ q - c
        if fp <= 0:
            out.append(p)
        if fp * fq < 0:
            t = fp / (fp - fq)
            out.append(p + t * (q - p))
    if len(out) >= 3:
        P = np.array(out)
        area = 0.5 * abs(np.dot(P[:, 0], np.roll(P[:, 1], -1)) - np.dot(P[:, 1], np.roll(P[:, 0], -1)))
    else:
        area = 0.0
    got = np.count_nonzero(lab == 0) / m ** 2
    assert abs(got - area) <= 4.0 / m


def test_moebius_apollonius_sphere():
    """eq. (2.1) case (iv): A_i = c_i I, w = 0.  Cell 0 of two seeds is the ball
    |y - z| <= rho with z = (c0 x0 - c1 x1) / (c0 - c1),
    rho^2 = c0 c1 |x0 - x1|^2 / (c0 - c1)^2 (for c0 > c1)."""
    g = _grid(2, 200)
    x = np.array([[0.45, 0.55], [0.6, 0.4]])
    c0, c1 = 3.0, 1.0
    A = np.stack([c0 * np.eye(2), c1 * np.eye(2)])
    lab = oracle.assign(g, x, A, np.zeros(2))
    z = (c0 * x[0] - c1 * x[1]) / (c0 - c1)
    rho2 = c0 * c1 * np.sum((x[0] - x[1]) ** 2) / (c0 - c1) ** 2
    y = oracle.pixel_centres(g)
    s = np.sum((y - z) ** 2, axis=1) - rho2
    clear = np.abs(s) > 1e-10
    np.testing.assert_array_equal(lab[clear], np.where(s[clear] < 0, 0, 1))


def test_bruteforce_tiny_random():
    """Full cost matrix with numpy (einsum) and argmin (first minimum) on tiny inputs."""
    for dim, m, n, seed in [(2, 12, 9, 1), (3, 6, 11, 2), (2, 7, 1, 3)]:
        inst = synth.make_instance(dim, n, m, seed, reject_c=0.0)
        w = 0.01 * synth.rng(seed + 100).standard_normal(n)
        y = oracle.pixel_centres(inst.grid)
        d = y[None, :, :] - inst.x[:, None, :]
        C = np.einsum("nja,nab,njb->nj", d, inst.A, d) - w[:, None]
        ref = np.argmin(C, axis=0)
        lab, gap = oracle.assign(inst.grid, inst.x, inst.A, w, with_gap=True)
        clear = gap > 1e-12
        np.testing.assert_array_equal(lab[clear], ref[clear])
        if n > 1:
            Cs = np.sort(C, axis=0)
            np.testing.assert_allclose((Cs[1] - Cs[0])[clear] > 0, True)


def test_single_seed():
    g = _grid(3, 9)
    x = np.array([[0.3, 0.6, 0.2]])
    lab, gap = oracle.assign(g, x, _identity(1, 3), np.zeros(1), with_gap=True)
    assert np.all(lab == 0) and np.all(np.isinf(gap))


def test_exact_tie_lowest_index():
    """Two identical seeds: every pixel ties; the lowest index is taken."""
    g = _grid(2, 16)
    x = np.array([[0.3, 0.3], [0.3, 0.3], [0.8, 0.8]])
    lab, gap = oracle.assign(g, x, _identity(3, 2), np.zeros(3), with_gap=True)
    assert not np.any(lab == 1)
    assert np.all(gap[lab == 0] == 0.0)


def test_ids_subset_matches_full():
    inst = synth.make_instance(3, 40, 12, 5)
    full = oracle.assign(inst.grid, inst.x, inst.A, inst.w)
    ids = synth.rng(3).integers(0, inst.grid.num_pixels, 200)
    sub = oracle.assign_ids(inst.grid, inst.x, inst.A, inst.w, ids)
    np.testing.assert_array_equal(sub, full[ids])


# ----------------------------------------------------------------------------- moments


@pytest.mark.parametrize("dim,res", [(2, (13, 9)), (3, (7, 5, 6))])
def test_moments_closed_form_totals(dim, res):
    g = synth.Grid(dim, res)
    n = 17
    x = synth.rng(4).random((n, dim))
    lab = oracle.assign(g, x, _identity(n, dim), np.zeros(n))
    mo = oracle.moments(g, lab, n)
    J = g.num_pixels
    assert mo[:, 0].sum() == J
    # sum over the grid of u_d = 2k_d + 1 is (J / M_d) * M_d^2
    for d in range(dim):
        assert mo[:, 1 + d].sum() == J * res[d]
    # second moments: sum u_a^2 = (J/M_a) * M_a (4 M_a^2 - 1) / 3 ; cross: (J/(M_a M_b)) M_a^2 M_b^2
    s = 1 + dim
    for a in range(dim):
        for b in range(a, dim):
            if a == b:
                ref = (J // res[a]) * res[a] * (4 * res[a] ** 2 - 1) // 3
            else:
                ref = (J // (res[a] * res[b])) * res[a] ** 2 * res[b] ** 2
            assert mo[:, s].sum() == ref
            s += 1


def test_moments_match_bincount():
    g = synth.Grid(3, (6, 4, 5))
    n = 9
    lab = synth.rng(5).integers(0, n, g.num_pixels).astype(np.int32)
    mo = oracle.moments(g, lab, n)
    j = np.arange(g.num_pixels)
    k0, k1, k2 = j % 6, (j // 6) % 4, j // 24
    u = np.stack([2 * k0 + 1, 2 * k1 + 1, 2 * k2 + 1], axis=1)
    assert np.array_equal(mo[:, 0], np.bincount(lab, minlength=n))
    for d in range(3):
        assert np.array_equal(mo[:, 1 + d], np.bincount(lab, weights=u[:, d], minlength=n).astype(np.int64))
    assert np.array_equal(mo[:, 4], np.bincount(lab, weights=u[:, 0] ** 2, minlength=n).astype(np.int64))
    assert np.array_equal(mo[:, 8], np.bincount(lab, weights=u[:, 1] * u[:, 2], minlength=n).astype(np.int64))


# ----------------------------------------------------------------------------- dual


def _sum_k(m):          # sum_{k=0}^{m-1} (k + 1/2)
    return m * m / 2.0


def _sum_k2(m):         # sum_{k=0}^{m-1} (k + 1/2)^2
    return m * (4.0 * m * m - 1.0) / 12.0


@pytest.mark.parametrize("dim,res", [(2, (40, 30)), (3, (9, 11, 7))])
def test_single_seed_dual_closed_form(dim, res):
    """N = 1: g~ = v w + |P| sum_j q_j with sum_j (y-x)(y-x)^T in closed form."""
    lo = (0.1, -0.2, 0.0)[:dim]
    hi = (1.1, 0.5, 2.0)[:dim]
    g = synth.Grid(dim, res, lo=lo, hi=hi)
    r = synth.rng(6)
    x = np.array(lo) + (np.array(hi) - np.array(lo)) * r.random((1, dim))
    A = synth.aniso_2d_lognormal(r, 1, 0.6) if dim == 2 else synth.aniso_3d_lognormal(r, 1, 0.6)
    w = np.array([0.37])
    v = np.array([g.measure])
    gval, grad, err = oracle.dual(g, x, A, w, v)
    h = oracle.grid_steps(g)
    J = g.num_pixels
    S = np.zeros((dim, dim))
    c = np.array(lo) - x[0]
    lin = [res[a] * c[a] + h[a] * _sum_k(res[a]) for a in range(dim)]
    for a in range(dim):
        for b in range(dim):
            if a == b:
                sq = res[a] * c[a] ** 2 + 2 * c[a] * h[a] * _sum_k(res[a]) + h[a] ** 2 * _sum_k2(res[a])
                S[a, a] = sq * J / res[a]
            else:
                S[a, b] = lin[a] * lin[b] * J / (res[a] * res[b])
    P = float(np.prod(h))
    ref = (v[0] - J * P) * w[0] + P * np.sum(A[0] * S)
    assert abs(gval - ref) <= 1e-12 * abs(ref)
    assert abs(grad[0]) <= 1e-12 and err <= 1e-12


def test_dual_equals_min_form():
    """g~(W) = sum_i v_i w_i + |P| sum_j min_i C_ij (eq. (2.7) rewritten), from a
    numpy brute-force cost matrix."""
    inst = synth.make_instance(2, 15, 24, 7)
    w = 0.01 * synth.rng(8).standard_normal(15)
    gval, grad, err = oracle.dual(inst.grid, inst.x, inst.A, w, inst.v)
    y = oracle.pixel_centres(inst.grid)
    d = y[None] - inst.x[:, None]
    C = np.einsum("nja,nab,njb->nj", d, inst.A, d) - w[:, None]
    P = oracle.pixel_volume(inst.grid)
    ref = float(inst.v @ w + P * C.min(axis=0).sum())
    assert abs(gval - ref) <= 1e-13 * max(1.0, abs(ref))
    lab = np.argmin(C, axis=0)
    np.testing.assert_allclose(grad, inst.v - P * np.bincount(lab, minlength=15), atol=1e-15)


def test_gauge_invariance():
    inst = synth.make_instance(3, 25, 12, 9)
    w = 0.01 * synth.rng(10).standard_normal(25)
    g1, gr1, _ = oracle.dual(inst.grid, inst.x, inst.A, w, inst.v)
    g2, gr2, _ = oracle.dual(inst.grid, inst.x, inst.A, w + 0.123, inst.v)
    assert abs(g1 - g2) <= 1e-12
    np.testing.assert_array_equal(gr1, gr2)


def test_gradient_sandwich_concavity():
    """g~ is concave and piecewise linear; v - |P| m is a supergradient, so for
    every h > 0: (g(W + h e_i) - g(W)) / h <= grad_i <= (g(W) - g(W - h e_i)) / h."""
    inst = synth.make_instance(2, 12, 48, 15)
    w = 0.003 * synth.rng(16).standard_normal(12)
    g0, grad, _ = oracle.dual(inst.grid, inst.x, inst.A, w, inst.v)
    tol = 1e-13
    for i in range(12):
        for h in (1e-2, 1e-3, 1e-4):
            e = np.zeros(12)
            e[i] = h
            gp, _, _ = oracle.dual(inst.grid, inst.x, inst.A, w + e, inst.v)
            gm, _, _ = oracle.dual(inst.grid, inst.x, inst.A, w - e, inst.v)
            assert (gp - g0) / h <= grad[i] + tol / h
            assert grad[i] <= (g0 - gm) / h + tol / h


def test_gradient_equals_difference_quotient_below_flip():
    """For steps too small to move any pixel, the one-sided quotient equals
    v_i - |P| m_i up to rounding (sign of eq. (2.8))."""
    inst = synth.make_instance(2, 10, 40, 17)
    w = np.zeros(10)
    lab0 = oracle.assign(inst.grid, inst.x, inst.A, w)
    g0, grad, _ = oracle.dual(inst.grid, inst.x, inst.A, w, inst.v)
    for i in range(10):
        e = np.zeros(10)
        e[i] = 1e-9
        assert np.array_equal(oracle.assign(inst.grid, inst.x, inst.A, w + e), lab0)
        gp, _, _ = oracle.dual(inst.grid, inst.x, inst.A, w + e, inst.v)
        assert abs((gp - g0) / 1e-9 - grad[i]) <= 1e-5 * max(1e-3, abs(grad[i]))
    # planted mistake: a gradient with the opposite sign breaks the sandwich
    e = np.zeros(10)
    i = int(np.argmax(np.abs(grad)))
    e[i] = 1e-3
    gp, _, _ = oracle.dual(inst.grid, inst.x, inst.A, w + e, inst.v)
    gm, _, _ = oracle.dual(inst.grid, inst.x, inst.A, w - e, inst.v)
    wrong = -grad[i]
    assert not ((gp - g0) / 1e-3 <= wrong + 1e-12 and wrong <= (g0 - gm) / 1e-3 + 1e-12)


# ----------------------------------------------------------------------------- Algorithms 2, 3


def test_solve_hits_targets_and_is_dual_optimal():
    inst = synth.make_instance(2, 20, 128, 18)
    W, info = oracle.solve_weights(inst.grid, inst.x, inst.A, inst.v, eps=0.01)
    assert info["converged"]
    gW, grad, err = oracle.dual(inst.grid, inst.x, inst.A, W, inst.v)
    assert err < 0.01
    P = oracle.pixel_volume(inst.grid)
    lab = oracle.assign(inst.grid, inst.x, inst.A, W)
    m = np.bincount(lab, minlength=20)
    assert np.all(np.abs(inst.v - m * P) < 0.01 * inst.v)
    g0, _, _ = oracle.dual(inst.grid, inst.x, inst.A, np.zeros(20), inst.v)
    assert gW >= g0
    r = synth.rng(19)
    for _ in range(5):
        d = r.standard_normal(20)
        for t in (1e-3, 1e-2):
            gt, _, _ = oracle.dual(inst.grid, inst.x, inst.A, W + t * d, inst.v)
            assert gt <= gW + t * grad @ d + 1e-13


def test_single_seed_centroid_is_box_centre():
    g = synth.Grid(3, (7, 8, 9), lo=(0.0, -1.0, 2.0), hi=(1.0, 1.0, 3.0))
    x = np.array([[0.2, 0.1, 2.9]])
    lab = oracle.assign(g, x, _identity(1, 3), np.zeros(1))
    c = oracle.centroids(g, x, lab)
    np.testing.assert_allclose(c[0], [0.5, 0.0, 2.5], atol=1e-14)


def test_symmetric_lloyd_fixed_point():
    """Four seeds placed symmetrically, A = I, equal volumes: the centroids of the
    four quadrants are (1/4 or 3/4, 1/4 or 3/4)."""
    g = _grid(2, 64)
    x = np.array([[0.3, 0.3], [0.7, 0.3], [0.3, 0.7], [0.7, 0.7]])
    v = np.full(4, 0.25)
    X, W, infos = oracle.lloyd(g, x, _identity(4, 2), v, K=2)
    np.testing.assert_allclose(X, [[0.25, 0.25], [0.75, 0.25], [0.25, 0.75], [0.75, 0.75]], atol=1e-12)
    assert all(i["converged"] for i in infos)


def test_centroids_match_numpy_means():
    inst = synth.make_instance(2, 9, 30, 21)
    lab = oracle.assign(inst.grid, inst.x, inst.A, inst.w)
    y = oracle.pixel_centres(inst.grid)
    c = oracle.centroids(inst.grid, inst.x, lab)
    for i in range(9):
        if np.any(lab == i):
            np.testing.assert_allclose(c[i], y[lab == i].mean(axis=0), rtol=1e-13)


def test_empty_cell_keeps_seed():
    g = _grid(2, 8)
    x = np.array([[0.5, 0.5], [0.5, 0.5]])      # seed 1 ties everywhere and loses
    lab = oracle.assign(g, x, _identity(2, 2), np.zeros(2))
    assert np.all(lab == 0)
    c = oracle.centroids(g, np.array([[0.5, 0.5], [0.1, 0.9]]), lab)
    np.testing.assert_array_equal(c[1], [0.1, 0.9])
