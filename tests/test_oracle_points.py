"""Pins of the non-uniform-discretisation oracle (oracle/points.py) against the
grid oracle (independent C code) and a k-d tree."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from oracle import points as op
from paper_2403_03571_gb300 import synth


@pytest.mark.parametrize("dim,n,m,seed", [(2, 40, 48, 3), (3, 25, 14, 4)])
def test_pixel_centres_reproduce_the_grid_oracle(dim, n, m, seed):
    inst = synth.make_instance(dim, n, m, seed)
    g = np.random.Generator(np.random.PCG64(seed))
    w = 0.2 * g.standard_normal(n) * n ** (-2.0 / dim)
    y = oracle.pixel_centres(inst.grid)
    cell = oracle.pixel_volume(inst.grid)
    mass = np.full(y.shape[0], cell)
    lab = op.assign(y, inst.x, inst.A, w)
    ref = oracle.assign(inst.grid, inst.x, inst.A, w)
    assert np.array_equal(lab, ref)
    # moments: m = count |P|, S1 = |P| sum y, S2 = |P| sum y y^T, with y = lo + (h/2) u
    mo = op.moments(y, mass, lab, n)
    im = oracle.moments(inst.grid, ref, n).astype(np.float64)
    h = oracle.grid_steps(inst.grid)
    lo = np.asarray(inst.grid.lo, dtype=np.float64)
    cnt = im[:, 0]
    assert np.allclose(mo[:, 0], cnt * cell, rtol=1e-13, atol=0)
    for a in range(dim):
        s1 = lo[a] * cnt + 0.5 * h[a] * im[:, 1 + a]
        assert np.allclose(mo[:, 1 + a], cell * s1, rtol=1e-12, atol=1e-15)
    k = 1 + dim
    for a in range(dim):
        for b in range(a, dim):
            s2 = (lo[a] * lo[b] * cnt + 0.5 * h[b] * lo[a] * im[:, 1 + b] + 0.5 * h[a] * lo[b] * im[:, 1 + a]
                  + 0.25 * h[a] * h[b] * im[:, k])
            assert np.allclose(mo[:, k], cell * s2, rtol=1e-11, atol=1e-15)
            k += 1
    # the dual of eqs. (2.7)-(2.8)
    v = inst.v
    g1, grad1, e1 = op.dual(y, mass, inst.x, inst.A, w, v)
    g0, grad0, e0 = oracle.dual(inst.grid, inst.x, inst.A, w, v)
    assert abs(g1 - g0) <= 1e-12 * max(1.0, abs(g0))
    assert np.allclose(grad1, grad0, rtol=0, atol=1e-13)
    assert abs(e1 - e0) <= 1e-10 * max(1.0, e0)


@pytest.mark.parametrize("dim", [2, 3])
def test_euclidean_voronoi_is_the_nearest_seed(dim):
    # A = I, w = 0: the cells are Voronoi cells (a special case named in Section 2)
    g = np.random.Generator(np.random.PCG64(10 + dim))
    x = g.random((60, dim))
    y = g.random((3000, dim))
    A = np.broadcast_to(np.eye(dim), (60, dim, dim))
    lab = op.assign(y, x, A, np.zeros(60))
    _, nn = cKDTree(x).query(y)
    assert np.array_equal(lab, nn)


def test_moments_and_dual_by_hand():
    # two seeds on a line, three points with masses; costs written out
    x = np.array([[0.0, 0.0], [1.0, 0.0]])
    A = np.array([np.eye(2), np.diag([4.0, 1.0])])
    w = np.array([0.0, 0.5])
    y = np.array([[0.2, 0.0], [0.7, 0.0], [0.9, 1.0]])
    mass = np.array([0.5, 0.25, 0.25])
    # point 0: c0 = 0.04, c1 = 4*0.64 - 0.5 = 2.06 -> 0
    # point 1: c0 = 0.49, c1 = 4*0.09 - 0.5 = -0.14 -> 1
    # point 2: c0 = 0.81 + 1 = 1.81, c1 = 4*0.01 + 1 - 0.5 = 0.54 -> 1
    lab = op.assign(y, x, A, w)
    assert lab.tolist() == [0, 1, 1]
    mo = op.moments(y, mass, lab, 2)
    assert np.allclose(mo[0], [0.5, 0.1, 0.0, 0.02, 0.0, 0.0])
    assert np.allclose(mo[1], [0.5, 0.25 * 0.7 + 0.25 * 0.9, 0.25, 0.25 * (0.49 + 0.81), 0.25 * 0.9, 0.25])
    v = np.array([0.4, 0.6])
    g, grad, err = op.dual(y, mass, x, A, w, v)
    assert g == pytest.approx(0.6 * 0.5 + 0.5 * 0.04 + 0.25 * -0.14 + 0.25 * 0.54, abs=1e-15)
    assert np.allclose(grad, [-0.1, 0.1])
    assert err == pytest.approx(0.25)
