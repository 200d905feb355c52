"""Pins of the oracle's slab moments and moment-form dual (CPU).

* ``moments_ids`` over all pixels equals ``moments`` (pinned by closed forms and
  bincounts elsewhere), and over the slabs of a partition of the last axis it
  sums to ``moments`` exactly: the moments of disjoint pixel sets add up.
* ``dual_from_moments`` (eq. (2.7) rewritten through the integer moments) equals
  ``dual_from_labels`` (the direct FP64 sum of the costs, eq. (2.7) as printed)
  to 1e-12 relative, with the gradient and the error bit-equal, on 2D and 3D
  boxes that are not the unit box and with non-symmetric A inputs.  A planted
  mistake (the cross term dropped) is caught.
"""
import numpy as np
import pytest

import oracle
from paper_2403_03571_gb300 import synth


def _inst(dim, n, res, seed, lo=None, hi=None, wscale=0.2):
    g = synth.rng(seed)
    grid = synth.Grid(dim, res, lo=lo, hi=hi)
    lo_a, hi_a = np.array(grid.lo), np.array(grid.hi)
    x = lo_a + (hi_a - lo_a) * g.random((n, dim))
    A = synth.aniso_2d_lognormal(g, n, 0.4) if dim == 2 else synth.aniso_3d_lognormal(g, n, 0.4)
    A = A + 0.05 * g.standard_normal(A.shape) * np.triu(np.ones((dim, dim)), 1)  # non-symmetric input
    v = synth.volumes_lognormal(g, n, 0.5, grid.measure)
    w = wscale * g.standard_normal(n) * (grid.measure / n) ** (2.0 / dim)
    return grid, x, A, w, v


@pytest.mark.parametrize("dim,res,world", [(2, (37, 29), 3), (3, (13, 11, 17), 4), (3, (9, 8, 3), 5)])
def test_slab_moments_partition(dim, res, world):
    grid, x, A, w, v = _inst(dim, 40, res, 3 + world)
    n = x.shape[0]
    lab = oracle.assign(grid, x, A, w)
    full = oracle.moments(grid, lab, n)
    np.testing.assert_array_equal(oracle.moments_ids(grid, np.arange(grid.num_pixels), lab, n), full)
    total = np.zeros_like(full)
    edges = [res[-1] * r // world for r in range(world + 1)]
    for r in range(world):
        ids = oracle.slab_ids(grid, edges[r], edges[r + 1] - edges[r])
        total += oracle.moments_ids(grid, ids, oracle.assign_ids(grid, x, A, w, ids), n)
    np.testing.assert_array_equal(total, full)
    # a slab's count column is the bincount of its labels, its coordinate sums the
    # closed-form sums of u = 2k + 1 over its rows
    ids = oracle.slab_ids(grid, 1, 2)
    sl = oracle.moments_ids(grid, ids, oracle.assign_ids(grid, x, A, w, ids), n)
    per = grid.num_pixels // res[-1]
    assert sl[:, 0].sum() == 2 * per
    assert sl[:, dim].sum() == per * ((2 * 1 + 1) + (2 * 2 + 1))


@pytest.mark.parametrize("dim,res,lo,hi", [(2, (41, 33), (-1.0, 0.5), (2.0, 1.5)),
                                           (3, (17, 14, 12), (0.0, -2.0, 1.0), (1.0, 0.5, 2.5)),
                                           (3, (16, 16, 16), None, None)])
def test_dual_from_moments_equals_direct_sums(dim, res, lo, hi):
    grid, x, A, w, v = _inst(dim, 30, res, 17, lo, hi)
    lab = oracle.assign(grid, x, A, w)
    g1, grad1, err1, m1, _ = oracle.dual_from_labels(grid, x, A, w, v, lab)
    mom = oracle.moments(grid, lab, x.shape[0])
    g2, grad2, err2 = oracle.dual_from_moments(grid, x, A, w, v, mom)
    assert abs(g2 - g1) <= 1e-12 * abs(g1)
    np.testing.assert_array_equal(grad2, grad1)
    assert err2 == err1
    # planted mistake: dropping the cross term 2 c^T A D S1 changes g~ far beyond rounding
    bad = mom.copy()
    bad[:, 1:1 + dim] = 0
    g3, _, _ = oracle.dual_from_moments(grid, x, A, w, v, bad)
    assert abs(g3 - g1) > 1e-6 * abs(g1)
