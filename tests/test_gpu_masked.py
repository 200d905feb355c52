"""Masked two-level discretisation on the GPU against the FP64 oracle
(oracle/masked.py): coarse labels and the fine grid's integer moments bit for
bit, the count of refined fine pixels exactly, the dual of eqs. (2.7)-(2.8) on
the fine grid within FP64 summation rounding."""
import numpy as np
import pytest

import oracle
from oracle import masked as om
from paper_2403_03571_gb300 import synth
from _gpu import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    require_gpu()
    from paper_2403_03571_gb300 import capi as c
    return c


def _weights(n, dim, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return 0.3 * g.standard_normal(n) * n ** (-2.0 / dim)


CASES = [
    (2, 40, (48, 48), 3, 1),
    (3, 60, (20, 20, 20), 2, 2),
    (2, 300, (61, 45), 2, 3),     # ragged, more than one seed chunk
    (3, 30, (10, 12, 9), 3, 4),   # ragged 3D
    (2, 25, (33, 31), 1, 5),      # r = 1: the coarse grid itself
    (2, 1, (16, 16), 4, 6),       # one seed: every pixel interior
    (3, 513, (9, 8, 7), 2, 7),    # three seed chunks
]


@pytest.mark.parametrize("dim,n,res,r,seed", CASES)
def test_masked_moments_match_oracle(capi, dim, n, res, r, seed):
    inst = synth.make_instance(dim, n, 8, seed)
    grid = synth.Grid(dim, res)
    w = _weights(n, dim, seed)
    ws = capi.Workspace(dim, n, grid.num_pixels)
    K = oracle.moment_width(dim)
    mom = torch.full((n, K), -1, dtype=torch.int64, device="cuda")
    lab = torch.full((grid.num_pixels,), -1, dtype=torch.int32, device="cuda")
    refined = torch.zeros(1, dtype=torch.int64, device="cuda")
    capi.apd_masked_moments(grid, r, dev(inst.x), dev(inst.A), dev(w), mom, lab, ws, refined=refined)
    assert ws.status() == capi.APD_OK
    hc, bnd, fine = om.labels(grid, r, inst.x, inst.A, w)
    assert np.array_equal(host(lab), hc)
    assert int(host(refined)[0]) == int(bnd.sum()) * r ** dim
    ref = oracle.moments(om.fine_grid(grid, r), fine, n)
    got = host(mom)
    assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]


@pytest.mark.parametrize("dim,n,res,r,seed", [(2, 80, (64, 50), 3, 8), (3, 40, (16, 14, 12), 2, 9)])
def test_masked_dual_matches_oracle(capi, dim, n, res, r, seed):
    inst = synth.make_instance(dim, n, 8, seed)
    grid = synth.Grid(dim, res)
    w = _weights(n, dim, seed)
    ws = capi.Workspace(dim, n, grid.num_pixels)
    lab = torch.empty(grid.num_pixels, dtype=torch.int32, device="cuda")
    g = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros(n, dtype=torch.float64, device="cuda")
    err = torch.zeros(1, dtype=torch.float64, device="cuda")
    capi.apd_masked_dual_value_grad(grid, r, dev(inst.x), dev(inst.A), dev(w), dev(inst.v), g, grad, err, lab, ws)
    assert ws.status() == capi.APD_OK
    g0, grad0, e0 = om.dual(grid, r, inst.x, inst.A, w, inst.v)
    assert abs(float(host(g)[0]) - g0) <= 1e-12 * max(1.0, abs(g0))
    assert np.allclose(host(grad), grad0, rtol=0, atol=1e-13)
    assert abs(float(host(err)[0]) - e0) <= 1e-10 * max(1.0, e0)


def test_masked_equals_the_fine_grid_across_a_straight_boundary(capi):
    # two seeds with A = I, boundary off the outer layer's corners: the masked
    # labelling equals the full fine grid's (oracle side), so do the moments
    dim, m, r = 3, 9, 8
    g = np.random.Generator(np.random.PCG64(7))
    c = np.full(dim, 0.5) + 0.05 * g.standard_normal(dim)
    d = np.ones(dim) + 0.05 * g.standard_normal(dim)
    x = np.stack([c - 0.1 * d, c + 0.1 * d])
    A = np.stack([np.eye(dim)] * 2)
    w = np.array([0.0, 0.02 * g.standard_normal()])
    coarse = synth.Grid.cube(dim, m)
    fg = om.fine_grid(coarse, r)
    ws = capi.Workspace(dim, 2, fg.num_pixels)
    mom = torch.zeros((2, 10), dtype=torch.int64, device="cuda")
    lab = torch.empty(coarse.num_pixels, dtype=torch.int32, device="cuda")
    capi.apd_masked_moments(coarse, r, dev(x), dev(A), dev(w), mom, lab, ws)
    full = torch.zeros((2, 10), dtype=torch.int64, device="cuda")
    capi.apd_cell_moments(fg, dev(x), dev(A), dev(w), full, ws)
    assert ws.status() == capi.APD_OK
    _, _, fine = om.labels(coarse, r, x, A, w)
    exact = oracle.assign(fg, x, A, w)
    assert np.array_equal(fine, exact)
    assert np.array_equal(host(full), oracle.moments(fg, exact, 2))
    assert np.array_equal(host(mom), host(full))
