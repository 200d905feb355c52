"""Non-uniform discretisation on the GPU against the FP64 oracle
(oracle/points.py): labels bit for bit, measure-weighted moments and the dual
of eqs. (2.7)-(2.8) within FP64 summation-order rounding."""
import numpy as np
import pytest

import oracle
from oracle import points as op
from paper_2403_03571_gb300 import synth
from _gpu import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    require_gpu()
    from paper_2403_03571_gb300 import capi as c
    return c


def _points(dim, count, seed, lo=0.0, hi=1.0):
    g = np.random.Generator(np.random.PCG64(seed))
    y = lo + (hi - lo) * g.random((count, dim))
    mass = g.uniform(0.5, 1.5, count) / count
    return y, mass


def _weights(n, dim, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return 0.3 * g.standard_normal(n) * n ** (-2.0 / dim)


def _check_moments(got, ref):
    scale = np.abs(ref).max(axis=0) + 1e-300
    assert np.all(np.abs(got - ref) <= 1e-12 * scale), np.abs(got - ref).max()


@pytest.mark.parametrize("dim,n,count,seed", [(2, 300, 20001, 1), (3, 257, 12345, 2), (2, 1, 777, 3),
                                             (3, 600, 5000, 4), (2, 50, 1, 7), (3, 513, 255, 8)])
def test_points_labels_and_moments_match_oracle(capi, dim, n, count, seed):
    inst = synth.make_instance(dim, n, 8, seed)
    w = _weights(n, dim, seed)
    y, mass = _points(dim, count, 100 + seed)
    ws = capi.Workspace(dim, n, 64)
    K = op.moment_width(dim)
    mom = torch.zeros((n, K), dtype=torch.float64, device="cuda")
    labels = torch.full((count,), -1, dtype=torch.int32, device="cuda")
    capi.apd_points_moments(dev(y), dev(mass), dev(inst.x), dev(inst.A), dev(w), mom, ws, labels=labels)
    assert ws.status() == capi.APD_OK
    ref = op.assign(y, inst.x, inst.A, w)
    got = host(labels)
    assert np.array_equal(got, ref), f"{np.count_nonzero(got != ref)} label mismatches"
    _check_moments(host(mom), op.moments(y, mass, ref, n))


def test_points_on_pixel_centres_equal_the_grid_path(capi):
    # the regular grid as a point set: labels equal apd_assign's, moments the integer moments converted
    inst = synth.make_instance(3, 200, 24, 9)
    w = _weights(200, 3, 9)
    y = oracle.pixel_centres(inst.grid)
    cell = oracle.pixel_volume(inst.grid)
    mass = np.full(y.shape[0], cell)
    ws = capi.Workspace(3, 200, inst.grid.num_pixels)
    lab_pts = torch.empty(y.shape[0], dtype=torch.int32, device="cuda")
    mom = torch.zeros((200, 10), dtype=torch.float64, device="cuda")
    capi.apd_points_moments(dev(y), dev(mass), dev(inst.x), dev(inst.A), dev(w), mom, ws, labels=lab_pts)
    lab_grid = torch.empty(y.shape[0], dtype=torch.int32, device="cuda")
    capi.apd_assign(inst.grid, dev(inst.x), dev(inst.A), dev(w), lab_grid, ws)
    assert ws.status() == capi.APD_OK
    assert np.array_equal(host(lab_pts), host(lab_grid))
    assert np.array_equal(host(lab_pts), oracle.assign(inst.grid, inst.x, inst.A, w))
    _check_moments(host(mom), op.moments(y, mass, host(lab_grid), 200))


@pytest.mark.parametrize("dim,n,count,seed", [(2, 150, 30000, 5), (3, 120, 20000, 6)])
def test_points_dual_matches_oracle(capi, dim, n, count, seed):
    inst = synth.make_instance(dim, n, 8, seed)
    w = _weights(n, dim, seed)
    y, mass = _points(dim, count, 200 + seed, lo=-0.5, hi=1.5)
    v = inst.v * mass.sum() / inst.v.sum()
    ws = capi.Workspace(dim, n, 64)
    g_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    e_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros(n, dtype=torch.float64, device="cuda")
    capi.apd_points_dual_value_grad(dev(y), dev(mass), dev(inst.x), dev(inst.A), dev(w), dev(v), g_out, grad,
                                    e_out, ws)
    assert ws.status() == capi.APD_OK
    g_ref, grad_ref, err_ref = op.dual(y, mass, inst.x, inst.A, w, v)
    gg = float(host(g_out)[0])
    assert abs(gg - g_ref) <= 1e-10 * max(1e-12, abs(g_ref)) + 1e-15
    np.testing.assert_allclose(host(grad), grad_ref, rtol=0, atol=1e-13)
    assert float(host(e_out)[0]) == pytest.approx(err_ref, rel=1e-10)


def test_points_exact_ties_go_to_the_lowest_index(capi):
    # two seeds with the same A and w, points on their bisector: equal FP64 costs
    x = np.array([[0.25, 0.5], [0.75, 0.5], [0.5, 0.9]])
    A = np.stack([np.eye(2)] * 3)
    w = np.zeros(3)
    y = np.stack([np.full(64, 0.5), np.linspace(0.0, 0.6, 64)], axis=1)
    mass = np.full(64, 1.0 / 64)
    ws = capi.Workspace(2, 3, 64)
    mom = torch.zeros((3, 6), dtype=torch.float64, device="cuda")
    labels = torch.full((64,), -1, dtype=torch.int32, device="cuda")
    capi.apd_points_moments(dev(y), dev(mass), dev(x), dev(A), dev(w), mom, ws, labels=labels)
    assert ws.status() == capi.APD_OK
    ref = op.assign(y, x, A, w)
    assert np.array_equal(host(labels), ref)
    assert (ref[y[:, 1] < 0.5] == 0).all()
