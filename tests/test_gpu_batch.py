"""Batched solves through the C ABI (apd_batch_*), judged by the FP64 oracle.

Moments of every instance of a batch must equal the oracle's (labels are
exact, near ties rescored in FP64) for every tile shape of the persistent
kernel; a batched solve must meet the stop rule of Algorithm 2 for every
instance by the oracle's own evaluation at the returned weights."""
import numpy as np
import pytest

import oracle
from paper_2403_03571_gb300 import synth
from _gpu import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    require_gpu()
    from paper_2403_03571_gb300 import capi as c
    return c


def _mixed(dim, seed, specs, wscale=0.0):
    """Instances from (n, res) specs with the workload laws and random weights."""
    out = []
    for k, (n, res) in enumerate(specs):
        g = synth.rng(seed * 100 + k)
        x = synth.seeds_with_rejection(g, n, dim, 0.2)
        A = synth.aniso_2d_lognormal(g, n, 0.3) if dim == 2 else synth.aniso_3d_lognormal(g, n, 0.3)
        v = synth.volumes_lognormal(g, n, 0.5)
        w = wscale * g.standard_normal(n) * n ** (-2.0 / dim)
        out.append(synth.Instance(synth.Grid(dim, res), x, A, w, v, f"m{k}"))
    return out


SPECS_2D = [(37, (100, 77)), (300, (129, 300)), (1, (33, 17)), (5000, (40, 40)), (700, (64, 256)),
            (50, (256, 256))]
SPECS_3D = [(20, (19, 23, 17)), (300, (40, 33, 29)), (600, (16, 16, 16)), (1, (9, 5, 7))]


def _tensors(insts):
    x, A, w, v = synth.concat(insts)
    return dev(x), dev(A), dev(w), dev(v)


def _oracle_moments(insts):
    return np.concatenate([oracle.moments(i.grid, oracle.assign(i.grid, i.x, i.A, i.w), i.n) for i in insts])


@pytest.mark.parametrize("dim,specs", [(2, SPECS_2D), (3, SPECS_3D)])
def test_batch_moments_every_tile_shape(capi, dim, specs):
    insts = _mixed(dim, 7 + dim, specs, wscale=0.2)
    x, A, w, _ = _tensors(insts)
    ref = _oracle_moments(insts)
    K = oracle.moment_width(dim)
    total = sum(i.n for i in insts)
    _, _, shapes = capi.Batch(dim, [i.grid for i in insts], [i.n for i in insts], tile=0).tile_info()
    for tile in range(len(shapes)):
        b = capi.Batch(dim, [i.grid for i in insts], [i.n for i in insts], tile=tile)
        b.set_pruning(tile % 2 == 1)  # every other shape with seed-group pruning
        for _ in range(2):  # two calls in a row on one batch
            mom = torch.full((total, K), -3, dtype=torch.int64, device="cuda")
            assert capi.apd_batch_cell_moments(b, x, A, w, mom) == capi.APD_OK
            np.testing.assert_array_equal(host(mom), ref, err_msg=f"tile shape {shapes[tile]}")


def test_batch_autotune_picks_timed_shape(capi):
    insts = _mixed(2, 3, [(200, (300, 200)), (60, (128, 128)), (900, (256, 256))])
    x, A, w, _ = _tensors(insts)
    b = capi.Batch(2, [i.grid for i in insts], [i.n for i in insts])
    assert b.tile_info()[0] == -1
    mom = torch.zeros((sum(i.n for i in insts), 6), dtype=torch.int64, device="cuda")
    assert capi.apd_batch_cell_moments(b, x, A, w, mom) == capi.APD_OK
    tile, ms, shapes = b.tile_info()
    assert 0 <= tile < len(shapes)
    assert all(t > 0 for t in ms)
    assert ms[tile] == min(ms)
    np.testing.assert_array_equal(host(mom), _oracle_moments(insts))


def _check_solved(insts, W_all, infos, capi, eps=0.01):
    off = 0
    for inst, info in zip(insts, infos):
        W = W_all[off:off + inst.n]
        off += inst.n
        assert info.status in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE), info.as_dict()
        _, _, err = oracle.dual(inst.grid, inst.x, inst.A, W, inst.v)
        assert err < eps, (inst.name, err, info.as_dict())
        assert abs(info.max_rel_err - err) <= 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_batch_solve_meets_stop_rule(capi, dim):
    if dim == 2:
        insts = [synth.make_instance(2, n, m, 40 + k) for k, (n, m) in
                 enumerate([(20, 96), (150, 200), (60, 128), (400, 320), (1, 32), (90, 150)])]
    else:
        insts = [synth.make_instance(3, n, m, 50 + k) for k, (n, m) in
                 enumerate([(40, 32), (120, 48), (15, 24)])]
    x, A, w, v = _tensors(insts)
    b = capi.Batch(dim, [i.grid for i in insts], [i.n for i in insts])
    b.set_pruning(dim == 3)
    w_out = torch.zeros_like(w)
    rc, infos = capi.apd_batch_solve_weights(b, x, A, w, v, w_out, capi.solve_opts(eps=0.01))
    assert rc in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE)
    _check_solved(insts, host(w_out), infos, capi)
    # the same solve one instance at a time takes a comparable number of evaluations
    for inst, info in zip(insts, infos):
        ws = capi.Workspace(dim, inst.n, inst.grid.num_pixels)
        xs, As, ws_w, vs = dev(inst.x), dev(inst.A), dev(inst.w), dev(inst.v)
        wo = torch.zeros_like(ws_w)
        _, single = capi.apd_solve_weights(inst.grid, xs, As, ws_w, vs, wo, ws, capi.solve_opts(eps=0.01))
        assert info.evaluations <= 2 * single.evaluations + 10, (info.as_dict(), single.as_dict())
    # a second solve on the same batch (graph reused) from the solution converges at once
    rc2, infos2 = capi.apd_batch_solve_weights(b, x, A, w_out.clone(), v, w_out, capi.solve_opts(eps=0.01))
    assert all(i.evaluations == 1 for i in infos2)


def test_batch_errors(capi):
    insts = _mixed(2, 11, [(30, (200, 200)), (25, (250, 160))])
    x, A, w, v = _tensors(insts)
    b = capi.Batch(2, [i.grid for i in insts], [i.n for i in insts])
    Abad = A.clone()
    Abad[31] = torch.tensor([[1.0, 2.0], [2.0, 1.0]], dtype=torch.float64)  # second instance, seed 1
    w_out = torch.zeros_like(w)
    rc, infos = capi.apd_batch_solve_weights(b, x, Abad, w, v, w_out)
    assert rc == capi.APD_ERR_NOT_SPD
    assert infos[1].status == capi.APD_ERR_NOT_SPD
    assert infos[0].status in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE)
    rc, _ = capi.apd_batch_solve_weights(b, x, A, w, v, w_out, capi.solve_opts(precision=capi.APD_TC_TF32))
    assert rc == capi.APD_ERR_UNSUPPORTED
    # the batch is still usable after the errors
    rc, infos = capi.apd_batch_solve_weights(b, x, A, w, v, w_out)
    _check_solved(insts, host(w_out), infos, capi)


def test_batch_coarse_to_fine(capi):
    insts = [synth.make_instance(3, n, m, 60 + k) for k, (n, m) in enumerate([(200, 48), (80, 32), (400, 64)])]
    x, A, w, v = _tensors(insts)
    b = capi.Batch(3, [i.grid for i in insts], [i.n for i in insts])
    w_out = torch.zeros_like(w)
    rc, infos, used = capi.apd_batch_solve_weights_multires(b, x, A, w, v, w_out)
    assert rc in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE)
    assert all(i.coarse_evaluations >= 1 and i.solves == 2 for i in infos)
    _check_solved(insts, host(w_out), infos, capi)
    w2 = torch.zeros_like(w)
    _, plain = capi.apd_batch_solve_weights(b, x, A, w, v, w2)
    assert sum(i.evaluations for i in infos) < sum(i.evaluations for i in plain)
