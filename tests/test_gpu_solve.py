"""Weight solve (Algorithm 2) and Lloyd (Algorithm 3) through the C ABI, judged
by the FP64 oracle: at the weights the GPU returns, the oracle's own
evaluation must meet the stop rule max_i |v_i - m_i|P|| / v_i < eps; centroids
must equal the oracle's discrete centroids at the GPU's (X, W)."""
import numpy as np
import pytest

import oracle
from paper_2403_03571_gb300 import synth
from _gpu import dev, host, instance_tensors, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    require_gpu()
    from paper_2403_03571_gb300 import capi as c
    return c


def _solve(capi, inst, eps=0.01, ws=None):
    x, A, w, v = instance_tensors(inst)
    ws = ws or capi.Workspace(inst.grid.dim, inst.n, inst.grid.num_pixels)
    w_out = torch.zeros(inst.n, dtype=torch.float64, device="cuda")
    rc, info = capi.apd_solve_weights(inst.grid, x, A, w, v, w_out, ws, capi.solve_opts(eps=eps))
    return rc, info, host(w_out)


def test_solve_2d_20_seeds_256(capi):
    inst = synth.workload_2d_20()
    rc, info, W = _solve(capi, inst)
    assert rc == capi.APD_OK, info.as_dict()
    _, _, err = oracle.dual(inst.grid, inst.x, inst.A, W, inst.v)
    assert err < 0.01
    assert abs(info.max_rel_err - err) <= 1e-12
    assert info.evaluations < 200


@pytest.mark.parametrize("dim,n,m,seed", [(2, 150, 200, 3), (3, 120, 48, 4)])
def test_solve_multiphase(capi, dim, n, m, seed):
    inst = synth.make_instance(dim, n, m, seed)
    rc, info, W = _solve(capi, inst)
    assert rc in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE), info.as_dict()
    g_w, _, err = oracle.dual(inst.grid, inst.x, inst.A, W, inst.v)
    assert err < 0.01
    g_0, _, _ = oracle.dual(inst.grid, inst.x, inst.A, np.zeros(n), inst.v)
    assert g_w >= g_0


def test_lloyd_step_centroids(capi):
    inst = synth.make_instance(2, 60, 128, 5)
    x, A, w, v = instance_tensors(inst)
    ws = capi.Workspace(2, 60, inst.grid.num_pixels)
    x_out = torch.zeros_like(x)
    w_out = torch.zeros_like(w)
    rc, info = capi.apd_lloyd_step(inst.grid, x, A, w, v, x_out, w_out, ws)
    assert rc in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE)
    W = host(w_out)
    lab = oracle.assign(inst.grid, inst.x, inst.A, W)
    ref = oracle.centroids(inst.grid, inst.x, lab)
    np.testing.assert_allclose(host(x_out), ref, rtol=0, atol=1e-12)
    _, _, err = oracle.dual(inst.grid, inst.x, inst.A, W, inst.v)
    assert err < 0.01


def test_lloyd_full(capi):
    inst = synth.make_instance(2, 40, 128, 6)
    x, A, w, v = instance_tensors(inst)
    ws = capi.Workspace(2, 40, inst.grid.num_pixels)
    x_out = torch.zeros_like(x)
    w_out = torch.zeros_like(w)
    rc, info = capi.apd_lloyd(inst.grid, x, A, w, v, 3, x_out, w_out, ws)
    assert rc in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE), info.as_dict()
    assert info.solves == 4
    X, W = host(x_out), host(w_out)
    _, _, err = oracle.dual(inst.grid, X, inst.A, W, inst.v)
    assert err < 0.01
    # X after round k is the centroid of the previous round's diagram: one more
    # oracle centroid step from (X, W) moves the seeds by less than a cell radius
    lab = oracle.assign(inst.grid, X, inst.A, W)
    C = oracle.centroids(inst.grid, X, lab)
    assert np.max(np.abs(C - X)) < 0.5 * 40 ** -0.5


def test_not_converged_reports_best(capi):
    inst = synth.make_instance(2, 80, 128, 7)
    x, A, w, v = instance_tensors(inst)
    ws = capi.Workspace(2, 80, inst.grid.num_pixels)
    w_out = torch.zeros_like(w)
    rc, info = capi.apd_solve_weights(inst.grid, x, A, w, v, w_out, ws,
                                      capi.solve_opts(eps=1e-9, max_evals=15))
    assert rc == capi.APD_NOT_CONVERGED
    assert info.evaluations <= 16
    _, _, err = oracle.dual(inst.grid, inst.x, inst.A, host(w_out), inst.v)
    assert abs(err - info.max_rel_err) <= 1e-12


@pytest.mark.parametrize("dim,n,m,seed", [(3, 300, 64, 12), (2, 400, 384, 13)])
def test_coarse_to_fine_solve(capi, dim, n, m, seed):
    inst = synth.make_instance(dim, n, m, seed)
    x, A, w, v = instance_tensors(inst)
    ws = capi.Workspace(dim, n, inst.grid.num_pixels)
    w_out = torch.zeros_like(w)
    rc, info, used = capi.apd_solve_weights_multires(inst.grid, x, A, w, v, w_out, ws,
                                                     mopts=capi.multires_opts(min_cell_span=0))
    assert rc in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE), info.as_dict()
    assert used == 0 and info.coarse_evaluations >= 1 and info.solves == 2
    _, _, err = oracle.dual(inst.grid, inst.x, inst.A, host(w_out), inst.v)
    assert err < 0.01 and abs(info.max_rel_err - err) <= 1e-12
    # the fine grid needs fewer evaluations from the coarse weights than from zero
    w2 = torch.zeros_like(w)
    rc2, plain = capi.apd_solve_weights(inst.grid, x, A, w, v, w2, ws)
    assert info.evaluations < plain.evaluations, (info.as_dict(), plain.as_dict())


def test_lloyd_coarse_to_fine(capi):
    from paper_2403_03571_gb300 import warmstart
    inst = synth.make_instance(3, 150, 40, 17)
    x, A, w, v = instance_tensors(inst)
    ws = capi.Workspace(3, inst.n, inst.grid.num_pixels)
    ws.set_pruning(True)
    x_out, w_out = torch.zeros_like(x), torch.zeros_like(w)
    rc, info, used = capi.apd_lloyd_multires(inst.grid, x, A, w, v, 3, x_out, w_out, ws,
                                             mopts=capi.multires_opts(2, 0.02, 60, min_cell_span=0),
                                             net=warmstart.load(3))
    assert rc in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE), info.as_dict()
    assert info.solves == 8 and info.coarse_evaluations >= 4
    X, W = host(x_out), host(w_out)
    # the returned weights solve the final positions (oracle's own evaluation) ...
    _, _, err = oracle.dual(inst.grid, X, inst.A, W, inst.v)
    assert err < 0.01
    # ... and the positions moved: they are the discrete centroids of an earlier round
    assert np.abs(X - inst.x).max() > 1e-3


def test_coarse_solve_skipped_for_small_cells(capi):
    # 300 seeds on 64^3: the 32^3 coarse grid has ~109 pixels per seed (< 8^3), so
    # the default options solve on the fine grid alone; min_cell_span = 0 forces
    # the coarse solve; both results meet the stop rule (oracle)
    inst = synth.make_instance(3, 300, 64, 12)
    x, A, w, v = instance_tensors(inst)
    ws = capi.Workspace(3, inst.n, inst.grid.num_pixels)
    for span, solves in ((None, 1), (0, 2)):
        w_out = torch.zeros_like(w)
        mo = capi.multires_opts() if span is None else capi.multires_opts(min_cell_span=span)
        rc, info, _ = capi.apd_solve_weights_multires(inst.grid, x, A, w, v, w_out, ws, mopts=mo)
        assert rc in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE), info.as_dict()
        assert info.solves == solves and (info.coarse_evaluations == 0) == (solves == 1)
        _, _, err = oracle.dual(inst.grid, inst.x, inst.A, host(w_out), inst.v)
        assert err < 0.01


def test_coarse_solve_stops_when_it_stalls(capi):
    # a coarse tolerance no coarse grid can reach: with coarse_stall_evals = 30 the
    # coarse solve stops after 30 evaluations without a 2 % better error instead of
    # running to its cap of 300,
    # and the fine solve still meets the stop rule (oracle)
    inst = synth.make_instance(2, 400, 384, 13)
    x, A, w, v = instance_tensors(inst)
    ws = capi.Workspace(2, inst.n, inst.grid.num_pixels)
    w_out = torch.zeros_like(w)
    rc, info, _ = capi.apd_solve_weights_multires(inst.grid, x, A, w, v, w_out, ws,
                                                  mopts=capi.multires_opts(2, 1e-6, 300, coarse_stall_evals=30))
    assert rc in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE), info.as_dict()
    assert info.solves == 2 and 30 <= info.coarse_evaluations < 300
    _, _, err = oracle.dual(inst.grid, inst.x, inst.A, host(w_out), inst.v)
    assert err < 0.01


@pytest.mark.parametrize("prec", ["fp32", "tc_tf32"])
def test_lloyd_coarse_history_carried(capi, prec):
    # the coarse solves of successive rounds continue one L-BFGS history: the
    # result still solves the final positions to 1 % (oracle), the run is
    # deterministic, and the main history is untouched by it (a plain solve
    # afterwards on the same workspace matches one on a fresh workspace)
    inst = synth.make_instance(3, 300, 48, 31)
    x, A, w, v = instance_tensors(inst)
    pc = capi.APD_FP32 if prec == "fp32" else capi.APD_TC_TF32
    opts = capi.solve_opts(eps=0.01, precision=pc)
    outs = []
    for _ in range(2):
        ws = capi.Workspace(3, inst.n, inst.grid.num_pixels)
        ws.set_pruning(True)
        x_out, w_out = torch.zeros_like(x), torch.zeros_like(w)
        rc, info, _ = capi.apd_lloyd_multires(inst.grid, x, A, w, v, 4, x_out, w_out, ws, opts,
                                              capi.multires_opts(2, 0.015, 200, carry_history=True,
                                                                 min_cell_span=0))
        assert rc in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE), info.as_dict()
        assert info.solves == 10
        outs.append((host(x_out), host(w_out), info.as_dict()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    X, W = outs[0][0], outs[0][1]
    _, _, err = oracle.dual(inst.grid, X, inst.A, W, inst.v)
    assert err < 0.01
    w_a = torch.zeros_like(w)
    capi.apd_solve_weights(inst.grid, x, A, w, v, w_a, ws, opts)
    ws2 = capi.Workspace(3, inst.n, inst.grid.num_pixels)
    ws2.set_pruning(True)
    w_b = torch.zeros_like(w)
    capi.apd_solve_weights(inst.grid, x, A, w, v, w_b, ws2, opts)
    assert np.array_equal(host(w_a), host(w_b))


def test_refining_solve_raises_the_resolution(capi):
    # Algorithm 2 with its step 4: on a 40^2 grid the smallest cell is a few
    # pixels, so 1 % is out of reach; the solve refines the grid of the same box,
    # restarts from the weights found, and converges on the finer grid
    inst = synth.make_instance(2, 60, 40, 23)
    x, A, w, v = instance_tensors(inst)
    ws = capi.Workspace(2, inst.n, 400 * 400)
    w_out = torch.zeros_like(w)
    rc, info, grid = capi.apd_solve_weights_refine(inst.grid, x, A, w, v, w_out, ws,
                                                   capi.solve_opts(max_evals=120),
                                                   capi.refine_opts(growth=1.5, max_rounds=4))
    assert rc in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE), info.as_dict()
    assert info.solves >= 2 and grid.res[0] > 40 and grid.res[0] == grid.res[1]
    assert grid.lo == inst.grid.lo and grid.hi == inst.grid.hi and grid.num_pixels <= 400 * 400
    # eq. (2.10) for the smallest target volume drives the first refinement
    need = 4.0 / (0.01 * inst.v.min())
    assert grid.num_pixels >= min(need, 400 * 400) * 0.999 or grid.num_pixels >= 1.5 ** 2 * 40 * 40
    # the oracle confirms the 1 % rule on the final grid
    _, _, err = oracle.dual(grid, inst.x, inst.A, host(w_out), inst.v)
    assert err < 0.01 and abs(info.max_rel_err - err) <= 1e-12
    # a cap below the next grid keeps the first grid and reports its status
    w2 = torch.zeros_like(w)
    rc2, info2, grid2 = capi.apd_solve_weights_refine(inst.grid, x, A, w, v, w2, ws,
                                                      capi.solve_opts(max_evals=60),
                                                      capi.refine_opts(max_res=(40, 40, 0)))
    assert grid2.res == (40, 40) and info2.solves == 1
    assert rc2 in (capi.APD_NOT_CONVERGED, capi.APD_WARN_TOL_INFEASIBLE)
