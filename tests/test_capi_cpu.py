"""C-ABI checks that need no GPU: the library builds, loads and exports every
symbol include/apd.h declares; host-only entry points and argument checks that
return before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2403_03571_gb300 import build, capi
from conftest import ROOT, golden_rows


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "apd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(apd_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    declared = _declared_symbols()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(capi.EXPORTED)


def test_version_and_strings(lib):
    assert lib.apd_version() >= 100
    for code in (0, 1, 2, -1, -2, -3, -4, -5, -6):
        assert len(capi.status_string(code)) > 0


def test_choose_resolution_matches_eq_2_10(lib):
    for d, n, eps, m in golden_rows("choice_of_m_example.txt"):
        assert capi.apd_choose_resolution(int(d), 1.0 / int(n), float(eps), 1.0) == int(m)
    for d in (2, 3):
        for vmin in (1e-3, 3.7e-4, 2e-5, 0.05):
            assert capi.apd_choose_resolution(d, vmin, 0.01, 1.0) == oracle.resolution_practical(d, vmin, 0.01)
    assert capi.apd_choose_resolution(4, 0.1, 0.01, 1.0) == -1
    assert capi.apd_choose_resolution(2, 0.0, 0.01, 1.0) == -1


def test_argument_errors_before_cuda(lib):
    g = capi.ApdGrid()
    g.dim = 4
    s = capi.ApdSeeds()
    s.n = 3
    assert lib.apd_assign(ctypes.byref(g), ctypes.byref(s), 0, None, None, None, None) == capi.APD_ERR_ARG
    g.dim = 2
    g.res[0], g.res[1] = 8, 0
    g.hi[0], g.hi[1] = 1.0, 1.0
    assert lib.apd_assign(ctypes.byref(g), ctypes.byref(s), 0, None, None, None, None) == capi.APD_ERR_ARG
    g.res[1] = 8
    # seeds with null pointers
    assert lib.apd_assign(ctypes.byref(g), ctypes.byref(s), 0, ctypes.c_void_p(16), None, None,
                          None) == capi.APD_ERR_ARG
    # wait-limit knob: null workspace or a limit beyond 32 bits
    assert lib.apd_workspace_set_wait_limit(None, 5) == capi.APD_ERR_ARG
    h = ctypes.c_void_p()
    assert lib.apd_workspace_create(ctypes.byref(h), 5, 10, 100) == capi.APD_ERR_ARG
    assert lib.apd_workspace_create(ctypes.byref(h), 2, 0, 100) == capi.APD_ERR_ARG
    assert lib.apd_workspace_create(None, 2, 10, 100) == capi.APD_ERR_ARG
    lib.apd_workspace_destroy(None)
    # batches: bad dimension, count, null arrays, tile index out of range
    grids = (capi.ApdGrid * 2)(g, g)
    ns = (ctypes.c_int32 * 2)(5, 6)
    assert lib.apd_batch_create(ctypes.byref(h), 4, 2, grids, ns, -1) == capi.APD_ERR_ARG
    assert lib.apd_batch_create(ctypes.byref(h), 2, 0, grids, ns, -1) == capi.APD_ERR_ARG
    assert lib.apd_batch_create(ctypes.byref(h), 2, 2, None, ns, -1) == capi.APD_ERR_ARG
    assert lib.apd_batch_create(ctypes.byref(h), 2, 2, grids, None, -1) == capi.APD_ERR_ARG
    assert lib.apd_batch_create(ctypes.byref(h), 2, 2, grids, ns, 99) == capi.APD_ERR_ARG
    assert lib.apd_batch_create(None, 2, 2, grids, ns, -1) == capi.APD_ERR_ARG
    assert lib.apd_batch_solve_weights(None, None, None, None, None, None, None, None,
                                       None) == capi.APD_ERR_ARG
    assert lib.apd_batch_cell_moments(None, None, None, None, None, None) == capi.APD_ERR_ARG
    assert lib.apd_batch_kernel_launches(None) == -1
    lib.apd_batch_destroy(None)
    assert lib.apd_batch_set_pruning(None, 1) == capi.APD_ERR_ARG
    assert lib.apd_workspace_set_pruning(None, 1) == capi.APD_ERR_ARG
    assert lib.apd_batch_solve_weights_multires(None, None, None, None, None, None, None, None, 0, None, None,
                                                None) == capi.APD_ERR_ARG
    # coarse-to-fine and warm-start solves: a bad grid is rejected before any CUDA call
    g.dim = 4
    assert lib.apd_solve_weights_multires(ctypes.byref(g), ctypes.byref(s), None, None, None, None, None,
                                          None, None, None, None) == capi.APD_ERR_ARG
    assert lib.apd_lloyd_multires(ctypes.byref(g), ctypes.byref(s), None, 1, None, None, None, None, None,
                                  None, None, None, None) == capi.APD_ERR_ARG
    assert lib.apd_solve_weights_warm(ctypes.byref(g), ctypes.byref(s), None, None, None, None, None, None,
                                      None, None) == capi.APD_ERR_ARG
    # refining solve: options checked first, then the grid, before any CUDA call
    r = capi.ApdRefineOpts()
    lib.apd_refine_opts_default(ctypes.byref(r))
    assert (r.growth, list(r.max_res), r.max_rounds) == (1.5, [0, 0, 0], 4)
    assert lib.apd_solve_weights_refine(ctypes.byref(g), ctypes.byref(s), None, None, None, ctypes.byref(r), None,
                                        None, None, None) == capi.APD_ERR_ARG
    g.dim = 2
    for bad in ({"growth": 1.0}, {"growth": float("nan")}, {"max_rounds": -1}):
        rb = capi.ApdRefineOpts()
        lib.apd_refine_opts_default(ctypes.byref(rb))
        for k, val in bad.items():
            setattr(rb, k, val)
        assert lib.apd_solve_weights_refine(ctypes.byref(g), ctypes.byref(s), None, None, None, ctypes.byref(rb),
                                            None, None, None, None) == capi.APD_ERR_ARG
    assert lib.apd_solve_weights_refine(None, None, None, None, None, None, None, None, None,
                                        None) == capi.APD_ERR_ARG
    # the refinement rule on the host: eq. (2.10) for the smallest volume, or the growth factor
    gr = capi.ApdGrid()
    gr.dim = 2
    gr.res[0] = gr.res[1] = 40
    gr.lo[0] = gr.lo[1] = 0.0
    gr.hi[0] = gr.hi[1] = 1.0
    ro = capi.ApdRefineOpts()
    lib.apd_refine_opts_default(ctypes.byref(ro))
    nxt = capi.ApdGrid()
    vmin = 0.005
    assert lib.apd_refine_next_grid(ctypes.byref(gr), vmin, 0.01, ctypes.byref(ro), 0, ctypes.byref(nxt)) == 0
    f = max(1.5, (4.0 / (0.01 * vmin) / 1600.0) ** 0.5)
    assert nxt.res[0] == nxt.res[1] == int(np.ceil(40 * f)) == 283
    assert (nxt.lo[0], nxt.hi[1]) == (0.0, 1.0)
    assert lib.apd_refine_next_grid(ctypes.byref(gr), 0.5, 0.01, ctypes.byref(ro), 0, ctypes.byref(nxt)) == 0
    assert nxt.res[0] == 60  # eq. (2.10) already holds: the growth factor 1.5
    ro.max_res[0] = 200
    assert lib.apd_refine_next_grid(ctypes.byref(gr), vmin, 0.01, ctypes.byref(ro), 0, ctypes.byref(nxt)) == 1
    ro.max_res[0] = 0
    assert lib.apd_refine_next_grid(ctypes.byref(gr), vmin, 0.01, ctypes.byref(ro), 283 * 283 - 1,
                                    ctypes.byref(nxt)) == 1
    assert lib.apd_refine_next_grid(ctypes.byref(gr), 0.0, 0.01, ctypes.byref(ro), 0,
                                    ctypes.byref(nxt)) == capi.APD_ERR_ARG
    g3 = capi.ApdGrid()
    g3.dim = 3
    for d in range(3):
        g3.res[d], g3.lo[d], g3.hi[d] = 32, 0.0, 2.0
    assert lib.apd_refine_next_grid(ctypes.byref(g3), 1e-3, 0.01, ctypes.byref(ro), 0, ctypes.byref(nxt)) == 0
    f3 = max(1.5, (8.0 * 8.0 / (0.01 * 1e-3) / 32 ** 3) ** (1 / 3))
    assert nxt.res[0] == nxt.res[2] == int(np.ceil(32 * f3))
    # non-uniform discretisation: argument checks before any CUDA call
    pts = capi.ApdPoints()
    pts.dim, pts.count = 2, 10
    assert lib.apd_points_moments(ctypes.byref(pts), ctypes.byref(s), None, None, None, None) == capi.APD_ERR_ARG
    pts.y = pts.mass = 16  # non-null, never dereferenced on this path
    assert lib.apd_points_moments(ctypes.byref(pts), None, None, None, None, None) == capi.APD_ERR_ARG
    pts.dim = 4
    assert lib.apd_points_dual_value_grad(ctypes.byref(pts), ctypes.byref(s), None, None, None, None, None,
                                          None) == capi.APD_ERR_ARG
    pts.dim, pts.count = 2, 0
    assert lib.apd_points_moments(ctypes.byref(pts), ctypes.byref(s), None, None, None, None) == capi.APD_ERR_ARG
    assert lib.apd_points_moments(None, None, None, None, None, None) == capi.APD_ERR_ARG
    # warm-start network: sizes, argument checks without a device
    f, p = ctypes.c_int32(), ctypes.c_int32()
    assert lib.apd_warmstart_sizes(2, ctypes.byref(f), ctypes.byref(p)) == capi.APD_OK
    assert (f.value, p.value) == (28, 10241)
    assert lib.apd_warmstart_sizes(3, ctypes.byref(f), ctypes.byref(p)) == capi.APD_OK
    assert (f.value, p.value) == (32, 10497)
    assert lib.apd_warmstart_sizes(4, None, None) == capi.APD_ERR_ARG
    assert lib.apd_warmstart_create(ctypes.byref(h), 4, None, None) == capi.APD_ERR_ARG
    assert lib.apd_warmstart_create(ctypes.byref(h), 2, None, None) == capi.APD_ERR_ARG
    assert lib.apd_warmstart_train_step(None, 1, None, None, None, ctypes.c_float(0.0), None, None,
                                        None) == capi.APD_ERR_ARG
    assert lib.apd_warmstart_train_step_pairs(None, 1, None, None, None, None, None, None, ctypes.c_float(0.0),
                                              ctypes.c_float(0.0), None, None, None) == capi.APD_ERR_ARG
    lib.apd_warmstart_destroy(None)
    assert lib.apd_tensor_core_check(0, 3, ctypes.byref(ctypes.c_int32()),
                                     ctypes.byref(ctypes.c_float())) == capi.APD_ERR_ARG
    gp = ctypes.c_double()
    assert lib.apd_lbfgs_check(4, 0, None, None, None, 0, None, ctypes.byref(gp)) == capi.APD_ERR_ARG
    assert lib.apd_lbfgs_check(4, 32, None, None, None, 0, None, ctypes.byref(gp)) == capi.APD_ERR_ARG
    assert lib.apd_lbfgs_check(0, 1, None, None, None, 1, None, ctypes.byref(gp)) == capi.APD_ERR_ARG
    assert lib.apd_lbfgs_check(4, 1, None, None, None, 2, None, ctypes.byref(gp)) == capi.APD_ERR_ARG
    assert lib.apd_workspace_set_graphs(None, 1) == capi.APD_ERR_ARG
    assert lib.apd_workspace_set_incremental(None, 1) == capi.APD_ERR_ARG


def test_masked_argument_errors_before_cuda(lib):
    g = capi.ApdGrid()
    g.dim = 2
    g.res[0], g.res[1] = 8, 8
    g.hi[0], g.hi[1] = 1.0, 1.0
    s = capi.ApdSeeds()
    s.n = 3
    s.x = s.A = s.w = 16  # non-null, never dereferenced on this path
    lab = ctypes.c_void_p(16)
    mom = ctypes.c_void_p(16)
    one = ctypes.c_void_p(16)
    # refinement factor below one, null coarse labels, a fine grid of 2^31 pixels or more
    for r in (0, -2):
        assert lib.apd_masked_moments(ctypes.byref(g), r, ctypes.byref(s), mom, lab, None, None,
                                      None) == capi.APD_ERR_ARG
    assert lib.apd_masked_moments(ctypes.byref(g), 2, ctypes.byref(s), mom, None, None, None,
                                  None) == capi.APD_ERR_ARG
    assert lib.apd_masked_moments(ctypes.byref(g), 8192, ctypes.byref(s), mom, lab, None, None,
                                  None) == capi.APD_ERR_ARG
    assert lib.apd_masked_moments(ctypes.byref(g), 1 << 30, ctypes.byref(s), mom, lab, None, None,
                                  None) == capi.APD_ERR_ARG
    # no workspace, bad grid, bad seeds
    assert lib.apd_masked_moments(ctypes.byref(g), 2, ctypes.byref(s), mom, lab, None, None,
                                  None) == capi.APD_ERR_ARG
    assert lib.apd_masked_dual_value_grad(ctypes.byref(g), 2, ctypes.byref(s), one, one, None, one, lab, None,
                                          None) == capi.APD_ERR_ARG
    g.dim = 4
    assert lib.apd_masked_moments(ctypes.byref(g), 2, ctypes.byref(s), mom, lab, None, None,
                                  None) == capi.APD_ERR_ARG
    g.dim = 2
    s.n = 0
    assert lib.apd_masked_dual_value_grad(ctypes.byref(g), 2, ctypes.byref(s), one, one, None, one, lab, None,
                                          None) == capi.APD_ERR_ARG
    assert lib.apd_masked_moments(None, 2, None, None, None, None, None, None) == capi.APD_ERR_ARG
