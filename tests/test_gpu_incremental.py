"""Incremental evaluations of the weight solve: the same results as full passes.

The weights enter every cost of eq. (2.1) linearly: between the recording's
weights w0 and w, C_k - C_a changes by exactly -(D_k - D_a), D = w - w0.  A
recording pass keeps each pixel's label a, runner-up b and certified bounds on
C_b - C_a and on every other seed's C_k - C_a; a re-decision pass keeps a
where the drift cannot close those margins, picks between a and b where only
they can win, and re-decides the rest over the tile's candidate list (FP64
where FP32 cannot decide), adding the label changes to the recorded moments.
The device chooses per pass between re-deciding and recording afresh.  Labels
and moments being the same as a full pass's, every evaluation's dual value
and gradient are too, so a whole solve (weights, evaluation counts, the stop
rule's error) must be bit-identical with and without incremental passes,
with and without graphs, through the plain, coarse-to-fine and Lloyd entry
points; the oracle confirms the stop rule at the result, and the profile
shows that scoring passes were skipped.  The grids here are small, so the
tests ask for incremental passes on every grid (mode 2)."""
import numpy as np
import pytest

import oracle
from paper_2403_03571_gb300 import synth
from _gpu import host, instance_tensors, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    require_gpu()
    from paper_2403_03571_gb300 import capi as c
    return c


def _run(capi, inst, kind, prec, incremental, graphs=True, eps=0.01):
    # incremental: 0 off, 1 default (grids of at least 2^20 pixels), 2 every grid
    x, A, w, v = instance_tensors(inst)
    ws = capi.Workspace(inst.grid.dim, inst.n, inst.grid.num_pixels)
    ws.set_pruning(True)
    ws.set_graphs(graphs)
    ws.set_incremental(incremental)
    ws.profile(True)
    opts = capi.solve_opts(eps=eps, precision=prec)
    x_out = torch.zeros_like(x)
    w_out = torch.zeros_like(w)
    mo = capi.multires_opts(2, 0.015, 200, min_cell_span=0)
    if kind == "solve":
        rc, info = capi.apd_solve_weights(inst.grid, x, A, w, v, w_out, ws, opts)
        x_out.copy_(x)
    elif kind == "multires":
        rc, info, _ = capi.apd_solve_weights_multires(inst.grid, x, A, w, v, w_out, ws, opts, mo)
        x_out.copy_(x)
    else:
        rc, info, _ = capi.apd_lloyd_multires(inst.grid, x, A, w, v, 2, x_out, w_out, ws, opts, mo)
    prof = ws.profile_read()
    return rc, info.as_dict(), host(x_out), host(w_out), prof


def _same(r0, r1):
    assert r1[0] == r0[0]
    for key in ("evaluations", "coarse_evaluations", "iterations", "solves"):
        assert r1[1][key] == r0[1][key], key
    assert r1[1]["max_rel_err"] == r0[1]["max_rel_err"]
    assert np.array_equal(r1[2], r0[2]) and np.array_equal(r1[3], r0[3])


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("kind", ["solve", "multires", "lloyd"])
def test_incremental_changes_nothing(capi, kind, prec):
    p = capi.APD_TC_TF32 if prec == "tf32" else capi.APD_TC_BF16
    inst = synth.make_instance(3, 300, 48, 31)
    r0 = _run(capi, inst, kind, p, incremental=False)
    r1 = _run(capi, inst, kind, p, incremental=2)
    _same(r0, r1)
    # every full pass times one scoring launch; incremental passes launch none
    assert r0[4][1] == r0[1]["evaluations"] + r0[1]["coarse_evaluations"]
    assert r1[4][1] < r0[4][1]
    if kind != "lloyd":
        _, _, err = oracle.dual(inst.grid, r1[2], inst.A, r1[3], inst.v)
        assert abs(err - r1[1]["max_rel_err"]) <= 1e-12


@pytest.mark.parametrize("graphs", [False, True])
def test_incremental_2d_and_anisotropic(capi, graphs):
    # 2D, anisotropic seeds (the alpha = 0.3 law, conditioning ~4)
    inst = synth.make_instance(2, 200, 192, 32, alpha=0.3)
    r0 = _run(capi, inst, "solve", capi.APD_TC_TF32, incremental=False, graphs=graphs)
    r1 = _run(capi, inst, "solve", capi.APD_TC_TF32, incremental=2, graphs=graphs)
    _same(r0, r1)
    _, _, err = oracle.dual(inst.grid, r1[2], inst.A, r1[3], inst.v)
    assert abs(err - r1[1]["max_rel_err"]) <= 1e-12


def test_incremental_tight_tolerance(capi):
    # a tight stop rule (about 1300 pixels per cell): long runs of small steps
    inst = synth.make_instance(3, 200, 64, 33)
    r0 = _run(capi, inst, "solve", capi.APD_TC_TF32, incremental=False, eps=0.004)
    r1 = _run(capi, inst, "solve", capi.APD_TC_TF32, incremental=2, eps=0.004)
    _same(r0, r1)
    assert r1[4][1] < r0[4][1]


def test_incremental_modes(capi):
    # mode 1 leaves grids below 2^20 pixels to full passes; other values are refused
    inst = synth.make_instance(3, 300, 48, 34)
    r0 = _run(capi, inst, "solve", capi.APD_TC_TF32, incremental=0)
    r1 = _run(capi, inst, "solve", capi.APD_TC_TF32, incremental=1)
    _same(r0, r1)
    assert r1[4][1] == r0[4][1] == r0[1]["evaluations"]
    ws = capi.Workspace(3, inst.n, inst.grid.num_pixels)
    for bad in (-1, 3):
        with pytest.raises(capi.ApdError):
            ws.set_incremental(bad)
