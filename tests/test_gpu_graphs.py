"""Evaluation graphs of the weight solve: the same results with and without.

After a solve's first evaluation, every evaluation (trial weights, scoring,
rescoring, moments, the dual of eqs. (2.7)-(2.8), the read-back) is replayed
from a captured CUDA graph with only the trial step changing.  The arithmetic
is the same launches on the same data, so weights, positions, evaluation counts
and statuses must be bit-identical to the run without graphs, for every scoring
form, through the plain, coarse-to-fine and Lloyd entry points; the oracle
confirms the stop rule at the result."""
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


FORMS = [("fp32", False), ("fp32", True), ("tc_tf32", True), ("tc_bf16", False)]


def _prec(capi, name):
    return {"fp32": capi.APD_FP32, "tc_tf32": capi.APD_TC_TF32, "tc_bf16": capi.APD_TC_BF16}[name]


def _run(capi, inst, kind, prec, prune, graphs, profile=False):
    x, A, w, v = instance_tensors(inst)
    ws = capi.Workspace(inst.grid.dim, inst.n, inst.grid.num_pixels)
    ws.set_pruning(prune)
    ws.set_graphs(graphs)
    if profile:
        ws.profile(True)
    opts = capi.solve_opts(eps=0.01, precision=_prec(capi, prec))
    x_out = torch.zeros_like(x)
    w_out = torch.zeros_like(w)
    if kind == "solve":
        rc, info = capi.apd_solve_weights(inst.grid, x, A, w, v, w_out, ws, opts)
        x_out.copy_(x)
    elif kind == "multires":
        rc, info, _ = capi.apd_solve_weights_multires(inst.grid, x, A, w, v, w_out, ws, opts,
                                                      capi.multires_opts(2, 0.015, 200, min_cell_span=0))
        x_out.copy_(x)
    else:
        rc, info, _ = capi.apd_lloyd_multires(inst.grid, x, A, w, v, 2, x_out, w_out, ws, opts,
                                              capi.multires_opts(2, 0.015, 200, min_cell_span=0))
    prof = ws.profile_read() if profile else None
    return rc, info.as_dict(), host(x_out), host(w_out), prof


@pytest.mark.parametrize("prec,prune", FORMS)
@pytest.mark.parametrize("kind", ["solve", "multires", "lloyd"])
def test_graphs_change_nothing(capi, kind, prec, prune):
    inst = synth.make_instance(3, 300, 48, 21)
    r0 = _run(capi, inst, kind, prec, prune, graphs=False)
    r1 = _run(capi, inst, kind, prec, prune, graphs=True)
    assert r1[0] == r0[0]
    for key in ("evaluations", "coarse_evaluations", "iterations", "solves", "rescored_fp64"):
        assert r1[1][key] == r0[1][key], key
    assert r1[1]["max_rel_err"] == r0[1]["max_rel_err"]
    assert np.array_equal(r1[2], r0[2]) and np.array_equal(r1[3], r0[3])
    if kind != "lloyd":  # a Lloyd run ends with the seeds moved to the last cells' centroids
        _, _, err = oracle.dual(inst.grid, r1[2], inst.A, r1[3], inst.v)
        assert abs(err - r1[1]["max_rel_err"]) <= 1e-12


def test_graphs_2d_and_profiling(capi):
    inst = synth.make_instance(2, 400, 256, 22)
    r0 = _run(capi, inst, "solve", "tc_tf32", True, graphs=False, profile=True)
    r1 = _run(capi, inst, "solve", "tc_tf32", True, graphs=True, profile=True)
    assert np.array_equal(r1[3], r0[3]) and r1[1]["evaluations"] == r0[1]["evaluations"]
    # every full pass's scoring launch is timed either way (incremental passes
    # launch none); so are the launches counted
    ms0, n0, pairs0, kl0 = r0[4]
    ms1, n1, pairs1, kl1 = r1[4]
    assert n1 == n0 and 0 < n0 <= r0[1]["evaluations"] and pairs1 == pairs0 and kl1 == kl0
    assert ms1 > 0.0 and ms0 > 0.0
