"""apd_cell_moments_noalloc: the moments entry point for callers that cannot
allocate device memory (a fixed device-memory budget, a host framework whose
allocator owns all device memory, or a loop that cannot take cudaMalloc's
implicit synchronisation).  Its scratch is a static device array, so it is
checked through the C ABI against the FP64 oracle's moments and against the
workspace entry point apd_cell_moments, on two calls in a row (the second call
must not see the first one's state).

This file is collected last on purpose: it must pass alone in a fresh process
and after every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2403_03571_gb300 import synth
from _gpu import host, instance_tensors, require_gpu, torch

pytestmark = pytest.mark.gpu


def _moments_with_workspace(capi, inst):
    x, A, w, _ = instance_tensors(inst)
    ws = capi.Workspace(inst.grid.dim, inst.n, inst.grid.num_pixels)
    K = 1 + inst.grid.dim + inst.grid.dim * (inst.grid.dim + 1) // 2
    out = torch.full((inst.n, K), -1, dtype=torch.int64, device="cuda")
    capi.apd_cell_moments(inst.grid, x, A, w, out, ws)
    assert ws.status() == capi.APD_OK
    return host(out)


def _moments_no_alloc(capi, inst):
    x, A, w, _ = instance_tensors(inst)
    K = 1 + inst.grid.dim + inst.grid.dim * (inst.grid.dim + 1) // 2
    out = torch.full((inst.n, K), -1, dtype=torch.int64, device="cuda")
    rc = capi.apd_cell_moments_noalloc(inst.grid, x, A, w, out)
    assert rc == capi.APD_OK, capi.status_string(rc)
    return host(out)


def test_no_alloc_matches_workspace_entry_point_twice():
    require_gpu()
    from paper_2403_03571_gb300 import capi
    g = synth.rng(2024)
    # two different problems back to back: 3D with weights, then 2D with a single
    # seed chunk; integer moments must be identical to the workspace path
    a = synth.make_instance(3, 700, 40, 11)
    a.w = 0.2 * g.standard_normal(700) * 700 ** (-2.0 / 3)
    b = synth.make_instance(2, 150, 300, 12)
    b.w = 0.2 * g.standard_normal(150) / 150
    for inst in (a, b):
        got = _moments_no_alloc(capi, inst)
        ref = _moments_with_workspace(capi, inst)
        np.testing.assert_array_equal(got, ref)
        exact = oracle.moments(inst.grid, oracle.assign(inst.grid, inst.x, inst.A, inst.w), inst.n)
        np.testing.assert_array_equal(got, exact)
        assert got[:, 0].sum() == inst.grid.num_pixels


def test_no_alloc_rejects_sizes_beyond_its_limits():
    require_gpu()
    from paper_2403_03571_gb300 import capi
    big_n = synth.make_instance(2, 4097, 8, 13, reject_c=0.0)
    x, A, w, _ = instance_tensors(big_n)
    out = torch.zeros((4097, 6), dtype=torch.int64, device="cuda")
    assert capi.apd_cell_moments_noalloc(big_n.grid, x, A, w, out) == capi.APD_ERR_WORKSPACE
    small = synth.make_instance(2, 10, 8, 14)
    big_grid = synth.Grid(2, (2048, 1025))
    x, A, w, _ = instance_tensors(small)
    out = torch.zeros((10, 6), dtype=torch.int64, device="cuda")
    assert capi.apd_cell_moments_noalloc(big_grid, x, A, w, out) == capi.APD_ERR_WORKSPACE
