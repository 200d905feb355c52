"""Anisotropic seeds (the paper's alpha laws of Section 3.2) through every
scoring arithmetic.

* alpha = 0.25 in 3D and 0.3 in 2D (max ||A||_F / min lambda_min ~ 7 and ~4):
  the tensor-core form runs, with candidate lists from the centre-form bounds;
  every label equals the oracle's, at W = 0 and at solve-sized weights.
* alpha = 0.3 in 3D (~12) and 0.7 (3D ~1600): a tensor-core request scores
  with the FP32 kernel (the conditioning read back after the seed preparation
  is above 10), which the launch count shows; the labels equal the oracle's.
"""
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


def _pc(capi, name):
    return {"fp32": capi.APD_FP32, "tc_tf32": capi.APD_TC_TF32, "tc_bf16": capi.APD_TC_BF16}[name]


def _labels(capi, inst, w, prec, prune=True):
    x, A, ww, _ = instance_tensors(inst, w)
    ws = capi.Workspace(inst.grid.dim, inst.n, inst.grid.num_pixels)
    ws.set_pruning(prune)
    lab = torch.empty(inst.grid.num_pixels, dtype=torch.int32, device="cuda")
    ws.profile(True)
    capi.apd_assign(inst.grid, x, A, ww, lab, ws, precision=_pc(capi, prec))
    assert ws.status() == capi.APD_OK
    _, _, _, launches = ws.profile_read()
    return host(lab), launches


@pytest.mark.parametrize("prec", ["fp32", "tc_tf32", "tc_bf16"])
@pytest.mark.parametrize("dim,n,alpha,wscale", [(3, 500, 0.25, 0.0), (3, 500, 0.25, 0.3), (2, 800, 0.3, 0.3),
                                                (3, 500, 0.3, 0.3)])
def test_anisotropic_labels_match_oracle(capi, dim, n, alpha, wscale, prec):
    inst = synth.runtime_test_instance(dim, n, alpha, False, 4242 + n)
    g = np.random.default_rng(n)
    w = wscale * g.standard_normal(n) * n ** (-2.0 / dim)
    lab, _ = _labels(capi, inst, w, prec)
    ref = oracle.assign(inst.grid, inst.x, inst.A, w)
    assert np.array_equal(lab, ref)


@pytest.mark.parametrize("alpha", [0.3, 0.7])
def test_ill_conditioned_tensor_core_request_scores_with_fp32(capi, alpha):
    inst = synth.runtime_test_instance(3, 300, alpha, False, 777)
    w = np.zeros(inst.n)
    lab_tc, l_tc = _labels(capi, inst, w, "tc_tf32")
    lab_fp, l_fp = _labels(capi, inst, w, "fp32")
    assert l_tc == l_fp  # no candidate pre-pass launched
    assert np.array_equal(lab_tc, oracle.assign(inst.grid, inst.x, inst.A, w))
    assert np.array_equal(lab_tc, lab_fp)
    # a well-conditioned set keeps the tensor-core path (its pre-pass adds launches)
    iso = synth.runtime_test_instance(3, 300, 0.0, False, 778)
    _, l_iso_tc = _labels(capi, iso, w, "tc_tf32")
    _, l_iso_fp = _labels(capi, iso, w, "fp32")
    assert l_iso_tc > l_iso_fp
