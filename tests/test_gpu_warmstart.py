"""Learned warm start on the GPU against the FP64 oracle (oracle/warmstart.py):
features, inference, the back-propagated gradient and the Adam step of the
hand-written kernels; training on a known target; and, with the stored
networks, what the prediction gains over the zero start on held-out
instances."""
import os

import numpy as np
import pytest

from oracle import warmstart as ow
import oracle
from paper_2403_03571_gb300 import synth
from _gpu import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    require_gpu()
    from paper_2403_03571_gb300 import capi as c
    return c


def _insts(dim, specs, seed):
    out = []
    for k, (n, m) in enumerate(specs):
        out.append(synth.make_instance(dim, n, m, seed + k))
    return out


def _random_net(dim, seed, scale=0.15):
    g = np.random.Generator(np.random.PCG64(seed))
    F, P = ow.n_features(dim), ow.n_params(dim)
    params = (g.normal(0, 1.0, P) * scale).astype(np.float32)
    norm = np.concatenate([g.normal(0, 0.5, F), np.exp(g.normal(0, 0.3, F))]).astype(np.float32)
    return params, norm


@pytest.mark.parametrize("dim,specs", [(2, [(300, 64), (5, 16), (1, 8), (1200, 64)]),
                                       (3, [(200, 16), (9, 8), (700, 16)])])
def test_features_and_prediction_match_oracle(capi, dim, specs):
    insts = _insts(dim, specs, 70 + dim)
    # a non-unit domain for one instance: the density scaling must use |O|
    insts[0].grid = synth.Grid(dim, insts[0].grid.res, lo=(0.0,) * dim, hi=(2.0,) + (1.0,) * (dim - 1))
    insts[0].x = insts[0].x * np.array([2.0] + [1.0] * (dim - 1))
    insts[0].v = insts[0].v * 2.0
    params, norm = _random_net(dim, 5)
    net = capi.WarmStart(dim, params, norm)
    x, A, w, v = (dev(a) for a in synth.concat(insts))
    counts = [i.n for i in insts]
    grids = [i.grid for i in insts]
    F = ow.n_features(dim)
    feats = torch.zeros((sum(counts), F), dtype=torch.float32, device="cuda")
    net.features(counts, grids, x, A, v, feats)
    wp = torch.zeros(sum(counts), dtype=torch.float64, device="cuda")
    net.predict(counts, grids, feats, wp)
    f_gpu, w_gpu = host(feats), host(wp)
    off = 0
    for inst in insts:
        ref = ow.features(inst.x, inst.A, inst.v, inst.grid.lo, inst.grid.hi)
        got = f_gpu[off:off + inst.n]
        # FP32 rounding of FP64 values; the volume-excess terms are differences
        # of sums and carry FP64 summation-order noise relative to their parts
        np.testing.assert_allclose(got, ref, rtol=2e-7, atol=1e-12)
        # inference from the GPU's own features (FP32 network vs FP64 oracle)
        pred = ow.predict(params, norm, got.astype(np.float64), inst.n, inst.grid.measure, dim)
        np.testing.assert_allclose(w_gpu[off:off + inst.n], pred, rtol=2e-4,
                                   atol=2e-5 * np.abs(pred).max())
        off += inst.n


@pytest.mark.parametrize("dim,B", [(2, 300), (3, 257), (2, 64)])
def test_gradient_matches_oracle(capi, dim, B):
    params, norm = _random_net(dim, 9 + dim)
    net = capi.WarmStart(dim, params, norm)
    g = np.random.Generator(np.random.PCG64(3))
    F, P = ow.n_features(dim), ow.n_params(dim)
    S = B + 40
    feats = g.normal(0.3, 1.5, (S, F)).astype(np.float32)
    targets = g.normal(0, 1, S).astype(np.float32)
    idx = g.choice(S, size=B, replace=False).astype(np.int32)
    grad = torch.zeros(P, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.train_step(dev(idx), dev(feats), dev(targets), 0.0, grad_out=grad, loss_out=loss)
    L_ref, g_ref = ow.loss_grad(params.astype(np.float64), norm.astype(np.float64),
                                feats[idx].astype(np.float64), targets[idx].astype(np.float64), dim)
    assert float(host(loss)[0]) == pytest.approx(L_ref * B, rel=1e-4)
    gg = host(grad)
    scale = np.abs(g_ref).max()
    np.testing.assert_allclose(gg, g_ref, rtol=1e-3, atol=1e-4 * scale)
    # lr = 0 leaves the parameters unchanged
    p2, _ = net.get()
    np.testing.assert_array_equal(p2, params)


def test_adam_first_step(capi):
    dim = 2
    params, norm = _random_net(dim, 21)
    net = capi.WarmStart(dim, params, norm)
    g = np.random.Generator(np.random.PCG64(4))
    F, P = ow.n_features(dim), ow.n_params(dim)
    feats = dev(g.normal(0, 1, (128, F)).astype(np.float32))
    targets = dev(g.normal(0, 1, 128).astype(np.float32))
    idx = dev(np.arange(128, dtype=np.int32))
    grad = torch.zeros(P, dtype=torch.float32, device="cuda")
    lr = 1e-3
    net.train_step(idx, feats, targets, lr, grad_out=grad)
    p1, _ = net.get()
    gg = host(grad).astype(np.float64)
    # first Adam step with bias correction: m_hat = g, v_hat = g^2
    expect = params - lr * gg / (np.abs(gg) + 1e-8)
    np.testing.assert_allclose(p1, expect, rtol=1e-5, atol=1e-7)


def test_training_fits_a_known_target(capi):
    # targets from a fixed random network of the same shape: the training kernels
    # must bring the loss down by an order of magnitude
    dim = 3
    F, P = ow.n_features(dim), ow.n_params(dim)
    teacher, tnorm = _random_net(dim, 31, scale=0.12)
    g = np.random.Generator(np.random.PCG64(8))
    S = 8192
    feats = g.normal(0, 1, (S, F))
    t, _ = ow.forward(teacher.astype(np.float64), tnorm.astype(np.float64), feats, dim)
    from paper_2403_03571_gb300 import warmstart
    net = capi.WarmStart(dim, warmstart.init_params(dim, 1))
    fd, td = dev(feats.astype(np.float32)), dev(t.astype(np.float32))
    net.fit_norm(fd)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    all_idx = dev(np.arange(S, dtype=np.int32))
    net.train_step(all_idx, fd, td, 0.0, loss_out=loss)
    l0 = float(host(loss)[0]) / S
    for ep in range(30):
        perm = dev(g.permutation(S).astype(np.int32))
        for k in range(0, S, 512):
            net.train_step(perm[k:k + 512], fd, td, 2e-3)
    net.train_step(all_idx, fd, td, 0.0, loss_out=loss)
    l1 = float(host(loss)[0]) / S
    assert l1 < 0.1 * l0, (l0, l1)


def test_solve_weights_warm_single_instance(capi):
    from paper_2403_03571_gb300 import warmstart
    inst = synth.make_instance(2, 200, 256, 91)
    params, norm = _random_net(2, 41, scale=0.05)
    net = capi.WarmStart(2, params, norm)
    x, A, w, v = (dev(a) for a in (inst.x, inst.A, inst.w, inst.v))
    ws = capi.Workspace(2, inst.n, inst.grid.num_pixels)
    w_out = torch.zeros_like(w)
    rc, info, used = capi.apd_solve_weights_warm(inst.grid, x, A, v, w_out, ws, net)
    assert rc in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE)
    assert used in (0, 1)
    _, _, err = oracle.dual(inst.grid, inst.x, inst.A, host(w_out), inst.v)
    assert err < 0.01
    # the judged start costs at most one extra evaluation over the better start's solve
    assert info.evaluations >= 2


@pytest.mark.parametrize("dim,count", [(2, 32), (3, 12)])
def test_trained_network_gain_on_held_out_instances(capi, dim, count):
    from paper_2403_03571_gb300 import warmstart
    net = warmstart.load(dim)
    if net is None:
        pytest.skip(f"no trained {dim}D network stored")
    insts = warmstart.draw(dim, count, warmstart.HELD_OUT_SEED[dim])
    x, A, w, v = warmstart.instance_arrays(insts)
    b = capi.Batch(dim, [i.grid for i in insts], [i.n for i in insts])
    w0 = torch.zeros_like(w)
    w_plain = torch.zeros_like(w)
    rc0, info0 = capi.apd_batch_solve_weights(b, x, A, w0, v, w_plain)
    wp = warmstart.predict(net, insts, x, A, v)
    w_warm = torch.zeros_like(w)
    rc1, info1, used = capi.apd_batch_solve_weights_judged(b, x, A, wp, v, w_warm)
    ok = (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE)
    assert all(i.status in ok for i in info0) and all(i.status in ok for i in info1)
    e0 = np.array([i.evaluations for i in info0], float)
    e1 = np.array([i.evaluations for i in info1], float)
    # the oracle confirms the warm-started volumes
    W = host(w_warm)
    off = 0
    for inst in insts[:4]:
        _, _, err = oracle.dual(inst.grid, inst.x, inst.A, W[off:off + inst.n], inst.v)
        assert err < 0.01
        off += inst.n
    print(f"{dim}D held-out: evaluations plain {e0.mean():.1f}, warm {e1.mean():.1f}, "
          f"prediction kept {sum(used)}/{count}")
    # the prediction beats the zero start by the judge's own measure (g~) on most
    # instances and, counting the judge's extra evaluation, shortens the solves
    assert sum(used) >= 0.75 * count, used
    assert e1.mean() < e0.mean(), (e0.mean(), e1.mean())


def test_pair_loss_gradient_matches_oracle(capi):
    dim = 3
    insts = _insts(dim, [(150, 16), (60, 8), (7, 8)], 88)
    params, norm = _random_net(dim, 13)
    net = capi.WarmStart(dim, params, norm)
    x, A, w, v = (dev(a) for a in synth.concat(insts))
    counts = [i.n for i in insts]
    S, F, P = sum(counts), ow.n_features(dim), ow.n_params(dim)
    feats = torch.zeros((S, F), dtype=torch.float32, device="cuda")
    knn = torch.zeros((S, 8), dtype=torch.int32, device="cuda")
    net.features(counts, [i.grid for i in insts], x, A, v, feats, knn=knn)
    # the neighbour rows equal the oracle's (per instance, offset to global rows)
    kn = host(knn)
    off = 0
    for inst in insts:
        ref = ow.knn_rows(inst.x)
        np.testing.assert_array_equal(kn[off:off + inst.n], np.where(ref >= 0, ref + off, -1))
        off += inst.n
    g = np.random.Generator(np.random.PCG64(6))
    targets = g.normal(0, 1, S).astype(np.float32)
    idx = dev(np.arange(S, dtype=np.int32))
    y_buf = torch.zeros(S, dtype=torch.float32, device="cuda")
    dy_buf = torch.zeros(S, dtype=torch.float32, device="cuda")
    grad = torch.zeros(P, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    mu = 0.05
    net.train_step_pairs(idx, feats, dev(targets), knn, y_buf, dy_buf, 0.0, mu=mu, grad_out=grad, loss_out=loss)
    L_ref, g_ref = ow.pair_loss_grad(params.astype(np.float64), norm.astype(np.float64),
                                     host(feats).astype(np.float64), targets.astype(np.float64), kn, dim, mu)
    assert float(host(loss)[0]) == pytest.approx(L_ref, rel=1e-4)
    np.testing.assert_allclose(host(grad), g_ref, rtol=2e-3, atol=2e-4 * np.abs(g_ref).max())
