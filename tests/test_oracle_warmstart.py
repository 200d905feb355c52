"""Pins of the warm-start oracle (oracle/warmstart.py) against things other
than itself: brute-force neighbours, finite differences of the FP64 loss, the
layer sizes, and the scale invariance the feature definition implies."""
import numpy as np
import pytest

from oracle import warmstart as ow
from paper_2403_03571_gb300 import synth


def _instance(dim, n, seed):
    g = synth.rng(seed)
    x = synth.seeds_with_rejection(g, n, dim, 0.2)
    A = synth.aniso_2d_lognormal(g, n, 0.3) if dim == 2 else synth.aniso_3d_lognormal(g, n, 0.3)
    v = synth.volumes_lognormal(g, n, 0.5)
    return x, A, v


def test_parameter_counts_from_layer_sizes():
    # F -> 64 -> 64 -> 64 -> 1 with biases: F = 28 (2D), 32 (3D)
    assert ow.n_features(2) == 1 + 3 + 16 + 2 + 6 == 28
    assert ow.n_features(3) == 1 + 6 + 16 + 3 + 6 == 32
    assert ow.n_params(2) == 28 * 64 + 64 + 2 * (64 * 64 + 64) + 64 + 1 == 10241
    assert ow.n_params(3) == 10497


@pytest.mark.parametrize("dim,n", [(2, 300), (3, 200), (2, 5)])
def test_features_match_brute_force_neighbours(dim, n):
    x, A, v = _instance(dim, n, 3 + dim)
    f = ow.features(x, A, v)
    s = n / 1.0
    d = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1))
    np.fill_diagonal(d, np.inf)
    order = np.argsort(d, axis=1, kind="stable")
    k = min(8, n - 1)
    c = 1 + dim * (dim + 1) // 2
    np.testing.assert_allclose(f[:, 0], v * s, rtol=1e-15)
    np.testing.assert_allclose(f[:, c:c + k], np.take_along_axis(d, order[:, :k], 1) * s ** (1 / dim), rtol=1e-12)
    np.testing.assert_allclose(f[:, c + 8:c + 8 + k], v[order[:, :k]] * s, rtol=1e-15)
    assert np.all(f[:, c + k:c + 8] == 4.0) and np.all(f[:, c + 8 + k:c + 16] == 0.0)
    # A entries: upper triangle of the symmetric part, row by row
    iu = np.triu_indices(dim)
    np.testing.assert_allclose(f[:, 1:c], A[:, iu[0], iu[1]], rtol=1e-15)
    # wall distances and ball counts / volume excess from the distance matrix
    ls = s ** (1 / dim)
    o = c + 16
    np.testing.assert_allclose(f[:, o:o + dim], np.minimum(x, 1 - x) * ls, rtol=1e-15)
    ball = np.pi if dim == 2 else 4 * np.pi / 3
    for q, r in enumerate((2.0, 4.0, 8.0)):
        inside = d < r / ls
        cnt = inside.sum(1).astype(float)
        V = (inside * v[None, :]).sum(1)
        e = ball * r ** dim
        np.testing.assert_allclose(f[:, o + dim + 2 * q], cnt / e, rtol=1e-14)
        np.testing.assert_allclose(f[:, o + dim + 2 * q + 1], (V * s - cnt) / e, rtol=1e-12, atol=1e-14)


def test_features_scale_invariant():
    # x -> c x, v -> c^D v, |O| -> c^D |O| leaves every feature unchanged
    x, A, v = _instance(3, 150, 9)
    f1 = ow.features(x, A, v)
    c = 2.5
    shift = np.array([-1.0, 3.0, 0.5])
    f2 = ow.features(c * x + shift, A, c ** 3 * v, shift, shift + c)
    np.testing.assert_allclose(f1, f2, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_matches_finite_differences(dim):
    g = np.random.Generator(np.random.PCG64(11 + dim))
    F, P = ow.n_features(dim), ow.n_params(dim)
    # He-scale weights keep y = O(1), so the FP64 rounding of the loss stays far
    # below the finite-difference step's truncation error
    params = g.normal(0, 1.0, P) * 0.15
    norm = np.concatenate([g.normal(0, 0.1, F), np.exp(g.normal(0, 0.1, F))])
    feats = g.normal(0, 1, (24, F))
    targets = g.normal(0, 1, 24)
    L, grad = ow.loss_grad(params, norm, feats, targets, dim)
    assert L == pytest.approx(ow.loss(params, norm, feats, targets, dim), rel=1e-15)
    # every layer's weights and biases are represented in the sampled coordinates
    F64 = 64 * F
    bounds = [0, F64, F64 + 64, F64 + 64 + 4096, F64 + 128 + 4096, F64 + 128 + 8192, F64 + 192 + 8192,
              F64 + 256 + 8192, P]
    picks = np.concatenate([g.choice(np.arange(a, b), size=min(25, b - a), replace=False)
                            for a, b in zip(bounds[:-1], bounds[1:])])
    h = 1e-6
    tol_abs = 16 * 2.3e-16 * max(1.0, L) / h  # rounding of the two loss values over the step
    for p in picks:
        e = np.zeros(P)
        e[p] = h
        fd = (ow.loss(params + e, norm, feats, targets, dim) - ow.loss(params - e, norm, feats, targets, dim)) / (2 * h)
        assert fd == pytest.approx(grad[p], rel=2e-6, abs=tol_abs), p


def test_gradient_check_catches_a_dropped_relu_mask():
    # a plausible mistake (no ReLU derivative in the first hidden layer) must fail the pin above
    dim = 2
    g = np.random.Generator(np.random.PCG64(5))
    F, P = ow.n_features(dim), ow.n_params(dim)
    params = g.normal(0, 0.3, P)
    norm = np.concatenate([np.zeros(F), np.ones(F)])
    feats = g.normal(0, 1, (16, F))
    targets = g.normal(0, 1, 16)
    W1, b1, W2, b2, W3, b3, w4, b4 = ow.unpack(params, dim)
    y, (z, h1, h2, h3) = ow.forward(params, norm, feats, dim)
    dy = 2 * (y - targets) / 16
    d3 = np.outer(dy, w4) * (h3 > 0)
    d2 = (d3 @ W3) * (h2 > 0)
    d1_wrong = d2 @ W2                      # mask dropped
    gW1_wrong = d1_wrong.T @ z
    _, grad = ow.loss_grad(params, norm, feats, targets, dim)
    assert not np.allclose(gW1_wrong.ravel(), grad[:64 * F], rtol=1e-6)


def test_pair_loss_gradient_matches_finite_differences():
    dim = 2
    g = np.random.Generator(np.random.PCG64(17))
    F, P = ow.n_features(dim), ow.n_params(dim)
    params = g.normal(0, 1.0, P) * 0.15
    norm = np.concatenate([g.normal(0, 0.1, F), np.exp(g.normal(0, 0.1, F))])
    x = g.random((30, dim))
    feats = g.normal(0, 1, (30, F))
    targets = g.normal(0, 1, 30)
    knn = ow.knn_rows(x)
    mu = 0.05
    L, grad = ow.pair_loss_grad(params, norm, feats, targets, knn, dim, mu)
    # the vectorised loss equals the loop over pairs written out
    assert L == pytest.approx(ow.pair_loss(params, norm, feats, targets, knn, dim, mu), rel=1e-13)
    # without the anchor, a constant shift of the targets (the gauge) does not change the loss
    L0 = ow.pair_loss_grad(params, norm, feats, targets, knn, dim)[0]
    assert L0 == pytest.approx(ow.pair_loss_grad(params, norm, feats, targets + 3.0, knn, dim)[0], rel=1e-12)
    h = 1e-6
    tol_abs = 16 * 2.3e-16 * max(1.0, L) / h
    for p in g.choice(P, size=60, replace=False):
        e = np.zeros(P)
        e[p] = h
        fd = (ow.pair_loss(params + e, norm, feats, targets, knn, dim, mu)
              - ow.pair_loss(params - e, norm, feats, targets, knn, dim, mu)) / (2 * h)
        assert fd == pytest.approx(grad[p], rel=2e-6, abs=tol_abs), p


def test_knn_rows_match_brute_force():
    g = np.random.Generator(np.random.PCG64(2))
    x = g.random((50, 3))
    d = np.sqrt(((x[:, None] - x[None]) ** 2).sum(-1))
    np.fill_diagonal(d, np.inf)
    np.testing.assert_array_equal(ow.knn_rows(x), np.argsort(d, 1, kind="stable")[:, :8])
    assert np.all(ow.knn_rows(x[:3])[:, 2:] == -1)
