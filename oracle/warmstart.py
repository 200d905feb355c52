"""FP64 CPU oracle of the learned warm start (features and the per-seed network).

TEST INFRASTRUCTURE ONLY: tests/ may import it; the library path never does.
It shares no code with the CUDA path: neighbours come from scipy's k-d tree,
the network and its gradient are plain numpy in FP64, written from the
definitions below.

The paper seeds the weight solve with W = 0 and motivates a better initial
guess; the predictor these functions describe is this project's addition, so
there is no passage to follow -- the definitions are:

* features of seed i of an instance with n seeds on the box [lo, hi] of
  measure |O|, s = n / |O|, lengths in units of s^(-1/D):  [v_i s, upper
  triangle of (A_i + A_i^T)/2, distances to the 8 nearest other seeds
  (ascending), target volumes of those seeds times s, distance to the nearer
  wall per axis, and for r = 2, 4, 8: c_r / E_r and (V_r s - c_r) / E_r with
  c_r the number and V_r the summed target volume of the other seeds within
  distance r, E_r = (unit-ball volume) r^D]; missing neighbours (n <= 8) give
  distance 4 and volume 0;
* network  y = w4 . relu(W3 relu(W2 relu(W1 z + b1) + b2) + b3) + b4,
  z = (f - mean) * inv_std, hidden width 64, flat parameter order
  W1 [64][F], b1, W2 [64][64], b2, W3 [64][64], b3, w4 [64], b4;
* prediction  w_i = y_i s^(-2/D);
* training losses over a batch: L = (1/B) sum_s (y_s - t_s)^2, and the
  neighbour-difference loss L = (1/(8B)) sum_i sum_{j in kNN(i)}
  ((y_i - y_j) - (t_i - t_j))^2 + (mu/B) sum_i (y_i - t_i)^2.

Pins (tests/test_oracle_warmstart.py): the k-d tree neighbours and ball counts
against a brute-force distance matrix; the wall distances and scale invariance;
the gradient against central finite differences of the FP64 loss; the
parameter counts against the layer sizes.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

H = 64
KNN = 8
RADII = (2.0, 4.0, 8.0)


def n_features(dim: int) -> int:
    return 1 + dim * (dim + 1) // 2 + 2 * KNN + dim + 2 * len(RADII)


def n_params(dim: int) -> int:
    F = n_features(dim)
    return H * F + H + 2 * (H * H + H) + H + 1


def features(x, A, v, lo=None, hi=None) -> np.ndarray:
    """Feature rows [n][F] of one instance on the box [lo, hi] (default unit box), FP64."""
    x = np.asarray(x, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    n, dim = x.shape
    lo = np.zeros(dim) if lo is None else np.asarray(lo, dtype=np.float64)[:dim]
    hi = np.ones(dim) if hi is None else np.asarray(hi, dtype=np.float64)[:dim]
    s = n / float(np.prod(hi - lo))
    ls = s ** (1.0 / dim)
    k = min(KNN, n - 1)
    dist = np.full((n, KNN), 4.0)
    vol = np.zeros((n, KNN))
    tree = cKDTree(x)
    if k > 0:
        d, idx = tree.query(x, k=k + 1)
        # column 0 is the point itself (distance 0); ties between neighbours at equal
        # distance are measure-zero for continuous positions
        dist[:, :k] = d[:, 1:] * ls
        vol[:, :k] = v[idx[:, 1:]] * s
    sym = 0.5 * (A + np.transpose(A, (0, 2, 1)))
    iu = np.triu_indices(dim)
    upper = sym[:, iu[0], iu[1]]
    walls = np.minimum(x - lo, hi - x) * ls
    ball = np.pi if dim == 2 else 4.0 * np.pi / 3.0
    scales = []
    for r in RADII:
        members = tree.query_ball_point(x, r / ls)
        c = np.array([len(m) - 1 for m in members], dtype=np.float64)
        V = np.array([v[m].sum() - v[i] for i, m in enumerate(members)])
        e = ball * r ** dim
        scales += [c / e, (V * s - c) / e]
    return np.concatenate([v[:, None] * s, upper, dist, vol, walls, np.stack(scales, 1)], axis=1)


def unpack(params, dim: int):
    """(W1, b1, W2, b2, W3, b3, w4, b4) views of the flat parameter vector."""
    F = n_features(dim)
    p = np.asarray(params, dtype=np.float64)
    shapes = [(H, F), (H,), (H, H), (H,), (H, H), (H,), (H,), (1,)]
    out, o = [], 0
    for sh in shapes:
        size = int(np.prod(sh))
        out.append(p[o:o + size].reshape(sh))
        o += size
    assert o == p.size
    return out


def forward(params, norm, feats, dim: int):
    """Network outputs y [S] and the activations (z, h1, h2, h3)."""
    F = n_features(dim)
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(params, dim)
    norm = np.asarray(norm, dtype=np.float64)
    z = (np.asarray(feats, dtype=np.float64) - norm[:F]) * norm[F:]
    h1 = np.maximum(z @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    h3 = np.maximum(h2 @ W3.T + b3, 0.0)
    y = h3 @ w4 + b4[0]
    return y, (z, h1, h2, h3)


def predict(params, norm, feats, n: int, measure: float, dim: int):  # measure = |O|
    """Predicted weights of one instance: y s^(-2/D)."""
    y, _ = forward(params, norm, feats, dim)
    return y * (n / measure) ** (-2.0 / dim)


def loss(params, norm, feats, targets, dim: int) -> float:
    y, _ = forward(params, norm, feats, dim)
    r = y - np.asarray(targets, dtype=np.float64)
    return float(np.mean(r * r))


def loss_grad(params, norm, feats, targets, dim: int):
    """(L, dL/dparams) by the chain rule, layer by layer (FP64)."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(params, dim)
    y, (z, h1, h2, h3) = forward(params, norm, feats, dim)
    B = y.shape[0]
    r = y - np.asarray(targets, dtype=np.float64)
    dy = 2.0 * r / B                       # dL/dy
    g_w4 = h3.T @ dy
    g_b4 = np.array([dy.sum()])
    d3 = np.outer(dy, w4) * (h3 > 0)       # dL/d(pre-activation of layer 3)
    g_W3, g_b3 = d3.T @ h2, d3.sum(0)
    d2 = (d3 @ W3) * (h2 > 0)
    g_W2, g_b2 = d2.T @ h1, d2.sum(0)
    d1 = (d2 @ W2) * (h1 > 0)
    g_W1, g_b1 = d1.T @ z, d1.sum(0)
    grad = np.concatenate([g.ravel() for g in (g_W1, g_b1, g_W2, g_b2, g_W3, g_b3, g_w4, g_b4)])
    return float(np.mean(r * r)), grad


def knn_rows(x) -> np.ndarray:
    """[n][8] rows of the 8 nearest other seeds (-1 where missing), distance order."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    out = np.full((n, KNN), -1, dtype=np.int64)
    k = min(KNN, n - 1)
    if k > 0:
        _, idx = cKDTree(x).query(x, k=k + 1)
        out[:, :k] = idx[:, 1:]
    return out


def pair_loss_grad(params, norm, feats, targets, knn, dim: int, mu: float = 0.0):
    """(L, dL/dparams) of the neighbour-difference loss; knn rows index feats."""
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(params, dim)
    y, (z, h1, h2, h3) = forward(params, norm, feats, dim)
    t = np.asarray(targets, dtype=np.float64)
    B = y.shape[0]
    ii = np.repeat(np.arange(B), KNN)
    jj = np.asarray(knn).reshape(-1)
    ok = jj >= 0
    ii, jj = ii[ok], jj[ok]
    r = (y[ii] - y[jj]) - (t[ii] - t[jj])
    scale = 1.0 / (B * KNN)
    e = y - t
    L = float(np.sum(r * r) * scale + mu * np.sum(e * e) / B)
    dy = 2.0 * mu * e / B
    np.add.at(dy, ii, 2.0 * r * scale)
    np.add.at(dy, jj, -2.0 * r * scale)
    g_w4 = h3.T @ dy
    g_b4 = np.array([dy.sum()])
    d3 = np.outer(dy, w4) * (h3 > 0)
    g_W3, g_b3 = d3.T @ h2, d3.sum(0)
    d2 = (d3 @ W3) * (h2 > 0)
    g_W2, g_b2 = d2.T @ h1, d2.sum(0)
    d1 = (d2 @ W2) * (h1 > 0)
    g_W1, g_b1 = d1.T @ z, d1.sum(0)
    grad = np.concatenate([g.ravel() for g in (g_W1, g_b1, g_W2, g_b2, g_W3, g_b3, g_w4, g_b4)])
    return L, grad


def pair_loss(params, norm, feats, targets, knn, dim: int, mu: float = 0.0) -> float:
    y, _ = forward(params, norm, feats, dim)
    t = np.asarray(targets, dtype=np.float64)
    B = y.shape[0]
    tot = mu * KNN * float(np.sum((y - t) ** 2))
    for i in range(B):
        for j in knn[i]:
            if j >= 0:
                r = (y[i] - y[j]) - (t[i] - t[j])
                tot += r * r
    return tot / (B * KNN)
