"""The L-BFGS direction kernels of the weight solve (Algorithm 2) against the
oracle's two-loop recursion.

The device stores the Gram entries s_i.y_j and y_i.y_j of its pairs when they
are pushed and runs the recursion on them, so its direction equals the
two-loop one in exact arithmetic and differs only by rounding; the bar is a
relative error of 1e-10 (FP64 throughout, well-conditioned pairs).  The
newest pair is taken only if it passes the curvature test; otherwise the
direction uses the older pairs with gamma = 1.  Both device paths are
checked: the direction kernels after plain pushes (a solve's first step and
restarts) and the push kernel that also forms the direction (every accepted
step), where the newest pair enters as y = g - (g - y) rounded in FP64."""
import numpy as np
import pytest

import oracle
from _gpu import require_gpu

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def capi():
    require_gpu()
    from paper_2403_03571_gb300 import capi as c
    return c


def pairs(rng, m, n):
    d = rng.uniform(0.5, 3.0, size=n)          # a diagonal-dominant curvature, as near a solve's optimum
    S = rng.standard_normal((m, n))
    Y = S * d + 0.05 * rng.standard_normal((m, n)) * np.sqrt(d)
    assert all(S[k] @ Y[k] > 0 for k in range(m))
    return S, Y


def as_pushed(Y, g, fused):
    if not fused:
        return Y
    Y = Y.copy()
    Y[-1] = g - (g - Y[-1])  # the fused path's newest pair, rounded as on the device
    return Y


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("n,hist", [(1, 1), (37, 3), (1000, 1), (1000, 10), (1000, 31), (10000, 10),
                                    (100003, 7)])
def test_direction_matches_two_loop(capi, n, hist, fused):
    rng = np.random.default_rng(n + hist)
    S, Y = pairs(rng, hist, n)
    g = rng.standard_normal(n)
    rc, p, gp = capi.apd_lbfgs_check(S, Y, g, fused)
    assert rc == capi.APD_OK
    Y = as_pushed(Y, g, fused)
    gamma = (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1])
    q = oracle.lbfgs_direction(S, Y, g, gamma)
    assert np.max(np.abs(p - q)) <= RTOL * np.max(np.abs(q))
    assert abs(gp - g @ q) <= RTOL * (np.abs(g) @ np.abs(q))
    assert gp < 0.0  # a descent direction of the minimised -g~


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("hist", [1, 4])
def test_rejected_newest_pair(capi, hist, fused):
    rng = np.random.default_rng(50 + hist)
    n = 500
    S, Y = pairs(rng, hist, n)
    Y[-1] = -Y[-1]                              # s.y < 0: fails the curvature test
    g = rng.standard_normal(n)
    rc, p, gp = capi.apd_lbfgs_check(S, Y, g, fused)
    assert rc == capi.APD_OK
    q = oracle.lbfgs_direction(S[:-1], Y[:-1], g, 1.0)
    assert np.max(np.abs(p - q)) <= RTOL * np.max(np.abs(q))
    assert abs(gp - g @ q) <= RTOL * (np.abs(g) @ np.abs(q))


def test_arguments(capi):
    g = np.ones(4)
    S = np.ones((32, 4))
    assert capi.apd_lbfgs_check(S, S, g)[0] == capi.APD_ERR_ARG   # hist > 31
    assert capi.apd_lbfgs_check(S[:0], S[:0], g)[0] == capi.APD_ERR_ARG
