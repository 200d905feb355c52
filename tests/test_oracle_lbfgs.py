"""Pins of the oracle's limited-memory BFGS direction (Algorithm 2's ascent).

The two-loop recursion (Nocedal and Wright, Algorithm 7.4) is checked against
things it does not share code with:
* the dense inverse-Hessian updates H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T
  from H0 = gamma I, applied oldest pair first, then p = -H g;
* the secant equation of the newest pair, H y = s;
* on a quadratic with Hessian Q and Q-conjugate steps s_k (y_k = Q s_k), n pairs
  give H = Q^-1 whatever gamma is (the hereditary property of BFGS);
* no pairs: p = -gamma g.
A copy with the loops' orders exchanged (a plausible slip) fails the dense pin."""
import numpy as np
import pytest

import oracle


def dense_direction(S, Y, g, gamma):
    n = g.shape[0]
    H = gamma * np.eye(n)
    I = np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / (s @ y)
        H = (I - rho * np.outer(s, y)) @ H @ (I - rho * np.outer(y, s)) + rho * np.outer(s, s)
    return -H @ g


def random_pairs(rng, m, n):
    Q = rng.standard_normal((n, n))
    Q = Q @ Q.T + n * np.eye(n)
    S = rng.standard_normal((m, n))
    Y = S @ Q + 0.1 * rng.standard_normal((m, n))
    assert all(S[k] @ Y[k] > 0 for k in range(m))
    return S, Y


@pytest.mark.parametrize("m,n", [(1, 3), (3, 7), (10, 20), (31, 40)])
def test_matches_dense_updates(m, n):
    rng = np.random.default_rng(100 + m)
    S, Y = random_pairs(rng, m, n)
    g = rng.standard_normal(n)
    gamma = (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1])
    p = oracle.lbfgs_direction(S, Y, g, gamma)
    q = dense_direction(S, Y, g, gamma)
    assert np.max(np.abs(p - q)) <= 1e-11 * np.max(np.abs(q))


def test_secant_equation_of_the_newest_pair():
    rng = np.random.default_rng(7)
    S, Y = random_pairs(rng, 6, 15)
    p = oracle.lbfgs_direction(S, Y, -Y[-1], 0.37)  # p = H y
    assert np.allclose(p, S[-1], rtol=0, atol=1e-12 * np.max(np.abs(S[-1])))


def test_quadratic_with_conjugate_steps_gives_the_inverse_hessian():
    rng = np.random.default_rng(8)
    n = 9
    B = rng.standard_normal((n, n))
    Q = B @ B.T + np.eye(n)
    _, V = np.linalg.eigh(Q)          # eigenvectors: orthogonal and Q-conjugate
    S = V.T * rng.uniform(0.5, 2.0, size=(n, 1))
    Y = S @ Q
    g = rng.standard_normal(n)
    for gamma in (1.0, 0.01, 50.0):
        p = oracle.lbfgs_direction(S, Y, g, gamma)
        assert np.allclose(p, -np.linalg.solve(Q, g), rtol=1e-9, atol=1e-12)


def test_no_pairs_is_scaled_steepest_descent():
    g = np.array([1.0, -2.0, 0.5])
    assert np.array_equal(oracle.lbfgs_direction(np.zeros((0, 3)), np.zeros((0, 3)), g, 2.0), -2.0 * g)


def test_planted_loop_order_slip_fails_the_dense_pin():
    def slipped(S, Y, g, gamma):  # the first loop run oldest to newest, the second newest to oldest
        q = np.array(g, dtype=np.float64)
        m = S.shape[0]
        rho = [1.0 / (S[k] @ Y[k]) for k in range(m)]
        alpha = [0.0] * m
        for k in range(m):
            alpha[k] = rho[k] * (S[k] @ q)
            q = q - alpha[k] * Y[k]
        r = gamma * q
        for k in range(m - 1, -1, -1):
            r = r + (alpha[k] - rho[k] * (Y[k] @ r)) * S[k]
        return -r

    rng = np.random.default_rng(9)
    S, Y = random_pairs(rng, 5, 12)
    g = rng.standard_normal(12)
    q = dense_direction(S, Y, g, 0.5)
    assert np.max(np.abs(slipped(S, Y, g, 0.5) - q)) > 1e-6 * np.max(np.abs(q))
    assert np.max(np.abs(oracle.lbfgs_direction(S, Y, g, 0.5) - q)) <= 1e-11 * np.max(np.abs(q))
