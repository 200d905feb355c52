"""The closed form the masked kernel adds for an interior coarse pixel, checked
on the CPU against direct sums over its r^D fine pixels.

Coarse pixel K (U = 2K + 1 per axis) covers the fine indices k = r K + j,
j = 0..r-1, whose odd coordinates u = 2k + 1 are r U - (r - 1) + 2j: they sum
to r^2 U with squares summing to r^3 U^2 + (r^3 - r) / 3.  Hence
    count = r^D,  sum u_a = r^(D+1) U_a,  sum u_a u_b = r^(D+2) U_a U_b (a != b),
    sum u_a^2 = r^(D+2) U_a^2 + r^D (r^2 - 1) / 3,
in the word order of the moments (count, sum u, upper triangle of sum u u^T)."""
import itertools

import pytest


def closed_form(K, r, D):
    rD, r2 = r ** D, r * r
    U = [2 * k + 1 for k in K]
    val = [rD] + [rD * r * U[a] for a in range(D)]
    for a in range(D):
        for b in range(a, D):
            val.append(rD * r2 * U[a] * U[b] + (rD * (r2 - 1) // 3 if a == b else 0))
    return val


def direct(K, r, D):
    val = [0] * (1 + D + D * (D + 1) // 2)
    for j in itertools.product(range(r), repeat=D):
        u = [2 * (K[a] * r + j[a]) + 1 for a in range(D)]
        val[0] += 1
        for a in range(D):
            val[1 + a] += u[a]
        e = 1 + D
        for a in range(D):
            for b in range(a, D):
                val[e] += u[a] * u[b]
                e += 1
    return val


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("r", [1, 2, 3, 4, 6, 9])
def test_block_moments_closed_form(D, r):
    for K in itertools.product((0, 1, 7, 40), repeat=D):
        assert closed_form(K, r, D) == direct(K, r, D), K


def test_diagonal_term_is_an_integer():
    # r^D (r - 1)(r + 1) holds the three consecutive integers (r - 1) r (r + 1)
    assert all((r ** d * (r * r - 1)) % 3 == 0 for r in range(1, 200) for d in (2, 3))
