"""Pins of the masked two-level discretisation oracle (oracle/masked.py):
brute force on tiny grids (pure-Python loops over pixels, neighbourhoods and
seeds), the straight boundary of two seeds with equal A (where the masked
labelling equals the full fine grid's away from the outer layer, a fact of
convex geometry), and the special cases r = 1 and one seed."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import masked as om
from paper_2403_03571_gb300 import synth


def _weights(n, dim, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    return 0.3 * g.standard_normal(n) * n ** (-2.0 / dim)


def _brute_labels(res, lo, hi, r, x, A, w):
    """Steps 1-3 with loops: coarse labels, boundary flags, fine labels (fine linear order)."""
    D = len(res)
    n = len(w)

    def label(rs, k):
        y = [lo[a] + (k[a] + 0.5) * ((hi[a] - lo[a]) / rs[a]) for a in range(D)]
        best, bi = None, -1
        for i in range(n):
            d = [y[a] - x[i][a] for a in range(D)]
            q = 0.0
            for a in range(D):
                for b in range(D):
                    q = q + d[a] * A[i][a][b] * d[b]
            c = q - w[i]
            if best is None or c < best:
                best, bi = c, i
        return bi

    coarse = {k: label(res, k) for k in itertools.product(*[range(m) for m in res])}
    bnd = {}
    for k, lk in coarse.items():
        b = False
        for off in itertools.product((-1, 0, 1), repeat=D):
            nb = tuple(k[a] + off[a] for a in range(D))
            if all(0 <= nb[a] < res[a] for a in range(D)) and coarse[nb] != lk:
                b = True
        bnd[k] = b
    fres = [m * r for m in res]
    fine = {}
    for k in itertools.product(*[range(m) for m in fres]):
        parent = tuple(k[a] // r for a in range(D))
        fine[k] = label(fres, k) if bnd[parent] else coarse[parent]

    def linear(d, rs):
        out = np.empty(int(np.prod(rs)), dtype=np.int64)
        for k, v in d.items():
            j = 0
            for a in reversed(range(D)):
                j = j * rs[a] + k[a]
            out[j] = v
        return out

    return linear(coarse, res), linear(bnd, res).astype(bool), linear(fine, fres)


@pytest.mark.parametrize("dim,res,r,n,seed", [(2, (7, 5), 3, 6, 1), (3, (4, 3, 5), 2, 5, 2), (2, (6, 6), 1, 4, 3)])
def test_masked_labels_match_brute_force(dim, res, r, n, seed):
    inst = synth.make_instance(dim, n, 8, seed)
    grid = synth.Grid(dim, res, lo=(-0.1,) * dim, hi=(1.2,) * dim)
    w = _weights(n, dim, seed)
    hc, bnd, fine = om.labels(grid, r, inst.x, inst.A, w)
    bc, bb, bf = _brute_labels(res, grid.lo, grid.hi, r, inst.x.tolist(), inst.A.tolist(), w.tolist())
    assert np.array_equal(hc, bc)
    assert np.array_equal(bnd, bb)
    assert np.array_equal(fine, bf)
    assert bnd.any() and (r == 1 or not bnd.all() or n == 1)


def _two_seed_halfspace(dim, seed):
    # A = I: the cells are half-spaces; the normal x2 - x1 near (1, .., 1) makes
    # the boundary cut corners of pixels whose face neighbours lie on one side
    g = np.random.Generator(np.random.PCG64(seed))
    c = np.full(dim, 0.5) + 0.05 * g.standard_normal(dim)
    dvec = np.ones(dim) + 0.05 * g.standard_normal(dim)
    x = np.stack([c - 0.1 * dvec, c + 0.1 * dvec])
    A = np.stack([np.eye(dim)] * 2)
    w = np.array([0.0, 0.02 * g.standard_normal()])
    return x, A, w


def _inner_parent(coarse, r):
    """bool [J_F]: the fine pixel's coarse parent has its whole 3^D neighbourhood inside the grid."""
    inner = np.ones(tuple(reversed(coarse.res)), dtype=bool)
    for ax in range(coarse.dim):
        idx = [slice(None)] * coarse.dim
        idx[ax] = 0
        inner[tuple(idx)] = False
        idx[ax] = -1
        inner[tuple(idx)] = False
    return om._lift(coarse, r, inner)


@pytest.mark.parametrize("dim,m,r,seed", [(2, 24, 3, 5), (3, 8, 6, 6), (3, 9, 8, 7)])
def test_straight_boundary_is_resolved_exactly(dim, m, r, seed):
    # a pixel box cut by a hyperplane has a vertex across it, and the neighbour
    # centre beyond that vertex lies across too: every cut coarse pixel off the
    # outer layer is a boundary pixel, so the masked labels equal the fine grid's
    x, A, w = _two_seed_halfspace(dim, seed)
    coarse = synth.Grid.cube(dim, m)
    _, bnd, fine = om.labels(coarse, r, x, A, w)
    exact = oracle.assign(om.fine_grid(coarse, r), x, A, w)
    inner = _inner_parent(coarse, r)
    assert np.array_equal(fine[inner], exact[inner])
    assert bnd.any() and not bnd.all()


def test_straight_boundary_catches_a_face_only_mask():
    # planted mistake: faces only (no edge or corner neighbours) misses the
    # corner cuts of the 3D case above, and the comparison sees it
    dim, m, r = 3, 9, 8
    x, A, w = _two_seed_halfspace(dim, 7)
    coarse = synth.Grid.cube(dim, m)
    hc = oracle.assign(coarse, x, A, w)
    L = hc.reshape((m,) * dim)
    face = np.zeros(L.shape, dtype=bool)
    for ax in range(dim):
        for o in (1, -1):
            own = [slice(None)] * dim
            nb = [slice(None)] * dim
            own[ax], nb[ax] = (slice(0, -1), slice(1, None)) if o == 1 else (slice(1, None), slice(0, -1))
            face[tuple(own)] |= L[tuple(own)] != L[tuple(nb)]
    fine = om._lift(coarse, r, hc).astype(np.int32)
    ids = np.flatnonzero(om._lift(coarse, r, face.ravel()))
    fine[ids] = oracle.assign_ids(om.fine_grid(coarse, r), x, A, w, ids)
    exact = oracle.assign(om.fine_grid(coarse, r), x, A, w)
    inner = _inner_parent(coarse, r)
    assert not np.array_equal(fine[inner], exact[inner])


@pytest.mark.parametrize("dim,m", [(2, 30), (3, 12)])
def test_refinement_one_is_the_coarse_grid(dim, m):
    inst = synth.make_instance(dim, 15, m, 11)
    w = _weights(15, dim, 11)
    hc, _, fine = om.labels(inst.grid, 1, inst.x, inst.A, w)
    assert np.array_equal(fine, hc)
    assert np.array_equal(om.moments(inst.grid, 1, inst.x, inst.A, w), oracle.moments(inst.grid, hc, 15))
    g1, gr1, e1 = om.dual(inst.grid, 1, inst.x, inst.A, w, inst.v)
    g0, gr0, e0 = oracle.dual(inst.grid, inst.x, inst.A, w, inst.v)
    assert g1 == g0 and np.array_equal(gr1, gr0) and e1 == e0


@pytest.mark.parametrize("dim,m,r", [(2, 10, 4), (3, 5, 3)])
def test_one_seed_fills_the_fine_grid(dim, m, r):
    coarse = synth.Grid.cube(dim, m)
    x = np.full((1, dim), 0.3)
    A = np.eye(dim)[None]
    hc, bnd, fine = om.labels(coarse, r, x, A, np.zeros(1))
    assert not bnd.any() and (fine == 0).all()
    mo = om.moments(coarse, r, x, A, np.zeros(1))[0]
    M = m * r
    # sum over the fine grid of u = 2k + 1 per axis: M^(D-1) * M^2; of u_a^2: M^(D-1) * M (4 M^2 - 1) / 3
    assert mo[0] == M ** dim
    assert all(mo[1 + a] == M ** (dim - 1) * M * M for a in range(dim))
    assert mo[1 + dim] == M ** (dim - 1) * M * (4 * M * M - 1) // 3
