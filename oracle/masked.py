"""Masked two-level discretisation, FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library path never does.

Section 4 of the paper names adaptable pixel sizes, found by masking the pixels
at cell boundaries, as the next step, without an algorithm.  The reading
followed here (and by the library):

1. Algorithm 1 on the coarse grid G gives labels H^G.
2. A coarse pixel is a boundary pixel when a pixel of its 3^D neighbourhood
   inside the grid carries another label; otherwise it is interior.
3. The fine grid F has r times the resolution of G on the same box.  A fine
   pixel inside an interior coarse pixel takes that pixel's label; a fine pixel
   inside a boundary coarse pixel is labelled by Algorithm 1 on F.

The labelling of F then enters the moments and eqs. (2.7)-(2.8) of the
regular grid F.  Built on the brute-force grid oracle (``oracle.assign``,
``assign_ids``, ``moments``, ``dual_from_labels``) plus numpy slicing.
"""
from __future__ import annotations

import itertools

import numpy as np

import oracle


def fine_grid(coarse, r: int):
    """The grid of the same box with r times the resolution per axis."""
    return type(coarse)(coarse.dim, tuple(int(m) * int(r) for m in coarse.res), lo=coarse.lo, hi=coarse.hi)


def boundary_mask(coarse, labels) -> np.ndarray:
    """bool [J_G]: a pixel of the 3^D neighbourhood inside the grid has another label (step 2)."""
    D = coarse.dim
    L = np.asarray(labels).reshape(tuple(reversed(coarse.res)))  # array axes: last grid axis first
    mask = np.zeros(L.shape, dtype=bool)
    for off in itertools.product((-1, 0, 1), repeat=D):
        own, nb = [], []
        for o in off:
            if o == 1:
                own.append(slice(0, -1))
                nb.append(slice(1, None))
            elif o == -1:
                own.append(slice(1, None))
                nb.append(slice(0, -1))
            else:
                own.append(slice(None))
                nb.append(slice(None))
        mask[tuple(own)] |= L[tuple(own)] != L[tuple(nb)]
    return mask.ravel()


def _lift(coarse, r: int, values) -> np.ndarray:
    """Per-coarse-pixel values repeated over the r^D fine pixels of each (fine linear order)."""
    a = np.asarray(values).reshape(tuple(reversed(coarse.res)))
    for ax in range(coarse.dim):
        a = np.repeat(a, r, axis=ax)
    return a.ravel()


def labels(coarse, r: int, x, A, w):
    """(coarse labels [J_G], boundary mask [J_G], fine labels [J_F]) of steps 1-3."""
    hc = oracle.assign(coarse, x, A, w)
    bnd = boundary_mask(coarse, hc)
    fine = _lift(coarse, r, hc).astype(np.int32)
    ids = np.flatnonzero(_lift(coarse, r, bnd))
    if ids.size:
        fine[ids] = oracle.assign_ids(fine_grid(coarse, r), x, A, w, ids)
    return hc, bnd, fine


def moments(coarse, r: int, x, A, w) -> np.ndarray:
    """Integer moments [n, K] of the fine labelling, in fine-grid units."""
    _, _, fine = labels(coarse, r, x, A, w)
    return oracle.moments(fine_grid(coarse, r), fine, np.asarray(x).shape[0])


def dual(coarse, r: int, x, A, w, v):
    """Eqs. (2.7)-(2.8) on the fine grid for the masked labelling: (g~, grad, max_rel_err)."""
    _, _, fine = labels(coarse, r, x, A, w)
    g, grad, err, _, _ = oracle.dual_from_labels(fine_grid(coarse, r), x, A, w, v, fine)
    return g, grad, err
