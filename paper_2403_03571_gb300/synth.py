"""Seeded synthetic inputs for anisotropic power diagrams (APDs).

This module only *draws* inputs: seed points, anisotropy matrices and target
volumes, plus the regular grid that discretises the box.  It holds none of the
method's arithmetic (no costs, no assignment, no reductions), so both the FP64
oracle and the CUDA path take their inputs from here.

Laws (Section 3.2 "Runtime tests" of the paper, with the substitutions the
workload definitions make):

* seeds: uniform in the box, drawn sequentially and accepted only when farther
  than ``C * N**(-1/D)`` from every seed already accepted, ``C = 0.2``;
* 2D anisotropy: ``A = R(theta) diag(a, 1/a) R(theta)^T`` with theta uniform on
  [0, pi) and ``ln a ~ N(0, 0.3^2)`` (det A = 1, the normalisation of
  Section 2.1);
* 3D anisotropy: ``A = Q diag(s) Q^T`` with Q the rotation of a uniform random
  unit quaternion (Shoemake's subgroup algorithm) and ``ln s_k ~ N(0, 0.3^2)``,
  rescaled by ``(s_1 s_2 s_3)^(-1/3)`` so that det A = 1;
* the paper's own alpha-law (Section 3.2): 2D ``a_hat ~ U(1-alpha, 1)``,
  ``A_hat(1/a_hat, a_hat, theta)`` of eq. (2.2);
* volumes: equal (single phase) or lognormal with shape sigma, normalised so
  that they sum to the measure of the box (Section 2.1).

Every draw uses numpy's PCG64 with an explicit integer seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

BASE_SEED = 2403035710


@dataclasses.dataclass(frozen=True)
class Grid:
    """Regular pixel/voxel grid on the box [lo, hi] (eq. (2.6) of the paper).

    Pixel ``k = (k_0, .., k_{D-1})`` has centre ``lo + (k + 1/2) * h`` with
    ``h = (hi - lo) / res``; the linear pixel id is ``k_0 + res_0 * (k_1 + res_1 * k_2)``
    (first axis fastest).
    """

    dim: int
    res: tuple
    lo: tuple = None
    hi: tuple = None

    def __post_init__(self):
        if self.dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        if len(self.res) != self.dim:
            raise ValueError("res must have dim entries")
        if self.lo is None:
            object.__setattr__(self, "lo", (0.0,) * self.dim)
        if self.hi is None:
            object.__setattr__(self, "hi", (1.0,) * self.dim)
        object.__setattr__(self, "res", tuple(int(r) for r in self.res))
        object.__setattr__(self, "lo", tuple(float(v) for v in self.lo))
        object.__setattr__(self, "hi", tuple(float(v) for v in self.hi))

    @property
    def num_pixels(self) -> int:
        return int(np.prod(self.res, dtype=np.int64))

    @property
    def measure(self) -> float:
        return float(np.prod([h - l for l, h in zip(self.lo, self.hi)]))

    @staticmethod
    def cube(dim: int, m: int) -> "Grid":
        return Grid(dim, (m,) * dim)


@dataclasses.dataclass
class Instance:
    """One APD problem: grid, seeds x [N, D], anisotropy A [N, D, D], weights w [N],
    target volumes v [N].  All arrays are float64 and C-contiguous."""

    grid: Grid
    x: np.ndarray
    A: np.ndarray
    w: np.ndarray
    v: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def seeds_with_rejection(g: np.random.Generator, n: int, dim: int, c: float = 0.2,
                         lo: Sequence[float] = None, hi: Sequence[float] = None,
                         max_tries: int = 10_000_000) -> np.ndarray:
    """Uniform seeds in the box, drawn one at a time, a candidate being kept only when
    its distance to every kept seed exceeds ``c * n**(-1/dim)`` (Section 3.2, test (b)).
    ``c = 0`` gives plain uniform sampling."""
    lo = np.zeros(dim) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = np.ones(dim) if hi is None else np.asarray(hi, dtype=np.float64)
    if c <= 0.0:
        return lo + (hi - lo) * g.random((n, dim))
    rmin = c * n ** (-1.0 / dim)
    # bucket grid with cell side rmin: a candidate only needs the 3^D neighbouring buckets
    nb = np.maximum(1, np.floor((hi - lo) / rmin).astype(np.int64))
    buckets: dict = {}
    out = np.empty((n, dim))
    kept = 0
    tries = 0
    offsets = np.array(np.meshgrid(*([[-1, 0, 1]] * dim), indexing="ij")).reshape(dim, -1).T
    while kept < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("seed rejection sampler did not terminate")
        p = lo + (hi - lo) * g.random(dim)
        b = np.minimum(((p - lo) / rmin).astype(np.int64), nb - 1)
        ok = True
        for off in offsets:
            lst = buckets.get(tuple(b + off))
            if lst is None:
                continue
            q = out[lst]
            if np.any(np.sum((q - p) ** 2, axis=1) <= rmin * rmin):
                ok = False
                break
        if not ok:
            continue
        out[kept] = p
        buckets.setdefault(tuple(b), []).append(kept)
        kept += 1
    return out


def aniso_2d_lognormal(g: np.random.Generator, n: int, sigma: float = 0.3) -> np.ndarray:
    """A = R(theta) diag(a, 1/a) R(theta)^T, theta ~ U[0, pi), ln a ~ N(0, sigma^2)."""
    theta = g.uniform(0.0, math.pi, n)
    a = np.exp(g.normal(0.0, sigma, n))
    return _rot2_diag(theta, a, 1.0 / a)


def aniso_2d_alpha(g: np.random.Generator, n: int, alpha: float) -> np.ndarray:
    """The paper's 2D law: a_hat ~ U(1-alpha, 1), theta ~ U(0, pi), matrix A_hat(1/a_hat, a_hat,
    theta) of eq. (2.2): axes 1/a_hat (major) and a_hat (minor), i.e.
    D = diag(a_hat^2, a_hat^-2) in the rotated frame."""
    a_hat = g.uniform(1.0 - alpha, 1.0, n) if alpha > 0 else np.ones(n)
    theta = g.uniform(0.0, math.pi, n)
    major = 1.0 / a_hat
    minor = a_hat
    return _rot2_diag(theta, major ** -2, minor ** -2)


def _rot2_diag(theta: np.ndarray, d0: np.ndarray, d1: np.ndarray) -> np.ndarray:
    c, s = np.cos(theta), np.sin(theta)
    A = np.empty((theta.shape[0], 2, 2))
    A[:, 0, 0] = c * c * d0 + s * s * d1
    A[:, 0, 1] = c * s * (d0 - d1)
    A[:, 1, 0] = A[:, 0, 1]
    A[:, 1, 1] = s * s * d0 + c * c * d1
    return A


def uniform_rotations(g: np.random.Generator, n: int) -> np.ndarray:
    """Haar-uniform rotations from unit quaternions (Shoemake's subgroup algorithm)."""
    u1, u2, u3 = g.random(n), g.random(n), g.random(n)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    qx = a * np.sin(2 * math.pi * u2)
    qy = a * np.cos(2 * math.pi * u2)
    qz = b * np.sin(2 * math.pi * u3)
    qw = b * np.cos(2 * math.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (qy * qy + qz * qz)
    R[:, 0, 1] = 2 * (qx * qy - qz * qw)
    R[:, 0, 2] = 2 * (qx * qz + qy * qw)
    R[:, 1, 0] = 2 * (qx * qy + qz * qw)
    R[:, 1, 1] = 1 - 2 * (qx * qx + qz * qz)
    R[:, 1, 2] = 2 * (qy * qz - qx * qw)
    R[:, 2, 0] = 2 * (qx * qz - qy * qw)
    R[:, 2, 1] = 2 * (qy * qz + qx * qw)
    R[:, 2, 2] = 1 - 2 * (qx * qx + qy * qy)
    return R


def _rot_zyz(theta: np.ndarray, phi: np.ndarray, gamma: np.ndarray) -> np.ndarray:
    """R = Rz(theta) Ry(phi) Rz(gamma) per seed (the z-y-z Euler convention)."""
    def rz(t):
        c, s = np.cos(t), np.sin(t)
        R = np.zeros((t.shape[0], 3, 3))
        R[:, 0, 0], R[:, 0, 1], R[:, 1, 0], R[:, 1, 1], R[:, 2, 2] = c, -s, s, c, 1.0
        return R

    def ry(t):
        c, s = np.cos(t), np.sin(t)
        R = np.zeros((t.shape[0], 3, 3))
        R[:, 0, 0], R[:, 0, 2], R[:, 2, 0], R[:, 2, 2], R[:, 1, 1] = c, s, -s, c, 1.0
        return R

    return rz(theta) @ ry(phi) @ rz(gamma)


def aniso_3d_alpha(g: np.random.Generator, n: int, alpha: float) -> np.ndarray:
    """The paper's 3D runtime-test law: axes a_hat ~ U(1-alpha, 1), b_hat ~
    U(1-alpha, 1/(1-alpha)) and 1/(a_hat b_hat) (det A = 1), angles theta, phi,
    gamma ~ U(0, 2 pi) of a z-y-z rotation R (the paper does not name the
    convention); A = R diag(axes^-2) R^T as in eq. (2.2)."""
    if alpha > 0:
        a_hat = g.uniform(1.0 - alpha, 1.0, n)
        b_hat = g.uniform(1.0 - alpha, 1.0 / (1.0 - alpha), n)
    else:
        a_hat, b_hat = np.ones(n), np.ones(n)
    ang = g.uniform(0.0, 2.0 * math.pi, (3, n))
    R = _rot_zyz(ang[0], ang[1], ang[2])
    axes = np.stack([a_hat, b_hat, 1.0 / (a_hat * b_hat)], axis=1)
    A = np.einsum("nij,nj,nkj->nik", R, axes ** -2, R)
    return 0.5 * (A + np.transpose(A, (0, 2, 1)))


def runtime_test_instance(dim: int, n: int, alpha: float, multiphase: bool, seed: int,
                          m: Optional[int] = None, eps: float = 0.01, m_cap: Optional[int] = None) -> Instance:
    """An instance of the paper's runtime tests (Section 3.2): seeds uniform on
    [0,1]^D with the sequential rejection C = 0.2, the alpha anisotropy law,
    equal volumes (single phase) or lognormal volumes with shape 1.0 normalised
    to |Omega| = 1 (multi phase), and M from eq. (2.10) for the smallest volume
    (capped at m_cap) unless given."""
    g = rng(seed)
    x = seeds_with_rejection(g, n, dim, c=0.2)
    A = aniso_2d_alpha(g, n, alpha) if dim == 2 else aniso_3d_alpha(g, n, alpha)
    v = volumes_lognormal(g, n, 1.0, 1.0) if multiphase else volumes_equal(n, 1.0)
    if m is None:
        m = required_resolution(dim, float(v.min()), eps)
        if m_cap is not None:
            m = min(m, m_cap)
    return Instance(Grid.cube(dim, m), _contig(x), _contig(A), np.zeros(n), _contig(v),
                    f"runtime_{dim}d_n{n}_a{alpha}_{'multi' if multiphase else 'single'}")


def aniso_3d_lognormal(g: np.random.Generator, n: int, sigma: float = 0.3) -> np.ndarray:
    """A = Q diag(s) Q^T, Q uniform rotation, ln s_k ~ N(0, sigma^2) rescaled to det 1."""
    Q = uniform_rotations(g, n)
    s = np.exp(g.normal(0.0, sigma, (n, 3)))
    s = s / np.cbrt(np.prod(s, axis=1))[:, None]
    A = np.einsum("nij,nj,nkj->nik", Q, s, Q)
    return 0.5 * (A + np.transpose(A, (0, 2, 1)))


def volumes_equal(n: int, measure: float = 1.0) -> np.ndarray:
    return np.full(n, measure / n)


def volumes_lognormal(g: np.random.Generator, n: int, sigma: float = 0.5,
                      measure: float = 1.0) -> np.ndarray:
    v = np.exp(g.normal(0.0, sigma, n))
    return v * (measure / v.sum())


def _contig(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_instance(dim: int, n: int, m: int, seed: int, *, volumes: str = "lognormal",
                  sigma_a: float = 0.3, sigma_v: float = 0.5, reject_c: float = 0.2,
                  alpha: Optional[float] = None, name: str = "") -> Instance:
    """Draw one instance on the unit box with an ``m^dim`` grid and zero weights."""
    g = rng(seed)
    grid = Grid.cube(dim, m)
    x = seeds_with_rejection(g, n, dim, c=reject_c)
    if dim == 2:
        A = aniso_2d_alpha(g, n, alpha) if alpha is not None else aniso_2d_lognormal(g, n, sigma_a)
    else:
        if alpha is not None:
            raise ValueError("the alpha law is provided for 2D only")
        A = aniso_3d_lognormal(g, n, sigma_a)
    if volumes == "equal":
        v = volumes_equal(n, grid.measure)
    else:
        v = volumes_lognormal(g, n, sigma_v, grid.measure)
    return Instance(grid, _contig(x), _contig(A), np.zeros(n), _contig(v), name)


# ---------------------------------------------------------------------------
# the five workloads (sizes, laws and seeds); index k seeds with BASE_SEED + k*1e6
# ---------------------------------------------------------------------------

def workload_seed(k: int, instance: int = 0) -> int:
    return BASE_SEED + 1_000_000 * k + instance


def workload_2d_20(instance: int = 0) -> Instance:
    """2D, 20 seeds, lognormal 2D anisotropy, equal volumes 1/20, 256^2 pixels."""
    return make_instance(2, 20, 256, workload_seed(0, instance), volumes="equal",
                         name="2d_n20_256sq")


def workload_3d_1000(instance: int = 0, m: int = 256) -> Instance:
    """3D, 1000 seeds, quaternion anisotropy, lognormal(0.5) volumes, 256^3 voxels."""
    return make_instance(3, 1000, m, workload_seed(1, instance), name=f"3d_n1000_{m}cube")


def workload_3d_10000(instance: int = 0, m: int = 512) -> Instance:
    """3D, 10,000 seeds, as the 1000-seed law, 512^3 voxels."""
    return make_instance(3, 10000, m, workload_seed(2, instance), name=f"3d_n10000_{m}cube")


def workload_2d_2000(instance: int = 0) -> Instance:
    """2D, 2000 seeds, lognormal volumes, 1024^2 pixels: the largest instance class
    of the batched 2D workload, for single-instance kernel measurements."""
    return make_instance(2, 2000, 1024, workload_seed(3, 10_000 + instance), name="2d_n2000_1024sq")


def required_resolution(dim: int, v_min: float, eps: float = 0.01, measure: float = 1.0) -> int:
    """Smallest M with measure / M^dim <= eps v_min / 2^dim (the resolution rule of
    eq. (2.10), non-strict), used to size the grids of the batched workloads."""
    target = (2.0 ** dim) * measure / (eps * v_min)
    m = max(1, int(math.floor(target ** (1.0 / dim))))
    while m ** dim < target:
        m += 1
    return m


def batched_table(count: int = 256, seed: Optional[int] = None, k: int = 3):
    """Per-instance seed counts N (log-uniform in [50, 2000]) and generator seeds of a
    batched workload."""
    g = rng(workload_seed(k) if seed is None else seed)
    ns = np.exp(g.uniform(math.log(50), math.log(2000), count)).round().astype(int)
    return ns, g.integers(0, 2**31 - 1, count)


BATCH_2D_RES = (256, 384, 512, 768, 1024)


def batched_2d_instances(count: int = 256, seed: Optional[int] = None) -> List[Instance]:
    """The batched 2D workload: N log-uniform in [50, 2000], seeds with rejection
    (C = 0.2), 2D lognormal anisotropy (sigma 0.3), lognormal volumes (sigma 0.5)
    normalised to 1, and per instance the smallest grid of 256^2 .. 1024^2 that
    meets eq. (2.10) at eps = 1% (1024^2 when none does)."""
    ns, seeds = batched_table(count, seed, k=3)
    out = []
    for b, (n, sd) in enumerate(zip(ns, seeds)):
        inst = make_instance(2, int(n), BATCH_2D_RES[0], int(sd), name=f"b2d_{b}")
        need = required_resolution(2, float(inst.v.min()))
        m = next((r for r in BATCH_2D_RES if r >= need), BATCH_2D_RES[-1])
        inst.grid = Grid.cube(2, m)
        out.append(inst)
    return out


def batched_3d_instances(count: int, seed: int, m_cap: int = 256, n_lo: int = 50,
                         n_hi: int = 2000) -> List[Instance]:
    """3D instances with the 1000-seed workload's laws, N log-uniform in
    [n_lo, n_hi] and M from eq. (2.10) at eps = 1%, capped at m_cap (the
    training distribution of the learned warm start)."""
    g = rng(seed)
    ns = np.exp(g.uniform(math.log(n_lo), math.log(n_hi), count)).round().astype(int)
    seeds = g.integers(0, 2**31 - 1, count)
    out = []
    for b, (n, sd) in enumerate(zip(ns, seeds)):
        inst = make_instance(3, int(n), 16, int(sd), name=f"b3d_{b}")
        m = min(m_cap, required_resolution(3, float(inst.v.min())))
        inst.grid = Grid.cube(3, m)
        out.append(inst)
    return out


def concat(instances: List[Instance]):
    """Concatenated (x, A, w, v) of a batch, in instance order."""
    return (np.concatenate([i.x for i in instances]), np.concatenate([i.A for i in instances]),
            np.concatenate([i.w for i in instances]), np.concatenate([i.v for i in instances]))
