"""Seeded input generators: laws of Section 3.2 and the workload substitutions."""
import numpy as np

import oracle
from paper_2403_03571_gb300 import synth


def test_deterministic():
    a = synth.make_instance(3, 50, 8, 123)
    b = synth.make_instance(3, 50, 8, 123)
    for f in ("x", "A", "v"):
        assert np.array_equal(getattr(a, f), getattr(b, f))


def test_2d_anisotropy_law():
    A = synth.aniso_2d_lognormal(synth.rng(1), 20000, 0.3)
    assert np.allclose(A, np.transpose(A, (0, 2, 1)))
    assert np.allclose(np.linalg.det(A), 1.0, atol=1e-12)
    ev = np.linalg.eigvalsh(A)
    assert np.all(ev > 0)
    # eigenvalues are a and 1/a with ln a ~ N(0, 0.3^2): ln(max eig) = |ln a|
    la = np.log(ev[:, 1])
    assert abs(np.mean(la) - 0.3 * np.sqrt(2 / np.pi)) < 0.01


def test_3d_anisotropy_law():
    A = synth.aniso_3d_lognormal(synth.rng(2), 20000, 0.3)
    assert np.allclose(A, np.transpose(A, (0, 2, 1)))
    assert np.allclose(np.linalg.det(A), 1.0, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(A) > 0)
    # Haar-uniform rotations: E[Q] = 0 and E[Q_00^2] = 1/3
    Q = synth.uniform_rotations(synth.rng(3), 50000)
    assert np.allclose(np.einsum("nij,nkj->nik", Q, Q), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(Q), 1.0)
    assert np.abs(Q.mean(axis=0)).max() < 0.01
    assert abs(np.mean(Q[:, 0, 0] ** 2) - 1 / 3) < 0.01


def test_alpha_law_2d():
    A = synth.aniso_2d_alpha(synth.rng(4), 5000, 0.7)
    ev = np.linalg.eigvalsh(A)
    assert np.allclose(ev[:, 0] * ev[:, 1], 1.0)
    # minor axis a_hat in (0.3, 1): eigenvalues a_hat^2 and a_hat^-2
    a_hat = np.sqrt(ev[:, 0])
    assert a_hat.min() >= 0.3 - 1e-12 and a_hat.max() <= 1.0 + 1e-12
    assert np.allclose(synth.aniso_2d_alpha(synth.rng(4), 10, 0.0), np.eye(2))


def test_volumes():
    v = synth.volumes_lognormal(synth.rng(5), 1000, 0.5)
    assert abs(v.sum() - 1.0) < 1e-12 and np.all(v > 0)
    lv = np.log(v)
    assert abs(lv.std() - 0.5) < 0.05
    assert np.allclose(synth.volumes_equal(20), 1 / 20)


def test_rejection_distance():
    for dim, n in ((2, 400), (3, 600)):
        x = synth.seeds_with_rejection(synth.rng(6), n, dim, 0.2)
        d = np.sqrt(((x[:, None] - x[None]) ** 2).sum(-1)) + np.eye(n) * 10
        assert d.min() > 0.2 * n ** (-1.0 / dim)
        assert x.min() >= 0 and x.max() <= 1


def test_workloads_shapes():
    w0 = synth.workload_2d_20()
    assert w0.x.shape == (20, 2) and w0.grid.res == (256, 256)
    assert np.allclose(w0.v, 1 / 20)
    w1 = synth.workload_3d_1000(m=16)
    assert w1.x.shape == (1000, 3) and abs(w1.v.sum() - 1) < 1e-12


def test_batched_2d_workload_shape():
    insts = synth.batched_2d_instances(256)
    ns = np.array([i.n for i in insts])
    assert ns.min() >= 50 and ns.max() <= 2000
    for inst in insts:
        m = inst.grid.res[0]
        assert m in synth.BATCH_2D_RES and inst.grid.res[1] == m
        assert abs(inst.v.sum() - 1.0) < 1e-12
        # the grid is the smallest listed one meeting eq. (2.10), as the oracle's
        # own resolution rule computes it
        need = oracle.resolution_practical(2, float(inst.v.min()))
        assert m >= need or m == synth.BATCH_2D_RES[-1]
        smaller = [r for r in synth.BATCH_2D_RES if r < m]
        assert not smaller or smaller[-1] < need
    total = sum(i.n * i.grid.num_pixels for i in insts)
    assert 5e10 < total < 3e11


def test_required_resolution_matches_oracle():
    for dim, vmin in [(2, 1 / 20), (3, 1e-4), (3, 2.3e-4), (2, 3.7e-5)]:
        assert synth.required_resolution(dim, vmin) == oracle.resolution_practical(dim, vmin)


def test_runtime_test_anisotropy_laws():
    # the paper's runtime-test laws (Section 3.2): det A = 1, eigenvalues the
    # inverse squared axes, identity at alpha = 0
    g = synth.rng(5)
    A = synth.aniso_3d_alpha(g, 200, 0.7)
    assert np.allclose(A, np.transpose(A, (0, 2, 1)), atol=0)
    assert np.allclose(np.linalg.det(A), 1.0, rtol=1e-12)
    ev = np.linalg.eigvalsh(A)
    assert (ev > 0).all()
    # axes a in [0.3, 1], b in [0.3, 1/0.3]: every eigenvalue a^-2, b^-2 or (ab)^2 lies in range
    assert ev.min() >= 0.3 ** 2 * 0.3 ** 2 * (1 - 1e-12) and ev.max() <= 0.3 ** -2 * 0.3 ** -2 * (1 + 1e-12)
    assert np.allclose(synth.aniso_3d_alpha(synth.rng(6), 10, 0.0), np.eye(3), atol=1e-14)
    A2 = synth.aniso_2d_alpha(synth.rng(7), 50, 0.3)
    assert np.allclose(np.linalg.det(A2), 1.0, rtol=1e-12)
    # the z-y-z rotation is orthogonal
    R = synth._rot_zyz(*synth.rng(8).uniform(0, 6.3, (3, 20)))
    assert np.allclose(np.einsum("nij,nkj->nik", R, R), np.eye(3), atol=1e-14)


def test_runtime_test_instances():
    single = synth.runtime_test_instance(3, 500, 0.3, False, 11)
    assert np.allclose(single.v, 1.0 / 500) and abs(single.v.sum() - 1.0) < 1e-12
    assert single.grid.res[0] == synth.required_resolution(3, 1.0 / 500, 0.01)
    multi = synth.runtime_test_instance(2, 300, 0.7, True, 12, m_cap=1000)
    assert abs(multi.v.sum() - 1.0) < 1e-12 and multi.v.std() > 0
    assert multi.grid.res[0] == min(1000, synth.required_resolution(2, float(multi.v.min()), 0.01))
    # the resolution the paper states for N = 10^4 single-phase grains in 3D: M = 200
    assert synth.required_resolution(3, 1e-4, 0.01) == 200
    # the rejection rule keeps seeds at least 0.2 N^(-1/D) apart
    d = np.linalg.norm(single.x[:, None] - single.x[None], axis=-1) + np.eye(500)
    assert d.min() > 0.2 * 500 ** (-1 / 3)
