"""Slabs and sharded evaluation on one GPU (the split of one APD across ranks).

The per-cell sums of eq. (2.7) are the only cross-slab data, so:
* the integer moments of the slabs of any partition of the last axis sum to
  the whole grid's moments bit for bit (and therefore to the oracle's);
* a weight solve or a Lloyd run whose workspace scores only one slab, with a
  reduction hook that adds the other slabs' moments, follows exactly the same
  path as the unsharded run: the final weights and positions are bit-identical.
The hook here emulates the other ranks on the same GPU by scoring their slabs
at the weights the solver passes; with one process per GPU the hook is an
NCCL allreduce instead (``paper_2403_03571_gb300.shard.allreduce_hook``).
"""
import numpy as np
import pytest

import oracle
from paper_2403_03571_gb300 import synth
from _gpu import host, instance_tensors, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    require_gpu()
    from paper_2403_03571_gb300 import capi as c
    return c


def _case(dim, n, res, seed, wscale=0.3):
    g = synth.rng(seed)
    x = synth.seeds_with_rejection(g, n, dim, 0.2)
    A = synth.aniso_2d_lognormal(g, n, 0.3) if dim == 2 else synth.aniso_3d_lognormal(g, n, 0.3)
    v = synth.volumes_lognormal(g, n, 0.5)
    w = wscale * g.standard_normal(n) * n ** (-2.0 / dim)
    return synth.Instance(synth.Grid(dim, res), x, A, w, v, f"d{dim}n{n}")


@pytest.mark.parametrize("prec", ["fp32", "fp32_pruned", "tc_bf16", "tc_tf32_pruned"])
@pytest.mark.parametrize("dim,n,res,world", [(3, 300, (40, 33, 29), 2), (3, 1000, (64, 64, 64), 4),
                                             (2, 200, (130, 97), 3), (3, 50, (20, 20, 5), 8)])
def test_slabs_sum_to_the_whole_grid(capi, dim, n, res, world, prec):
    inst = _case(dim, n, res, 11 + world)
    x, A, w, _ = instance_tensors(inst)
    pc = {"fp32": capi.APD_FP32, "tc_bf16": capi.APD_TC_BF16, "tc_tf32": capi.APD_TC_TF32}[prec.replace("_pruned", "")]
    K = oracle.moment_width(dim)
    ws = capi.Workspace(dim, n, inst.grid.num_pixels)
    ws.set_pruning(prec.endswith("_pruned"))
    full = torch.zeros((n, K), dtype=torch.int64, device="cuda")
    capi.apd_cell_moments(inst.grid, x, A, w, full, ws, precision=pc)
    total = np.zeros((n, K), dtype=np.int64)
    for r in range(world):
        kb, kc = capi.apd_shard_range(res[-1], r, world)
        if kc == 0:
            continue
        part = torch.full((n, K), -1, dtype=torch.int64, device="cuda")
        capi.apd_cell_moments_slab(inst.grid, kb, kc, x, A, w, part, ws, precision=pc)
        assert ws.status() == capi.APD_OK
        p = host(part)
        # each slab against the oracle's moments of its pixels, in full-grid coordinates
        ids = oracle.slab_ids(inst.grid, kb, kc)
        lab = oracle.assign_ids(inst.grid, inst.x, inst.A, inst.w, ids)
        np.testing.assert_array_equal(p, oracle.moments_ids(inst.grid, ids, lab, n))
        total += p
    np.testing.assert_array_equal(total, host(full))
    np.testing.assert_array_equal(total, oracle.moments(inst.grid, oracle.assign(inst.grid, inst.x, inst.A,
                                                                                 inst.w), n))


def _emulating_hook(capi, inst, world, rank, prec):
    """A reduction hook for `rank` that adds the other ranks' slab moments,
    scored on this GPU for the generators of the evaluation (the positions,
    matrices and trial weights the library passes)."""
    from paper_2403_03571_gb300 import shard
    helpers = {}
    calls = []

    def hook(ctx, mom_ptr, words, seeds, stream_ptr):
        try:
            sd = seeds.contents
            n, dim = sd.n, inst.grid.dim
            mom = shard.device_view(mom_ptr, words, "int64")
            w = shard.device_view(sd.w, n, "float64")
            x = shard.device_view(sd.x, n * dim, "float64").view(n, dim)
            A = shard.device_view(sd.A, n * dim * dim, "float64").view(n, dim, dim)
            with torch.cuda.stream(shard._stream_of(stream_ptr)):
                K = words // n
                for r in range(world):
                    if r == rank:
                        continue
                    grid = helpers["grid"]  # the one grid these solves use
                    kb, kc = capi.apd_shard_range(grid.res[-1], r, world)
                    if kc == 0:
                        continue
                    ws2 = helpers.setdefault(("ws", grid.res), capi.Workspace(grid.dim, n, grid.num_pixels))
                    part = torch.empty((n, K), dtype=torch.int64, device="cuda")
                    capi.apd_cell_moments_slab(grid, kb, kc, x, A, w, part, ws2, precision=prec,
                                               stream=torch.cuda.current_stream())
                    mom += part.view(-1)
            calls.append(1)
            return 0
        except Exception as e:  # noqa: BLE001
            print("hook failed:", e)
            return 1

    return capi.REDUCE_FN(hook), helpers, calls


@pytest.mark.parametrize("world,rank", [(2, 0), (2, 1), (3, 2)])
def test_sharded_solve_is_bit_identical(capi, world, rank):
    inst = _case(3, 400, (48, 40, 36), 31, 0.0)
    x, A, w0, v = instance_tensors(inst)
    n, J = inst.n, inst.grid.num_pixels
    opts = capi.solve_opts(eps=0.01)
    ws_full = capi.Workspace(3, n, J)
    w_full = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc0, info0 = capi.apd_solve_weights(inst.grid, x, A, w0, v, w_full, ws_full, opts)
    ws = capi.Workspace(3, n, J)
    hook, helpers, calls = _emulating_hook(capi, inst, world, rank, capi.APD_FP32)
    helpers["grid"] = inst.grid
    ws.set_shard(rank, world, hook)
    w_sh = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc1, info1 = capi.apd_solve_weights(inst.grid, x, A, w0, v, w_sh, ws, opts)
    assert rc1 == rc0 and info1.evaluations == info0.evaluations and len(calls) == info1.evaluations
    np.testing.assert_array_equal(host(w_sh), host(w_full))
    assert info1.max_rel_err == info0.max_rel_err and info1.g == info0.g
    # the oracle's max relative volume error at the sharded weights is the one reported
    _, _, err = oracle.dual(inst.grid, inst.x, inst.A, host(w_sh), inst.v)
    assert err == info1.max_rel_err
    ws.set_shard(0, 1)


def test_sharded_lloyd_is_bit_identical(capi):
    inst = _case(3, 300, (40, 40, 40), 41, 0.0)
    x, A, w0, v = instance_tensors(inst)
    n, J = inst.n, inst.grid.num_pixels
    opts = capi.solve_opts(eps=0.01)
    outs = []
    for world in (1, 2):
        ws = capi.Workspace(3, n, J)
        if world > 1:
            hook, helpers, _ = _emulating_hook(capi, inst, world, 1, capi.APD_FP32)
            helpers["grid"] = inst.grid
            ws.set_shard(1, world, hook)
        x_out = torch.zeros_like(x)
        w_out = torch.zeros(n, dtype=torch.float64, device="cuda")
        rc, info = capi.apd_lloyd(inst.grid, x, A, w0, v, 2, x_out, w_out, ws, opts)
        outs.append((host(x_out), host(w_out), info.evaluations))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


def test_shard_arguments(capi):
    assert capi.apd_shard_range(10, 0, 3) == (0, 3)
    assert capi.apd_shard_range(10, 2, 3) == (6, 4)
    with pytest.raises(capi.ApdError):
        capi.apd_shard_range(10, 3, 3)
    inst = _case(2, 20, (30, 20), 3)
    x, A, w, _ = instance_tensors(inst)
    ws = capi.Workspace(2, 20, 600)
    mom = torch.zeros((20, 6), dtype=torch.int64, device="cuda")
    for kb, kc in ((-1, 3), (0, 0), (18, 3)):
        with pytest.raises(capi.ApdError) as e:
            capi.apd_cell_moments_slab(inst.grid, kb, kc, x, A, w, mom, ws)
        assert e.value.code == capi.APD_ERR_ARG
    with pytest.raises(capi.ApdError):
        ws.set_shard(0, 2, None)  # a sharded workspace needs a hook
