"""The sharded evaluation protocol of one APD on two gloo ranks (CPU).

Each rank owns the slab ``apd_shard_range(res, rank, 2)`` of the last axis,
computes that slab's integer moments (here with the oracle, standing in for
the GPU scoring), and one int64 sum-allreduce gives both ranks the full
moments (eq. (2.7)'s per-cell sums are the only cross-slab data).  The dual
value and gradient follow from the moments alone, so a replicated L-BFGS run
takes identical steps on both ranks: the weights must be bit-identical across
ranks and equal to a one-process run on the whole grid.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
scipy_opt = pytest.importorskip("scipy.optimize")


def _instance():
    from paper_2403_03571_gb300 import synth
    return synth.make_instance(3, 60, 1, 5, volumes="lognormal"), synth.Grid(3, (24, 20, 18))


def _solve(grid, inst, moments_at):
    """Replicated L-BFGS (scipy) on -g~ computed from the (reduced) moments."""
    import oracle

    def f(W):
        g, grad, _ = oracle.dual_from_moments(grid, inst.x, inst.A, W, inst.v, moments_at(W))
        return -g, -grad

    r = scipy_opt.minimize(f, np.zeros(inst.n), jac=True, method="L-BFGS-B",
                           options={"maxiter": 25, "maxfun": 40, "gtol": 0.0, "ftol": 0.0})
    return r.x


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import oracle
    from paper_2403_03571_gb300 import build, capi
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    build.build()
    capi.load()
    inst, grid = _instance()
    inst.v = inst.v * grid.measure
    kb, kc = capi.apd_shard_range(grid.res[-1], rank, world)
    ids = oracle.slab_ids(grid, kb, kc)
    reductions = []

    def moments_at(W):
        lab = oracle.assign_ids(grid, inst.x, inst.A, W, ids, nthreads=2)
        m = torch.from_numpy(oracle.moments_ids(grid, ids, lab, inst.n, nthreads=2))
        dist.all_reduce(m, op=dist.ReduceOp.SUM)
        reductions.append(1)
        return m.numpy()

    w_probe = 0.01 * np.arange(inst.n) / inst.n
    reduced = moments_at(w_probe)
    W = _solve(grid, inst, moments_at)
    dist.barrier()
    out.put((rank, kb, kc, reduced, W.tobytes(), len(reductions)))
    dist.destroy_process_group()


def test_two_gloo_ranks_solve_one_apd():
    import oracle
    from paper_2403_03571_gb300 import build
    build.build()
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    inst, grid = _instance()
    inst.v = inst.v * grid.measure
    # the two slabs partition the last axis
    assert (res[0][1], res[0][1] + res[0][2]) == (0, res[1][1]) and res[1][1] + res[1][2] == grid.res[-1]
    # the reduced moments are the whole grid's
    w_probe = 0.01 * np.arange(inst.n) / inst.n
    full = oracle.moments(grid, oracle.assign(grid, inst.x, inst.A, w_probe), inst.n)
    for r in res:
        np.testing.assert_array_equal(r[3], full)
    # identical weights on both ranks, equal to the one-process run
    assert res[0][4] == res[1][4] and res[0][5] == res[1][5]
    W1 = _solve(grid, inst, lambda W: oracle.moments(grid, oracle.assign(grid, inst.x, inst.A, W), inst.n))
    assert np.frombuffer(res[0][4]).tobytes() == W1.tobytes()
