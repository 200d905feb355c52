"""Learned warm start of the weight solve: data generation, training, storage.

Every numeric step runs in the library's kernels (include/apd.h): the training
instances are solved by the plain method (batched FP32 solves from W = 0,
``apd_batch_solve_weights``), features come from ``apd_warmstart_features``,
and training is ``apd_warmstart_train_step`` (hand-written forward, backward
and Adam kernels).  This module only draws instances, moves arrays and
schedules the steps.

Targets: the solved weights of each instance, centred (the dual is invariant to
adding a constant to all weights) and scaled to units of the mean cell size
squared, t_i = (w_i - mean w) (n / |O|)^(2/D), the inverse of the scaling the
prediction applies.  The loss compares differences between neighbouring
seeds (apd_warmstart_train_step_pairs): the dual penalises an error that
changes from cell to cell far more than one that varies slowly, and local
features can only ever predict the former.

Usage (on a GPU): ``python -m paper_2403_03571_gb300.warmstart --dim 2 --instances 5000``
writes ``data/warmstart_2d.npz``.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time
from typing import List, Optional

import numpy as np

from . import capi, synth

_HERE = os.path.dirname(os.path.abspath(__file__))
DATA_DIR = os.path.join(_HERE, "data")
TRAIN_SEED = {2: 2403_035_720, 3: 2403_035_730}   # instance draws for training
HELD_OUT_SEED = {2: 2403_035_721, 3: 2403_035_731}  # never used in training


def path(dim: int) -> str:
    return os.path.join(DATA_DIR, f"warmstart_{dim}d.npz")


def init_params(dim: int, seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases, in the flat order of include/apd.h."""
    F, P = capi.warmstart_sizes(dim)
    g = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fan_in, fan_out in ((F, 64), (64, 64), (64, 64), (64, 1)):
        lim = math.sqrt(6.0 / fan_in)
        parts.append(g.uniform(-lim, lim, fan_in * fan_out))
        parts.append(np.zeros(fan_out))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == P
    return p


def load(dim: int) -> Optional[capi.WarmStart]:
    """The stored network for dim, or None if none has been trained."""
    p = path(dim)
    if not os.path.exists(p):
        return None
    z = np.load(p)
    return capi.WarmStart(dim, z["params"], z["norm"])


def meta(dim: int) -> dict:
    z = np.load(path(dim))
    return json.loads(str(z["meta"]))


def draw(dim: int, count: int, seed: int) -> List[synth.Instance]:
    if dim == 2:
        return synth.batched_2d_instances(count, seed)
    return synth.batched_3d_instances(count, seed)


def instance_arrays(insts, device="cuda"):
    import torch
    x, A, w, v = synth.concat(insts)
    return tuple(torch.from_numpy(a).to(device) for a in (x, A, w, v))


def predict(net: capi.WarmStart, insts, x, A, v):
    """Predicted weights (device, concatenated) for the instances."""
    import torch
    counts = [i.n for i in insts]
    grids = [i.grid for i in insts]
    feats = torch.empty((sum(counts), net.n_features), dtype=torch.float32, device=x.device)
    net.features(counts, grids, x, A, v, feats)
    w = torch.empty(sum(counts), dtype=torch.float64, device=x.device)
    net.predict(counts, grids, feats, w)
    return w


def generate(dim: int, count: int, seed: int, chunk: int = 256, log=print):
    """Solve `count` drawn instances with the plain batched method; returns the
    features (device FP32 [S][F]), targets (device FP32 [S]), the per-instance
    sample counts and statistics.  Unconverged instances are dropped."""
    import torch
    F, _ = capi.warmstart_sizes(dim)
    feat_net = capi.WarmStart(dim, np.zeros(capi.warmstart_sizes(dim)[1], np.float32))
    feats, targets, counts, knns = [], [], [], []
    base = 0  # rows kept so far
    stats = {"instances": 0, "dropped": 0, "evaluations": 0, "seconds": 0.0}
    insts_all = draw(dim, count, seed)
    opts = capi.solve_opts(eps=0.01, max_evals=1000)
    for c0 in range(0, count, chunk):
        insts = insts_all[c0:c0 + chunk]
        x, A, w, v = instance_arrays(insts)
        t0 = time.time()
        b = capi.Batch(dim, [i.grid for i in insts], [i.n for i in insts])
        w_out = torch.zeros_like(w)
        rc, infos = capi.apd_batch_solve_weights(b, x, A, w, v, w_out, opts)
        f = torch.empty((x.shape[0], F), dtype=torch.float32, device="cuda")
        kn = torch.empty((x.shape[0], 8), dtype=torch.int32, device="cuda")
        feat_net.features([i.n for i in insts], [i.grid for i in insts], x, A, v, f, knn=kn)
        W = w_out.cpu().numpy()
        stats["seconds"] += time.time() - t0
        off = 0
        keep_rows = []
        for inst, info in zip(insts, infos):
            rows = slice(off, off + inst.n)
            off += inst.n
            stats["evaluations"] += info.evaluations
            if info.status not in (capi.APD_OK, capi.APD_WARN_TOL_INFEASIBLE):
                stats["dropped"] += 1
                continue
            wi = W[rows]
            s = inst.n / inst.grid.measure
            targets.append(((wi - wi.mean()) * s ** (2.0 / dim)).astype(np.float32))
            keep_rows.append(np.arange(rows.start, rows.stop))
            counts.append(inst.n)
            stats["instances"] += 1
        keep_np = np.concatenate(keep_rows)
        keep = torch.from_numpy(keep_np).to("cuda")
        feats.append(f[keep])
        # neighbour rows of the kept instances, renumbered to rows of the kept set
        remap = np.full(x.shape[0], -1, dtype=np.int64)
        remap[keep_np] = base + np.arange(keep_np.size)
        k_np = kn.cpu().numpy()[keep_np]
        knns.append(np.where(k_np >= 0, remap[np.maximum(k_np, 0)], -1).astype(np.int32))
        base += keep_np.size
        b.close()
        log(f"  chunk {c0 // chunk}: {len(insts)} instances, {stats['seconds']:.1f} s so far")
    F_all = torch.cat(feats)
    T_all = torch.from_numpy(np.concatenate(targets)).to("cuda")
    K_all = torch.from_numpy(np.concatenate(knns)).to("cuda")
    return F_all, T_all, K_all, counts, stats


def train(dim: int, feats, targets, knn, counts, epochs: int = 40, batch: int = 4096, lr: float = 2e-3,
          mu: float = 0.02, val_frac: float = 0.05, seed: int = 0, log=print):
    """Adam on the neighbour-difference loss (apd_warmstart_train_step_pairs) with a
    small squared-error anchor mu; mini-batches are whole instances (so every
    neighbour of a batch row is in the batch).  The last val_frac of the
    instances is held out.  Returns (params, norm, history)."""
    import torch
    net = capi.WarmStart(dim, init_params(dim, seed))
    n_inst = len(counts)
    n_val = max(1, int(round(val_frac * n_inst)))
    starts = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    S_train = int(starts[n_inst - n_val])
    S = int(starts[-1])
    net.fit_norm(feats[:S_train])
    g = np.random.Generator(np.random.PCG64(seed + 1))
    y_buf = torch.zeros(S, dtype=torch.float32, device="cuda")
    dy_buf = torch.zeros(S, dtype=torch.float32, device="cuda")
    loss_buf = torch.zeros(1, dtype=torch.float32, device="cuda")

    def batches(inst_ids):
        rows, size = [], 0
        for b in inst_ids:
            rows.append(np.arange(starts[b], starts[b + 1], dtype=np.int32))
            size += rows[-1].size
            if size >= batch:
                yield np.concatenate(rows)
                rows, size = [], 0
        if rows:
            yield np.concatenate(rows)

    val_batches = [torch.from_numpy(r).to("cuda") for r in batches(range(n_inst - n_val, n_inst))]

    def val_loss():
        tot, cnt = 0.0, 0
        for r in val_batches:
            net.train_step_pairs(r, feats, targets, knn, y_buf, dy_buf, 0.0, mu=mu, loss_out=loss_buf)
            tot += float(loss_buf.item()) * r.shape[0]
            cnt += r.shape[0]
        return tot / max(1, cnt)

    hist = {"val0": val_loss(), "val": []}
    steps_per_epoch = max(1, S_train // batch)
    total = epochs * steps_per_epoch
    step = 0
    t0 = time.time()
    for ep in range(epochs):
        for r in batches(g.permutation(n_inst - n_val)):
            lr_k = lr * 0.5 * (1.0 + math.cos(math.pi * min(step, total) / total))
            net.train_step_pairs(torch.from_numpy(r).to("cuda"), feats, targets, knn, y_buf, dy_buf, lr_k, mu=mu)
            step += 1
        hist["val"].append(val_loss())
        log(f"  epoch {ep}: val loss {hist['val'][-1]:.4f} ({time.time() - t0:.1f} s)")
    # the same loss for the zero prediction (the plain start), for scale
    hist["zero_val"] = None
    params, norm = net.get()
    return params, norm, hist


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=2, choices=[2, 3])
    ap.add_argument("--instances", type=int, default=5000)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    from . import build
    build.build()
    capi.load()
    t0 = time.time()
    feats, targets, knn, counts, stats = generate(args.dim, args.instances, TRAIN_SEED[args.dim])
    print(json.dumps({"generate": stats, "samples": int(feats.shape[0])}))
    params, norm, hist = train(args.dim, feats, targets, knn, counts, epochs=args.epochs)
    meta_d = {"dim": args.dim, "instances_drawn": args.instances, "instances_used": stats["instances"],
              "samples": int(feats.shape[0]), "train_seed": TRAIN_SEED[args.dim], "epochs": args.epochs,
              "val_loss": hist["val"][-1], "val_loss_init": hist["val0"],
              "loss": "neighbour-difference + 0.02 squared error", "generate_seconds": stats["seconds"],
              "total_seconds": time.time() - t0}
    out = args.out or path(args.dim)
    os.makedirs(os.path.dirname(out), exist_ok=True)
    np.savez(out, params=params, norm=norm, meta=json.dumps(meta_d))
    print(json.dumps(meta_d))


if __name__ == "__main__":
    main()
