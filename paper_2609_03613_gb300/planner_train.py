"""Train the bin planner on per-tile statistics the pipeline logs itself.

Data (one "render" = one seeded scene and camera, EXACT mode, K = 64):
  * the frame's binned stream is built once (projection, tile intersection,
    depth range, bins);
  * gs_tile_features gives each tile's 8 features;
  * the raster runs once per chunk class c = 0..5 with every tile forced to c
    (gs_rasterize_fwd_plan) and records each tile's clock64() cycles, `reps`
    times; the label of a tile is the class of its smallest median cycles
    (softmax cross entropy on these labels saved more cycles on a held-out
    split than an expected-cost loss or labels that keep the default class
    within a few percent).
Training: mini-batch Adam on the GPU, entirely through the library's own
kernels (gs_mlp_forward, gs_mlp_loss_grad, gs_mlp_backward, gs_adam_step).
Feature standardisation is folded into the first layer afterwards, so the
inference kernel takes raw features.

    python -m paper_2609_03613_gb300.planner_train --out planner_weights.npy

writes the float32 parameters (GS_PLAN_PARAMS values) and prints a summary.
The committed `planner_weights.npy` next to this file was written this way.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import scenes
from . import tilegs as G

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "planner_weights.npy")


def training_renders(n_scenes, views_per_scene, scene_seed0, cam_seed0, sizes=(300_000, 600_000, 1_000_000)):
    """(scene, camera) pairs: scenes of the mid workload's distribution, cameras
    on spheres around them with resolutions 512^2 .. 1080p."""
    for i in range(n_scenes):
        sc = scenes.mixture_scene(sizes[i % len(sizes)], scene_seed0 + i)
        for cam in scenes.batch_cameras(views_per_scene, cam_seed0 + 97 * i):
            yield sc, cam


def frame(ctx, ds, cam):
    proj = ctx.project(ds, cam)
    isect, m_cap, m_dev, m = ctx.tile_intersect(proj, ds.n, cam)
    words, offsets, _ = ctx.sort_or_bin(proj, ds.scales, ds.n, cam, isect, m_cap, m_dev)
    return proj, words, offsets


def log_tiles(ctx, ds, cam, reps=3):
    """features [T][8] (numpy) and median cycles [T][6] (numpy) of one render."""
    import torch
    proj, words, offsets = frame(ctx, ds, cam)
    feat = ctx.tile_features(cam, offsets)
    T = feat.shape[0]
    cyc = np.zeros((reps, G.PLAN_CLASSES, T))
    for r in range(reps):
        for c in range(G.PLAN_CLASSES):
            plan = torch.full((T,), c, dtype=torch.uint8, device=feat.device)
            _, _, _, cy = ctx.rasterize_fwd_plan(proj, ds.n, cam, words, offsets, plan=plan, cycles=True)
            cyc[r, c] = cy.cpu().numpy()
    torch.cuda.synchronize()
    return feat.cpu().numpy(), np.median(cyc, axis=0).T


def collect(renders, reps=3):
    import torch
    ctx = G.Context("exact")
    feats, cycles = [], []
    last_sc, ds = None, None
    for sc, cam in renders:
        if sc is not last_sc:
            ds = G.DeviceScene.from_numpy(sc)
            last_sc = sc
        f, c = log_tiles(ctx, ds, cam, reps)
        keep = f[:, 0] > 0.0  # tiles with entries
        feats.append(f[keep])
        cycles.append(c[keep])
    assert ctx.error() == 0
    torch.cuda.synchronize()
    return np.concatenate(feats), np.concatenate(cycles)


def init_params(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    F, H, C = G.PLAN_FEATURES, G.PLAN_HIDDEN, G.PLAN_CLASSES
    parts = [rng.normal(0, np.sqrt(2.0 / F), H * F), np.zeros(H), rng.normal(0, np.sqrt(2.0 / H), H * H),
             np.zeros(H), rng.normal(0, np.sqrt(1.0 / H), C * H), np.zeros(C)]
    return np.concatenate(parts).astype(np.float32)


def fold_standardisation(params, mu, sd):
    """Parameters taking raw features: W1' = W1 / sd, b1' = b1 - W1' mu."""
    F, H = G.PLAN_FEATURES, G.PLAN_HIDDEN
    p = params.astype(np.float64).copy()
    W1 = p[:H * F].reshape(H, F) / sd
    p[:H * F] = W1.ravel()
    p[H * F:H * F + H] -= W1 @ mu
    return p.astype(np.float32)


def train(X, y, epochs=20, batch=4096, lr=3e-3, seed=0):
    """Adam on the GPU through the library kernels; returns (params, loss history)."""
    import torch
    dev = torch.device("cuda")
    mu, sd = X.mean(axis=0), X.std(axis=0) + 1e-6
    Xs = torch.from_numpy(((X - mu) / sd).astype(np.float32)).to(dev)
    ys = torch.from_numpy(y.astype(np.int32)).to(dev)
    P = torch.from_numpy(init_params(seed)).to(dev)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    rng = np.random.Generator(np.random.PCG64(seed))
    n = Xs.shape[0]
    step, hist = 0, []
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(n)).to(dev)
        tot = 0.0
        for b0 in range(0, n - batch + 1, batch):
            idx = order[b0:b0 + batch]
            xb, yb = Xs[idx].contiguous(), ys[idx].contiguous()
            acts, logits = G.mlp_forward(P, xb)
            loss, dz = G.mlp_loss_grad(logits, yb)
            grads = G.mlp_backward(P, xb, acts, dz)
            step += 1
            G.adam_step(P, grads, m, v, step, lr)
            tot += float(loss.item()) if b0 == 0 else 0.0
        hist.append(tot)
    torch.cuda.synchronize()
    return fold_standardisation(P.cpu().numpy(), mu, sd), hist


def labels_of(cycles, default_class=2, margin=0.0):
    """argmin class per tile; with margin > 0, tiles whose best class is within
    `margin` of the default's cycles keep the default."""
    best = np.argmin(cycles, axis=1)
    dflt = cycles[:, default_class]
    keep_default = cycles[np.arange(len(best)), best] >= (1.0 - margin) * dflt
    return np.where(keep_default, default_class, best)


def evaluate(params, renders, iters=20):
    """Raster ms per render with the planner's per-tile plan and with the
    fixed chunk size (every tile class 2 = the default 256 entries), on the
    same stream; images compared bit for bit.  Returns a list of
    (fixed_ms, planned_ms)."""
    import torch
    ctx = G.Context("exact")
    ctx.set_planner_weights(torch.from_numpy(params))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = []
    last_sc, ds = None, None
    for sc, cam in renders:
        if sc is not last_sc:
            ds = G.DeviceScene.from_numpy(sc)
            last_sc = sc
        proj, words, offsets = frame(ctx, ds, cam)
        plan = ctx.plan_tiles(ctx.tile_features(cam, offsets))
        ref = ctx.rasterize_fwd_plan(proj, ds.n, cam, words, offsets)
        got = ctx.rasterize_fwd_plan(proj, ds.n, cam, words, offsets, plan=plan)
        assert all(torch.equal(a, b) for a, b in zip(ref[:3], got[:3]))
        ms = []
        for p in (None, plan):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(iters)]
            for i in range(iters):
                flush.zero_()
                ev[i][0].record()
                ctx.rasterize_fwd_plan(proj, ds.n, cam, words, offsets, plan=p)
                ev[i][1].record()
            torch.cuda.synchronize()
            ms.append(float(np.median([a.elapsed_time(b) for a, b in ev])))
        out.append(tuple(ms))
    assert ctx.error() == 0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--scenes", type=int, default=20)
    ap.add_argument("--views", type=int, default=10)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--dump", default=None, help="npz of a 300k-tile sample of the logged data")
    args = ap.parse_args()
    t0 = time.time()
    X, cyc = collect(training_renders(args.scenes, args.views, 7000, 20000), args.reps)
    t1 = time.time()
    y = labels_of(cyc)
    params, hist = train(X, y, epochs=args.epochs)
    t2 = time.time()
    np.save(args.out, params)
    if args.dump:
        rng = np.random.Generator(np.random.PCG64(1))
        sel = rng.choice(len(y), min(len(y), 300_000), replace=False)
        np.savez_compressed(args.dump, X=X[sel].astype(np.float32), cycles=cyc[sel].astype(np.float32))
    counts = np.bincount(y, minlength=G.PLAN_CLASSES)
    perfect = 1.0 - cyc[np.arange(len(y)), np.argmin(cyc, axis=1)].sum() / cyc[:, 2].sum()
    held = evaluate(params, training_renders(4, 5, 9000, 30000))
    fixed, planned = np.array(held).T
    print(json.dumps({"samples": int(len(y)), "label_counts": counts.tolist(),
                      "cycles_sum_gain_if_perfect_vs_class2": round(float(perfect), 4),
                      "loss_first_batch_per_epoch": [round(h, 4) for h in hist],
                      "held_out_raster_ms_fixed": round(float(fixed.sum()), 4),
                      "held_out_raster_ms_planned": round(float(planned.sum()), 4),
                      "held_out_gain": round(float(1.0 - planned.sum() / fixed.sum()), 4),
                      "held_out_per_render": [[round(a, 4), round(b, 4)] for a, b in held],
                      "collect_s": round(t1 - t0, 1), "train_s": round(t2 - t1, 1), "out": args.out}))


if __name__ == "__main__":
    main()
