"""Train the bin planner on per-tile statistics the pipeline logs itself.

Data (one "render" = one seeded scene and camera, EXACT mode, K = 64):
  * the frame's binned stream is built once (projection, tile intersection,
    depth range, bins);
  * gs_tile_features gives each tile's 8 features;
  * the counting raster (gs_rasterize_fwd_plan) logs each tile's bins
    needed: 1 + the bin holding the last entry any of its pixels visits;
  * the label of a tile is the smallest class whose first-pass bins (class
    c < 5: the fewest bins from the front holding 64 << c entries; class 5:
    all) cover the bins it needs.
Training: mini-batch Adam on softmax cross entropy, on the GPU, entirely
through the library's own kernels (gs_mlp_forward, gs_mlp_loss_grad,
gs_mlp_backward, gs_adam_step).  Feature standardisation is folded into the
first layer afterwards, so the inference kernel takes raw features.  At
inference the planner takes the smallest class whose cumulative probability
reaches cfg.planner_quantile.

    python -m paper_2609_03613_gb300.planner_train --out planner_weights.npy

writes the float32 parameters (GS_PLAN_PARAMS values) and prints a summary,
with a held-out evaluation of whole frames (planned against every bin in one
pass).  The committed `planner_weights.npy` next to this file was written
this way.
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
    """(scene, camera) pairs: scenes of the mid workload's distribution, half
    the cameras on spheres around them (resolutions 512^2 .. 1080p), half
    inside one of their dense clusters (deep tiles, like the heavy
    workloads)."""
    for i in range(n_scenes):
        seed = scene_seed0 + i
        sc = scenes.mixture_scene(sizes[i % len(sizes)], seed)
        cams = scenes.batch_cameras(views_per_scene - views_per_scene // 2, cam_seed0 + 97 * i)
        for j in range(views_per_scene // 2):
            w, h = scenes.BATCH_RESOLUTIONS[(i + j) % len(scenes.BATCH_RESOLUTIONS)]
            cams.append(scenes.heavy_camera(seed, cam_seed0 + 97 * i + 50 + j, w, h, w * (1100.0 / 1920.0)))
        for cam in cams:
            yield sc, cam


def frame(ctx, ds, cam):
    proj = ctx.project(ds, cam)
    isect, m_cap, m_dev, m = ctx.tile_intersect(proj, ds.n, cam)
    words, offsets, _ = ctx.sort_or_bin(proj, ds.scales, ds.n, cam, isect, m_cap, m_dev)
    return proj, words, offsets


def class_bins(off, K, c):
    """First-pass bins of class c for every tile (off: [T*K + 1] numpy)."""
    T = (len(off) - 1) // K
    if c >= G.PLAN_CLASSES - 1:
        return np.full(T, K, np.int64)
    o = off[:T * K + 1].astype(np.int64)
    cum = o[1:].reshape(T, K) - o[0:T * K:K][:, None]
    hit = cum >= (64 << c)
    return np.where(hit.any(axis=1), np.argmax(hit, axis=1) + 1, K)


def labels_of(needed, off, K):
    """Smallest class whose first-pass bins cover each tile's bins needed."""
    y = np.full(len(needed), G.PLAN_CLASSES - 1, np.int64)
    for c in range(G.PLAN_CLASSES - 2, -1, -1):
        y = np.where(class_bins(off, K, c) >= needed, c, y)
    return y


def log_tiles(ctx, ds, cam):
    """features [T][8], labels [T] and offsets (numpy) of one render."""
    import torch
    proj, words, offsets = frame(ctx, ds, cam)
    feat = ctx.tile_features(cam, offsets)
    needed = ctx.rasterize_fwd_plan(proj, ds.n, cam, words, offsets, needed=True)[4]
    torch.cuda.synchronize()
    off = offsets.cpu().numpy().astype(np.int64)
    return feat.cpu().numpy(), labels_of(needed.cpu().numpy(), off, ctx.stride), off


def collect(renders):
    import torch
    ctx = G.Context("exact")
    feats, labels = [], []
    last_sc, ds = None, None
    for sc, cam in renders:
        if sc is not last_sc:
            ds = G.DeviceScene.from_numpy(sc)
            last_sc = sc
        f, y, _ = log_tiles(ctx, ds, cam)
        keep = f[:, 0] > 0.0  # tiles with entries
        feats.append(f[keep])
        labels.append(y[keep])
    assert ctx.error() == 0
    torch.cuda.synchronize()
    return np.concatenate(feats), np.concatenate(labels)


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


def evaluate(params, renders, iters=10, q=0.9):
    """Whole frames (gs_render, un-captured, stage events) of each held-out
    render with the planner (two passes) and with every bin in one pass;
    images compared bit for bit.  Returns per render a dict of frame and
    bin-stage ms for both, and the tiles the planner left to the second
    pass."""
    import torch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    fixed = G.Context("exact")
    planned = G.Context("exact", planner=1, planner_quantile=q)
    planned.set_planner_weights(torch.from_numpy(params))
    out = []
    last_sc, ds = None, None
    for sc, cam in renders:
        if sc is not last_sc:
            ds = G.DeviceScene.from_numpy(sc)
            last_sc = sc
        a = fixed.render(ds, cam)
        b = planned.render(ds, cam)
        torch.cuda.synchronize()
        assert all(torch.equal(x, y) for x, y in zip(a, b))
        r = {}
        for name, ctx in (("fixed", fixed), ("planned", planned)):
            ctx.enable_timing(True)
            ev, st = [], {}
            for i in range(iters):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ctx.render(ds, cam, flags=G.RENDER_NO_SYNC)
                e1.record()
                for k, v in ctx.stage_times().items():
                    st.setdefault(k, []).append(v)
                ev.append((e0, e1))
            torch.cuda.synchronize()
            fr = [a.elapsed_time(b) for a, b in ev]
            ctx.enable_timing(False)
            r[name] = {"frame_ms": float(np.median(fr)), "bin_ms": float(np.median(st["bin"])),
                       "complete_ms": float(np.median(st["complete"]))}
        T = G.n_tiles(cam.width, cam.height, 16)
        r["flagged"] = int(planned.flagged_tiles())
        r["tiles"] = T
        out.append(r)
    assert fixed.error() == 0 and planned.error() == 0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--scenes", type=int, default=20)
    ap.add_argument("--views", type=int, default=10)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--quantile", type=float, default=0.9)
    args = ap.parse_args()
    t0 = time.time()
    X, y = collect(training_renders(args.scenes, args.views, 7000, 20000))
    t1 = time.time()
    params, hist = train(X, y, epochs=args.epochs)
    t2 = time.time()
    np.save(args.out, params)
    counts = np.bincount(y, minlength=G.PLAN_CLASSES)
    held = evaluate(params, training_renders(4, 4, 9000, 30000), q=args.quantile)
    fx = sum(h["fixed"]["frame_ms"] for h in held)
    pl = sum(h["planned"]["frame_ms"] for h in held)
    print(json.dumps({"samples": int(len(y)), "label_counts": counts.tolist(),
                      "loss_first_batch_per_epoch": [round(h, 4) for h in hist],
                      "held_out_frame_ms_fixed": round(fx, 4), "held_out_frame_ms_planned": round(pl, 4),
                      "held_out_gain": round(1.0 - pl / fx, 4),
                      "held_out_flagged_tiles": [h["flagged"] for h in held],
                      "held_out_tiles": [h["tiles"] for h in held],
                      "held_out_per_render": held,
                      "collect_s": round(t1 - t0, 1), "train_s": round(t2 - t1, 1), "out": args.out}))


if __name__ == "__main__":
    main()
