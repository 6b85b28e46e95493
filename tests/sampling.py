"""Test helpers (no GPU): per-tile entry counts of the oracle's projected
rects and (depth, gid)-sorted brute-force lists of a few sampled tiles, so
that full-size frames can be checked tile by tile against the oracle's
compositing without building every tile's list."""
import numpy as np


def tile_counts(P, tx, ty):
    """Per-tile entry counts of the visible rects (2D difference array)."""
    r = P["rect"].astype(np.int64)[P["visible"] == 1]
    D = np.zeros((ty + 1, tx + 1), np.int64)
    np.add.at(D, (r[:, 1], r[:, 0]), 1)
    np.add.at(D, (r[:, 1], r[:, 2]), -1)
    np.add.at(D, (r[:, 3], r[:, 0]), -1)
    np.add.at(D, (r[:, 3], r[:, 2]), 1)
    return D.cumsum(0).cumsum(1)[:ty, :tx].ravel()


def sampled_stream(P, tiles, tx, ty):
    """Offsets [T+1] and stream words with the (depth, gid)-sorted lists of
    the sampled tiles only (every other tile empty)."""
    r = P["rect"]
    vis = np.nonzero(P["visible"] == 1)[0]
    zb = P["depth"].view(np.uint32).astype(np.uint64)
    rv = r[vis]
    lists = {}
    for t in tiles:
        y, x = divmod(int(t), tx)
        g = vis[(rv[:, 0] <= x) & (x < rv[:, 2]) & (rv[:, 1] <= y) & (y < rv[:, 3])]
        lists[int(t)] = np.sort((zb[g] << np.uint64(32)) | g.astype(np.uint64))
    counts = np.zeros(tx * ty, np.int64)
    for t, l in lists.items():
        counts[t] = l.shape[0]
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    stream = np.concatenate([lists[t] for t in sorted(lists)]) if lists else np.zeros(0, np.uint64)
    return off, stream
