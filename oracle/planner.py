"""CPU oracle of the bin planner's arithmetic (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's reference leg may use
this module; the CUDA library never calls it and shares no code with it.

What it restates, in float64 numpy, one plain step at a time:
  * the per-tile features of a binned stream (from the K fine-bin offsets of
    each tile): log1p(n), log1p(max bin), nonempty/K, first/K, last/K,
    log1p(first bin count), log1p(entries in the K/8 bins from the first
    nonempty one), log1p(n / nonempty);
  * the planner network 8 -> 64 -> 64 -> 6 with ReLU, parameters packed as
    W1[64][8] b1[64] W2[64][64] b2[64] W3[6][64] b3[6];
  * mean softmax cross entropy and its gradient, backpropagation through the
    network, and one Adam step (Kingma & Ba, 2015: m, v moving averages of the
    gradient and its square, bias-corrected, step lr * m_hat / (sqrt(v_hat) + eps));
  * the decision: the smallest class whose cumulative softmax probability
    reaches the quantile q, and the first-pass bins of a class (class c < 5:
    the fewest bins from the tile's front holding at least 64 << c entries,
    all K for class 5);
  * the training label of a tile: the bins it needs, 1 + the bin holding the
    last entry any of its pixels visits when compositing its whole list (the
    stopping entry, or the list's last for a pixel that never stops), and the
    smallest class whose bins cover them.
The paper has no planner (it uses one bin count and spacing for every tile,
Sec. 5.3, and leaves distribution-dependent settings to future work, Sec. 7);
these definitions are the project's.
"""
from __future__ import annotations

import numpy as np

F, H, C = 8, 64, 6
N_PARAMS = H * F + H + H * H + H + C * H + C


def unpack(params):
    p = np.asarray(params, np.float64)
    assert p.shape == (N_PARAMS,)
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + C * H].reshape(C, H); o += C * H
    b3 = p[o:o + C]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(a) for a in (W1, b1, W2, b2, W3, b3)]).astype(np.float64)


def tile_features(offsets, K, n_tiles):
    """Features [T][8] from offsets [T*K + 1] (tile t's bins are offsets[t*K .. t*K + K])."""
    off = np.asarray(offsets, np.int64)
    out = np.zeros((n_tiles, F))
    for t in range(n_tiles):
        cnt = np.diff(off[t * K:t * K + K + 1])
        n = int(off[t * K + K] - off[t * K])
        nz = np.nonzero(cnt > 0)[0]
        ne = len(nz)
        first = int(nz[0]) if ne else K
        last = int(nz[-1]) if ne else -1
        span = max(K // 8, 1)
        front = int(cnt[first:first + span].sum()) if ne else 0
        out[t] = [np.log1p(n), np.log1p(cnt.max() if K else 0), ne / K,
                  first / K if ne else 1.0, last / K if ne else 0.0,
                  np.log1p(cnt[first] if ne else 0), np.log1p(front),
                  np.log1p(n / ne) if ne else 0.0]
    return out


def forward(params, X):
    """(h1, h2, logits) for X [B][8]."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    X = np.asarray(X, np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h1, h2, h2 @ W3.T + b3


def xent(logits, labels):
    """Mean softmax cross entropy and its gradient w.r.t. the logits."""
    z = np.asarray(logits, np.float64)
    B = z.shape[0]
    m = z.max(axis=1, keepdims=True)
    e = np.exp(z - m)
    s = e.sum(axis=1, keepdims=True)
    y = np.asarray(labels, np.int64)
    loss = float(np.mean(np.log(s[:, 0]) + m[:, 0] - z[np.arange(B), y]))
    d = e / s
    d[np.arange(B), y] -= 1.0
    return loss, d / B


def backward(params, X, h1, h2, dlogits):
    """Parameter gradient (packed like params) of sum_s dlogits[s] . logits[s]."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    X = np.asarray(X, np.float64)
    dz = np.asarray(dlogits, np.float64)
    dW3 = dz.T @ h2
    db3 = dz.sum(axis=0)
    d2 = (dz @ W3) * (h2 > 0.0)
    dW2 = d2.T @ h1
    db2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (h1 > 0.0)
    dW1 = d1.T @ X
    db1 = d1.sum(axis=0)
    return pack(dW1, db1, dW2, db2, dW3, db3)


def adam(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step; returns (params, m, v)."""
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * grads
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * grads * grads
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return np.asarray(params, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


def decide(logits, q):
    """Smallest class whose cumulative softmax probability reaches q (the
    last class when none before it does)."""
    z = np.asarray(logits, np.float64)
    e = np.exp(z - z.max(axis=1, keepdims=True))
    cum = np.cumsum(e, axis=1) / e.sum(axis=1, keepdims=True)
    hit = cum[:, :C - 1] >= q
    return np.where(hit.any(axis=1), np.argmax(hit, axis=1), C - 1)


def class_bins(offsets, K, n_tiles, classes):
    """First-pass bins per tile for the given class of each tile."""
    off = np.asarray(offsets, np.int64)
    out = np.zeros(n_tiles, np.int64)
    for t in range(n_tiles):
        c = int(classes[t])
        if c >= C - 1:
            out[t] = K
            continue
        cum = off[t * K + 1:t * K + K + 1] - off[t * K]
        hit = np.nonzero(cum >= (64 << c))[0]
        out[t] = hit[0] + 1 if len(hit) else K
    return out


def plan(params, X, offsets, K, n_tiles, q=0.9):
    """(classes, first-pass bins) per tile."""
    cls = decide(forward(params, X)[2], q)
    return cls, class_bins(offsets, K, n_tiles, cls)


def bins_needed(offsets, K, n_tiles, tile_end):
    """Bins each tile needs given tile_end[t], the stream position after the
    last entry any of its pixels visits: 1 + the bin holding tile_end - 1;
    0 for an empty tile."""
    off = np.asarray(offsets, np.int64)
    out = np.zeros(n_tiles, np.int64)
    for t in range(n_tiles):
        s0 = off[t * K]
        e = int(tile_end[t])
        if e <= s0:
            continue
        seg = off[t * K:t * K + K + 1]
        out[t] = int(np.searchsorted(seg, e - 1, side="right") - 1) + 1
    return out


def tile_end_from_visits(offsets, K, tile, width, height, ntests):
    """tile_end per tile from the per-pixel visit counts of compositing the
    tiles' whole lists in order (ntests [H][W]: entries each pixel visited,
    the stopping one included): the span start plus the largest count."""
    off = np.asarray(offsets, np.int64)
    tx = (width + tile - 1) // tile
    ty = (height + tile - 1) // tile
    out = np.zeros(tx * ty, np.int64)
    for t in range(tx * ty):
        x0, y0 = (t % tx) * tile, (t // tx) * tile
        blk = ntests[y0:min(y0 + tile, height), x0:min(x0 + tile, width)]
        out[t] = off[t * K] + (int(blk.max()) if blk.size else 0)
    return out


def label(needed, offsets, K, n_tiles):
    """Smallest class whose first-pass bins cover the bins a tile needs."""
    out = np.full(n_tiles, C - 1, np.int64)
    for c in range(C - 2, -1, -1):
        b = class_bins(offsets, K, n_tiles, np.full(n_tiles, c))
        out = np.where(b >= needed, c, out)
    return out
