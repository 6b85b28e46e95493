"""CPU oracle of the scene's spatial order (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's reference leg may use
this module; the CUDA library never calls it and shares no code with it.

Raster-order-aware storage (the geometry-layout direction of Sec. 6.2): the
Gaussians are stored in the Z-order (Morton order) of their means.  The paper
names the direction, not an order; this definition is the project's, written
out plainly in float32 numpy (each step one correctly rounded operation):
  lo_a = min over Gaussians of x_a, hi_a = max, ext_a = hi_a - lo_a,
  s_a = 1024 / ext_a (0 when ext_a == 0),
  c_a = min(1023, trunc((x_a - lo_a) * s_a)),
  code = bits of c_x at 3k, of c_y at 3k+1, of c_z at 3k+2 (k = 0..9),
  perm = the gids stably sorted by code (equal codes keep gid order).
"""
from __future__ import annotations

import numpy as np


def cells(means):
    """Per-axis grid cells c [n][3] (int64) of the means [n][3]."""
    x = np.asarray(means, np.float32)
    n = x.shape[0]
    if n == 0:
        return np.zeros((0, 3), np.int64)
    lo = x.min(axis=0)
    hi = x.max(axis=0)
    ext = (hi - lo).astype(np.float32)
    s = np.zeros(3, np.float32)
    for a in range(3):
        if ext[a] > 0:
            s[a] = np.float32(1024.0) / ext[a]
    d = (x - lo).astype(np.float32)
    q = (d * s).astype(np.float32)
    c = np.trunc(q).astype(np.int64)
    return np.clip(c, 0, 1023)


def morton_codes(means):
    """30-bit codes [n] (int64): bit k of the x, y, z cells at 3k, 3k+1, 3k+2."""
    c = cells(means)
    code = np.zeros(c.shape[0], np.int64)
    for k in range(10):
        for a in range(3):
            code |= ((c[:, a] >> k) & 1) << (3 * k + a)
    return code


def spatial_order(means):
    """perm [n] (int32): position i of the reordered scene holds Gaussian perm[i]."""
    return np.argsort(morton_codes(means), kind="stable").astype(np.int32)


def permute_scene(scene, perm):
    """A scenes.Scene-like object with every per-Gaussian array taken in perm order."""
    import dataclasses
    p = np.asarray(perm)
    fields = {f.name: getattr(scene, f.name) for f in dataclasses.fields(scene)}
    for k, v in fields.items():
        if isinstance(v, np.ndarray) and v.ndim >= 1 and v.shape[0] == len(p):
            fields[k] = np.ascontiguousarray(v[p])
    return type(scene)(**fields)
