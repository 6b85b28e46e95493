"""Pins for the planner oracle (oracle/planner.py): the tile features on
hand-made bin histograms, the network's gradient by central finite
differences, the cross-entropy gradient and its closed form at uniform
logits, and Adam's first step (update = -lr g / (|g| + eps)).
None of these runs the CUDA path."""
import math

import numpy as np

from oracle import planner as PL


def _offsets(per_tile_counts):
    counts = np.concatenate(per_tile_counts)
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)


def test_features_by_hand():
    K = 16
    t0 = np.zeros(K, int); t0[3] = 5; t0[4] = 2; t0[10] = 9          # first 3, last 10
    t1 = np.zeros(K, int)                                              # empty tile
    t2 = np.zeros(K, int); t2[0] = 1                                   # one entry in bin 0
    f = PL.tile_features(_offsets([t0, t1, t2]), K, 3)
    # K/8 = 2 bins from the first nonempty one: bins 3, 4 -> 7 entries
    np.testing.assert_allclose(f[0], [math.log1p(16), math.log1p(9), 3 / 16, 3 / 16, 10 / 16,
                                      math.log1p(5), math.log1p(7), math.log1p(16 / 3)])
    np.testing.assert_allclose(f[1], [0, 0, 0, 1, 0, 0, 0, 0])
    np.testing.assert_allclose(f[2], [math.log1p(1), math.log1p(1), 1 / 16, 0, 0, math.log1p(1),
                                      math.log1p(1), math.log1p(1)])


def _rand_params(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(0.0, 0.3, PL.N_PARAMS)


def test_network_gradient_matches_central_differences():
    rng = np.random.Generator(np.random.PCG64(3))
    P = _rand_params(2)
    X = rng.normal(0.0, 1.0, (7, PL.F))
    y = rng.integers(0, PL.C, 7)

    def loss(p):
        return PL.xent(PL.forward(p, X)[2], y)[0]

    h1, h2, z = PL.forward(P, X)
    _, dz = PL.xent(z, y)
    g = PL.backward(P, X, h1, h2, dz)
    idx = rng.choice(PL.N_PARAMS, 300, replace=False)
    idx = np.concatenate([idx, np.arange(PL.N_PARAMS - 2 * PL.C * PL.H // PL.H, PL.N_PARAMS)])
    for i in idx:
        h = 1e-6
        p = P.copy(); p[i] += h
        lp = loss(p)
        p[i] -= 2 * h
        lm = loss(p)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_xent_uniform_logits_and_gradient():
    z = np.zeros((4, PL.C))
    y = np.array([0, 1, 5, 2])
    loss, d = PL.xent(z, y)
    assert abs(loss - math.log(PL.C)) < 1e-15
    expect = np.full((4, PL.C), 1.0 / PL.C)
    expect[np.arange(4), y] -= 1.0
    np.testing.assert_allclose(d, expect / 4, atol=1e-15)
    # gradient rows sum to zero (softmax sums to one)
    rng = np.random.Generator(np.random.PCG64(4))
    _, d2 = PL.xent(rng.normal(0, 3, (9, PL.C)), rng.integers(0, PL.C, 9))
    np.testing.assert_allclose(d2.sum(axis=1), 0.0, atol=1e-15)


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p, m, v = PL.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_plan_is_argmax_with_lowest_class_on_ties():
    P = np.zeros(PL.N_PARAMS)
    W1, b1, W2, b2, W3, b3 = PL.unpack(P)
    b3 = np.array([0.0, 1.0, 1.0, -1.0, 0.5, 1.0])
    P2 = PL.pack(W1, b1, W2, b2, W3, b3)
    assert list(PL.plan(P2, np.zeros((2, PL.F)))) == [1, 1]
