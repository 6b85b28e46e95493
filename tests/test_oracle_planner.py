"""Pins for the planner oracle (oracle/planner.py): the tile features on
hand-made bin histograms, the network's gradient by central finite
differences, the cross-entropy gradient and its closed form at uniform
logits, Adam's first step (update = -lr g / (|g| + eps)), and the decision
rule, class-to-bins map and training label on hand-computed cases.
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


def test_plan_of_a_bias_only_network():
    """Zero weights: every tile gets the classes of the output bias alone.
    Bias (0, 0, log 2, -50, ...) has cumulative probabilities .25 .5 1 ...,
    so q = 0.5 picks class 1 and q = 0.9 class 2, whatever the features."""
    P = np.zeros(PL.N_PARAMS)
    W1, b1, W2, b2, W3, b3 = PL.unpack(P)
    b3 = np.array([0.0, 0.0, math.log(2.0), -50.0, -50.0, -50.0])
    P2 = PL.pack(W1, b1, W2, b2, W3, b3)
    K = 8
    off = _offsets([np.array([10, 0, 60, 0, 100, 500, 0, 30]), np.zeros(K, int)])
    X = PL.tile_features(off, K, 2)
    cls, bins = PL.plan(P2, X, off, K, 2, q=0.5)
    assert cls.tolist() == [1, 1] and bins.tolist() == [5, 8]
    cls, bins = PL.plan(P2, X, off, K, 2, q=0.9)
    assert cls.tolist() == [2, 2] and bins.tolist() == [6, 8]


def test_decision_rule_by_hand():
    # softmax of (0, 0, log 2, ...) etc.: cumulative probabilities by hand
    z = np.array([[0.0, 0.0, math.log(2.0), -50.0, -50.0, -50.0],   # p = .25 .25 .5 ~0 ~0 ~0
                  [-50.0, -50.0, -50.0, -50.0, -50.0, 0.0],       # all mass on class 5
                  [0.0] * 6])                                    # uniform: cum = (c+1)/6
    np.testing.assert_array_equal(PL.decide(z, 0.5), [1, 5, 2])
    np.testing.assert_array_equal(PL.decide(z, 0.9), [2, 5, 5])   # 5/6 < 0.9 -> class 5
    np.testing.assert_array_equal(PL.decide(z, 0.2), [0, 5, 1])


def test_class_bins_by_hand():
    K = 8
    t0 = np.array([10, 0, 60, 0, 100, 500, 0, 30])   # cumulative 10 10 70 70 170 670 670 700
    t1 = np.zeros(K, int)                            # empty: never reaches -> K
    t2 = np.array([3000, 0, 0, 0, 0, 0, 0, 1])       # the first bin alone holds 3000
    off = _offsets([t0, t1, t2])
    for c, want in ((0, [3, 8, 1]), (1, [5, 8, 1]), (2, [6, 8, 1]), (3, [6, 8, 1]), (4, [8, 8, 1]),
                    (5, [8, 8, 8])):
        np.testing.assert_array_equal(PL.class_bins(off, K, 3, [c] * 3), want, err_msg=str(c))


def test_bins_needed_and_label_by_hand():
    K = 8
    t0 = np.array([10, 0, 60, 0, 100, 500, 0, 30])
    off = _offsets([t0, np.zeros(K, int)])
    # tile 0 spans [0, 700): an end inside bin 2 ([10, 70)) needs 3 bins
    assert PL.bins_needed(off, K, 2, [40, 700]).tolist() == [3, 0]
    assert PL.bins_needed(off, K, 2, [70, 700]).tolist() == [3, 0]   # the last visit is entry 69
    assert PL.bins_needed(off, K, 2, [71, 700]).tolist() == [5, 0]   # entry 70 sits in bin 4 ([70, 170))
    assert PL.bins_needed(off, K, 2, [700, 700]).tolist() == [8, 0]
    need = np.array([3, 0])
    # class 0 keeps 3 bins (64 entries reached in bin 2): it covers 3 bins
    assert PL.label(need, off, K, 2).tolist() == [0, 0]
    assert PL.label(np.array([5, 0]), off, K, 2).tolist() == [1, 0]
    assert PL.label(np.array([6, 0]), off, K, 2).tolist() == [2, 0]
    assert PL.label(np.array([8, 0]), off, K, 2).tolist() == [4, 0]


def test_tile_end_from_visits_by_hand():
    # a 2x1 tile grid of 2x2 tiles on a 3x2 image (ragged right column)
    off = np.array([0, 5, 9])
    nt = np.array([[1, 4, 2], [0, 3, 1]])
    np.testing.assert_array_equal(PL.tile_end_from_visits(off, 1, 2, 3, 2, nt), [4, 7])
