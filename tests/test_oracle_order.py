"""Pins for the spatial-order oracle (oracle/order.py): hand-computed codes,
the cube's corner order, stability on duplicates, the degenerate extent,
Z-order locality, and that the oracle's image of a permuted scene is the
original image (the reorder changes storage, not the picture).
None of these runs the CUDA path."""
import numpy as np

import oracle as O
from oracle import order as OR
from paper_2609_03613_gb300 import scenes


def test_codes_by_hand():
    # extent 1 on every axis (points at 0 and 1), so s = 1024 and cells are
    # 1024 * coordinate: (0.25, 0.5, 0.75) -> cells (256, 512, 768):
    # x bit 8 -> code bit 24; y bit 9 -> bit 28; z bits 8, 9 -> bits 26, 29
    pts = np.array([[0, 0, 0], [1, 1, 1], [0.25, 0.5, 0.75], [0.5, 0, 0], [0, 0, 1.0 / 1024.0]], np.float32)
    code = OR.morton_codes(pts)
    assert code[0] == 0
    assert code[1] == (1 << 30) - 1  # the top corner clamps to cell 1023 on every axis
    assert code[2] == 2**24 + 2**28 + 2**26 + 2**29 == 889192448
    assert code[3] == 2**27  # x cell 512 = bit 9 -> code bit 27
    assert code[4] == 4  # z cell 1 -> code bit 2


def test_cube_corners_in_z_order():
    corners = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
    rng = np.random.Generator(np.random.PCG64(3))
    shuffled = rng.permutation(8)
    pts = np.array([corners[i] for i in shuffled], np.float32) * 5.0 - 2.0
    perm = OR.spatial_order(pts)
    assert [tuple(int(v) for v in (pts[p] + 2.0) / 5.0) for p in perm] == corners


def test_ties_keep_gid_order_and_degenerate_extent():
    pts = np.array([[1, 2, 3], [0, 0, 0], [1, 2, 3], [0, 0, 0], [1, 2, 3]], np.float32)
    assert list(OR.spatial_order(pts)) == [1, 3, 0, 2, 4]
    same = np.full((6, 3), 0.7, np.float32)
    assert list(OR.spatial_order(same)) == list(range(6))
    assert OR.spatial_order(np.zeros((0, 3), np.float32)).shape == (0,)


def test_z_order_locality():
    # consecutive Gaussians in Z-order are spatial neighbours: on a uniform
    # cloud the mean step is a small multiple of the mean spacing n^(-1/3),
    # far below the ~0.66 of two random points in the unit cube
    rng = np.random.Generator(np.random.PCG64(4))
    pts = rng.random((20_000, 3)).astype(np.float32)
    step_z = np.linalg.norm(np.diff(pts[OR.spatial_order(pts)], axis=0), axis=1).mean()
    step_r = np.linalg.norm(np.diff(pts, axis=0), axis=1).mean()
    assert step_r > 0.6
    assert step_z < 4.0 * 20_000 ** (-1.0 / 3.0)


def test_permuted_scene_gives_the_same_image():
    sc = scenes.tiny_scene(6000, 11)
    cam = scenes.tiny_camera()
    perm = OR.spatial_order(sc.means)
    assert sorted(perm.tolist()) == list(range(sc.n))
    psc = OR.permute_scene(sc, perm)
    np.testing.assert_array_equal(psc.means, sc.means[perm])
    np.testing.assert_array_equal(psc.sh, sc.sh[perm])
    _, _, _, (rgb0, alpha0, last0) = O.render(sc, cam, bg=(0.2, 0.1, 0.0))
    _, _, _, (rgb1, alpha1, last1) = O.render(psc, cam, bg=(0.2, 0.1, 0.0))
    # no two visible Gaussians share a depth in this scene, so the (depth, gid)
    # order is the same list of Gaussians and the image is bit-identical
    np.testing.assert_array_equal(rgb1.view(np.uint32), rgb0.view(np.uint32))
    np.testing.assert_array_equal(alpha1.view(np.uint32), alpha0.view(np.uint32))
    hit = last0 >= 0
    np.testing.assert_array_equal(np.where(hit, perm[np.maximum(last1, 0)], -1), last0)
