"""Pins of the oracle renderer (Section 3.3, Algorithm 1) against closed forms.  CPU only.

A model returning a constant value through a transfer function of constant opacity alpha makes every
sample identical, so along a ray of n occupied samples the pixel opacity is 1 - (1-alpha)^n and the
colour is rgb * (1 - (1-alpha)^n), with n cut at the first sample that pushes the opacity above 0.99.
An axis-aligned ray through the box centre with spacing a power of two has exactly computable sample
positions, which pins the sample count and the nearest-voxel occupancy test.
"""
import math

import numpy as np

from oracle import render


def _const_model(v):
    return lambda u: np.full(u.shape[0], v, np.float64)


def _tf_const(alpha, rgb=(0.2, 0.4, 0.6)):
    tf = np.zeros((256, 4), np.float32)
    tf[:, :3] = rgb
    tf[:, 3] = alpha
    return tf


AXIS_CAM = (np.array([2, 0, 0], np.float32), np.array([0, 0.5, 0], np.float32), np.array([0, 0, 0.5], np.float32),
            np.array([-1, 0, 0], np.float32))


def test_axis_ray_sample_count_and_opacity():
    S = [9, 9, 9]  # spacing 1/8 world units
    occ = np.ones((1, 9, 9, 9), bool)
    # 1x1 image: the pixel centre looks exactly along -x, enters at x=1 (t=1), leaves at x=-1 (t=3)
    img, cnt = render.render(_const_model(0.5), AXIS_CAM, 1, 1, S, occ, 0.0, _tf_const(0.2))
    n = 17  # t = 1 + k/8 <= 3
    a = float(np.float32(0.2))  # the table stores float32
    rgb = np.array([0.2, 0.4, 0.6], np.float32).astype(np.float64)
    assert cnt[0, 0] == n
    assert abs(img[0, 0, 3] - (1 - (1 - a) ** n)) < 1e-12
    assert np.allclose(img[0, 0, :3], rgb * (1 - (1 - a) ** n), atol=1e-12)


def test_early_termination_count():
    S = [9, 9, 9]
    occ = np.ones((1, 9, 9, 9), bool)
    img, cnt = render.render(_const_model(0.5), AXIS_CAM, 1, 1, S, occ, 0.0, _tf_const(0.5))
    n = math.ceil(math.log(0.01) / math.log(0.5) + 1e-12)  # first n with 1 - 0.5^n > 0.99 -> 7
    assert n == 7 and cnt[0, 0] == n
    assert abs(img[0, 0, 3] - (1 - 0.5 ** 7)) < 1e-12


def test_nearest_voxel_occupancy():
    # Only the centre voxel (4,4,4) is occupied.  Sample k sits at x = 1 - k/8, voxel coordinate
    # q = 8 - k/2, nearest voxel floor(q + 0.5) = 4 for k = 8 and 9 only.
    S = [9, 9, 9]
    occ = np.zeros((1, 9, 9, 9), bool)
    occ[0, 4, 4, 4] = True
    r, u = render.ray_samples(AXIS_CAM, 1, 1, S, occ, 0.0)
    assert r.tolist() == [0, 0]
    assert np.allclose(u[:, 0], [0.5, 0.4375])  # u = (x + 1)/2 at x = 0 (k = 8) and x = -1/8 (k = 9)


def test_empty_occupancy_is_black_and_misses_are_zero():
    S = [9, 9, 9]
    img, cnt = render.render(_const_model(0.5), AXIS_CAM, 8, 6, S, np.zeros((1, 9, 9, 9), bool), 0.0, _tf_const(0.3))
    assert (img == 0).all() and (cnt == 0).all()
    away = (np.array([0, 0, 3], np.float32), np.array([0.1, 0, 0], np.float32), np.array([0, 0.1, 0], np.float32),
            np.array([0, 0, 1], np.float32))  # looking away from the box
    img, cnt = render.render(_const_model(0.5), away, 4, 4, S, np.ones((1, 9, 9, 9), bool), 0.0, _tf_const(0.3))
    assert (img == 0).all()


def test_unseen_time_uses_either_key_frame():
    S = [9, 9, 9]
    occ = np.zeros((3, 9, 9, 9), bool)
    occ[2, 4, 4, 4] = True  # only in the last key frame
    for t, n in ((0.25, 0), (0.5, 0), (0.75, 2), (1.0, 2)):
        r, _ = render.ray_samples(AXIS_CAM, 1, 1, S, occ, t)
        assert r.size == n, t


def test_transfer_function_interpolates_entries():
    tf = np.random.default_rng(0).random((256, 4)).astype(np.float32)
    v = np.arange(256) / 255.0
    assert np.allclose(render.transfer(v, tf), tf, atol=1e-12)
    mid = render.transfer(np.array([(10.5) / 255.0]), tf)[0]
    assert np.allclose(mid, 0.5 * (tf[10].astype(np.float64) + tf[11]), atol=1e-12)
    assert np.allclose(render.transfer(np.array([-3.0, 7.0]), tf), tf[[0, 255]], atol=1e-12)


def test_decode_grid_hits_vertices():
    u, shape = render.decode_coords([5, 3, 9], 2, 0.25)
    assert shape == (17, 5, 9)
    assert u[0].tolist() == [0, 0, 0, 0.25] and u[-1].tolist() == [1, 1, 1, 0.25]
    xs = np.unique(u[:, 0])
    assert np.array_equal(xs, (np.arange(9) / 8).astype(np.float32))
