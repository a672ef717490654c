"""Pins of the oracle's dilation, feature merging, bounding boxes and RNG.  CPU only."""
import numpy as np
from scipy import ndimage

import synth
from oracle import index, rng


def test_dilation_vs_scipy():
    r = np.random.default_rng(0)
    m = r.random((3, 9, 11, 13)) < 0.03
    d = index.dilate(m)
    ref = np.stack([ndimage.binary_dilation(m[k], structure=np.ones((3, 3, 3), bool)) for k in range(3)])
    assert np.array_equal(d, ref)


def test_fbb_brute_force():
    r = np.random.default_rng(1)
    for _ in range(20):
        m = r.random((4, 7, 8, 9)) < 0.01
        if not m.any():
            continue
        d = index.dilate(m)
        lo, size = index.fbb(d)
        zs, ys, xs = [], [], []
        for t in range(4):
            for z in range(7):
                for y in range(8):
                    for x in range(9):
                        if d[t, z, y, x]:
                            xs.append(x); ys.append(y); zs.append(z)
        assert lo == [min(xs), min(ys), min(zs)]
        assert size == [max(xs) - min(xs) + 1, max(ys) - min(ys) + 1, max(zs) - min(zs) + 1]


def test_single_voxel_boxes():
    m = np.zeros((2, 10, 10, 10), bool)
    m[0, 5, 5, 5] = True
    assert index.fbb(index.dilate(m)) == ([4, 4, 4], [3, 3, 3])
    m[1, 0, 0, 9] = True  # clipped at the border
    assert index.fbb(index.dilate(m)) == ([4, 0, 0], [6, 7, 7])  # x 4..9, y,z 0..6


def test_merge_features_hand_built():
    # two one-voxel features in different frames: each frame's region is one clipped 3x3x3 cube, and the
    # box of the union spans both cubes
    a = np.zeros((2, 8, 8, 8), bool)
    b = np.zeros_like(a)
    a[0, 1, 1, 1] = True                  # (t, z, y, x)
    b[1, 4, 5, 6] = True
    d = index.merge_features([a, b])
    assert d[0].sum() == 27 and d[1].sum() == 27
    assert d[0, 0:3, 0:3, 0:3].all() and d[1, 3:6, 4:7, 5:8].all()
    assert index.fbb(d) == ([0, 0, 0], [8, 7, 6])          # x 0..7, y 0..6, z 0..5
    # overlapping features in one frame: cubes x 1..3 and x 2..4 over y, z 1..3 give 4 x 3 x 3 voxels
    c = np.zeros((1, 6, 6, 6), bool)
    e = np.zeros_like(c)
    c[0, 2, 2, 2] = True
    e[0, 2, 2, 3] = True
    d = index.merge_features([c, e])
    assert d.sum() == 36 and index.fbb(d) == ([1, 1, 1], [4, 3, 3])
    # a feature at the volume corner is clipped: 2 x 2 x 2 voxels
    f = np.zeros((1, 5, 5, 5), bool)
    f[0, 0, 0, 0] = True
    assert index.merge_features([f]).sum() == 8


def test_merge_features_is_dilation_of_union():
    """Dilation distributes over union, so merging the dilated features equals dilating the union of the
    masks (a different computation), and one feature is its own dilation."""
    r = np.random.default_rng(4)
    for k in (1, 2, 3, 5):
        masks = [r.random((3, 6, 7, 9)) < 0.02 for _ in range(k)]
        union = np.zeros_like(masks[0])
        for m in masks:
            union |= m
        ref = np.stack([ndimage.binary_dilation(union[t], structure=np.ones((3, 3, 3), bool)) for t in range(3)])
        assert np.array_equal(index.merge_features(masks), ref)
    assert np.array_equal(index.merge_features(masks[:1]), index.dilate(masks[0]))


def test_splitmix64_published_values():
    # First outputs of SplitMix64 seeded with 0, as published with the generator.
    assert int(rng.at(0, 0)) == 0xE220A8397B1DCDAF
    assert int(rng.at(0, 1)) == 0x6E789E6AA1B965F4
    # the input module's independent C implementation agrees
    assert synth.splitmix64_at(0, 0) == 0xE220A8397B1DCDAF


def test_init_table_matches_input_generator():
    t = rng.InitTable(5, 2)
    rows = np.array([0, 1, 7, 1000])
    ref = synth.init_tables(5, 2002).reshape(-1, 2)[rows]
    assert np.array_equal(t[rows], ref)


def test_init_mlp_matches_input_generator():
    for dims in ([8, 32, 32, 1], [32, 64, 64, 1], [64, 64, 64, 64, 1]):
        assert np.array_equal(rng.init_mlp(9, dims), synth.init_mlp(9, dims))
