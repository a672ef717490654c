"""Pins of the oracle's dilation, bounding boxes and RNG.  CPU only."""
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
