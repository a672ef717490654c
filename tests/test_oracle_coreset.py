"""Pins of the oracle's coreset (Section 3.1) and its epoch shuffle.  CPU only.

- The coreset of a one-voxel feature is the 3x3x3 cube of its 26-neighbourhood at that key frame
  (clipped at the border), listed in (z, y, x) order with the volume's values; frames without a
  feature contribute nothing; the union over key frames concatenates them.
- Coordinates are FBB-normalised: the FBB corners map to 0 and 1 exactly, and lo + u (S - 1) gives
  back the voxel.
- The shuffle is a bijection of [0, N) for sizes around powers of two (brute force), the Feistel
  network alone is a bijection of its whole 2^k domain, epochs and seeds give different orders, and
  the batches of an epoch cover the coreset exactly once.  Over many epochs every position is
  equally likely for a given sample (chi-square against uniform).
"""
import numpy as np
import pytest

from oracle import coreset


def _vol(shape):
    return np.arange(np.prod(shape), dtype=np.float32).reshape(shape) * 0.5


def test_single_voxel_feature_gives_its_neighbourhood_cube():
    shape = (3, 10, 10, 10)  # T, Z, Y, X
    m = np.zeros(shape, np.uint8)
    m[1, 7, 6, 5] = 1
    v = _vol(shape)
    ents, labels, lo, size = coreset.build(m, v, [0, 1, 2])
    assert lo == [4, 5, 6] and size == [3, 3, 3]
    assert ents.shape == (27, 4)
    want = [(x, y, z, 1) for z in (6, 7, 8) for y in (5, 6, 7) for x in (4, 5, 6)]  # (z, y, x) order
    assert [tuple(e) for e in ents] == want
    assert np.array_equal(labels, np.array([v[1, z, y, x] for x, y, z, _ in want], np.float32))
    # frames without a feature add nothing
    e0, l0, _, _ = coreset.build(m, v, [0])
    assert e0.shape == (0, 4) and l0.shape == (0,)


def test_border_clipping_and_union_over_key_frames():
    shape = (4, 6, 6, 6)
    m = np.zeros(shape, np.uint8)
    m[0, 0, 0, 0] = 1        # corner: 2 x 2 x 2 after clipping
    m[3, 2, 3, 5] = 1        # on the x = 5 face: 2 x 3 x 3
    v = _vol(shape)
    ents, labels, lo, size = coreset.build(m, v, [0, 3])
    assert ents.shape[0] == 8 + 18
    assert (ents[:8, 3] == 0).all() and (ents[8:, 3] == 3).all()
    assert lo == [0, 0, 0] and size == [6, 5, 4]
    assert np.array_equal(labels, v[ents[:, 3], ents[:, 2], ents[:, 1], ents[:, 0]])


def test_coordinates_are_fbb_normalised():
    lo, size, nt = [3, 4, 5], [10, 1, 7], 9
    ents = np.array([[3, 4, 5, 0], [12, 4, 11, 8], [7, 4, 8, 4]], np.int64)
    u = coreset.coords_of(ents, lo, size, nt)
    assert u.dtype == np.float32
    assert np.array_equal(u[0], [0, 0, 0, 0]) and np.array_equal(u[1], [1, 0, 1, 1])
    back = np.array(lo, np.float64) + u[2, :3].astype(np.float64) * (np.array(size) - 1)
    assert np.allclose(back, [7, 4, 8], atol=1e-5) and abs(u[2, 3] * (nt - 1) - 4) < 1e-6


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 17, 255, 256, 257, 1000, 4097, 65537])
def test_shuffle_is_a_bijection(N):
    for seed, epoch in ((0, 0), (7, 3)):
        p = coreset.permute(seed, epoch, N, np.arange(N))
        assert np.array_equal(np.sort(p), np.arange(N))


def test_feistel_network_alone_is_a_bijection_of_its_domain():
    for k in (2, 4, 10):
        N = 1 << k  # no cycle walking needed
        p = coreset.permute(3, 1, N, np.arange(N))
        assert np.array_equal(np.sort(p), np.arange(N))


def test_epochs_and_seeds_differ_and_batches_cover_once():
    N = 1000
    a = coreset.permute(1, 0, N, np.arange(N))
    b = coreset.permute(1, 1, N, np.arange(N))
    c = coreset.permute(2, 0, N, np.arange(N))
    assert not np.array_equal(a, b) and not np.array_equal(a, c) and not np.array_equal(a, np.arange(N))
    ents = np.stack([np.arange(N), np.zeros(N), np.zeros(N), np.zeros(N)], 1).astype(np.int64)
    labels = np.arange(N, dtype=np.float32)
    seen = []
    for bi in range((N + 127) // 128):
        _, lab = coreset.batch(ents, labels, [0, 0, 0], [N, 1, 1], 1, 1, 0, bi, 128)
        assert lab.size == min(128, N - 128 * bi)
        seen.append(lab)
    assert np.array_equal(np.sort(np.concatenate(seen)), labels)


def test_shuffle_positions_are_uniform():
    N, E = 37, 3700
    pos_of_0 = np.empty(E, np.int64)
    for e in range(E):
        p = coreset.permute(5, e, N, np.arange(N))
        pos_of_0[e] = int(np.nonzero(p == 0)[0][0])
    counts = np.bincount(pos_of_0, minlength=N)
    chi2 = float(((counts - E / N) ** 2 / (E / N)).sum())
    assert chi2 < 80.0, chi2  # 36 degrees of freedom: the 0.9999 quantile is about 75
