"""Pins of the masked compact tables in the oracle (oracle/masked.py), independent of its own formulas.

- Per-axis vertex ranges against a brute force over cells with exact fractions: a vertex is active when
  one of its cells, as the float32 cell step assigns points to cells ([c, c+1), the first cell open
  below, the last closed above), meets the widened footprint.  Exhaustive over small S, R, v and k,
  including R == 1, R == 2, S == 1 and R > S.
- Hand-worked ranges (S = 5, R = 3).
- No mask: every vertex active, compact rows equal to Eq. 9 rows.
- Compact rows are 0 .. N-1 in Eq. 9 order (a bijection from the active vertices).
- Soundness: all 16 corners of every level are active at random and face points of footprints.
- Equivalence: a masked table holding a rectangular table's vertex values encodes footprint points
  exactly like it; at any point the masked encoding equals the rectangular one with the inactive rows
  set to 0, and the gradients of the active rows agree.
- Product structure: OR-resampling the dilated mask one axis at a time gives the same active grid.
"""
from fractions import Fraction

import numpy as np

from oracle import encode, index, masked, schedule

LEVELS = [[2, 3, 2, 1], [3, 5, 4, 2], [7, 6, 9, 3], [13, 11, 10, 5]]


def _brute_range(lo, hi, R):
    """Vertices of the cells (as the cell step assigns points) that meet [lo, hi] (exact fractions)."""
    if R == 1:
        return {0}
    out = set()
    for c in range(R - 1):
        a = Fraction(-10 ** 9) if c == 0 else Fraction(c)           # first cell: everything below 1
        b = Fraction(10 ** 9) if c == R - 2 else Fraction(c + 1)    # last cell: everything from R-2
        closed_hi = c == R - 2
        meets = lo <= b and hi >= a if closed_hi else lo < b and hi >= a
        if meets:
            out |= {c, c + 1}
    return out


def test_vertex_ranges_against_exact_cells():
    m = Fraction(1, 64)
    for S in range(1, 12):
        for R in range(1, 15):
            for v in range(S):
                if S == 1:
                    want = set(range(R))
                else:
                    lo = Fraction(2 * v - 1, 2) * Fraction(R - 1, S - 1) - m
                    hi = Fraction(2 * v + 1, 2) * Fraction(R - 1, S - 1) + m
                    want = _brute_range(lo, hi, R)
                a, b = masked.vertex_range(v, S, R)
                assert set(range(a, b + 1)) == want, (S, R, v)
    for T in range(1, 10):
        for R in range(1, 12):
            for k in range(T):
                if T == 1:
                    want = set(range(R))
                else:
                    lo = Fraction(k - 1) * Fraction(R - 1, T - 1) - m
                    hi = Fraction(k + 1) * Fraction(R - 1, T - 1) + m
                    want = _brute_range(lo, hi, R)
                a, b = masked.time_range(k, T, R)
                assert set(range(a, b + 1)) == want, (T, R, k)


def test_hand_worked_ranges():
    # S = 5 voxels, R = 3 vertices: p = u * 2 and u = q / 4, so voxel v covers p in [(v - 1/2)/2, (v + 1/2)/2].
    # v = 0: p in [-1/4, 1/4] -> cell 0 -> vertices 0..1.  v = 2: p in [3/4, 5/4] -> cells 0, 1 -> 0..2.
    # v = 4: p in [7/4, 9/4] -> cell 1 (the last) -> vertices 1..2.
    assert masked.vertex_range(0, 5, 3) == (0, 1)
    assert masked.vertex_range(2, 5, 3) == (0, 2)
    assert masked.vertex_range(4, 5, 3) == (1, 2)
    # time: T = 5 steps, R = 3: step k covers p in [(k - 1)/2, (k + 1)/2]; k = 0 -> [-1/2, 1/2] -> cell 0.
    assert masked.time_range(0, 5, 3) == (0, 1)
    assert masked.time_range(2, 5, 3) == (0, 2)
    # the finest level on the data grid (R = S): voxel v touches cells v - 1 and v
    assert masked.vertex_range(3, 8, 8) == (2, 4)


def _small_mask(seed=3):
    rs = np.random.default_rng(seed)
    m = np.zeros((5, 11, 10, 13), np.uint8)                # [T][Z][Y][X]
    m[1, 3:5, 4:6, 2:4] = 1
    m[3, 6, 2, 8:10] = 1
    m[4, rs.integers(0, 11), rs.integers(0, 10), rs.integers(0, 13)] = 1
    d = index.dilate(m)
    lo, size = index.fbb(d)
    return masked.fbb_mask(d, lo, size)


def test_no_mask_is_eq9():
    dil = np.ones((5, 7, 6, 9), bool)
    lay = masked.MaskedLayout(LEVELS, dil)
    b, total = schedule.bases(LEVELS)
    assert lay.bases == b and lay.rows_total == total
    for l, R in enumerate(LEVELS):
        assert np.array_equal(lay.level(l).rank, b[l] + np.arange(schedule.level_rows(R)))


def test_compact_rows_are_a_bijection_in_eq9_order():
    lay = masked.MaskedLayout(LEVELS, _small_mask())
    seen = []
    for l in range(len(LEVELS)):
        r = lay.level(l).rank
        act = r[r >= 0]
        assert np.all(np.diff(act) == 1)                    # increasing in Eq. 9 order, no gaps
        seen.append(act)
    allr = np.concatenate(seen)
    assert np.array_equal(allr, np.arange(lay.rows_total))
    dense = schedule.bases(LEVELS)[1]
    assert 0 < lay.rows_total < dense                       # the point of the variant


def test_footprint_corners_are_active():
    dil = _small_mask()
    lay = masked.MaskedLayout(LEVELS, dil)
    for edge in (False, True):
        pts = masked.footprint_points(dil, 4000, 5 + edge, edge=edge)
        for l, R in enumerate(LEVELS):
            rows, _ = encode.level_corners(pts, R, lay.bases[l], lay.level(l))
            assert (rows >= 0).all(), (l, edge)


def test_equivalence_with_the_rectangular_table():
    dil = _small_mask()
    lay = masked.MaskedLayout(LEVELS, dil)
    b, total = schedule.bases(LEVELS)
    F = 2
    rs = np.random.default_rng(11)
    T_lin = rs.uniform(-1, 1, (total, F))
    T_m = np.zeros((lay.rows_total, F))
    T_zero = np.zeros_like(T_lin)                          # rectangular table, inactive rows 0
    for l in range(len(LEVELS)):
        r = lay.level(l).rank
        idx = np.flatnonzero(r >= 0)
        T_m[r[idx]] = T_lin[b[l] + idx]
        T_zero[b[l] + idx] = T_lin[b[l] + idx]
    pts = masked.footprint_points(dil, 3000, 9)
    assert np.array_equal(encode.encode(LEVELS, lay.bases, pts, T_m, lay), encode.encode(LEVELS, b, pts, T_lin))
    anyp = rs.uniform(0, 1, (3000, 4)).astype(np.float32)
    e_m = encode.encode(LEVELS, lay.bases, anyp, T_m, lay)
    assert np.array_equal(e_m, encode.encode(LEVELS, b, anyp, T_zero))
    assert (encode.encode(LEVELS, lay.bases, anyp, np.ones_like(T_m), lay) < 1 - 1e-12).any()  # some inactive
    d_enc = rs.normal(size=(3000, len(LEVELS) * F))
    rm, gm = encode.encode_backward(LEVELS, lay.bases, anyp, d_enc, F, lay)
    rl, gl = encode.encode_backward(LEVELS, b, anyp, d_enc, F)
    full = np.zeros_like(T_lin)
    full[rl] = gl
    want = np.zeros_like(T_m)
    for l in range(len(LEVELS)):
        r = lay.level(l).rank
        idx = np.flatnonzero(r >= 0)
        want[r[idx]] = full[b[l] + idx]
    got = np.zeros_like(T_m)
    got[rm] = gm
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


def test_active_grid_is_separable():
    """The definition marks, for every occupied voxel, the product of its per-axis vertex ranges.  The
    same grid comes out of OR-resampling the dilated mask one axis at a time, each vertex taking the OR
    over the voxels whose range holds it (the form a parallel build can use): a product structure the
    definition must have."""
    dil = _small_mask(8)
    T, Sz, Sy, Sx = dil.shape

    def resample(a, axis, S, R, time):
        rng = [masked.time_range(v, S, R) if time else masked.vertex_range(v, S, R) for v in range(S)]
        out_shape = list(a.shape)
        out_shape[axis] = R
        out = np.zeros(out_shape, bool)
        for X in range(R):
            vs = [v for v in range(S) if rng[v][0] <= X <= rng[v][1]]
            if vs:
                idx = [slice(None)] * a.ndim
                idx[axis] = X
                out[tuple(idx)] = np.take(a, vs, axis=axis).any(axis=axis)
        return out

    for R in LEVELS + [[40, 3, 50, 12]]:
        g = resample(dil, 3, Sx, R[0], False)
        g = resample(g, 2, Sy, R[1], False)
        g = resample(g, 1, Sz, R[2], False)
        g = resample(g, 0, T, R[3], True)
        assert np.array_equal(g, masked.active_grid(dil, R)), R
