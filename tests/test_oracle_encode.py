"""Pins of the oracle's encoding (Section 3.2.4, Eqs. 9-12) against closed forms, brute force and a
library interpolator.  CPU only."""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

from oracle import encode, schedule


def _coords(rng, n):
    c = rng.random((n, 4)).astype(np.float32)
    c[:5] = [[0, 0, 0, 0], [1, 1, 1, 1], [1, 0, 1, 0], [0.5, 0.5, 0.5, 0.5], [np.nan, -3, 7, 1]]
    return c


def test_locate_definition():
    c, c1, w = encode.locate(np.array([0.0, 1.0, 0.5, np.nan, -1, 2, 0.999999], np.float32), 5)
    assert list(c) == [0, 3, 2, 0, 0, 3, 3] and list(c1) == [1, 4, 3, 1, 1, 4, 4]
    assert list(w[:6]) == [0, 1, 0, 0, 0, 1]
    c, c1, w = encode.locate(np.array([0.3, 1.0], np.float32), 1)  # single-vertex axis
    assert list(c) == [0, 0] and list(c1) == [0, 0] and list(w) == [0, 0]


def test_weights_partition_of_unity():
    rng = np.random.default_rng(1)
    co = _coords(rng, 4000)
    for R in ([4, 4, 4, 1], [7, 3, 5, 2], [33, 17, 9, 8]):
        _, w = encode.level_corners(co, R, 0)
        assert (w >= 0).all()
        assert np.abs(w.sum(1) - 1.0).max() <= 4 * np.finfo(np.float64).eps


def test_vertex_reproduction():
    # At a vertex the encoding returns the stored embedding exactly (R-1 powers of two make
    # j/(R-1) exact in float32).
    rng = np.random.default_rng(2)
    levels = [[5, 9, 3, 2], [17, 5, 9, 5]]
    b, rows = schedule.bases(levels)
    F = 3
    table = rng.standard_normal((rows, F))
    for l, R in enumerate(levels):
        idx = np.stack([rng.integers(0, R[d], 500) for d in range(4)], 1)
        co = (idx / (np.array(R) - 1)).astype(np.float32)
        enc = encode.encode(levels, b, co, table)[:, l * F:(l + 1) * F]
        row = b[l] + encode.fhash(idx[:, 3], idx[:, 0], idx[:, 1], idx[:, 2], R)
        assert np.array_equal(enc, table[row])


def test_multilinear_field_exact():
    # Any field multilinear in (x, y, z, t) written into a level's table is reproduced exactly at
    # the float32 cell position c + w (the interpolant of Eqs. 10-12 is exact on that space).
    rng = np.random.default_rng(3)
    R = [6, 5, 7, 4]
    coef = rng.standard_normal(16)

    def f(x, y, z, t):
        out = 0.0
        for m in range(16):
            out = out + coef[m] * (x if m & 1 else 1) * (y if m & 2 else 1) * (z if m & 4 else 1) * (t if m & 8 else 1)
        return out

    t, z, y, x = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in (R[3], R[2], R[1], R[0])], indexing="ij")
    table = np.zeros((np.prod(R), 1))
    table[encode.fhash(t.astype(int).ravel(), x.astype(int).ravel(), y.astype(int).ravel(),
                       z.astype(int).ravel(), R), 0] = f(x, y, z, t).ravel()
    co = _coords(rng, 3000)
    enc = encode.encode([R], [0], co, table)[:, 0]
    pos = []
    for d in range(4):
        c, _, w = encode.locate(co[:, d], R[d])
        pos.append(c + w.astype(np.float64))
    assert np.abs(enc - f(*pos)).max() <= 1e-12 * max(1.0, np.abs(enc).max())


def test_matches_library_quadrilinear():
    # Single level, F=1: the encoding equals scipy's linear RegularGridInterpolator on the vertex
    # grid, queried at the float32 cell positions.
    rng = np.random.default_rng(4)
    R = [5, 4, 6, 3]
    vals = rng.standard_normal((R[3], R[2], R[1], R[0]))
    table = np.zeros((np.prod(R), 1))
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (R[3], R[2], R[1], R[0])], indexing="ij")
    table[encode.fhash(t.ravel(), x.ravel(), y.ravel(), z.ravel(), R), 0] = vals.ravel()
    co = _coords(rng, 2000)
    pos = []
    for d in range(4):
        c, _, w = encode.locate(co[:, d], R[d])
        pos.append((c + w.astype(np.float64)) / (R[d] - 1))
    axes = [np.arange(n) / (n - 1) for n in (R[3], R[2], R[1], R[0])]
    ref = RegularGridInterpolator(axes, vals)(np.stack([pos[3], pos[2], pos[1], pos[0]], 1))
    enc = encode.encode([R], [0], co, table)[:, 0]
    assert np.abs(enc - ref).max() <= 1e-12


def test_time_spans_nest():
    # The nesting of neighbouring time steps across levels shown in Figure 6 holds for vertex-aligned
    # temporal grids with Rt = 2^k + 1.
    t = np.random.default_rng(5).random(5000).astype(np.float32)
    spans = []
    for Rt in (9, 5, 3, 2):
        c, c1, _ = encode.locate(t, Rt)
        spans.append((c / (Rt - 1), c1 / (Rt - 1)))
    for (a0, a1), (b0, b1) in zip(spans[:-1], spans[1:]):
        assert (b0 <= a0).all() and (a1 <= b1).all()


def test_backward_is_transpose_of_forward():
    # <d_enc, J table> = <J^T d_enc, table> for random table and d_enc (the scatter is the exact
    # adjoint of the gather), and the scatter of a one-hot d_enc row equals that sample's weights.
    rng = np.random.default_rng(6)
    levels = [[3, 3, 3, 2], [5, 4, 3, 3]]
    b, rows = schedule.bases(levels)
    F = 2
    co = _coords(rng, 300)
    table = rng.standard_normal((rows, F))
    d = rng.standard_normal((300, len(levels) * F))
    lhs = np.sum(d * encode.encode(levels, b, co, table))
    r, g = encode.encode_backward(levels, b, co, d, F)
    rhs = np.sum(g * table[r])
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


@pytest.mark.parametrize("R", [(5, 6, 7, 3), (4, 4, 4, 2), (9, 1, 2, 1), (8, 12, 3, 2)])
def test_brick_rows_are_the_rank_of_the_brick_order(R):
    """The brick linearisation (Section 3.2.3 allows locality-preserving orders): every vertex's row is
    its rank in lexicographic (t, bz, by, bx, iz, iy, ix) order, brute force over all vertices, partial
    bricks included; so it is a bijection onto [0, Rx*Ry*Rz*Rt) like Eq. 9."""
    Rx, Ry, Rz, Rt = R
    t, z, y, x = (a.ravel() for a in np.meshgrid(np.arange(Rt), np.arange(Rz), np.arange(Ry), np.arange(Rx),
                                                 indexing="ij"))
    rows = encode.fhash(t, x, y, z, R, "brick")
    key = np.lexsort((x % 4, y % 4, z % 4, x // 4, y // 4, z // 4, t))  # last key is primary
    rank = np.empty_like(key)
    rank[key] = np.arange(key.size)
    assert np.array_equal(rows, rank)
    assert np.array_equal(np.sort(rows), np.arange(Rx * Ry * Rz * Rt))


def test_brick_layout_is_a_relabelling_of_eq9():
    """With the same vertex values stored at each layout's rows, both layouts give the same encoding
    and the same gradient per vertex: only where a vertex lives changes."""
    levels = [[3, 4, 5, 2], [6, 7, 9, 3]]
    bases, total = schedule.bases(levels)
    F = 2
    rng = np.random.default_rng(3)
    t_lin = rng.standard_normal((total, F))
    t_brk = np.empty_like(t_lin)
    for R, b in zip(levels, bases):
        Rx, Ry, Rz, Rt = R
        t, z, y, x = (a.ravel() for a in np.meshgrid(*[np.arange(k) for k in (Rt, Rz, Ry, Rx)], indexing="ij"))
        t_brk[b + encode.fhash(t, x, y, z, R, "brick")] = t_lin[b + encode.fhash(t, x, y, z, R)]
    c = rng.random((500, 4)).astype(np.float32)
    assert np.allclose(encode.encode(levels, bases, c, t_lin), encode.encode(levels, bases, c, t_brk, "brick"),
                       rtol=0, atol=1e-12)
    d = rng.standard_normal((500, len(levels) * F))
    r1, g1 = encode.encode_backward(levels, bases, c, d, F)
    r2, g2 = encode.encode_backward(levels, bases, c, d, F, "brick")
    m = np.empty(total, np.int64)  # brick row -> linear row
    for R, b in zip(levels, bases):
        Rx, Ry, Rz, Rt = R
        t, z, y, x = (a.ravel() for a in np.meshgrid(*[np.arange(k) for k in (Rt, Rz, Ry, Rx)], indexing="ij"))
        m[b + encode.fhash(t, x, y, z, R, "brick")] = b + encode.fhash(t, x, y, z, R)
    order = np.argsort(m[r2])
    assert np.array_equal(m[r2][order], r1) and np.allclose(g2[order], g1, rtol=0, atol=1e-12)
