"""Multi-resolution Tesseract encoding, forward and backward (oracle; test infrastructure only).

Section 3.2.4 gives four steps per level: (1) locate the neighbouring time steps
t_Previous / t_Next, (2) locate the embedding cell containing (x, y, z), (3) map the 8
corners of that cell at both time steps to table rows through the F-Hash of Eq. 9 (16
look-ups), (4) interpolate trilinearly in space (Eqs. 10-11) and then linearly in time
(Eq. 12).  The per-level results are concatenated (coarse level first) as the MLP input.

Readings taken where the paper is silent or garbled:
* Resolutions count VERTICES: level grid vertex j of an axis with R vertices sits at
  normalised coordinate j/(R-1) of [0, 1] (the paper's [-1, 1] cube, shifted and halved).
  Inputs are FBB-normalised u in [0,1]^4 in (x, y, z, t) order.
* Cell location in float32, because it decides integer rows and the GPU takes the same
  decision in float32: u <- min(max(u, 0), 1) (NaN -> 0), p = u*(R-1) rounded to nearest,
  c = clamp(floor(p), 0, R-2), w = p - c (exact), upper corner min(c+1, R-1).  An axis with
  R == 1 has c = 0, w = 0 and both corners on vertex 0.
* Eq. 12 is garbled in the source; the reading is V = (1-w_t) V^Previous + w_t V^Next.
Everything after the float32 cell step is float64.

Corner order used for row/weight arrays: c = i + 2j + 4k + 8s with i, j, k the upper/lower
corner on x, y, z and s = 0 for t_Previous, 1 for t_Next.

`layout` is "linear" (Eq. 9), "brick", or a masked layout (oracle/masked.py: rows only for the
vertices near the features; an inactive corner has row -1, reads 0 and takes no gradient).
"""
import numpy as np


def locate(u, R):
    """Steps 1-2 on one axis: float32 cell index c, upper corner c1 and fraction w."""
    u = np.asarray(u, np.float32)
    u = np.fmin(np.fmax(u, np.float32(0.0)), np.float32(1.0))   # fmax(NaN, 0) = 0
    p = u * np.float32(R - 1)                                    # float32 multiply, round to nearest
    c = np.floor(p).astype(np.int64)
    c = np.maximum(np.minimum(c, R - 2), 0)
    w = (p - c.astype(np.float32)).astype(np.float32)            # exact
    c1 = np.minimum(c + 1, R - 1)
    return c, c1, w


def fhash(t, x, y, z, R, layout="linear"):
    """Row of vertex (t, x, y, z) within level l.

    "linear" is Eq. 9: F-Hash^l(t, x, y, z) = t*Rx*Ry*Rz + z*Rx*Ry + y*Rx + x.
    "brick" is the locality-preserving linearisation that Section 3.2.3 allows: each time slice is cut
    into 4x4x4 spatial bricks (narrower at the high end of an axis when R is not a multiple of 4),
    bricks in (bz, by, bx) order and vertices inside a brick in (iz, iy, ix) order.  With b = v // 4,
    i = v % 4 and w(b) = min(4, R - 4b) per axis, the row is
        t*Rx*Ry*Rz + 4 bz Rx Ry + wz 4 by Rx + wz wy 4 bx + (iz wy + iy) wx + ix,
    a bijection onto [0, Rx*Ry*Rz*Rt) like Eq. 9 (no bucket is wasted)."""
    Rx, Ry, Rz = (np.int64(R[0]), np.int64(R[1]), np.int64(R[2]))
    if layout == "linear":
        return t * (Rx * Ry * Rz) + z * (Rx * Ry) + y * Rx + x
    x, y, z, t = (np.asarray(a, np.int64) for a in (x, y, z, t))
    bx, by, bz = x // 4, y // 4, z // 4
    ix, iy, iz = x % 4, y % 4, z % 4
    wx, wy, wz = np.minimum(4, Rx - 4 * bx), np.minimum(4, Ry - 4 * by), np.minimum(4, Rz - 4 * bz)
    return (t * (Rx * Ry * Rz) + 4 * bz * Rx * Ry + wz * 4 * by * Rx + wz * wy * 4 * bx
            + (iz * wy + iy) * wx + ix)


def _level_layout(layout, l):
    return layout if isinstance(layout, str) else layout.level(l)


def _rows(t, x, y, z, R, base, layout):
    """Concatenated-table rows of vertices (t, x, y, z) of one level; -1 for an inactive vertex of a
    masked level."""
    if isinstance(layout, str):
        return base + fhash(t, x, y, z, R, layout)
    return layout.rows(t, x, y, z)


def level_corners(coords, R, base, layout="linear"):
    """Rows [N][16] (int64, concatenated-table rows; -1 = inactive corner of a masked level) and
    float64 weights [N][16] of one level.  `layout` is a string or one level of a masked layout."""
    coords = np.asarray(coords, np.float32)
    cx, cx1, wx = locate(coords[:, 0], R[0])
    cy, cy1, wy = locate(coords[:, 1], R[1])
    cz, cz1, wz = locate(coords[:, 2], R[2])
    tp, tn, wt = locate(coords[:, 3], R[3])
    wx, wy, wz, wt = (a.astype(np.float64) for a in (wx, wy, wz, wt))
    N = coords.shape[0]
    rows = np.empty((N, 16), np.int64)
    wts = np.empty((N, 16), np.float64)
    for s, (tt, ws) in enumerate(((tp, 1.0 - wt), (tn, wt))):
        for k, (zz, wk) in enumerate(((cz, 1.0 - wz), (cz1, wz))):
            for j, (yy, wj) in enumerate(((cy, 1.0 - wy), (cy1, wy))):
                for i, (xx, wi) in enumerate(((cx, 1.0 - wx), (cx1, wx))):
                    c = i + 2 * j + 4 * k + 8 * s
                    rows[:, c] = _rows(tt, xx, yy, zz, R, base, layout)
                    wts[:, c] = ws * wk * wj * wi
    return rows, wts


def interpolate_level(coords, R, base, table, layout="linear"):
    """Steps 3-4 for one level: Eqs. 10-11 (trilinear at t_Previous and t_Next), then Eq. 12."""
    coords = np.asarray(coords, np.float32)
    cx, cx1, wx = locate(coords[:, 0], R[0])
    cy, cy1, wy = locate(coords[:, 1], R[1])
    cz, cz1, wz = locate(coords[:, 2], R[2])
    tp, tn, wt = locate(coords[:, 3], R[3])
    x, y, z, t = (a.astype(np.float64)[:, None] for a in (wx, wy, wz, wt))

    def V(tt):
        acc = 0.0
        for i, xx in ((0, cx), (1, cx1)):
            for j, yy in ((0, cy), (1, cy1)):
                for k, zz in ((0, cz), (1, cz1)):
                    r = _rows(tt, xx, yy, zz, R, base, layout)
                    Vijk = np.asarray(table[np.maximum(r, 0)], np.float64)
                    Vijk = np.where((r >= 0)[:, None], Vijk, 0.0)        # inactive corner reads 0
                    acc = acc + Vijk * (x ** i * (1 - x) ** (1 - i)) * (y ** j * (1 - y) ** (1 - j)) \
                        * (z ** k * (1 - z) ** (1 - k))
        return acc

    return (1.0 - t) * V(tp) + t * V(tn)


def encode(levels, level_bases, coords, table, layout="linear"):
    """Concatenated encoding [N][L*F] float64; `table` is indexable by int64 row arrays and
    returns [n][F] values (a dense [rows][F] array, or any lazy equivalent)."""
    parts = [interpolate_level(coords, R, b, table, _level_layout(layout, l))
             for l, (R, b) in enumerate(zip(levels, level_bases))]
    return np.concatenate(parts, axis=1)


def encode_backward(levels, level_bases, coords, d_enc, F, layout="linear"):
    """Gradient of sum(d_enc * enc) with respect to the table: each of the 16 corner rows of every
    level receives weight * d_enc of that level (Eqs. 10-12 are linear in the table).
    Returns (unique rows int64, gradient [n_rows][F] float64)."""
    all_rows, all_vals = [], []
    for l, (R, b) in enumerate(zip(levels, level_bases)):
        rows, wts = level_corners(coords, R, b, _level_layout(layout, l))
        g = np.asarray(d_enc, np.float64)[:, l * F:(l + 1) * F]
        all_rows.append(rows.reshape(-1))
        all_vals.append((wts[:, :, None] * g[:, None, :]).reshape(-1, F))
    rows = np.concatenate(all_rows)
    vals = np.concatenate(all_vals)
    keep = rows >= 0                                     # inactive corners take no gradient
    rows, vals = rows[keep], vals[keep]
    # per-row sums of the contributions: sort by row, then sum each run of equal rows
    order = np.argsort(rows, kind="stable")
    rs = rows[order]
    starts = np.flatnonzero(np.concatenate([[True], rs[1:] != rs[:-1]]))
    uniq = rs[starts]
    grad = np.stack([np.add.reduceat(vals[order, f], starts) for f in range(F)], 1)
    return uniq, grad
