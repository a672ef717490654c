"""Masked compact tables (oracle; test infrastructure only).

Section 3.1 mentions a more aggressive variant of the coreset: embedding entries only where the
features are, so that the multi-resolution grids take irregular shapes and hold fewer encoding
parameters; the paper found its dictionary look-ups too slow and kept rectangular FBB grids.  This
module is the plain definition of that variant as the library builds it (FHASH_LAYOUT_MASKED).

Readings (the paper does not define which entries the irregular grids keep):
* Footprint of a dilated-feature voxel (Section 3.1's d_k), index v on a spatial axis of the Feature
  Bounding Box with S voxels: the coordinates whose nearest voxel is v, u (S - 1) in [v - 1/2, v + 1/2].
  On the time axis (T steps) the footprint of step k is t (T - 1) in [k - 1, k + 1]: a render at an
  unseen time between two steps uses the occupancy of both (Section 3.3).  In level units p = u (R - 1)
  the footprint is widened by 1/64 on each side, far more than float32 rounding of a coordinate.
* A vertex of level l is active when it is a corner of a cell that the float32 cell step of Section
  3.2.4 assigns to some point of some footprint.  Per axis these cells are
  clamp(floor(p_lo), 0, R - 2) .. clamp(floor(p_hi), 0, R - 2), so the vertices are that range extended
  by one at the top.  An axis with S == 1 maps every coordinate to its one voxel, so all of its vertices
  are active; an axis with R == 1 has vertex 0 only.
* Rows: the active vertices of a level, in Eq. 9 order, numbered consecutively from the level's base
  (the active counts of the coarser levels added up).  An inactive corner reads 0 and receives no
  gradient.  Every point of a footprint therefore sees only active corners, and there the encoding
  equals that of the rectangular table holding the same vertex values.
The widening is a rational 1/64, so every bound below is exact integer arithmetic.
"""
import numpy as np

from . import encode


def vertex_range(v, S, R):
    """Active vertex range [lo, hi] on a spatial axis for voxel index v (FBB-relative)."""
    if R == 1:
        return 0, 0
    if S == 1:
        return 0, R - 1
    den = 64 * (S - 1)
    p_lo = ((2 * v - 1) * (R - 1) * 32 - (S - 1)) // den      # floor(p - 1/64), exact
    p_hi = ((2 * v + 1) * (R - 1) * 32 + (S - 1)) // den
    c_lo = min(max(p_lo, 0), R - 2)
    c_hi = min(max(p_hi, 0), R - 2)
    return c_lo, c_hi + 1


def time_range(k, T, R):
    """Active vertex range [lo, hi] on the time axis for time step k of T."""
    if R == 1:
        return 0, 0
    if T == 1:
        return 0, R - 1
    den = 64 * (T - 1)
    p_lo = ((k - 1) * (R - 1) * 64 - (T - 1)) // den
    p_hi = ((k + 1) * (R - 1) * 64 + (T - 1)) // den
    c_lo = min(max(p_lo, 0), R - 2)
    c_hi = min(max(p_hi, 0), R - 2)
    return c_lo, c_hi + 1


def active_grid(dil_fbb, R):
    """Active vertices of one level, bool [Rt][Rz][Ry][Rx], from the dilated mask over the FBB,
    bool [T][Sz][Sy][Sx]: every occupied voxel marks the box of its per-axis vertex ranges."""
    T, Sz, Sy, Sx = dil_fbb.shape
    Rx, Ry, Rz, Rt = (int(r) for r in R)
    act = np.zeros((Rt, Rz, Ry, Rx), bool)
    for t, z, y, x in zip(*np.nonzero(dil_fbb)):
        tl, th = time_range(int(t), T, Rt)
        zl, zh = vertex_range(int(z), Sz, Rz)
        yl, yh = vertex_range(int(y), Sy, Ry)
        xl, xh = vertex_range(int(x), Sx, Rx)
        act[tl:th + 1, zl:zh + 1, yl:yh + 1, xl:xh + 1] = True
    return act


class MaskedLevel:
    """Row map of one level: Eq. 9 row -> compact row (base + rank among the active rows), or -1."""

    def __init__(self, R, active, base):
        self.R = [int(r) for r in R]
        flat = active.reshape(-1)                       # [t][z][y][x] order is Eq. 9's
        self.rank = np.full(flat.shape[0], -1, np.int64)
        self.rank[flat] = base + np.arange(int(flat.sum()), dtype=np.int64)
        self.base = int(base)
        self.count = int(flat.sum())

    def rows(self, t, x, y, z):
        return self.rank[encode.fhash(t, x, y, z, self.R)]


class MaskedLayout:
    """All levels of a masked model (coarse to fine), built from the dilated mask over the FBB."""

    def __init__(self, levels, dil_fbb):
        self.levels, acc = [], 0
        for R in levels:
            lvl = MaskedLevel(R, active_grid(dil_fbb, R), acc)
            self.levels.append(lvl)
            acc += lvl.count
        self.rows_total = acc
        self.bases = [lvl.base for lvl in self.levels]

    def level(self, l):
        return self.levels[l]


def fbb_mask(dilated, lo, size):
    """The dilated mask restricted to the Feature Bounding Box, [T][Sz][Sy][Sx]."""
    return np.asarray(dilated, bool)[:, lo[2]:lo[2] + size[2], lo[1]:lo[1] + size[1], lo[0]:lo[0] + size[0]]


def footprint_points(dil_fbb, n, seed, edge=False):
    """n random FBB-normalised float32 points [n][4], each in the footprint of a random occupied voxel;
    with edge=True the points sit at the footprint's faces (at most 1/200 of a voxel inside)."""
    rs = np.random.default_rng(seed)
    T, Sz, Sy, Sx = dil_fbb.shape
    occ = np.stack(np.nonzero(dil_fbb), 1)              # (t, z, y, x)
    pick = occ[rs.integers(0, occ.shape[0], n)]
    if edge:
        off = rs.choice([-0.495, 0.495], size=(n, 3))
        offt = rs.choice([-0.995, 0.995], size=n)
    else:
        off = rs.uniform(-0.5, 0.5, (n, 3))
        offt = rs.uniform(-1.0, 1.0, n)
    out = np.empty((n, 4), np.float64)
    for a, (col, S) in enumerate(((3, Sx), (2, Sy), (1, Sz))):
        out[:, a] = (pick[:, col] + off[:, a]) / max(S - 1, 1) if S > 1 else 0.0
    out[:, 3] = (pick[:, 0] + offt) / max(T - 1, 1) if T > 1 else 0.0
    return np.clip(out, 0.0, 1.0).astype(np.float32)
