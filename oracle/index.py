"""Feature dilation, bounding boxes and occupancy (Section 3.1; oracle, test infrastructure only).

Masks are numpy arrays [T][Z][Y][X] (x fastest), truthy where a vertex belongs to the
extracted feature f_k of key frame k.
"""
import numpy as np


def dilate(mask):
    """Feature dilation (Section 3.1): d_k = f_k plus every vertex whose 26-neighbourhood
    (Chebyshev radius 1, spatial only, same time step) touches f_k, clipped at the volume border.
    Written as the OR of the 27 shifted copies of the mask."""
    m = np.asarray(mask).astype(bool)
    T, Z, Y, X = m.shape
    p = np.zeros((T, Z + 2, Y + 2, X + 2), bool)
    p[:, 1:-1, 1:-1, 1:-1] = m
    out = np.zeros_like(m)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                out |= p[:, 1 + dz:1 + dz + Z, 1 + dy:1 + dy + Y, 1 + dx:1 + dx + X]
    return out


def merge_features(masks):
    """Several features in one model: Section 3.1 merges the occupancy grids of several features for
    rendering.  Each feature mask is dilated on its own (as above) and the dilated regions are OR-ed;
    the Feature Bounding Box and the occupancy grid are then those of the union."""
    out = None
    for m in masks:
        d = dilate(m)
        out = d if out is None else (out | d)
    return out


def frame_boxes(d):
    """Bounding box b_k of each frame's dilated feature (Section 3.1): inclusive [lo, hi] in
    (x, y, z) order, or None for an empty frame."""
    boxes = []
    for k in range(d.shape[0]):
        idx = np.nonzero(d[k])
        if len(idx[0]) == 0:
            boxes.append(None)
            continue
        z, y, x = idx
        boxes.append(((int(x.min()), int(y.min()), int(z.min())), (int(x.max()), int(y.max()), int(z.max()))))
    return boxes


def fbb(d):
    """Temporal fusion (Section 3.1): the Feature Bounding Box is the smallest box containing every
    b_k.  Returns (lo[3], size[3]) in (x, y, z) order with size = hi - lo + 1 (vertex counts)."""
    boxes = [b for b in frame_boxes(d) if b is not None]
    if not boxes:
        raise ValueError("empty feature mask")
    lo = [min(b[0][a] for b in boxes) for a in range(3)]
    hi = [max(b[1][a] for b in boxes) for a in range(3)]
    return lo, [hi[a] - lo[a] + 1 for a in range(3)]


def occupancy(d, lo, size):
    """Occupancy grid (Section 3.1): one bit per voxel, set where the dilated feature d_k covers
    it; kept over the FBB only (it is empty outside).  Returns bool [T][Sz][Sy][Sx]."""
    return d[:, lo[2]:lo[2] + size[2], lo[1]:lo[1] + size[1], lo[0]:lo[0] + size[0]].copy()
