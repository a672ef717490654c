"""Rendering of a trained F-Hash INR (Section 3.3, Algorithm 1) and time-slice decode (oracle; test
infrastructure only).

The paper renders by sample streaming: rays are marched through the volume, samples in occupied
space are sent to the INR with the time step concatenated, the values go through a transfer function
and are composited front to back, finished rays leave.  Adaptive ray marching (ARM) only changes HOW
MANY samples each alive ray contributes per round (the pace N_s = max(min(N_r/N_a, 64), 1)); it does
not change which samples a ray takes or their order, so the image it produces is the one written
here ray by ray.  The readings of the steps the paper leaves open:

* World space is the Feature Bounding Box scaled to [-1, 1]^3 (Section 3.1, Eqs. 1-2); the model
  coordinate is u = (p + 1) / 2 per axis, t_norm on time.
* Camera: rays from eye through pixel centres; pixel (i, j), row 0 at the top, looks along
  fwd + sx*right + sy*up, sx = (2i+1)/W - 1, sy = 1 - (2j+1)/H, normalised.
* Samples at fixed spacing delta = 1/(S_max - 1) world units (half the smallest voxel edge) from the
  entry point into the box: s_k = t_min + k*delta while s_k <= t_max; t_min is clamped at 0.
* Empty-space skipping (occupancy grid, Section 3.1 and 3.3): a sample is evaluated only when the
  voxel nearest to it, v = floor(u*(S-1) + 0.5), is occupied at time step floor(t) or - when t is
  between key frames - at the next one (the interpolated occupancy of an unseen time step is non-zero
  wherever either neighbour is occupied).
* Transfer function: 256 RGBA entries indexed by v clamped to [0,1] times 255 with linear
  interpolation; its alpha is already corrected for the spacing.  Front to back:
  C += T * alpha * rgb, T *= 1 - alpha, stop after the sample that makes 1 - T > 0.99; pixel =
  (C, 1 - T).  Rays that miss the box stay (0, 0, 0, 0).
The geometry (ray directions, box entry/exit, sample positions, voxel and time indices) decides
which integer samples exist, so it is evaluated in float32 with round-to-nearest and no fused
multiply-add, exactly as the GPU does; model values, transfer function and compositing are float64.
"""
import numpy as np

from . import encode, mlp

f32 = np.float32


def ray_setup(cam, width, height):
    """Per pixel: unit direction d [H*W][3] float32, t_min, t_max float32, hit mask."""
    eye, right, up, fwd = (np.asarray(v, f32) for v in cam)
    j, i = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    sx = (np.asarray(2 * i + 1, f32) / f32(width)) - f32(1.0)
    sy = f32(1.0) - (np.asarray(2 * j + 1, f32) / f32(height))
    sx, sy = sx.ravel(), sy.ravel()
    d = np.stack([(fwd[a] + sx * right[a]) + sy * up[a] for a in range(3)], 1).astype(f32)
    ln = np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])
    d = (d / ln[:, None]).astype(f32)
    tn = np.full(d.shape[0], -np.inf, f32)
    tf = np.full(d.shape[0], np.inf, f32)
    hit = np.ones(d.shape[0], bool)
    with np.errstate(divide="ignore", invalid="ignore"):
        for a in range(3):
            nz = d[:, a] != 0
            t0 = (f32(-1.0) - eye[a]) / d[:, a]
            t1 = (f32(1.0) - eye[a]) / d[:, a]
            lo, hi = np.minimum(t0, t1), np.maximum(t0, t1)
            tn = np.where(nz, np.maximum(tn, lo), tn)
            tf = np.where(nz, np.minimum(tf, hi), tf)
            if eye[a] < -1 or eye[a] > 1:
                hit &= nz
    tmin = np.maximum(tn, f32(0.0)).astype(f32)
    tmax = tf.astype(f32)
    hit &= tmin <= tmax
    return d, tmin, tmax, hit


def step_size(fbb_size):
    return f32(1.0 / (max(fbb_size) - 1))


def occupied(occ, fbb_size, t_norm, u):
    """Occupancy test of samples u [n][3] (float32) at t_norm (float32); occ bool [T][Sz][Sy][Sx]."""
    nt = occ.shape[0]
    v = [np.floor(u[:, a] * f32(fbb_size[a] - 1) + f32(0.5)).astype(np.int64) for a in range(3)]
    inside = np.ones(u.shape[0], bool)
    for a in range(3):
        inside &= (v[a] >= 0) & (v[a] < fbb_size[a])
    vc = [np.clip(v[a], 0, fbb_size[a] - 1) for a in range(3)]
    tq = f32(t_norm) * f32(nt - 1)
    tp = int(min(max(np.floor(tq), 0), nt - 1))
    wt = tq - f32(tp)
    tn = min(tp + 1, nt - 1)
    o = occ[tp][vc[2], vc[1], vc[0]]
    if wt > 0:
        o = o | occ[tn][vc[2], vc[1], vc[0]]
    return inside & o


def ray_samples(cam, width, height, fbb_size, occ, t_norm):
    """All occupied samples of every ray in marching order: (ray index, u [n][4] float32)."""
    d, tmin, tmax, hit = ray_setup(cam, width, height)
    eye = np.asarray(cam[0], f32)
    delta = step_size(fbb_size)
    rays, us = [], []
    k = 0
    active = np.nonzero(hit)[0]
    while active.size:
        s = tmin[active] + f32(k) * delta
        keep = s <= tmax[active]
        active, s = active[keep], s[keep]
        if not active.size:
            break
        p = np.stack([eye[a] + s * d[active, a] for a in range(3)], 1).astype(f32)
        u = ((p + f32(1.0)) * f32(0.5)).astype(f32)
        occd = occupied(occ, fbb_size, t_norm, u)
        rays.append(active[occd])
        us.append(u[occd])
        k += 1
    if not rays:
        return np.zeros(0, np.int64), np.zeros((0, 4), f32)
    r = np.concatenate(rays)
    u = np.concatenate(us)
    order = np.argsort(r, kind="stable")  # per ray, in k order
    u4 = np.concatenate([u[order], np.full((r.size, 1), f32(t_norm), f32)], 1)
    return r[order], u4


def transfer(v, tf):
    """RGBA from values v (float64) through the 256-entry table tf with linear interpolation."""
    x = np.clip(v, 0.0, 1.0) * 255.0
    i0 = np.minimum(np.floor(x).astype(np.int64), 254)
    f = (x - i0)[:, None]
    tf = np.asarray(tf, np.float64)
    return tf[i0] * (1.0 - f) + tf[i0 + 1] * f


def render(model_eval, cam, width, height, fbb_size, occ, t_norm, tf):
    """Image [H][W][4] float64 and per-pixel count of composited samples.  model_eval(u [n][4]) ->
    values [n] (float64)."""
    r, u = ray_samples(cam, width, height, fbb_size, occ, t_norm)
    vals = model_eval(u) if r.size else np.zeros(0)
    rgba = transfer(vals, tf)
    img = np.zeros((width * height, 4))
    counts = np.zeros(width * height, np.int64)
    T = np.ones(width * height)
    done = np.zeros(width * height, bool)
    for n in range(r.size):  # front to back, ray by ray in order
        ray = r[n]
        if done[ray]:
            continue
        a = rgba[n, 3]
        img[ray, :3] += T[ray] * a * rgba[n, :3]
        T[ray] *= 1.0 - a
        counts[ray] += 1
        if 1.0 - T[ray] > 0.99:
            done[ray] = True
    img[:, 3] = 1.0 - T
    hit = counts > 0
    img[~hit] = 0.0
    return img.reshape(height, width, 4), counts.reshape(height, width)


def model_eval_fn(levels, level_bases, table, mlp_params, dims, layout="linear"):
    def f(u):
        return mlp.forward(mlp_params, dims, encode.encode(levels, level_bases, u, table, layout))[0]
    return f


def decode_coords(fbb_size, upsample, t_norm):
    """Regular grid over the FBB at fractional t: n'_d = upsample*(S_d - 1) + 1 points per axis,
    u_d = j / (n'_d - 1) in float32.  Returns (u [n][4] float32 in [z][y][x] order, shape)."""
    n = [upsample * (s - 1) + 1 for s in fbb_size]
    ax = [(np.arange(n[a], dtype=f32) / f32(n[a] - 1)).astype(f32) for a in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    u = np.stack([x.ravel(), y.ravel(), z.ravel(), np.full(x.size, f32(t_norm), f32)], 1)
    return u, (n[2], n[1], n[0])
