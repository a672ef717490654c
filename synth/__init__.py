"""Seeded synthetic inputs shared by the CUDA path (tests, bench) and the oracle.

Only input data is made here: scalar fields shaped like the paper's datasets
(Table 2), threshold masks, uniform sample coordinates, training targets sampled
from a voxel field, initial parameter values, cameras and transfer functions.
Nothing in this package computes any step of the F-Hash method.  The heavy
generators are plain C (``synth.c``) compiled on first use with gcc.
"""
import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_synth.so")
_lib = None
_lock = threading.Lock()


def build(force=False):
    """Compile synth.c into _synth.so next to it (gcc, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i64, u64, f64, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
            lib.synth_splitmix64_at.restype = u64
            lib.synth_splitmix64_at.argtypes = [u64, u64]
            lib.synth_uniform.argtypes = [u64, u64, u64, i64, f64, f64, vp]
            lib.synth_field.restype = ctypes.c_int
            lib.synth_field.argtypes = [ctypes.c_int, u64, i64, i64, i64, i64, i64, i64, vp]
            lib.synth_rescale.argtypes = [vp, i64, f64, f64]
            lib.synth_minmax.argtypes = [vp, i64, ctypes.POINTER(f64), ctypes.POINTER(f64)]
            lib.synth_quantile.restype = ctypes.c_float
            lib.synth_quantile.argtypes = [vp, i64, f64, i64]
            lib.synth_mask.argtypes = [vp, i64, ctypes.c_float, ctypes.c_float, vp]
            lib.synth_sample.argtypes = [vp, i64, i64, i64, i64, vp, vp, vp, i64, vp]
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def splitmix64_at(seed, i):
    """i-th output (0-based) of SplitMix64 seeded with `seed`."""
    return int(_L().synth_splitmix64_at(seed & (2**64 - 1), i))


def uniform(seed, stream, n, lo=0.0, hi=1.0, offset=0):
    out = np.empty(int(n), np.float32)
    if n:
        _L().synth_uniform(seed, stream, offset, int(n), lo, hi, _p(out))
    return out


def field(kind, seed, nx, ny, nz, nt, normalise=None):
    """Scalar field [nt][nz][ny][nx] float32 of the given kind (see synth.c).
    Kinds 2-4 are normalised to [0,1] over the 4D domain (the paper normalises values to [0,1])."""
    out = np.empty((nt, nz, ny, nx), np.float32)
    rc = _L().synth_field(kind, seed, nx, ny, nz, nt, 0, nt, _p(out))
    if rc:
        raise ValueError("synth_field failed (%d)" % rc)
    if normalise is None:
        normalise = kind != 1
    if normalise:
        lo, hi = ctypes.c_double(), ctypes.c_double()
        _L().synth_minmax(_p(out), out.size, ctypes.byref(lo), ctypes.byref(hi))
        _L().synth_rescale(_p(out), out.size, lo.value, hi.value)
    return out


def quantile(v, q, stride=97):
    v = np.ascontiguousarray(v, np.float32)
    return float(_L().synth_quantile(_p(v), v.size, q, stride))


def mask(v, thr, hi=None):
    """u8 mask: v > thr, or thr < v < hi (interval feature) when hi is given."""
    v = np.ascontiguousarray(v, np.float32)
    out = np.empty(v.shape, np.uint8)
    _L().synth_mask(_p(v), v.size, thr, -np.inf if hi is None else hi, _p(out))
    return out


def coords(seed, n, stream=100, offset=0):
    """n uniform points in [0,1)^4, layout [n][4] = (x, y, z, t), FBB-normalised."""
    return uniform(seed, stream, 4 * int(n), offset=4 * int(offset)).reshape(int(n), 4)


def sample(fld, fbb_lo, fbb_size, pts):
    """Targets: field sampled at FBB-normalised points (trilinear in space, linear in time)."""
    fld = np.ascontiguousarray(fld, np.float32)
    nt, nz, ny, nx = fld.shape
    pts = np.ascontiguousarray(pts, np.float32)
    lo = np.ascontiguousarray(fbb_lo, np.int64)
    sz = np.ascontiguousarray(fbb_size, np.int64)
    out = np.empty(pts.shape[0], np.float32)
    _L().synth_sample(_p(fld), nx, ny, nz, nt, _p(lo), _p(sz), _p(pts), pts.shape[0], _p(out))
    return out


def init_tables(seed, n_params, r=1e-4):
    """Embedding initial values U(-r, r) (the paper: uniform initialisation)."""
    return uniform(seed, 200, n_params, -r, r)


def init_mlp(seed, dims):
    """Initial MLP parameters with PyTorch nn.Linear's default bounds U(-1/sqrt(fan_in), 1/sqrt(fan_in)).
    Flat layout per layer: W[out][in] then b[out]."""
    parts = []
    for k in range(len(dims) - 1):
        fi, fo = dims[k], dims[k + 1]
        b = 1.0 / math.sqrt(fi)
        parts.append(uniform(seed, 300 + 2 * k, fo * fi, -b, b))
        parts.append(uniform(seed, 301 + 2 * k, fo, -b, b))
    return np.concatenate(parts).astype(np.float32)


def camera(eye, width, height, fov_deg=60.0):
    """Pinhole camera looking at the origin, up +z (or +y when the view is nearly vertical).

    Returns (eye, right, up, fwd) as float32 [3] each, with right/up pre-scaled by the half extents
    of the image plane at unit distance, so pixel (i, j) looks along
    fwd + sx*right + sy*up, sx = (2i+1)/W - 1, sy = 1 - (2j+1)/H."""
    e = np.asarray(eye, np.float64)
    f = -e / np.linalg.norm(e)
    upv = np.array([0.0, 0.0, 1.0])
    if abs(f @ upv) > 0.999:
        upv = np.array([0.0, 1.0, 0.0])
    r = np.cross(f, upv)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(math.radians(fov_deg) / 2)
    return (e.astype(np.float32), (r * th * width / height).astype(np.float32),
            (u * th).astype(np.float32), f.astype(np.float32))


def sphere_eye(seed, i, radius=2.0):
    """i-th camera position uniform on the sphere of the given radius."""
    u = uniform(seed, 400, 2, offset=2 * i).astype(np.float64)
    z = 2 * u[0] - 1
    phi = 2 * math.pi * u[1]
    s = math.sqrt(max(0.0, 1 - z * z))
    return radius * np.array([s * math.cos(phi), s * math.sin(phi), z])


def transfer_function(step_voxels=0.5, kind=0):
    """256-entry RGBA table, float32 [256][4], alpha already corrected for the sample spacing:
    alpha' = 1 - (1 - alpha)^step (alpha is given per unit voxel)."""
    x = np.linspace(0.0, 1.0, 256)
    r = np.clip(1.5 * x, 0, 1)
    g = np.clip(1.5 * x - 0.5, 0, 1)
    b = np.clip(0.8 - x, 0, 1)
    if kind == 0:
        a = np.clip((x - 0.3) / 0.6, 0, 1) ** 2 * 0.6
    else:
        a = np.full_like(x, 0.2)
    a = 1.0 - (1.0 - a) ** step_voxels
    return np.stack([r, g, b, a], 1).astype(np.float32)
