"""Workload descriptions (input recipes) used by the tests and the bench.

Each workload names a synthetic field (kind and seed of synth.field), how its feature mask is
made, the level schedule, embedding size, MLP shape, batch and Adam settings.  These are
inputs and hyper-parameters only.
"""
import numpy as np

from . import field as _field
from . import mask as _mask
from . import quantile as _quantile

# 32^3 x 8 field of 4 moving Gaussian blobs; 4 levels doubling from 4^3x1 to 32^3x8; F=2; MLP 2x32.
SMALL = dict(name="blobs-32^3x8", kind=1, seed=0, dims=(32, 32, 32, 8), mask=("gt", 0.5),
             schedule=dict(mode="explicit", res=[[4, 4, 4, 1], [8, 8, 8, 2], [16, 16, 16, 4], [32, 32, 32, 8]]),
             F=2, hidden=2, width=32, batch=16384, adam=(1e-2, 0.9, 0.99, 1e-8), init_range=1e-4)

# 256^3 x 64 field of 64 advecting blobs + 3-octave value noise; mask above the 80th percentile;
# 16 levels geometric 8^3x2 -> 256^3x64; F=2; MLP 2x64; batch 2^18; Adam lr 1e-2, betas 0.9/0.99.
LARGE = dict(name="advect-256^3x64", kind=2, seed=1, dims=(256, 256, 256, 64), mask=("quantile", 0.8),
             schedule=dict(mode="geometric", n_levels=16, r0=[8, 8, 8, 2], r1=[256, 256, 256, 64]),
             F=2, hidden=2, width=64, batch=2 ** 18, adam=(1e-2, 0.9, 0.99, 1e-8), init_range=1e-4)

# 128^3 x 32 version of LARGE (same recipe; about 3.3 GB of training state, still larger than L2):
# the size used for detailed profiler captures and full-launch parity checks.
MEDIUM = dict(LARGE, name="advect-128^3x32", dims=(128, 128, 128, 32),
              schedule=dict(mode="geometric", n_levels=16, r0=[8, 8, 8, 2], r1=[128, 128, 128, 32]))

# Combustion-shaped precision workload: 480x720x120 x 100 flame-like front along a noisy surface
# advancing 2 voxels/step + 4-octave noise; interval feature 0.05 < v < 0.95; 16 levels geometric
# from about 1/32 of the volume to the volume in space and 2 -> 10 in time (10 key-frame levels);
# F=4; MLP 3x64; batch 2^20.
FRONT = dict(name="front-480x720x120x100", kind=3, seed=2, dims=(480, 720, 120, 100), mask=("interval", 0.05, 0.95),
             schedule=dict(mode="geometric", n_levels=16, r0=[15, 23, 4, 2], r1=[480, 720, 120, 10]),
             F=4, hidden=3, width=64, batch=2 ** 20, adam=(1e-2, 0.9, 0.99, 1e-8), init_range=1e-4)

# Supernova-shaped serving workload: 432^3 x 60 expanding radial shell + 4-octave noise; feature
# v > 0.5; 16 levels geometric 14^3x2 -> 432^3x16; F=2; MLP 2x64; batch 2^18.
SHELL = dict(name="shell-432^3x60", kind=4, seed=3, dims=(432, 432, 432, 60), mask=("gt", 0.5),
             schedule=dict(mode="geometric", n_levels=16, r0=[14, 14, 14, 2], r1=[432, 432, 432, 16]),
             F=2, hidden=2, width=64, batch=2 ** 18, adam=(1e-2, 0.9, 0.99, 1e-8), init_range=1e-4)


def make_field_and_mask(w, dims=None):
    nx, ny, nz, nt = dims or w["dims"]
    f = _field(w["kind"], w["seed"], nx, ny, nz, nt)
    how = w["mask"][0]
    if how == "gt":
        return f, _mask(f, w["mask"][1])
    if how == "interval":
        return f, _mask(f, w["mask"][1], w["mask"][2])
    return f, _mask(f, _quantile(f, w["mask"][1]))
