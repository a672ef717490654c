"""Deferred Adam (fhash_set_adam_deferral) is bit-identical to the dense update (GPU, through the C ABI).

Two models start from the same parameters; one updates every parameter every step (deferral off), the
other defers the Adam update of its fine levels' rows to the next step that reads them.  After every
sequence below, parameters, gradients and both moments must be equal bit for bit.

For the comparison to be exact the two runs must see identical gradients, and the table scatter adds
with atomics in no fixed order.  So each step's batch holds samples whose cells share no vertex on any
level: one sample in each of a set of coarsest-level cells spaced far enough apart that no finer cell
spans two of them.  Every table row then receives its additions from a single thread, in program
order, and the whole step is deterministic.  The groups a batch touches change from step to step, so
replays of many lengths occur (the deferred rows of a group not touched for j steps replay j steps).

Covered: float32 and bf16 models (the bf16 shadow is refreshed by the replay), Eq. 9, brick and masked
rows, F = 1, 2 and 8, a flush in the middle of training (reading the state) followed by more deferred
steps, and plain fhash_compute_grads / fhash_apply_adam calls interleaved with deferred steps.  At the
bench size (advect-256^3x64, the default threshold of 2^25 rows, levels 12-15 deferred) the same
comparison runs on 20000 sampled rows of the deferred levels and every row the batches touched.
"""
import numpy as np
import pytest

import synth
from synth import workloads

from _util import fh, read, to_dev, torch

pytestmark = pytest.mark.gpu
W1 = workloads.SMALL


def disjoint_batch(rng, res, n=None):
    """Points in coarsest-level cells spaced S cells apart (S large enough that two of them are more than
    two cells apart on every finer level), one uniform point per chosen cell, t uniform."""
    R0 = res[0][:3]
    R1 = [min(r[a] for r in res[1:]) if len(res) > 1 else R0[a] for a in range(3)]
    S = [int(np.floor(0.9 + 2.0 * (R0[a] - 1) / max(R1[a] - 1, 1))) + 1 for a in range(3)]
    cells = [np.arange(0, R0[a] - 1, S[a]) for a in range(3)]
    grid = np.stack(np.meshgrid(*cells, indexing="ij"), -1).reshape(-1, 3)
    if n is not None and n < grid.shape[0]:
        grid = grid[rng.choice(grid.shape[0], n, replace=False)]
    u = (grid + 0.05 + 0.9 * rng.random(grid.shape)) / (np.array(R0) - 1)
    t = rng.random((grid.shape[0], 1))
    return np.concatenate([u, t], 1).astype(np.float32)


def _build(m, F=2, dtype=0, layout=0, res=None, seed=5):
    nx, ny, nz, nt = W1["dims"]
    sched = dict(mode="explicit", res=res) if res else W1["schedule"]
    return fh().fhash_build(nx, ny, nz, nt, mask=m, schedule=fh().make_schedule(**sched), F=F, dtype=dtype,
                            mlp_hidden_layers=W1["hidden"], mlp_width=W1["width"], seed=seed, init_range=0.3,
                            layout=layout)


def _state(model, n_all):
    return [read(model, w, 0, n_all).view(np.uint32) for w in
            (fh().STATE_PARAM, fh().STATE_GRAD, fh().STATE_ADAM_M, fh().STATE_ADAM_V)]


def _equal(a, b, n_all):
    sa, sb = _state(a, n_all), _state(b, n_all)
    for name, x, y in zip(("param", "grad", "m", "v"), sa, sb):
        bad = np.flatnonzero(x != y)
        assert bad.size == 0, (name, bad[:10], bad.size)


@pytest.fixture(scope="module")
def field_mask():
    return workloads.make_field_and_mask(W1)


RES_MIXED = [[4, 4, 4, 1], [9, 7, 8, 2], [16, 15, 17, 4], [32, 31, 30, 8]]


@pytest.mark.parametrize("F,dtype,layout,res", [(2, "fp32", "linear", None), (2, "fp32", "brick", None),
                                                (2, "bf16", "brick", None), (1, "fp32", "linear", RES_MIXED),
                                                (8, "fp32", "brick", RES_MIXED), (2, "fp32", "masked", None)])
def test_deferred_equals_dense(field_mask, F, dtype, layout, res):
    f, m = field_mask
    lay = {"linear": fh().LAYOUT_LINEAR, "brick": fh().LAYOUT_BRICK, "masked": fh().LAYOUT_MASKED}[layout]
    dt = fh().BF16 if dtype == "bf16" else fh().FP32
    dense = _build(m, F, dt, lay, res)
    lazy = _build(m, F, dt, lay, res)
    fh().fhash_set_adam_deferral(dense, 0)
    fh().fhash_set_adam_deferral(lazy, 500)  # every level with at least 500 rows: all but the coarsest
    info = fh().fhash_get_info(lazy)
    n_all = info["n_table_params"] + info["n_mlp_params"]
    st = fh().fhash_get_adam_stats(lazy)
    assert st["first_deferred_level"] == 1 and st["deferred_params"] > 0.9 * info["n_table_params"]
    assert fh().fhash_get_adam_stats(dense)["first_deferred_level"] == -1
    rng = np.random.default_rng(11)
    hp = (1e-2, 0.9, 0.99, 1e-8)
    replayed = 0

    def step(k):
        nonlocal replayed
        # every fourth step reuses the previous batch's cells (touched again one step later: replays of
        # length 0 and 1); the others draw a new subset (long gaps)
        c = disjoint_batch(np.random.default_rng(1000 + (k // 4 if k % 4 == 1 else k)), info["res"], n=6)
        tgt = synth.sample(f, info["fbb_lo"], info["fbb_size"], c)
        ld, ll = np.zeros(1), np.zeros(1)
        fh().fhash_train_step(dense, to_dev(c), to_dev(tgt), hp, ld)
        fh().fhash_train_step(lazy, to_dev(c), to_dev(tgt), hp, ll)
        assert ld[0] == ll[0], (k, ld[0], ll[0])
        replayed += fh().fhash_get_adam_stats(lazy)["last_replayed_steps"]

    for k in range(25):
        step(k)
    assert fh().fhash_get_adam_stats(lazy)["clean_step"] < 25
    _equal(dense, lazy, n_all)  # reading the state brings every deferred group to step 25
    assert fh().fhash_get_adam_stats(lazy)["clean_step"] == 25
    # plain calls between deferred steps: a gradient accumulated outside the step, a dense update
    c = disjoint_batch(rng, info["res"], n=5)
    tgt = synth.sample(f, info["fbb_lo"], info["fbb_size"], c)
    for mdl in (dense, lazy):
        fh().fhash_compute_grads(mdl, to_dev(c), to_dev(tgt))
    for k in range(25, 32):
        step(k)
    for mdl in (dense, lazy):
        fh().fhash_apply_adam(mdl, hp)
    for k in range(32, 50):
        step(k)
    assert replayed > 0
    pts = synth.coords(3, 4000)
    outs = []
    for mdl in (dense, lazy):
        o = torch().empty(4000, dtype=torch().float32, device="cuda")
        fh().fhash_forward(mdl, to_dev(pts), o)  # the forward reads the (bf16 shadow of the) settled tables
        outs.append(o.cpu().numpy())
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))
    _equal(dense, lazy, n_all)
    assert fh().fhash_get_info(lazy)["step"] == fh().fhash_get_info(dense)["step"] == 51
    fh().fhash_check(lazy)


def test_deferral_threshold_and_checkpoint(field_mask, tmp_path):
    """Changing the threshold mid-training settles first; a checkpoint of a model with deferred groups holds
    the settled state and training resumes from it exactly."""
    f, m = field_mask
    a, b = _build(m), _build(m)
    fh().fhash_set_adam_deferral(a, 0)
    fh().fhash_set_adam_deferral(b, 100)
    info = fh().fhash_get_info(b)
    n_all = info["n_table_params"] + info["n_mlp_params"]
    hp = (1e-2, 0.9, 0.99, 1e-8)

    def run(models, ks):
        for k in ks:
            c = disjoint_batch(np.random.default_rng(50 + k), info["res"], n=7)
            tgt = to_dev(synth.sample(f, info["fbb_lo"], info["fbb_size"], c))
            for mdl in models:
                fh().fhash_train_step(mdl, to_dev(c), tgt, hp)

    run((a, b), range(8))
    fh().fhash_set_adam_deferral(b, 20000)   # only the finest level
    assert fh().fhash_get_adam_stats(b)["first_deferred_level"] == 3
    run((a, b), range(8, 16))
    path = str(tmp_path / "deferred.fhc")
    fh().fhash_save(b, path)
    c2 = fh().fhash_load(path)
    fh().fhash_set_adam_deferral(c2, 100)
    run((a, b, c2), range(16, 24))
    _equal(a, b, n_all)
    _equal(a, c2, n_all)


def test_fullsize_deferred_equals_dense():
    """advect-256^3x64 in the bench's configuration (brick rows, default threshold: levels 12-15, 3.47e9
    parameters deferred) against deferral off, 10 steps of deterministic batches."""
    W = workloads.LARGE
    f, m = workloads.make_field_and_mask(W)
    nx, ny, nz, nt = W["dims"]
    models = [fh().fhash_build(nx, ny, nz, nt, mask=m, schedule=fh().make_schedule(**W["schedule"]), F=W["F"],
                               mlp_hidden_layers=W["hidden"], mlp_width=W["width"], seed=3, init_range=0.1,
                               layout=fh().LAYOUT_BRICK) for _ in range(2)]
    del m
    dense, lazy = models
    fh().fhash_set_adam_deferral(dense, 0)
    info = fh().fhash_get_info(lazy)
    st = fh().fhash_get_adam_stats(lazy)
    assert st["first_deferred_level"] == 12, st
    F = info["F"]
    touched = []
    hp = W["adam"]
    for k in range(10):
        c = disjoint_batch(np.random.default_rng(70 + k), info["res"])
        assert c.shape[0] == 27
        tgt = to_dev(synth.sample(f, info["fbb_lo"], info["fbb_size"], c))
        ld, ll = np.zeros(1), np.zeros(1)
        fh().fhash_train_step(dense, to_dev(c), tgt, hp, ld)
        fh().fhash_train_step(lazy, to_dev(c), tgt, hp, ll)
        assert ld[0] == ll[0], k
        rows = torch().empty((c.shape[0], info["n_levels"], 16), dtype=torch().int64, device="cuda")
        fh().fhash_lookup(lazy, to_dev(c), rows)
        touched.append(rows.cpu().numpy()[:, 12:, :].ravel())
    touched = np.unique(np.concatenate(touched))
    lo = info["base"][12]
    sample = np.random.default_rng(1).integers(lo, info["total_rows"], 20000)
    rows = np.unique(np.concatenate([touched, sample]))
    for which in (fh().STATE_PARAM, fh().STATE_ADAM_M, fh().STATE_ADAM_V, fh().STATE_GRAD):
        got = [np.empty((rows.size, F), np.float32) for _ in range(2)]
        one = np.empty(F, np.float32)
        for g, mdl in zip(got, models):
            for i, r in enumerate(rows):
                fh().fhash_read_state(mdl, which, int(r) * F, one)
                g[i] = one
        assert np.array_equal(got[0].view(np.uint32), got[1].view(np.uint32)), which
    n_t = info["n_table_params"]
    mlp = [read(mdl, fh().STATE_PARAM, n_t, info["n_mlp_params"]) for mdl in models]
    assert np.array_equal(mlp[0].view(np.uint32), mlp[1].view(np.uint32))
    fh().fhash_check(lazy)
    del models, dense, lazy
