"""Checkpoint save/load through the C ABI: the loaded model is bit-identical in every state vector,
description and occupancy grid, and training continues from it as from the original."""
import os

import numpy as np
import pytest

import synth
from synth import workloads

from _util import build, fh, read, to_dev, torch

pytestmark = pytest.mark.gpu
W1 = workloads.SMALL


@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
def test_save_load_roundtrip_and_continue(tmp_path, dtype):
    f, m = workloads.make_field_and_mask(W1)
    dt = fh().FP32 if dtype == "fp32" else fh().BF16
    a = build(W1, mask=m, dtype=dt, seed=29)
    info = fh().fhash_get_info(a)
    batches = []
    for k in range(30):
        c = synth.coords(900 + k, 4096)
        batches.append((to_dev(c), to_dev(synth.sample(f, info["fbb_lo"], info["fbb_size"], c))))
    for c, t in batches[:20]:
        fh().fhash_train_step(a, c, t, W1["adam"])
    path = os.path.join(tmp_path, "model.fhck")
    fh().fhash_save(a, path)
    b = fh().fhash_load(path)
    ia, ib = fh().fhash_get_info(a), fh().fhash_get_info(b)
    for k in ("res", "base", "fbb_lo", "fbb_size", "mlp_dims", "step", "n_table_params", "dtype", "nt"):
        assert ia[k] == ib[k], k
    n = ia["n_table_params"] + ia["n_mlp_params"]
    for which in (fh().STATE_PARAM, fh().STATE_GRAD, fh().STATE_ADAM_M, fh().STATE_ADAM_V):
        assert np.array_equal(read(a, which, 0, n), read(b, which, 0, n)), which
    s = ia["fbb_size"]
    for t in range(ia["nt"]):
        oa = np.empty((s[2], s[1], s[0]), np.uint8)
        ob = np.empty_like(oa)
        fh().fhash_read_occupancy(a, t, oa)
        fh().fhash_read_occupancy(b, t, ob)
        assert np.array_equal(oa, ob)
    la, lb = [], []
    for c, t in batches[20:]:
        for mm, out in ((a, la), (b, lb)):
            loss = np.zeros(1)
            fh().fhash_train_step(mm, c, t, W1["adam"], loss)
            out.append(loss[0])
    # same state, same inputs: only the atomic summation order of the table gradients differs
    assert np.allclose(la, lb, rtol=1e-5, atol=0)


def test_load_rejects_foreign_and_truncated(tmp_path):
    bad = os.path.join(tmp_path, "bad.fhck")
    open(bad, "wb").write(b"not a checkpoint" * 100)
    with pytest.raises(fh().FHashError) as e:
        fh().fhash_load(bad)
    assert e.value.status == 7
    f, m = workloads.make_field_and_mask(W1)
    a = build(W1, mask=m, seed=2)
    good = os.path.join(tmp_path, "good.fhck")
    fh().fhash_save(a, good)
    data = open(good, "rb").read()
    open(bad, "wb").write(data[: len(data) // 2])
    with pytest.raises(fh().FHashError) as e:
        fh().fhash_load(bad)
    assert e.value.status == 7
    with pytest.raises(fh().FHashError):
        fh().fhash_load(os.path.join(tmp_path, "missing.fhck"))
