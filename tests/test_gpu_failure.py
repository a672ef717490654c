"""Failure detection without a GPU fault: bounded device waits report through the model's error word,
invalid arguments are rejected on the host before anything is launched, and the model stays usable."""
import time

import numpy as np
import pytest

import synth
from synth import workloads

from _util import build, fh, to_dev, torch

pytestmark = pytest.mark.gpu
W1 = workloads.SMALL


def test_bounded_wait_times_out_and_reports():
    f, m = workloads.make_field_and_mask(W1)
    model = build(W1, mask=m, dtype=fh().BF16)
    fh().fhash_check(model)
    t0 = time.perf_counter()
    fh().fhash_diag_wait_timeout(model, 2_000_000)  # 2 ms: nothing ever arrives on the barrier
    with pytest.raises(fh().FHashError) as e:
        fh().fhash_check(model)
    assert e.value.status == 4 and time.perf_counter() - t0 < 5.0
    fh().fhash_check(model)  # the word is cleared by the check that reported it
    c = synth.coords(3, 1000)
    out = torch().empty(1000, dtype=torch().float32, device="cuda")
    fh().fhash_forward(model, to_dev(c), out)  # the context is still healthy
    fh().fhash_check(model)
    assert np.isfinite(out.cpu().numpy()).all()


def test_invalid_arguments_are_rejected():
    f, m = workloads.make_field_and_mask(W1)
    model = build(W1, mask=m)
    c = to_dev(synth.coords(3, 16))
    out = torch().empty(16, device="cuda")
    cases = [
        lambda: fh().fhash_build(1, 8, 8, 1),                                  # volume too small
        lambda: fh().fhash_build(8, 8, 8, 1, F=3),                             # F without kernels
        lambda: fh().fhash_build(8, 8, 8, 1, mlp_width=48),                    # width not 16/32/64
        lambda: fh().fhash_build(8, 8, 8, 1, mask=np.zeros((1, 8, 8, 8), np.uint8)),  # empty feature
        lambda: fh().fhash_apply_adam(model, (1e-2, 1.5, 0.99, 1e-8)),          # beta1 out of range
        lambda: fh().fhash_read_state(model, 0, 1 << 40, np.zeros(4, np.float32)),  # out of bounds
        lambda: fh().fhash_render(model, synth.camera([2, 0, 0], 4, 4), 1.5, to_dev(synth.transfer_function()), 4, 4,
                                  torch().empty((4, 4, 4), device="cuda")),    # t outside [0, 1]
        lambda: fh().fhash_decode(model, 0.5, 0, out),                          # upsample 0
        lambda: fh().fhash_diag_wait_timeout(model, 0),
    ]
    for i, fn in enumerate(cases):
        with pytest.raises(fh().FHashError) as e:
            fn()
        assert e.value.status == 1, i
    fh().fhash_forward(model, c, out)
    fh().fhash_check(model)
