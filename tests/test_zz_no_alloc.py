"""fhash_compute_grads_noalloc against fhash_compute_grads (GPU, through the C ABI).

The no-allocation variant exists for callers that cannot call cudaMalloc (an application that has
given all device memory to its own pool, or a loop that cannot take the implicit device
synchronisation of cudaMalloc/cudaFree).  It must give the same loss and gradients as the regular
entry point: checked here on two calls in a row (gradients accumulate), within the tolerance of the
gradient parity test (1e-4 relative to the magnitude of the entries; the atomic scatter order differs
between runs).  This file is collected last so that a first-failure stop has run every other test.
"""
import numpy as np
import pytest

import synth
from synth import workloads

from _util import build, fh, read, set_params, to_dev, torch

pytestmark = pytest.mark.gpu
W1 = workloads.SMALL


def _close(a, b):
    scale = np.abs(a) + np.abs(b) + 1e-6 * max(np.abs(a).max(), np.abs(b).max(), 1e-30)
    return (np.abs(a - b) <= 1e-4 * scale).all()


def test_noalloc_matches_regular_entry_point():
    f, m = workloads.make_field_and_mask(W1)
    ref = build(W1, mask=m, seed=4)
    alt = build(W1, mask=m, seed=4)
    info = fh().fhash_get_info(ref)
    table = synth.uniform(8, 50, info["n_table_params"], -0.5, 0.5)
    p = synth.init_mlp(8, info["mlp_dims"])
    set_params(ref, table, p)
    set_params(alt, table, p)
    n_all = info["n_table_params"] + info["n_mlp_params"]
    for call, n in enumerate((fh().NOALLOC_MAX_SAMPLES, 777)):
        c = synth.coords(60 + call, n)
        tgt = synth.sample(f, info["fbb_lo"], info["fbb_size"], c)
        cd, td = to_dev(c), to_dev(tgt)
        l_ref = np.zeros(1, np.float64)
        l_alt = torch().zeros(1, dtype=torch().float64, device="cuda")
        fh().fhash_compute_grads(ref, cd, td, l_ref)
        fh().fhash_compute_grads_noalloc(alt, cd, td, l_alt)
        torch().cuda.synchronize()
        assert abs(l_alt.item() - l_ref[0]) <= 1e-6 * l_ref[0], call
        g_ref = read(ref, fh().STATE_GRAD, 0, n_all)
        g_alt = read(alt, fh().STATE_GRAD, 0, n_all)
        assert np.abs(g_ref).max() > 0
        assert _close(g_alt, g_ref), call
    fh().fhash_check(alt)


def test_noalloc_rejects_oversized_batch():
    f, m = workloads.make_field_and_mask(W1)
    model = build(W1, mask=m)
    n = fh().NOALLOC_MAX_SAMPLES + 1
    c = to_dev(synth.coords(1, n))
    t = to_dev(np.zeros(n, np.float32))
    with pytest.raises(fh().FHashError) as e:
        fh().fhash_compute_grads_noalloc(model, c, t)
    assert e.value.status == 1 and "n <=" in str(e.value)
