"""fhash_compute_grads_noalloc against fhash_compute_grads (GPU, through the C ABI).

The no-allocation variant exists for callers that cannot call cudaMalloc (an application that has
given all device memory to its own pool, or a loop that cannot take the implicit device
synchronisation of cudaMalloc/cudaFree).  It must give the same loss and gradients as the regular
entry point: checked here on two calls in a row (gradients accumulate), within the tolerance of the
gradient parity tests (both within 1e-4 x the sum of the magnitudes of each entry's terms of the
exact gradient, so within 2e-4 of each other), for both rectangular row layouts, embedding sizes F = 1, 2, 4 and 8, and a model built
in the bf16 precision form (whose float32 form this call evaluates: it is compared with a float32
model holding the same parameters).  The call must also leave the device's free memory unchanged.
This file is collected last so that a first-failure stop has run every other test.
"""
import numpy as np
import pytest

import synth
from synth import workloads
from oracle import encode, mlp

from _util import fh, read, set_params, to_dev, torch

pytestmark = pytest.mark.gpu
W1 = workloads.SMALL


def _build(m, F, dtype, layout, seed=4):
    nx, ny, nz, nt = W1["dims"]
    return fh().fhash_build(nx, ny, nz, nt, mask=m, schedule=fh().make_schedule(**W1["schedule"]), F=F, dtype=dtype,
                            mlp_hidden_layers=W1["hidden"], mlp_width=W1["width"], seed=seed,
                            init_range=W1["init_range"], layout=layout)


@pytest.fixture(scope="module")
def field_mask():
    return workloads.make_field_and_mask(W1)


@pytest.mark.parametrize("layout,F,dtype", [("linear", 2, "fp32"), ("brick", 2, "fp32"), ("linear", 4, "fp32"),
                                            ("brick", 1, "fp32"), ("brick", 8, "fp32"), ("brick", 2, "bf16"),
                                            ("linear", 4, "bf16")])
def test_noalloc_matches_regular_entry_point(field_mask, layout, F, dtype):
    f, m = field_mask
    lay = fh().LAYOUT_BRICK if layout == "brick" else fh().LAYOUT_LINEAR
    ref = _build(m, F, fh().FP32, lay)
    alt = _build(m, F, fh().BF16 if dtype == "bf16" else fh().FP32, lay)
    info = fh().fhash_get_info(ref)
    table = synth.uniform(8, 50, info["n_table_params"], -0.5, 0.5)
    p = synth.init_mlp(8, info["mlp_dims"])
    set_params(ref, table, p)
    set_params(alt, table, p)
    n_t, n_all = info["n_table_params"], info["n_table_params"] + info["n_mlp_params"]
    T = table.reshape(-1, F).astype(np.float64)
    pd = p.astype(np.float64)
    abs_mlp = np.zeros(info["n_mlp_params"])
    abs_tab = np.zeros(n_t)
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
        # Both entry points are within 1e-4 x the sum of the magnitudes of each entry's terms of the exact
        # gradient (the bound of the gradient parity tests; the regular one forms the MLP gradients on the
        # tensor cores with 3xTF32 products, this one with float32 products on the CUDA cores, and their
        # atomic scatter orders differ), so they are within 2e-4 of each other.  Terms from the oracle.
        y, a, z = mlp.forward(pd, info["mlp_dims"], encode.encode(info["res"], info["base"], c, T, layout))
        _, gy = mlp.mse(y, tgt)
        g_abs, d_abs = mlp.backward(np.abs(pd), info["mlp_dims"], [np.abs(x) for x in a],
                                    [np.where(x > 0, 1.0, -1.0) for x in z], np.abs(gy))
        abs_mlp += g_abs
        rows, t_abs = encode.encode_backward(info["res"], info["base"], c, d_abs, F, layout)
        abs_tab[(rows[:, None] * F + np.arange(F)).ravel()] += t_abs.ravel()
        assert (np.abs(g_alt[:n_t] - g_ref[:n_t]) <= 2e-4 * abs_tab + 1e-12).all(), call
        assert (np.abs(g_alt[n_t:] - g_ref[n_t:]) <= 2e-4 * abs_mlp + 1e-12).all(), call
    fh().fhash_check(alt)


def test_noalloc_leaves_free_memory_unchanged(field_mask):
    f, m = field_mask
    model = _build(m, 2, fh().FP32, fh().LAYOUT_BRICK, seed=9)
    info = fh().fhash_get_info(model)
    batches = []
    for n in (fh().NOALLOC_MAX_SAMPLES, 1, 333, 2048):
        c = synth.coords(90 + n, n)
        batches.append((to_dev(c), to_dev(synth.sample(f, info["fbb_lo"], info["fbb_size"], c))))
    loss = torch().zeros(1, dtype=torch().float64, device="cuda")
    fh().fhash_compute_grads_noalloc(model, *batches[0], loss)  # loads the library's kernels and array
    torch().cuda.synchronize()
    free0 = torch().cuda.mem_get_info()[0]
    for cd, td in batches:
        fh().fhash_compute_grads_noalloc(model, cd, td, loss)
    torch().cuda.synchronize()
    assert torch().cuda.mem_get_info()[0] == free0
    fh().fhash_check(model)


def test_noalloc_rejects_oversized_batch(field_mask):
    f, m = field_mask
    model = _build(m, 2, fh().FP32, fh().LAYOUT_LINEAR)
    n = fh().NOALLOC_MAX_SAMPLES + 1
    c = to_dev(synth.coords(1, n))
    t = to_dev(np.zeros(n, np.float32))
    with pytest.raises(fh().FHashError) as e:
        fh().fhash_compute_grads_noalloc(model, c, t)
    assert e.value.status == 1 and "n <=" in str(e.value)
