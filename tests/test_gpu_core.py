"""GPU parity of the index builder, encoding, forward, gradients, Adam and training against the oracle.

Every test calls the CUDA path through the C ABI (Python binding = marshalling only) and compares it
with the FP64 oracle on the same seeded inputs.  Tolerances: table rows bit-exact; FP32 encoding
|g - o| <= 1e-5 * sum_c |w_c T_c| + 1e-30; FP32 MLP output |g - o| <= 1e-4 * max(|o|, RMS(o)).
"""
import numpy as np
import pytest

import synth
from synth import workloads
from oracle import adam, encode, index, mlp, rng, schedule, train

from _util import build, fh, oracle_levels, read, set_params, to_dev, torch

pytestmark = pytest.mark.gpu
W1 = workloads.SMALL


@pytest.fixture(scope="module")
def small():
    f, m = workloads.make_field_and_mask(W1)
    model = build(W1, mask=m)
    info = fh().fhash_get_info(model)
    return dict(field=f, mask=m, model=model, info=info)


EDGE = np.array([[0, 0, 0, 0], [1, 1, 1, 1], [0.5, 0.5, 0.5, 0.5], [1, 0, 1, 0], [-0.25, 1.5, 0.3, 2.0],
                 [np.nan, 0.2, 0.7, np.nan]], np.float32)
# The C ABI takes float32 hyper-parameters; the oracle is given exactly those values.
HP32 = tuple(float(np.float32(x)) for x in W1["adam"])
R32 = float(np.float32(W1["init_range"]))


def _coords(n, seed=11):
    c = synth.coords(seed, n)
    k = min(n, len(EDGE))
    c[:k] = EDGE[:k]
    return c


def _random_params(info, seed=3, r=1.0):
    table = synth.uniform(seed, 50, info["n_table_params"], -r, r)
    p = synth.init_mlp(seed, info["mlp_dims"])
    return table, p


def test_build_fbb_and_occupancy(small):
    d = index.dilate(small["mask"])
    lo, size = index.fbb(d)
    info = small["info"]
    assert info["fbb_lo"] == lo and info["fbb_size"] == size
    occ = index.occupancy(d, lo, size)
    for t in range(info["nt"]):
        got = np.empty((size[2], size[1], size[0]), np.uint8)
        fh().fhash_read_occupancy(small["model"], t, got)
        assert np.array_equal(got.astype(bool), occ[t]), t


def test_levels_and_bases(small):
    info = small["info"]
    lv = oracle_levels(W1)
    b, total = schedule.bases(lv)
    assert info["res"] == lv and info["base"] == b and info["total_rows"] == total
    assert info["mlp_dims"] == [8, 32, 32, 1]


@pytest.mark.parametrize("mode", ["fold-max", "fold-min", "geometric"])
def test_schedules_match_oracle(mode):
    m = np.zeros((5, 40, 30, 50), np.uint8)
    m[1, 10:15, 4:20, 7:31] = 1
    m[3, 30:33, 25:28, 40:44] = 1
    lo, size = index.fbb(index.dilate(m))
    if mode == "geometric":
        w = dict(W1, schedule=dict(mode="geometric", n_levels=7, r0=[3, 4, 2, 2], r1=[40, 33, 17, 5]))
    else:
        w = dict(W1, schedule=dict(mode="fold", fold=2, levels_rule=0 if mode == "fold-max" else 1))
    model = build(w, mask=m, dims=(50, 30, 40, 5))
    info = fh().fhash_get_info(model)
    assert info["fbb_lo"] == lo and info["fbb_size"] == size
    assert info["res"] == oracle_levels(w, size, 5)


def test_initial_parameters(small):
    info = small["info"]
    idx = np.unique(np.concatenate([np.arange(64), np.random.default_rng(0).integers(0, info["n_table_params"], 4000),
                                    [info["n_table_params"] - 1]]))
    got = np.array([read(small["model"], 0, int(i), 1)[0] for i in idx[:64]])
    assert np.array_equal(got, rng.uniform_range(7, 200, idx[:64].astype(np.uint64), -R32, R32))
    allt = read(small["model"], 0, 0, info["n_table_params"])
    assert np.array_equal(allt[idx], rng.uniform_range(7, 200, idx.astype(np.uint64), -R32, R32))
    p = read(small["model"], 0, info["n_table_params"], info["n_mlp_params"])
    assert np.array_equal(p, synth.init_mlp(7, info["mlp_dims"]))


def test_lookup_rows_bit_exact(small):
    info = small["info"]
    lv, b = info["res"], info["base"]
    c = _coords(3001)
    L = len(lv)
    rows = torch().empty((c.shape[0], L, 16), dtype=torch().int64, device="cuda")
    w = torch().empty((c.shape[0], L, 16), dtype=torch().float32, device="cuda")
    fh().fhash_lookup(small["model"], to_dev(c), rows, w)
    rows = rows.cpu().numpy().view(np.uint64)
    w = w.cpu().numpy()
    for l in range(L):
        r_o, w_o = encode.level_corners(c, lv[l], b[l])
        assert np.array_equal(rows[:, l, :], r_o.astype(np.uint64)), l
        assert np.abs(w[:, l, :] - w_o).max() <= 4e-7


def test_encode_parity(small):
    info = small["info"]
    table, p = _random_params(info)
    set_params(small["model"], table, p)
    c = _coords(5003)
    enc = torch().empty((c.shape[0], info["n_levels"] * info["F"]), dtype=torch().float32, device="cuda")
    fh().fhash_encode(small["model"], to_dev(c), enc)
    got = enc.cpu().numpy()
    T = table.reshape(-1, info["F"]).astype(np.float64)
    ref = encode.encode(info["res"], info["base"], c, T)
    scale = encode.encode(info["res"], info["base"], c, np.abs(T))  # sum_c |w_c T_c|
    assert (np.abs(got - ref) <= 1e-5 * scale + 1e-30).all(), np.abs(got - ref).max()


def test_forward_parity_host_and_device(small):
    info = small["info"]
    table, p = _random_params(info, seed=4, r=0.5)
    set_params(small["model"], table, p)
    c = _coords(4099)
    T = table.reshape(-1, info["F"]).astype(np.float64)
    ref = mlp.forward(p, info["mlp_dims"], encode.encode(info["res"], info["base"], c, T))[0]
    out = torch().empty(c.shape[0], dtype=torch().float32, device="cuda")
    fh().fhash_forward(small["model"], to_dev(c), out)
    got_d = out.cpu().numpy()
    got_h = np.empty(c.shape[0], np.float32)
    fh().fhash_forward(small["model"], c, got_h)  # host buffers, staged by the library
    tol = 1e-4 * np.maximum(np.abs(ref), np.sqrt(np.mean(ref ** 2)))
    assert (np.abs(got_d - ref) <= tol).all(), np.abs(got_d - ref).max()
    assert np.array_equal(got_d, got_h)


def test_empty_and_ragged_batches(small):
    f = fh()
    out = torch().empty(0, dtype=torch().float32, device="cuda")
    f.fhash_forward(small["model"], torch().empty((0, 4), device="cuda"), out)
    for n in (1, 127, 129, 1000):
        c = _coords(n, seed=20 + n)
        a = torch().empty(n, dtype=torch().float32, device="cuda")
        f.fhash_forward(small["model"], to_dev(c), a)
        b = torch().empty(n + 5, dtype=torch().float32, device="cuda")
        f.fhash_forward(small["model"], to_dev(np.concatenate([c, _coords(5, 99)])), b)
        assert torch().equal(a, b[:n])  # per-sample results independent of batch size / position


def test_gradients_parity(small):
    info = small["info"]
    model = build(W1, mask=small["mask"])
    table, p = _random_params(info, seed=5, r=0.5)
    set_params(model, table, p)
    c = _coords(3000, seed=12)
    tgt = synth.sample(small["field"], info["fbb_lo"], info["fbb_size"], np.nan_to_num(np.clip(c, 0, 1)))
    loss = np.zeros(1, np.float64)
    fh().fhash_compute_grads(model, to_dev(c), to_dev(tgt), loss)
    T = table.reshape(-1, info["F"]).astype(np.float64)
    L, _, g_mlp, (rows, g_rows) = train.loss_and_grads(info["res"], info["base"], info["F"], info["mlp_dims"], T, p, c, tgt)
    assert abs(loss[0] - L) <= 1e-5 * L
    n_t = info["n_table_params"]
    g = read(model, 1, 0, n_t + info["n_mlp_params"])
    # scale: the same backward on absolute values bounds the sum of |terms| of every gradient entry
    enc = encode.encode(info["res"], info["base"], c, T)
    y, a, z = mlp.forward(p, info["mlp_dims"], enc)
    _, gy = mlp.mse(y, tgt)
    Wabs = np.abs(p)
    abs_mlp, abs_denc = mlp.backward(Wabs, info["mlp_dims"], [np.abs(x) for x in a],
                                     [np.where(x > 0, 1.0, -1.0) for x in z], np.abs(gy))
    assert (np.abs(g[n_t:] - g_mlp) <= 1e-4 * abs_mlp + 1e-12).all()
    _, g_abs = encode.encode_backward(info["res"], info["base"], c, abs_denc, info["F"])
    gt = g[:n_t].reshape(-1, info["F"])
    assert (np.abs(gt[rows] - g_rows) <= 1e-4 * g_abs + 1e-12).all()
    untouched = np.ones(gt.shape[0], bool)
    untouched[rows] = False
    assert (gt[untouched] == 0).all()


def test_adam_parity(small):
    # Each step is checked from the GPU's own state before it (p, m, v read back), fed the GPU's
    # gradient, so fp32 rounding of earlier steps does not compound.  Scales: m and v are sums of two
    # terms, so their error is bounded relative to the sum of the terms' magnitudes.
    info = small["info"]
    model = build(W1, mask=small["mask"])
    table, p = _random_params(info, seed=6, r=0.5)
    set_params(model, table, p)
    n = info["n_table_params"] + info["n_mlp_params"]
    lr, b1, b2, eps = HP32
    for k in range(1, 4):
        c = _coords(2048, seed=30 + k)
        tgt = synth.sample(small["field"], info["fbb_lo"], info["fbb_size"], np.nan_to_num(np.clip(c, 0, 1)))
        fh().fhash_compute_grads(model, to_dev(c), to_dev(tgt))
        P0, M0, V0 = (read(model, w, 0, n).astype(np.float64) for w in (0, 2, 3))
        g = read(model, 1, 0, n).astype(np.float64)  # the same gradient feeds both sides
        fh().fhash_apply_adam(model, HP32)
        P, M, V = adam.step(P0, g, M0, V0, k, lr, b1, b2, eps)
        got_p, got_m, got_v = (read(model, w, 0, n) for w in (0, 2, 3))
        assert (read(model, 1, 0, n) == 0).all()
        sm = b1 * np.abs(M0) + (1 - b1) * np.abs(g)
        sv = b2 * V0 + (1 - b2) * g * g
        assert (np.abs(got_m - M) <= 1e-6 * sm + 1e-30).all(), k
        assert (np.abs(got_v - V) <= 1e-6 * sv + 1e-38).all(), k
        assert (np.abs(got_p - P) <= 1e-6 * lr + 3e-7 * np.abs(P)).all(), k


def test_training_curve_parity(small):
    info = small["info"]
    model = build(W1, mask=small["mask"], seed=9)
    n_t = info["n_table_params"]
    table = read(model, 0, 0, n_t)
    p = read(model, 0, n_t, info["n_mlp_params"])
    om = train.Model(info["res"], info["F"], info["mlp_dims"], table.reshape(-1, info["F"]), p)
    losses_g, losses_o = [], []
    for k in range(50):
        c = synth.coords(100 + k, W1["batch"])
        tgt = synth.sample(small["field"], info["fbb_lo"], info["fbb_size"], c)
        loss = np.zeros(1, np.float64)
        fh().fhash_train_step(model, to_dev(c), to_dev(tgt), W1["adam"], loss)
        losses_g.append(loss[0])
        losses_o.append(train.train_step(om, c, tgt, *HP32))
    lg, lo = np.array(losses_g), np.array(losses_o)
    assert lo[-1] < 0.5 * lo[0]
    assert (np.abs(lg - lo) <= 1e-4 * lo).all(), np.max(np.abs(lg - lo) / lo)


def test_params_and_level_info_entry_points(small):
    info, model = small["info"], small["model"]
    res, base, fbb = fh().fhash_level_info(model)
    assert res == info["res"] and base == info["base"] and fbb == info["fbb_lo"] + info["fbb_size"]
    table, p = _random_params(info, seed=17)
    t0 = np.empty_like(table)
    p0 = np.empty_like(p)
    fh().fhash_get_params(model, t0, p0)
    fh().fhash_set_params(model, table, p)  # host buffers
    t1 = torch().empty(table.size, dtype=torch().float32, device="cuda")
    p1 = torch().empty(p.size, dtype=torch().float32, device="cuda")
    fh().fhash_get_params(model, t1, p1)  # device buffers
    torch().cuda.synchronize()
    assert np.array_equal(t1.cpu().numpy(), table) and np.array_equal(p1.cpu().numpy(), p)
    assert np.array_equal(read(model, fh().STATE_PARAM, 0, table.size), table)
    fh().fhash_set_params(model, t0, p0)  # restore the module fixture's parameters
