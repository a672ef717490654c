"""Parity at the full size of the bench workload (advect-256^3x64: 16 levels up to 256^3 x 64, F=2,
3.56e9 parameters, batch 2^18), in the launch configuration bench.py times.

The oracle computes only what it can afford, from its own inputs: initial tables and MLP from its own
SplitMix64 (the library's documented initialisation), the seeded field and mask from synth.  Checked:
- the Feature Bounding Box and two time steps of the occupancy grid, bit-exact;
- forward outputs on 4096 sampled points, within 1e-4 x max(|o|, RMS(o));
- the full-batch loss of one training step, within 1e-5 relative;
- MLP gradients and the table gradient on 20000 sampled touched rows, within 1e-4 x the sum of
  the magnitudes of their terms; 2000 sampled untouched rows exactly zero;
- the Adam update of the same rows, fed the same gradient, within 1e-6 x lr + 3e-7 x |p|;
- the bf16 precision form at this size (brick rows, tables U(-0.5, 0.5)): forward on 4096 points
  against the bf16 emulation, and the loss, MLP gradients and 20000 sampled table-row gradients of
  one full-batch step against the emulation's backward (bounds of the small-workload bf16 tests);
- masked compact tables at this size: the active bit of 20000 sampled vertices on each of four levels
  against the definition (a box query over the dilated mask), level bases equal to the running
  popcount of the bits, and the rows of all corners of 4096 footprint points active and equal to the
  level base plus the rank of their Eq. 9 row among the active ones.
"""
import numpy as np
import pytest

import synth
from synth import workloads
from oracle import adam, encode, index, masked, mlp, precision, rng, schedule, train

from _util import fh, to_dev, torch

pytestmark = pytest.mark.gpu
W = workloads.LARGE
SEED = 3
HP32 = tuple(float(np.float32(x)) for x in W["adam"])
R32 = float(np.float32(W["init_range"]))


@pytest.fixture(scope="module")
def large():
    f, m = workloads.make_field_and_mask(W)
    nx, ny, nz, nt = W["dims"]
    model = fh().fhash_build(nx, ny, nz, nt, mask=m, schedule=fh().make_schedule(**W["schedule"]), F=W["F"],
                             mlp_hidden_layers=W["hidden"], mlp_width=W["width"], seed=SEED, init_range=W["init_range"])
    return dict(field=f, mask=m, model=model, info=fh().fhash_get_info(model))


def test_fullsize_build(large):
    info = large["info"]
    lv = schedule.geometric_schedule(W["schedule"]["r0"], W["schedule"]["r1"], W["schedule"]["n_levels"])
    b, total = schedule.bases(lv)
    assert info["res"] == lv and info["base"] == b and info["total_rows"] == total == 1778559385
    d = index.dilate(large["mask"])
    lo, size = index.fbb(d)
    assert info["fbb_lo"] == lo and info["fbb_size"] == size
    occ = index.occupancy(d, lo, size)
    for t in (0, 37):
        got = np.empty((size[2], size[1], size[0]), np.uint8)
        fh().fhash_read_occupancy(large["model"], t, got)
        assert np.array_equal(got.astype(bool), occ[t]), t


def test_fullsize_forward_train_step(large):
    _forward_train_step(large["model"], large["info"], large["field"], "linear")


def test_fullsize_brick_forward_train_step(large):
    """The same checks on a model in the brick row layout (the bench's default layout)."""
    nx, ny, nz, nt = W["dims"]
    model = fh().fhash_build(nx, ny, nz, nt, mask=large["mask"], schedule=fh().make_schedule(**W["schedule"]),
                             F=W["F"], mlp_hidden_layers=W["hidden"], mlp_width=W["width"], seed=SEED,
                             init_range=W["init_range"], layout=fh().LAYOUT_BRICK)
    _forward_train_step(model, fh().fhash_get_info(model), large["field"], "brick")
    del model


def _forward_train_step(model, info, field, layout):
    lv, b, F, dims = info["res"], info["base"], info["F"], info["mlp_dims"]
    table = rng.InitTable(SEED, F, R32)
    p = rng.init_mlp(SEED, dims)
    n_t = info["n_table_params"]

    # forward on sampled points
    c = synth.coords(31, 4096)
    out = torch().empty(c.shape[0], dtype=torch().float32, device="cuda")
    fh().fhash_forward(model, to_dev(c), out)
    ref = mlp.forward(p, dims, encode.encode(lv, b, c, table, layout))[0]
    tol = 1e-4 * np.maximum(np.abs(ref), np.sqrt(np.mean(ref ** 2)))
    assert (np.abs(out.cpu().numpy() - ref) <= tol).all()

    # one full training step at the bench's batch
    B = W["batch"]
    c = synth.coords(10_000, B)
    tgt = synth.sample(field, info["fbb_lo"], info["fbb_size"], c)
    loss = np.zeros(1, np.float64)
    fh().fhash_compute_grads(model, to_dev(c), to_dev(tgt), loss)
    L, _, g_mlp, (rows, g_rows) = train.loss_and_grads(lv, b, F, dims, table, p, c, tgt, layout)
    assert abs(loss[0] - L) <= 1e-5 * L, (loss[0], L)

    g_dev = np.empty(info["n_mlp_params"], np.float32)
    fh().fhash_read_state(model, fh().STATE_GRAD, n_t, g_dev)
    enc = encode.encode(lv, b, c, table, layout)
    y, a, z = mlp.forward(p, dims, enc)
    _, gy = mlp.mse(y, tgt)
    abs_mlp, abs_denc = mlp.backward(np.abs(p), dims, [np.abs(x) for x in a], [np.where(x > 0, 1.0, -1.0) for x in z],
                                     np.abs(gy))
    assert (np.abs(g_dev - g_mlp) <= 1e-4 * abs_mlp + 1e-12).all()

    r_abs, g_abs = encode.encode_backward(lv, b, c, abs_denc, F, layout)
    assert np.array_equal(r_abs, rows)
    pick = np.random.default_rng(0).choice(rows.size, 20000, replace=False)
    touched = rows[pick]
    gt = np.empty((touched.size, F), np.float32)
    one = np.empty(F, np.float32)
    for k, r in enumerate(touched):
        fh().fhash_read_state(model, fh().STATE_GRAD, int(r) * F, one)
        gt[k] = one
    assert (np.abs(gt - g_rows[pick]) <= 1e-4 * g_abs[pick] + 1e-12).all()
    cand = np.random.default_rng(1).integers(0, info["total_rows"], 40000)
    untouched = cand[~np.isin(cand, rows)][:2000]
    for r in untouched:
        fh().fhash_read_state(model, fh().STATE_GRAD, int(r) * F, one)
        assert (one == 0).all()

    # Adam on the same rows, same gradient
    fh().fhash_apply_adam(model, HP32)
    p0 = table[touched].astype(np.float64)
    p1, _, _ = adam.step(p0, gt.astype(np.float64), np.zeros_like(p0), np.zeros_like(p0), 1, *HP32)
    got = np.empty_like(gt)
    for k, r in enumerate(touched):
        fh().fhash_read_state(model, fh().STATE_PARAM, int(r) * F, one)
        got[k] = one
    assert (np.abs(got - p1) <= 1e-6 * HP32[0] + 3e-7 * np.abs(p1)).all()
    fh().fhash_check(model)


def test_fullsize_bf16_forward_and_gradients(large):
    """The precision form at the bench size, in the launch configuration the bench uses (brick rows,
    persistent tensor-core forward, tensor-core weight gradients).  Forward: every output within
    4e-3 x max(|o|, RMS(o)) of the bf16 emulation and 99% within 5e-4.  One step at batch 2^18: loss
    within 2e-3 relative, MLP gradients and the gradients of 20000 sampled touched table rows within
    3e-3 x the sum of the magnitudes of their terms."""
    nx, ny, nz, nt = W["dims"]
    seed, r = 29, float(np.float32(0.5))
    model = fh().fhash_build(nx, ny, nz, nt, mask=large["mask"], schedule=fh().make_schedule(**W["schedule"]),
                             F=W["F"], dtype=fh().BF16, mlp_hidden_layers=W["hidden"], mlp_width=W["width"],
                             seed=seed, init_range=0.5, layout=fh().LAYOUT_BRICK)
    info = fh().fhash_get_info(model)
    lv, b, F, dims = info["res"], info["base"], info["F"], info["mlp_dims"]
    table = rng.InitTable(seed, F, r)
    p = rng.init_mlp(seed, dims).astype(np.float64)

    c = synth.coords(41, 4096)
    c[:3] = [[0, 0, 0, 0], [1, 1, 1, 1], [np.nan, 2.0, -1.0, 0.5]]
    out = torch().empty(c.shape[0], dtype=torch().float32, device="cuda")
    fh().fhash_forward(model, to_dev(c), out)
    ref = precision.forward_bf16(lv, b, table, p, dims, c, "brick")
    err = np.abs(out.cpu().numpy() - ref) / np.maximum(np.abs(ref), np.sqrt(np.mean(ref ** 2)))
    assert err.max() <= 4e-3 and np.mean(err <= 5e-4) >= 0.99, (err.max(), np.mean(err <= 5e-4))

    B = W["batch"]
    c = synth.coords(12_000, B)
    tgt = synth.sample(large["field"], info["fbb_lo"], info["fbb_size"], c)
    loss = np.zeros(1, np.float64)
    fh().fhash_compute_grads(model, to_dev(c), to_dev(tgt), loss)
    L, g_mlp, g_abs, d_enc, d_abs = precision.grads_bf16(lv, b, table, p, dims, c, tgt.astype(np.float64), "brick")
    assert abs(loss[0] - L) <= 2e-3 * L, (loss[0], L)
    g_dev = np.empty(info["n_mlp_params"], np.float32)
    fh().fhash_read_state(model, fh().STATE_GRAD, info["n_table_params"], g_dev)
    assert (np.abs(g_dev - g_mlp) <= 3e-3 * g_abs + 1e-9).all(), np.max(np.abs(g_dev - g_mlp) / (g_abs + 1e-9))
    rows, g_rows = encode.encode_backward(lv, b, c, d_enc, F, "brick")
    r_abs, g_rows_abs = encode.encode_backward(lv, b, c, d_abs, F, "brick")
    assert np.array_equal(rows, r_abs)
    pick = np.random.default_rng(3).choice(rows.size, 20000, replace=False)
    got = np.empty((pick.size, F), np.float32)
    one = np.empty(F, np.float32)
    for k, rr in enumerate(rows[pick]):
        fh().fhash_read_state(model, fh().STATE_GRAD, int(rr) * F, one)
        got[k] = one
    assert (np.abs(got - g_rows[pick]) <= 3e-3 * g_rows_abs[pick] + 1e-9).all()
    fh().fhash_check(model)
    del model


def test_fullsize_finite_differences(large):
    """Central differences of the full-batch loss (2^18 samples, the bench's launch configuration)
    against the GPU's analytic gradient on 48 touched table entries across the levels and 16 MLP
    parameters.  The loss is piecewise quadratic in each parameter, so the quotient is exact up to
    float32 rounding unless a ReLU flips inside +-h: a point whose quotients at h and h/10 disagree
    by more than 5% is dropped (at least 48 of the 64 must be checked; at h/10 a table entry moves the
    outputs of the few samples that see it by about 1e-5, so float32 rounding alone gives about 1%).  h = 1e-2 for table entries
    (only a few samples see them, so a larger step keeps float32 rounding of the outputs small) and
    1e-3 for MLP parameters.  Bound: 2% relative."""
    info, model = large["info"], large["model"]
    lv, b, F = info["res"], info["base"], info["F"]
    n_t = info["n_table_params"]
    c = synth.coords(20_000, W["batch"])
    tgt = synth.sample(large["field"], info["fbb_lo"], info["fbb_size"], c)
    dc, dt = to_dev(c), to_dev(tgt)
    loss = np.zeros(1, np.float64)
    g = np.zeros(1, np.float32)
    # a clean gradient: the previous test ended with an Adam step, which clears the buffer
    fh().fhash_compute_grads(model, dc, dt, loss)
    pick = np.random.default_rng(5)
    params = []
    for level in (0, 3, 6, 9, 12, 15, 15, 15):
        rows, _ = encode.level_corners(c[:64], lv[level], b[level])
        for r in pick.choice(rows.ravel(), 6, replace=False):
            params.append(int(r) * F + int(pick.integers(0, F)))
    params += [n_t + int(k) for k in pick.choice(info["n_mlp_params"], 16, replace=False)]
    grads = []
    for off in params:
        fh().fhash_read_state(model, fh().STATE_GRAD, off, g)
        grads.append(float(g[0]))

    def L(off, v):
        fh().fhash_write_state(model, fh().STATE_PARAM, off, np.array([v], np.float32))
        fh().fhash_compute_grads(model, dc, dt, loss)
        return loss[0]

    p = np.zeros(1, np.float32)
    checked = 0
    for off, gr in zip(params, grads):
        fh().fhash_read_state(model, fh().STATE_PARAM, off, p)
        v0 = float(p[0])
        fd = []
        for h in ((1e-2, 1e-3) if off < n_t else (1e-3, 1e-4)):
            vp, vm = float(np.float32(v0 + h)), float(np.float32(v0 - h))
            fd.append((L(off, vp) - L(off, vm)) / (vp - vm))
        fh().fhash_write_state(model, fh().STATE_PARAM, off, np.array([v0], np.float32))
        if abs(fd[0] - fd[1]) > 5e-2 * max(abs(fd[0]), 1e-12):
            continue  # a ReLU kink inside +-h
        # absolute floor: the float32 rounding of the outputs of the few samples that see a table entry
        # moves the loss by about 5e-14 per sample, 2.5e-12 in the quotient at h = 1e-2
        assert abs(fd[0] - gr) <= 2e-2 * abs(fd[0]) + (4e-12 if off < n_t else 1e-12), (off, fd, gr)
        checked += 1
    assert checked >= 48, checked
    fh().fhash_check(model)


def test_fullsize_render_and_decode(large):
    """The ARM renderer and the time-slice decode on a model of the full bench shape (16 levels to
    256^3 x 64, F=2, MLP 2x64, 3.56e9 parameters), in the launch configuration the serving leg uses:
    a 32 x 24 image through fhash_render and a 256^3 decode at fractional t, against the oracle on
    the same parameters (the library's initial tables, U(-0.5, 0.5), and MLP from its documented
    SplitMix64 streams; output bias 0.45).  Tolerances as on the small workload: composited sample
    counts equal on >= 99.9% of pixels, matched pixels within 2e-4, PSNR >= 60 dB; decode values on
    3000 sampled grid points within 1e-4 x max(|o|, RMS(o))."""
    from oracle import render
    nx, ny, nz, nt = W["dims"]
    seed = 17
    model = fh().fhash_build(nx, ny, nz, nt, mask=large["mask"], schedule=fh().make_schedule(**W["schedule"]),
                             F=W["F"], mlp_hidden_layers=W["hidden"], mlp_width=W["width"], seed=seed, init_range=0.5)
    info = fh().fhash_get_info(model)
    lv, b, F, dims = info["res"], info["base"], info["F"], info["mlp_dims"]
    p = rng.init_mlp(seed, dims).astype(np.float64)
    p[-1] = 0.45
    fh().fhash_write_state(model, fh().STATE_PARAM, info["n_table_params"] + info["n_mlp_params"] - 1,
                           np.array([0.45], np.float32))
    table = rng.InitTable(seed, F, float(np.float32(0.5)))
    ev = render.model_eval_fn(lv, b, table, p, dims)

    if "occ" not in large:
        d = index.dilate(large["mask"])
        large["occ"] = index.occupancy(d, info["fbb_lo"], info["fbb_size"])
    w, h, t = 32, 24, np.float32(0.41)
    cam = synth.camera(synth.sphere_eye(8, 2), w, h)
    tf = synth.transfer_function(0.5)
    rgba = torch().empty((h, w, 4), dtype=torch().float32, device="cuda")
    cnt = torch().empty((h, w), dtype=torch().int32, device="cuda")
    fh().fhash_render(model, cam, float(t), to_dev(tf), w, h, rgba, cnt)
    img, cnt = rgba.cpu().numpy(), cnt.cpu().numpy()
    ref, rcnt = render.render(ev, cam, w, h, info["fbb_size"], large["occ"], t, tf)
    same = cnt == rcnt
    assert rcnt.sum() > 0 and same.mean() >= 0.999, (same.mean(), int((~same).sum()))
    assert np.abs(img[same] - ref[same]).max() <= 2e-4
    mse = np.mean((img - ref) ** 2)
    assert mse == 0 or 10 * np.log10(1.0 / mse) >= 60

    up, tq = 1, np.float32(0.37)
    ddims = fh().fhash_decode_dims(model, up)
    out = torch().empty((ddims[2], ddims[1], ddims[0]), dtype=torch().float32, device="cuda")
    fh().fhash_decode(model, float(tq), up, out)
    got = out.cpu().numpy().ravel()
    u, shape = render.decode_coords(info["fbb_size"], up, tq)
    assert list(shape) == [ddims[2], ddims[1], ddims[0]]
    pick = np.random.default_rng(2).choice(u.shape[0], 3000, replace=False)
    refd = ev(u[pick])
    tol = 1e-4 * np.maximum(np.abs(refd), np.sqrt(np.mean(refd ** 2)))
    assert (np.abs(got[pick] - refd) <= tol).all(), np.abs(got[pick] - refd).max()
    fh().fhash_check(model)
    del model


def test_fullsize_masked_directory(large):
    nx, ny, nz, nt = W["dims"]
    model = fh().fhash_build(nx, ny, nz, nt, mask=large["mask"], schedule=fh().make_schedule(**W["schedule"]),
                             F=W["F"], mlp_hidden_layers=W["hidden"], mlp_width=W["width"], seed=SEED,
                             init_range=W["init_range"], layout=fh().LAYOUT_MASKED)
    info = fh().fhash_get_info(model)
    lv, base = info["res"], info["base"]
    d = index.dilate(large["mask"])
    lo, size = index.fbb(d)
    dil = masked.fbb_mask(d, lo, size)
    del d
    T, Sz, Sy, Sx = dil.shape
    pop = np.array([bin(i).count("1") for i in range(256)], np.uint8)
    rs = np.random.default_rng(12)
    bits, cum = [], []
    for l, R in enumerate(lv):
        nw = (int(np.prod(R, dtype=np.int64)) + 63) // 64
        b = np.empty(nw, np.uint64)
        fh().fhash_read_active(model, l, 0, b)
        per_word = pop[b.view(np.uint8)].reshape(-1, 8).sum(1, dtype=np.int64)
        bits.append(b)
        cum.append(np.concatenate([[0], np.cumsum(per_word)]))
        nxt = base[l + 1] if l + 1 < len(lv) else info["total_rows"]
        assert cum[l][-1] == nxt - base[l], l
    for l in (0, 8, 12, len(lv) - 1):
        Rx, Ry, Rz, Rt = lv[l]
        ranges = [np.array([masked.vertex_range(v, S, R) for v in range(S)]) for S, R in ((Sx, Rx), (Sy, Ry), (Sz, Rz))]
        ranges.append(np.array([masked.time_range(k, T, Rt) for k in range(T)]))
        # a box query reads about prod(S/R + 3) voxels: coarse levels get fewer samples
        box = np.prod([S / R + 3 for S, R in ((Sx, Rx), (Sy, Ry), (Sz, Rz), (T, Rt))])
        for _ in range(int(min(20000, max(20, 4e7 / box)))):
            X = [int(rs.integers(0, r)) for r in (Rx, Ry, Rz, Rt)]
            vs = [np.flatnonzero((rg[:, 0] <= x) & (x <= rg[:, 1])) for rg, x in zip(ranges, X)]
            want = bool(dil[np.ix_(vs[3], vs[2], vs[1], vs[0])].any()) if all(v.size for v in vs) else False
            r = int(encode.fhash(X[3], X[0], X[1], X[2], lv[l]))
            got = bool((int(bits[l][r >> 6]) >> (r & 63)) & 1)
            assert got == want, (l, X)
    # footprint points: random occupied voxels, offsets inside their footprints
    pts = []
    while sum(len(p) for p in pts) < 4096:
        v = np.stack([rs.integers(0, n, 100000) for n in (T, Sz, Sy, Sx)], 1)
        pts.append(v[dil[v[:, 0], v[:, 1], v[:, 2], v[:, 3]]])
    v = np.concatenate(pts)[:4096]
    u = np.empty((4096, 4))
    for a, (col, S) in enumerate(((3, Sx), (2, Sy), (1, Sz))):
        u[:, a] = (v[:, col] + rs.uniform(-0.5, 0.5, 4096)) / (S - 1)
    u[:, 3] = (v[:, 0] + rs.uniform(-1.0, 1.0, 4096)) / (T - 1)
    u = np.clip(u, 0, 1).astype(np.float32)
    rows = torch().empty((4096, len(lv), 16), dtype=torch().int64, device="cuda")
    fh().fhash_lookup(model, to_dev(u), rows)
    rows = rows.cpu().numpy().view(np.uint64)
    for l, R in enumerate(lv):
        r_lin, _ = encode.level_corners(u, R, 0)
        w, i = r_lin >> 6, (r_lin & 63).astype(np.uint64)
        word = bits[l][w]
        assert ((word >> i) & np.uint64(1) == 1).all(), l
        below = word & ((np.uint64(1) << i) - np.uint64(1))
        rank = cum[l][w] + pop[below.view(np.uint8).reshape(below.shape + (8,))].sum(-1, dtype=np.int64)
        assert np.array_equal(rows[:, l, :], (base[l] + rank).astype(np.uint64)), l
    fh().fhash_check(model)
    del model
