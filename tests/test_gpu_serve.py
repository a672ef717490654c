"""GPU tests of the continuous-batching serving loop (include/fhash_serve.h).

Each request's result in a mix - renders of different sizes, cameras and fractional times, and
decodes at different upsampling and times, over an FP32, a bf16 and an FP32 masked-table model
(FHASH_LAYOUT_MASKED), interleaved across many
ticks of a small packed buffer - must be bit-identical to the same request run alone through
fhash_render / fhash_decode (per-sample arithmetic does not depend on batch position, and the image
does not depend on the ARM pace).  Served results are also checked against the oracle directly:
renders and decodes of the float32 model against oracle/render.py with the tolerances of the
standalone render and decode tests, the masked model against the oracle's masked layout, and the bf16
model against oracle/render.py evaluated through the bf16 emulation (oracle/precision.py).  Admission
follows the memory budget; cancellation releases memory.
"""
import numpy as np
import pytest

import synth
from synth import workloads
from oracle import encode, index, masked, mlp, precision, render

from _util import build, fh, set_params, to_dev, torch

pytestmark = pytest.mark.gpu
W1 = workloads.SMALL


@pytest.fixture(scope="module")
def models():
    f, m = workloads.make_field_and_mask(W1)
    out = []
    nx, ny, nz, nt = W1["dims"]
    for dt in (fh().FP32, fh().BF16, "masked"):
        if dt == "masked":
            model = fh().fhash_build(nx, ny, nz, nt, mask=m, schedule=fh().make_schedule(**W1["schedule"]), F=W1["F"],
                                     mlp_hidden_layers=W1["hidden"], mlp_width=W1["width"], seed=17,
                                     init_range=W1["init_range"], layout=fh().LAYOUT_MASKED)
        else:
            model = build(W1, mask=m, dtype=dt, seed=17)
        info = fh().fhash_get_info(model)
        table = synth.uniform(51, 50, info["n_table_params"], -0.6, 0.6)
        p = synth.init_mlp(51, info["mlp_dims"])
        p[-1] = 0.45
        set_params(model, table, p)
        out.append(model)
    return out


def _alone_render(model, cam, t, w, h, tf):
    rgba = torch().empty((h, w, 4), dtype=torch().float32, device="cuda")
    cnt = torch().empty((h, w), dtype=torch().int32, device="cuda")
    fh().fhash_render(model, cam, t, tf, w, h, rgba, cnt)
    return rgba.cpu().numpy(), cnt.cpu().numpy()


def _alone_decode(model, t, up):
    d = fh().fhash_decode_dims(model, up)
    out = torch().empty((d[2], d[1], d[0]), dtype=torch().float32, device="cuda")
    fh().fhash_decode(model, t, up, out)
    return out.cpu().numpy()


def _run(srv, ids, max_ticks=10000):
    for _ in range(max_ticks):
        if all(fh().fhash_server_poll(srv, i)[0] in (fh().REQ_DONE, fh().REQ_CANCELLED) for i in ids):
            return
        fh().fhash_server_tick(srv)
    raise AssertionError("requests did not finish")


def test_mix_equals_alone(models):
    tf = to_dev(synth.transfer_function(0.5))
    srv = fh().fhash_server_create(models, budget_bytes=1 << 30, max_live=8, tick_samples=8192)
    specs = [("r", 0, 0.0, 40, 30, 0), ("d", 1, 0.37, 2), ("r", 1, 0.55, 64, 48, 1), ("d", 0, 1.0, 1),
             ("r", 2, 0.45, 48, 36, 4), ("r", 0, 0.9, 24, 24, 2), ("r", 1, 0.2, 72, 40, 3), ("d", 2, 0.6, 1),
             ("d", 0, 0.5, 2)]
    subs = []
    for sp in specs:
        if sp[0] == "r":
            _, mi, t, w, h, v = sp
            cam = synth.camera(synth.sphere_eye(3, v), w, h)
            out = torch().empty((h, w, 4), dtype=torch().float32, device="cuda")
            cnt = torch().empty((h, w), dtype=torch().int32, device="cuda")
            rid = fh().fhash_server_submit(srv, fh().make_request(fh().REQ_RENDER, mi, t, cam, w, h, 64, tf, out=out,
                                                                  counts=cnt))
            subs.append((sp, rid, out, cnt, cam))
        else:
            _, mi, t, up = sp
            d = fh().fhash_decode_dims(models[mi], up)
            out = torch().empty((d[2], d[1], d[0]), dtype=torch().float32, device="cuda")
            rid = fh().fhash_server_submit(srv, fh().make_request(fh().REQ_DECODE, mi, t, upsample=up, out=out))
            subs.append((sp, rid, out, None, None))
        fh().fhash_server_tick(srv)  # requests arrive while others are on the GPU
    _run(srv, [s[1] for s in subs])
    st = fh().fhash_server_get_stats(srv)
    assert st["ticks"] > len(specs) and st["pool_used"] == 0 and st["live"] == 0
    # launches per tick do not grow with the live requests: one generation and one compositing launch
    # (plus one ray set-up launch on ticks that admit renders) and one graph per model with samples
    assert st["packed_launches"] <= 3 * st["ticks"] and st["model_launches"] <= 3 * st["ticks"]
    for sp, rid, out, cnt, cam in subs:
        state, lat = fh().fhash_server_poll(srv, rid)
        assert state == fh().REQ_DONE and lat >= 0
        if sp[0] == "r":
            a, c = _alone_render(models[sp[1]], cam, sp[2], sp[3], sp[4], tf)
            assert np.array_equal(out.cpu().numpy(), a) and np.array_equal(cnt.cpu().numpy(), c), sp
        else:
            assert np.array_equal(out.cpu().numpy(), _alone_decode(models[sp[1]], sp[2], sp[3])), sp


def test_budget_admission_and_cancel(models):
    tf = to_dev(synth.transfer_function(0.5))
    w, h = 64, 64
    probe = fh().fhash_server_create([models[0]], budget_bytes=1 << 28, max_live=8, tick_samples=4096)
    fixed = (1 << 28) - fh().fhash_server_get_stats(probe)["pool_bytes"]  # models + packed buffers
    need = 4096 * 48 + 3 * 4096 * 4  # one 64x64 render: ray states + two alive lists + counts
    del probe
    srv = fh().fhash_server_create([models[0]], budget_bytes=fixed + need * 3 // 2, max_live=8, tick_samples=4096)
    outs, ids = [], []
    for v in range(3):
        out = torch().empty((h, w, 4), dtype=torch().float32, device="cuda")
        cam = synth.camera(synth.sphere_eye(4, v), w, h)
        ids.append(fh().fhash_server_submit(srv, fh().make_request(fh().REQ_RENDER, 0, 0.3, cam, w, h, 64, tf, out=out)))
        outs.append((out, cam))
    fh().fhash_server_tick(srv)
    states = [fh().fhash_server_poll(srv, i)[0] for i in ids]
    assert states.count(fh().REQ_LIVE) + states.count(fh().REQ_DONE) == 1 and states.count(fh().REQ_QUEUED) == 2
    fh().fhash_server_cancel(srv, ids[2])
    _run(srv, ids)
    assert fh().fhash_server_poll(srv, ids[2])[0] == fh().REQ_CANCELLED
    for i, (out, cam) in zip(ids[:2], outs[:2]):
        assert fh().fhash_server_poll(srv, i)[0] == fh().REQ_DONE
        a, _ = _alone_render(models[0], cam, 0.3, w, h, tf)
        assert np.array_equal(out.cpu().numpy(), a)
    assert fh().fhash_server_get_stats(srv)["pool_used"] == 0


def test_invalid_requests(models):
    srv = fh().fhash_server_create([models[0]], budget_bytes=1 << 28, max_live=2, tick_samples=1024)
    out = torch().empty(16, device="cuda")
    tf = to_dev(synth.transfer_function(0.5))
    bad = [fh().make_request(fh().REQ_RENDER, 5, 0.1, synth.camera([2, 0, 0], 4, 4), 4, 4, 64, tf, out=out),
           fh().make_request(fh().REQ_RENDER, 0, 1.5, synth.camera([2, 0, 0], 4, 4), 4, 4, 64, tf, out=out),
           fh().make_request(fh().REQ_RENDER, 0, 0.1, synth.camera([2, 0, 0], 64, 64), 64, 64, 64, tf, out=out),
           fh().make_request(fh().REQ_DECODE, 0, 0.1, upsample=9, out=out), fh().make_request(7, 0, 0.1, out=out)]
    for r in bad:
        with pytest.raises(fh().FHashError) as e:
            fh().fhash_server_submit(srv, r)
        assert e.value.status == 1


def _oracle_eval(model, kind, m):
    """The oracle's float64 evaluation of a served model: (function of u [n][4], FBB size, occupancy)."""
    info = fh().fhash_get_info(model)
    table = synth.uniform(51, 50, info["n_table_params"], -0.6, 0.6)
    p = synth.init_mlp(51, info["mlp_dims"])
    p[-1] = 0.45
    d = index.dilate(m)
    occ = index.occupancy(d, info["fbb_lo"], info["fbb_size"])
    T = table.reshape(-1, info["F"])
    res, dims = info["res"], info["mlp_dims"]
    if kind == "bf16":
        return (lambda u: precision.forward_bf16(res, info["base"], T, p.astype(np.float64), dims, u)), info, occ
    if kind == "masked":
        lo, size = index.fbb(d)
        lay = masked.MaskedLayout(res, masked.fbb_mask(d, lo, size))
        assert list(info["base"][:len(res)]) == lay.bases
        return (lambda u: mlp.forward(p.astype(np.float64), dims,
                                      encode.encode(res, lay.bases, u, T.astype(np.float64), lay))[0]), info, occ
    return render.model_eval_fn(res, info["base"], T.astype(np.float64), p.astype(np.float64), dims), info, occ


def test_served_results_match_oracle(models, capsys):
    """Renders and decodes of all three models, served together, against the oracle.  float32 and masked:
    composited-sample counts equal on >= 99.9% of pixels, matched pixels within 2e-4, image PSNR >= 60 dB;
    decodes within 1e-4 x max(|o|, RMS).  bf16 against the bf16 emulation (float32 accumulation against
    float64, and the rare layer input on a bf16 rounding tie): counts equal on >= 99.5% of pixels, 99% of
    matched pixels within 2e-4, image PSNR >= 50 dB; decodes within 4e-3 x max(|o|, RMS), 99% within 5e-4."""
    f, m = workloads.make_field_and_mask(W1)
    tf_host = synth.transfer_function(0.5)
    tf = to_dev(tf_host)
    srv = fh().fhash_server_create(models, budget_bytes=1 << 30, max_live=8, tick_samples=4096)
    subs = []
    for mi in range(3):
        w, h, t = 48, 36, 0.45 + 0.1 * mi
        cam = synth.camera(synth.sphere_eye(6, mi), w, h)
        out = torch().empty((h, w, 4), dtype=torch().float32, device="cuda")
        cnt = torch().empty((h, w), dtype=torch().int32, device="cuda")
        rid = fh().fhash_server_submit(srv, fh().make_request(fh().REQ_RENDER, mi, t, cam, w, h, 64, tf, out=out,
                                                              counts=cnt))
        subs.append(("r", mi, rid, out, cnt, (cam, w, h, t)))
        d = fh().fhash_decode_dims(models[mi], 2)
        dout = torch().empty((d[2], d[1], d[0]), dtype=torch().float32, device="cuda")
        rid = fh().fhash_server_submit(srv, fh().make_request(fh().REQ_DECODE, mi, 0.37, upsample=2, out=dout))
        subs.append(("d", mi, rid, dout, None, (0.37, 2)))
        fh().fhash_server_tick(srv)
    _run(srv, [s[2] for s in subs])
    kinds = ["fp32", "bf16", "masked"]
    for kind, mi, rid, out, cnt, arg in subs:
        assert fh().fhash_server_poll(srv, rid)[0] == fh().REQ_DONE
        ev, info, occ = _oracle_eval(models[mi], kinds[mi], m)
        name = kinds[mi]
        if kind == "r":
            cam, w, h, t = arg
            img, c = out.cpu().numpy(), cnt.cpu().numpy()
            ref, rc = render.render(ev, cam, w, h, info["fbb_size"], occ, np.float32(t), tf_host)
            same = c == rc
            assert rc.sum() > 0
            err = np.abs(img[same] - ref[same]).max(axis=-1)
            mse = np.mean((img - ref) ** 2)
            psnr = np.inf if mse == 0 else 10 * np.log10(1.0 / mse)
            with capsys.disabled():
                print("\nserved render %s: counts equal %.5f, matched max err %.3g, PSNR %.1f dB"
                      % (name, same.mean(), err.max(), psnr))
            if name == "bf16":
                assert same.mean() >= 0.995 and np.mean(err <= 2e-4) >= 0.99 and psnr >= 50, name
            else:
                assert same.mean() >= 0.999 and err.max() <= 2e-4 and psnr >= 60, name
        else:
            t, up = arg
            u, shape = render.decode_coords(info["fbb_size"], up, np.float32(t))
            ref = ev(u).reshape(shape)
            got = out.cpu().numpy()
            e = np.abs(got - ref) / np.maximum(np.abs(ref), np.sqrt(np.mean(ref ** 2)))
            with capsys.disabled():
                print("served decode %s: max rel err %.3g" % (name, e.max()))
            if name == "bf16":
                assert e.max() <= 4e-3 and np.mean(e <= 5e-4) >= 0.99, name
            else:
                assert e.max() <= 1e-4, name
