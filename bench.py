#!/usr/bin/env python
"""Benchmark of the F-Hash training step on one GB300 (replicas over N GPUs).

One step = one full pass of the training hot path over one batch of 2^18 synthetic samples of the
256^3 x 64 workload: encode (16 levels, F=2) -> MLP 2x64 forward -> MSE -> MLP backward -> table
scatter-add -> dense Adam over all 3.56e9 parameters.  Inputs are resident in HBM before the timed
region; the 57 GB of training state streamed every step is far larger than L2, so no extra flush is
needed.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload large|small]
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")  # the oracle legs are timed single-threaded

import argparse
import json
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "train samples/s (enc+MLP fwd+bwd); render p50/p99 ms; BF16 vs FP32 @PSNR"
# DRAM traffic of k_adam from one ncu capture of the kernel on advect-128^3x32: 4.106 GB read + 3.323 GB written for 256,431,321
# parameters, 28.97 B/param, when 21% of the 4-parameter gradient groups were non-zero (algorithmic
# 28 + 4 x 0.21 = 28.84 B/param).  The written part depends on that fraction, so the capture does not
# scale to the full launch in proportion; the bench reports it as a small-case ratio instead.
ADAM_SMALL_CASE = {"workload": "advect-128^3x32", "bytes_per_param_measured": (4.106175e9 + 3.323173e9) / 256431321,
                   "bytes_per_param_algorithmic": 28.84, "grad_groups_touched": 0.2097}
ADAM_SMALL_CASE["ratio"] = ADAM_SMALL_CASE["bytes_per_param_measured"] / ADAM_SMALL_CASE["bytes_per_param_algorithmic"]


# DRAM traffic of k_defer_replay per caught-up group of 32 floats, from one ncu capture of the kernel on
# advect-128^3x32 after 100 aging steps: 0.7668 GB read + 0.5926 GB written, over the 1,473,749 groups per
# step that the same command's live phase loop reported (algorithmic: 896 B per group).
REPLAY_DRAM_BYTES_PER_GROUP = (0.766776832e9 + 0.59256832e9) / 1473749


def _layout(args):
    """Row layout of the tables: brick (4x4x4 bricks per time slice, a linearisation Section 3.2.3
    allows; the bench's default because it gathers faster) or linear (Eq. 9, the library's default)."""
    return {"linear": 0, "brick": 1}[getattr(args, "layout", "brick")]


def max_over_ranks(dist, x, device="cuda"):
    """The slowest rank's value, on every rank (x itself without a process group).  Replicas run the
    same work on their own GPU, so the job's time is the maximum over ranks."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def _touched_fraction(fh, model, info, coords, tgt, hp, n_deferred=0, chunk=1 << 28):
    """One more training step, untimed: the fraction of 4-parameter gradient groups that are non-zero
    before its Adam update, over the parameters Adam updates densely (all but the n_deferred parameters of
    the deferred levels, which end the table)."""
    import torch
    n = info["n_table_params"] + info["n_mlp_params"]
    lo = info["n_table_params"] - n_deferred
    lo -= lo % 8
    ranges = [(0, lo), (lo + n_deferred, n)] if n_deferred else [(0, n)]
    fh.fhash_compute_grads(model, coords, tgt)
    buf = torch.empty(min(chunk, n), dtype=torch.float32, device="cuda")
    hit = total = 0
    for a, b in ranges:
        b -= (b - a) % 4
        for off in range(a, b, chunk):
            k = min(chunk, b - off)
            fh.fhash_read_state(model, fh.STATE_GRAD, off, buf[:k])
            hit += int(buf[:k].view(-1, 4).ne(0).any(1).sum())
            total += k // 4
    fh.fhash_apply_adam(model, hp)
    torch.cuda.synchronize()
    return hit / max(1, total)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 9 for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def _workload(name):
    from synth import workloads
    return {"large": workloads.LARGE, "medium": workloads.MEDIUM, "small": workloads.SMALL}[name]


def _levels(w):
    from oracle import schedule
    s = w["schedule"]
    if s["mode"] == "geometric":
        return schedule.geometric_schedule(s["r0"], s["r1"], s["n_levels"])
    return [list(r) for r in s["res"]]


def _oracle_phases(w, n_sample, seed, adam_slice):
    """Seconds the oracle takes for encode -> MLP -> MSE -> backward -> scatter on n_sample samples and for
    dense Adam on adam_slice parameters (inputs made before the clock starts), and the step's parameter
    count."""
    import synth
    from oracle import adam, rng, schedule, train
    lv = _levels(w)
    b, rows = schedule.bases(lv)
    F = w["F"]
    dims = [len(lv) * F] + [w["width"]] * w["hidden"] + [1]
    n_params = rows * F + sum(dims[k] * dims[k + 1] + dims[k + 1] for k in range(len(dims) - 1))
    table = rng.InitTable(seed, F, w["init_range"])
    p = synth.init_mlp(seed, dims).astype(np.float64)
    c = synth.coords(1000 + seed, n_sample)
    tgt = synth.uniform(seed, 77, n_sample)
    t0 = time.perf_counter()
    train.loss_and_grads(lv, b, F, dims, table, p, c, tgt)
    t1 = time.perf_counter()
    z = np.zeros(adam_slice)
    P = synth.uniform(seed, 78, adam_slice).astype(np.float64)
    adam.step(P, P * 1e-3, z, z, 1)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, n_params


def oracle_step_sample(w, n_sample, seed=0, adam_slice=1 << 20):
    """Times the oracle on a bounded sample of one step: encode -> MLP -> MSE -> backward -> scatter for
    n_sample samples, plus dense Adam on a slice of adam_slice parameters.  Returns (seconds for the
    whole step extrapolated to the full batch and parameter count, description)."""
    a, b, n_params = _oracle_phases(w, n_sample, seed, adam_slice)
    full = a * w["batch"] / n_sample + b * n_params / adam_slice
    desc = ("oracle (numpy FP64, 1 thread): encode+MLP+MSE+backward+scatter on %d of %d samples and dense Adam on "
            "%d of %d parameters, extrapolated linearly to one full step" % (n_sample, w["batch"], adam_slice, n_params))
    return full, desc


def _oracle_worker(job):
    w, n_sample, seed, adam_slice = job
    return _oracle_phases(w, n_sample, seed, adam_slice)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The oracle on every host core: one single-threaded process per core (spawned, so safe after CUDA
    is initialised), each timing its own bounded sample at the same time.  A step's time is extrapolated
    from the slowest process: P processes handle P x n_sample samples and P x adam_slice parameters in
    that time."""

    def __init__(self, procs=None):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.procs = max(1, min(procs or host_cores(), 64))
        self.ex = cf.ProcessPoolExecutor(self.procs, mp_context=mp.get_context("spawn"))
        list(self.ex.map(_oracle_worker, [(_workload("small"), 64, i, 1024) for i in range(self.procs)],
                         timeout=300))  # start every process and import the oracle before timing

    def step(self, w, n_sample, adam_slice, seed=0, timeout=600):
        jobs = [(w, n_sample, seed * 1000 + i, adam_slice) for i in range(self.procs)]
        res = list(self.ex.map(_oracle_worker, jobs, timeout=timeout))
        a = max(r[0] for r in res)
        b = max(r[1] for r in res)
        n_params = res[0][2]
        full = a * w["batch"] / (n_sample * self.procs) + b * n_params / (adam_slice * self.procs)
        desc = ("oracle (numpy FP64) in %d single-threaded processes at once, one per host core, each on "
                "encode+MLP+MSE+backward+scatter of %d of %d samples and dense Adam on %d of %d parameters; the "
                "slowest process's times extrapolated linearly to one full step"
                % (self.procs, n_sample, w["batch"], adam_slice, n_params))
        return full, desc

    def close(self):
        self.ex.shutdown(wait=True, cancel_futures=True)


def run_reference(args):
    """Reference arm: the FP64 oracle as it stands, on the host cores, bounded samples per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = _workload(args.workload)
    n_sample = 4096
    cores = 1
    try:
        pool = OraclePool()
    except Exception as e:  # no process pool on this host: the single-process oracle
        print("oracle process pool unavailable (%s); timing one process" % e, file=sys.stderr)
        pool = None
    times = []
    desc = ""
    for k in range(args.warmup + args.steps):
        if pool is not None:
            t, desc = pool.step(w, n_sample, 1 << 20, seed=k)
        else:
            t, desc = oracle_step_sample(w, n_sample, seed=k)
        if k >= args.warmup:
            times.append(t)
    if pool is not None:
        cores = pool.procs
        pool.close()
    sec = float(np.mean(times))
    v = w["batch"] / sec
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "global_batch": w["batch"]},
        "extrapolated": True,
        "sample": "ms_per_step extrapolated from bounded samples: " + desc,
        "cpu_baseline": {"value": v, "unit": "samples/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def _copy_params(src, dst, n, chunk=1 << 28):
    """Trained float32 parameters of one model into another of the same shape, through the C ABI."""
    import torch
    import paper_2507_03836_gb300 as fh
    buf = torch.empty(min(n, chunk), dtype=torch.float32, device="cuda")
    for o in range(0, n, chunk):
        k = min(chunk, n - o)
        fh.fhash_read_state(src, fh.STATE_PARAM, o, buf[:k])
        fh.fhash_write_state(dst, fh.STATE_PARAM, o, buf[:k])
    torch.cuda.synchronize()


def precision_leg(args, w, model, info, field, mask, rank):
    """The trained model served in FP32 and in the precision form (bf16 + tensor cores, the same weights):
    PSNR and max error of both forms on 1M held-out points against the field."""
    import torch
    import synth
    import paper_2507_03836_gb300 as fh
    nx, ny, nz, nt = w["dims"]
    m16 = fh.fhash_build(nx, ny, nz, nt, mask=mask, schedule=fh.make_schedule(**w["schedule"]), F=w["F"],
                         dtype=fh.BF16, mlp_hidden_layers=w["hidden"], mlp_width=w["width"], seed=1 + rank,
                         init_range=w["init_range"], layout=_layout(args))
    n_all = info["n_table_params"] + info["n_mlp_params"]
    _copy_params(model, m16, n_all)

    # precision: the same trained weights served in both forms, on 1M held-out points
    held = synth.coords(777, 1 << 20)
    truth = synth.sample(field, info["fbb_lo"], info["fbb_size"], held).astype(np.float64)
    hd = torch.from_numpy(held).cuda()
    prec = {"held_out_points": int(held.shape[0]), "reference": "field sampled at the held-out points"}
    rngv = truth.max() - truth.min()
    for name, mm in (("fp32", model), ("bf16", m16)):
        o = torch.empty(held.shape[0], dtype=torch.float32, device="cuda")
        fh.fhash_forward(mm, hd, o)
        pred = o.cpu().numpy().astype(np.float64)
        mse = np.mean((pred - truth) ** 2)
        prec["psnr_" + name] = float(10 * np.log10(rngv ** 2 / mse))
        prec["max_abs_err_" + name] = float(np.abs(pred - truth).max())
    prec["psnr_drop_db"] = prec["psnr_fp32"] - prec["psnr_bf16"]

    del m16
    return prec


def _build(w, dtype, seed, mask, layout=0):
    import paper_2507_03836_gb300 as fh
    nx, ny, nz, nt = w["dims"]
    m = fh.fhash_build(nx, ny, nz, nt, mask=mask, schedule=fh.make_schedule(**w["schedule"]), F=w["F"], dtype=dtype,
                       mlp_hidden_layers=w["hidden"], mlp_width=w["width"], seed=seed, init_range=w["init_range"],
                       layout=layout)
    return m, fh.fhash_get_info(m)


def _batches(w, info, field, k, seed):
    import torch
    import synth
    out = []
    for i in range(k):
        c = synth.coords(seed + i, w["batch"])
        out.append((torch.from_numpy(c).cuda(), torch.from_numpy(synth.sample(field, info["fbb_lo"], info["fbb_size"], c)).cuda()))
    return out


def _train(model, batches, hp, warmup=3):
    """Trains on the batches; returns ms per step over all but the first `warmup` (CUDA events)."""
    import torch
    import paper_2507_03836_gb300 as fh
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i, (c, t) in enumerate(batches):
        if i == warmup:
            torch.cuda.synchronize()
            e0.record(st)
        fh.fhash_train_step(model, c, t, hp)
    e1.record(st)
    torch.cuda.synchronize()
    fh.fhash_check(model)
    return e0.elapsed_time(e1) / max(1, len(batches) - warmup)


def _psnr(model, info, field, n=1 << 20, seed=777):
    import torch
    import synth
    import paper_2507_03836_gb300 as fh
    held = synth.coords(seed, n)
    truth = synth.sample(field, info["fbb_lo"], info["fbb_size"], held).astype(np.float64)
    o = torch.empty(n, dtype=torch.float32, device="cuda")
    fh.fhash_forward(model, torch.from_numpy(held).cuda(), o)
    pred = o.cpu().numpy().astype(np.float64)
    rng = truth.max() - truth.min()
    return float(10 * np.log10(rng ** 2 / np.mean((pred - truth) ** 2))), float(np.abs(pred - truth).max())


def leg_precision_front(args, steps):
    """Precision form against float32 on the Combustion-shaped front: both trained from the same start on the
    same batches; samples/s of each, and PSNR / max abs error on 1M held-out points against the field."""
    import paper_2507_03836_gb300 as fh
    from synth import workloads
    w = workloads.FRONT
    t0 = time.time()
    field, mask = workloads.make_field_and_mask(w)
    res = {"workload": w["name"], "steps": steps, "batch": w["batch"],
           "note": "both forms trained from the same fresh start; ms_per_step over all but 3 warm-up steps"}
    for name, dt in (("fp32", fh.FP32), ("bf16", fh.BF16)):
        model, info = _build(w, dt, 5, mask, _layout(args))
        batches = _batches(w, info, field, steps + 3, 50_000)
        ms = _train(model, batches, w["adam"])
        p, e = _psnr(model, info, field)
        res[name] = {"ms_per_step": ms, "samples_s": w["batch"] / ms * 1e3, "psnr_db": p, "max_abs_err": e,
                     "params": info["n_table_params"] + info["n_mlp_params"]}
        del model, batches
    res["psnr_drop_db"] = res["fp32"]["psnr_db"] - res["bf16"]["psnr_db"]
    res["bf16_over_fp32_samples_s"] = res["bf16"]["samples_s"] / res["fp32"]["samples_s"]
    res["setup_s"] = time.time() - t0
    return res


def suite_precision(args):
    res = leg_precision_front(args, args.steps)
    res["suite"] = "precision"
    print(json.dumps(res))


def suite_coreset(args):
    """Coreset training (Section 3.1) on advect-256^3x64: the union of the dilated feature at 10 key frames,
    the paper's batch of 2^21, epochs shuffled by the library.  Reports the coreset size and build time,
    samples/s of coreset training steps, and PSNR of the coreset-trained model and of a model trained
    for the same steps on uniform samples, on 1M held-out coreset samples (the feature region at the key
    frames) and on 1M uniform points."""
    import torch
    import paper_2507_03836_gb300 as fh
    from synth import workloads
    w = dict(workloads.LARGE, batch=1 << 21)
    keys = [int(round(k * (w["dims"][3] - 1) / 9)) for k in range(10)]
    t0 = time.time()
    field, mask = workloads.make_field_and_mask(w)
    setup_s = time.time() - t0
    hp = w["adam"]
    B, K, W0 = w["batch"], args.steps, 3
    res = {"suite": "coreset", "workload": w["name"], "key_frames": keys, "batch": B, "steps": K}
    model, info = _build(w, fh.FP32, 5, mask, _layout(args))
    torch.cuda.synchronize()
    t1 = time.time()
    N = fh.fhash_coreset_build(model, field, keys)
    res["coreset_samples"] = N
    res["coreset_build_s"] = time.time() - t1
    per_epoch = (N + B - 1) // B
    res["batches_per_epoch"] = per_epoch
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(K + W0):
        if i == W0:
            torch.cuda.synchronize()
            e0.record(st)
        fh.fhash_coreset_train_step(model, 1, i // per_epoch, i % per_epoch, B, hp)
    e1.record(st)
    torch.cuda.synchronize()
    fh.fhash_check(model)
    ms = e0.elapsed_time(e1) / K
    res["coreset_train"] = {"ms_per_step": ms, "samples_s": B / ms * 1e3}
    # held-out evaluation sets: coreset samples of another shuffle, and uniform points
    hc = torch.empty((1 << 20, 4), dtype=torch.float32, device="cuda")
    ht = torch.empty(1 << 20, dtype=torch.float32, device="cuda")
    n_h = fh.fhash_coreset_batch(model, 4242, 0, 0, 1 << 20, hc, ht)
    hc, ht = hc[:n_h], ht[:n_h].cpu().numpy().astype(np.float64)

    def feature_psnr(m):
        o = torch.empty(n_h, dtype=torch.float32, device="cuda")
        fh.fhash_forward(m, hc, o)
        pred = o.cpu().numpy().astype(np.float64)
        rng = ht.max() - ht.min()
        return float(10 * np.log10(rng ** 2 / np.mean((pred - ht) ** 2)))

    res["coreset_train"]["psnr_feature_db"] = feature_psnr(model)
    res["coreset_train"]["psnr_uniform_db"] = _psnr(model, info, field)[0]
    del model
    uni, info = _build(w, fh.FP32, 5, mask, _layout(args))
    ms = _train(uni, _batches(w, info, field, K + W0, 60_000), hp, warmup=W0)
    res["uniform_train"] = {"ms_per_step": ms, "samples_s": B / ms * 1e3, "psnr_feature_db": feature_psnr(uni),
                            "psnr_uniform_db": _psnr(uni, info, field)[0]}
    res["setup_s"] = setup_s
    print(json.dumps(res))


def suite_masked(args):
    """Masked compact tables (FHASH_LAYOUT_MASKED, Section 3.1's feature-only grids) against the default
    brick layout, both trained on the coreset of advect-256^3x64 (10 key frames, batch 2^21): table size,
    directory build time, coreset-training samples/s, float32 forward samples/s on 4M held-out coreset
    points and PSNR there."""
    import torch
    import paper_2507_03836_gb300 as fh
    from synth import workloads
    w = dict(workloads.LARGE, batch=1 << 21)
    keys = [int(round(k * (w["dims"][3] - 1) / 9)) for k in range(10)]
    field, mask = workloads.make_field_and_mask(w)
    hp = w["adam"]
    B, K, W0 = w["batch"], args.steps, 3
    res = {"suite": "masked", "workload": w["name"], "key_frames": keys, "batch": B, "steps": K}
    st = torch.cuda.current_stream()
    for name, layout in (("brick", fh.LAYOUT_BRICK), ("masked", fh.LAYOUT_MASKED)):
        torch.cuda.synchronize()
        t0 = time.time()
        model, info = _build(w, fh.FP32, 5, mask, layout)
        build_s = time.time() - t0
        N = fh.fhash_coreset_build(model, field, keys)
        per_epoch = (N + B - 1) // B
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i in range(K + W0):
            if i == W0:
                torch.cuda.synchronize()
                e0.record(st)
            fh.fhash_coreset_train_step(model, 1, i // per_epoch, i % per_epoch, B, hp)
        e1.record(st)
        torch.cuda.synchronize()
        fh.fhash_check(model)
        ms = e0.elapsed_time(e1) / K
        n_h = 1 << 22
        hc = torch.empty((n_h, 4), dtype=torch.float32, device="cuda")
        ht = torch.empty(n_h, dtype=torch.float32, device="cuda")
        n_h = fh.fhash_coreset_batch(model, 4242, 0, 0, n_h, hc, ht)
        hc, ht = hc[:n_h], ht[:n_h]
        o = torch.empty(n_h, dtype=torch.float32, device="cuda")
        for _ in range(3):
            fh.fhash_forward(model, hc, o)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(10):
            fh.fhash_forward(model, hc, o)
        e1.record(st)
        torch.cuda.synchronize()
        fwd_ms = e0.elapsed_time(e1) / 10
        pred, lab = o.cpu().numpy().astype(np.float64), ht.cpu().numpy().astype(np.float64)
        psnr = float(10 * np.log10((lab.max() - lab.min()) ** 2 / np.mean((pred - lab) ** 2)))
        res[name] = {"table_rows": info["total_rows"], "table_params": info["n_table_params"],
                     "device_bytes": info["device_bytes"], "build_s": build_s, "coreset_samples": N,
                     "train_ms_per_step": ms, "train_samples_s": B / ms * 1e3,
                     "forward_samples_s": n_h / fwd_ms * 1e3, "psnr_feature_db": psnr}
        del model, hc, ht, o
        torch.cuda.empty_cache()
    res["table_fraction"] = res["masked"]["table_rows"] / res["brick"]["table_rows"]
    print(json.dumps(res))


def suite_forward(args):
    """The two evaluation paths of the precision form on uniform points: the fused kernel and the split
    pair (bf16 encoding rows, then the TMA-fed tensor-core MLP).  --workload picks the model (random
    initial tables, U(-0.5, 0.5)), --forward-points the batch, --steps the timed calls after 3 warm-up
    calls; --forward-paths restricts the paths.  Both paths give bit-identical outputs (checked)."""
    import torch
    import synth
    import paper_2507_03836_gb300 as fh
    from synth import workloads
    w = dict(_workload(args.workload), init_range=0.5)
    field, mask = workloads.make_field_and_mask(w)
    model, info = _build(w, fh.BF16, 1, mask, _layout(args))
    n = args.forward_points
    c = torch.from_numpy(synth.coords(5, n)).cuda()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    res = {"suite": "forward", "workload": w["name"], "layout": args.layout, "points": n, "steps": args.steps}
    sums = {}
    st = torch.cuda.current_stream()
    for name in args.forward_paths.split(","):
        fh.fhash_set_forward_path(model, {"fused": fh.FORWARD_FUSED, "split": fh.FORWARD_SPLIT}[name])
        for _ in range(3):
            fh.fhash_forward(model, c, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            fh.fhash_forward(model, c, out)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[name] = {"ms": ms, "samples_s": n / ms * 1e3}
        sums[name] = out.clone()
    fh.fhash_check(model)
    if len(sums) == 2:
        res["bit_identical"] = bool(torch.equal(sums["fused"], sums["split"]))
    print(json.dumps(res))


def suite_peaks(args):
    """Ceilings of the encoding's access pattern on this GPU: random gathers of 4, 8 and 16 bytes from a
    64 MB table (resident in the 129 MB L2) and from an 8 GB table (HBM), through the library's
    fhash_diag_random_gather kernel.  Reports gathers/s, useful GB/s and 32-byte-sector GB/s, plus
    MEASURED_PEAKS.json for reference."""
    import torch
    import paper_2507_03836_gb300 as fh
    res = {"suite": "peaks", "measured_peaks": _peaks()[0]}
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    for name, nbytes in (("l2_64MB", 64 << 20), ("hbm_8GB", 8 << 30)):
        table = torch.rand(nbytes // 4, dtype=torch.float32, device="cuda")
        for width in (4, 8, 16):
            n = 1 << 28
            for _ in range(2):
                fh.fhash_diag_random_gather(table, width, n, 7, out)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            reps = 5
            for r in range(reps):
                fh.fhash_diag_random_gather(table, width, n, 100 + r, out)
            e1.record(st)
            torch.cuda.synchronize()
            s = e0.elapsed_time(e1) / 1e3 / reps
            res["%s_w%d" % (name, width)] = {"gathers_s": n / s, "useful_gbs": n * width / s / 1e9,
                                              "sector_gbs": n * 32 / s / 1e9}
        del table
    print(json.dumps(res))


def _serve(models, kinds, n_req, rate, budget, tf, seed=1234, decode_every=0):
    """Poisson stream through one server; kinds[i] = model index of request i; every `decode_every`-th
    request (0: none) is a time-slice decode (upsample 1 or 2), the rest renders of 256^2/512^2/1024^2.
    rate None: closed loop, each request submitted when the previous one is done (service time alone)."""
    import torch
    import synth
    import paper_2507_03836_gb300 as fh
    rng = np.random.default_rng(seed)
    closed = rate is None
    arrivals = np.cumsum(rng.exponential(1.0 / (rate or 1.0), n_req))
    if closed:
        arrivals[:] = np.inf
    sizes = rng.choice([256, 512, 1024], n_req)
    times = rng.random(n_req)
    ups = rng.choice([1, 2], n_req)
    srv = fh.fhash_server_create(models, budget_bytes=budget, max_live=64, tick_samples=1 << 22)
    reqs, outs = [], []
    for i in range(n_req):
        mi = kinds[i]
        if decode_every and i % decode_every == decode_every - 1:
            d = fh.fhash_decode_dims(models[mi], int(ups[i]))
            out = torch.empty((d[2], d[1], d[0]), dtype=torch.float32, device="cuda")
            reqs.append(fh.make_request(fh.REQ_DECODE, mi, float(times[i]), upsample=int(ups[i]), out=out))
        else:
            s_ = int(sizes[i])
            out = torch.empty((s_, s_, 4), dtype=torch.float32, device="cuda")
            cam = synth.camera(synth.sphere_eye(7, i), s_, s_)
            reqs.append(fh.make_request(fh.REQ_RENDER, mi, float(times[i]), cam, s_, s_, 64, tf, out=out))
        outs.append(out)
    # warm-up (kernels, graphs)
    wid = fh.fhash_server_submit(srv, reqs[0])
    while fh.fhash_server_poll(srv, wid)[0] != fh.REQ_DONE:
        fh.fhash_server_tick(srv)
    st0 = fh.fhash_server_get_stats(srv)
    torch.cuda.synchronize()
    lat = np.zeros(n_req)
    done = np.zeros(n_req, bool)
    ids = {}
    nxt = 0
    t0 = time.perf_counter()
    while not done.all():
        now = time.perf_counter() - t0
        if closed and nxt < n_req and all(done[k] for k in ids):  # one at a time: arrival = now
            arrivals[nxt] = now
        while nxt < n_req and arrivals[nxt] <= now:
            ids[nxt] = fh.fhash_server_submit(srv, reqs[nxt])
            nxt += 1
        if not ids or all(done[k] for k in ids):
            time.sleep(max(0.0, min(arrivals[nxt] - (time.perf_counter() - t0), 0.01)) if nxt < n_req else 0)
            continue
        fh.fhash_server_tick(srv)
        tnow = time.perf_counter() - t0
        for k, rid in ids.items():
            if not done[k] and fh.fhash_server_poll(srv, rid)[0] == fh.REQ_DONE:
                done[k] = True
                lat[k] = (tnow - arrivals[k]) * 1e3
    elapsed = time.perf_counter() - t0
    st = fh.fhash_server_get_stats(srv)
    samples = st["samples"] - st0["samples"]
    is_dec = np.array([bool(decode_every and i % decode_every == decode_every - 1) for i in range(n_req)])
    out = {"p50_ms": float(np.percentile(lat, 50)), "p95_ms": float(np.percentile(lat, 95)),
           "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
           "throughput_samples_s": samples / elapsed, "requests_s": n_req / elapsed,
           "ticks": st["ticks"] - st0["ticks"], "graph_launches": st["model_launches"] - st0["model_launches"]}
    if is_dec.any():
        out["render_p50_ms"] = float(np.percentile(lat[~is_dec], 50))
        out["render_p99_ms"] = float(np.percentile(lat[~is_dec], 99))
        out["decode_p50_ms"] = float(np.percentile(lat[is_dec], 50))
        out["decode_p99_ms"] = float(np.percentile(lat[is_dec], 99))
    del srv
    return out


def leg_serve_shell(args, steps, n_req, rate, alone=0):
    """Render serving on the Supernova-shaped shell model (trained as the default workload for `steps`
    steps): Poisson stream at `rate` req/s, FP32 form and the precision form (same weights), p50/p95/p99 and
    samples/s; PSNR of both forms; with alone > 0 also the latency of the first `alone` requests served one
    at a time (service time without queueing)."""
    import torch
    import synth
    import paper_2507_03836_gb300 as fh
    from synth import workloads
    w = workloads.SHELL
    t0 = time.time()
    field, mask = workloads.make_field_and_mask(w)
    m32, info = _build(w, fh.FP32, 6, mask, _layout(args))
    ms = _train(m32, _batches(w, info, field, steps + 3, 60_000), w["adam"])
    m16, _ = _build(w, fh.BF16, 6, mask, _layout(args))
    del mask
    _copy_params(m32, m16, info["n_table_params"] + info["n_mlp_params"])
    tf = torch.from_numpy(synth.transfer_function(0.5)).cuda()
    res = {"workload": w["name"], "model_params": info["n_table_params"] + info["n_mlp_params"],
           "train_steps": steps + 3, "train_ms_per_step": ms, "requests": n_req, "rate_req_s": rate,
           "images": "uniform in {256^2, 512^2, 1024^2}, cameras on the radius-2 sphere, t uniform in [0,1]"}
    for name, mi in (("fp32", 0), ("bf16", 1)):
        res[name] = _serve([m32, m16], [mi] * n_req, n_req, rate, 96 << 30, tf)
        if alone:
            res[name]["alone"] = _serve([m32, m16], [mi] * alone, alone, None, 96 << 30, tf)
        res[name]["psnr_db"], res[name]["max_abs_err"] = _psnr(m32 if mi == 0 else m16, info, field)
    res["setup_s"] = time.time() - t0
    del m32, m16
    return res


def suite_serve(args):
    res = leg_serve_shell(args, args.steps, args.serve_requests, args.serve_rate)
    res["suite"] = "serve"
    print(json.dumps(res))


def suite_mixed(args):
    """Mixed stream over three resident models (the advect-256^3x64 model in FP32, the front model and a second
    256^3x64 model in the precision form) under a 64 GB budget; decode:render 1:3."""
    import torch
    import synth
    import paper_2507_03836_gb300 as fh
    from synth import workloads
    t0 = time.time()
    models, infos = [], []
    for w, dt, seed in ((workloads.LARGE, fh.FP32, 7), (workloads.FRONT, fh.BF16, 8),
                        (dict(workloads.LARGE, seed=4, name="advect2-256^3x64"), fh.BF16, 9)):
        field, mask = workloads.make_field_and_mask(w)
        m, info = _build(w, dt, seed, mask, _layout(args))
        _train(m, _batches(w, info, field, args.steps + 3, 70_000 + seed * 1000), w["adam"])
        models.append(m)
        infos.append((w["name"], info))
        del field, mask
    tf = torch.from_numpy(synth.transfer_function(0.5)).cuda()
    kinds = list(np.random.default_rng(5).integers(0, 3, args.serve_requests))
    res = {"suite": "mixed", "models": [n for n, _ in infos], "budget_bytes": 64 << 30,
           "requests": args.serve_requests, "rate_req_s": args.serve_rate, "decode_to_render": "1:3"}
    res.update(_serve(models, kinds, args.serve_requests, args.serve_rate, 64 << 30, tf, decode_every=4))
    res["setup_s"] = time.time() - t0
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "medium", "small"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"],
                    help="training form: float32, or the bf16 precision form (tensor-core MLP)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving and precision legs")
    ap.add_argument("--batch", type=int, default=0,
                    help="samples per step (0: the workload's batch; other values are for profiling cases only)")
    ap.add_argument("--age-steps", type=int, default=512,
                    help="untimed training steps on fresh batches before the warm-up (steady-state Adam deferral)")
    ap.add_argument("--adam-deferral", type=int, default=-1,
                    help="levels with at least this many rows defer their Adam update (0: dense Adam every "
                         "step; -1: the library default, 2^25)")
    ap.add_argument("--serve-requests", type=int, default=60)
    ap.add_argument("--serve-alone", type=int, default=12, help="requests also served one at a time (no queueing)")
    ap.add_argument("--serve-train-steps", type=int, default=40, help="training steps of the served shell model")
    ap.add_argument("--precision-steps", type=int, default=20, help="training steps per form on the front model")
    ap.add_argument("--no-precision-suite", action="store_true", help="skip the front-model bf16 vs fp32 leg")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--layout", default="brick", choices=["linear", "brick"],
                    help="table row layout: 4x4x4 bricks per time slice (the default: the faster F-Hash "
                         "linearisation on this GPU), or Eq. 9")
    ap.add_argument("--forward-points", type=int, default=1 << 22, help="--suite forward: points per call")
    ap.add_argument("--forward-paths", default="fused,split", help="--suite forward: paths to time")
    ap.add_argument("--suite", default="train", choices=["train", "precision", "serve", "mixed", "coreset", "masked", "forward",
                                                    "peaks"],
                    help="train: the default line; precision / serve / mixed: the other workloads")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.suite != "train":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        return {"precision": suite_precision, "serve": suite_serve, "mixed": suite_mixed,
                "coreset": suite_coreset, "masked": suite_masked, "forward": suite_forward,
                "peaks": suite_peaks}[args.suite](args)

    import torch
    import synth
    import paper_2507_03836_gb300 as fh

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    w = _workload(args.workload)
    from synth import workloads
    t0 = time.time()
    field, mask = workloads.make_field_and_mask(w)
    nx, ny, nz, nt = w["dims"]
    model = fh.fhash_build(nx, ny, nz, nt, mask=mask, schedule=fh.make_schedule(**w["schedule"]), F=w["F"],
                           dtype=fh.BF16 if args.dtype == "bf16" else fh.FP32,
                           mlp_hidden_layers=w["hidden"], mlp_width=w["width"], seed=1 + rank,
                           init_range=w["init_range"], layout=_layout(args))
    mask_for_bf16 = mask if not args.no_serve else None
    del mask
    info = fh.fhash_get_info(model)
    setup_s = time.time() - t0

    # batches: coords uniform in [0,1]^4 (FBB-normalised), targets sampled from the field
    if args.batch > 0:
        w = dict(w, batch=args.batch)
    B = w["batch"]
    # fresh batches for every loop below (warm-up, timed, phase breakdown, end to end): a batch seen a few
    # steps earlier would find its table groups almost current and understate the deferred Adam's replay
    nb = args.warmup + 3 * args.steps + 2
    coords_h = [synth.coords(10_000 + 100 * rank + k, B) for k in range(nb)]
    tgt_h = [synth.sample(field, info["fbb_lo"], info["fbb_size"], c) for c in coords_h]
    coords_d = [torch.from_numpy(c).cuda() for c in coords_h]
    tgt_d = [torch.from_numpy(t).cuda() for t in tgt_h]
    loss_d = torch.zeros(nb, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    hp = w["adam"]

    if args.adam_deferral >= 0:
        fh.fhash_set_adam_deferral(model, args.adam_deferral)
    # aging (untimed): steps on fresh batches, so that the deferred Adam state (how many steps each table
    # group is behind when a batch reads it) has the distribution of a long training run, not of a
    # fresh model (a fresh model's first steps replay almost nothing)
    t_age = time.time()
    for k in range(args.age_steps):
        c = synth.coords(50_000 + 1000 * rank + k, B)
        fh.fhash_train_step(model, torch.from_numpy(c).cuda(),
                            torch.from_numpy(synth.sample(field, info["fbb_lo"], info["fbb_size"], c)).cuda(), hp)
    torch.cuda.synchronize()
    age_s = time.time() - t_age
    for k in range(args.warmup):
        fh.fhash_train_step(model, coords_d[k], tgt_d[k], hp, loss_d[k:k + 1])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    K = args.steps
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    e_start.record(st)
    for k in range(K):
        i = args.warmup + k
        fh.fhash_train_step(model, coords_d[i], tgt_d[i], hp, loss_d[i:i + 1])
    e_end.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed = max_over_ranks(dist, e_start.elapsed_time(e_end) / 1e3)
    losses = loss_d.cpu().numpy()

    # phase breakdown (untimed for the headline): the same batches again with the library's events around
    # the phases of fhash_train_step on its stream
    fh.fhash_set_timing(model, True)
    ph, groups, gsteps = [], [], []
    for k in range(K):
        i = args.warmup + K + k
        fh.fhash_train_step(model, coords_d[i], tgt_d[i], hp)
        a = fh.fhash_get_adam_stats(model)
        ph.append(a["last_ms"] + [a["last_side_ms"]])
        groups.append(a["last_replayed_groups"])
        gsteps.append(a["last_replayed_steps"])
    fh.fhash_set_timing(model, False)
    ph = np.mean(np.array(ph), 0)
    adam_stats = fh.fhash_get_adam_stats(model)
    claim_ms, replay_ms, encode_ms, mlp_ms, scatter_ms, dw_ms, dense_ms, side_ms = (float(x) for x in ph)
    # with deferred levels the dense-range update runs on a second stream beside the next step's replay
    # (last_side_ms); the step's own Adam phase then only records its scalars
    overlapped = side_ms > 0
    if overlapped:
        tab_ms, dense_ms = dense_ms, side_ms
    replay_groups, replay_steps = float(np.mean(groups)), float(np.mean(gsteps))
    n_deferred = int(adam_stats["deferred_params"])
    gsize = int(adam_stats["group_params"])

    # end to end through the public API: host (pinned) inputs copied in, loss read back, every step
    e0 = args.warmup + 2 * K
    pin_c = [torch.from_numpy(c).pin_memory() for c in coords_h[e0:e0 + K + 2]]
    pin_t = [torch.from_numpy(t).pin_memory() for t in tgt_h[e0:e0 + K + 2]]
    lh = np.zeros(1, np.float64)
    for k in range(K, K + 2):  # warm-up of the host-input path (its staging buffers) on two more batches
        fh.fhash_train_step(model, pin_c[k].numpy(), pin_t[k].numpy(), hp, lh)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t1 = time.perf_counter()
    for k in range(K):
        fh.fhash_train_step(model, pin_c[k].numpy(), pin_t[k].numpy(), hp, lh)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t1)
    fh.fhash_check(model)

    # fraction of 4-parameter groups with a non-zero gradient after one step in the densely updated range
    # (untimed, after every timed loop: reading the gradient brings every deferred group up to date, which
    # would shorten the replays of the steps after it): k_adam writes the cleared gradient back only
    # there, so its algorithmic bytes are 28 B/param + 4 B x that fraction
    touched = _touched_fraction(fh, model, info, coords_d[args.warmup], tgt_d[args.warmup], hp, n_deferred)

    prec = None
    if not args.no_serve:
        prec = precision_leg(args, w, model, info, field, mask_for_bf16, rank)
    del mask_for_bf16

    n_params = info["n_table_params"] + info["n_mlp_params"]
    peaks, peak_kind = _peaks()
    hbm = peaks["hbm_gbs"]
    L, F = len(info["res"]), info["F"]
    bf16 = args.dtype == "bf16"
    n_dense = n_params - n_deferred
    # Algorithmic bytes per launch of each phase kernel (each phase below is one launch, except the MLP and
    # weight-gradient phases):
    #  k_adam (dense range): read p, g, m, v; write p, m, v, and the cleared g where it was not zero
    #    (+ the bf16 shadow of p in the precision form);
    #  k_defer_replay: per caught-up group of G floats, G x 4 bytes each of p, g, m, v read and of p,
    #    m, v written (+16 bytes of bf16 shadow);
    #  k_encode_cols: per sample 16 corner rows of F float32 per level, the 16-byte coordinates and the
    #    L*F encoding values written;
    #  k_scatter_cols (its two launches): the same corner rows reduced, coordinates, d(encoding) read.
    adam_bpp = (30.0 if bf16 else 28.0) + 4.0 * touched
    elem = 2 if bf16 else 4
    kern = {
        "k_adam": (adam_bpp * n_dense, dense_ms, "dense Adam over %d parameters (levels below the deferred ones "
                                                 "and the MLP), %.2f B/param%s" % (n_dense, adam_bpp,
                                                 "; runs beside the replay, sharing the GPU" if overlapped else "")),
        "k_defer_replay": (replay_groups * gsize * (7 * 4 + (2 if bf16 else 0)), replay_ms,
                           "%.0f caught-up groups of %d floats per step, %.1f replayed steps each on average"
                           % (replay_groups, gsize, replay_steps / max(replay_groups, 1))),
        "k_encode_cols": (B * (16 * L * F * 4 + 16 + L * F * 4), encode_ms,
                          "%d samples x (16 x %d levels x %d floats gathered + 16 B coordinates + %d floats written)"
                          % (B, L, F, L * F)),
        "k_scatter_cols": (B * (16 * L * F * 4 + 16 + L * F * 4), scatter_ms,
                           "%d samples x (16 x %d levels x %d floats reduced + 16 B coordinates + %d floats read)"
                           % (B, L, F, L * F)),
    }
    dims = info["mlp_dims"]
    nh_m, in_m = len(dims) - 2, dims[0]
    if not bf16 and in_m in (16, 32, 64) and 1 <= nh_m <= 2 and all(d == 64 for d in dims[1:-1]):
        # the float32 MLP fused on the tensor cores (its phase also holds the one-block loss reduction):
        # per sample the encoding and target read; hidden activations, every delta and d(encoding) written
        mlp_b = 4 * (in_m + 1) + 4 * (nh_m * 64 + nh_m * 64 + 1 + in_m)
        kern["k_mlp_f32tc"] = (B * mlp_b, mlp_ms, "%d samples x %d B (encoding and target read; activations, "
                                                  "deltas and d(encoding) written)" % (B, mlp_b))
    if bf16:  # the fused tensor-core forward replaces k_encode_cols in the precision form
        kern["k_forward_tc"] = (B * (16 * L * F * elem + 16), encode_ms, "%d samples x (16 x %d levels x %d bf16 "
                                "gathered + 16 B coordinates)" % (B, L, F))
        del kern["k_encode_cols"]
    phases = {}
    for name, (by, ms, note) in kern.items():
        ach = by / (ms / 1e3) / 1e9 if ms > 0 else 0.0
        phases[name] = {"ms": ms, "bytes_per_launch": by, "achieved": ach, "frac": ach / hbm, "unit": "GB/s",
                        "bytes": note}
    top = max(phases, key=lambda k: phases[k]["ms"])
    roofline = dict(kernel=top, bound="hbm", achieved=phases[top]["achieved"], peak=hbm, unit="GB/s",
                    frac=phases[top]["frac"], traffic=None, peak_source=peak_kind,
                    bytes_per_launch=phases[top]["bytes_per_launch"], bytes=phases[top]["bytes"], phases=phases)
    if top == "k_defer_replay" and replay_ms > 0:
        # The replay is bound by special-function arithmetic, not by streamed bytes: every parameter-step
        # takes one approximate square root and one approximate division.  Peak: 16 special-function
        # results per clock per SM (4 per sub-partition) x 152 SMs x the maximum SM clock, two per
        # parameter-step.  traffic: DRAM bytes per caught-up group from one ncu capture of this kernel on
        # advect-128^3x32 (a launch of the full workload exceeds the capture size rule; the replay's
        # memory traffic grows with the groups it catches up, not with their replay lengths).
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        peak_steps = 152 * 16 * sm_mhz * 1e6 / 2 / 1e9
        steps_s = replay_steps * gsize / (replay_ms / 1e3) / 1e9
        roofline.update(bound="alu", unit="G parameter-steps/s", achieved=steps_s, peak=peak_steps,
                        frac=steps_s / peak_steps, peak_source="derived: 152 SMs x 16 special-function results "
                        "per clock x %.0f MHz / 2 per parameter-step" % sm_mhz,
                        traffic=REPLAY_DRAM_BYTES_PER_GROUP * replay_groups if REPLAY_DRAM_BYTES_PER_GROUP else None,
                        traffic_note="ncu dram__bytes_read.sum + dram__bytes_write.sum per caught-up group on "
                                     "advect-128^3x32 (%.0f B), times the groups of this launch" % REPLAY_DRAM_BYTES_PER_GROUP,
                        hbm_algorithmic_frac=phases[top]["frac"])
    value = job_rate(world, B * K, elapsed)
    deferred = adam_stats["first_deferred_level"] >= 0
    # float32 without the fused tensor-core MLP: separate forward and backward MLP kernels
    per_step = (7 if (bf16 or "k_mlp_f32tc" in kern) else 8) + (3 + 3 if deferred else 1)

    out = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": elapsed / K * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": w["name"], "global_batch": B * world, "levels": L, "F": F,
                   "layout": args.layout,
                   "mlp": info["mlp_dims"], "table_params": info["n_table_params"],
                   "parallelism": "replicas" if world > 1 else "single",
                   "adam": "deferred from level %d (%d of %d parameters), bit-identical to dense"
                           % (adam_stats["first_deferred_level"], n_deferred, n_params) if deferred else "dense",
                   "aged_steps": args.age_steps,
                   "l2": "inputs larger than L2: %.1f GB of training state; every step's gathers, replays and "
                         "scatters reach it at random" % (16.0 * n_params / 1e9)},
        "phases_ms": {"catch_up_claim_sort": claim_ms, "catch_up_replay": replay_ms, "encode": encode_ms,
                      "mlp_fwd_loss_bwd": mlp_ms, "scatter": scatter_ms, "weight_grads": dw_ms,
                      "adam_dense": dense_ms, "adam_scalars": tab_ms if overlapped else 0.0},
        "phases_note": "adam_dense runs on a second stream beside catch_up_replay (not on the step's critical "
                       "path)" if overlapped else "phases in sequence on one stream",
        "adam_deferral": {"replayed_groups_per_step": replay_groups, "replayed_group_steps_per_step": replay_steps,
                          "first_deferred_level": adam_stats["first_deferred_level"],
                          "deferred_params": n_deferred},
        # per step, float32: encode, the fused MLP (forward, loss and backward; other shapes: forward and
        # backward apart), loss reduction, 2 scatters; precision form: fused forward, loss reduction, MLP
        # backward, 2 scatters; both: the tensor-core weight gradients and their reduction; then the
        # deferred catch-up (claim, sort, replay), the previous step's Adam over the dense ranges (2
        # launches) and the step's scalar record, or one dense Adam launch
        "gpu_launches": K * per_step,
        "roofline": roofline,
        "clocks": clk,
        "e2e": {"value": job_rate(world, B * K, e2e_s), "unit": "samples/s", "h2d_bytes_per_step": B * 20,
                "d2h_bytes_per_step": 8},
        "loss_first_last": [float(losses[0]), float(losses[-1])],
        "setup_s": setup_s,
    }
    if prec:
        out["precision"] = prec
    if not args.no_serve:
        # the other configurations, after the training model is released: renders served on the shell model
        # (config 4: Poisson stream at 200 req/s, and the same requests one at a time), and bf16 against
        # float32 training on the front model (config 3)
        del model
        torch.cuda.synchronize()
        out["render"] = leg_serve_shell(args, args.serve_train_steps, args.serve_requests, args.serve_rate,
                                        alone=args.serve_alone)
        if not args.no_precision_suite:
            out["precision_front"] = leg_precision_front(args, args.precision_steps)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t, desc = oracle_step_sample(w, 32768, adam_slice=1 << 25)
        one = {"value": B / t, "unit": "samples/s", "cores": 1, "kind": "oracle", "sample": desc}
        out["cpu_baseline"] = one
        try:  # the same oracle on every host core at once
            pool = OraclePool()
            tp, descp = pool.step(w, 8192, 1 << 22, seed=3)
            pool.close()
            out["cpu_baseline"] = {"value": B / tp, "unit": "samples/s", "cores": pool.procs, "kind": "oracle",
                                   "sample": descp, "single_process": one}
        except Exception as e:
            one["all_cores_error"] = str(e)[:200]
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
