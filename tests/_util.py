"""Helpers shared by the GPU parity tests: build models through the C ABI and mirror them in the oracle."""
import numpy as np

import synth
from oracle import index, schedule


def fh():
    import paper_2507_03836_gb300 as m
    return m


def torch():
    import torch as t
    return t


def sched_of(w):
    s = dict(w["schedule"])
    return fh().make_schedule(**s)


def oracle_levels(w, fbb_size=None, nt=None):
    s = w["schedule"]
    if s["mode"] == "explicit":
        return [list(r) for r in s["res"]]
    if s["mode"] == "geometric":
        return schedule.geometric_schedule(s["r0"], s["r1"], s["n_levels"])
    return schedule.fold_schedule(fbb_size, nt, s.get("fold", 2), "min" if s.get("levels_rule", 0) else "max")


def build(w, mask=None, dtype=0, seed=7, dims=None):
    nx, ny, nz, nt = dims or w["dims"]
    return fh().fhash_build(nx, ny, nz, nt, mask=mask, schedule=sched_of(w), F=w["F"], dtype=dtype,
                            mlp_hidden_layers=w["hidden"], mlp_width=w["width"], seed=seed,
                            init_range=w["init_range"])


def set_params(model, table, mlp):
    """Writes host float32 table [rows*F] and MLP vector into the model (parameters as inputs)."""
    f = fh()
    table = np.ascontiguousarray(table, np.float32).ravel()
    mlp = np.ascontiguousarray(mlp, np.float32).ravel()
    f.fhash_write_state(model, f.STATE_PARAM, 0, table)
    f.fhash_write_state(model, f.STATE_PARAM, table.size, mlp)


def read(model, which, offset, n):
    f = fh()
    out = np.empty(int(n), np.float32)
    f.fhash_read_state(model, which, offset, out)
    torch().cuda.synchronize()
    return out


def to_dev(a):
    return torch().from_numpy(np.ascontiguousarray(a)).cuda()
