"""The library's host-side schedule and sizing (fhash_plan: no CUDA call, so it runs here on the CPU)
against the oracle's schedules and the parameter counts Table 3 prints.

- Fold schedules (both level-count rules) on the Table 3 bounding boxes: levels equal to the oracle's
  and the Combustion encoding parameters equal to the printed 24.20 Mi (25,374,176 with Eq. 6's
  maximum, 25,374,080 with the minimum rule).
- Geometric and explicit schedules: levels, table rows, parameters (tables plus MLP) and state bytes
  (16 B per parameter, 18 B with the bf16 shadow) equal to the oracle's counts; the bench workload
  has 3,557,118,770 table parameters.
- Refusals: L*F above 64, fold < 2, bad F, MLP width or FBB size.
- The masked layout's per-axis active-vertex rule (fhash_active_range) equals the oracle's.
"""
import os

import numpy as np
import pytest

from oracle import schedule
from synth import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table3_params.txt")


def fh():
    import __graft_entry__
    __graft_entry__._build_module().build()  # in-tree library (a no-op when it is up to date)
    import paper_2507_03836_gb300 as m
    return m


def _rows():
    out = []
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            out.append(dict(name=f[0], fbb=[int(x) for x in f[1:4]], keys=int(f[4]), F=int(f[5])))
    return out


@pytest.mark.parametrize("rule", ["max", "min"])
@pytest.mark.parametrize("row", _rows(), ids=lambda r: r["name"])
def test_fold_plan_matches_oracle(row, rule):
    f = fh()
    s = f.make_schedule(mode="fold", fold=2, levels_rule=f.LEVELS_MAX if rule == "max" else f.LEVELS_MIN)
    p = f.fhash_plan(row["fbb"], row["keys"], s, F=row["F"], mlp_hidden_layers=2, mlp_width=64)
    lv = schedule.fold_schedule(row["fbb"], row["keys"], 2, rule)
    assert p["res"] == lv
    assert p["table_rows"] == schedule.bases(lv)[1]
    dims = [len(lv) * row["F"], 64, 64, 1]
    assert p["n_params"] == schedule.param_count(lv, row["F"], dims)
    assert p["state_bytes"] == 16 * p["n_params"]
    if row["name"] == "combustion":
        assert p["table_rows"] * row["F"] == {"max": 25374176, "min": 25374080}[rule]
        assert round(p["table_rows"] * row["F"] / 2 ** 20, 2) == 24.20


def test_geometric_and_explicit_plans():
    f = fh()
    w = workloads.LARGE
    s = w["schedule"]
    p = f.fhash_plan((256, 256, 256), 64, f.make_schedule(**s), F=w["F"], dtype=f.BF16,
                     mlp_hidden_layers=w["hidden"], mlp_width=w["width"])
    lv = schedule.geometric_schedule(s["r0"], s["r1"], s["n_levels"])
    assert p["res"] == lv
    assert p["table_rows"] * w["F"] == 3557118770
    dims = [len(lv) * w["F"]] + [w["width"]] * w["hidden"] + [1]
    assert p["n_params"] == schedule.param_count(lv, w["F"], dims)
    assert p["state_bytes"] == 18 * p["n_params"]
    res = [[3, 5, 2, 1], [6, 9, 7, 2], [13, 10, 17, 3]]
    q = f.fhash_plan((30, 30, 30), 4, f.make_schedule(mode="explicit", res=res), F=4, mlp_hidden_layers=1,
                     mlp_width=16)
    assert q["res"] == res and q["table_rows"] == schedule.bases(res)[1]
    assert q["n_params"] == schedule.param_count(res, 4, [12, 16, 1])


def test_plan_refusals():
    f = fh()
    res16 = [[2, 2, 2, 2]] * 17
    with pytest.raises(f.FHashError):  # 17 levels x F=4 > 64 MLP inputs
        f.fhash_plan((8, 8, 8), 2, f.make_schedule(mode="explicit", res=res16), F=4)
    with pytest.raises(f.FHashError):
        f.fhash_plan((8, 8, 8), 2, f.make_schedule(mode="fold", fold=1))
    with pytest.raises(f.FHashError):
        f.fhash_plan((8, 8, 8), 2, f.make_schedule(mode="fold", fold=2), F=3)
    with pytest.raises(f.FHashError):
        f.fhash_plan((8, 8, 8), 2, f.make_schedule(mode="fold", fold=2), mlp_width=48)
    with pytest.raises(f.FHashError):
        f.fhash_plan((0, 8, 8), 2, f.make_schedule(mode="fold", fold=2))
    assert np.isfinite(f.fhash_plan((8, 8, 8), 1, f.make_schedule(mode="fold", fold=2))["state_bytes"])


def test_masked_active_range_matches_oracle():
    """The library's per-axis rule of the masked layout (the host arithmetic its GPU build uses) equals
    the oracle's, exhaustively over small axes and on bench-sized ones."""
    from oracle import masked
    f = fh()
    for S in list(range(1, 14)) + [256, 431]:
        for R in list(range(1, 16)) + [64, 256, 432]:
            for v in (range(S) if S < 20 else (0, 1, S // 3, S - 2, S - 1)):
                assert f.fhash_active_range(v, S, R) == masked.vertex_range(v, S, R), (S, R, v)
                assert f.fhash_active_range(v, S, R, is_time=True) == masked.time_range(v, S, R), (S, R, v)
    with pytest.raises(f.FHashError):
        f.fhash_active_range(5, 5, 3)
