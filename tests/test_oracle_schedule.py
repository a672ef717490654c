"""Pins of the oracle's level schedule and table sizing against numbers the paper prints.

CPU only.  Fixtures: tests/golden/table3_params.txt (Table 3, Section 5.2.2; FBB sizes from the
evolution-visualisation figure of Section 5.3.1; key frames from Section 5.1.1).
"""
import os

import numpy as np
import pytest

from oracle import schedule
from oracle.encode import fhash

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table3_params.txt")


def _rows():
    out = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        out.append(dict(name=f[0], S=[int(f[1]), int(f[2]), int(f[3])], T=int(f[4]), F=int(f[5]),
                        mi=float(f[6]), res_level=int(f[7]), frame=[int(f[8]), int(f[9]), int(f[10])],
                        pct=float(f[11]), status=f[12]))
    return out


def test_ceil_log():
    assert [schedule.ceil_log(2, s) for s in (1, 2, 3, 4, 5, 54, 64, 65, 200)] == [0, 1, 2, 2, 3, 6, 6, 7, 8]
    assert schedule.ceil_log(3, 27) == 3 and schedule.ceil_log(3, 28) == 4


@pytest.mark.parametrize("row", [r for r in _rows() if r["status"] != "unreproduced"], ids=lambda r: r["name"])
def test_table3_parameter_count(row):
    # Both level-count readings (Eq. 6 max, Table 3 min) give the printed mebi count.
    for rule in ("max", "min"):
        lv = schedule.fold_schedule(row["S"], row["T"], 2, rule)
        mi = schedule.param_count(lv, row["F"]) / 2**20
        if row["status"] == "exact":
            assert round(mi, 1) == row["mi"], (rule, mi)
        else:
            assert abs(mi - row["mi"]) / row["mi"] < 1e-3, (rule, mi)


def test_combustion_exact_counts():
    # 200x110x54, 10 key frames, fold 2, F=2: both readings land on 24.20 Mi.
    assert schedule.param_count(schedule.fold_schedule([200, 110, 54], 10, 2, "max"), 2) == 25374176
    assert schedule.param_count(schedule.fold_schedule([200, 110, 54], 10, 2, "min"), 2) == 25374080


@pytest.mark.parametrize("row", _rows(), ids=lambda r: r["name"])
def test_table3_res_level_is_min_rule(row):
    assert len(schedule.fold_schedule(row["S"], row["T"], 2, "min")) == row["res_level"]


@pytest.mark.parametrize("row", _rows(), ids=lambda r: r["name"])
def test_fbb_caption_mapping(row):
    # The reading of the garbled caption order reproduces its printed percentages.
    pct = 100.0 * np.prod(row["S"]) / np.prod(row["frame"])
    assert round(pct, 2) == row["pct"]


def test_fold_recursion_closed_form():
    # Eqs. 7-8 on the Combustion FBB, written out: x halves (rounding up) down to 2, shorter axes pad
    # with 2 at the tail, time 10 -> 5 -> 3 -> 2.
    lv = schedule.fold_schedule([200, 110, 54], 10, 2, "max")
    fine_to_coarse = lv[::-1]
    assert [r[0] for r in fine_to_coarse] == [200, 100, 50, 25, 13, 7, 4, 2]
    assert [r[1] for r in fine_to_coarse] == [110, 55, 28, 14, 7, 4, 2, 2]
    assert [r[2] for r in fine_to_coarse] == [54, 27, 14, 7, 4, 2, 2, 2]
    assert [r[3] for r in fine_to_coarse] == [10, 5, 3, 2, 2, 2, 2, 2]
    # fold 4: fewer levels (Table 1 reports 4 levels at fold 4 for its 8-level fold-2 case)
    assert len(schedule.fold_schedule([200, 110, 54], 10, 4, "max")) == 4


def test_geometric_schedule_256():
    lv = schedule.geometric_schedule([8, 8, 8, 2], [256, 256, 256, 64], 16)
    assert [r[0] for r in lv] == [8, 10, 13, 16, 20, 25, 32, 40, 51, 64, 81, 102, 128, 161, 203, 256]
    assert [r[3] for r in lv] == [2, 3, 3, 4, 5, 6, 8, 10, 13, 16, 20, 25, 32, 40, 51, 64]
    assert schedule.bases(lv)[1] == 1778559385


def test_fhash_bijective_brute_force():
    # Eq. 9 is a minimal perfect hash per level; with per-level bases the concatenated rows of every
    # vertex of every level cover [0, total) exactly once.
    levels = [[3, 4, 5, 2], [2, 3, 2, 1], [5, 2, 3, 3], [1, 1, 2, 4]]
    b, total = schedule.bases(levels)
    rows = []
    for R, base in zip(levels, b):
        t, z, y, x = np.meshgrid(*[np.arange(n) for n in (R[3], R[2], R[1], R[0])], indexing="ij")
        rows.append(base + fhash(t.ravel(), x.ravel(), y.ravel(), z.ravel(), R))
    rows = np.sort(np.concatenate(rows))
    assert np.array_equal(rows, np.arange(total))


def test_fhash_eq9_hand_values():
    # Eq. 9 evaluated by hand on R = (Rx, Ry, Rz, Rt) = (3, 4, 5, 2):
    #   (t,x,y,z) = (1,2,3,4): 1*60 + 4*12 + 3*3 + 2 = 119 (the last row);
    #   (0,1,0,0) -> 1 (x is the fastest axis), (0,0,1,0) -> 3, (0,0,0,1) -> 12, (1,0,0,0) -> 60.
    R = [3, 4, 5, 2]
    assert int(fhash(1, 2, 3, 4, R)) == 119
    assert [int(fhash(*v, R)) for v in ((0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (1, 0, 0, 0))] == [1, 3, 12, 60]
