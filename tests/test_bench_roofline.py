"""bench.py's per-stage roofline arithmetic on a plan summary shaped like the 262k sphere's
(float32 level 2, double-float levels 3-4, symmetric float32 near field); no GPU."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

INFO = {
    "lf": 4, "near_precision": "fp32", "near_symmetric": True,
    "p2p_pairs": 897195640, "p2p_self_pairs": 83243070,
    "levels": {2: {"nbox": 56, "K": 7336, "precision": "fp32", "ilist_total": 2504},
               3: {"nbox": 272, "K": 4284, "precision": "df", "ilist_total": 12216},
               4: {"nbox": 1159, "K": 1200, "precision": "df", "ilist_total": 53880}},
}
MS = {"permute_in": 0.01, "near_field": 1.6, "s2m": 0.93, "m2m": 0.62, "m2l": 0.37, "l2l": 0.57,
      "l2t": 0.92, "permute_out": 0.006}
N = 262144


def test_stage_rooflines():
    r = bench.stage_rooflines(INFO, MS, N, N, fp32_peak=40273.92, hbm=6800.0)
    assert set(r) == {"near_field", "s2m", "l2t", "m2l", "m2m", "l2l"}
    off = 897195640 - 83243070
    ops = 38.0 * 83243070 + 51.0 * off / 2
    assert r["near_field"]["kernel"] == "k_p2p_mixed_sym_warp"
    assert r["near_field"]["achieved"] == pytest.approx(ops / 1.6e-3 / 1e9)
    assert r["s2m"]["achieved"] == pytest.approx(156.0 * 600 * N / 0.93e-3 / 1e9)
    m2l = 4.0 * 2504 * 7336 + 48.0 * (12216 * 4284 + 53880 * 1200)
    assert r["m2l"]["bound"] == "alu" and r["m2l"]["achieved"] == pytest.approx(m2l / 0.37e-3 / 1e9)
    m2m = (272 * 4284 * 16 + 56 * 7336 * 8) + (1159 * 1200 * 16 + 272 * 4284 * 16)
    assert r["m2m"]["bound"] == "hbm" and r["m2m"]["achieved"] == pytest.approx(m2m / 0.62e-3 / 1e9)
    for v in r.values():
        assert v["frac"] == pytest.approx(v["achieved"] / v["peak"]) and 0.0 < v["frac"] < 1.5


def test_float64_levels_keep_the_byte_bound_for_m2l():
    info = dict(INFO, levels={2: dict(INFO["levels"][2], precision="fp64")}, lf=2)
    r = bench.stage_rooflines(info, MS, N, N, fp32_peak=40273.92, hbm=6800.0)
    assert r["m2l"]["bound"] == "hbm" and "s2m" not in r
