"""The roofline arithmetic of bench.py: achieved = algorithmic M2L flops
(2 r^2 per interaction pair per product pass per RHS) / stage time, against
the measured BF16 peak (TF32 forms: that peak x the nominal 1.1 / 2.25
ratio), frac = achieved / peak."""
import json
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def peaks():
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("precision,passes,ratio", [("fp16x3", 3, 1.0), ("bf16x3", 3, 1.0),
                                                    ("tf32x3", 3, 1.1 / 2.25), ("tf32", 1, 1.1 / 2.25)])
def test_m2l_roofline(precision, passes, ratio):
    if not os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        pytest.skip("no measured peaks")
    info = SimpleNamespace(m2l_pairs=6039504, rank=89)
    r = bench.roofline(precision, info, 2, 0.5, {"sm_mhz": 2070.0}, None, None, "uniform-1M-p5-d5")
    flops = 2.0 * 89 * 89 * 6039504 * passes * 2
    assert r["achieved"] == pytest.approx(flops / 0.5e-3 / 1e12)
    assert r["peak"] == pytest.approx(peaks()["bf16_tflops"] * ratio)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    if precision == "fp16x3":
        assert r["traffic"] == bench.M2L_TRAFFIC[("uniform-1M-p5-d5", "fp16x3")]
