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
        assert r["traffic"] == bench.measured_traffic("k_m2l_tc", "uniform-1M-p5-d5", "fp16x3")


def test_traffic_counts_only_for_the_captured_sources(tmp_path, monkeypatch):
    """A traffic figure is used only while the kernel's sources have the
    digest recorded with it."""
    f = tmp_path / "traffic.txt"
    good = bench.source_digest("k_m2l_tc")
    f.write_text("# kernel workload precision digest bytes\n"
                 "k_m2l_tc uniform-1M-p5-d5 fp16x3 %s 1234\n"
                 "k_m2l_tc uniform-1M-p5-d6 fp16x3 0000000000000000 999\n" % good)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.measured_traffic("k_m2l_tc", "uniform-1M-p5-d5", "fp16x3") == 1234
    assert bench.measured_traffic("k_m2l_tc", "uniform-1M-p5-d6", "fp16x3") is None
    assert bench.measured_traffic("k_m2l_tc", "uniform-1M-p5-d5", "tf32x3") is None


def test_stage_rooflines_arithmetic():
    """Per-stage work over time against each stage's bound, and the overall
    fraction = sum of ideal stage times / matvec time."""
    if not os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        pytest.skip("no measured peaks")

    class Props:
        multi_processor_count = 152

    class Cuda:
        @staticmethod
        def get_device_properties(dev):
            return Props()

    torch = SimpleNamespace(cuda=Cuda)
    info = SimpleNamespace(m2l_pairs=6039504, rank=89, p2p_evals=441_000_000, p2p_pairs=851_000_000,
                           near_symmetric=1)
    c = {"n": 1 << 20, "p": 5, "depth": 5, "kernel": 1}
    stage = [0.014, 0.15, 0.36, 0.16, 0.0, 0.72, 0.018, 0.92]
    m2l = bench.roofline("fp16x3", info, 1, 0.36, {"sm_mhz": 2070.0}, None, None, "uniform-1M-p5-d5")
    r = bench.stage_rooflines(info, c, 1, stage, "fp16x3", {"sm_mhz": 2070.0}, torch, None, m2l, 0.90)
    mufu = 152 * 16 * 2070e6
    assert r["p2p"]["achieved"] == pytest.approx(441e6 / 0.72e-3 / 1e9)
    assert r["p2p"]["frac"] == pytest.approx(441e6 / 0.72e-3 / mufu)
    hbm = peaks()["hbm_gbs"] * 1e9
    n = float(1 << 20)
    assert r["combine"]["frac"] == pytest.approx((4 * n * 4 + 52 * n) / 0.018e-3 / hbm)
    assert r["m2l"]["ideal_ms"] == pytest.approx(m2l["frac"] * 0.36)
    ideal = sum(v["ideal_ms"] for k, v in r.items() if k != "overall")
    assert r["overall"]["frac"] == pytest.approx(ideal / 0.90)
