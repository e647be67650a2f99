"""Host arithmetic of bench.py's roofline figures (no GPU): the dominant
kernel's algorithmic bytes per launch when one launch runs every SOR round,
the whole-step figure against the compulsory bytes of a step, and the shape
of the captured DRAM-traffic table."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    argv, sys.argv = sys.argv, ["bench.py"]
    try:
        spec.loader.exec_module(m)
    finally:
        sys.argv = argv
    return m


def test_sor_launch_accounting(bench):
    km = {"force": 0.013, "collide": 0.027, "stream": 0.012, "grad": 0.011, "sor": 0.044,
          "surf": 0.014}
    cells, rounds = 262144, 2
    one = bench.roofline2(km, cells, "f32", rounds, 6780.0, "measured", sor_launches=1)
    per = bench.roofline2(km, cells, "f32", rounds, 6780.0, "measured", sor_launches=2)
    assert one["kernel"] == per["kernel"] == "sor"
    # one launch for both rounds: twice the bytes in twice the time
    assert one["alg_bytes_per_launch"] == 2 * per["alg_bytes_per_launch"] == 2 * 32 * cells
    assert one["avg_launch_ms"] == pytest.approx(2 * per["avg_launch_ms"])
    assert one["achieved"] == pytest.approx(per["achieved"])
    assert one["achieved"] == pytest.approx(2 * 32 * cells / 0.044e-3 / 1e9)
    assert one["frac"] == pytest.approx(one["achieved"] / 6780.0)
    # FP64 fields double the bytes
    d = bench.roofline2(km, cells, "f64", rounds, 6780.0, "measured", sor_launches=1)
    assert d["alg_bytes_per_launch"] == 2 * one["alg_bytes_per_launch"]


def test_step_roofline(bench):
    r = bench.step_roofline(2000.0, "d2q9", "f32", 6780.0, "L2")
    assert r["b_alg_per_cell"] == 176 and r["achieved_gbs"] == pytest.approx(352.0)
    assert bench.step_roofline(1.0, "d3q19", "bf16", 1.0, "")["b_alg_per_cell"] == 184
    assert bench.step_roofline(1.0, "d3q19", "f32", 1.0, "")["b_alg_per_cell"] == 336
    assert bench.step_roofline(1.0, "d2q9", "f16", 1.0, "")["b_alg_per_cell"] == 104


def test_traffic_table_shape(bench):
    # a figure per tuner tile choice, tied to the hash of the SOR kernel's own
    # sources (the bench reports it only while that hash matches)
    t = bench.TRAFFIC
    assert len(t["kernel_sha"]) == 16 and int(t["kernel_sha"], 16) >= 0
    assert t["sor_launches_per_step"] == 1 and set(t["bytes_per_launch"]) >= {4, 5, 6}
    assert all(b > 0 for b in t["bytes_per_launch"].values())
    assert set(bench.SOR2_FILES) == {"lbs_dev.cuh", "lbs_k2d.cuh"}
    assert bench.src_hash(bench.SOR2_FILES) != bench.src_hash()
