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


def test_fused_step_accounting(bench):
    """The fused 2D step: the SOR group is one launch carrying every sweep
    (32 B a cell and sweep in FP32) plus the gradient (7 fields), the total's
    weights (2) and the rescale (4); the fused LB-FD kernel moves its
    populations and 27 fields once."""
    km = {"force": 0.0, "collide": 0.030, "stream": 0.0, "grad": 0.0, "sor": 0.050,
          "surf": 0.0}
    cells, sweeps = 262144, 8
    r = bench.roofline2(km, cells, "f32", sweeps, 6780.0, "measured", sor_launches=1)
    assert r["kernel"] == "sor"
    assert r["alg_bytes_per_cell"] == 32 * sweeps + 13 * 4
    assert r["alg_bytes_per_launch"] == (32 * sweeps + 52) * cells
    assert r["achieved"] == pytest.approx((32 * sweeps + 52) * cells / 0.050e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6780.0)
    # FP64 fields double every field byte
    d = bench.roofline2(km, cells, "f64", sweeps, 6780.0, "measured", sor_launches=1)
    assert d["alg_bytes_per_cell"] == 2 * r["alg_bytes_per_cell"]
    # one launch a round: the sweeps' bytes spread over the launches, the
    # gradient, total and rescale in groups of their own
    per = bench.roofline2(km, cells, "f32", sweeps, 6780.0, "measured", sor_launches=2)
    assert per["alg_bytes_per_cell"] == 32 * sweeps
    assert per["alg_bytes_per_launch"] == 32 * sweeps * cells / 2
    assert per["avg_launch_ms"] == pytest.approx(0.025)
    # the fused LB-FD kernel
    assert bench.alg_bytes_2d("collide", "f32") == 2 * (16 * 4 + 2 * 4 + 1) + 27 * 4
    assert bench.alg_bytes_2d("collide", "f16") == 2 * (16 * 2 + 2 * 4 + 1) + 27 * 4
    km2 = dict(km, collide=0.060)
    c = bench.roofline2(km2, cells, "f32", sweeps, 6780.0, "measured", sor_launches=1)
    assert c["kernel"] == "collide" and c["alg_bytes_per_cell"] == 254


def test_step_roofline(bench):
    r = bench.step_roofline(2000.0, "d2q9", "f32", 6780.0, "L2")
    assert r["b_alg_per_cell"] == 176 and r["achieved_gbs"] == pytest.approx(352.0)
    assert bench.step_roofline(1.0, "d3q19", "bf16", 1.0, "")["b_alg_per_cell"] == 184
    assert bench.step_roofline(1.0, "d3q19", "f32", 1.0, "")["b_alg_per_cell"] == 336
    assert bench.step_roofline(1.0, "d2q9", "f16", 1.0, "")["b_alg_per_cell"] == 104


def test_traffic_table_shape(bench):
    # DRAM bytes a cell of each fused 2D kernel from an ncu capture, tied to
    # the hash of the files that hold the kernels' device code (the bench
    # reports them only while that hash matches)
    t = bench.TRAFFIC
    assert len(t["kernel_sha"]) == 16 and int(t["kernel_sha"], 16) >= 0
    for table in ("bytes_per_cell", "bytes_per_cell_hbm"):
        for variant, per in t[table].items():
            assert 0 <= int(variant) <= 8
            for k, v in per.items():
                assert k in ("collide", "sor") and v > 0
    # valid only for the captured source, form and tile variants
    ok = bench.src_hash(bench.FUSED2_FILES) == t["kernel_sha"]
    v = int(next(iter(t["bytes_per_cell"])))
    assert bench.traffic_valid(1, v) == ok
    assert not bench.traffic_valid(3, v)
    missing = next(k for k in range(9) if str(k) not in t["bytes_per_cell"])
    assert not bench.traffic_valid(1, missing)
    assert set(bench.FUSED2_FILES) == {"lbs_dev.cuh", "lbs_k2d.cuh", "lbs_fused2.cuh"}
    assert bench.src_hash(bench.FUSED2_FILES) != bench.src_hash()
