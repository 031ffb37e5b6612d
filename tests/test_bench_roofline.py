"""bench.py's roofline arithmetic: per class, achieved = algorithmic bytes
summed over the timed launches / their summed event time, frac = achieved /
peak; the roofline record is the class with the most time per step, with its
DRAM traffic scaled from the ncu ratio of bytes moved per algorithmic byte."""
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def _prof(ms, launches, bytes_per_launch):
    return {"ms": ms, "launches": launches, "bytes": bytes_per_launch * launches}


def _bench():
    sys.path.insert(0, str(ROOT))
    import bench
    return bench


def test_achieved_bandwidth_and_dominant_class():
    bench = _bench()
    steps = 20
    # per step: 18 Chebyshev launches of 808.45 MB in 2.5225 ms, and so on
    prof = {
        "helm_sweep": _prof(2.522462 * steps, 18 * steps, 808452096.0),
        "multidot": _prof(1.016678 * steps, 14 * steps, 354718281.0),
        "axpy_norm": _prof(1.101381 * steps, 14 * steps, 421827145.0),
        "laplacian_f64": _prof(1.297525 * steps, 16 * steps, 150994944.0),
        "mg_smooth_fine": _prof(1.838854 * steps, 42 * steps, 178956971.0),
    }
    roof, classes = bench.roofline(prof, steps, 6787.9, "measured")
    assert roof["kernel"].startswith("k_helm_cheb_v4")
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s" and roof["peak"] == 6787.9
    # 18 x 808.45 MB in 2.5225 ms
    expect = 18 * 808452096.0 / 2.522462e-3 / 1e9
    assert roof["achieved"] == pytest.approx(expect, rel=1e-12)
    assert roof["frac"] == pytest.approx(expect / 6787.9, rel=1e-12)
    assert roof["avg_launch_ms"] == pytest.approx(2.522462 / 18, rel=1e-12)
    assert roof["bytes_per_launch"] == pytest.approx(808452096.0)
    # no ncu ratio taken on the current build of the Chebyshev step: traffic null
    assert "helm_sweep" not in bench.NCU_TRAFFIC_RATIO and roof["traffic"] is None
    assert len(classes) == 5
    for v in classes.values():
        assert v["achieved_gbs"] == pytest.approx(
            v["bytes_per_launch"] / (v["avg_launch_ms"] * 1e-3) / 1e9, rel=1e-12)


def test_class_without_launches_reads_zero():
    bench = _bench()
    prof = {c: _prof(0.0, 0, 0.0) for c in bench.ROOFLINE_CLASSES.values()}
    prof["multidot"] = _prof(4.0, 8, 1e8)
    roof, classes = bench.roofline(prof, 2, 1000.0, "fallback")
    assert roof["kernel"].startswith("k_multidot_sp4")
    assert roof["traffic"] == pytest.approx(bench.NCU_TRAFFIC_RATIO["multidot"] * 1e8)
    assert roof["achieved"] == pytest.approx(8 * 1e8 / 4e-3 / 1e9)
    assert roof["peak_kind"] == "fallback"
    zero = [v for v in classes.values() if v["ms_per_step"] == 0.0]
    assert len(zero) == 4 and all(v["achieved_gbs"] == 0.0 for v in zero)
