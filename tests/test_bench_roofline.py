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
        "schur_markers": _prof(1.03 * steps, 16 * steps, 125e6),
        "mg_smooth_fine": _prof(1.838854 * steps, 42 * steps, 178956971.0),
        "vcycle": _prof(4.07 * steps, 14 * steps, 0.95e9),
        "solve": _prof(9.53 * steps, steps, 26.0e9),
    }
    roof, classes, solve = bench.roofline(prof, steps, 6787.9, "measured")
    # the predictor's Chebyshev step takes longest but is not part of the
    # solve: the record names the solve's longest class
    assert roof["kernel"].startswith("k_first_v4 + k_sweep_v4")
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s" and roof["peak"] == 6787.9
    expect = 42 * 178956971.0 / 1.838854e-3 / 1e9
    assert roof["achieved"] == pytest.approx(expect, rel=1e-12)
    assert roof["frac"] == pytest.approx(expect / 6787.9, rel=1e-12)
    assert roof["avg_launch_ms"] == pytest.approx(1.838854 / 42, rel=1e-12)
    assert roof["bytes_per_launch"] == pytest.approx(178956971.0)
    assert roof["traffic"] == pytest.approx(bench.NCU_TRAFFIC_RATIO["mg_smooth_fine"] * 178956971.0)
    assert len(classes) == len(bench.ROOFLINE_CLASSES)
    for v in classes.values():
        assert v["achieved_gbs"] == pytest.approx(
            v["bytes_per_launch"] / (v["avg_launch_ms"] * 1e-3) / 1e9, rel=1e-12)
    # the whole solve: 26 GB in 9.53 ms
    assert solve["bytes_per_solve"] == pytest.approx(26.0e9)
    assert solve["ms_per_solve"] == pytest.approx(9.53)
    assert solve["frac"] == pytest.approx(26.0e9 / 9.53e-3 / 1e9 / 6787.9, rel=1e-12)


def test_class_without_launches_reads_zero():
    bench = _bench()
    prof = {c: _prof(0.0, 0, 0.0) for c in bench.ROOFLINE_CLASSES.values()}
    prof["solve"] = _prof(0.0, 0, 0.0)
    prof["multidot"] = _prof(4.0, 8, 1e8)
    roof, classes, solve = bench.roofline(prof, 2, 1000.0, "fallback")
    assert roof["kernel"].startswith("k_multidot_sp4")
    assert roof["traffic"] == pytest.approx(bench.NCU_TRAFFIC_RATIO["multidot"] * 1e8)
    assert roof["achieved"] == pytest.approx(8 * 1e8 / 4e-3 / 1e9)
    assert roof["peak_kind"] == "fallback"
    zero = [v for v in classes.values() if v["ms_per_step"] == 0.0]
    assert len(zero) == len(classes) - 1 and all(v["achieved_gbs"] == 0.0 for v in zero)
    assert solve["achieved"] == 0.0
