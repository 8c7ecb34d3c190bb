"""Host logic of bench.py's roofline (no GPU): the per-class fractions are
the algorithmic flops per launch over the launch time and the FP64 peak
derived from the unit count, the measured FP64 issue rate per SM per clock
and the clock, with the nominal peak (2 per SM per clock) beside them; the
dominant class is the one with the most device time; the flops per
zone-cycle are the per-unit counts scaled to the grid's own faces and
zones."""
import math

import pytest

import bench
from paper_2110_10191_gb300 import problems as pb


class _Pr:
    def __init__(self, n, precision=0):
        self.n = n
        self.precision = precision


CPU = {"_face_flops_per_face": 1000.0, "_recon_flops_per_face": 700.0,
       "_update_flops_per_zone_stage": 2500.0}


def _prof(n, ms):
    return {"flux": (3 * ms["flux"], 3), "recon": (3 * ms["recon"], 3),
            "update": (ms["update"], 1), "ct": (0.1, 2)}


def test_derived_peaks():
    assert bench.FP64_PEAK_NOMINAL == pytest.approx(152 * 2 * 2 * 2.07e9)
    assert bench.fp64_peak_sustained(2.0) == pytest.approx(bench.FP64_PEAK_NOMINAL)
    assert bench.fp64_peak_sustained(1.683) == pytest.approx(152 * 1.683 * 2 * 2.07e9)


FP64 = {"rate": 1.5, "mhz": 2070.0}


def test_fractions_and_dominant_class():
    n = (16, 12, 8)
    zones = n[0] * n[1] * n[2]
    faces = bench.faces_per_launch(n)
    ms = {"flux": 0.5, "recon": 0.9, "update": 1.2}
    peak = 152 * 1.5 * 2 * 2.07e9
    roof, kernels, fzc = bench.build_roofline(_prof(n, ms), CPU, _Pr(n), zones, FP64, "torus128")
    flops = {"flux": CPU["_face_flops_per_face"] * sum(faces) / 3.0,
             "recon": CPU["_recon_flops_per_face"] * sum(faces) / 3.0,
             "update": CPU["_update_flops_per_zone_stage"] * zones}
    for c in ("flux", "recon", "update"):
        rate = flops[c] / (ms[c] * 1e-3)
        assert kernels[c]["avg_launch_ms"] == pytest.approx(ms[c])
        assert kernels[c]["frac"] == pytest.approx(rate / peak)
        assert kernels[c]["frac_of_nominal"] == pytest.approx(rate / bench.FP64_PEAK_NOMINAL)
    # most device time: recon (3 x 0.9 ms) over flux (1.5) and update (1.2)
    assert roof["kernel"].startswith("kp_recon")
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert roof["peak"] == pytest.approx(peak / 1e12)
    assert roof["peak_nominal"] == pytest.approx(bench.FP64_PEAK_NOMINAL / 1e12)
    assert roof["frac"] == pytest.approx(kernels["recon"]["frac"])
    assert roof["achieved"] == pytest.approx(roof["frac"] * roof["peak"])
    # per zone-cycle: two stages of every face and zone
    want = 2 * ((1000.0 + 700.0) * sum(faces) + 2500.0 * zones) / zones
    assert fzc == pytest.approx(want)


def test_no_roofline_off_the_fp64_headline():
    n = (16, 12, 8)
    zones = n[0] * n[1] * n[2]
    prof = _prof(n, {"flux": 0.5, "recon": 0.9, "update": 1.2})
    for pr, variant, cpu in ((_Pr(n, precision=1), "none", CPU), (_Pr(n), "drift", CPU),
                             (_Pr(n), "none", None)):
        roof, kernels, fzc = bench.build_roofline(prof, cpu, pr, zones, FP64, "torus128", variant)
        assert roof is None and kernels == {} and fzc is None


def test_traffic_only_for_the_captured_sources(monkeypatch):
    n = (16, 12, 8)
    zones = n[0] * n[1] * n[2]
    prof = _prof(n, {"flux": 0.5, "recon": 0.9, "update": 1.2})
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: bench.NCU_TRAFFIC["src_hash"])
    roof, kernels, _ = bench.build_roofline(prof, CPU, _Pr(n), zones, FP64, "torus128")
    assert roof["traffic"] == bench.NCU_TRAFFIC["torus128"]["recon"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    roof, kernels, _ = bench.build_roofline(prof, CPU, _Pr(n), zones, FP64, "torus128")
    assert roof["traffic"] is None and kernels["update"]["fp64_pipe_ncu"] is None


def test_headline_workload_recipe():
    pr = bench.make_problem("torus128")
    assert tuple(pr.n) == (128, 128, 128) and pr.recon == pb.RECON_WENO5
    assert math.isclose(pr.a, 0.9375)
