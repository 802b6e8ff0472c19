"""bench.py's roofline arithmetic on made-up inputs (CPU only): achieved = algorithmic work per
launch / measured time, frac = achieved / the measured peak, the work counts of the two
rooflines (the field's evaluations M * E * Q * Nk, the LU's (8/3) N^3 per system)."""
import os
import sys
from types import SimpleNamespace

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _w(N, E):
    return SimpleNamespace(mesh=SimpleNamespace(N=N, E=E))


def test_field_roofline_arithmetic():
    w = _w(2884, 1440)
    peaks = {"ffma_tflops": 78.0, "sm_count": 152}
    r = bench.roofline_field(w, 500.0, 16384, 512, 2, peaks)
    evals = 16384 * 1440 * 16 * 512
    assert r["evals_per_s"] == pytest.approx(evals / 0.5)
    assert r["achieved"] == pytest.approx(bench.FIELD_FLOPS_PER_EVAL * evals / 0.5 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 78.0)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["launches_per_step"] == 1
    assert r["traffic"] == bench.FIELD_LAUNCH_DRAM_BYTES[2]
    assert bench.roofline_field(w, 500.0, 16384, 1024, 1, peaks)["launches_per_step"] == 2
    assert bench.roofline_field(w, 500.0, 16384, 512, 1, peaks)["traffic"] is None  # no capture


def test_lu_roofline_arithmetic():
    w = _w(2884, 1440)
    ph = {"systems": 512, "factor_ms": 200.0, "assembly_ms": 1.0, "refine_ms": 2.0, "reassembly_ms": 3.0}
    r = bench.roofline_lu(w, ph, {"tf32_tflops": 1200.0})
    flops = 512 * (8.0 / 3.0) * 2884.0 ** 3
    assert r["achieved"] == pytest.approx(flops / 0.2 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1200.0)
    assert r["bound"] == "tensor" and r["phase_ms"]["reassembly_ms"] == 3.0
    ph0 = dict(ph, factor_ms=0.0)
    assert bench.roofline_lu(w, ph0, {"tf32_tflops": 1200.0})["frac"] is None
