"""Host-side pieces of the benchmark, on CPU: the closed forms its parity checks use against the
oracle, the roofline arithmetic, and the rule that a recorded DRAM traffic figure is used only
while the kernel sources it was taken on are unchanged."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402

BC = {bench.W.PER: oracle.PER, bench.W.UNB: oracle.UNB}


def _oracle_field(name):
    wl = bench.workload(name)
    prob = oracle.Problem(bc=tuple((BC[a], BC[b]) for a, b in wl["bc"]), h=tuple(1.0 / n for n in wl["n"]),
                          center=oracle.CELL, kernel=wl["kernel"])
    return wl, oracle.solve(wl["rhs"](), prob)


@pytest.mark.parametrize("name,tol", [("per32_f64", 1e-13), ("unb32_f64", 1e-5)])
def test_closed_form_planes_agree_with_the_oracle(name, tol):
    # periodic sine products: the spectral solve is exact; unbounded Gaussian: the HEJ2-smoothed
    # potential, up to the blob's truncation at the box and the sampling of the right-hand side
    wl, ref = _oracle_field(name)
    z = bench.sample_planes(wl["n"][2])
    cf = bench.closed_form_planes(wl, z)
    assert bench.rel_linf(ref[z], cf) < tol


def test_roofline_of_the_dominant_pass(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: (6790.0, "measured"))
    monkeypatch.setattr(bench, "traffic_record", lambda k, w: None)
    pinfo = [{"kind": 0, "bytes": 1e9, "flops": 1e9}, {"kind": 5, "bytes": 4e9, "flops": 8e9}]
    roof = bench.roofline(pinfo, np.array([0.5, 2.0]), 0, {}, "unb512_f32")
    assert roof["kernel"] == "k_fused_c2c" and roof["bound"] == "hbm"
    assert roof["achieved"] == pytest.approx(4e9 / 2e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6790.0)
    # native FP64 against the measured FP64 FMA rate
    roof64 = bench.roofline(pinfo, np.array([0.5, 2.0]), 1, {"fp64_tflops": 1.25}, "unb512_f64")
    assert roof64["bound"] == "alu" and roof64["frac"] == pytest.approx(8e9 / 2e-3 / 1e12 / 1.25)


def test_traffic_record_needs_the_current_kernel_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    sha = bench.kernel_source_sha()
    (prof / "traffic.json").write_text(json.dumps({
        "k_fused_c2c@unb512_f32": {"source_sha": sha, "dram_bytes_per_launch": 4.6e9},
        "k_fused_c2c@unb512_f64": {"source_sha": "0" * 16, "dram_bytes_per_launch": 9.9e9}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: sha)
    assert bench.traffic_record("k_fused_c2c", "unb512_f32") == 4.6e9
    assert bench.traffic_record("k_fused_c2c", "unb512_f64") is None      # other sources
    assert bench.traffic_record("k_inv_real", "unb512_f32") is None       # no record
