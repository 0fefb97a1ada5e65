"""Host-side logic of bench.py (CPU only): the algorithmic-bytes and FLOP models behind the
roofline entry, the DRAM-traffic record's binding to the kernel sources, the clock-sample
parser, the plaquette used for the clover coefficients and the sizing of the oracle sample."""

import json
import os

import numpy as np
import pytest

import bench
import synthetic as S
from oracle import clover as CL

ODD_SITES_24C128 = 24 ** 3 * 128 // 2


def test_algorithmic_bytes_of_the_schur_apply():
    """Per odd site and source: K-a 96, K-b 192 + 6 links, K-c 288 + 6 links (FP32, two-row links of 48 B)."""
    n = ODD_SITES_24C128
    assert bench.apply_bytes(n, 1) == n * 1152
    assert bench.apply_bytes(n, 12) == n * (12 * 576 + 576)                    # 6.63 GB per 12-source apply
    assert bench.launch_bytes("schur_c_hop_tinv_axpy_f32", n, 12) == n * (12 * 288 + 288)
    assert bench.launch_bytes("schur_a_tdag_f32", n, 12) == n * 12 * 96        # reads no link
    assert bench.launch_bytes("schur_b_hop_tsolve_f64", n, 1) == n * (2 * 192 + 6 * 144)
    assert bench.launch_bytes("cg_xr_f32", n, 1) is None
    assert bench.eo4d_launch_bytes("eo4d_dslash_oe_axpy_f32", n, 2) == n * (2 * 288 + 6 * 48)


def test_paper_flop_model():
    """(3432 N_t - 576)(V_s / 2) per M-hat apply (App. B, Wilson temporal + 3-D Schur)."""
    assert bench.paper_flops_per_apply(24, 128) == (3432 * 128 - 576) * (24 ** 3 // 2)


def test_traffic_record_binding(tmp_path, monkeypatch):
    """A DRAM traffic record counts only for its kernel sources, workload, source count and the
    hop-kernel configuration it was captured in."""
    cfg = bench.hop_config_key({"variant": "one thread per site", "tile_rows": 6})
    assert cfg == "variant=one thread per site;tile_rows=6"
    assert bench.hop_config_key({"variant": "bulk-copy-fed", "tile_rows": 4, "sources_per_unit": 1, "stages": 3}) == \
        "variant=bulk-copy-fed;tile_rows=4;sources=1;stages=3"
    assert bench.hop_config_key(None) is None
    rec = {"source_hash": bench.source_hash(),
           "kernels": {"schur_c_hop_tinv_axpy_f32": {"workload": bench.WORKLOAD, "nrhs": 12, "config": cfg,
                                                     "dram_bytes_per_launch": 3.6e9}}}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    k = "schur_c_hop_tinv_axpy_f32"
    assert bench.traffic_for(k, 12, cfg, str(path)) == 3.6e9
    assert bench.traffic_for(k, 1, cfg, str(path)) is None                                  # other source count
    assert bench.traffic_for(k, 12, "variant=one thread per site;tile_rows=8", str(path)) is None  # other traversal
    assert bench.traffic_for("schur_b_hop_tsolve_f32", 12, cfg, str(path)) is None          # not captured
    assert bench.traffic_for(k, 12, cfg, str(tmp_path / "absent.json")) is None
    # several captured configurations of one kernel
    cfg8 = "variant=one thread per site;tile_rows=8"
    rec["kernels"][k] = [rec["kernels"][k], dict(rec["kernels"][k], config=cfg8, dram_bytes_per_launch=3.9e9)]
    path.write_text(json.dumps(rec))
    assert bench.traffic_for(k, 12, cfg, str(path)) == 3.6e9
    assert bench.traffic_for(k, 12, cfg8, str(path)) == 3.9e9
    assert bench.traffic_for(k, 12, "variant=one thread per site;tile_rows=4", str(path)) is None
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 16)                             # kernels changed
    assert bench.traffic_for(k, 12, cfg, str(path)) is None


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_parses_nvidia_smi_rows(tmp_path):
    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "0, 2070, 2070, 1380.5, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "garbage line\n")
    c = bench.ClockSampler(0)
    c.path, c.proc, c.fh = str(path), _DoneProc(), open(os.devnull, "w")
    r = c.stop()
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_sampler_flags_thermal_slowdown(tmp_path):
    path = tmp_path / "clocks.csv"
    path.write_text("0, 1500, 2070, 1400.0, 0x40, Not Active, Active, Not Active, Active\n")
    c = bench.ClockSampler(0)
    c.path, c.proc, c.fh = str(path), _DoneProc(), open(os.devnull, "w")
    assert c.stop()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_sampler_without_nvidia_smi():
    c = bench.ClockSampler(0)
    c.proc = None
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_spatial_plaquette():
    assert bench.spatial_plaquette(S.unit_gauge(4, 4)) == pytest.approx(1.0, abs=1e-15)
    U = S.random_gauge(4, 6, 0.3, 5)
    leaves = np.mean([np.real(np.trace(CL.clover_leaves(U, i, j), axis1=-2, axis2=-1)).mean() / 12.0
                      for (i, j) in CL.SPATIAL_PLANES])   # four leaves per site, each averaging the plaquette
    assert bench.spatial_plaquette(U) == pytest.approx(leaves, rel=1e-13)


def test_oracle_sample_is_small_and_even():
    """The CPU baseline runs one spawned process per core, all applying at once."""
    prm = dict(S.WORKLOADS["wilson_4c16_xi3"])
    gbs, desc, procs, dt = bench.oracle_sample(0.01, prm, procs=2)
    assert gbs > 0 and procs == 2 and dt > 0
    assert "4^3x16" in desc and "2 concurrent" in desc
