"""Host-side helpers of bench.py that the reported JSON line depends on (no GPU):
the comment-free kernel hash that keys the committed DRAM-traffic record, the
lookup of that record, and the summary of the clock samples taken during the
timed region (throttle reasons flagged)."""
import json
import os
import shutil

import pytest

import bench

CSRC = os.path.join(bench.ROOT, "paper_1612_06424_gb300", "csrc")


def test_strip_comments():
    src = "int a = 1;  // one\n// a whole comment line\n\n  float b;   \n"
    assert bench._strip_comments(src) == "int a = 1;\n  float b;"


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    d = tmp_path / "paper_1612_06424_gb300" / "csrc"
    d.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(CSRC, f), d / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_kernel_hash_ignores_comments_only(fake_root):
    h0 = bench._kernel_hash()
    p = fake_root / "paper_1612_06424_gb300" / "csrc" / "dslash.cuh"
    p.write_text(p.read_text() + "\n// a note that changes no code\n")
    assert bench._kernel_hash() == h0
    p.write_text(p.read_text() + "\nnamespace lq { constexpr int k_extra = 1; }\n")
    assert bench._kernel_hash() != h0


def test_traffic_record_used_only_for_matching_source(fake_root):
    rec = {"32:1": {"kernel_hash": bench._kernel_hash(), "dram_bytes_per_launch": 123456, "system_sites": 1000}}
    path = fake_root / "profiles" / "dslash_traffic.json"
    path.write_text(json.dumps(rec))
    assert bench._traffic(32, 1) == pytest.approx(123.456)
    assert bench._traffic(32, 2) is None
    assert bench._traffic(16, 1) is None
    rec["32:1"]["kernel_hash"] = "0" * 16
    path.write_text(json.dumps(rec))
    assert bench._traffic(32, 1) is None


def test_cpu_cost_counts_site_applications():
    """The extrapolated oracle time: every solve's sites x (2 per iteration + 2), scaled by the
    measured seconds per round over the sample's sites."""
    wl = dict(bench.WL16)
    s3 = 16 ** 3
    iters = {"gamma": 10, "gamma_bar": 20, "gamma_star": 30, "full": 40}
    sites = {"gamma": 14 * s3, "gamma_bar": 18 * s3, "gamma_star": 18 * s3, "full": 32 * s3}
    want = sum(sites[k] * (2 * iters[k] + 2) for k in iters) * 2.0 / s3
    assert bench._cpu_cost(2.0, s3, wl, iters) == pytest.approx(want)


def test_clock_summary_flags_throttle_reasons():
    c = bench.Clocks()
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2070, 1390.5, 0x8, Active, Not Active, Not Active, Not Active"]
    c.f.write("\n".join(rows) + "\n")
    s = c.summary()
    os.unlink(c.f.name)
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples():
    c = bench.Clocks()
    s = c.summary()
    os.unlink(c.f.name)
    assert s["reasons"] == ["unsampled"] and s["sm_mhz"] is None


def test_nucleon_roofline_counts_three_tf32_passes(fake_root):
    """The tensor-core block contraction is reported against the TF32 peak derived from the
    measured bf16 peak (x 1.1 / 2.25), with three TF32 passes per contraction flop."""
    (fake_root / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6000.0, "bf16_tflops": 2250.0}))
    r = bench._nucleon_roofline(1.0e14, 1.0, 77.0, 120, 41, 13824)
    assert r["bound"] == "tensor" and r["peak"] == pytest.approx(1100.0)
    assert r["contraction_tflops"] == pytest.approx(100.0)
    assert r["achieved"] == pytest.approx(300.0) and r["frac"] == pytest.approx(300.0 / 1100.0, rel=1e-3)
    (fake_root / "MEASURED_PEAKS.json").unlink()
    assert bench._tf32_peak()[1].startswith("fallback")
