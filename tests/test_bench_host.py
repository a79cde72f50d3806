"""Host logic of bench.py, on the CPU: the clock samples kept for the timed
region, the gating of the committed ncu figures by the kernel-source hash,
and the whole-job throughput."""
import datetime
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _row(t, sm, reasons=("Not Active",) * 4):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([ts, "0", str(sm), "2070", "900.00", "0x0"] + list(reasons))


def _clocks(tmp_path, rows, t0, t1):
    c = bench.Clocks.__new__(bench.Clocks)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    c.f = open(c.path, "a")

    class P:  # a finished sampler process
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.proc = P()
    c.t0, c.t1 = t0, t1
    return c


def test_clock_samples_inside_the_region(tmp_path):
    t0 = 1_700_000_000.0
    rows = [_row(t0 - 0.5, 1400), _row(t0 + 0.01, 2070), _row(t0 + 0.03, 2060),
            _row(t0 + 0.5, 1500, ("Not Active", "Not Active", "Not Active", "Active"))]
    out = _clocks(tmp_path, rows, t0, t0 + 0.05).stop()
    assert out["samples"] == 2 and out["sm_mhz"] == 2065.0
    assert out["reasons"] == [] and out["sm_max_mhz"] == 2070.0


def test_clock_nearest_sample_for_a_short_region(tmp_path):
    t0 = 1_700_000_000.0
    rows = [_row(t0 - 0.2, 1300),
            _row(t0 + 0.06, 2070, ("Active", "Not Active", "Not Active", "Not Active"))]
    out = _clocks(tmp_path, rows, t0, t0 + 0.01).stop()
    assert out["samples"] == 1 and out["sm_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown"]


def test_ncu_figures_only_for_the_hashed_sources(tmp_path, monkeypatch):
    f = tmp_path / "traffic.txt"
    f.write_text(f"# comment\nkernel_hash = {bench.kernel_hash('depth_first')}\n"
                 "dram_bytes_per_segment = 8.5\nissue_active_pct = 77.0\n")
    monkeypatch.setitem(bench.TRAFFIC_FILE, "depth_first", str(f))
    assert bench.ncu_summary("depth_first") == {"dram_bytes_per_segment": 8.5,
                                                 "issue_active_pct": 77.0}
    f.write_text("kernel_hash = 0000000000000000\ndram_bytes_per_segment = 8.5\n")
    assert bench.ncu_summary("depth_first") is None


def test_kernel_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    src = tmp_path / "k.cuh"
    src.write_text("// a kernel\n__device__ int f(int x) { return x + 1; }  /* one */\n")
    monkeypatch.setitem(bench.KERNEL_SOURCES, "depth_first", [str(src)])
    monkeypatch.setattr(bench, "ROOT", "/")
    h0 = bench.kernel_hash("depth_first")
    src.write_text("// the same kernel, reworded\n__device__ int f(int x)\n{\n  return x + 1;\n}\n")
    assert bench.kernel_hash("depth_first") == h0
    src.write_text("__device__ int f(int x) { return x + 2; }\n")
    assert bench.kernel_hash("depth_first") != h0


def test_committed_traffic_files_match_the_sources():
    # the committed captures were taken on the code now in the tree
    for form in ("depth_first", "breadth_first"):
        assert bench.ncu_summary(form) is not None, form


def test_committed_traffic_files_parse():
    for form in ("depth_first", "breadth_first"):
        kv = {}
        for line in open(bench.TRAFFIC_FILE[form]):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
        assert len(kv["kernel_hash"]) == 16
        assert float(kv["dram_bytes_per_segment"]) > 0


def test_job_throughput():
    assert bench.job_throughput(1000, 4, 500.0) == pytest.approx(8000.0)


def test_traversal_roofline_issue_bound():
    ncu = {"warp_inst_per_segment": 140.0, "dram_bytes_per_segment": 9.0, "l2_hit_pct": 82.0}
    clk = {"sm_mhz": 2000.0}
    r = bench.traversal_roofline(2.0e11, 8.0e7, 0.01, 6800.0, "measured", ncu, clk)
    issue_peak = 152 * 4 * 2000e6 / 1e9
    assert r["bound"] == "issue" and r["peak"] == pytest.approx(issue_peak)
    assert r["achieved"] == pytest.approx(140.0 * 8.0e7 / 0.01 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / issue_peak)
    assert r["traffic"] == pytest.approx(9.0 * 8.0e7)
    assert r["dram"]["frac"] == pytest.approx(9.0 * 8.0e7 / 0.01 / 1e9 / 6800.0)
    assert r["algorithmic"]["frac_of_hbm_peak"] == pytest.approx(2.0e11 / 0.01 / 1e9 / 6800.0)
    assert r["ncu"] == {"l2_hit_pct": 82.0}
    # without a capture of this kernel source: no issue or DRAM figure
    r = bench.traversal_roofline(2.0e11, 8.0e7, 0.01, 6800.0, "measured", None, None)
    assert r["frac"] is None and r["traffic"] is None and r["dram"]["frac"] is None
    assert "maximum SM clock" in r["peak_source"]


def test_cpu_baseline_scales_only_the_ray_work():
    from paper_2303_10521_gb300 import scenes
    sc = scenes.toy_scene(seed=0)
    r = bench.run_cpu_baseline(sc, sc.frame(0), stride=50)
    frame_s = r["setup_s"] + 50 * (r["discovery_s"] + r["accept_field_s"])
    assert r["frame_s_extrapolated"] == pytest.approx(frame_s)
    assert r["value"] == pytest.approx(len(sc.frame(0).rx_pos) / frame_s)
    assert r["segments"] > 0 and r["s_per_segment"] > 0


def test_oracle_check_counts_and_errors():
    """The bench's untimed FP64 check on records and fields it is handed: a
    path set the oracle accepts with its own fields gives no rejection and
    zero error; a field perturbed by 1e-3 shows up as that error."""
    import numpy as np
    import oracle
    from paper_2303_10521_gb300 import scenes
    sc = scenes.toy_scene(seed=0)
    fr = sc.frame(0)
    o = oracle.OracleScene(sc, fr)
    p = oracle.enumerate_paths(o, 2)
    acc, _ = oracle.validate(o, p)
    p = p[acc][:40]
    rec = np.zeros((len(p), 8), np.uint32)
    rec[:, 0], rec[:, 1] = p["tx"], p["rx"]
    rec[:, 2] = p["depth"] | 0x100
    rec[:, 3:7] = p["face"]
    fields = []
    for f in sc.freqs:
        a, tau, fd = oracle.field(o, p, f)
        fields.append(np.column_stack([a.real, a.imag, tau, fd]))
    r = bench.oracle_check(sc, fr, rec, fields, rec)
    assert r["paths"] == len(p) and r["oracle_rejects"] == 0
    assert r["acceptance_disagreements"] == 0
    e = r["field_vs_fp64_oracle"][f"{sc.freqs[0] / 1e9:g} GHz"]
    assert e["max_rel_amplitude_error"] == 0.0 and e["max_phase_error_rad"] < 1e-15
    fields[0][3, 0:2] *= 1.001
    r = bench.oracle_check(sc, fr, rec, fields, None)
    e = r["field_vs_fp64_oracle"][f"{sc.freqs[0] / 1e9:g} GHz"]
    assert e["max_rel_amplitude_error"] == pytest.approx(1e-3, rel=1e-6)
