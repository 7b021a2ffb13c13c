"""Host-side logic of bench.py (CPU only): the kernel-source hash that decides
whether a committed ncu figure still describes the kernels, and the lookup of
that figure."""
import json

import bench


def test_code_only_drops_comments_and_whitespace():
    a = "int f(int x) {  // the identity\n  return x; /* plain */ }\n"
    b = "int f(int x){return x;}"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only("int f(int x){return x+1;}")


def test_committed_traffic_is_used_only_for_the_hashed_sources(tmp_path, monkeypatch):
    rec = {"fp64_volume_3d_n3": {"bytes_per_node": 182.4, "fp64_flops_executed_per_node": 497.2,
                                 "src_sha": bench.source_sha()}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_sha", lambda: rec["fp64_volume_3d_n3"]["src_sha"])
    assert bench.ncu_traffic("fp64_volume_3d_n3") == 182.4
    assert bench.ncu_record("fp64_volume_3d_n3", "fp64_flops_executed_per_node") == 497.2
    assert bench.ncu_traffic("fp64_volume_2d_n3") is None
    monkeypatch.setattr(bench, "source_sha", lambda: "000000000000")
    assert bench.ncu_traffic("fp64_volume_3d_n3") is None


def test_volume_flops_per_node_formula():
    # 3D N = 3: 4.5 pairs per node of 81 flop, a 12-flop prologue and the
    # lifting at the line ends
    assert abs(bench.volume_flops_per_node(3, 3) - 391.5) < 1e-9


def test_traffic_records_of_other_kernel_families_use_their_own_sources(tmp_path, monkeypatch):
    files = bench.MHD_KERNEL_SOURCES
    rec = {"fp64_mhd_volume_n3": {"bytes_per_node": 130.0, "sources": list(files),
                                  "src_sha": bench.source_sha(files)}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))
    real_root = bench.ROOT
    sha = bench.source_sha(files)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_sha",
                        lambda f=bench.KERNEL_SOURCES: sha if f == files else "000000000000")
    assert bench.ncu_traffic("fp64_mhd_volume_n3") == 130.0
    monkeypatch.setattr(bench, "source_sha", lambda f=bench.KERNEL_SOURCES: "111111111111")
    assert bench.ncu_traffic("fp64_mhd_volume_n3") is None
    assert real_root


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle on a bounded sample, CPU only)
    prints one JSON line with the contract's keys."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--workload",
                        "euler3d_n3_32cubed_wave"], capture_output=True, text=True, timeout=600,
                       cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_mhd_cpu_baseline_times_both_solvers():
    out = bench.mhd_cpu_baseline(6, seconds=0.3)
    assert out["kind"] == "oracle" and out["cores"] >= 1
    for key in ("weak_form_hll", "ec_flux_differencing"):
        assert out[key]["value"] > 0 and "oracle rhs" in out[key]["sample"]
