"""The benchmark's JSON-line contract, checked on its CPU reference arm (the
oracle on the host cores) for two workloads."""
import json
import os
import subprocess
import sys

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def reference_line(workload, *extra):
    out = subprocess.run([sys.executable, os.path.join(REPO, "bench.py"), "--impl", "reference", "--workload",
                          workload, "--steps", "1", "--warmup", "0", *extra], cwd=REPO, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("workload", ["web-10k", "kpid-1m", "kpid-sim"])
def test_reference_arm_prints_one_contract_line(workload):
    d = reference_line(workload)
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["data"] == "synthetic" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]
    if workload == "web-10k":
        # the native line's headline: solves per second to the tolerance
        assert d["metric"] == "solves_per_s_to_tol" and d["unit"] == "solves/s" and d["higher_is_better"] is True


def test_kpid_reference_with_the_completion():
    # the oracle's K-PID emulation with completed dangling columns, on its
    # smaller sample; the line names the completion
    plain = reference_line("kpid-1m")
    d = reference_line("kpid-1m", "--dangling")
    assert d["config"]["dangling"] == "uniform 1/N completion"
    assert plain["config"]["dangling"] == "zero columns"
    assert "N=2e+04" in d["config"]["sample"] and "N=1e+05" in plain["config"]["sample"]
    # a completed column counts N elementary diffusions: far above the plain cost
    assert d["value"] > 10 * plain["value"]


def test_warm_start_reference_uses_the_native_metric():
    # the native warm-start line reports time to tol (lower is better); its
    # reference arm must report the same metric and unit
    d = reference_line("warmstart")
    assert d["metric"] == "time_to_tol_ms" and d["unit"] == "ms" and d["higher_is_better"] is False


def test_kpid_simulation_line_covers_the_papers_grid():
    # the host-core simulation of K PIDs (no GPU): every K of the grid, both
    # partitions, the delays at K = 8; idle shares in [0, 1) and speed-ups > 1
    out = subprocess.run([sys.executable, os.path.join(REPO, "bench.py"), "--workload", "kpid-sim"], cwd=REPO,
                         capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][0])
    assert d["metric"] == "kpid_speedup" and d["value"] > 1
    rows = d["rows"]
    assert {r["K"] for r in rows} == {1, 2, 4, 8, 16, 32, 64}
    assert {r["delay_proba"] for r in rows} == {0.0, 0.5, 0.8}
    assert all(r["status"] == 0 and 0.0 <= r["idle_share"] < 1.0 for r in rows)
    assert all(r["speedup"] > 1 for r in rows if r["K"] > 1 and r["delay_proba"] == 0.0)


def test_level_traffic_lookup_reads_the_committed_captures():
    # the roofline's "traffic" comes from profiles/level_traffic.txt, keyed by
    # workload, precision, propagation and slice sweeps per level; a
    # configuration without a capture reports null
    sys.path.insert(0, REPO)
    import bench
    with_sweeps = bench.level_traffic("web-1m", "f32", 3, 1)
    without = bench.level_traffic("web-1m", "f32", 3, 0)
    assert with_sweeps is not None and without is not None
    assert 1e7 < with_sweeps < 2e8 and 1e7 < without < 2e8
    assert bench.level_traffic("stress-16m", "f32", 3, 1) is None
    assert bench.level_traffic("web-1m", "f64", 3, 1) is None
