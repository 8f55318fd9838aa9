"""bench.py's roofline bookkeeping: the algorithmic bytes per cell update of each kernel and
step, the DRAM traffic it reports only for the kernel sources the counters were taken on, and
the CPU-baseline plan entry."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("precision,psi,fused,step", [("fp32", 80, 156, 236), ("fp16s", 42, 80, 122),
                                                      ("fp16s_sr", 42, 80, 122), ("fp64", 160, 312, 472)])
def test_two_pass_byte_model(precision, psi, fused, step):
    # D3Q19: psi pass reads 19 populations and writes psi; the fused pass reads 19 populations
    # and psi and writes 19 populations
    b = bench.bytes_per_cell(precision)
    assert (b["psi_pass"], b["fused_pass"], b["step"]) == (psi, fused, step)


@pytest.mark.parametrize("precision,step", [("fp32", 152), ("fp16s", 76)])
def test_single_pass_byte_model(precision, step):
    b = bench.bytes_per_cell(precision, streaming="fused")
    assert b["step"] == b["fused_pass"] == step and b["psi_pass"] == 0


def test_d2q9_byte_model():
    assert bench.bytes_per_cell("fp32", q=9)["step"] == 3 * 9 * 4 + 2 * 4 == 116


def test_traffic_is_reported_only_for_the_recorded_sources(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    table = ("| workload | kernel | dram bytes per launch at full size | per cell | algorithmic |\n"
             "|---|---|---|---|---|\n"
             "| wl_a | k_collide_pair | 4.705e9 | x | y |\n"
             "| wl_a | k_fused_pair | 5.94e9 | x | y |\n")
    sha = bench.kernel_source_sha()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # kernel_source_sha reads the CUDA sources under ROOT; keep the real ones
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: sha)
    (tmp_path / "profiles" / "roofline_traffic.md").write_text(f"kernel_source_sha: {sha}\n\n" + table)
    assert bench.recorded_traffic("wl_a", "k_collide_pair") == 4.705e9
    assert bench.recorded_traffic("wl_a", "k_fused_pair") == 5.94e9
    assert bench.recorded_traffic("wl_b", "k_collide_pair") is None
    (tmp_path / "profiles" / "roofline_traffic.md").write_text("kernel_source_sha: 0123456789abcdef\n\n" + table)
    assert bench.recorded_traffic("wl_a", "k_collide_pair") is None


def test_cpu_plan_entry_times_the_oracle_in_a_child_process():
    """One entry of the CPU-baseline plan (the oracle alone, thread count from OMP_NUM_THREADS)
    runs in its own process and reports three positive rates."""
    import json
    import subprocess
    import sys
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-plan-child", "d2q9_bgk_256x256_droplet:2"],
                       env=env, capture_output=True, text=True, check=True, timeout=300)
    mlups = json.loads(r.stdout.strip().splitlines()[-1])["mlups"]
    assert len(mlups) == 3 and all(v > 0 for v in mlups)
