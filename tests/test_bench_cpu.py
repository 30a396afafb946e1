"""The benchmark's host-side helpers on CPU tensors: the check that the step's
three products agree, and the profiling cases of the argument parser."""
import subprocess
import sys

import pytest
import torch

import bench


def test_consistency_check_accepts_agreeing_products():
    y = torch.linspace(-3.0, 5.0, 1000, dtype=torch.float64)
    ys = y * (1 + 1e-16)
    y32 = y.float()
    out = bench.consistency_check(y, ys, y32)
    assert out["ok"]
    assert out["split_vs_plain"] <= 1e-12
    assert out["fp32_vs_plain"] <= 1e-4


@pytest.mark.parametrize("which", ["split", "fp32"])
def test_consistency_check_rejects_a_wrong_product(which):
    y = torch.linspace(-3.0, 5.0, 1000, dtype=torch.float64)
    ys = y.clone()
    y32 = y.float()
    if which == "split":
        ys[17] += 1e-9 * 5.0          # above FP64 rounding of the largest |y|
    else:
        y32[3] += 1e-3 * 5.0          # above FP32 rounding of values and x
    with pytest.raises(RuntimeError):
        bench.consistency_check(y, ys, y32)


def test_profiling_cases_in_the_parser():
    out = subprocess.run([sys.executable, bench.__file__, "--help"], capture_output=True, text=True, check=True)
    for case in ("plain", "poisson7", "stencil27"):
        assert case in out.stdout


def _small_workload():
    from paper_1106_5908_gb300 import workloads as W
    A = W.hamiltonian_like(20000, seed=61)
    return A, W.uniform(A.n_rows, 62)


def test_cpu_baseline_reports_both_node_level_forms():
    A, x = _small_workload()
    from paper_1106_5908_gb300 import model
    out = bench.cpu_baseline(A, x, model.bytes_plain(A.n_rows, A.n_cols, A.nnz), budget_s=0.4)
    assert out["kind"] == "oracle" and out["unit"] == "GB/s"
    assert out["value"] > 0 and out["cores"] >= 1
    assert out["single_thread"]["cores"] == 1 and out["single_thread"]["value"] > 0


def test_reference_arm_line(monkeypatch, capsys):
    import json
    import types
    monkeypatch.setattr(bench, "hamiltonian_workload", _small_workload)
    args = types.SimpleNamespace(steps=2, warmup=3, gpus=1)
    bench.run_reference(args, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "GB/s"
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["gpu_launches"] == 0
    bench.run_reference(args, 1)  # other ranks print nothing
    assert capsys.readouterr().out == ""
