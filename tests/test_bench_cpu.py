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
