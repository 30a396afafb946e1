"""Pins of the code-balance model (Eq. 1, Eq. 2, kappa of Sect. 2) against the
numbers the paper prints."""
import json
import os

import pytest

from paper_1106_5908_gb300 import model

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_model_numbers.json")))


def test_eq1_upper_limits_nehalem():
    g = GOLD["nehalem_hmep"]
    # 18.1 GB/s / B_CRS(15, 0) = 2.66 GF/s; 21.2 GB/s -> 3.12 GF/s (Sect. 2)
    assert model.max_performance(g["spmvm_bandwidth_gbs"], g["nnzr"]) == pytest.approx(
        g["max_perf_spmvm_bw_gfs"], abs=0.005)
    assert model.max_performance(g["stream_bandwidth_gbs"], g["nnzr"]) == pytest.approx(
        g["max_perf_stream_bw_gfs"], abs=0.005)


def test_kappa_hmep():
    g = GOLD["nehalem_hmep"]
    k = model.kappa_from(g["spmvm_bandwidth_gbs"], g["measured_perf_gfs"], g["nnzr"])
    assert k == pytest.approx(g["kappa"], abs=0.05)
    assert k * g["nnzr"] == pytest.approx(g["extra_bytes_per_row"], abs=0.1)
    assert round(model.rhs_loads(k, g["nnzr"])) == g["rhs_loads_approx"]


def test_kappa_hmep_electron_order():
    g = GOLD["nehalem_hmep_electron_order"]
    base = model.kappa_from(18.1, 2.25, 15)
    assert g["kappa"] / base - 1 == pytest.approx(g["extra_traffic_increase_approx"], abs=0.03)
    # performance ratio implied by the code balance: a drop of roughly 10 %
    drop = 1 - model.b_crs(15, base) / model.b_crs(15, g["kappa"])
    assert 0.05 < drop < 0.12
    assert drop == pytest.approx(g["perf_drop_approx"], abs=0.03)


def test_kappa_uhbr():
    g = GOLD["uhbr"]
    k = model.kappa_from(g["spmvm_bandwidth_gbs"], g["measured_perf_gfs"], g["nnzr"])
    # The printed inputs give 0.447; the paper prints 0.43.  Both round the
    # right-hand-side load count to 8.
    assert k == pytest.approx(g["kappa_printed"], abs=0.02)
    assert round(model.rhs_loads(k, g["nnzr"])) == g["rhs_loads_approx"]
    assert round(model.rhs_loads(g["kappa_printed"], g["nnzr"])) == g["rhs_loads_approx"]


def test_eq2_split_penalty():
    g = GOLD["split_penalty"]
    assert model.split_penalty(g["nnzr_low"]) == pytest.approx(g["penalty_low_approx"], abs=0.005)
    assert model.split_penalty(g["nnzr_high"]) == pytest.approx(g["penalty_high_approx"], abs=0.005)
    # and the penalty shrinks when kappa > 0 (Sect. 3.4: "even less if kappa > 0")
    assert model.split_penalty(15, 2.5) < model.split_penalty(15, 0.0)


def test_eq1_terms():
    # B_CRS = (12 + 24/N + kappa)/2: 8 B val + 4 B index, 16/N for the result,
    # 8/N for one load of the right-hand side, 2 flops
    for n in (1, 7, 15, 123):
        for k in (0.0, 1.0, 3.79):
            assert model.b_crs(n, k) == pytest.approx((8 + 4 + 16 / n + 8 / n + k) / 2)
            assert model.b_split(n, k) - model.b_crs(n, k) == pytest.approx(8 / n)


def test_gpu_byte_counts():
    # plain FP64, beta = 0: 12 B/entry + row_ptr + x once + y once
    assert model.bytes_plain(10, 10, 30) == 12 * 30 + 4 * 11 + 80 + 80
    assert model.bytes_plain(10, 10, 30, beta_nonzero=True) == 12 * 30 + 4 * 11 + 160 + 80
    assert model.bytes_plain(10, 10, 30, val_bytes=4, x_bytes=4, y_bytes=4) == 8 * 30 + 44 + 40 + 40
    assert model.bytes_spmm(10, 10, 30, 4) == 12 * 30 + 44 + 8 * 4 * 20
    assert model.bytes_split(10, 10, 30, 5) == model.bytes_plain(10, 10, 30) + 160 + 44 + 140
    assert model.flops(30, 4) == 240
