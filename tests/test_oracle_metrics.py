"""Pins of the oracle's accuracy measures (RMSE, MAE, iRMSE, iMAE over
pixels with valid ground truth; the KITTI measures of Section V, Tables 1-3)
by closed forms on constructed maps."""
import numpy as np
import pytest

import oracle


def test_perfect_prediction_scores_zero():
    g = np.full((7, 9), 12.5, np.float32)
    m = oracle.metrics(g, g)
    assert m["valid"] == 63 and m["rmse_mm"] == 0 and m["mae_mm"] == 0
    assert m["irmse_per_km"] == 0 and m["imae_per_km"] == 0


def test_constant_offset_closed_form():
    g = np.full((8, 8), 10.0, np.float32)
    p = np.full((8, 8), 20.0, np.float32)
    m = oracle.metrics(p, g)
    assert m["rmse_mm"] == pytest.approx(10000.0) and m["mae_mm"] == pytest.approx(10000.0)
    # |1/20 - 1/10| = 0.05 per metre = 50 per kilometre
    assert m["irmse_per_km"] == pytest.approx(50.0) and m["imae_per_km"] == pytest.approx(50.0)


def test_rmse_and_mae_differ_as_they_should():
    # errors of 0 and 2 m on two halves: MAE 1 m, RMSE sqrt(2) m
    g = np.full((4, 6), 30.0, np.float32)
    p = g.copy()
    p[:, 3:] = 32.0
    m = oracle.metrics(p, g)
    assert m["mae_mm"] == pytest.approx(1000.0) and m["rmse_mm"] == pytest.approx(1000.0 * np.sqrt(2.0))


def test_invalid_ground_truth_is_ignored_and_empty_prediction_counts():
    g = np.zeros((5, 5), np.float32)
    g[2, 2] = 4.0
    p = np.full((5, 5), 99.0, np.float32)
    p[2, 2] = 0.0                      # empty prediction where truth exists
    m = oracle.metrics(p, g)
    assert m["valid"] == 1
    assert m["mae_mm"] == pytest.approx(4000.0)
    assert m["imae_per_km"] == pytest.approx(250.0)      # |0 - 1/4| per metre
    assert oracle.metrics(p, np.zeros((5, 5), np.float32))["valid"] == 0
