"""Host logic of the surrogate's temperature placement: the chi-peak
estimators against peaks fixed by construction."""
import math

import numpy as np

from paper_1208_2080_gb300 import surrogate as sg


def _lorentz(T, T0, w, A=100.0):
    return A / (1.0 + ((T - T0) / w) ** 2)


def test_dense_estimator_finds_a_gaussian_peak_exactly():
    # log chi of a Gaussian peak is a parabola: the vertex is exact
    T = np.linspace(0.985, 1.015, 96)
    chi = 50.0 * np.exp(-0.5 * ((T - 1.0031) / 0.004) ** 2)
    assert abs(sg.peak_estimate_dense(T, chi) - 1.0031) < 1e-9


def test_dense_estimator_averages_out_point_noise():
    rng = np.random.default_rng(3)
    T = np.linspace(0.985, 1.015, 96)
    errs = []
    for _ in range(50):
        chi = _lorentz(T, 1.0042, 0.006) * (1 + 0.03 * rng.normal(size=T.size))
        errs.append(sg.peak_estimate_dense(T, chi) - 1.0042)
    # 3% point noise: the fitted vertex stays within a few grid spacings
    spacing = T[1] - T[0]
    assert abs(np.mean(errs)) < spacing and np.std(errs) < 3 * spacing


def test_grid_estimator_on_a_coarse_grid_is_off_by_up_to_its_spacing():
    # the 32-point uniform grid over [0.9, 1.1] against a narrow peak between
    # two grid points: the parabola through the maximum and its neighbours
    # cannot place it closer than a fraction of the spacing
    T = np.linspace(0.9, 1.1, 32)
    chi = _lorentz(T, 1.0031, 0.003)
    est = sg.peak_estimate(T, chi)
    spacing = T[1] - T[0]
    assert abs(est - 1.0031) < spacing
    # a dense grid around it gets the peak to a small fraction of that
    Td = np.linspace(est * 0.985, est * 1.015, 96)
    assert abs(sg.peak_estimate_dense(Td, _lorentz(Td, 1.0031, 0.003)) - 1.0031) < 0.1 * spacing


def test_edge_cases():
    T = np.linspace(0.9, 1.1, 5)
    # a monotone chi has its maximum at the edge: the estimators stay inside the grid
    chi = np.exp(T)
    assert T[0] <= sg.peak_estimate(T, chi) <= T[-1]
    assert T[0] <= sg.peak_estimate_dense(T, chi) <= T[-1]
    # fewer than three points above the cut: the arg max
    chi = np.array([1.0, 1.0, 10.0, 1.0, 1.0])
    assert sg.peak_estimate_dense(T, chi) == T[2]
    assert math.isfinite(sg.peak_estimate(T, chi))
