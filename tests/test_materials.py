"""The tabulated silver permittivity (input data for wavelength sweeps):
pinned to the values the paper prints (the table of n and kappa of its
silver spheroid benchmark, and eps_r ~ -10.15 + 0.32i quoted at the 506 nm
resonance)."""

import numpy as np
import pytest

import workloads


def test_tabulated_points_are_exact_squares_of_n_plus_i_kappa():
    t = workloads.SILVER_JC
    eps = workloads.eps_silver(t[:, 0])
    np.testing.assert_allclose(eps, (t[:, 1] + 1j * t[:, 2]) ** 2, rtol=1e-15, atol=0)


def test_quoted_resonance_permittivity():
    e = workloads.eps_silver(506.0)[0]
    assert abs(e.real - (-10.15)) < 0.005 and abs(e.imag - 0.32) < 0.005


def test_table_is_sorted_and_refuses_extrapolation():
    t = workloads.SILVER_JC
    assert np.all(np.diff(t[:, 0]) > 0) and t.shape == (22, 3)
    with pytest.raises(ValueError):
        workloads.eps_silver(250.0)
    with pytest.raises(ValueError):
        workloads.eps_silver(900.0)
