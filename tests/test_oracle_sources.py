"""Pins of the oracle's source terms to their closed forms."""
import numpy as np
import pytest

from oracle import sources


def test_ricker_closed_form():
    f0 = 5.0
    t0 = 1.0 / f0
    assert sources.ricker(t0, f0) == 1.0
    tz = t0 + 1.0 / (np.sqrt(2.0) * np.pi * f0)          # 1 - 2 pi^2 f0^2 tau^2 = 0
    assert abs(sources.ricker(tz, f0)) < 1e-15 * 4
    assert sources.ricker(0.0, f0) == pytest.approx((1.0 - 2.0 * np.pi ** 2) * np.exp(-np.pi ** 2), rel=1e-14)


def test_gaussian_derivative_eq_ft():
    fs = 2.0
    t0, s = 1.0 / fs, 1.0 / (2.0 * np.pi * fs)
    assert sources.gaussian_derivative(t0, fs) == 0.0
    # extrema at t0 -+ sigma_t with value +- exp(-1/2) / (sqrt(2 pi) sigma_t^2)
    peak = np.exp(-0.5) / (np.sqrt(2.0 * np.pi) * s * s)
    assert sources.gaussian_derivative(t0 - s, fs) == pytest.approx(peak, rel=1e-13)
    ts = np.linspace(0, 1, 20001)
    assert np.abs(sources.gaussian_derivative(ts, fs)).max() == pytest.approx(peak, rel=1e-6)


def test_sine_burst():
    fs = 20e3
    assert float(sources.sine_burst(2.0 / fs + 1e-9, fs)) == 0.0
    assert float(sources.sine_burst(1.0 / fs, fs)) == pytest.approx(0.0, abs=1e-12)
    t = 0.25 / fs
    assert float(sources.sine_burst(t, fs)) == pytest.approx(np.sin(np.pi / 8) ** 2, rel=1e-12)
    # The second of the two cycles: sin(2 pi 1.25) = 1, envelope sin^2(5 pi / 8).
    t = 1.25 / fs
    assert float(sources.sine_burst(t, fs)) == pytest.approx(np.sin(5 * np.pi / 8) ** 2, rel=1e-12)


def test_bell_eq_fx():
    fx = sources.bell(np.array([[1.0, 2.0]]), 0.06, 10.0)
    assert fx(np.array([[1.0, 2.0]]))[0] == 10.0
    x = np.array([[1.06, 2.0]])
    assert fx(x)[0] == pytest.approx(10.0 * np.exp(-0.5), rel=1e-14)
