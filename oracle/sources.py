"""Source terms (oracle, test infrastructure).

The load separates into f(t) = f_t(t) f_x (Sec. Spatial discretization).
  * ricker: f_t(t) = (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2), t0 = 1/f0
    (the workloads' wavelet; the paper's own 2D wavelet is the next one).
  * gaussian_derivative: Eq. ft, derivative of a Gaussian centred at t0 = 1/f_s
    with sigma_t = 1 / (2 pi f_s).
  * sine_burst: the two-cycle sine burst of the 3D example (n_c cycles).
  * bell: Eq. fx, amp * exp(-|x - x_s|^2 / (2 sigma^2)) (the paper uses amp 10).

Pins: tests/test_oracle_sources.py (closed-form values: Ricker peak 1 at t0,
zeros at t0 +- 1/(sqrt(2) pi f0); Eq. ft zero at t0 and extremum at t0 -+ sigma_t;
burst zero beyond n_c / f_s and its value inside the second cycle).
"""
import numpy as np

RICKER, GAUSS_DERIV, SINE_BURST = 0, 1, 2


def ricker(t, f0):
    t0 = 1.0 / f0
    a = (np.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def gaussian_derivative(t, fs):
    t0 = 1.0 / fs
    s = 1.0 / (2.0 * np.pi * fs)
    return -(t - t0) / (np.sqrt(2.0 * np.pi) * s ** 3) * np.exp(-((t - t0) ** 2) / (2.0 * s * s))


def sine_burst(t, fs, ncycles=2):
    t = np.asarray(t, dtype=np.float64)
    val = np.sin(2.0 * np.pi * fs * t) * np.sin(np.pi * fs * t / ncycles) ** 2
    return np.where(t <= ncycles / fs, val, 0.0)


def wavelet(kind, f0):
    if kind == RICKER:
        return lambda t: float(ricker(t, f0))
    if kind == GAUSS_DERIV:
        return lambda t: float(gaussian_derivative(t, f0))
    if kind == SINE_BURST:
        return lambda t: float(sine_burst(t, f0))
    raise ValueError(kind)


def bell(pos, sigma, amp):
    """Spatial Gaussian bell(s); pos (nsrc, dim).  Sum over sources."""
    pos = np.atleast_2d(np.asarray(pos, dtype=np.float64))

    def fx(x):
        x = np.atleast_2d(x)
        out = np.zeros(len(x))
        for s in pos:
            out += amp * np.exp(-((x - s) ** 2).sum(axis=1) / (2.0 * sigma * sigma))
        return out

    return fx
