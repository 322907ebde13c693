"""Pins of the oracle's second source signal, the first derivative of a
Gaussian (Sec. 3.2), read as the tau-derivative of the Ricker's Gaussian
envelope exp(-pi^2 tau^2 / T^2) scaled to unit peak magnitude, delay 1.5 T."""
import numpy as np

import oracle
from paper_2009_11742_gb300 import inputs


def test_special_points_and_antisymmetry():
    T = 7.5
    t0 = 1.5 * T
    ts = T / (np.pi * np.sqrt(2.0))  # extrema of tau exp(-pi^2 tau^2 / T^2)
    f, _ = oracle.wavelet(1, np.array([t0, t0 + ts, t0 - ts]), T)
    np.testing.assert_allclose(f, [0.0, -1.0, 1.0], atol=1e-15)
    tau = np.linspace(0.0, 3 * T, 301)
    fp, _ = oracle.wavelet(1, t0 + tau, T)
    fm, _ = oracle.wavelet(1, t0 - tau, T)
    np.testing.assert_allclose(fp, -fm, atol=1e-15)
    assert np.max(np.abs(fp)) <= 1.0 + 1e-15


def test_is_the_derivative_of_the_gaussian_envelope():
    """f(t) = c d/dt exp(-pi^2 (t - t0)^2 / T^2) with c = T e^{1/2} / (pi sqrt 2),
    the derivative taken by central differences of the envelope alone."""
    T = 11.0
    t = np.linspace(0.0, 4 * T, 401)
    env = lambda x: np.exp(-np.pi ** 2 * (x - 1.5 * T) ** 2 / T ** 2)  # noqa: E731
    h = 1e-5
    d = (env(t + h) - env(t - h)) / (2 * h)
    c = T * np.exp(0.5) / (np.pi * np.sqrt(2.0))
    f, _ = oracle.wavelet(1, t, T)
    np.testing.assert_allclose(f, c * d, atol=1e-8)


def test_period_derivative_vs_finite_differences():
    t = np.linspace(0.0, 90.0, 181)
    for T in (20.0, 33.0):
        _, d = oracle.wavelet(1, t, T)
        h = 1e-6 * T
        fp, _ = oracle.wavelet(1, t, T + h)
        fm, _ = oracle.wavelet(1, t, T - h)
        np.testing.assert_allclose(d, (fp - fm) / (2 * h), atol=1e-7)


def test_ricker_kind_is_unchanged():
    t = np.linspace(0.0, 60.0, 61)
    f0, d0 = oracle.wavelet(0, t, 12.0)
    f1, d1 = oracle.ricker(t, 12.0)
    np.testing.assert_array_equal(f0, f1)
    np.testing.assert_array_equal(d0, d1)


def test_forward_with_gaussian_source_equals_its_forcing_table():
    p = inputs.make_problem(12, 10, 5, 3, seed=2)
    N = 120
    Z1, Z2 = np.zeros((12, 5)), np.zeros((10, 5))
    tn = (np.arange(N) + 4) * p.dt
    ft, _ = oracle.wavelet(1, tn[:, None], p.T.astype(np.float64)[None, :])
    a = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z1, Z2, N, T=p.T, n0=4, r=6, wavelet=1)
    b = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z1, Z2, N, ftab=ft, n0=4, r=6)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    c = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z1, Z2, N, T=p.T, n0=4, r=6)
    assert np.linalg.norm(c[0] - a[0]) > 1e-3 * np.linalg.norm(a[0])  # the signal matters


def test_adjoint_period_gradient_with_gaussian_source():
    p = inputs.make_problem(10, 9, 3, 2, seed=6)
    N = 80
    Z1, Z2 = np.zeros((10, 3)), np.zeros((9, 3))
    _, _, ys = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z1, Z2, N, T=1.05 * p.T.astype(np.float64),
                              r=1, wavelet=1)
    L, _, _, gT = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, Z1, Z2, p.T, N, ys, wavelet=1)
    T0 = p.T.astype(np.float64)
    for m in range(3):
        h = 1e-6 * T0[m]
        Tp, Tm = T0.copy(), T0.copy()
        Tp[m] += h
        Tm[m] -= h
        Lp = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, Z1, Z2, Tp, N, ys, wavelet=1)[0]
        Lm = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, Z1, Z2, Tm, N, ys, wavelet=1)[0]
        assert abs((Lp - Lm) / (2 * h) - gT[m]) <= 1e-5 * abs(gT[m]) + 1e-12
