"""Pins of the Womersley closed form used by the oscillatory-pipe check (no GPU)."""
import math

import numpy as np

from oracle import womersley as Wo


def test_modes_satisfy_the_ode_and_wall_condition():
    R, rho, mu, omega = 1.0, 1.0, 0.04, 0.64
    a = np.array([2 * math.pi, 1.0, 0.5])
    b = np.array([0.0, -0.7, 0.3])
    G = Wo.pressure_gradient_modes(a, b, R, rho, mu, omega)
    r = np.linspace(0.05, 0.95, 50)
    h = 1e-4
    W = Wo.velocity_modes(r, G, R, rho, mu, omega)
    Wp = Wo.velocity_modes(r + h, G, R, rho, mu, omega)
    Wm = Wo.velocity_modes(r - h, G, R, rho, mu, omega)
    d1 = (Wp - Wm) / (2 * h)
    d2 = (Wp - 2 * W + Wm) / (h * h)
    for k in range(len(G)):
        lhs = 1j * rho * k * omega * W[:, k]
        rhs = G[k] + mu * (d2[:, k] + d1[:, k] / r)
        assert np.allclose(lhs, rhs, atol=1e-5 * max(1.0, abs(G[k])))
    assert np.allclose(Wo.velocity_modes([R], G, R, rho, mu, omega), 0, atol=1e-12)


def test_flow_rate_integral_reproduces_the_waveform():
    R, rho, mu, omega = 1.3, 1.06, 0.04, 9.0
    a = np.array([3.0, 0.8, -0.2, 0.1])
    b = np.array([0.0, 0.4, 0.3, -0.05])
    G = Wo.pressure_gradient_modes(a, b, R, rho, mu, omega)
    r = np.linspace(0, R, 20001)
    W = Wo.velocity_modes(r, G, R, rho, mu, omega)
    Q = np.trapezoid(2 * math.pi * r[:, None] * W, r, axis=0)
    series = Wo.to_real_series(Q)[0]
    ref = np.zeros(2 * len(a) - 1)
    ref[0] = a[0]
    ref[1::2] = a[1:]
    ref[2::2] = b[1:]
    assert np.allclose(series, ref, rtol=1e-6, atol=1e-8)


def test_low_frequency_limit_is_quasi_steady_poiseuille():
    R, rho, mu = 1.0, 1.0, 1.0
    omega = 1e-4
    a = np.array([1.0, 0.5])
    b = np.array([0.0, 0.0])
    G = Wo.pressure_gradient_modes(a, b, R, rho, mu, omega)
    r = np.linspace(0, R, 7)
    W = Wo.velocity_modes(r, G, R, rho, mu, omega)
    # mode 1 carries flow rate Q_1 = (a_1 - i b_1) / 2 = 0.25: Poiseuille profile 2 Q_1 / (pi R^2) (1 - r^2 / R^2)
    pois = 2 * 0.25 / (math.pi * R * R) * (1 - (r / R) ** 2)
    assert np.allclose(W[:, 1], pois, rtol=1e-3, atol=1e-6)
