"""Womersley's closed form for fully developed oscillatory flow in a straight pipe (test infrastructure).

A textbook exact solution of the Navier-Stokes equations, not a case of the paper: it checks the unsteady
solution of both the HB method (Sec. 2) and the conventional time marching (Sec. 3) on a pipe.

For axial velocity w(r, t) in a pipe of radius R driven by G(t) = -dp/dz, rho dw/dt = G + mu (w'' + w'/r)
with w(R) = 0.  Mode k >= 1 (time factor e^{i k w t}): W_k(r) = G_k / (i rho k w) (1 - J0(b r) / J0(b R)),
b = i^{3/2} sqrt(k w / nu); mode 0 is Poiseuille flow, W_0 = G_0 (R^2 - r^2) / (4 mu).  The flow rate of
mode k is Q_k = G_k pi R^2 / (i rho k w) (1 - 2 J1(b R) / (b R J0(b R))), Q_0 = G_0 pi R^4 / (8 mu).
The convective term vanishes identically (w depends on r only), so the solution is exact for the
Navier-Stokes equations, and it is band-limited in time when the flow rate is.

Real series convention: f(t) = a0 + sum_k a_k cos(k w t) + b_k sin(k w t) = f_0 + 2 Re sum_k f_k e^{i k w t},
f_k = (a_k - i b_k) / 2.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import jv


def pressure_gradient_modes(a, b, R, rho, mu, omega):
    """Complex modes G_k (k = 0..n_h) of G = -dp/dz that drive the flow rate with real series (a, b)."""
    nu = mu / rho
    n_h = len(a) - 1
    G = np.zeros(n_h + 1, dtype=complex)
    G[0] = a[0] * 8.0 * mu / (math.pi * R ** 4)
    for k in range(1, n_h + 1):
        Qk = 0.5 * (a[k] - 1j * b[k])
        bR = (1j ** 1.5) * R * math.sqrt(k * omega / nu)
        f = 1.0 - 2.0 * jv(1, bR) / (bR * jv(0, bR))
        G[k] = Qk * 1j * rho * k * omega / (math.pi * R * R * f)
    return G


def velocity_modes(r, G, R, rho, mu, omega):
    """Complex modes W_k(r) [len(r), n_h + 1] of the axial velocity (the Bessel-function solution of the
    module docstring)."""
    nu = mu / rho
    r = np.asarray(r, dtype=float)
    W = np.zeros((r.size, len(G)), dtype=complex)
    W[:, 0] = G[0] * (R * R - r * r) / (4.0 * mu)
    for k in range(1, len(G)):
        b = (1j ** 1.5) * math.sqrt(k * omega / nu)
        W[:, k] = G[k] / (1j * rho * k * omega) * (1.0 - jv(0, b * r) / jv(0, b * R))
    return W


def to_real_series(modes):
    """(a0, a1, b1, ...) from complex modes f_k: a_k = 2 Re f_k, b_k = -2 Im f_k."""
    modes = np.atleast_2d(modes)
    n_h = modes.shape[1] - 1
    out = np.zeros((modes.shape[0], 2 * n_h + 1))
    out[:, 0] = modes[:, 0].real
    out[:, 1::2] = 2.0 * modes[:, 1:].real
    out[:, 2::2] = -2.0 * modes[:, 1:].imag
    return out


def pipe_solution(xyz, a, b, R, L, rho, mu, omega):
    """Exact harmonics [n, 4, 2 n_h + 1] of (u1, u2, u3, p) at points xyz for a pipe along +z from z = 0
    to z = L with a traction-free outlet (p = 0 at z = L)."""
    G = pressure_gradient_modes(a, b, R, rho, mu, omega)
    r = np.minimum(np.hypot(xyz[:, 0], xyz[:, 1]), R)
    W = velocity_modes(r, G, R, rho, mu, omega)
    out = np.zeros((xyz.shape[0], 4, 2 * (len(G) - 1) + 1))
    out[:, 2] = to_real_series(W)
    out[:, 3] = to_real_series(np.outer(L - xyz[:, 2], G))
    return out
