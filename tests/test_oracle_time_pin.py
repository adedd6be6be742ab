"""Brute-force time discretisation against the HB oracle: does the spectral coupling H of Sec. 2.1
(H = E^-1 Omega E standing for d/dt across the N instances) give the periodic solution of the
time-continuous problem?

The time-continuous counterpart of the HB residual replaces H by d/dt: momentum Q(u, du/dt, p) +
d/dt T(u, du/dt, p) = 0 and continuity Q^c = 0 (Eqs. NS-harm and Rmc with H -> d/dt).  Marching it
forward from an initial state is ill-posed: T carries - int N tau L with L = rho du/dt + ..., so the
momentum equation gains - rho^2 tau d^2u/dt^2 (the time derivative of the least-squares weight), a
backward-parabolic term whose modes grow like exp(t / tau) forward in time.  Its periodic solution is
well defined, though, and the brute-force way to reach it is a fine uniform time grid of M >> N levels
with the second-order central difference D = (S - S^-1) / (2 dt) in place of H, solved for its periodic
state by Newton (the oracle's own residual and exact Jacobian with H replaced by D).  The harmonics of
that solution converge to the HB solution's as dt^2; a wrong sign, frequency or placement of the
spectral coupling breaks that.
"""
import numpy as np
import pytest

from oracle import hb_oracle as O
from tests import problems as P


def central_difference(M: int, T: float) -> np.ndarray:
    """Periodic second-order central difference on t_m = m T / M."""
    dt = T / M
    D = np.zeros((M, M))
    for m in range(M):
        D[m, (m + 1) % M] += 0.5 / dt
        D[m, (m - 1) % M] -= 0.5 / dt
    return D


M1, M2 = 15, 25


def hb_harmonics(spec, h_scale: float = 1.0) -> np.ndarray:
    """HB solution (N = 9) of the channel; h_scale != 1 plants a mistake in the oracle's H."""
    spec.n_h = 4
    pr = P.oracle_problem(spec)
    pr.H = h_scale * pr.H
    y, hist = O.solve(pr, rtol=1e-12)
    assert hist[-1] <= 1e-12 * hist[0]
    return O.instances_to_harmonics(y, 4)


def fd_periodic_harmonics(spec, c_start, M: int) -> np.ndarray:
    """Periodic solution on M time levels with the central difference, from c_start sampled on the fine
    grid (exact Newton throughout); its first 9 real harmonics."""
    spec.n_h = (M - 1) // 2
    pr = P.oracle_problem(spec)
    pr.H = central_difference(M, spec.T)
    y0 = O.harmonics_to_instances(c_start, M, spec.T)
    y, hist = O.solve(pr, y0=y0, switch_tol=10.0, rtol=1e-9, gmres_tol=1e-3)
    assert hist[-1] <= 1e-10 * hist[0]
    return O.instances_to_harmonics(y, (M - 1) // 2)[:, :, :c_start.shape[-1]]


@pytest.fixture(scope="module")
def brute_force():
    """Channel forced by two inflow harmonics: its HB solution with N = 9 (4 harmonics, room for the
    products the convective term forms) and the central-difference periodic solutions on 15 and 25
    levels."""
    spec = P.channel_spec(n_h=2)
    c_hb = hb_harmonics(spec)
    return spec, c_hb, fd_periodic_harmonics(spec, c_hb, M1), fd_periodic_harmonics(spec, c_hb, M2)


def convergence(c_hb, c1, c2):
    """(e1, e2, Richardson error) of the two grids' harmonics against c_hb, relative."""
    nrm = np.linalg.norm(c_hb)
    rich = (M2 * M2 * c2 - M1 * M1 * c1) / (M2 * M2 - M1 * M1)
    return (np.linalg.norm(c1 - c_hb) / nrm, np.linalg.norm(c2 - c_hb) / nrm, np.linalg.norm(rich - c_hb) / nrm)


def second_order_to(c_hb, c1, c2) -> bool:
    e1, e2, er = convergence(c_hb, c1, c2)
    return 0.9 * (M2 / M1) ** 2 < e1 / e2 < 1.1 * (M2 / M1) ** 2 and er < 0.1 * e2


def test_central_difference_periodic_solution_converges_to_hb_at_second_order(brute_force):
    spec, c_hb, c1, c2 = brute_force
    e1, e2, er = convergence(c_hb, c1, c2)
    # measured: 1.97e-2 and 7.25e-3, ratio 2.72 against (25 / 15)^2 = 2.78; Richardson extrapolation
    # removes the dt^2 term and what is left (dt^4, HB's own truncation) is 2.6e-4
    assert e2 < 1.5e-2
    assert second_order_to(c_hb, c1, c2), (e1, e2, er)


@pytest.mark.parametrize("h_scale", [-1.0, 1.01])
def test_planted_mistake_in_H_breaks_the_agreement(brute_force, h_scale):
    """The same check against an oracle whose H has the wrong sign (time reversed) or a 1 % frequency
    error: the brute-force solutions no longer converge to its HB solution."""
    spec, c_hb, c1, c2 = brute_force
    c_wrong = hb_harmonics(spec, h_scale)
    assert not second_order_to(c_wrong, c1, c2)
