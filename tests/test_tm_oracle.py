"""Pins of the time-marching oracle (oracle/tm_oracle.py) against what the paper and the mathematics fix:

* rho_inf = 0 gives the c1 = 1.5 that Sec. 2.3 quotes for its generalized-alpha pseudo-time term;
* with zero acceleration and omega_hat = 0 one time level is the steady GLS problem, i.e. the HB residual,
  tangent and Jacobi diagonal at N = 1 (H = 0), which the HB oracle's own pins fix;
* a moving plug flow u = a(t) e_x, p = -rho a'(t) x is an exact solution of the time-domain GLS
  equations for P1 (L = 0, grad u = 0) at every time and every omega_hat;
* generalized-alpha marching of that plug flow is second-order accurate in the time step.
"""
import math

import numpy as np
import pytest

from oracle import hb_oracle as O
from oracle import tm_oracle as TM
from paper_2411_14315_gb300 import inputs as I


def test_rho_inf_zero_gives_the_papers_c1():
    am, af, gam = TM.galpha(0.0)
    assert (am, af, gam) == (1.5, 1.0, 1.0)
    assert am / (af * gam) == 1.5
    am, af, gam = TM.galpha(1.0)                      # trapezoidal limit
    assert (am, af, gam) == (0.5, 0.5, 0.5)


def _random_problem(n_h, seed=5, n=(3, 2, 2)):
    m = I.box_mesh(*n, lx=1.5, jitter=0.2, seed=seed)
    tag = m.face_tag.copy()
    tag[(tag == 3) | (tag == 4)] = 0
    pr = O.HBProblem(m.xyz, m.tets, m.faces, tag, 1.1, 0.07, 1.7, n_h, beta_bf=0.2)
    a, b = I.waveform_harmonics(n_h, 1.0, seed)
    pr.set_inflow(1, I.uniform_profile(m, [1], [1.0, 0.2, 0.0]), a, b)
    pa, pb = I.waveform_harmonics(n_h, 0.5, seed + 1)
    pr.set_outlet_pressure(2, pa, pb)
    pr.set_outlet_resistance(5, 0.7, pa * 0.3, pb * 0.3)
    return m, pr


def test_zero_acceleration_is_the_steady_hb_problem():
    m, pr = _random_problem(0)
    rng = np.random.default_rng(3)
    y = rng.uniform(-1, 1, (m.n_nodes, 4))
    y = pr.apply_dirichlet(y[:, :, None])[:, :, 0]
    v = rng.uniform(-1, 1, (m.n_nodes, 4))
    r_tm = TM.residual(pr, y, np.zeros_like(y), 0.3, 0.0)
    r_hb = O.residual(pr, y[:, :, None])[:, :, 0]
    assert np.max(np.abs(r_tm - r_hb)) <= 1e-12 * np.max(np.abs(r_hb))
    # without a step (no acceleration term) the tangent and its diagonal are the steady ones
    j_tm = TM.jv_paper(pr, y, v, 0.0, 0.0)
    j_hb = O.jv_paper(pr, y[:, :, None], v[:, :, None], shift=0.0)[:, :, 0]
    assert np.max(np.abs(j_tm - j_hb)) <= 1e-12 * np.max(np.abs(j_hb))
    d_tm = TM.jacobi_diag(pr, y, 0.0, 0.0)
    d_hb = O.jacobi_diag(pr, y[:, :, None], shift=0.0)[:, :, 0]
    assert np.max(np.abs(d_tm - d_hb)) <= 1e-12 * np.max(np.abs(d_hb))
    # the acceleration term of tau_hat only lowers tau: a large omega_hat changes the residual
    assert np.max(np.abs(TM.residual(pr, y, np.zeros_like(y), 0.3, 1e3) - r_tm)) > 1e-6


@pytest.mark.parametrize("omega2", [0.0, 2.0])
def test_tangent_acceleration_terms_are_exact(omega2):
    """For a given omega_hat the residual is affine in du/dt, so the part of the tangent that the step
    adds (shift M v and the least-squares c1 rho / dt v terms of both rows) must equal the central
    difference of r along du/dt = shift / rho v_velocity, at any state; at rest with a uniform pressure
    (L = 0) the whole tangent is the exact derivative along (v, shift / rho v_velocity)."""
    m, pr = _random_problem(1)
    rng = np.random.default_rng(8)
    mask, g = TM.dirichlet_at(pr, 0.2)
    v = rng.uniform(-1, 1, (m.n_nodes, 4))
    v[mask, :3] = 0.0
    rho, shift, eps = pr.rho, 7.3, 1e-3
    dyd = np.zeros_like(v)
    dyd[:, :3] = shift / rho * v[:, :3]
    # any state: the acceleration part
    y = rng.uniform(-1, 1, (m.n_nodes, 4))
    y[mask, :3] = g[mask]
    yd = rng.uniform(-1, 1, (m.n_nodes, 4))
    fd = (TM.residual(pr, y, yd + eps * dyd, 0.2, omega2) - TM.residual(pr, y, yd - eps * dyd, 0.2, omega2)) / (2 * eps)
    part = TM.jv_paper(pr, y, v, omega2, shift) - TM.jv_paper(pr, y, v, omega2, 0.0)
    assert np.max(np.abs(part - fd)) <= 1e-10 * np.max(np.abs(fd))
    # at rest with a uniform pressure: the whole tangent
    y = np.zeros((m.n_nodes, 4))
    y[:, 3] = 0.7
    yd = np.zeros((m.n_nodes, 4))
    fd = (TM.residual(pr, y + eps * v, yd + eps * dyd, 0.2, omega2)
          - TM.residual(pr, y - eps * v, yd - eps * dyd, 0.2, omega2)) / (2 * eps)
    jv = TM.jv_paper(pr, y, v, omega2, shift)
    jv[mask, :3] = 0.0                        # Dirichlet rows: identity on v vs zero rows of r
    # (the backflow term is one-sided at rest: its central difference is O(eps))
    assert np.max(np.abs(jv - fd)) <= eps * np.max(np.abs(fd))
    # Jacobi diagonal = e_k^T J e_k, J without the least-squares acceleration term, for free velocity and
    # pressure unknowns off the Neumann faces (the diagonal holds the volume terms) at a random state
    y = rng.uniform(-1, 1, (m.n_nodes, 4))
    y[mask, :3] = g[mask]
    d = TM.jacobi_diag(pr, y, omega2, shift)
    on_faces = np.zeros(m.n_nodes, dtype=bool)
    on_faces[pr.faces[pr.neumann_faces()].ravel()] = True
    nodes = np.nonzero(~mask & ~on_faces)[0][:4]
    assert nodes.size > 0
    for node in nodes:
        for f in (0, 3):
            e = np.zeros_like(v)
            e[node, f] = 1.0
            jk = TM.jv_paper(pr, y, e, omega2, shift, ls_acceleration=False)[node, f]
            assert abs(jk - d[node, f]) <= 1e-12 * abs(d[node, f])


def _plug(T=2.0, rho=1.3, mu=0.05, seed=1, n=(4, 3, 3), a1=0.12, b1=-0.08):
    m = I.box_mesh(*n, lx=2.0, ly=1.0, lz=1.0, jitter=0.2, seed=seed)
    a = np.array([1.0, a1])
    b = np.array([0.0, b1])
    pr = O.HBProblem(m.xyz, m.tets, m.faces, m.face_tag, rho, mu, T, 1)
    prof = I.uniform_profile(m, [1, 3, 4, 5, 6], [1, 0, 0])
    for tag in [1, 3, 4, 5, 6]:
        pr.set_inflow(tag, prof, a, b)
    w = 2 * math.pi / T
    # p = -rho a'(t) x, so the outlet x = 2 carries P(t) = -2 rho a'(t)
    pr.set_outlet_pressure(2, np.array([0.0, -rho * 2.0 * w * b1]), np.array([0.0, rho * 2.0 * w * a1]))

    def exact(t):
        at = a[0] + a1 * math.cos(w * t) + b1 * math.sin(w * t)
        ad = w * (-a1 * math.sin(w * t) + b1 * math.cos(w * t))
        add = -w * w * (a1 * math.cos(w * t) + b1 * math.sin(w * t))
        y = np.zeros((m.n_nodes, 4))
        y[:, 0] = at
        y[:, 3] = -rho * ad * m.xyz[:, 0]
        yd = np.zeros((m.n_nodes, 4))
        yd[:, 0] = ad
        yd[:, 3] = -rho * add * m.xyz[:, 0]
        return y, yd
    return m, pr, exact


@pytest.mark.parametrize("t,omega2", [(0.0, 0.0), (0.37, 0.0), (1.21, 4.0), (1.9, 0.3)])
def test_moving_plug_flow_is_an_exact_solution(t, omega2):
    m, pr, exact = _plug()
    y, yd = exact(t)
    r = TM.residual(pr, y, yd, t, omega2)
    scale = 1.3 * np.max(np.abs(yd)) * np.max(pr.geo.V) ** (2 / 3)
    assert np.max(np.abs(r)) < 1e-12 * max(scale, 1.0)
    # a wrong sign of the acceleration is caught
    r_bad = TM.residual(pr, y, -yd, t, omega2)
    assert np.max(np.abs(r_bad)) > 1e-4


def test_generalized_alpha_march_is_second_order():
    """The plug flow's velocity is fixed by its Dirichlet data; the time error shows in the pressure,
    p = -rho x a'(t), which must fall ~4x when the step is halved."""
    errs = []
    for spp in (24, 48):
        m, pr, exact = _plug(n=(2, 2, 2))
        y0, _ = exact(0.0)
        y, _, _ = TM.march(pr, spp, 0.5, rho_inf=0.5, y0=y0, newton_tol=1e-11, gmres_tol=1e-12)
        ye, _ = exact(0.5 * pr.T)
        assert np.max(np.abs(y[:, 0] - ye[:, 0])) < 1e-12
        errs.append(np.max(np.abs(y[:, 3] - ye[:, 3])))
    assert errs[1] < errs[0] / 3.5


def test_omega_hat_is_the_velocity_norm_ratio():
    """Reading R14: omega_hat^2 = ||du/dt||^2 / ||u||^2 over the nodal velocity vectors only; for
    du/dt = c u on the velocity it is c^2 whatever the pressures."""
    rng = np.random.default_rng(5)
    y = rng.uniform(-1, 1, (40, 4))
    yd = np.empty_like(y)
    yd[:, :3] = -2.5 * y[:, :3]
    yd[:, 3] = rng.uniform(-50, 50, 40)
    assert abs(TM.omega_hat2(y, yd) - 6.25) < 1e-12
