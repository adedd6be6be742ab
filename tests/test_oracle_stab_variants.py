"""Pins of the oracle's stabilisation variants (Sec. 2.2, remarks after Eq. tau; readings R17, R18).

  * full RBVMS adds the cross- and Reynolds-stress terms of the subscale velocity u' = -tau L / rho: on one
    tetrahedron with a spatially constant tau L (no convection in tau or L, u = a(t) + B x with B constant
    in time, p linear) they have the closed forms -(V/4) (tau L . grad) u_i and -(V/rho) (tau L . grad N_a)
    (tau L)_i per node; the plug-flow patch (L = 0) stays an exact solution; the Reynolds stress sums to 0
    over an element's nodes; the exact Jacobian matches central differences;
  * the time-discretisation term of tau, ct (1/dt)^2 with dt = T / N, enters tau under the root (closed form
    on the reference tetrahedron) and leaves the plug-flow solution exact.
"""
import math

import numpy as np
import pytest

from oracle import hb_oracle as O
from paper_2411_14315_gb300 import inputs as I
from tests.test_oracle_pins import _plug_problem, _random_problem


def _one_tet_problem(n_h=2, rho=1.2, mu=0.3, T=1.3):
    xyz = np.array([[0.1, 0.0, 0.05], [1.2, 0.1, 0.0], [0.2, 0.9, 0.1], [0.05, 0.2, 1.1]])
    tets = np.array([[0, 1, 2, 3]])
    faces = I.boundary_faces(tets, 4).astype(np.int32)
    pr = O.HBProblem(xyz, tets, faces, np.full(4, 7, dtype=np.int32), rho, mu, T, n_h, beta_bf=0.0,
                     convection=False)
    return xyz, pr


def test_rbvms_terms_closed_form_on_one_tetrahedron():
    xyz, pr = _one_tet_problem()
    N, rho = pr.N, pr.rho
    rng = np.random.default_rng(3)
    t = O.instance_times(N, pr.T)
    w = 2 * math.pi / pr.T
    a = np.stack([0.3 + 0.2 * np.cos(w * t + k) for k in range(3)])      # a_i(t), band limited
    B = rng.uniform(-1, 1, (3, 3))                                       # non-symmetric, constant in time
    c = rng.uniform(-1, 1, 3)
    g = np.stack([0.5 * np.sin(w * t + k) for k in range(3)])            # grad p (t)
    y = np.zeros((4, 4, N))
    y[:, :3, :] = a[None] + (xyz @ B.T)[:, :, None]
    y[:, 3, :] = c.sum() + np.einsum("ai,in->an", xyz, g)
    gls = O.residual(pr, y)
    pr.stab = "rbvms"
    rb = O.residual(pr, y)
    # closed form: H a is the exact derivative of a (band limited), L = rho a' + grad p, tau constant
    adot = np.stack([-0.2 * w * np.sin(w * t + k) for k in range(3)])
    tau = 1.0 / math.sqrt(O.C_I * pr.nu ** 2 * pr.geo.GG[0])
    tL = tau * (rho * adot + g)                                          # [i, n]
    V, gN = pr.geo.V[0], pr.geo.gradN[0]
    cross = -(V / 4.0) * np.einsum("jn,ij->in", tL, B)                   # same for every node
    reyn = -(V / rho) * np.einsum("jn,aj,in->ain", tL, gN, tL)
    expect = cross[None] + reyn
    assert np.allclose(rb[:, :3] - gls[:, :3], expect, rtol=1e-12, atol=1e-14)
    assert np.allclose(rb[:, 3], gls[:, 3])                              # continuity rows unchanged
    # a transposed velocity gradient would give another answer (B is not symmetric)
    assert not np.allclose(expect, (-(V / 4.0) * np.einsum("jn,ji->in", tL, B))[None] + reyn)


def test_rbvms_reynolds_stress_sums_to_zero_over_element_nodes():
    m, pr = _random_problem(seed=31, resistance=False, beta=0.0)
    y = I.random_state(m.n_nodes, pr.N, 41)
    s = O._element_state(pr, y, np.arange(m.tets.shape[0]))
    HUq = np.einsum("qa,eain->eqin", O.NQ, O._apply_H(pr, s["U"]))
    conv = np.einsum("eqjn,eijn->eqin", s["Uq"], s["gradU"])
    tL = s["tau"][:, :, None, :] * (pr.rho * HUq + pr.rho * conv + s["gradP"][:, None])
    zero_grad = np.zeros_like(s["gradU"])
    reyn = O._rbvms_terms(pr, s["V"] / 4.0, s["gN"], zero_grad, tL)
    assert np.abs(reyn.sum(axis=1)).max() < 1e-13 * np.abs(reyn).max()


@pytest.mark.parametrize("stab,ct", [("rbvms", 0.0), ("gls", 1.0), ("rbvms", 4.0)])
def test_plug_flow_stays_exact_under_variants(stab, ct):
    m, pr, y = _plug_problem(2)
    pr.stab, pr.ct_dt = stab, ct
    r = O.residual(pr, y)
    scale = pr.rho * np.abs(y[:, :3]).max() * pr.geo.V.max() * (1 + pr.omega * 2)
    assert np.abs(r).max() < 1e-13 * max(scale, 1.0) + 1e-14


@pytest.mark.parametrize("stab,ct", [("rbvms", 0.0), ("rbvms", 1.0), ("gls", 1.0)])
def test_exact_jv_of_variants_matches_central_differences(stab, ct):
    m, pr = _random_problem(seed=32)
    pr.stab, pr.ct_dt = stab, ct
    N = pr.N
    y = pr.apply_dirichlet(I.random_state(m.n_nodes, N, 9))
    v = I.random_state(m.n_nodes, N, 10)
    mask, _ = pr.dirichlet()
    v[mask, :3] = 0
    eps = 1e-6
    fd = (O.residual(pr, y + eps * v) - O.residual(pr, y - eps * v)) / (2 * eps)
    je = O.jv_exact(pr, y, v)
    assert np.linalg.norm(fd - je) / np.linalg.norm(je) < 1e-8
    if stab == "rbvms":                      # the added terms are really in the Jacobian
        pr.stab = "gls"
        assert np.linalg.norm(O.jv_exact(pr, y, v) - je) > 1e-6 * np.linalg.norm(je)


def test_tau_with_time_discretisation_term_on_reference_tet():
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    tets = np.array([[0, 1, 2, 3]])
    faces = I.boundary_faces(tets, 4).astype(np.int32)
    nu, T, n_h, ct = 0.2, 0.8, 3, 2.5
    pr = O.HBProblem(xyz, tets, faces, np.ones(4, dtype=np.int32), 1.0, nu, T, n_h)
    pr.ct_dt = ct
    N = pr.N
    y = np.zeros((4, 4, N))
    y[:, 0, :] = 1.0
    st = O._element_state(pr, y, np.array([0]))
    dt = 2 * math.pi / (N * 2 * math.pi / T)                 # the paper's equivalent step 2 pi / (N w)
    assert np.allclose(st["tau"], (ct / dt ** 2 + 1.0 + 3.0 * nu * nu * 3.0) ** -0.5)
