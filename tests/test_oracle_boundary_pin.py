"""Closed-form pin of the oracle's outlet terms (Sec. 2.3 and readings R5, R8): for a velocity that is
uniform over an outlet, the traction term - int N_A h n_i with h = -P (or -(P_d + R Q) at a resistance
outlet, Q = sum over the outlet's faces of |f| u.n) and the backflow stabilisation
- int N_A (rho/2) beta ((u.n - |u.n|)/2) u_i reduce to

    r_{A,i}(t_n) = sum over outlet faces f containing A of |f| / 3 (P(t_n) n_i + (rho/2) beta max(0, -u.n) u_i),

since int_f N_A = |f| / 3 and (u.n - |u.n|)/2 = -max(0, -u.n) is constant on the face.  Face normals and
areas are computed here from the coordinates, independently of the oracle."""
import math

import numpy as np
import pytest

from oracle import hb_oracle as O
from tests import problems as P


def _outlet_faces(spec):
    m = spec.mesh
    f = np.nonzero(spec.face_tag == 2)[0]                  # the x-max pressure outlet of the channel
    p = m.xyz[m.faces[f]]
    cr = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    n = cr / (2.0 * area[:, None])
    n *= np.sign(n[:, 0])[:, None]                         # outward: towards +x at the x-max outlet
    return m.faces[f], area, n


@pytest.mark.parametrize("resistance", [0.0, 2.5])       # pressure outlet, or resistance outlet (R8)
@pytest.mark.parametrize("ux", [-0.7, 0.7])               # inflow through the outlet (backflow) or outflow
def test_outlet_traction_and_backflow_match_the_closed_form(ux, resistance):
    spec = P.channel_spec(n_h=1)
    pr = P.oracle_problem(spec)                            # inflow cap Dirichlet; the outlet is the only
    assert set(spec.face_tag[pr.neumann_faces()].tolist()) == {2}       # Neumann part of the boundary
    (tag, pa, pb), = spec.outlets_p
    if resistance:
        # h = -(P_d + R Q) with Q the outlet flow rate: for a uniform velocity Q = sum_f |f| (u . n_f)
        pr.outlet_p.clear()
        pr.set_outlet_resistance(tag, resistance, pa, pb)
    N = pr.N
    t = spec.T * np.arange(N) / N
    w = 2.0 * math.pi / spec.T
    Pn = pa[0] + sum(pa[k] * np.cos(k * w * t) + pb[k] * np.sin(k * w * t) for k in range(1, len(pa)))
    u = np.array([ux, 0.4, 0.25])
    y = np.zeros((pr.n_nodes, 4, N))
    y[:, :3, :] = u[None, :, None]
    y[:, 3, :] = 1.7                                       # pressure does not enter the boundary terms
    faces, area, n = _outlet_faces(spec)
    if resistance:
        Pn = Pn + resistance * sum(area[f] * float(u @ n[f]) for f in range(len(faces)))
    expect = np.zeros((pr.n_nodes, 3, N))
    for f in range(len(faces)):
        back = 0.5 * spec.rho * spec.beta * max(0.0, -float(u @ n[f]))
        contrib = area[f] / 3.0 * (Pn[None, :] * n[f][:, None] + back * u[:, None])
        for a in faces[f]:
            expect[a] += contrib
    got = O.boundary_residual(pr, y)
    assert np.abs(got - expect).max() <= 1e-13 * np.abs(expect).max()
    if ux > 0:
        assert all(float(u @ n[f]) > 0 for f in range(len(faces)))   # outflow: no backflow term at all


@pytest.mark.parametrize("exact", [False, True])
@pytest.mark.parametrize("resistance", [0.0, 2.5])
@pytest.mark.parametrize("ux", [-0.7, 0.7])
def test_outlet_tangent_matches_the_closed_form(ux, resistance, exact):
    """The derivative of the outlet terms along a direction v, for u and v uniform over the outlet:
    the paper's tangent freezes the backflow coefficient (reading R7), -(rho/2) beta (u.n)_- v_i; the
    exact derivative adds -(rho/2) beta (v.n) u_i where u.n < 0; a resistance outlet contributes
    R Q(v) n_i with Q(v) = sum_f |f| v.n_f (R8), in both."""
    spec = P.channel_spec(n_h=1)
    pr = P.oracle_problem(spec)
    (tag, pa, pb), = spec.outlets_p
    if resistance:
        pr.outlet_p.clear()
        pr.set_outlet_resistance(tag, resistance, pa, pb)
    N = pr.N
    u = np.array([ux, 0.4, 0.25])
    vv = np.array([0.3, -0.2, 0.5])
    y = np.zeros((pr.n_nodes, 4, N))
    y[:, :3, :] = u[None, :, None]
    v = np.zeros((pr.n_nodes, 4, N))
    v[:, :3, :] = vv[None, :, None]
    faces, area, n = _outlet_faces(spec)
    Qv = sum(area[f] * float(vv @ n[f]) for f in range(len(faces)))
    expect = np.zeros((pr.n_nodes, 3, N))
    k = 0.5 * spec.rho * spec.beta
    for f in range(len(faces)):
        un = float(u @ n[f])
        back = k * max(0.0, -un) * vv
        if exact and un < 0:
            back = back - k * float(vv @ n[f]) * u
        contrib = area[f] / 3.0 * (resistance * Qv * n[f] + back)
        for a in faces[f]:
            expect[a] += contrib[:, None]
    got = O.boundary_jv(pr, y, v, exact)
    scale = max(np.abs(expect).max(), 1e-300)
    assert np.abs(got - expect).max() <= 1e-13 * scale
