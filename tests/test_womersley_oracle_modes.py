"""The oracle against Womersley's closed form for oscillatory pipe flow, on the CPU.

Womersley's solution u = w(r, t) e_z, p = G(t) (L - z) has no convection (u . grad u = 0), so it also
solves the Stokes limit of the HB equations.  Without convection and backflow the oracle's HB residual
(Eq. Rmc with tau of Eq. tau at U = 0) is linear and time invariant, so its root decouples into one
complex system per Fourier mode k (H -> i k w, Eq. NS-harm): written out here by hand from the GLS weak
form, assembled sparse and solved directly.  Two checks pin the oracle to the closed form:
  * the instance values built from those modes zero the oracle's residual (so the oracle's linear part,
    Dirichlet rows and traction-free outlet are this discretisation of the equations), and
  * their velocity error against Womersley's solution falls at second order in the cell size (P1), on
    the pipe of the Womersley workload (~3,000 tetrahedra) and its refinement (~24,000).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import hb_oracle as O
from oracle import womersley as Wo
from paper_2411_14315_gb300 import workloads as W


def _problem(level):
    spec = W.womersley_spec(level=level)
    tag, _, a, b = spec.inflows[0]
    omega = 2 * math.pi / spec.T
    exact = Wo.pipe_solution(spec.mesh.xyz, a, b, 1.0, 5.0, spec.rho, spec.mu, omega)
    m = spec.mesh
    pr = O.HBProblem(m.xyz, m.tets, m.faces, m.face_tag, spec.rho, spec.mu, spec.T, spec.n_h, beta_bf=0.0,
                     convection=False)
    pr.set_inflow_harmonics(tag, exact[:, :3])
    return pr, exact


def _mode_solution(pr, exact):
    """Instance values [n, 4, N] of the Stokes-limit HB root, one sparse complex solve per mode.

    Per element (volume V, shape gradients gN, tau = (C_I nu^2 G:G)^(-1/2) at U = 0) and node pair a, b,
    with M_ab = V (1 + delta_ab) / 20 and S_ab = V gN_a . gN_b, mode k (om = k w) contributes
      velocity i / velocity i:  (i om rho + tau rho om^2) M_ab + mu S_ab   (Galerkin mass, viscous, and the
                                 least-squares term -H N_A tau rho H u)
      velocity i / pressure:    -V/4 d_i N_a - i om tau V/4 d_i N_b
      pressure / velocity i:    V/4 d_i N_b + i om tau V/4 d_i N_a        (continuity, PSPG of rho H u)
      pressure / pressure:      tau / rho S_ab
    """
    n, N, n_h = pr.n_nodes, pr.N, pr.n_h
    w = 2 * math.pi / pr.T
    g = pr.geo
    tets = pr.tets
    V, gN = g.V, g.gradN
    tau = 1.0 / np.sqrt(3.0 * pr.nu ** 2 * g.GG)
    rho, mu = pr.rho, pr.mu
    eye = np.eye(4)
    M = V[:, None, None] * (1.0 + eye)[None] / 20.0                 # [e, a, b]
    S = V[:, None, None] * np.einsum("eai,ebi->eab", gN, gN)
    A = np.repeat(tets[:, :, None], 4, axis=2)                       # row node [e, a, b]
    B = np.repeat(tets[:, None, :], 4, axis=1)                       # column node
    mask, _ = pr.dirichlet()
    fixed = np.zeros(4 * n, dtype=bool)
    fixed.reshape(n, 4)[mask, :3] = True
    free = ~fixed
    sol = []
    for k in range(n_h + 1):
        om = k * w
        rows, cols, vals = [], [], []

        def add(r, c, v):
            rows.append(r.ravel())
            cols.append(c.ravel())
            vals.append(np.broadcast_to(v, r.shape).ravel())

        kvv = (1j * om * rho + tau[:, None, None] * rho * om * om) * M + mu * S
        for i in range(3):
            add(4 * A + i, 4 * B + i, kvv)
            gi_a = gN[:, :, i][:, :, None] * np.ones((1, 1, 4))     # d_i N_a over b
            gi_b = gN[:, :, i][:, None, :] * np.ones((1, 4, 1))     # d_i N_b over a
            t4 = (tau * V / 4.0)[:, None, None]
            add(4 * A + i, 4 * B + 3, -V[:, None, None] / 4.0 * gi_a - 1j * om * t4 * gi_b)
            add(4 * A + 3, 4 * B + i, V[:, None, None] / 4.0 * gi_b + 1j * om * t4 * gi_a)
        add(4 * A + 3, 4 * B + 3, (tau / rho)[:, None, None] * S)
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(4 * n, 4 * n))
        # Dirichlet data of mode k from the real harmonics (a0, a1, b1, ...): a0, (a_k - i b_k) / 2
        ud = np.zeros((n, 4), dtype=complex)
        h = exact[:, :3]
        ud[:, :3] = h[:, :, 0] if k == 0 else (h[:, :, 2 * k - 1] - 1j * h[:, :, 2 * k]) / 2.0
        ud[~mask, :3] = 0.0
        wall = np.unique(pr.faces[pr.face_tag == 0].ravel())
        ud[wall, :3] = 0.0
        ud = ud.ravel()
        rhs = -(K @ ud)                                              # traction-free outlet: no boundary load
        x = ud.copy()
        x[free] = spla.spsolve(K[free][:, free].tocsc(), rhs[free])
        sol.append(x.reshape(n, 4))
    t = O.instance_times(N, pr.T)
    y = np.zeros((n, 4, N)) + sol[0].real[:, :, None]
    for k in range(1, n_h + 1):
        y += 2.0 * (sol[k][:, :, None] * np.exp(1j * k * w * t)[None, None, :]).real
    return y


def test_stokes_limit_root_matches_womersley_at_second_order():
    errs = []
    for level in (1, 2):
        pr, exact = _problem(level)
        y = _mode_solution(pr, exact)
        r = O.residual(pr, y)
        scale = np.abs(O.residual(pr, pr.initial_state())).max()
        assert np.abs(r).max() < 1e-9 * scale, level
        hm = O.instances_to_harmonics(y, pr.n_h)
        errs.append(float(np.linalg.norm(hm[:, :3] - exact[:, :3]) / np.linalg.norm(exact[:, :3])))
    print("Womersley velocity errors (oracle, Stokes limit):", errs)
    assert errs[0] < 0.08
    assert errs[1] < errs[0] / 3.0            # second order in h gives ~4x per halving


def test_mode_solution_notices_a_wrong_viscosity():
    """The same construction with the viscosity changed by 10 % no longer zeroes the oracle's residual
    (the check above is not satisfied by construction)."""
    pr, exact = _problem(1)
    mu0 = pr.mu
    pr.mu = 1.1 * mu0
    pr.nu = pr.mu / pr.rho
    y = _mode_solution(pr, exact)
    pr.mu = mu0
    pr.nu = mu0 / pr.rho
    r = O.residual(pr, y)
    scale = np.abs(O.residual(pr, pr.initial_state())).max()
    assert np.abs(r).max() > 1e-4 * scale
