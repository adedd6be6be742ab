"""Plain FP64 CPU oracle of the conventional time-stepping GLS solver the paper compares against.

TEST INFRASTRUCTURE ONLY: the tests use it to check the GPU time-marching path; it shares no code with
the CUDA library.  It reuses the mesh geometry, quadrature and boundary-face data of the HB oracle
(hb_oracle.py), which is pinned on its own.

The paper (Sec. 3, Eq. tauhat) runs the same GLS stabilisation in the time domain with the acceleration
in the stabilisation parameter:
    tau_hat = (omega_hat^2 + u . xi u + C_I nu^2 xi : xi)^(-1/2),   omega_hat = ||du/dt|| / ||u||
and a time integrator of generalized-alpha type (the pseudo-time term of Sec. 2.3 uses one, with
rho_inf = 0 giving c1 = 1.5).  One time level's residual, with u, p and du/dt given:
    r^m_A,i = int N_A rho du_i/dt + rho N_A u . grad u_i + mu grad N_A . grad u_i - dN_A/dx_i p
              + (u . grad N_A) tau_hat L_i                                       (+ Neumann, backflow)
    r^c_A   = int N_A div u + (1 / rho) grad N_A . tau_hat L
    L_i     = rho du_i/dt + rho u . grad u_i + dp/dx_i
i.e. Eq. (NS-weak) with H u replaced by du/dt and without the least-squares H term (test functions do
not depend on time).  Readings of what the paper leaves open (Sec. 3, Eq. tauhat, Sec. 2.3):
  R13 Generalized-alpha for first-order systems (Jansen, Whiting & Hulbert 2000): alpha_m =
      (3 - rho_inf) / (2 (1 + rho_inf)), alpha_f = 1 / (1 + rho_inf), gamma = 1/2 + alpha_m - alpha_f;
      the residual is taken at (u, p)_{n+alpha_f} and du/dt_{n+alpha_m} (the pressure at the same
      level as the velocity keeps it second-order accurate); Dirichlet values at t_{n+1}, outlet
      pressures at t_{n+alpha_f}.  rho_inf = 0.5 unless stated.
  R14 omega_hat^2 = ||du/dt||^2 / ||u||^2 over the nodal velocity vectors (discrete 2-norms) of the
      current iterate.
  R15 The tangent is the paper's (Eqs. K_mat, ctangent) at N = 1 with U and tau_hat frozen, plus the
      acceleration's derivative: c1 rho / dt M on the velocity (Galerkin) and c1 rho / dt v inside the
      least-squares L of both rows, c1 = alpha_m / (alpha_f gamma).  (The HB tangent has no such term:
      its time coupling is the F block.)  The Jacobi preconditioner takes the diagonal of this tangent
      without the least-squares acceleration cross term (u . grad N_A) tau c1 rho / dt N_A, which has no
      sign and can cancel the Galerkin mass diagonal; the Galerkin c1 rho / dt M_AA stays in it.

Array layouts: one time level is [n_nodes, 4] (u1, u2, u3, p).
"""
from __future__ import annotations

import math

import numpy as np

from oracle import hb_oracle as HB

C_I = HB.C_I
NQ, MREF, MID = HB.NQ, HB.MREF, HB._MID


def galpha(rho_inf: float = 0.5):
    """(alpha_m, alpha_f, gamma) of generalized-alpha for first-order systems (reading R13)."""
    am = (3.0 - rho_inf) / (2.0 * (1.0 + rho_inf))
    af = 1.0 / (1.0 + rho_inf)
    return am, af, 0.5 + am - af


def series(a, b, omega: float, t: float) -> float:
    """a0 + sum_k (a_k cos k omega t + b_k sin k omega t): the boundary data's real series (Eq. upgh_def)
    at time t."""
    k = np.arange(1, len(a))
    return float(a[0] + np.sum(a[1:] * np.cos(k * omega * t)) + np.sum(b[1:] * np.sin(k * omega * t)))


def dirichlet_at(prob: HB.HBProblem, t: float):
    """(mask [n], g [n, 3]) at time t: inflow profile x waveform(t), or per-point harmonics at t; walls 0
    (reading R11, evaluated at one time instead of the instances)."""
    mask = np.zeros(prob.n_nodes, dtype=bool)
    g = np.zeros((prob.n_nodes, 3))
    w = prob.omega
    for tag, (prof, a, b) in prob.inflow.items():
        nodes = np.unique(prob.faces[prob.face_tag == tag].ravel())
        if isinstance(prof, str):
            c = a[nodes]                                   # [m, 3, 2 n_h + 1]: a0, a1, b1, a2, b2, ...
            nh = (c.shape[2] - 1) // 2
            val = c[:, :, 0].copy()
            for k in range(1, nh + 1):
                val += c[:, :, 2 * k - 1] * math.cos(k * w * t) + c[:, :, 2 * k] * math.sin(k * w * t)
            g[nodes] = val
        else:
            g[nodes] = prof[nodes] * series(a, b, w, t)
        mask[nodes] = True
    wall = np.unique(prob.faces[prob.face_tag == 0].ravel())
    g[wall] = 0.0
    mask[wall] = True
    return mask, g


def _outlet_h(prob: HB.HBProblem, y: np.ndarray, t: float) -> np.ndarray:
    """Traction level h per face at time t: -P(t) (reading R5), or -(P_d(t) + R Q) for resistance outlets
    (R8)."""
    h = np.zeros(prob.faces.shape[0])
    for tag, (a, b) in prob.outlet_p.items():
        h[prob.face_tag == tag] = -series(a, b, prob.omega, t)
    for tag, (R, a, b) in prob.outlet_r.items():
        f = np.nonzero(prob.face_tag == tag)[0]
        Q = float(np.sum(prob.face_area[f] / 3.0 * np.einsum("fbi,fi->f", y[prob.faces[f]][:, :, :3],
                                                                 prob.face_normal[f])))
        h[f] = -(series(a, b, prob.omega, t) + R * Q)
    return h


def _boundary(prob: HB.HBProblem, y: np.ndarray, h: np.ndarray) -> np.ndarray:
    """- int N_A h n_i - int N_A (rho/2) beta |u.n|_- u_i over the Neumann faces (reading R5)."""
    out = np.zeros((prob.n_nodes, 3))
    fn = prob.neumann_faces()
    if fn.size == 0:
        return out
    S, nrm, nodes = prob.face_area[fn], prob.face_normal[fn], prob.faces[fn]
    neu = -(S / 3.0)[:, None] * nrm * h[fn][:, None]
    um = np.einsum("mb,fbi->fmi", MID, y[nodes][:, :, :3])
    s = np.einsum("fmi,fi->fm", um, nrm)
    sm = 0.5 * (s - np.abs(s))
    bf = -(0.5 * prob.rho * prob.beta_bf) * np.einsum("f,mb,fm,fmi->fbi", S / 3.0, MID, sm, um)
    for b in range(3):
        np.add.at(out, nodes[:, b], neu + bf[:, b])
    return out


def _state(prob: HB.HBProblem, y: np.ndarray, omega2: float):
    """Per element and quadrature point: u and tau_hat of Eq. (tauhat) with omega_hat^2 = omega2 (R14)."""
    t = prob.tets
    g = prob.geo
    U = y[t][:, :, :3]                                     # [e, a, i]
    Uq = np.einsum("qa,eai->eqi", NQ, U)
    g2 = C_I * prob.nu ** 2 * g.GG
    uGu = np.einsum("eqi,eij,eqj->eq", Uq, g.G, Uq)
    tau = 1.0 / np.sqrt(omega2 + uGu + g2[:, None])        # Eq. (tauhat)
    return t, U, Uq, tau


def residual(prob: HB.HBProblem, y: np.ndarray, ydot: np.ndarray, t: float, omega2: float) -> np.ndarray:
    """Time-domain GLS residual [n, 4] of one time level of the conventional solver of Sec. 3 (module
    docstring; readings R13, R14); Dirichlet momentum rows 0."""
    rho, mu = prob.rho, prob.mu
    tt, U, Uq, tau = _state(prob, y, omega2)
    gN, V = prob.geo.gradN, prob.geo.V
    P = y[tt][:, :, 3]
    Ud = ydot[tt][:, :, :3]
    Udq = np.einsum("qa,eai->eqi", NQ, Ud)
    gradU = np.einsum("eai,eaj->eij", U, gN)
    gradP = np.einsum("ea,eaj->ej", P, gN)
    conv = np.einsum("eqj,eij->eqi", Uq, gradU)
    L = rho * Udq + rho * conv + gradP[:, None, :]
    tL = tau[:, :, None] * L
    udN = np.einsum("eqj,eaj->eqa", Uq, gN)
    w = V / 4.0
    Qm = (rho * V[:, None, None] * np.einsum("ab,ebi->eai", MREF, Ud)
          + rho * np.einsum("e,qa,eqi->eai", w, NQ, conv)
          + np.einsum("e,eqa,eqi->eai", w, udN, tL)
          + mu * V[:, None, None] * np.einsum("eaj,eij->eai", gN, gradU)
          - V[:, None, None] * gN * P.mean(axis=1)[:, None, None])
    Qc = (w * np.einsum("eii->e", gradU))[:, None] + (1.0 / rho) * np.einsum("e,eai,eqi->ea", w, gN, tL)
    rm = np.zeros((prob.n_nodes, 3))
    rc = np.zeros(prob.n_nodes)
    for a in range(4):
        np.add.at(rm, tt[:, a], Qm[:, a])
        np.add.at(rc, tt[:, a], Qc[:, a])
    rm += _boundary(prob, y, _outlet_h(prob, y, t))
    mask, _ = dirichlet_at(prob, t)
    rm[mask] = 0.0
    return np.concatenate([rm, rc[:, None]], axis=1)


def jv_paper(prob: HB.HBProblem, y: np.ndarray, v: np.ndarray, omega2: float, shift: float,
             ls_acceleration: bool = True) -> np.ndarray:
    """Paper tangent at N = 1 with U and tau_hat frozen at y, plus the acceleration's derivative (R15):
    shift M on the velocity and, with ls_acceleration, shift v inside the least-squares L of both rows.
    Dirichlet velocity rows are the identity on v, whose Dirichlet velocity entries count as 0."""
    rho, mu = prob.rho, prob.mu
    mask, _ = dirichlet_at(prob, 0.0)
    vm = v.copy()
    vm[mask, :3] = 0.0
    tt, U, Uq, tau = _state(prob, y, omega2)
    gN, V = prob.geo.gradN, prob.geo.V
    dU = vm[tt][:, :, :3]
    dP = vm[tt][:, :, 3]
    gradV = np.einsum("eai,eaj->eij", dU, gN)
    gradVp = np.einsum("ea,eaj->ej", dP, gN)
    ugv = np.einsum("eqj,eij->eqi", Uq, gradV)
    udN = np.einsum("eqj,eaj->eqa", Uq, gN)
    w = V / 4.0
    Vb = V[:, None, None]
    dUq = np.einsum("qa,eai->eqi", NQ, dU) * (1.0 if ls_acceleration else 0.0)
    Kv = (rho * np.einsum("e,qa,eqi->eai", w, NQ, ugv)
          + mu * Vb * np.einsum("eaj,eij->eai", gN, gradV)
          + rho * np.einsum("e,eq,eqa,eqi->eai", w, tau, udN, ugv)
          + shift * Vb * np.einsum("ab,ebi->eai", MREF, dU)
          + shift * np.einsum("e,eq,eqa,eqi->eai", w, tau, udN, dUq))
    Gv = -Vb * gN * dP.mean(axis=1)[:, None, None] + np.einsum("e,eq,eqa,ei->eai", w, tau, udN, gradVp)
    Dv = ((w * np.einsum("eii->e", gradV))[:, None] + np.einsum("e,eq,eaj,eqj->ea", w, tau, gN, ugv)
          + (shift / rho) * np.einsum("e,eq,eaj,eqj->ea", w, tau, gN, dUq))
    Lv = (1.0 / rho) * np.einsum("e,eq,eaj,ej->ea", w, tau, gN, gradVp)
    rm = np.zeros((prob.n_nodes, 3))
    rc = np.zeros(prob.n_nodes)
    for a in range(4):
        np.add.at(rm, tt[:, a], (Kv + Gv)[:, a])
        np.add.at(rc, tt[:, a], (Dv + Lv)[:, a])
    # boundary: backflow with its coefficient frozen, resistance rank-one term
    fn = prob.neumann_faces()
    if fn.size:
        S, nrm, nodes = prob.face_area[fn], prob.face_normal[fn], prob.faces[fn]
        dh = np.zeros(prob.faces.shape[0])
        for tag, (R, a, b) in prob.outlet_r.items():
            f = np.nonzero(prob.face_tag == tag)[0]
            Qv = float(np.sum(prob.face_area[f] / 3.0 * np.einsum("fbi,fi->f", vm[prob.faces[f]][:, :, :3],
                                                                      prob.face_normal[f])))
            dh[f] = -R * Qv
        neu = -(S / 3.0)[:, None] * nrm * dh[fn][:, None]
        um = np.einsum("mb,fbi->fmi", MID, y[nodes][:, :, :3])
        vmid = np.einsum("mb,fbi->fmi", MID, vm[nodes][:, :, :3])
        s = np.einsum("fmi,fi->fm", um, nrm)
        sm = 0.5 * (s - np.abs(s))
        bf = -(0.5 * prob.rho * prob.beta_bf) * np.einsum("f,mb,fm,fmi->fbi", S / 3.0, MID, sm, vmid)
        for b in range(3):
            np.add.at(rm, nodes[:, b], neu + bf[:, b])
    rm[mask] = v[mask, :3]
    return np.concatenate([rm, rc[:, None]], axis=1)


def jacobi_diag(prob: HB.HBProblem, y: np.ndarray, omega2: float, shift: float) -> np.ndarray:
    """Diagonal of the volume part of jv_paper without the least-squares acceleration term (R15); 1 on
    Dirichlet velocity rows; [n, 4]."""
    rho, mu = prob.rho, prob.mu
    tt, U, Uq, tau = _state(prob, y, omega2)
    gN, V = prob.geo.gradN, prob.geo.V
    udN = np.einsum("eqj,eaj->eqa", Uq, gN)
    w = V / 4.0
    gg = np.einsum("eaj,eaj->ea", gN, gN)
    dv = (rho * np.einsum("e,qa,eqa->ea", w, NQ, udN) + rho * np.einsum("e,eq,eqa->ea", w, tau, udN ** 2)
          + mu * V[:, None] * gg + shift * V[:, None] * MREF[0, 0])
    dp = (1.0 / rho) * np.einsum("e,eq,ea->ea", w, tau, gg)
    d = np.zeros((prob.n_nodes, 4))
    for a in range(4):
        np.add.at(d[:, 0], tt[:, a], dv[:, a])
        np.add.at(d[:, 3], tt[:, a], dp[:, a])
    d[:, 1] = d[:, 0]
    d[:, 2] = d[:, 0]
    mask, _ = dirichlet_at(prob, 0.0)
    d[mask, :3] = 1.0
    return d


def omega_hat2(y: np.ndarray, ydot: np.ndarray) -> float:
    """Reading R14: ||du/dt||^2 / ||u||^2 over the nodal velocity vectors."""
    uu = float(np.sum(y[:, :3] ** 2))
    return float(np.sum(ydot[:, :3] ** 2)) / uu if uu > 0 else 0.0


def march(prob: HB.HBProblem, steps_per_period: int, periods: float, rho_inf: float = 0.5,
          newton_tol: float = 1e-12, newton_max: int = 30, gmres_tol: float = 1e-13, use_omega: bool = True,
          y0=None, record_every: int = 0):
    """Generalized-alpha time marching from y0 (default: zero interior velocity, Dirichlet values at 0,
    pressure 0) with zero initial acceleration.  Each step: predictor (same velocity and pressure, du/dt
    scaled by (gamma - 1) / gamma, Dirichlet nodes moved to their values), then Newton on the paper
    tangent (R15) with GMRES, each correction solving (K + c1 rho / dt M) d = -r / alpha_f and updating
    (u, p) += d, du/dt += d_u / (gamma dt).  Returns (y, ydot, records) with records the states every
    record_every steps."""
    dt = prob.T / steps_per_period
    am, af, gam = galpha(rho_inf)
    c1 = am / (af * gam)
    n = prob.n_nodes
    mask, g = dirichlet_at(prob, 0.0)
    y = np.zeros((n, 4)) if y0 is None else np.array(y0, dtype=np.float64)
    y[mask, :3] = g[mask]
    yd = np.zeros((n, 4))
    recs = []
    nsteps = int(round(steps_per_period * periods))
    for k in range(nsteps):
        t1 = (k + 1) * dt
        _, g1 = dirichlet_at(prob, t1)
        y1 = y.copy()
        yd1 = (gam - 1.0) / gam * yd
        y1[mask, :3] = g1[mask]
        yd1[mask, :3] = (g1[mask] - y[mask, :3]) / (gam * dt) + (gam - 1.0) / gam * yd[mask, :3]
        r0 = None
        for _ in range(newton_max):
            ya = y + af * (y1 - y)
            yda = yd + am * (yd1 - yd)
            om2 = omega_hat2(ya, yda) if use_omega else 0.0
            r = residual(prob, ya, yda, k * dt + af * dt, om2)
            rn = np.linalg.norm(r)
            r0 = rn if r0 is None else r0
            if rn <= newton_tol * max(r0, 1e-300) or rn == 0.0:
                break
            shp = r.shape
            mv = lambda x: jv_paper(prob, ya, x.reshape(shp), om2, c1 * prob.rho / dt).ravel()  # noqa: E731
            dg = jacobi_diag(prob, ya, om2, c1 * prob.rho / dt).ravel()
            d, _ = HB.gmres(mv, -r.ravel() / af, lambda z: z / dg, gmres_tol, restart=60)
            d = d.reshape(shp)
            d[mask, :3] = 0.0
            y1 += d
            yd1[:, :3] += d[:, :3] / (gam * dt)
        y, yd = y1, yd1
        if record_every and (k + 1) % record_every == 0:
            recs.append(y.copy())
    return y, yd, recs
