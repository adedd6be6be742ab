"""Plain FP64 CPU oracle of the harmonic balance (HB) Galerkin/least-squares Navier-Stokes method.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct statement of what the GPU path
computes; only the tests, the smoke check and the CPU-baseline leg of the benchmark may import it.  It
shares no code with the CUDA library (the only common inputs come from the seeded input generators).

Everything follows the paper's Sec. 2 (arXiv 2411.14315):
  * Eq. (NS-harm): HB Navier-Stokes, H = E^-1 Omega E acting across the N = 2 N_h + 1 time instances;
  * Eq. (NS-weak) / Eq. (Rmc): the GLS weak form and its discrete residual for P1 tetrahedra;
  * Eq. (tau): the per-instance stabilisation parameter;
  * Eqs. (splitK), (ptangent), (K_mat), (ctangent), (F_mat): the paper's tangent L~ = C + P;
  * Sec. 2.3 pseudo time stepping (c1 = 1.5), CFL rule, backflow stabilisation, Jacobi + GMRES.

Readings of points the paper leaves open, each with the passage it interprets (the labels R1-R9, R17 and R18 are
the same in the library's headers and tests):
  R1  (Eq. NS-harm, Eqs. upghdft/upghharm) H is the real Fourier spectral differentiation matrix on
      t_n = n T / N (odd N):
      H[j,k] = (w/2) (-1)^(j-k) / sin(pi (j-k) / N), H[j,j] = 0.  This is what E^-1 Omega E means once
      Omega's mode index is taken as the signed frequency of each DFT row.
  R2  (Eq. Rmc; the paper names no rule) Volume integrals use the 4-point degree-2 Gauss rule; tau is evaluated per quadrature point.
  R3  (Eq. tau) xi is the metric of the map to the parent tetrahedron (0,0,0),(1,0,0),(0,1,0),(0,0,1)
      with local node 0 at the origin: G = J^-T J^-1, so tau depends on the local vertex order.
  R4  (Eq. Rmc) The "-H N_A" least-squares term and the Galerkin rho N_A H u term are applied as one H product
      after spatial assembly: r^m = Q^m + H T, T_A = rho M u - sum_e int N_A tau L (exact algebra).
  R5  (Sec. 2.1 traction condition; Sec. 2.3 backflow) Outlet pressure P gives h = -P; backflow term kept literally as printed, (rho/2) beta |u.n|_-
      with |x|_- = (x - |x|)/2, integrated with the 3-point edge-midpoint face rule.
  R6  (Sec. 2.3, Eq. NR) Pseudo time stepping is pseudo-transient continuation: each pseudo step solves
      (L~ + c1 rho / dt M_vel) d = -r(y), r the steady HB residual, so the root is unchanged.
  R7  (Eqs. splitK, ptangent, K_mat, ctangent, F_mat) The paper's tangent freezes U and tau at y and keeps only the Galerkin H term (Eq. F_mat); the
      backflow term enters it with its coefficient frozen.  The exact Jacobian is the full derivative.
  R8  (Sec. 3, Sec. 4 future work) Resistance outlets (h = -(P_d + R Q), Q the instantaneous outlet flux) are an extension; the
      paper leaves them out of scope (Sec. 3).
  R9  (Sec. 2.3) The Jacobi preconditioner is diag(P) + c1 rho/dt M_AA over the volume terms (Sec. 2.3); C has a
      zero diagonal because H does.
  R17 (Sec. 2.2, remark 2 after Eq. tau) "Full RBVMS": the subscale velocity u' = -tau L / rho, which the
      least-squares terms already place in the time coupling and the advected velocity, is also added to
      the advecting velocity: cross stress int N_a rho u' . grad u_i and Reynolds stress
      - int rho (u' . grad N_a) u'_i; no other term.  The paper's tangent keeps the GLS blocks; the exact
      Jacobian includes the added terms.
  R18 (Sec. 2.2, remark 4 after Eq. tau) The time-discretisation term of tau is ct_dt (1 / dt)^2 under the
      root with the equivalent step dt = 2 pi / (N w) = T / N; ct_dt = 1 takes the remark's (1/dt)^2.

Array layouts: instance vectors are [n_nodes, 4, N] (u1, u2, u3, p; N instances contiguous).
"""
from __future__ import annotations

import math

import numpy as np

C_I = 3.0                          # Eq. (tau): shape-function constant for tetrahedra
C1_PSEUDO = 1.5                    # Sec. 2.3: generalized-alpha with rho_inf = 0
QA = 0.5854101966249685            # 4-point Gauss rule on a tetrahedron: barycentric coordinates
QB = 0.1381966011250105
NQ = np.full((4, 4), QB) + np.eye(4) * (QA - QB)     # NQ[q, a] = N_a at quadrature point q
MREF = (np.ones((4, 4)) + np.eye(4)) / 20.0          # int N_a N_b = V (1 + delta_ab) / 20


# ---------------------------------------------------------------------------------------------------
# time operators (Sec. 2.1)


def n_instances(n_h: int) -> int:
    """N = 2M - 1 with M - 1 = n_h retained harmonics (Sec. 2.1, after Eq. upghdft)."""
    return 2 * n_h + 1


def instance_times(N: int, T: float) -> np.ndarray:
    """Equally spaced instances t_n = n T / N, n = 0..N-1 (Eq. upghharm)."""
    return T * np.arange(N) / N


def dft_E(N: int) -> np.ndarray:
    """E[j,k] = (1/N) exp(-2 pi i j k / N) (Sec. 2.1, Eq. upghdft)."""
    j = np.arange(N)
    return np.exp(-2j * np.pi * np.outer(j, j) / N) / N


def spectral_H(N: int, omega: float) -> np.ndarray:
    """H = E^-1 Omega E in real closed form (reading R1): the Fourier differentiation matrix."""
    H = np.zeros((N, N))
    for j in range(N):
        for k in range(N):
            if j != k:
                d = j - k
                H[j, k] = 0.5 * omega * (-1.0) ** d / math.sin(math.pi * d / N)
    return H


def sample_waveform(a, b, N: int, T: float) -> np.ndarray:
    """q(t_n) for q(t) = a0 + sum_k a_k cos(k w t) + b_k sin(k w t): the truncated Fourier series of a
    boundary condition (Eq. upgh_def) evaluated at the instances (Eq. upghdft)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    t = instance_times(N, T)
    w = 2.0 * math.pi / T
    q = np.full(N, a[0])
    for k in range(1, len(a)):
        q += a[k] * np.cos(k * w * t) + b[k] * np.sin(k * w * t)
    return q


def instances_to_harmonics(y: np.ndarray, n_h: int) -> np.ndarray:
    """Fourier coefficients of instance values (Sec. 3.2 reconstruction; u* = E u, Eq. upghdft) in real
    form (a0, a1, b1, ..., a_nh, b_nh) with a_k = 2 Re u*_k, b_k = -2 Im u*_k.  y [..., N]."""
    N = y.shape[-1]
    c = y @ dft_E(N).T                      # c[..., m] = sum_n E[m, n] y[..., n]
    out = np.empty(y.shape[:-1] + (2 * n_h + 1,))
    out[..., 0] = c[..., 0].real
    for k in range(1, n_h + 1):
        out[..., 2 * k - 1] = 2.0 * c[..., k].real
        out[..., 2 * k] = -2.0 * c[..., k].imag
    return out


def harmonics_to_instances(coef: np.ndarray, N: int, T: float) -> np.ndarray:
    """Inverse of instances_to_harmonics: the real series of Eq. (upgh_def) evaluated at the instances
    of Eq. (upghharm)."""
    n_h = (coef.shape[-1] - 1) // 2
    t = instance_times(N, T)
    w = 2.0 * math.pi / T
    y = np.repeat(coef[..., :1], N, axis=-1).astype(np.float64)
    for k in range(1, n_h + 1):
        y = y + coef[..., 2 * k - 1:2 * k] * np.cos(k * w * t) + coef[..., 2 * k:2 * k + 1] * np.sin(k * w * t)
    return y


# ---------------------------------------------------------------------------------------------------
# geometry of P1 tetrahedra (Sec. 2.3, Eq. tau)


class Geometry:
    """Per-element shape gradients, volume and parent-map metric (reading R3)."""

    def __init__(self, xyz: np.ndarray, tets: np.ndarray):
        x = xyz[tets]                                   # [E, 4, 3]
        J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)  # columns
        det = np.linalg.det(J)
        Jinv = np.linalg.inv(J)                         # row k = grad of parent coordinate xi_k
        g = np.empty((tets.shape[0], 4, 3))
        g[:, 1:] = Jinv
        g[:, 0] = -Jinv.sum(axis=1)
        self.V = np.abs(det) / 6.0
        self.gradN = g                                  # [E, a, j] = dN_a / dx_j
        self.G = np.einsum("eki,ekj->eij", Jinv, Jinv)  # xi = J^-T J^-1
        self.GG = np.einsum("eij,eij->e", self.G, self.G)


# ---------------------------------------------------------------------------------------------------
# problem definition (Eq. NS-time boundary conditions; Sec. 2.3 Dirichlet built into the unknowns)


class HBProblem:
    """Mesh + fluid + boundary conditions of one HB solve (the problem statement of Sec. 2.1: domain,
    rho, mu, period, N_h; inflow and outlet data as harmonics, Sec. 2.1 and Sec. 3).

    Face tags: 0 = no-slip wall.  Inflow tags carry Dirichlet g = profile(x) q(t); pressure outlets
    h = -P(t); resistance outlets h = -(P_d(t) + R Q(t)); other tags are traction-free (h = 0).
    Backflow stabilisation acts on every Neumann face."""

    def __init__(self, xyz, tets, faces, face_tag, rho: float, mu: float, T: float, n_h: int,
                 beta_bf: float = 0.2, convection: bool = True):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        self.faces = np.asarray(faces, dtype=np.int64)
        self.face_tag = np.asarray(face_tag, dtype=np.int64)
        self.rho, self.mu, self.T, self.n_h = float(rho), float(mu), float(T), int(n_h)
        self.nu = self.mu / self.rho
        self.N = n_instances(n_h)
        self.omega = 2.0 * math.pi / self.T
        self.H = spectral_H(self.N, self.omega)
        self.beta_bf = float(beta_bf)
        self.convection = convection      # False only for the Stokes-mode check of the tests
        # stabilisation variants of Sec. 2.2 (remarks after Eq. tau), readings R17 and R18:
        #   stab = "gls": Eq. (NS-weak) as printed; "rbvms": the subscale velocity u' = -tau L / rho is added
        #   to every velocity of the Galerkin convective term (cross- and Reynolds-stress terms);
        #   ct_dt > 0: ct_dt (1 / dt)^2 under the root of Eq. (tau), dt = 2 pi / (N w) = T / N
        self.stab = "gls"
        self.ct_dt = 0.0
        self.n_nodes = self.xyz.shape[0]
        self.geo = Geometry(self.xyz, self.tets)
        self.inflow = {}
        self.outlet_p = {}
        self.outlet_r = {}
        self._face_geometry()

    # boundary faces: outward unit normal (away from the owning tetrahedron's opposite vertex) and area
    def _face_geometry(self):
        """Outward unit normal and area of every boundary face (for the surface integrals of Eq. NS-weak)."""
        loc = np.array([(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)])
        tf = np.sort(self.tets[:, loc].reshape(-1, 3), axis=1)
        n = self.n_nodes
        key_t = (tf[:, 0] * n + tf[:, 1]) * n + tf[:, 2]
        sf = np.sort(self.faces, axis=1)
        key_f = (sf[:, 0] * n + sf[:, 1]) * n + sf[:, 2]
        order = np.argsort(key_t)
        pos = np.searchsorted(key_t[order], key_f)
        if np.any(pos >= len(order)) or np.any(key_t[order][np.minimum(pos, len(order) - 1)] != key_f):
            raise ValueError("boundary face not found in any tetrahedron")
        owner = order[pos]
        tet = owner // 4
        opp = self.tets[tet, owner % 4]
        p = self.xyz[self.faces]
        cr = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
        area = 0.5 * np.linalg.norm(cr, axis=1)
        nrm = cr / (2.0 * area[:, None])
        away = p.mean(axis=1) - self.xyz[opp]
        nrm *= np.sign(np.einsum("fi,fi->f", nrm, away))[:, None]
        self.face_area = area
        self.face_normal = nrm

    def set_inflow(self, tag: int, profile, a, b):
        """Separable Dirichlet data g = profile(x) q(t), q a real Fourier series (Eq. upgh_def)."""
        self.inflow[int(tag)] = (np.asarray(profile, dtype=np.float64), np.asarray(a, float), np.asarray(b, float))

    def set_inflow_harmonics(self, tag: int, harmonics):
        """General Dirichlet data: per-point real harmonics [n_nodes, 3, 2 n_h + 1] (Eq. upgh_def)."""
        self.inflow[int(tag)] = ("harmonics", np.asarray(harmonics, dtype=np.float64), None)

    def set_outlet_pressure(self, tag: int, a, b):
        """Outlet pressure P(t) as a real Fourier series; traction h = -P (reading R5)."""
        self.outlet_p[int(tag)] = (np.asarray(a, float), np.asarray(b, float))

    def set_outlet_resistance(self, tag: int, R: float, a, b):
        """Resistance outlet h = -(P_d(t) + R Q(t)) (reading R8; an extension, not in the paper)."""
        self.outlet_r[int(tag)] = (float(R), np.asarray(a, float), np.asarray(b, float))

    # derived boundary data
    def dirichlet(self):
        """(mask [n_nodes] bool, g [n_nodes, 3, N]) at the instances: wall nodes (u = 0) take priority over
        inflow (reading R11)."""
        N = self.N
        mask = np.zeros(self.n_nodes, dtype=bool)
        g = np.zeros((self.n_nodes, 3, N))
        for tag, (prof, a, b) in self.inflow.items():
            nodes = np.unique(self.faces[self.face_tag == tag].ravel())
            if isinstance(prof, str):
                g[nodes] = harmonics_to_instances(a[nodes], N, self.T)
            else:
                q = sample_waveform(a, b, N, self.T)
                g[nodes] = prof[nodes][:, :, None] * q[None, None, :]
            mask[nodes] = True
        wall = np.unique(self.faces[self.face_tag == 0].ravel())
        g[wall] = 0.0
        mask[wall] = True
        return mask, g

    def neumann_faces(self) -> np.ndarray:
        """Faces of the Neumann part of the boundary (every tag that is neither wall nor inflow)."""
        dir_tags = set(self.inflow) | {0}
        return np.nonzero(~np.isin(self.face_tag, list(dir_tags)))[0]

    def initial_state(self) -> np.ndarray:
        """y0: Dirichlet values built in (Sec. 2.3), zero interior velocity, pressure at the mean outlet
        level (mean over pressure / resistance outlets of P_d at each instance)."""
        mask, g = self.dirichlet()
        y = np.zeros((self.n_nodes, 4, self.N))
        y[mask, :3] = g[mask]
        levels = [sample_waveform(a, b, self.N, self.T) for (a, b) in self.outlet_p.values()]
        levels += [sample_waveform(a, b, self.N, self.T) for (_, a, b) in self.outlet_r.values()]
        if levels:
            y[:, 3, :] = np.mean(levels, axis=0)[None, :]
        return y

    def apply_dirichlet(self, y: np.ndarray) -> np.ndarray:
        """y with the prescribed velocities of Sec. 2.3 built in."""
        mask, g = self.dirichlet()
        y = y.copy()
        y[mask, :3] = g[mask]
        return y


# ---------------------------------------------------------------------------------------------------
# element terms of the residual (Eq. Rmc with readings R2-R4)


def tau_dt_term(prob: HBProblem) -> float:
    """ct_dt (1 / dt)^2 with the equivalent step dt = 2 pi / (N w) = T / N of the remark on the
    time-discretisation term of tau (Sec. 2.2, reading R18); 0 for Eq. (tau) as printed."""
    dt = prob.T / prob.N
    return prob.ct_dt / (dt * dt)


def _apply_H(prob: HBProblem, x: np.ndarray) -> np.ndarray:
    """Instance coupling of Eq. (NS-harm): (H x)[..., j] = sum_k H[j, k] x[..., k]."""
    return x @ prob.H.T


def _element_state(prob: HBProblem, y: np.ndarray, elems):
    """Per element and quadrature point: u, H u, grad u, grad p and tau of Eq. (tau) at every instance
    (readings R2, R3)."""
    t = prob.tets[elems]
    g = prob.geo
    U = y[t][:, :, :3, :]                               # [e, a, i, n]
    P = y[t][:, :, 3, :]                                # [e, a, n]
    gN = g.gradN[elems]
    V = g.V[elems]
    G = g.G[elems]
    g2 = C_I * prob.nu ** 2 * g.GG[elems] + tau_dt_term(prob)
    Uq = np.einsum("qa,eain->eqin", NQ, U)
    if not prob.convection:
        Uq_tau = np.zeros_like(Uq)
    else:
        Uq_tau = Uq
    uGu = np.einsum("eqin,eij,eqjn->eqn", Uq_tau, G, Uq_tau)
    tau = 1.0 / np.sqrt(uGu + g2[:, None, None])         # Eq. (tau), per quadrature point and instance
    gradU = np.einsum("eain,eaj->eijn", U, gN)          # d u_i / d x_j
    gradP = np.einsum("ean,eaj->ejn", P, gN)
    return dict(t=t, U=U, P=P, gN=gN, V=V, G=G, Uq=Uq, Uq_tau=Uq_tau, tau=tau, gradU=gradU, gradP=gradP)


def element_residual(prob: HBProblem, y: np.ndarray, elems=None):
    """Per-element (Qm [e,a,i,n], T [e,a,i,n], Qc [e,a,n]) such that the assembled residual is
    r^m = Qm + H T and r^c = Qc (reading R4)."""
    if elems is None:
        elems = np.arange(prob.tets.shape[0])
    s = _element_state(prob, y, elems)
    rho, mu = prob.rho, prob.mu
    V, gN, U, P = s["V"], s["gN"], s["U"], s["P"]
    HU = _apply_H(prob, U)
    HUq = np.einsum("qa,eain->eqin", NQ, HU)
    conv = np.einsum("eqjn,eijn->eqin", s["Uq"], s["gradU"]) if prob.convection else np.zeros_like(HUq)
    L = rho * HUq + rho * conv + s["gradP"][:, None, :, :]      # momentum operator (no viscous term, P1)
    tL = s["tau"][:, :, None, :] * L
    udN = np.einsum("eqjn,eaj->eqan", s["Uq_tau"], gN)       # u_q . grad N_a (zero without convection)
    w = V / 4.0
    pbar = P.mean(axis=1)                                      # int p dOmega / V for P1
    div = np.einsum("eiin->en", s["gradU"])
    Qm = (rho * np.einsum("e,qa,eqin->eain", w, NQ, conv)
          + np.einsum("e,eqan,eqin->eain", w, udN, tL)
          + mu * V[:, None, None, None] * np.einsum("eaj,eijn->eain", gN, s["gradU"])
          - V[:, None, None, None] * gN[:, :, :, None] * pbar[:, None, None, :])
    if prob.stab == "rbvms":
        # u' = -tau L / rho (so rho u' = -tau L): cross stress int N_a rho u' . grad u_i and Reynolds stress
        # - int rho (u' . grad N_a) u'_i (reading R17)
        Qm = Qm + _rbvms_terms(prob, w, gN, s["gradU"], tL)
    T = (rho * V[:, None, None, None] * np.einsum("ab,ebin->eain", MREF, U)
         - np.einsum("e,qa,eqin->eain", w, NQ, tL))
    Qc = (w[:, None, None] * div[:, None, :]
          + (1.0 / rho) * np.einsum("e,eai,eqin->ean", w, gN, tL))
    return s["t"], Qm, T, Qc


def _rbvms_terms(prob: HBProblem, w, gN, gradU, tL):
    """Cross- and Reynolds-stress terms of full RBVMS per element node (reading R17), with tL = tau L:
    - sum_q w [N_a(q) (tL_q . grad) u_i + (1 / rho) (tL_q . grad N_a) tL_q,i]."""
    cross = np.einsum("e,qa,eqjn,eijn->eain", w, NQ, tL, gradU)
    tdN = np.einsum("eqjn,eaj->eqan", tL, gN)
    reyn = np.einsum("e,eqan,eqin->eain", w, tdN, tL) / prob.rho
    return -(cross + reyn)


def _assemble(prob: HBProblem, t, Qm, T, Qc):
    """Element-to-node sums of Q^m, T and Q^c (the assembly behind Eq. Rmc; reading R4)."""
    n, N = prob.n_nodes, prob.N
    rm = np.zeros((n, 3, N))
    tm = np.zeros((n, 3, N))
    rc = np.zeros((n, N))
    for a in range(4):
        np.add.at(rm, t[:, a], Qm[:, a])
        np.add.at(tm, t[:, a], T[:, a])
        np.add.at(rc, t[:, a], Qc[:, a])
    return rm, tm, rc


# ---------------------------------------------------------------------------------------------------
# boundary terms (Eq. NS-time Neumann condition, Sec. 2.3 backflow, reading R5 / R8)

_MID = np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]])   # N at the 3 edge midpoints


def _outlet_h(prob: HBProblem, y: np.ndarray) -> np.ndarray:
    """Traction level h per face and instance [n_faces, N]: -P (reading R5) or -(P_d + R Q) (R8)."""
    N = prob.N
    h = np.zeros((prob.faces.shape[0], N))
    for tag, (a, b) in prob.outlet_p.items():
        h[prob.face_tag == tag] = -sample_waveform(a, b, N, prob.T)[None, :]
    for tag, (R, a, b) in prob.outlet_r.items():
        Q = outlet_flux(prob, y, tag)
        h[prob.face_tag == tag] = -(sample_waveform(a, b, N, prob.T) + R * Q)[None, :]
    return h


def outlet_flux(prob: HBProblem, y: np.ndarray, tag: int) -> np.ndarray:
    """Q_n = int_Gamma u_n . n for P1 velocity (exact: face area / 3 times the nodal sum); the flow rate
    of a resistance outlet (reading R8)."""
    f = np.nonzero(prob.face_tag == tag)[0]
    un = np.einsum("fbin,fi->fbn", y[prob.faces[f]][:, :, :3, :], prob.face_normal[f])
    return np.einsum("f,fbn->n", prob.face_area[f] / 3.0, un)


def boundary_residual(prob: HBProblem, y: np.ndarray) -> np.ndarray:
    """Momentum contributions of the Neumann faces [n_nodes, 3, N]: the traction term of Eq. (NS-weak)
    and the backflow stabilisation of Sec. 2.3 as printed (reading R5)."""
    out = np.zeros((prob.n_nodes, 3, prob.N))
    fn = prob.neumann_faces()
    if fn.size == 0:
        return out
    h = _outlet_h(prob, y)[fn]
    S = prob.face_area[fn]
    nrm = prob.face_normal[fn]
    nodes = prob.faces[fn]
    # - int N_A h n_i : h uniform on a face, int N_A = S / 3
    neu = -(S / 3.0)[:, None, None] * nrm[:, :, None] * h[:, None, :]          # [f, i, n]
    # backflow: - int N_A (rho/2) beta |u.n|_- u_i  (3-point edge-midpoint rule)
    uf = y[nodes][:, :, :3, :]                                                    # [f, b, i, n]
    um = np.einsum("mb,fbin->fmin", _MID, uf)
    s = np.einsum("fmin,fi->fmn", um, nrm)
    sm = 0.5 * (s - np.abs(s))
    bf = -(0.5 * prob.rho * prob.beta_bf) * np.einsum("f,mb,fmn,fmin->fbin", S / 3.0, _MID, sm, um)
    for b in range(3):
        np.add.at(out, nodes[:, b], neu + bf[:, b])
    return out


def residual(prob: HBProblem, y: np.ndarray) -> np.ndarray:
    """Assembled HB-GLS residual [n_nodes, 4, N] (Eq. Rmc); Dirichlet momentum rows are zero."""
    t, Qm, T, Qc = element_residual(prob, y)
    rm, tm, rc = _assemble(prob, t, Qm, T, Qc)
    rm = rm + _apply_H(prob, tm) + boundary_residual(prob, y)
    mask, _ = prob.dirichlet()
    rm[mask] = 0.0
    return np.concatenate([rm, rc[:, None, :]], axis=1)


# ---------------------------------------------------------------------------------------------------
# Jacobian-vector products


def _mask_v(prob: HBProblem, v: np.ndarray):
    """(mask, v with its prescribed velocity entries zeroed): they are not unknowns (Sec. 2.3)."""
    mask, _ = prob.dirichlet()
    vm = v.copy()
    vm[mask, :3] = 0.0
    return mask, vm


def jv_paper(prob: HBProblem, y: np.ndarray, v: np.ndarray, shift: float = 0.0) -> np.ndarray:
    """(P + C + shift M_vel) v with U and tau frozen at y (Eqs. ptangent, K_mat, ctangent, F_mat, R7).
    Dirichlet velocity rows are the identity on v."""
    mask, vm = _mask_v(prob, v)
    elems = np.arange(prob.tets.shape[0])
    s = _element_state(prob, y, elems)
    rho, mu = prob.rho, prob.mu
    V, gN, tau = s["V"], s["gN"], s["tau"]
    t = s["t"]
    dU = vm[t][:, :, :3, :]
    dP = vm[t][:, :, 3, :]
    gradV = np.einsum("eain,eaj->eijn", dU, gN)
    gradVp = np.einsum("ean,eaj->ejn", dP, gN)
    Uconv = s["Uq"] if prob.convection else np.zeros_like(s["Uq"])
    ugv = np.einsum("eqjn,eijn->eqin", Uconv, gradV)              # U_k dv_i/dx_k at q
    udN = np.einsum("eqjn,eaj->eqan", s["Uq_tau"], gN)           # U_k dN_a/dx_k at q
    w = V / 4.0
    Vb = V[:, None, None, None]
    # K block: Galerkin convection + viscosity + SUPG (rho tau) + pseudo-time mass
    Kv = (rho * np.einsum("e,qa,eqin->eain", w, NQ, ugv)
          + mu * Vb * np.einsum("eaj,eijn->eain", gN, gradV)
          + rho * np.einsum("e,eqn,eqan,eqin->eain", w, tau, udN, ugv)
          + shift * Vb * np.einsum("ab,ebin->eain", MREF, dU))
    # G block: - int dN_a/dx_i N_b + int U.grad N_a tau dN_b/dx_i
    Gv = (-Vb * gN[:, :, :, None] * dP.mean(axis=1)[:, None, None, :]
          + np.einsum("e,eqn,eqan,ein->eain", w, tau, udN, gradVp))
    # D block: int N_a dN_b/dx_j + int dN_a/dx_j tau U.grad N_b
    Dv = (w[:, None, None] * np.einsum("eiin->en", gradV)[:, None, :]
          + np.einsum("e,eqn,eaj,eqjn->ean", w, tau, gN, ugv))
    # L block: (1/rho) int tau grad N_a . grad N_b
    Lv = (1.0 / rho) * np.einsum("e,eqn,eaj,ejn->ean", w, tau, gN, gradVp)
    # F block: H (rho M v)
    Tv = rho * Vb * np.einsum("ab,ebin->eain", MREF, dU)
    rm, tm, rc = _assemble(prob, t, Kv + Gv, Tv, Dv + Lv)
    rm = rm + _apply_H(prob, tm) + boundary_jv(prob, y, vm, exact=False)
    rm[mask] = v[mask, :3]
    return np.concatenate([rm, rc[:, None, :]], axis=1)


def jv_exact(prob: HBProblem, y: np.ndarray, v: np.ndarray, shift: float = 0.0) -> np.ndarray:
    """Exact derivative of residual() (Eq. Rmc) along v (plus shift M_vel v); Dirichlet rows identity
    (reading R7: the Newton phase's Jacobian)."""
    mask, vm = _mask_v(prob, v)
    elems = np.arange(prob.tets.shape[0])
    s = _element_state(prob, y, elems)
    rho, mu = prob.rho, prob.mu
    V, gN, tau, G = s["V"], s["gN"], s["tau"], s["G"]
    t = s["t"]
    U = s["U"]
    dU = vm[t][:, :, :3, :]
    dP = vm[t][:, :, 3, :]
    Uq, Uq_tau = s["Uq"], s["Uq_tau"]
    conv_on = 1.0 if prob.convection else 0.0
    HU = _apply_H(prob, U)
    HUq = np.einsum("qa,eain->eqin", NQ, HU)
    dHUq = np.einsum("qa,eain->eqin", NQ, _apply_H(prob, dU))
    dUq = np.einsum("qa,eain->eqin", NQ, dU)
    dUq_tau = dUq * conv_on
    gradU = s["gradU"]
    gradV = np.einsum("eain,eaj->eijn", dU, gN)
    gradVp = np.einsum("ean,eaj->ejn", dP, gN)
    conv = conv_on * np.einsum("eqjn,eijn->eqin", Uq, gradU)
    dconv = conv_on * (np.einsum("eqjn,eijn->eqin", dUq, gradU) + np.einsum("eqjn,eijn->eqin", Uq, gradV))
    L = rho * HUq + rho * conv + s["gradP"][:, None, :, :]
    dL = rho * dHUq + rho * dconv + gradVp[:, None, :, :]
    duGu = 2.0 * np.einsum("eqin,eij,eqjn->eqn", Uq_tau, G, dUq_tau)
    dtau = -0.5 * tau ** 3 * duGu
    tL = tau[:, :, None, :] * L
    dtL = dtau[:, :, None, :] * L + tau[:, :, None, :] * dL
    udN = np.einsum("eqjn,eaj->eqan", Uq_tau, gN)
    dudN = np.einsum("eqjn,eaj->eqan", dUq_tau, gN)
    w = V / 4.0
    Vb = V[:, None, None, None]
    dQm = (rho * np.einsum("e,qa,eqin->eain", w, NQ, dconv)
           + np.einsum("e,eqan,eqin->eain", w, dudN, tL)
           + np.einsum("e,eqan,eqin->eain", w, udN, dtL)
           + mu * Vb * np.einsum("eaj,eijn->eain", gN, gradV)
           - Vb * gN[:, :, :, None] * dP.mean(axis=1)[:, None, None, :]
           + shift * Vb * np.einsum("ab,ebin->eain", MREF, dU))
    if prob.stab == "rbvms":
        # derivative of the cross- and Reynolds-stress terms (reading R17)
        tdN = np.einsum("eqjn,eaj->eqan", tL, gN)
        dtdN = np.einsum("eqjn,eaj->eqan", dtL, gN)
        dQm = dQm - (np.einsum("e,qa,eqjn,eijn->eain", w, NQ, dtL, gradU)
                     + np.einsum("e,qa,eqjn,eijn->eain", w, NQ, tL, gradV)
                     + (np.einsum("e,eqan,eqin->eain", w, dtdN, tL)
                        + np.einsum("e,eqan,eqin->eain", w, tdN, dtL)) / rho)
    dT = rho * Vb * np.einsum("ab,ebin->eain", MREF, dU) - np.einsum("e,qa,eqin->eain", w, NQ, dtL)
    dQc = (w[:, None, None] * np.einsum("eiin->en", gradV)[:, None, :]
           + (1.0 / rho) * np.einsum("e,eai,eqin->ean", w, gN, dtL))
    rm, tm, rc = _assemble(prob, t, dQm, dT, dQc)
    rm = rm + _apply_H(prob, tm) + boundary_jv(prob, y, vm, exact=True)
    rm[mask] = v[mask, :3]
    return np.concatenate([rm, rc[:, None, :]], axis=1)


def boundary_jv(prob: HBProblem, y: np.ndarray, v: np.ndarray, exact: bool) -> np.ndarray:
    """Derivative of boundary_residual along v.  exact=False freezes the backflow coefficient
    (reading R7); the resistance term is linear and identical in both."""
    out = np.zeros((prob.n_nodes, 3, prob.N))
    fn = prob.neumann_faces()
    if fn.size == 0:
        return out
    S = prob.face_area[fn]
    nrm = prob.face_normal[fn]
    nodes = prob.faces[fn]
    dh = np.zeros((prob.faces.shape[0], prob.N))
    for tag, (R, a, b) in prob.outlet_r.items():
        dh[prob.face_tag == tag] = -R * outlet_flux(prob, v, tag)[None, :]
    dh = dh[fn]
    neu = -(S / 3.0)[:, None, None] * nrm[:, :, None] * dh[:, None, :]
    uf = y[nodes][:, :, :3, :]
    vf = v[nodes][:, :, :3, :]
    um = np.einsum("mb,fbin->fmin", _MID, uf)
    vmid = np.einsum("mb,fbin->fmin", _MID, vf)
    s = np.einsum("fmin,fi->fmn", um, nrm)
    sm = 0.5 * (s - np.abs(s))
    term = sm[:, :, None, :] * vmid
    if exact:
        dsm = (s < 0).astype(np.float64) * np.einsum("fmin,fi->fmn", vmid, nrm)
        term = term + dsm[:, :, None, :] * um
    bf = -(0.5 * prob.rho * prob.beta_bf) * np.einsum("f,mb,fmin->fbin", S / 3.0, _MID, term)
    for b in range(3):
        np.add.at(out, nodes[:, b], neu + bf[:, b])
    return out


def jacobi_diag(prob: HBProblem, y: np.ndarray, shift: float = 0.0) -> np.ndarray:
    """Diagonal of P + shift M_vel (reading R9); 1 on Dirichlet velocity rows.  [n_nodes, 4, N]."""
    elems = np.arange(prob.tets.shape[0])
    s = _element_state(prob, y, elems)
    rho, mu = prob.rho, prob.mu
    V, gN, tau = s["V"], s["gN"], s["tau"]
    udN = np.einsum("eqjn,eaj->eqan", s["Uq_tau"], gN)
    udN_conv = udN if prob.convection else np.zeros_like(udN)
    w = V / 4.0
    g2 = np.einsum("eaj,eaj->ea", gN, gN)
    dv = (rho * np.einsum("e,qa,eqan->ean", w, NQ, udN_conv)
          + rho * np.einsum("e,eqn,eqan->ean", w, tau, udN ** 2)
          + (mu * V[:, None] * g2)[:, :, None]
          + (shift * V[:, None] * MREF[0, 0] * np.ones((1, 4)))[:, :, None])
    dp = (1.0 / rho) * np.einsum("e,eqn,ea->ean", w, tau, g2)
    t = s["t"]
    n, N = prob.n_nodes, prob.N
    d = np.zeros((n, 4, N))
    for a in range(4):
        np.add.at(d[:, 0], t[:, a], dv[:, a])
        np.add.at(d[:, 3], t[:, a], dp[:, a])
    d[:, 1] = d[:, 0]
    d[:, 2] = d[:, 0]
    mask, _ = prob.dirichlet()
    d[mask, :3] = 1.0
    return d


# ---------------------------------------------------------------------------------------------------
# Newton-Krylov solve (Eq. NR, Sec. 2.3)


def gmres(matvec, b: np.ndarray, precond_inv, tol: float, restart: int = 50, maxiter: int = 2000,
          x0=None):
    """Right-preconditioned restarted GMRES (Saad & Schultz; the linear solver of every Newton step,
    Sec. 2.3) with modified Gram-Schmidt and Givens rotations, all FP64.  Solves A x = b to ||b - A x|| <= tol ||b||.  Returns (x, iterations)."""
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0
    it = 0
    while it < maxiter:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            break
        Vk = np.zeros((restart + 1, n))
        Hh = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        Vk[0] = r / beta
        k_used = 0
        for k in range(restart):
            wv = matvec(precond_inv(Vk[k]))
            for j in range(k + 1):
                Hh[j, k] = np.dot(Vk[j], wv)
                wv = wv - Hh[j, k] * Vk[j]
            Hh[k + 1, k] = np.linalg.norm(wv)
            if Hh[k + 1, k] > 0:
                Vk[k + 1] = wv / Hh[k + 1, k]
            for j in range(k):
                tmp = cs[j] * Hh[j, k] + sn[j] * Hh[j + 1, k]
                Hh[j + 1, k] = -sn[j] * Hh[j, k] + cs[j] * Hh[j + 1, k]
                Hh[j, k] = tmp
            den = math.hypot(Hh[k, k], Hh[k + 1, k])
            cs[k] = Hh[k, k] / den
            sn[k] = Hh[k + 1, k] / den
            Hh[k, k] = den
            Hh[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            k_used = k + 1
            if abs(g[k + 1]) <= tol * bnorm or it >= maxiter:
                break
        yk = np.linalg.solve(np.triu(Hh[:k_used, :k_used]), g[:k_used])
        x = x + precond_inv(Vk[:k_used].T @ yk)
        if abs(g[k_used]) <= tol * bnorm:
            break
    return x, it


def pseudo_dt(prob: HBProblem) -> float:
    """CFL rule of Sec. 2.3: dt ~ h_c / u_c with h_c the edge of the regular tetrahedron of mean
    element volume and u_c the largest mean inlet velocity over the instances."""
    hc = (6.0 * math.sqrt(2.0) * prob.geo.V.mean()) ** (1.0 / 3.0)
    _, g = prob.dirichlet()
    uc = 0.0
    for tag in prob.inflow:
        f = np.nonzero(prob.face_tag == tag)[0]
        A = prob.face_area[f].sum()
        un = np.abs(np.einsum("fbin,fi->fbn", g[prob.faces[f]], prob.face_normal[f]))
        flux = np.einsum("f,fbn->n", prob.face_area[f] / 3.0, un)
        uc = max(uc, float(flux.max() / A))
    return hc / uc if uc > 0 else math.inf


def solve(prob: HBProblem, y0=None, dt=None, switch_tol: float = 1e-3, rtol: float = 1e-12,
          gmres_tol: float = 1e-4, restart: int = 50, max_steps: int = 200, verbose: bool = False):
    """Pseudo-transient Newton (reading R6): paper tangent + c1 rho/dt mass until ||r||/||r0|| <
    switch_tol, then Newton with the exact Jacobian until the update and residual both fall below rtol.
    Returns (y, history)."""
    y = prob.initial_state() if y0 is None else prob.apply_dirichlet(y0)
    if dt is None:
        dt = pseudo_dt(prob)
    shift = C1_PSEUDO * prob.rho / dt if math.isfinite(dt) else 0.0
    r = residual(prob, y)
    r0 = np.linalg.norm(r)
    hist = [r0]
    newton = False
    shp = y.shape
    for step in range(max_steps):
        rn = np.linalg.norm(r)
        if r0 == 0.0 or rn / r0 < switch_tol:
            newton = True
        sh = 0.0 if newton else shift
        if newton:
            mv = lambda x: jv_exact(prob, y, x.reshape(shp)).ravel()  # noqa: E731
        else:
            mv = lambda x: jv_paper(prob, y, x.reshape(shp), shift=sh).ravel()  # noqa: E731
        d = jacobi_diag(prob, y, shift=sh).ravel()
        tol = gmres_tol if newton else 0.03
        dx, its = gmres(mv, -r.ravel(), lambda z: z / d, tol, restart=restart)
        y = y + dx.reshape(shp)
        r = residual(prob, y)
        hist.append(np.linalg.norm(r))
        if verbose:
            print(f"step {step} newton={newton} gmres={its} |r|/|r0|={hist[-1] / r0:.3e}")
        if newton and np.linalg.norm(dx) <= rtol * np.linalg.norm(y) and hist[-1] <= rtol * r0 * 10:
            break
        if newton and hist[-1] <= 1e-14 * r0:
            break
    return y, hist
