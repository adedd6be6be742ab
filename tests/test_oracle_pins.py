"""Pins of the CPU oracle against facts the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed forms, an exact patch
solution, an identity of the discrete equations, finite differences, independently written element
matrices, a per-mode complex Stokes solve, or invariances of the continuous problem.
"""
import math

import numpy as np
import pytest

from oracle import hb_oracle as O
from paper_2411_14315_gb300 import inputs as I


def _signed_freq(N):
    j = np.arange(N)
    return np.where(j <= N // 2, j, j - N)


# --------------------------------------------------------------------------------------------------
# H and the DFT (Sec. 2.1)


@pytest.mark.parametrize("n_h", [0, 1, 2, 4, 10, 12])
def test_H_differentiates_trig_polynomials_exactly(n_h):
    N = 2 * n_h + 1
    T = 0.8
    w = 2 * math.pi / T
    H = O.spectral_H(N, w)
    t = O.instance_times(N, T)
    for k in range(0, n_h + 1):
        c, s = np.cos(k * w * t), np.sin(k * w * t)
        assert np.allclose(H @ c, -k * w * s, atol=1e-12 * max(1, k * w))
        assert np.allclose(H @ s, k * w * c, atol=1e-12 * max(1, k * w))


@pytest.mark.parametrize("N", [1, 3, 9, 21, 25])
def test_H_skew_zero_diagonal_imaginary_spectrum(N):
    w = 1.7
    H = O.spectral_H(N, w)
    assert np.all(np.diag(H) == 0)
    assert np.allclose(H, -H.T, atol=0)
    ev = np.sort(np.linalg.eigvals(H).imag)
    assert np.allclose(ev, w * np.arange(-(N // 2), N // 2 + 1), atol=1e-11)
    assert np.allclose(np.linalg.eigvals(H).real, 0, atol=1e-11)


@pytest.mark.parametrize("N", [3, 5, 13, 21])
def test_H_is_Einv_Omega_E(N):
    """Paper's definition H = E^-1 Omega E with Omega = diag(i m w), m the signed frequency of each DFT
    row (reading R1), built from the DFT matrix of Eq. (upghdft)."""
    w = 2.3
    E = O.dft_E(N)
    Om = np.diag(1j * w * _signed_freq(N))
    H2 = np.linalg.inv(E) @ Om @ E
    assert np.allclose(H2.imag, 0, atol=1e-12)
    assert np.allclose(O.spectral_H(N, w), H2.real, atol=1e-12)


def test_dft_round_trip_and_real_coefficients():
    rng = np.random.default_rng(3)
    n_h, T = 5, 1.3
    N = 2 * n_h + 1
    E = O.dft_E(N)
    assert np.allclose(np.linalg.inv(E) @ E, np.eye(N), atol=1e-13)
    # E^-1 = N^-1 ... conjugate: (E^-1)[j,k] = exp(+2 pi i j k / N)
    j = np.arange(N)
    assert np.allclose(np.linalg.inv(E), np.exp(2j * np.pi * np.outer(j, j) / N), atol=1e-12)
    coef = rng.normal(size=(7, 2 * n_h + 1))
    y = O.harmonics_to_instances(coef, N, T)
    assert np.allclose(O.instances_to_harmonics(y, n_h), coef, atol=1e-13)
    # a0 + a1 cos + b1 sin sampled directly
    t = O.instance_times(N, T)
    w = 2 * math.pi / T
    direct = coef[:, 0:1] + coef[:, 1:2] * np.cos(w * t) + coef[:, 2:3] * np.sin(w * t)
    for k in range(2, n_h + 1):
        direct = direct + coef[:, 2 * k - 1:2 * k] * np.cos(k * w * t) + coef[:, 2 * k:2 * k + 1] * np.sin(k * w * t)
    assert np.allclose(y, direct, atol=1e-13)


# --------------------------------------------------------------------------------------------------
# geometry and tau (Sec. 2.2, Eq. tau; reading R3)


def test_reference_tet_geometry_and_tau():
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    tets = np.array([[0, 1, 2, 3]])
    g = O.Geometry(xyz, tets)
    assert np.isclose(g.V[0], 1 / 6)
    assert np.allclose(g.gradN[0], [[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    assert np.allclose(g.G[0], np.eye(3)) and np.isclose(g.GG[0], 3.0)
    s = 0.25
    g2 = O.Geometry(xyz * s, tets)
    assert np.isclose(g2.V[0], s ** 3 / 6)
    assert np.allclose(g2.G[0], np.eye(3) / s ** 2)
    # tau at a quadrature point where u_q = (1, 0, 0): (1 + C_I nu^2 * 3)^-1/2 on the reference tet
    faces = I.boundary_faces(tets, 4).astype(np.int32)
    nu = 0.2
    pr = O.HBProblem(xyz, tets, faces, np.ones(4, dtype=np.int32), 1.0, nu, 1.0, 0)
    y = np.zeros((4, 4, 1))
    y[:, 0, 0] = 1.0
    st = O._element_state(pr, y, np.array([0]))
    assert np.allclose(st["tau"], (1.0 + 3.0 * nu * nu * 3.0) ** -0.5)


def test_shape_gradients_reproduce_linear_fields():
    m = I.box_mesh(2, 2, 2, jitter=0.25, seed=4)
    g = O.Geometry(m.xyz, m.tets.astype(np.int64))
    x = m.xyz[m.tets]
    assert np.allclose(g.gradN.sum(axis=1), 0, atol=1e-12)
    assert np.allclose(np.einsum("eai,eaj->eij", x, g.gradN), np.eye(3), atol=1e-12)
    vol = np.abs(np.linalg.det(np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], 2))) / 6
    assert np.isclose(vol.sum(), 1.0)


# --------------------------------------------------------------------------------------------------
# problem builders


def _plug_problem(n_h, T=2.0, rho=1.3, mu=0.05, seed=1, n=(4, 3, 3)):
    """Plug flow u = a(t) e_x, p = -rho a'(t) x in [0,2]x[0,1]^2: an exact solution of the HB-GLS
    equations for P1 (L = 0, grad u = 0), with Dirichlet data on all faces but the x = 2 outlet."""
    m = I.box_mesh(*n, lx=2.0, ly=1.0, lz=1.0, jitter=0.2, seed=seed)
    a = np.zeros(n_h + 1)
    b = np.zeros(n_h + 1)
    a[0] = 1.0
    rng = np.random.default_rng(seed)
    for k in range(1, n_h + 1):
        a[k], b[k] = rng.uniform(-0.15, 0.15, 2) / k
    pr = O.HBProblem(m.xyz, m.tets, m.faces, m.face_tag, rho, mu, T, n_h)
    prof = I.uniform_profile(m, [1, 3, 4, 5, 6], [1, 0, 0])
    for tag in [1, 3, 4, 5, 6]:
        pr.set_inflow(tag, prof, a, b)
    w = 2 * math.pi / T
    k = np.arange(n_h + 1)
    pr.set_outlet_pressure(2, -rho * 2.0 * k * w * b, rho * 2.0 * k * w * a)
    N = 2 * n_h + 1
    t = O.instance_times(N, T)
    at = np.full(N, a[0])
    adot = np.zeros(N)
    for j in range(1, n_h + 1):
        at += a[j] * np.cos(j * w * t) + b[j] * np.sin(j * w * t)
        adot += j * w * (-a[j] * np.sin(j * w * t) + b[j] * np.cos(j * w * t))
    y = np.zeros((m.n_nodes, 4, N))
    y[:, 0] = at[None, :]
    y[:, 3] = -rho * np.asarray(adot)[None, :] * m.xyz[:, :1]
    return m, pr, y


def _random_problem(seed=11, n_h=2, resistance=True, beta=0.2, n=(3, 2, 2)):
    """Box with an inlet (x-min, uniform profile), walls (y faces), a pressure outlet (x-max) and a
    resistance or traction-free outlet (z faces)."""
    m = I.box_mesh(*n, lx=1.5, jitter=0.2, seed=seed)
    tag = m.face_tag.copy()
    tag[(tag == 3) | (tag == 4)] = 0
    pr = O.HBProblem(m.xyz, m.tets, m.faces, tag, 1.1, 0.07, 1.7, n_h, beta_bf=beta)
    a, b = I.waveform_harmonics(n_h, 1.0, seed)
    pr.set_inflow(1, I.uniform_profile(m, [1], [1.0, 0.2, 0.0]), a, b)
    pa, pb = I.waveform_harmonics(n_h, 0.5, seed + 1)
    pr.set_outlet_pressure(2, pa, pb)
    if resistance:
        pr.set_outlet_resistance(5, 0.8, pa * 0.3, pb * 0.3)
    return m, pr


# --------------------------------------------------------------------------------------------------
# exact solutions and identities of the discrete equations


@pytest.mark.parametrize("n_h", [0, 1, 3])
def test_plug_flow_patch_residual_is_zero(n_h):
    m, pr, y = _plug_problem(n_h)
    r = O.residual(pr, y)
    scale = pr.rho * np.abs(y[:, :3]).max() * pr.geo.V.max() * (1 + pr.omega * n_h)
    assert np.abs(r).max() < 1e-13 * max(scale, 1.0) + 1e-14
    mask, g = pr.dirichlet()
    assert np.allclose(y[mask, :3], g[mask])


def test_plug_flow_patch_fails_on_wrong_outlet_sign():
    """The patch test is sensitive to the reading h = -P: flipping it leaves a residual."""
    m, pr, y = _plug_problem(2)
    for tag, (a, b) in list(pr.outlet_p.items()):
        pr.set_outlet_pressure(tag, -a, -b)
    assert np.abs(O.residual(pr, y)).max() > 1e-3


def test_continuity_rows_sum_to_boundary_flux():
    """sum_A r^c_A = int div u = flux of u through the boundary, at any state (sum_A grad N_A = 0
    removes the least-squares part)."""
    m, pr = _random_problem()
    y = I.random_state(m.n_nodes, pr.N, 5)
    r = O.residual(pr, y)
    un = np.einsum("fbin,fi->fbn", y[pr.faces][:, :, :3, :], pr.face_normal)
    flux = np.einsum("f,fbn->n", pr.face_area / 3, un)
    assert np.allclose(r[:, 3].sum(axis=0), flux, atol=1e-13)


def test_exact_jv_matches_central_differences():
    m, pr = _random_problem(seed=12)
    N = pr.N
    y = pr.apply_dirichlet(I.random_state(m.n_nodes, N, 7))
    v = I.random_state(m.n_nodes, N, 8)
    mask, _ = pr.dirichlet()
    v[mask, :3] = 0
    eps = 1e-6
    fd = (O.residual(pr, y + eps * v) - O.residual(pr, y - eps * v)) / (2 * eps)
    je = O.jv_exact(pr, y, v)
    assert np.linalg.norm(fd - je) / np.linalg.norm(je) < 1e-8
    # the shift adds the consistent mass on velocity rows only
    js = O.jv_exact(pr, y, v, shift=2.5)
    diff = js - je
    assert np.allclose(diff[:, 3], 0)


def test_time_instance_only_state_reduces_to_steady():
    """A state constant in time has H y = 0, so every instance's residual equals the N = 1 (steady GLS)
    residual of that state (the paper's own N = 1 case)."""
    m, pr3 = _random_problem(seed=13, n_h=1, resistance=False)
    pr1 = O.HBProblem(m.xyz, m.tets, m.faces, pr3.face_tag, pr3.rho, pr3.mu, pr3.T, 0)
    for tag, (prof, a, b) in pr3.inflow.items():
        pr1.set_inflow(tag, prof, a[:1], b[:1])
        pr3.set_inflow(tag, prof, a[:1] * np.r_[1, 0], b[:1] * np.r_[1, 0])
    for tag, (a, b) in pr3.outlet_p.items():
        pr1.set_outlet_pressure(tag, a[:1], b[:1])
        pr3.set_outlet_pressure(tag, np.r_[a[0], 0], np.r_[0, 0])
    y1 = I.random_state(m.n_nodes, 1, 9)
    y3 = np.repeat(y1, 3, axis=2)
    r1 = O.residual(pr1, y1)
    r3 = O.residual(pr3, y3)
    for n in range(3):
        assert np.allclose(r3[:, :, n], r1[:, :, 0], atol=1e-13)


# --------------------------------------------------------------------------------------------------
# invariances of the continuous problem


def test_time_shift_equivariance():
    """Shifting every boundary waveform by one instance rotates the residual by one instance."""
    m, pr = _random_problem(seed=14, n_h=3)
    N, T = pr.N, pr.T
    y = I.random_state(m.n_nodes, N, 10)
    r = O.residual(pr, y)
    d = T / N
    w = 2 * math.pi / T

    def shift(a, b):
        k = np.arange(len(a))
        return a * np.cos(k * w * d) + b * np.sin(k * w * d), b * np.cos(k * w * d) - a * np.sin(k * w * d)

    pr2 = O.HBProblem(m.xyz, m.tets, m.faces, pr.face_tag, pr.rho, pr.mu, T, pr.n_h)
    for tag, (prof, a, b) in pr.inflow.items():
        pr2.set_inflow(tag, prof, *shift(a, b))
    for tag, (a, b) in pr.outlet_p.items():
        pr2.set_outlet_pressure(tag, *shift(a, b))
    for tag, (R, a, b) in pr.outlet_r.items():
        pr2.set_outlet_resistance(tag, R, *shift(a, b))
    y2 = np.roll(y, -1, axis=2)      # y2(t_n) = y(t_n + d)
    r2 = O.residual(pr2, y2)
    assert np.allclose(r2, np.roll(r, -1, axis=2), atol=1e-12)


def test_rigid_motion_invariance():
    m, pr = _random_problem(seed=15)
    N = pr.N
    y = I.random_state(m.n_nodes, N, 11)
    r = O.residual(pr, y)
    Q, _ = np.linalg.qr(np.random.default_rng(1).normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    xyz2 = m.xyz @ Q.T + np.array([0.3, -1.2, 2.0])
    pr2 = O.HBProblem(xyz2, m.tets, m.faces, pr.face_tag, pr.rho, pr.mu, pr.T, pr.n_h)
    for tag, (prof, a, b) in pr.inflow.items():
        pr2.set_inflow(tag, prof @ Q.T, a, b)
    for tag, (a, b) in pr.outlet_p.items():
        pr2.set_outlet_pressure(tag, a, b)
    for tag, (R, a, b) in pr.outlet_r.items():
        pr2.set_outlet_resistance(tag, R, a, b)
    y2 = y.copy()
    y2[:, :3] = np.einsum("ij,njt->nit", Q, y[:, :3])
    r2 = O.residual(pr2, y2)
    r_rot = r.copy()
    r_rot[:, :3] = np.einsum("ij,njt->nit", Q, r[:, :3])
    assert np.allclose(r2, r_rot, atol=1e-12)


def test_node_renumbering_invariance():
    m, pr = _random_problem(seed=16)
    N = pr.N
    y = I.random_state(m.n_nodes, N, 12)
    r = O.residual(pr, y)
    perm = np.random.default_rng(2).permutation(m.n_nodes)   # new id of old node i is inv[i]
    inv = np.argsort(perm)
    xyz2 = m.xyz[perm]
    tets2 = inv[m.tets]
    faces2 = inv[m.faces]
    pr2 = O.HBProblem(xyz2, tets2, faces2, pr.face_tag, pr.rho, pr.mu, pr.T, pr.n_h)
    for tag, (prof, a, b) in pr.inflow.items():
        pr2.set_inflow(tag, prof[perm], a, b)
    for tag, (a, b) in pr.outlet_p.items():
        pr2.set_outlet_pressure(tag, a, b)
    for tag, (R, a, b) in pr.outlet_r.items():
        pr2.set_outlet_resistance(tag, R, a, b)
    r2 = O.residual(pr2, y[perm])
    assert np.allclose(r2, r[perm], atol=1e-12)


# --------------------------------------------------------------------------------------------------
# the paper's tangent against element matrices written out from Eq. (K_mat) and Eq. (F_mat)


def _dense_paper_tangent(pr, y, shift):
    """Dense L~ = P + C + shift M (volume terms only) from per-element matrices, with plain loops."""
    n, N = pr.n_nodes, pr.N
    nd = n * 4 * N
    Jd = np.zeros((nd, nd))
    idx = lambda A, f, t: (A * 4 + f) * N + t  # noqa: E731
    qa, qb = O.QA, O.QB
    NQ = [[qa if a == q else qb for a in range(4)] for q in range(4)]
    H = pr.H
    for e, tet in enumerate(pr.tets):
        x = pr.xyz[tet]
        J = np.column_stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]])
        Ji = np.linalg.inv(J)
        V = abs(np.linalg.det(J)) / 6
        gN = np.vstack([-Ji.sum(0), Ji])
        G = Ji.T @ Ji
        g2 = 3.0 * pr.nu ** 2 * np.sum(G * G)
        for t in range(N):
            uq = [sum(NQ[q][a] * y[tet[a], :3, t] for a in range(4)) for q in range(4)]
            tau = [1 / math.sqrt(uq[q] @ G @ uq[q] + g2) for q in range(4)]
            for a in range(4):
                for b in range(4):
                    Mab = V * (2.0 if a == b else 1.0) / 20
                    K = mu_term = pr.mu * V * (gN[a] @ gN[b])
                    del mu_term
                    K += shift * Mab
                    for q in range(4):
                        w = V / 4
                        K += w * pr.rho * NQ[q][a] * (uq[q] @ gN[b])
                        K += w * pr.rho * tau[q] * (uq[q] @ gN[a]) * (uq[q] @ gN[b])
                    Lab = sum(V / 4 * tau[q] * (gN[a] @ gN[b]) for q in range(4)) / pr.rho
                    A, B = tet[a], tet[b]
                    for i in range(3):
                        Jd[idx(A, i, t), idx(B, i, t)] += K
                        Gi = -V / 4 * gN[a][i] + sum(V / 4 * tau[q] * (uq[q] @ gN[a]) * gN[b][i] for q in range(4))
                        Jd[idx(A, i, t), idx(B, 3, t)] += Gi
                        Di = V / 4 * gN[b][i] + sum(V / 4 * tau[q] * gN[a][i] * (uq[q] @ gN[b]) for q in range(4))
                        Jd[idx(A, 3, t), idx(B, i, t)] += Di
                        for s in range(N):      # F = H int rho N_A N_B
                            Jd[idx(A, i, t), idx(B, i, s)] += H[t, s] * pr.rho * Mab
                    Jd[idx(A, 3, t), idx(B, 3, t)] += Lab
    return Jd


def test_paper_tangent_matches_element_matrices_of_Kmat():
    m = I.box_mesh(2, 1, 1, jitter=0.2, seed=17)
    tag = m.face_tag.copy()
    pr = O.HBProblem(m.xyz, m.tets, m.faces, tag, 1.2, 0.09, 1.1, 1, beta_bf=0.0)
    a, b = I.waveform_harmonics(1, 1.0, 3)
    pr.set_inflow(1, I.uniform_profile(m, [1], [1.0, 0.0, 0.0]), a, b)   # only x-min is Dirichlet
    N = pr.N
    y = I.random_state(m.n_nodes, N, 13)
    v = I.random_state(m.n_nodes, N, 14)
    mask, _ = pr.dirichlet()
    v[mask, :3] = 0
    shift = 0.7
    Jd = _dense_paper_tangent(pr, y, shift)
    jv = Jd @ v.ravel()
    jv = jv.reshape(v.shape)
    jv[mask, :3] = 0
    ref = O.jv_paper(pr, y, v, shift=shift)
    ref[mask, :3] = 0
    assert np.linalg.norm(ref - jv) / np.linalg.norm(jv) < 1e-13
    # Jacobi diagonal is the diagonal of the same matrix (no backflow here)
    d = O.jacobi_diag(pr, y, shift=shift)
    dd = np.diag(Jd).reshape(v.shape)
    free = ~mask
    assert np.allclose(d[free], dd[free], rtol=1e-13, atol=1e-15)
    assert np.allclose(d[~free, 3], dd[~free, 3], rtol=1e-13)


def test_exact_minus_paper_tangent_is_dropped_H_terms_without_convection():
    """With convection off, the exact Jacobian differs from the paper's tangent only by the
    least-squares H terms that Eq. (ctangent) drops: -H int N_A tau (rho H v + grad v_p) in the momentum
    rows and (1/rho) int grad N_A tau rho (H v) in the continuity rows."""
    m, pr = _random_problem(seed=18, resistance=False, beta=0.0)
    pr.convection = False
    N = pr.N
    y = I.random_state(m.n_nodes, N, 15)
    v = I.random_state(m.n_nodes, N, 16)
    mask, _ = pr.dirichlet()
    v[mask, :3] = 0
    d = O.jv_exact(pr, y, v) - O.jv_paper(pr, y, v)
    exp = np.zeros_like(d)
    Hv = v[:, :3] @ pr.H.T
    g = pr.geo
    tm = np.zeros((m.n_nodes, 3, N))
    for e, tet in enumerate(pr.tets):
        tau = 1.0 / math.sqrt(3.0 * pr.nu ** 2 * g.GG[e])
        gp = sum(np.outer(g.gradN[e, b], v[tet[b], 3]) for b in range(4))      # grad v_p [i, n]
        for a in range(4):
            for q in range(4):
                Nqa = O.QA if a == q else O.QB
                hq = sum((O.QA if b == q else O.QB) * Hv[tet[b]] for b in range(4))
                tm[tet[a]] -= g.V[e] / 4 * Nqa * tau * (pr.rho * hq + gp)
                exp[tet[a], 3] += g.V[e] / 4 * tau * np.einsum("i,in->n", g.gradN[e, a], hq)
    exp[:, :3] = tm @ pr.H.T
    exp[mask, :3] = 0
    assert np.linalg.norm(d - exp) / np.linalg.norm(exp) < 1e-12


# --------------------------------------------------------------------------------------------------
# Stokes limit: HB decouples into one complex system per Fourier mode


def test_stokes_modes_solve_hb_equations():
    """Without convection (U -> 0 in the residual and in tau) and without backflow, the HB equations are
    linear and time-invariant, so their solution is the per-mode solution of the frequency-domain
    equations (Eq. NS-spec with A -> 0), assembled here by hand and solved directly.  The real instance
    values built from those modes must zero the oracle's HB residual."""
    m = I.box_mesh(2, 2, 2, lx=1.5, jitter=0.15, seed=21)
    tag = m.face_tag.copy()
    tag[(tag == 3) | (tag == 4) | (tag == 5) | (tag == 6)] = 0
    n_h, rho, mu, T = 3, 1.05, 0.3, 0.9
    pr = O.HBProblem(m.xyz, m.tets, m.faces, tag, rho, mu, T, n_h, beta_bf=0.0, convection=False)
    ga, gb = I.waveform_harmonics(n_h, 1.0, 5)
    prof = I.uniform_profile(m, [1], [1.0, 0.0, 0.0])
    pr.set_inflow(1, prof, ga, gb)
    pa, pb = I.waveform_harmonics(n_h, 2.0, 6)
    pr.set_outlet_pressure(2, pa, pb)
    N = pr.N
    w = 2 * math.pi / T
    mask, _ = pr.dirichlet()
    n = m.n_nodes
    # per-mode complex data: q(t) = sum_m q_m e^{i m w t}
    gm = [ga[0] + 0j] + [(ga[k] - 1j * gb[k]) / 2 for k in range(1, n_h + 1)]
    pm = [pa[0] + 0j] + [(pa[k] - 1j * pb[k]) / 2 for k in range(1, n_h + 1)]
    out_faces = np.nonzero(tag == 2)[0]
    sol = []
    for k in range(n_h + 1):
        om = k * w
        K = np.zeros((4 * n, 4 * n), dtype=complex)
        f = np.zeros(4 * n, dtype=complex)
        for tet in pr.tets:
            x = pr.xyz[tet]
            J = np.column_stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]])
            Ji = np.linalg.inv(J)
            V = abs(np.linalg.det(J)) / 6
            gN = np.vstack([-Ji.sum(0), Ji])
            G = Ji.T @ Ji
            tau = 1 / math.sqrt(3.0 * pr.nu ** 2 * np.sum(G * G))
            for a in range(4):
                for b in range(4):
                    A, B = tet[a], tet[b]
                    Mab = V * (2.0 if a == b else 1.0) / 20
                    Sab = V * gN[a] @ gN[b]
                    for i in range(3):
                        # rho i w M + mu S + (-i w) tau rho (i w) M
                        K[4 * A + i, 4 * B + i] += (1j * om * rho + tau * rho * om * om) * Mab + mu * Sab
                        # -int d_i N_a N_b  + (-i w) tau int N_a d_i N_b
                        K[4 * A + i, 4 * B + 3] += -V / 4 * gN[a][i] - 1j * om * tau * V / 4 * gN[b][i]
                        # int N_a d_i N_b + (1/rho) tau int d_i N_a rho (i w) N_b
                        K[4 * A + 3, 4 * B + i] += V / 4 * gN[b][i] + 1j * om * tau * V / 4 * gN[a][i]
                    K[4 * A + 3, 4 * B + 3] += tau / rho * Sab
        for fi in out_faces:
            S = pr.face_area[fi]
            for A in pr.faces[fi]:
                for i in range(3):
                    f[4 * A + i] += S / 3 * (-pm[k]) * pr.face_normal[fi][i]    # int N_A h n_i, h = -P
        ud = np.zeros(4 * n, dtype=complex)
        for A in np.nonzero(mask)[0]:
            ud[4 * A:4 * A + 3] = prof[A] * gm[k]
        free = np.ones(4 * n, dtype=bool)
        for A in np.nonzero(mask)[0]:
            free[4 * A:4 * A + 3] = False
        rhs = f - K @ ud
        xk = ud.copy()
        xk[free] = np.linalg.solve(K[np.ix_(free, free)], rhs[free])
        sol.append(xk.reshape(n, 4))
    t = O.instance_times(N, T)
    y = np.zeros((n, 4, N))
    y += sol[0].real[:, :, None]
    for k in range(1, n_h + 1):
        y += 2 * (sol[k][:, :, None] * np.exp(1j * k * w * t)[None, None, :]).real
    r = O.residual(pr, y)
    scale = np.abs(O.residual(pr, np.zeros_like(y))).max()
    assert np.abs(r).max() < 1e-11 * scale


def test_pseudo_step_rule_on_a_regular_tetrahedron():
    """Sec. 2.3's CFL rule dt = h_c / u_c: on one regular tetrahedron of edge 2 sqrt(2) the edge of the
    regular tetrahedron of mean volume is that edge, and a uniform inflow U q(t) normal to the inlet face
    has the largest mean inlet speed U max_n |q(t_n)|."""
    xyz = np.array([[1.0, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]])
    tets = np.array([[0, 1, 2, 3]])
    faces = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    tags = np.array([1, 2, 2, 2])                  # inlet opposite vertex 0; the rest traction-free
    T, n_h, U = 0.8, 2, 1.7
    pr = O.HBProblem(xyz, tets, faces, tags, 1.0, 0.1, T, n_h)
    inward = xyz[0] - xyz[1:].mean(0)              # from the inlet face towards vertex 0
    inward /= np.linalg.norm(inward)
    profile = np.zeros((4, 3))
    profile[1:] = U * inward
    a, b = np.array([1.0, 0.6, -0.3]), np.array([0.0, 0.4, 0.2])
    pr.set_inflow(1, profile, a, b)
    t = T * np.arange(pr.N) / pr.N
    w = 2 * math.pi / T
    q = a[0] + sum(a[k] * np.cos(k * w * t) + b[k] * np.sin(k * w * t) for k in (1, 2))
    assert abs(O.pseudo_dt(pr) - 2 * math.sqrt(2) / (U * np.abs(q).max())) < 1e-12
