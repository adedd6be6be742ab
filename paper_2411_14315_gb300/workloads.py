"""Seeded workloads: one mesh plus fluid constants and boundary waveforms, as plain input data.

These are the synthetic stand-ins for the paper's three patient cases (Sec. 3; their geometries and
waveforms come from an external repository and are not available here).  A spec carries inputs only:
the library and the CPU oracle each turn it into their own boundary data.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from paper_2411_14315_gb300 import inputs as I


@dataclasses.dataclass
class Spec:
    mesh: I.Mesh
    rho: float
    mu: float
    T: float
    n_h: int
    beta: float = 0.2
    inflows: list = dataclasses.field(default_factory=list)      # (tag, profile or None, a, b)
    outlets_p: list = dataclasses.field(default_factory=list)    # (tag, a, b)
    outlets_r: list = dataclasses.field(default_factory=list)    # (tag, R, a, b)
    tags: np.ndarray | None = None                               # face tags override
    name: str = ""
    inflows_harm: list = dataclasses.field(default_factory=list)  # (tag, per-node harmonics [n, 3, M])

    @property
    def N(self):
        return 2 * self.n_h + 1

    @property
    def face_tag(self):
        return self.mesh.face_tag if self.tags is None else self.tags


def dirichlet_nodes(spec: Spec) -> np.ndarray:
    m = spec.mesh
    dtags = [0] + [t for t, *_ in spec.inflows]
    return np.unique(m.faces[np.isin(spec.face_tag, dtags)].ravel())




def box_spec(seed=11, n_h=2, n=(6, 4, 4), resistance=True, beta=0.2, jitter=0.2) -> Spec:
    """Box with an inlet (x-min, uniform profile), no-slip walls (y faces), a pressure outlet (x-max)
    and a resistance outlet (z faces)."""
    m = I.box_mesh(*n, lx=1.5, jitter=jitter, seed=seed)
    tag = m.face_tag.copy()
    tag[(tag == 3) | (tag == 4)] = 0
    a, b = I.waveform_harmonics(n_h, 1.0, seed)
    pa, pb = I.waveform_harmonics(n_h, 0.5, seed + 1)
    s = Spec(m, 1.1, 0.07, 1.7, n_h, beta=beta, tags=tag)
    s.inflows.append((1, I.uniform_profile(m, [1], [1.0, 0.2, 0.0]), a, b))
    s.outlets_p.append((2, pa, pb))
    if resistance:
        s.outlets_r.append((5, 0.8, pa * 0.3, pb * 0.3))
    return s


def channel_spec(n=(4, 3, 3), n_h: int = 2, mu: float = 0.3, seed: int = 90) -> Spec:
    """Jittered box channel: uniform inflow on x-min with harmonics 0.3/k (cos) and 0.2/k (sin) on a unit
    mean, a pressure outlet on x-max (mean 0.3, first harmonic 0.1 cos / -0.05 sin), no-slip on the other
    four faces; rho = 1.1, T = 1.7.  Small and well conditioned: the oracle's solve converges in seconds."""
    m = I.box_mesh(*n, lx=1.5, jitter=0.2, seed=seed)
    tag = m.face_tag.copy()
    tag[tag >= 3] = 0
    k = np.arange(1, n_h + 1)
    a = np.zeros(n_h + 1)
    b = np.zeros(n_h + 1)
    a[0] = 1.0
    a[1:] = 0.3 / k
    b[1:] = 0.2 / k
    pa = np.zeros(n_h + 1)
    pb = np.zeros(n_h + 1)
    pa[0] = 0.3
    if n_h >= 1:
        pa[1], pb[1] = 0.1, -0.05
    s = Spec(m, 1.1, mu, 1.7, n_h, beta=0.2, tags=tag)
    s.inflows.append((1, I.uniform_profile(m, [1], [1.0, 0.0, 0.0]), a, b))
    s.outlets_p.append((2, pa, pb))
    return s


def womersley_spec(level: int = 1, n_h: int = 4, seed: int = 1001, parabolic_none: bool = True) -> Spec:
    """Straight pipe R = 1, L = 5, rho = 1, mu = 0.04, Womersley number 4 (omega = 16 nu), mean
    Reynolds number 100 (mean velocity 2), parabolic inflow scaled by seeded harmonics, traction-free
    outlet."""
    m = I.womersley_mesh(level)
    nu = 0.04
    omega = 16.0 * nu
    T = 2.0 * math.pi / omega
    a, b = I.waveform_harmonics(n_h, 2.0 * math.pi, seed)
    s = Spec(m, 1.0, 0.04, T, n_h)
    s.inflows.append((1, None if parabolic_none else I.parabolic_profile(m, 1), a, b))
    return s


def glenn_spec(n_tets=1_000_000, n_h=10, seed=2000) -> Spec:
    """Glenn-like T-junction in cgs units: rho 1.06, mu 0.04, T 0.6979 s, parabolic inflow on both
    inflow tubes (10 seeded harmonics), resistance outlets at a mean level of 7.5 mmHg."""
    m = I.glenn_like(n_tets, seed)
    mmHg = 1333.22
    s = Spec(m, 1.06, 0.04, 0.6979, n_h)
    for k, tag in enumerate(m.inlet_tags):
        q_mean = 0.5 * math.pi * 0.36 * 30.0           # mean velocity 15 cm/s
        a, b = I.waveform_harmonics(n_h, q_mean, seed + 10 + k)
        s.inflows.append((tag, None, a, b))
    for k, tag in enumerate(m.outlet_tags):
        pa = np.zeros(n_h + 1)
        pb = np.zeros(n_h + 1)
        pa[0] = 7.0 * mmHg
        s.outlets_r.append((tag, 30.0, pa, pb))
    return s


def cerebral_spec(n_tets=2_000_000, n_h=10, seed=3000) -> Spec:
    """Cerebral-like vessel (tube of radius 0.2 cm along a seeded spline with a saccular bulge) in cgs
    units: rho 1.06, mu 0.04, T 1 s, parabolic inflow with 10 seeded harmonics at a mean velocity of
    15 cm/s, outlet at a steady 115 mmHg (Sec. 3.2 stand-in)."""
    m = I.cerebral_like(n_tets, seed)
    mmHg = 1333.22
    a, b = I.waveform_harmonics(n_h, math.pi * 0.04 * 15.0, seed + 11)
    pa = np.zeros(n_h + 1)
    pb = np.zeros(n_h + 1)
    pa[0] = 115.0 * mmHg
    s = Spec(m, 1.06, 0.04, 1.0, n_h, name=f"cerebral_s{seed}")
    s.inflows.append((1, None, a, b))
    s.outlets_p.append((2, pa, pb))
    return s


def coronary_spec(n_tets=300_000, n_h=10, seed=4000, reynolds=100.0, severity=(0.3, 0.7)) -> Spec:
    """Stenosed coronary-like tube (radius U(0.15, 0.25) cm, 30-70 % diameter reduction) in cgs units:
    rho 1.06, mu 0.04, T 0.8 s, parabolic inflow with 10 seeded harmonics at a mean Reynolds number of
    `reynolds`, outlet at a steady 70 mmHg (Sec. 3.3 stand-in)."""
    m = I.stenosed_tube(n_tets, seed, severity)
    rng = np.random.default_rng(seed + 7)
    R = float(np.max(np.linalg.norm(m.xyz[:, :2], axis=1)))
    nu = 0.04 / 1.06
    u_mean = reynolds * nu / (2.0 * R)
    a, b = I.waveform_harmonics(n_h, u_mean * math.pi * R * R, seed + 11, amp_lo=0.3, amp_hi=0.8)
    mmHg = 1333.22
    pa = np.zeros(n_h + 1)
    pb = np.zeros(n_h + 1)
    pa[0] = 70.0 * mmHg
    s = Spec(m, 1.06, 0.04, 0.8, n_h, name=f"coronary_s{seed}")
    s.inflows.append((1, None, a, b))
    s.outlets_p.append((2, pa, pb))
    del rng
    return s


def vessel_spec(seed: int, n_h: int = 4, n_core: int = 5, n_rim: int = 3, n_axial: int = 6) -> Spec:
    """Seeded vessel-like pipe (the learned warm start's training family): radius U(0.8, 1.2), length
    U(4, 6) radii, a cosine narrowing of U(0, 25) % of the diameter, rho 1, mu 0.04, Womersley number
    U(3, 5), mean Reynolds number U(50, 100), parabolic inflow times seeded harmonics, traction-free
    outlet."""
    rng = np.random.default_rng(seed)
    R = rng.uniform(0.8, 1.2)
    L = R * rng.uniform(4.0, 6.0)
    sev = rng.uniform(0.0, 0.25)
    zc = L * rng.uniform(0.35, 0.65)
    ls = R * rng.uniform(0.8, 1.5)

    def rfun(z):
        if abs(z - zc) < ls:
            return R * (1.0 - 0.5 * sev * (1.0 + math.cos(math.pi * (z - zc) / ls)))
        return R

    m = I.pipe_mesh(R, L, n_core, n_rim, n_axial, radius_fn=rfun, name=f"vessel_s{seed}")
    nu = 0.04
    alpha = rng.uniform(3.0, 5.0)
    omega = alpha * alpha * nu / (R * R)
    re = rng.uniform(50.0, 100.0)
    u_mean = re * nu / (2.0 * R)
    a, b = I.waveform_harmonics(n_h, u_mean * math.pi * R * R, seed + 1)
    s = Spec(m, 1.0, 0.04, 2.0 * math.pi / omega, n_h, name=f"vessel_s{seed}")
    s.inflows.append((1, None, a, b))
    return s


def batch_specs(n: int = 64, seed: int = 5000, lo: int = 20_000, hi: int = 400_000):
    """Batch of vessels of uneven size and N: sizes log-uniform in [lo, hi] tetrahedra, families drawn
    from {pipe (oscillatory pipe flow), T-junction (Glenn-like), stenosed tube (coronary-like)}, n_h drawn
    from {4, 6, 10}."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(n):
        size = int(math.exp(rng.uniform(math.log(lo), math.log(hi))))
        fam = int(rng.integers(3))
        n_h = int(rng.choice([4, 6, 10]))
        s = seed + 100 + k
        if fam == 0:
            m = I.pipe_by_size(size, s)
            nu = 0.04
            a, b = I.waveform_harmonics(n_h, 2.0 * math.pi, s)
            sp = Spec(m, 1.0, 0.04, 2.0 * math.pi / (16 * nu), n_h, name=f"pipe_{k}")
            sp.inflows.append((1, None, a, b))
        elif fam == 1:
            sp = glenn_spec(n_tets=size, n_h=n_h, seed=s)
        else:
            sp = coronary_spec(n_tets=size, n_h=n_h, seed=s)
        specs.append(sp)
    return specs
