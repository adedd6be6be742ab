"""Test adapters: apply one workload spec identically to the CPU oracle and to the library."""
from __future__ import annotations

from paper_2411_14315_gb300 import inputs as I
from paper_2411_14315_gb300.workloads import (Spec, box_spec, channel_spec, dirichlet_nodes,  # noqa: F401
                                              glenn_spec, womersley_spec)


def oracle_problem(spec: Spec, convection: bool = True):
    from oracle import hb_oracle as O
    m = spec.mesh
    pr = O.HBProblem(m.xyz, m.tets, m.faces, spec.face_tag, spec.rho, spec.mu, spec.T, spec.n_h,
                     beta_bf=spec.beta, convection=convection)
    for tag, prof, a, b in spec.inflows:
        if prof is None:
            prof = I.parabolic_profile(m, tag)
        pr.set_inflow(tag, prof, a, b)
    for tag, harm in spec.inflows_harm:
        pr.set_inflow_harmonics(tag, harm)
    for tag, a, b in spec.outlets_p:
        pr.set_outlet_pressure(tag, a, b)
    for tag, R, a, b in spec.outlets_r:
        pr.set_outlet_resistance(tag, R, a, b)
    return pr


def gpu_problem(spec: Spec, **kw):
    from paper_2411_14315_gb300 import hbgls
    return hbgls.Problem.from_spec(spec, **kw)
