"""Oscillatory pipe flow against Womersley's closed form (an exact Navier-Stokes solution).

The pipe is driven by the exact inflow harmonics (general per-point Dirichlet data); the outlet is
traction free.  Convection vanishes and the flow is band-limited in time, so the harmonic balance
error is purely spatial: the velocity error must fall at second order in the cell size (P1), fitted over
three refinements."""
import math

import numpy as np
import pytest

from oracle import hb_oracle as O
from oracle import womersley as Wo
from paper_2411_14315_gb300 import inputs as I
from paper_2411_14315_gb300 import workloads as W
from tests import problems as P

pytestmark = pytest.mark.gpu


def _spec(level):
    spec = W.womersley_spec(level=level)
    tag, _, a, b = spec.inflows[0]
    omega = 2 * math.pi / spec.T
    exact = Wo.pipe_solution(spec.mesh.xyz, a, b, 1.0, 5.0, spec.rho, spec.mu, omega)
    spec.inflows = []
    spec.inflows_harm = [(tag, exact[:, :3])]
    return spec, exact


def test_harmonic_inflow_residual_matches_oracle():
    spec, exact = _spec(1)
    ora = P.oracle_problem(spec)
    gp = P.gpu_problem(spec)
    gp.set_instances(None)
    assert np.allclose(gp.instances(), ora.initial_state(), atol=1e-12)
    y = ora.apply_dirichlet(I.smooth_state(spec.mesh, spec.N, 3, vel=2.0))
    r = gp.residual(y, 0)
    ref = O.residual(ora, y)
    assert np.linalg.norm(r - ref) <= 1e-12 * np.linalg.norm(ref)


def test_womersley_second_order_convergence():
    """Three refinements of the pipe (~3k, ~24k, ~196k tetrahedra, each halving the cell size): the solved
    velocity error against Womersley's solution falls at an observed order >= 1.8 in h between the two
    finest levels (P1 gives 2), and the least-squares fit over all three gives >= 1.7."""
    errs, hs = [], []
    for level in (1, 2, 3):
        spec, exact = _spec(level)
        gp = P.gpu_problem(spec)
        rep = gp.solve(precision=1, rtol=1e-9, max_steps=400, precond=2)
        assert rep["status"] == 0
        h = gp.harmonics()
        errs.append(float(np.linalg.norm(h[:, :3] - exact[:, :3]) / np.linalg.norm(exact[:, :3])))
        hs.append(2.0 ** (1 - level))
        gp.close()
    order = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    fine = np.log(errs[1] / errs[2]) / np.log(2.0)          # observed order between the two finest levels
    print("Womersley velocity errors by level:", errs, "fitted order:", order, "finest-pair order:", fine)
    assert errs[0] < 0.08
    # the order of accuracy is an asymptotic property: the coarsest pipe (5 x 5 core cells) is still
    # pre-asymptotic, so the bar is on the finest pair, the three-level fit gets a looser one
    assert fine >= 1.8
    assert order >= 1.7
