"""GPU parity of the stabilisation variants of Sec. 2.2 (remarks after Eq. tau) against the oracle:
full RBVMS (cross- and Reynolds-stress terms of u' = -tau L / rho) and the time-discretisation term
ct (1/dt)^2 under the root of tau.  FP64 1e-12, FP32 1e-5, per field, at random states."""
import numpy as np
import pytest

from oracle import hb_oracle as O
from paper_2411_14315_gb300 import inputs as I
from tests import problems as P

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}
VARIANTS = [(1, 0.0), (0, 1.0), (1, 2.0)]


def relerr(a, b):
    return max(np.linalg.norm(a[:, f] - b[:, f]) / max(np.linalg.norm(b[:, f]), 1e-300) for f in range(4))


def _pair(variant, ct, n_h=3, n=(7, 5, 4)):
    spec = P.box_spec(n=n, n_h=n_h)
    ora = P.oracle_problem(spec)
    ora.stab = "rbvms" if variant == 1 else "gls"
    ora.ct_dt = ct
    gp = P.gpu_problem(spec)
    gp.set_stabilization(variant, ct)
    return spec, ora, gp


@pytest.mark.parametrize("variant,ct", VARIANTS)
@pytest.mark.parametrize("precision", [0, 1])
def test_variant_residual_and_jacobians(variant, ct, precision):
    spec, ora, gp = _pair(variant, ct)
    y = I.random_state(spec.mesh.n_nodes, spec.N, 51)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 52)
    assert relerr(gp.residual(y, precision), O.residual(ora, y)) < TOL[precision]
    assert relerr(gp.jv(y, v, 1, precision, 0.4), O.jv_exact(ora, y, v, shift=0.4)) < TOL[precision]
    assert relerr(gp.jv(y, v, 0, precision, 0.4), O.jv_paper(ora, y, v, shift=0.4)) < TOL[precision]
    assert relerr(gp.jv(y, v, 2, precision, 0.4), O.jv_paper(ora, y, v, shift=0.4)) < TOL[precision]
    d = gp.jacobi_diag(y, precision, 0.4)
    assert relerr(d, O.jacobi_diag(ora, y, shift=0.4)) < TOL[precision]
    gp.close()


def test_variant_switch_back_restores_gls():
    spec, ora, gp = _pair(1, 2.0)
    y = I.random_state(spec.mesh.n_nodes, spec.N, 53)
    r1 = gp.residual(y, 0)
    gp.set_stabilization(0, 0.0)
    ora.stab, ora.ct_dt = "gls", 0.0
    r0 = gp.residual(y, 0)
    assert relerr(r0, O.residual(ora, y)) < 1e-12
    assert np.linalg.norm(r1 - r0) > 1e-6 * np.linalg.norm(r0)
    with pytest.raises(RuntimeError):
        gp.set_stabilization(2, 0.0)
    with pytest.raises(RuntimeError):
        gp.set_stabilization(0, -1.0)
    gp.close()


@pytest.mark.parametrize("variant,ct", [(1, 0.0), (0, 1.0)])
def test_variant_solve_reaches_a_root_of_the_oracle_residual(variant, ct):
    """The library's solve under a variant ends at a root of the oracle's residual of that variant."""
    spec = P.channel_spec()
    ora = P.oracle_problem(spec)
    ora.stab = "rbvms" if variant == 1 else "gls"
    ora.ct_dt = ct
    gp = P.gpu_problem(spec)
    gp.set_stabilization(variant, ct)
    rep = gp.solve(precision=0, rtol=1e-12, max_steps=200)
    assert rep["status"] == 0
    y = gp.instances()
    r = O.residual(ora, y)
    r0 = O.residual(ora, ora.initial_state())
    assert np.linalg.norm(r) < 1e-9 * np.linalg.norm(r0)
    gp.close()
