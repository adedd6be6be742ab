"""The deterministic element-to-node summation (hb_set_scatter(0)) on the GPU.

Every operator of the library -- residual (Eq. Rmc), the paper's tangent (Eqs. K_mat, ctangent, F_mat)
matrix-free and assembled, the exact Jacobian and the Jacobi diagonal -- is evaluated twice in the
deterministic mode and must come back bitwise equal; it must match the oracle to the usual bars (FP64
1e-12, FP32 1e-5, norm-wise relative per field) and the atomic mode to the same bars.  The box has a
resistance outlet (flow rates summed per outlet) and backflow faces, so the face slots and the
fixed-order outlet sums are exercised; its mesh spans many patches with a ragged last one.  A whole
mixed-precision solve run twice in that mode reproduces its iterates bit for bit.
"""
import numpy as np
import pytest

from oracle import hb_oracle as O
from paper_2411_14315_gb300 import inputs as I
from tests import problems as P

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def relerr(a, b):
    return max(np.linalg.norm(a[:, f] - b[:, f]) / max(np.linalg.norm(b[:, f]), 1e-300) for f in range(a.shape[1]))


@pytest.fixture(scope="module")
def box():
    spec = P.box_spec(n=(9, 7, 6), n_h=3)
    ora = P.oracle_problem(spec)
    gp = P.gpu_problem(spec)
    yield spec, ora, gp
    gp.close()


def _ops(gp, y, v, precision):
    return {
        "residual": gp.residual(y, precision),
        "jv_paper": gp.jv(y, v, 0, precision, 0.4),
        "jv_exact": gp.jv(y, v, 1, precision, 0.4),
        "jv_assembled": gp.jv(y, v, 2, precision, 0.4),
        "diag": gp.jacobi_diag(y, precision, 0.4),
    }


def _oracle(ora, y, v):
    return {
        "residual": O.residual(ora, y),
        "jv_paper": O.jv_paper(ora, y, v, shift=0.4),
        "jv_exact": O.jv_exact(ora, y, v, shift=0.4),
        "jv_assembled": O.jv_paper(ora, y, v, shift=0.4),
        "diag": O.jacobi_diag(ora, y, shift=0.4),
    }


@pytest.mark.parametrize("precision", [0, 1])
def test_deterministic_mode_is_bitwise_repeatable_and_matches_the_oracle(box, precision):
    spec, ora, gp = box
    y = I.random_state(spec.mesh.n_nodes, spec.N, 71)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 72)
    gp.set_scatter(0)
    assert gp.scatter() == 0
    try:
        first = _ops(gp, y, v, precision)
        second = _ops(gp, y, v, precision)
    finally:
        gp.set_scatter(1)
    atomic = _ops(gp, y, v, precision)
    ref = _oracle(ora, y, v)
    for name in first:
        assert np.array_equal(first[name], second[name]), name
        assert relerr(first[name], ref[name]) < TOL[precision], name
        assert relerr(first[name], atomic[name]) < TOL[precision], name


def test_deterministic_mode_with_rbvms_and_many_instances():
    """The residual and exact Jacobian carry 7 slot fields per node (the T rows go through H after the
    gather); full RBVMS and the dt term of tau at N = 9 (generic and fixed-N kernels alike)."""
    spec = P.box_spec(n=(7, 5, 4), n_h=4)
    ora = P.oracle_problem(spec)
    ora.stab, ora.ct_dt = "rbvms", 1.0
    gp = P.gpu_problem(spec)
    gp.set_stabilization(1, 1.0)
    gp.set_scatter(0)
    y = I.random_state(spec.mesh.n_nodes, spec.N, 73)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 74)
    for precision in (0, 1):
        r1, r2 = gp.residual(y, precision), gp.residual(y, precision)
        assert np.array_equal(r1, r2)
        assert relerr(r1, O.residual(ora, y)) < TOL[precision]
        j1, j2 = gp.jv(y, v, 1, precision, 0.3), gp.jv(y, v, 1, precision, 0.3)
        assert np.array_equal(j1, j2)
        assert relerr(j1, O.jv_exact(ora, y, v, shift=0.3)) < TOL[precision]
    gp.close()


def test_deterministic_solve_repeats_bit_for_bit():
    """Two mixed-precision solves from the same start in the deterministic mode (assembled multigrid
    preconditioner, so the row-wise assembly is in the loop) give identical reports and states, and the
    state is a root of the oracle's residual."""
    spec = P.channel_spec()
    ora = P.oracle_problem(spec)
    states, reports = [], []
    for _ in range(2):
        gp = P.gpu_problem(spec)
        rep = gp.solve(precision=1, rtol=1e-10, precond=2, scatter=0)
        assert rep["status"] == 0
        assert gp.scatter() == 0
        states.append(gp.instances())
        reports.append((rep["steps"], rep["gmres_iters"], rep["jv_calls"], rep["res_final"]))
        gp.close()
    assert reports[0] == reports[1]
    assert np.array_equal(states[0], states[1])
    r = O.residual(ora, states[0])
    r0 = O.residual(ora, ora.initial_state())
    assert np.linalg.norm(r) < 1e-8 * np.linalg.norm(r0)


def test_scatter_setting_is_checked(box):
    _, _, gp = box
    with pytest.raises(RuntimeError):
        gp.set_scatter(2)
    assert gp.scatter() == 1
