"""GPU solve against the oracle's solve: the periodic state the library converges to (plain FP64 path
and mixed FP32-operator path) is the oracle's root to 1e-8 relative per field, the bar for a final
solution.  The oracle's root comes from its own pseudo-transient Newton-GMRES (readings R6, R7) driven to
||r|| <= 1e-12 ||r0||."""
import numpy as np
import pytest

from oracle import hb_oracle as O
from tests import problems as P

pytestmark = pytest.mark.gpu


def relerr(a, b):
    out = 0.0
    for f in range(a.shape[1]):
        n = np.linalg.norm(b[:, f])
        d = np.linalg.norm(a[:, f] - b[:, f])
        out = max(out, d / n if n > 0 else d)
    return out


@pytest.fixture(scope="module")
def channel_root():
    spec = P.channel_spec()
    ora = P.oracle_problem(spec)
    y, hist = O.solve(ora, rtol=1e-13, gmres_tol=1e-10, max_steps=60)
    assert hist[-1] <= 1e-12 * hist[0]
    return spec, ora, y


@pytest.mark.parametrize("precision,precond", [(0, 0), (1, 0), (0, 1), (1, 1), (0, 2), (1, 2)])
def test_solution_matches_oracle_root(channel_root, precision, precond):
    """Plain Jacobi (the paper's), node-block and aggregation-multigrid preconditioning reach the same
    root."""
    spec, ora, y_ref = channel_root
    gp = P.gpu_problem(spec)
    rep = gp.solve(precision=precision, rtol=1e-12, precond=precond)
    assert rep["status"] == 0
    y = gp.instances()
    assert relerr(y, y_ref) < 1e-8
    # the state is a root of the oracle's residual too (its Dirichlet rows hold the prescribed values)
    r = O.residual(ora, y)
    assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(O.residual(ora, ora.initial_state()))
    gp.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_multigrid_preconditioner_on_the_pipe(precision):
    """On the Womersley pipe (~3,000 tets, N = 9; the multigrid hierarchy has a coarse level) the solve with
    the multigrid preconditioner ends at the state of the Jacobi-preconditioned solve (1e-8) with fewer
    GMRES iterations."""
    spec = P.womersley_spec()
    ref = P.gpu_problem(spec)
    r0 = ref.solve(precision=0, rtol=1e-12, max_steps=300)
    assert r0["status"] == 0
    yref = ref.instances()
    gp = P.gpu_problem(spec)
    rep = gp.solve(precision=precision, rtol=1e-11, max_steps=300, precond=2)
    assert rep["status"] == 0
    assert relerr(gp.instances(), yref) < 1e-8
    print("GMRES iterations: jacobi", r0["gmres_iters"], "multigrid", rep["gmres_iters"])
    assert rep["gmres_iters"] < r0["gmres_iters"]
    gp.close()
    ref.close()
