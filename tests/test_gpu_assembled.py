"""The assembled paper tangent (per node pair and instance K, G, D, L and the pair mass; applied as a
row-wise sparse product) against the oracle's matrix-free paper tangent, element by element (FP64 1e-12,
FP32 1e-5), for compile-time and generic instance counts, with prescribed velocities and resistance
outlets; the device path against the fused element pass; and a solve that uses it."""
import numpy as np
import pytest

from oracle import hb_oracle as O
from paper_2411_14315_gb300 import hbgls
from paper_2411_14315_gb300 import inputs as I
from tests import problems as P

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def relerr(a, b):
    out = 0.0
    for f in range(b.shape[1]):
        n = np.linalg.norm(b[:, f])
        d = np.linalg.norm(a[:, f] - b[:, f])
        out = max(out, d / n if n > 0 else d)
    return out


@pytest.mark.parametrize("n_h", [0, 1, 4, 10, 15])
def test_assembled_tangent_matches_oracle(n_h):
    spec = P.box_spec(seed=80 + n_h, n_h=n_h, n=(6, 5, 4))
    ora = P.oracle_problem(spec)
    gp = P.gpu_problem(spec)
    y = I.random_state(spec.mesh.n_nodes, spec.N, 81)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 82)
    ref = O.jv_paper(ora, y, v, shift=0.8)
    for prec in (0, 1):
        assert relerr(gp.jv(y, v, kind=hbgls.ASSEMBLED, precision=prec, shift=0.8), ref) < TOL[prec], prec
    gp.close()


def test_device_path_matches_element_pass():
    torch = pytest.importorskip("torch")
    spec = P.box_spec(seed=90, n_h=3, n=(7, 5, 4))
    gp = P.gpu_problem(spec)
    n, N = spec.mesh.n_nodes, spec.N
    y = torch.tensor(I.random_state(n, N, 91), dtype=torch.float32, device="cuda")
    v = torch.tensor(I.random_state(n, N, 92), dtype=torch.float32, device="cuda")
    o1 = torch.empty_like(y)
    o2 = torch.empty_like(y)
    with pytest.raises(hbgls.HBError):
        gp.jv_dev(y, v, o2, hbgls.ASSEMBLED, hbgls.FP32, 1.3)         # nothing assembled yet
    gp.jv_dev(y, v, o1, hbgls.PAPER, hbgls.FP32, 1.3)
    gp.assemble_dev(y, hbgls.FP32)
    for _ in range(2):                                                  # the assembly is reusable
        gp.jv_dev(y, v, o2, hbgls.ASSEMBLED, hbgls.FP32, 1.3)
        torch.cuda.synchronize()
        a, b = o2.double().cpu().numpy(), o1.double().cpu().numpy()
        assert relerr(a, b) < 1e-5
    gp.close()


def test_solve_through_assembled_tangent():
    spec = P.channel_spec()
    ora = P.oracle_problem(spec)
    y_ref, hist = O.solve(ora, rtol=1e-13, gmres_tol=1e-10, max_steps=60)
    gp = P.gpu_problem(spec)
    rep = gp.solve(precision=1, rtol=1e-12, assembled=1)
    assert rep["status"] == 0
    assert relerr(gp.instances(), y_ref) < 1e-8
    gp.close()
