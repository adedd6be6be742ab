"""hb_jv_dev_noalloc: the Jacobian-vector product for callers that cannot let the library allocate.

Such callers own all device memory through their own allocator (a caching pool can leave cudaMalloc
failing while the pool still holds free memory) or run latency-critical loops that a cudaMalloc or
cudaFree would stall by synchronising the device.  The entry point keeps its only scratch (per-outlet
flow rates of resistance outlets) in a fixed device array, so this test checks, through the C ABI,
that two calls in a row reproduce the allocating entry point's result on a problem with a resistance
outlet, and that device free memory does not change across the calls.

This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2411_14315_gb300 import inputs as I
from tests import problems as P

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.mark.parametrize("n_h", [3, 10])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind", [0, 1])
def test_noalloc_jv_matches_allocating_jv_twice(precision, kind, n_h):
    """N = 7 (generic in-patch H) and N = 21 (the circulant kernel in registers)."""
    torch = pytest.importorskip("torch")
    from paper_2411_14315_gb300 import hbgls
    spec = P.box_spec(seed=77, n=(6, 4, 4), n_h=n_h, resistance=True)
    gp = P.gpu_problem(spec)
    gp.info()                                   # prepares the boundary data (allocates, once)
    dt = torch.float64 if precision == 0 else torch.float32
    y = torch.tensor(I.random_state(spec.mesh.n_nodes, spec.N, 91), dtype=dt, device="cuda")
    v = torch.tensor(I.random_state(spec.mesh.n_nodes, spec.N, 92), dtype=dt, device="cuda")
    ref = torch.empty_like(y)
    out1 = torch.empty_like(y)
    out2 = torch.empty_like(y)
    s = torch.cuda.current_stream()
    gp.jv_dev(y, v, ref, kind, precision, 0.4, stream=s)
    gp.jv_dev_noalloc(y, v, out1, kind, precision, 0.4, stream=s)    # first call: device set-up
    s.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    gp.jv_dev_noalloc(y, v, out2, kind, precision, 0.4, stream=s)
    s.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before
    r = ref.double().cpu().numpy()
    for out in (out1, out2):
        o = out.double().cpu().numpy()
        assert np.linalg.norm(o - r) / np.linalg.norm(r) < TOL[precision]
    gp.close()
    assert hbgls.HB_OK == 0


def test_noalloc_jv_every_fp32_launch_variant():
    """The FP32 paper-tangent product through hb_jv_dev_noalloc under every launch variant (the pipelined
    variants need the allocating W pass and run variant 1 here) against hb_jv_dev, N = 21."""
    torch = pytest.importorskip("torch")
    spec = P.box_spec(seed=79, n=(6, 4, 4), n_h=10, resistance=True)
    gp = P.gpu_problem(spec)
    y = torch.tensor(I.random_state(spec.mesh.n_nodes, spec.N, 93), dtype=torch.float32, device="cuda")
    v = torch.tensor(I.random_state(spec.mesh.n_nodes, spec.N, 94), dtype=torch.float32, device="cuda")
    ref = torch.empty_like(y)
    out = torch.empty_like(y)
    s = torch.cuda.current_stream()
    for var in range(7):
        gp.set_launch_variant(var)
        gp.info()                               # the variant change asks for prepared data again
        gp.jv_dev(y, v, ref, 0, 1, 0.4, stream=s)
        gp.jv_dev_noalloc(y, v, out, 0, 1, 0.4, stream=s)
        s.synchronize()
        r = ref.double().cpu().numpy()
        assert np.linalg.norm(out.double().cpu().numpy() - r) / np.linalg.norm(r) < TOL[1], var
    gp.close()


def test_noalloc_jv_requires_prepared_boundary_data():
    torch = pytest.importorskip("torch")
    from paper_2411_14315_gb300 import hbgls
    spec = P.box_spec(seed=78, n=(3, 3, 3), n_h=1)
    gp = P.gpu_problem(spec)                    # boundary conditions set, not yet prepared
    y = torch.zeros(gp.shape, dtype=torch.float64, device="cuda")
    out = torch.empty_like(y)
    with pytest.raises(hbgls.HBError) as e:
        gp.jv_dev_noalloc(y, y.clone(), out, 0, 0)
    assert e.value.status == 8                  # HB_ERR_STATE
    gp.close()
