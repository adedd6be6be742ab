"""Batched operator application (one captured graph; one persistent element launch over many problems of
different N, or one per instance count) against the CPU oracle per member and per field, and against per-problem
calls; patch autotuning."""
import numpy as np
import pytest

from oracle import hb_oracle as O
from paper_2411_14315_gb300 import inputs as I
from tests import problems as P

pytestmark = pytest.mark.gpu


def _problems():
    specs = [P.box_spec(seed=71, n_h=4, n=(6, 4, 4)), P.box_spec(seed=72, n_h=6, n=(5, 4, 3)),
             P.box_spec(seed=73, n_h=10, n=(7, 5, 4)), P.box_spec(seed=74, n_h=2, n=(4, 4, 4)),
             P.womersley_spec()]
    return specs, [P.gpu_problem(s) for s in specs]


def _relerr_fields(a, b):
    """max over the four fields of ||a_f - b_f|| / ||b_f||."""
    return max(np.linalg.norm(a[:, f] - b[:, f]) / max(np.linalg.norm(b[:, f]), 1e-300) for f in range(4))


@pytest.mark.parametrize("grouping", [0, 1, 2])
@pytest.mark.parametrize("precision,kind", [(1, 0), (1, 1), (0, 0), (0, 1)])
def test_batch_matches_oracle(precision, kind, grouping):
    """Every member of a batch of five problems (N = 5, 9, 13, 21 and the Womersley pipe at 9; pressure,
    resistance and traction-free outlets; prescribed velocities) against the oracle's paper tangent
    (Eqs. ptangent, K_mat, ctangent, F_mat) or exact Jacobian, field by field: FP64 1e-12, FP32 1e-5."""
    torch = pytest.importorskip("torch")
    from paper_2411_14315_gb300 import hbgls
    specs, probs = _problems()
    dt = torch.float64 if precision == 0 else torch.float32
    ys = [torch.tensor(I.random_state(s.mesh.n_nodes, s.N, 180 + k), dtype=dt, device="cuda") for k, s in enumerate(specs)]
    vs = [torch.tensor(I.random_state(s.mesh.n_nodes, s.N, 190 + k), dtype=dt, device="cuda") for k, s in enumerate(specs)]
    outs = [torch.empty_like(y) for y in ys]
    shift = 0.6
    b = hbgls.Batch(probs, precision)
    b.set_grouping(grouping)
    st = torch.cuda.current_stream()
    b.jv_dev(ys, vs, outs, kind, shift, stream=st)
    st.synchronize()
    tol = 1e-12 if precision == 0 else 1e-5
    fn = O.jv_paper if kind == 0 else O.jv_exact
    for s, y, v, o in zip(specs, ys, vs, outs):
        ora = P.oracle_problem(s)
        # the oracle sees exactly the values the kernels saw (FP32 inputs widened without rounding)
        ref = fn(ora, y.double().cpu().numpy(), v.double().cpu().numpy(), shift=shift)
        err = _relerr_fields(o.double().cpu().numpy(), ref)
        assert err < tol, (s.N, err)
    b.close()


@pytest.mark.parametrize("precision,kind", [(1, 0), (1, 1), (0, 0)])
def test_batch_matches_individual_calls(precision, kind):
    torch = pytest.importorskip("torch")
    from paper_2411_14315_gb300 import hbgls
    specs, probs = _problems()
    dt = torch.float64 if precision == 0 else torch.float32
    ys = [torch.tensor(I.random_state(s.mesh.n_nodes, s.N, 80 + k), dtype=dt, device="cuda") for k, s in enumerate(specs)]
    vs = [torch.tensor(I.random_state(s.mesh.n_nodes, s.N, 90 + k), dtype=dt, device="cuda") for k, s in enumerate(specs)]
    outs = [torch.empty_like(y) for y in ys]
    refs = [torch.empty_like(y) for y in ys]
    s = torch.cuda.current_stream()
    for p, y, v, r in zip(probs, ys, vs, refs):
        p.jv_dev(y, v, r, kind, precision, 0.6, stream=s)
    b = hbgls.Batch(probs, precision)
    for _ in range(2):                      # second call replays the captured graph
        b.jv_dev(ys, vs, outs, kind, 0.6, stream=s)
    s.synchronize()
    tol = 1e-12 if precision == 0 else 2e-6
    for o, r in zip(outs, refs):
        o, r = o.double().cpu().numpy(), r.double().cpu().numpy()
        assert np.linalg.norm(o - r) <= tol * np.linalg.norm(r)
    assert b.launch_count() > 0
    b.close()


def test_patch_autotuning_keeps_results():
    spec = P.womersley_spec()
    gp = P.gpu_problem(spec)
    y = I.random_state(spec.mesh.n_nodes, spec.N, 5)
    v = I.random_state(spec.mesh.n_nodes, spec.N, 6)
    before = gp.jv(y, v, 1, 1, 0.2)
    best, ms = gp.tune_patches(1, [16, 32, 48, 64, 96], reps=3)
    assert best in (16, 32, 48, 64, 96) and ms > 0
    after = gp.jv(y, v, 1, 1, 0.2)
    assert np.linalg.norm(after - before) <= 2e-6 * np.linalg.norm(before)


def test_batch_member_with_deterministic_summation():
    """In the default layout each member runs its own operator, so a member set to deterministic
    summation (hb_set_scatter(0)) keeps it inside the batch: bitwise equal on a second replay and equal to
    its own per-problem call."""
    torch = pytest.importorskip("torch")
    from paper_2411_14315_gb300 import hbgls
    specs, probs = _problems()
    probs[2].set_scatter(0)
    ys = [torch.tensor(I.random_state(s.mesh.n_nodes, s.N, 280 + k), dtype=torch.float32, device="cuda")
          for k, s in enumerate(specs)]
    vs = [torch.tensor(I.random_state(s.mesh.n_nodes, s.N, 290 + k), dtype=torch.float32, device="cuda")
          for k, s in enumerate(specs)]
    outs = [torch.empty_like(y) for y in ys]
    st = torch.cuda.current_stream()
    b = hbgls.Batch(probs, 1)
    b.jv_dev(ys, vs, outs, 0, 0.6, stream=st)
    st.synchronize()
    first = outs[2].clone()
    b.jv_dev(ys, vs, outs, 0, 0.6, stream=st)
    ref = torch.empty_like(ys[2])
    probs[2].jv_dev(ys[2], vs[2], ref, 0, 1, 0.6, stream=st)
    st.synchronize()
    assert torch.equal(first, outs[2])
    assert torch.equal(first, ref)
    b.close()


def test_batch_recaptures_after_a_member_setting_changes():
    """A member switched to full RBVMS after the batch's first use (same operands, kind and shift) is
    applied with the new setting on the next batched call: its exact-Jacobian product then equals its own
    per-problem call and differs from the one before."""
    torch = pytest.importorskip("torch")
    from paper_2411_14315_gb300 import hbgls
    specs, probs = _problems()
    ys = [torch.tensor(I.random_state(s.mesh.n_nodes, s.N, 380 + k), dtype=torch.float32, device="cuda")
          for k, s in enumerate(specs)]
    vs = [torch.tensor(I.random_state(s.mesh.n_nodes, s.N, 390 + k), dtype=torch.float32, device="cuda")
          for k, s in enumerate(specs)]
    outs = [torch.empty_like(y) for y in ys]
    st = torch.cuda.current_stream()
    for grouping in (2, 0):
        probs[2].set_stabilization(0, 0.0)
        b = hbgls.Batch(probs, 1)
        b.set_grouping(grouping)
        b.jv_dev(ys, vs, outs, 1, 0.6, stream=st)
        st.synchronize()
        before = outs[2].double().cpu().numpy()
        probs[2].set_stabilization(1, 0.0)
        b.jv_dev(ys, vs, outs, 1, 0.6, stream=st)
        ref = torch.empty_like(ys[2])
        probs[2].jv_dev(ys[2], vs[2], ref, 1, 1, 0.6, stream=st)
        st.synchronize()
        after, ref = outs[2].double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.linalg.norm(after - ref) <= 2e-6 * np.linalg.norm(ref), grouping
        assert np.linalg.norm(after - before) > 1e-4 * np.linalg.norm(ref), grouping
        b.close()
