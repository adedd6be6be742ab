"""GPU parity of the learned warm-start network (BF16 weights, FP32 arithmetic) with its FP64 oracle."""
import math

import numpy as np
import pytest

from oracle import hb_oracle as O
from oracle import mpnn_oracle as MO
from paper_2411_14315_gb300 import inputs as I
from paper_2411_14315_gb300 import workloads as W
from tests import problems as P

pytestmark = pytest.mark.gpu


def _spec(n_h=3, seed=4100):
    return W.coronary_spec(n_tets=4000, n_h=n_h, seed=seed, reynolds=50.0)


def _oracle_inputs(spec):
    m = spec.mesh
    tag, prof, a, b = spec.inflows[0]
    prof = I.parabolic_profile(m, tag) if prof is None else prof
    wave = np.zeros(2 * spec.n_h + 1)
    wave[0] = a[0]
    wave[1::2] = a[1:]
    wave[2::2] = b[1:]
    return MO.graph_inputs(m.xyz, m.tets, m.faces, spec.face_tag, [t for t, *_ in spec.inflows], prof, wave)


def _refs(spec):
    """u_ref: largest mean inflow speed over instances and inflows; p_ref: mean outlet level."""
    ora = P.oracle_problem(spec)
    _, g = ora.dirichlet()
    u = 0.0
    for tag in ora.inflow:
        f = np.nonzero(ora.face_tag == tag)[0]
        A = ora.face_area[f].sum()
        un = np.abs(np.einsum("fbin,fi->fbn", g[ora.faces[f]], ora.face_normal[f]))
        u = max(u, float(np.einsum("f,fbn->n", ora.face_area[f] / 3.0, un).max() / A))
    lv = [O.sample_waveform(a, b, spec.N, spec.T) for (a, b) in ora.outlet_p.values()]
    lv += [O.sample_waveform(a, b, spec.N, spec.T) for (_, a, b) in ora.outlet_r.values()]
    return u, float(np.mean(lv)), spec.rho


def _bf16_exact(a):
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def test_graph_inputs_match_oracle_definition():
    from paper_2411_14315_gb300 import hbgls
    spec = _spec()
    gp = P.gpu_problem(spec)
    net = hbgls.MPNN(spec.n_h)
    x, src, dst, e = net.graph(gp)
    xo, so, do, eo = _oracle_inputs(spec)
    assert np.allclose(x, xo, atol=2e-6)
    assert len(src) == len(so)
    lib = {(int(a), int(b)): e[k] for k, (a, b) in enumerate(zip(src, dst))}
    for k in range(0, len(so), 7):
        assert np.allclose(lib[(int(so[k]), int(do[k]))], eo[k], atol=2e-6)


@pytest.mark.parametrize("tensor_cores", [True, False])
def test_loss_and_gradient_match_oracle(tensor_cores):
    """Loss and parameter gradient against the FP64 oracle with BF16-exact weights, with the forward MLPs on
    the tensor cores (TF32 head/tail split, FP32 accumulation) and on FP32 FMAs."""
    from paper_2411_14315_gb300 import hbgls
    spec = _spec()
    gp = P.gpu_problem(spec)
    net = hbgls.MPNN(spec.n_h, seed=5)
    net.set_tensor_cores(tensor_cores)
    M = 2 * spec.n_h + 1
    shapes = MO.layer_shapes(MO.F_IN, MO.F_E, 4 * M, hidden=64, layers=3)
    rng = np.random.default_rng(6)
    p = MO.flatten(MO.init_params(shapes, 7))
    p = p + rng.normal(0, 0.05, p.shape)          # non-zero biases
    p = _bf16_exact(p)
    assert p.size == net.num_params
    net.set_params(p)
    u, pr, rho = _refs(spec)
    t = rng.normal(size=(spec.mesh.n_nodes, 4, M))
    t[:, :3] *= u
    t[:, 3] *= rho * u * u
    t[:, 3, 0] += pr
    loss, grad = net.loss_grad(gp, t)
    x, src, dst, e = _oracle_inputs(spec)
    lo, go = MO.loss_and_grad(MO.unflatten(p.astype(np.float64), shapes), x, src, dst, e,
                              MO.normalise_target(t, u, pr, rho), layers=3)   # default pressure scale 1
    go = MO.flatten(go)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    assert np.linalg.norm(grad - go) <= 1e-4 * np.linalg.norm(go)


def test_training_reduces_loss_and_warm_start_sets_state():
    from paper_2411_14315_gb300 import hbgls
    spec = _spec()
    gp = P.gpu_problem(spec)
    net = hbgls.MPNN(spec.n_h, seed=8)
    gp.set_instances(None)
    target = gp.harmonics()                      # the default initial state, a smooth target
    l0 = net.train_step(gp, target, 1e-3)
    for _ in range(150):
        l1 = net.train_step(gp, target, 1e-3)
    assert l1 < 0.3 * l0
    pred = net.predict(gp)
    assert np.all(np.isfinite(pred))
    net.warm_start(gp)
    y = gp.instances()
    ora = P.oracle_problem(spec)
    mask, g = ora.dirichlet()
    assert np.allclose(y[mask, :3], g[mask], atol=1e-12)


def test_tensor_core_forward_matches_fma_forward():
    """The prediction with tensor-core MLPs equals the FP32-FMA prediction to FP32 accuracy (hidden 32 and
    64, output widths of N = 7 and N = 21)."""
    from paper_2411_14315_gb300 import hbgls
    for n_h, hidden in ((3, 64), (10, 64), (3, 32)):
        spec = _spec(n_h=n_h)
        gp = P.gpu_problem(spec)
        net = hbgls.MPNN(n_h, hidden=hidden, seed=9)
        p = net.get_params()
        net.set_params(p + np.random.default_rng(3).normal(0, 0.05, p.shape).astype(np.float32))
        net.set_tensor_cores(False)
        a = net.predict(gp)
        net.set_tensor_cores(True)
        b = net.predict(gp)
        assert np.linalg.norm(b - a) <= 2e-5 * np.linalg.norm(a), (n_h, hidden)
        net.close()
        gp.close()
