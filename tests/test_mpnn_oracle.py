"""Pins of the network oracle: its hand-written backward pass against central differences of its own
forward pass, and properties of its graph inputs (no GPU)."""
import numpy as np

from oracle import mpnn_oracle as MO
from paper_2411_14315_gb300 import inputs as I


def _tiny_graph(seed=0):
    m = I.box_mesh(2, 2, 1, jitter=0.1, seed=seed)
    prof = I.uniform_profile(m, [1], [1.0, 0.0, 0.0])
    wave = np.array([1.0, 0.3, -0.2, 0.1, 0.05])
    x, src, dst, e = MO.graph_inputs(m.xyz, m.tets, m.faces, m.face_tag, [1], prof, wave)
    return m, x, src, dst, e


def test_backward_matches_central_differences():
    m, x, src, dst, e = _tiny_graph()
    shapes = MO.layer_shapes(MO.F_IN, MO.F_E, 12, hidden=8, layers=2)
    params = MO.init_params(shapes, 3)
    rng = np.random.default_rng(4)
    # non-zero biases so every path is exercised
    params = [(W1, rng.normal(0, 0.1, b1.shape), W2, rng.normal(0, 0.1, b2.shape)) for (W1, b1, W2, b2) in params]
    target = rng.normal(size=(x.shape[0], 12))
    loss, grads = MO.loss_and_grad(params, x, src, dst, e, target, layers=2)
    flat = MO.flatten(params)
    g = MO.flatten(grads)
    idx = rng.choice(flat.size, 60, replace=False)
    eps = 1e-6
    for k in idx:
        fp = flat.copy(); fp[k] += eps
        fm = flat.copy(); fm[k] -= eps
        lp, _ = MO.loss_and_grad(MO.unflatten(fp, shapes), x, src, dst, e, target, layers=2)
        lm, _ = MO.loss_and_grad(MO.unflatten(fm, shapes), x, src, dst, e, target, layers=2)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_aggregation_is_a_sum_over_incoming_edges():
    """With one layer, zero message output weights except a bias, each node receives bias x in-degree."""
    m, x, src, dst, e = _tiny_graph(1)
    H = 4
    shapes = MO.layer_shapes(MO.F_IN, MO.F_E, 3, hidden=H, layers=1)
    params = [(np.zeros((i, h)), np.zeros(h), np.zeros((h, o)), np.zeros(o)) for (i, h, o) in shapes]
    bm = np.arange(1.0, H + 1)
    params[1] = (params[1][0], params[1][1], params[1][2], bm)               # msg: constant message bm
    params[2] = (np.vstack([np.zeros((H, H)), np.eye(H)]), np.zeros(H), np.eye(H), np.zeros(H))  # upd: relu(a)
    params[3] = (np.eye(H), np.zeros(H), np.ones((H, 3)), np.zeros(3))
    out, _ = MO.forward(params, x, src, dst, e, layers=1)
    deg = np.bincount(dst, minlength=x.shape[0])
    assert np.allclose(out[:, 0], deg * bm.sum())


def test_graph_inputs_edges_and_flags():
    m, x, src, dst, e = _tiny_graph(2)
    # both directions of each tetrahedron edge, no duplicates
    pairs = set(zip(src.tolist(), dst.tolist()))
    assert len(pairs) == src.size and all((b, a) in pairs for (a, b) in pairs)
    assert np.allclose(np.linalg.norm(e[:, :3], axis=1), e[:, 3])
    assert np.all(np.abs(x[:, :3]) <= 1.0 + 1e-12)
    assert set(np.unique(x[:, 3:6])) <= {0.0, 1.0}
