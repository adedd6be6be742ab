"""Plain FP64 CPU oracle of the message-passing network used as a learned warm start.

TEST INFRASTRUCTURE ONLY: the tests use it to check the GPU network's forward pass and gradients.
It shares no code with the CUDA library.

The network is not part of the paper's method.  The paper only suggests that harmonic balance
solutions could serve as machine-learning datasets (Sec. 4); this network is trained on solutions the
method itself generates.  Definition (H hidden width, L layers):

    mlp(p, X)   = relu(X W1 + b1) W2 + b2
    h           = mlp(enc, x)                                     node encoder
    for each layer l:
        m_e     = mlp(msg_l, [h[src_e], h[dst_e], e_e])           message on directed edge e
        a_i     = sum over edges e with dst_e = i of m_e          aggregation
        h       = h + mlp(upd_l, [h, a])                          residual node update
    out         = mlp(dec, h)
    loss        = mean over nodes and outputs of (out - target)^2

Parameters are a list of (W1, b1, W2, b2) tuples in the order enc, (msg_0, upd_0), ..., dec.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(f_in: int, f_e: int, f_out: int, hidden: int = 64, layers: int = 3):
    """(in, hidden, out) of every MLP in parameter order."""
    H = hidden
    shapes = [(f_in, H, H)]
    for _ in range(layers):
        shapes.append((2 * H + f_e, H, H))
        shapes.append((2 * H, H, H))
    shapes.append((H, H, f_out))
    return shapes


def init_params(shapes, seed: int):
    """Seeded parameters for the tests (an input of the definition above, not part of it)."""
    rng = np.random.default_rng(seed)
    ps = []
    for (i, h, o) in shapes:
        ps.append((rng.normal(0, (2.0 / i) ** 0.5, (i, h)), np.zeros(h),
                   rng.normal(0, (1.0 / h) ** 0.5, (h, o)), np.zeros(o)))
    return ps


def _mlp_fwd(p, X):
    """mlp(p, X) of the definition above; also returns what the backward pass needs."""
    W1, b1, W2, b2 = p
    Z = X @ W1 + b1
    A = np.maximum(Z, 0.0)
    return A @ W2 + b2, (X, A)


def _mlp_bwd(p, cache, dY):
    """Backward pass of mlp (chain rule): gradients of its parameters and of its input."""
    W1, b1, W2, b2 = p
    X, A = cache
    dW2 = A.T @ dY
    db2 = dY.sum(axis=0)
    dA = dY @ W2.T
    dZ = dA * (A > 0)
    dW1 = X.T @ dZ
    db1 = dZ.sum(axis=0)
    dX = dZ @ W1.T
    return dX, (dW1, db1, dW2, db2)


def forward(params, x, src, dst, e, layers: int):
    """The network of the definition above on one graph; returns (out, caches)."""
    H = params[0][2].shape[1]
    h, c_enc = _mlp_fwd(params[0], x)
    caches = [c_enc]
    for l in range(layers):
        pm, pu = params[1 + 2 * l], params[2 + 2 * l]
        xm = np.concatenate([h[src], h[dst], e], axis=1)
        m, cm = _mlp_fwd(pm, xm)
        a = np.zeros((h.shape[0], H))
        np.add.at(a, dst, m)
        du, cu = _mlp_fwd(pu, np.concatenate([h, a], axis=1))
        caches.append((cm, cu))
        h = h + du
    out, c_dec = _mlp_fwd(params[-1], h)
    caches.append(c_dec)
    return out, caches


def loss_and_grad(params, x, src, dst, e, target, layers: int):
    """The loss of the definition above and its gradient with respect to every parameter (backward pass
    through the layers in reverse order)."""
    H = params[0][2].shape[1]
    out, caches = forward(params, x, src, dst, e, layers)
    diff = out - target
    loss = float(np.mean(diff ** 2))
    dout = 2.0 * diff / diff.size
    grads = [None] * len(params)
    dh, grads[-1] = _mlp_bwd(params[-1], caches[-1], dout)
    n = x.shape[0]
    for l in reversed(range(layers)):
        pm, pu = params[1 + 2 * l], params[2 + 2 * l]
        cm, cu = caches[1 + l]
        dxu, grads[2 + 2 * l] = _mlp_bwd(pu, cu, dh)
        dh = dh + dxu[:, :H]
        da = dxu[:, H:]
        dm = da[dst]
        dxm, grads[1 + 2 * l] = _mlp_bwd(pm, cm, dm)
        np.add.at(dh, src, dxm[:, :H])
        np.add.at(dh, dst, dxm[:, H:2 * H])
    _, grads[0] = _mlp_bwd(params[0], caches[0], dh)
    del n
    return loss, grads


def flatten(ps):
    """Parameters in order as one vector (W1, b1, W2, b2 of each MLP, row-major)."""
    return np.concatenate([np.concatenate([W1.ravel(), b1, W2.ravel(), b2]) for (W1, b1, W2, b2) in ps])


def unflatten(vec, shapes):
    """Inverse of flatten."""
    ps = []
    o = 0
    for (i, h, out) in shapes:
        W1 = vec[o:o + i * h].reshape(i, h); o += i * h
        b1 = vec[o:o + h]; o += h
        W2 = vec[o:o + h * out].reshape(h, out); o += h * out
        b2 = vec[o:o + out]; o += out
        ps.append((W1, b1, W2, b2))
    return ps


# ---------------------------------------------------------------------------------------------------
# inputs of the network for one problem (restated here independently of the library)

F_IN, F_E = 32, 4


def graph_inputs(xyz, tets, faces, face_tag, inflow_tags, profile, wave):
    """Node features x [n, 32], directed edges (src, dst) and edge features e [n_edges, 4].

    x: (position - centroid) / L with L the largest half extent; wall, inflow and outlet flags (wall:
    node on a tag-0 face; inflow: node on an inflow cap and not on a wall; outlet: node on any other
    cap); the inflow profile at inflow nodes divided by its largest magnitude; the inflow waveform's
    real series divided by |a0|; zero padding.  Edges: both directions of every tetrahedron edge.
    e: (x_dst - x_src) / L and its length."""
    n = xyz.shape[0]
    c = xyz.mean(axis=0)
    L = float(np.max(0.5 * (xyz.max(axis=0) - xyz.min(axis=0))))
    L = L if L > 0 else 1.0
    wall = np.zeros(n, bool)
    wall[np.unique(faces[face_tag == 0].ravel())] = True
    inflow = np.zeros(n, bool)
    for t in inflow_tags:
        inflow[np.unique(faces[face_tag == t].ravel())] = True
    inflow &= ~wall
    outlet = np.zeros(n, bool)
    caps = (face_tag != 0) & ~np.isin(face_tag, list(inflow_tags))
    outlet[np.unique(faces[caps].ravel())] = True
    prof = np.where(inflow[:, None], profile, 0.0)
    pmax = float(np.max(np.linalg.norm(prof, axis=1)))
    pmax = pmax if pmax > 0 else 1.0
    x = np.zeros((n, F_IN))
    x[:, 0:3] = (xyz - c) / L
    x[:, 3] = wall
    x[:, 4] = inflow
    x[:, 5] = outlet
    x[:, 6:9] = prof / pmax
    a0 = abs(wave[0]) if abs(wave[0]) > 0 else 1.0
    m = min(len(wave), F_IN - 9)
    x[:, 9:9 + m] = np.asarray(wave[:m]) / a0
    pairs = np.array([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])
    ed = np.sort(tets[:, pairs].reshape(-1, 2), axis=1)
    ed = np.unique(ed, axis=0)
    src = np.concatenate([ed[:, 0], ed[:, 1]])
    dst = np.concatenate([ed[:, 1], ed[:, 0]])
    d = (xyz[dst] - xyz[src]) / L
    e = np.concatenate([d, np.linalg.norm(d, axis=1, keepdims=True)], axis=1)
    return x, src, dst, e


def normalise_target(harm, u_ref, p_ref, rho):
    """Velocity / u_ref; pressure (mean minus p_ref) / (rho u_ref^2); harm [n, 4, M] -> [n, 4 M]."""
    t = np.array(harm, dtype=np.float64, copy=True)
    t[:, :3] /= u_ref
    t[:, 3, 0] -= p_ref
    t[:, 3] /= rho * u_ref * u_ref
    return t.reshape(t.shape[0], -1)
