"""Learned warm start: data generation from the method's own solves, training and evaluation.

Every step runs in libhbgls (solves, network forward/backward/Adam); this module only sequences the
calls.  The network is not part of the paper's method (Sec. 4 only suggests harmonic balance solutions
as machine-learning data).
"""
from __future__ import annotations

import time

import numpy as np

from paper_2411_14315_gb300 import hbgls
from paper_2411_14315_gb300 import workloads as W


def family(seeds, n_h=4):
    """Vessel-like pipes (one spec per seed), see workloads.vessel_spec."""
    return [W.vessel_spec(int(s), n_h=n_h) for s in seeds]


def coronary_family(seeds, n_tets=30_000, n_h=10):
    """Stenosed coronary-like tubes (workloads.coronary_spec: radius U(0.15, 0.25) cm, 30-70 % stenosis,
    Re 100, N = 2 n_h + 1), one per seed, at n_tets tetrahedra."""
    return [W.coronary_spec(n_tets=n_tets, n_h=n_h, seed=int(s)) for s in seeds]


def solve_opts(**kw):
    o = dict(precision=1, rtol=1e-10, max_steps=300)
    o.update(kw)
    return o


def generate(specs, accept=1e-3, **kw):
    """Solve each spec from the default initial state and keep those whose residual fell below
    `accept` x its initial value (the paper's own convergence criterion is 1e-3, Sec. 2.3);
    returns [(problem, harmonics, report)] and the number of rejected specs."""
    out, rejected = [], 0
    for s in specs:
        p = hbgls.Problem.from_spec(s)
        rep = p.solve(check=False, **solve_opts(**kw))
        if rep["status"] == 0 or rep["res_final"] <= accept * rep["res0"]:
            out.append((p, p.harmonics(), rep))
        else:
            rejected += 1
            p.close()
    return out, rejected


def pressure_scale(specs_data):
    """Pressure normalisation factor for the network: the RMS over the training data of the pressure
    harmonics relative to the mean outlet level, in units of rho U^2 (U the largest mean inlet speed)."""
    acc, cnt = 0.0, 0
    for p, h, _ in specs_data:
        info = p.info()
        pp = np.array(h[:, 3, :], copy=True)
        pp[:, 0] -= info["p_ref"]
        rho = float(p.rho)
        pp /= rho * info["u_ref"] ** 2
        acc += float(np.sum(pp ** 2))
        cnt += pp.size
    return float(np.sqrt(acc / max(cnt, 1)))


def train(net: hbgls.MPNN, data, steps: int, lr: float = 2e-3, lr_final: float = 1e-4, seed: int = 0):
    """Adam over the samples in random order with a geometric learning-rate decay; returns losses."""
    rng = np.random.default_rng(seed)
    losses = []
    for k in range(steps):
        p, h, _ = data[int(rng.integers(len(data)))]
        a = lr * (lr_final / lr) ** (k / max(1, steps - 1))
        losses.append(net.train_step(p, h, a))
    return losses


def evaluate(net: hbgls.MPNN, specs, correction: bool = False, **kw):
    """Cold (default initial state) and warm (network prediction) solves of each spec to the same
    absolute residual; with correction, also a solve from the default state that takes learned
    correction steps (use_learned = 2).  Returns per-case dictionaries."""
    res = []
    for s in specs:
        cold = hbgls.Problem.from_spec(s)
        t0 = time.perf_counter()
        rc = cold.solve(check=False, **solve_opts(**kw))
        tc = time.perf_counter() - t0
        warm = hbgls.Problem.from_spec(s)
        pred = net.predict(warm)                       # for the error figures only (not timed)
        t0 = time.perf_counter()
        net.warm_start(warm)                           # one network forward, then the solve
        rw = warm.solve(check=False, **solve_opts(r_ref=rc["res0"], **kw))
        tw = time.perf_counter() - t0
        hc = cold.harmonics()
        err_pred = float(np.linalg.norm(pred - hc) / np.linalg.norm(hc))
        err_pred_vel = float(np.linalg.norm(pred[:, :3] - hc[:, :3]) / np.linalg.norm(hc[:, :3]))
        yw = warm.instances()
        yc = cold.instances()
        case = dict(cold=rc, warm=rw, t_cold=tc, t_warm=tw, pred_rel_err=err_pred,
                    pred_rel_err_velocity=err_pred_vel,
                    warm_vs_cold=float(np.linalg.norm(yw - yc) / np.linalg.norm(yc)))
        if correction:
            corr = hbgls.Problem.from_spec(s)
            net.attach(corr)
            t0 = time.perf_counter()
            rk = corr.solve(check=False, **solve_opts(r_ref=rc["res0"], use_learned=2, **kw))
            case["correction"] = rk
            case["t_correction"] = time.perf_counter() - t0
            case["correction_vs_cold"] = float(np.linalg.norm(corr.instances() - yc) / np.linalg.norm(yc))
            corr.close()
        res.append(case)
        cold.close()
        warm.close()
    return res
