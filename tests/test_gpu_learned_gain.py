"""What the trained warm-start network gains over the method without it.

Trains the network on solves the method generates for seeded vessel-like pipes, then solves held-out
vessels from the default initial state (cold), from the network's prediction (warm), and from the
default state with learned correction steps, to the same absolute residual, and compares the outer
(pseudo-time / Newton) steps.  All three end at the same state.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_learned_warm_start_reduces_outer_steps():
    from paper_2411_14315_gb300 import hbgls
    from paper_2411_14315_gb300 import learned as LR
    train_specs = LR.family(range(5000, 5024))
    test_specs = LR.family(range(6000, 6006))
    data, rejected = LR.generate(train_specs)
    assert len(data) >= 20
    net = hbgls.MPNN(4, seed=1, p_scale=LR.pressure_scale(data))
    losses = LR.train(net, data, steps=6000, lr=3e-3, lr_final=3e-5)
    assert np.mean(losses[-100:]) < 0.05 * losses[0]
    ev = LR.evaluate(net, test_specs, correction=True)
    cold = sum(e["cold"]["steps"] for e in ev)
    warm = sum(e["warm"]["steps"] for e in ev)
    for e in ev:
        assert e["cold"]["status"] == 0 and e["warm"]["status"] == 0 and e["correction"]["status"] == 0
        assert e["warm_vs_cold"] < 1e-8
        assert e["correction_vs_cold"] < 1e-8
    print(f"outer steps cold {cold} warm {warm}; GMRES iterations cold "
          f"{sum(e['cold']['gmres_iters'] for e in ev)} warm {sum(e['warm']['gmres_iters'] for e in ev)}")
    assert warm < cold
    for p, _, _ in data:
        p.close()
