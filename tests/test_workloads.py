"""Shapes of the seeded synthetic workloads (gate and parameter counts per recipe)."""
import numpy as np
import pytest

from paper_2009_02823_gb300 import workloads as W


@pytest.mark.parametrize("cfg,n,G,P,T", [(1, 10, 116, 80, 19), (2, 24, 1420, 960, 72),
                                         (3, 30, 745, 600, 200), (5, 26, 462, 936, 51)])
def test_counts(cfg, n, G, P, T):
    w = W.config(cfg)
    assert (w.n, w.n_gates, w.n_params, len(w.terms)) == (n, G, P, T)
    assert w.theta.shape == (P,)
    assert np.all((w.theta >= 0) & (w.theta < 2 * np.pi))
    # parameter indices follow gate order, each used once
    seen = [p for (_k, _a, _b, ps) in w.gates for p in ps if p >= 0]
    assert seen == list(range(P))


def test_seeded_reproducible():
    a, b = W.config(3), W.config(3)
    assert np.array_equal(a.theta, b.theta) and a.terms == b.terms


def test_random_pauli_recipe():
    w = W.config(3)
    ws = [len(ops) for _c, ops in w.terms]
    assert min(ws) >= 1 and max(ws) <= 4
    for _c, ops in w.terms:
        qs = [q for q, _l in ops]
        assert len(set(qs)) == len(qs)


def test_batched_recipe():
    ws = W.batched()
    assert len(ws) == 512
    assert {w.n for w in ws} <= set(range(12, 21))
    assert all(4 <= w.meta["layers"] <= 16 for w in ws)
    assert all(w.n_params == 2 * w.n * w.meta["layers"] for w in ws)
