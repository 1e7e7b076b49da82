"""Pins of the oracle's graph tables: the incident-edge slots E(v) and the
integer jump thresholds that sample b_v (Definition 4).

The thresholds are checked against exact rational arithmetic
(fractions.Fraction): T_j differs from floor(2^32 C_j) by at most one unit,
so each slot's probability is b_vj within 2^-32.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2512_02175_gb300 import workloads as W

TWO32 = 2 ** 32


def _graph(oracle, V, src, dst, wi, wt, length=None, kind=None):
    E = len(src)
    if length is None:
        length = [1.0 if d >= 0 else np.inf for d in dst]
    return oracle.Graph(V, src, dst, length, [0.0] * E, [0.0] * E, [1.0] * E, wi, wt, kind=kind)


def test_slot_order_and_self_loop(oracle):
    # edges: 0:(0->1) 1:(1->1 self-loop) 2:(2->0) 3:(1->-1)
    g = _graph(oracle, 3, [0, 1, 2, 1], [1, 1, 0, -1], [1, 2, 3, 4], [5, 6, 7, 0],
               length=[1, 1, 1, np.inf])
    off, se, send, T = g.slots()
    assert list(off) == [0, 2, 6, 7]
    # vertex 0: e0 init, e2 term; vertex 1: e0 term, e1 init, e1 term, e3 init; vertex 2: e2 init
    assert list(se) == [0, 2, 0, 1, 1, 3, 2]
    assert list(send) == [0, 1, 1, 0, 1, 0, 0]


def test_thresholds_exact(oracle):
    rng = np.random.default_rng(3)
    for trial in range(200):
        k = int(rng.integers(1, 20))
        w = rng.integers(0, 50, k).astype(float)
        if trial % 3 == 0:
            w = rng.uniform(0, 1, k)
        if w.sum() == 0:
            w[0] = 1.0
        d = W.star_brownian(k)
        g = oracle.Graph(k + 1, d["src"], d["dst"], d["length"], d["c0"], d["c1"], d["sigma"],
                         w, np.ones(k))
        off, se, send, T = g.slots()
        Tv = [int(t) for t in T[off[0]:off[1]]]
        tot = sum(Fraction(x) for x in w)
        cum = Fraction(0)
        for j in range(k):
            cum += Fraction(w[j])
            exact = (cum / tot) * TWO32
            assert abs(Tv[j] - int(exact)) <= 1, (w, j)
        assert Tv[-1] == TWO32
        assert all(a <= b for a, b in zip(Tv, Tv[1:]))
        # leaves (degree 1) always return to their only slot
        for v in range(1, k + 1):
            assert int(T[off[v]]) == TWO32


def test_choice_rule_boundaries(oracle):
    w = [1.0, 0.0, 2.0, 1.0]
    d = W.star_brownian(4)
    g = oracle.Graph(5, d["src"], d["dst"], d["length"], d["c0"], d["c1"], d["sigma"], w,
                     np.ones(4))
    off, se, send, T = g.slots()
    Tv = [int(t) for t in T[off[0]:off[1]]]
    assert Tv == [TWO32 // 4, TWO32 // 4, 3 * TWO32 // 4, TWO32]
    assert g.choose_slot(0, 0) == 0
    assert g.choose_slot(0, Tv[0] - 1) == 0
    assert g.choose_slot(0, Tv[0]) == 2          # the zero-weight slot 1 is skipped
    assert g.choose_slot(0, Tv[2] - 1) == 2
    assert g.choose_slot(0, Tv[2]) == 3
    assert g.choose_slot(0, TWO32 - 1) == 3
    # leaf vertex 3 has one slot whatever u is
    assert g.choose_slot(3, 0) == off[3] and g.choose_slot(3, TWO32 - 1) == off[3]


@pytest.mark.parametrize("bad", [
    dict(src=[0], dst=[2]),                      # vertex out of range
    dict(length=[0.0]),                          # length <= 0
    dict(length=[np.nan]),
    dict(length=[np.inf]),                       # infinite length on a finite edge
    dict(sigma=[0.0]),                           # sigma <= 0
    dict(wi=[0.0], wt=[1.0]),                    # vertex 0 has total weight 0
    dict(wi=[-1.0]),                             # negative weight
])
def test_invalid_graphs_rejected(oracle, bad):
    args = dict(V=2, src=[0], dst=[1], length=[1.0], sigma=[1.0], wi=[1.0], wt=[1.0])
    args.update(bad)
    with pytest.raises(ValueError):
        oracle.Graph(args["V"], args["src"], args["dst"], args["length"], [0.0], [0.0],
                     args["sigma"], args["wi"], args["wt"])


def test_absorbing_vertex_needs_no_weights(oracle):
    g = oracle.Graph(2, [0], [1], [1.0], [0.0], [0.0], [1.0], [1.0], [0.0], kind=[0, 1])
    assert g.n_slots == 2
