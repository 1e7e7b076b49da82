"""Pins of the oracle's histograms: the variable-width one against a
hand-worked case and against the uniform-width one, and both against the
count of living particles."""
import numpy as np

from paper_2512_02175_gb300 import workloads as W


def test_binned_histogram_hand_case(oracle):
    O = oracle
    # three edges: lengths 1, 2, 4; vertex 0 centre, 1..3 leaves
    d = W._desc(4, [0, 0, 0], [1, 2, 3], [1.0, 2.0, 4.0], 0.0, 0.0, 1.0, 1.0, 1.0)
    g = O.Graph.from_desc(d)
    # edge 0: bins [0,0.25) [0.25,0.5) [0.5,1]; edge 1: no bins;
    # edge 2: [0,3) [3,4]
    off = [0, 3, 3, 5]
    up = [0.25, 0.5, 1.0, 3.0, 4.0]
    e = np.array([0, 0, 0, 0, 0, 1, 2, 2, 2, -1, 0], np.int32)
    x = np.array([0.0, 0.25, 0.49, 0.5, 1.0, 1.5, 2.999, 3.0, 4.0, 0.3, 0.2499])
    h = O.histogram_binned(g, O.State(e, x), off, up)
    # x = 0.25 and 0.5 sit on inner boundaries and go up; 1.0 = the last
    # boundary stays in the last bin; edge 1 and the dead particle count nothing
    assert h.tolist() == [2, 2, 2, 1, 2]


def test_binned_histogram_reproduces_uniform_bins(oracle):
    O = oracle
    d = W.random_mixed(7)
    E = len(d["src"])
    # power-of-two ranges and bin counts: every boundary and every x * B /
    # range is exact, so both rules take the same decision
    rng = np.random.Generator(np.random.PCG64(5))
    ranges = 2.0 ** rng.integers(-2, 3, E)
    d = dict(d, hist_range=ranges)
    g = O.Graph.from_desc(d)
    e, x = W.uniform_on_edges(d, 20_000, 3)
    st = O.State(e, x)
    cnt = O.Counters(g)
    O.simulate(g, st, cnt, seed=1, instance=0, dt=2e-3, steps=40, M=8)
    B = 8
    uni = O.histogram(g, st, B)
    off = np.arange(E + 1, dtype=np.int32) * B
    up = np.concatenate([ranges[k] * np.arange(1, B + 1) / B for k in range(E)])
    var = O.histogram_binned(g, st, off, up)
    assert np.array_equal(uni, var)
    assert var.sum() == np.count_nonzero(st.edge >= 0)
