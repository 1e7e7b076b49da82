"""Brute-force pins of one EM-Step (Algorithms 1-2) with injected draws, the
orientation-flip symmetry, invariants, and bit-exact invariances.

Each case below is worked out by hand from the algorithm: the first normal W
and the hit draws (u_k, z_k) are injected, so every branch is hit on purpose
and the expected state is written down exactly.
"""
import math

import numpy as np
import pytest

from paper_2512_02175_gb300 import workloads as W

TWO32 = 2 ** 32


def _star(oracle, lengths=(1.0, 0.5, 2.0), c0=0.0, c1=0.0, sigma=1.0, w=None, kind=None):
    k = len(lengths)
    w = np.ones(k) if w is None else np.asarray(w, float)
    return oracle.Graph(k + 1, np.zeros(k, np.int32), np.arange(1, k + 1), lengths,
                        np.broadcast_to(c0, (k,)), np.broadcast_to(c1, (k,)),
                        np.broadcast_to(sigma, (k,)), w, np.ones(k), kind=kind)


def test_interior_step(oracle):
    g = _star(oracle)
    r = oracle.em_step_injected(g, 0, 0.5, 0.01, 8, [1.0], [])
    assert r["edge"] == 0 and r["x"] == 0.5 + math.sqrt(0.01)
    assert r["splits"] == 0 and r["hits"] == 0 and r["exits"].sum() == 0


def test_hit_centre_brownian(oracle):
    g = _star(oracle)
    off, se, send, T = g.slots()
    T0 = int(T[0])
    # x = 0.05, W = -1, h = 0.01: x~ = -0.05 -> alpha = 0.05^2/(0.01*1) = 0.25 -> h' = 0.0075
    for u, e_new in [(0, 0), (T0 - 1, 0), (T0, 1), (TWO32 - 1, 2)]:
        r = oracle.em_step_injected(g, 0, 0.05, 0.01, 8, [-1.0, -0.3], [u])
        assert r["edge"] == e_new
        # from the vertex the rest of the step goes into the edge with |z|
        assert abs(r["x"] - 0.3 * math.sqrt(0.0075)) < 1e-15
        assert r["hits"] == 1 and r["first_hits"] == 1 and r["splits"] == 1
        assert r["exits"][e_new] == 1 and r["exits"].sum() == 1  # slot j of vertex 0 is edge j


def test_hit_leaf_reflects(oracle):
    g = _star(oracle)
    # edge 0 has length 1; x = 0.95, W = +1, h = 0.01: leaf hit at alpha = 0.25
    r = oracle.em_step_injected(g, 0, 0.95, 0.01, 8, [1.0, 0.7], [12345])
    assert r["edge"] == 0
    assert abs(r["x"] - (1.0 - 0.7 * math.sqrt(0.0075))) < 1e-15
    off, se, send, T = g.slots()
    leaf_slot = off[1]
    assert r["exits"][leaf_slot] == 1


def test_drift_hit_init_end(oracle):
    # mu = -0.4, h = 0.25, x = 0.1, W = -0.3: 0.1 - 0.1 s^2 - 0.15 s = 0 at s = 1/2
    g = _star(oracle, lengths=(1.0, 1.0), c0=-0.4)
    r = oracle.em_step_injected(g, 0, 0.1, 0.25, 8, [-0.3, 1.0], [0])
    h2 = 0.25 * 0.75
    assert r["edge"] == 0
    assert abs(r["x"] - (-0.4 * h2 + math.sqrt(h2) * 1.0)) < 1e-14


def test_drift_hit_term_end_sign(oracle):
    # At the terminal end the increment enters with the opposite sign:
    # x = 0.9, mu = +0.4, h = 0.25, W = 0.3 on an edge of length 1:
    # (1 - 0.9) - 0.1 s^2 - 0.15 s = 0 at s = 1/2, alpha = 1/4.
    # (Solving with the unnegated increment has no root in (0,1].)
    g = _star(oracle, lengths=(1.0, 1.0), c0=0.4)
    r = oracle.em_step_injected(g, 0, 0.9, 0.25, 8, [0.3, 1.0], [0])
    h2 = 0.25 * 0.75
    assert r["edge"] == 0  # leaf: back onto edge 0 at its term end
    # from the term end into the edge: x = L + mu h2 - sqrt(h2) |z|
    assert abs(r["x"] - (1.0 + 0.4 * h2 - math.sqrt(h2) * 1.0)) < 1e-14


def test_return_to_vertex_then_exit(oracle):
    # at the centre on edge 0 with mu = -5, h = 0.01; |W| = 0.3:
    # x~ = -0.05 + 0.03 < 0 -> alpha = 0.09/(25*0.01) = 0.36 (Algorithm 1)
    g = _star(oracle, lengths=(1.0, 1.0), c0=-5.0)
    off, se, send, T = g.slots()
    r = oracle.em_step_injected(g, 0, 0.0, 0.01, 8, [-0.3, 2.0], [int(T[0])])
    h2 = 0.01 * (1 - 0.36)
    assert r["edge"] == 1
    assert abs(r["x"] - (-5.0 * h2 + math.sqrt(h2) * 2.0)) < 1e-14
    assert r["hits"] == 1 and r["first_hits"] == 0  # started at the vertex


def test_truncation_at_M(oracle):
    g = _star(oracle, lengths=(1.0, 1.0), c0=-5.0)
    off, se, send, T = g.slots()
    # M = 2: two returns to the vertex -> stop there on the second chosen edge
    r = oracle.em_step_injected(g, 0, 0.0, 0.01, 2, [0.3, 0.1], [0, int(T[0])])
    assert r["splits"] == 2 and r["truncations"] == 1
    assert r["edge"] == 1 and r["x"] == 0.0
    assert r["exits"].sum() == 0


def test_absorbing_vertex(oracle):
    g = _star(oracle, lengths=(1.0, 1.0), kind=[0, 1, 0])
    r = oracle.em_step_injected(g, 0, 0.99, 0.01, 8, [1.0], [0])
    assert r["edge"] == -1 and r["absorbed"][1] == 1 and r["hits"] == 1
    # a dead particle does not move
    r2 = oracle.em_step_injected(g, -1, 0.5, 0.01, 8, [1.0], [0])
    assert r2["edge"] == -1 and r2["x"] == 0.5 and r2["splits"] == 0


def test_semi_infinite_edge_never_hits_far_end(oracle):
    g = oracle.Graph(1, [0], [-1], [np.inf], [0.0], [0.0], [1.0], [1.0], [0.0])
    r = oracle.em_step_injected(g, 0, 1.0, 1.0, 8, [50.0], [])
    assert r["edge"] == 0 and r["x"] == 51.0


def test_exhaustive_one_step_enumeration(oracle):
    """All slot outcomes of one hit on the mixed graph: u at T_j - 1 and T_j."""
    d = W.random_mixed()
    g = oracle.Graph.from_desc(d)
    off, se, send, T = g.slots()
    L = d["length"]
    for e in range(len(L)):
        for side in (0, 1):
            if side == 1 and not np.isfinite(L[e]):
                continue
            v = d["src"][e] if side == 0 else d["dst"][e]
            if d["kind"][v] == 1:
                continue
            x0 = 0.01 if side == 0 else L[e] - 0.01
            Wn = -5.0 if side == 0 else 5.0
            for j in range(off[v], off[v + 1]):
                for u in (int(T[j]) - 1, int(T[j])):
                    if not (0 <= u < TWO32):
                        continue
                    exp_slot = g.choose_slot(v, u)
                    # independently: first slot with u < T
                    ref = next(s for s in range(off[v], off[v + 1]) if u < int(T[s]))
                    assert exp_slot == ref
                    r = oracle.em_step_injected(g, e, x0, 1e-4, 1, [Wn], [u])
                    assert r["edge"] == se[ref]
                    assert r["x"] == (0.0 if send[ref] == 0 else L[se[ref]])
                    assert r["truncations"] == 1


def _trajectory_with_injection(oracle, g, edge, x, seed, steps, dt, M, flip_edge=None,
                               length=None):
    """Step one particle with the Philox draws passed in through the
    injection hook; on ``flip_edge`` the normal of an interior sub-step is
    negated (the flipped frame)."""
    nd, hits, fh, fl = 0, 0, 0, 0
    out = []
    for t in range(steps):
        zs = [oracle.normal(seed, 0, 0, nd + i) for i in range(M + 1)]
        if flip_edge is not None and edge == flip_edge and 0.0 < x < length:
            zs[0] = -zs[0]
        us = [oracle.split_draw(seed, 0, 0, hits + j) for j in range(M)]
        r = oracle.em_step_injected(g, edge, x, dt, M, zs, us, nd, hits, fh, fl)
        edge, x, nd, hits = r["edge"], r["x"], r["n_draw"], r["hits"]
        fh, fl = r["first_hits"], r["flags"]
        out.append((edge, x))
    return out


def test_orientation_flip_mirrors_trajectories(oracle):
    """Reversing an edge (swap ends, c0 -> -(c0 + c1 L), x -> L - x, swap end
    weights) mirrors every trajectory when the interior normals on that edge
    are negated."""
    src, dst = [0, 1, 1], [1, 2, 3]
    L = [1.3, 0.7, 0.9]
    c0, c1 = [0.8, -0.5, 0.3], [-1.2, 0.4, -0.7]
    sig = [0.9, 1.1, 0.8]
    wi, wt = [1.0, 2.0, 1.5], [0.7, 1.0, 1.0]
    g = oracle.Graph(4, src, dst, L, c0, c1, sig, wi, wt)
    # flip edge 0: 1 -> 0
    c0f = [-(c0[0] + c1[0] * L[0])] + c0[1:]
    gf = oracle.Graph(4, [1, 1, 1], [0, 2, 3], L, c0f, c1, sig, [wt[0]] + wi[1:],
                      [wi[0]] + wt[1:])
    matched = 0
    for p in range(40):
        x0 = 0.1 + 0.02 * p
        a = _trajectory_with_injection(oracle, g, 0, x0, 100 + p, 150, 2e-3, 8)
        b = _trajectory_with_injection(oracle, gf, 0, L[0] - x0, 100 + p, 150, 2e-3, 8,
                                       flip_edge=0, length=L[0])
        ok = True
        for (ea, xa), (eb, xb) in zip(a, b):
            xm = L[0] - xb if eb == 0 else xb
            if ea != eb or abs(xa - xm) > 1e-9:
                ok = False
                break
        matched += ok
    assert matched >= 38


def _run(oracle, d, n, steps, dt, M, seed=1, pid=None, init=None):
    g = oracle.Graph.from_desc(d)
    e, x = init if init is not None else W.uniform_on_edges(d, n, 5)
    st = oracle.State(e, x, pid)
    cnt = oracle.Counters(g)
    oracle.simulate(g, st, cnt, seed=seed, instance=0, dt=dt, steps=steps, M=M)
    return g, st, cnt


def test_invariants_mixed_graph(oracle):
    d = W.random_mixed()
    n = 3000
    g, st, cnt = _run(oracle, d, n, 400, 2e-3, 6)
    alive = st.edge >= 0
    hist = oracle.histogram(g, st, 8)
    assert hist.sum() + cnt.absorbed.sum() == n          # mass conservation
    assert int(cnt.absorbed.sum()) == int((~alive).sum())
    L = d["length"][st.edge[alive]]
    assert np.all(st.x[alive] >= 0) and np.all(st.x[alive] <= L)
    assert np.all(st.first_hits <= st.hits)
    assert cnt.absorbed[:5].sum() == 0                  # only 5, 6 absorb
    assert cnt.exits.sum() > 0 and cnt.truncations[0] >= 0
    assert cnt.particle_steps[0] <= n * 400


def test_chunking_and_sharding_bit_exact(oracle):
    d = W.random_mixed(seed=11)
    n = 500
    init = W.uniform_on_edges(d, n, 9)
    g, a, ca = _run(oracle, d, n, 120, 3e-3, 5, init=init)
    # 4 chunks of 30 steps
    g2 = oracle.Graph.from_desc(d)
    b = oracle.State(*init)
    cb = oracle.Counters(g2)
    for c in range(4):
        oracle.simulate(g2, b, cb, seed=1, instance=0, dt=3e-3, steps=30, M=5)
    # 2 shards by particle id
    s1 = oracle.State(init[0][:200], init[1][:200], np.arange(200))
    s2 = oracle.State(init[0][200:], init[1][200:], np.arange(200, n))
    cs = oracle.Counters(g2)
    oracle.simulate(g2, s1, cs, seed=1, instance=0, dt=3e-3, steps=120, M=5)
    oracle.simulate(g2, s2, cs, seed=1, instance=0, dt=3e-3, steps=120, M=5)
    for other, co in [(b, cb)]:
        assert np.array_equal(a.edge, other.edge) and np.array_equal(a.x, other.x)
        assert np.array_equal(a.hits, other.hits) and np.array_equal(ca.exits, co.exits)
    assert np.array_equal(a.edge, np.concatenate([s1.edge, s2.edge]))
    assert np.array_equal(a.x, np.concatenate([s1.x, s2.x]))
    assert np.array_equal(ca.exits, cs.exits) and np.array_equal(ca.absorbed, cs.absorbed)
    assert ca.truncations[0] == cs.truncations[0] == cb.truncations[0]
