"""The synthetic workloads against the recipes they stand for (CPU):

* the vascular network: a 3-nearest-neighbour graph of 50 000 points pruned
  to degrees 1..4 (mostly 3 and 4, 85% of the vertices), one connected
  component, about 80 000 edges,
  lognormal lengths (median 50 um, sigma_log 0.6), Kirchhoff flows
  conserved at every interior vertex, drift = flow / area rescaled to median
  |u| = 1000 um/s, sigma = sqrt(2 D), jump weights proportional to the area
  at both ends, inlets reflecting and outlets absorbing, and a step of 10
  times the explicit one-cell finite-volume limit;
* the 16-edge Langevin star: lengths U[0.5, 2], V_e = a_e (x - c_e)^2 with
  a_e in [0.5, 4] and c_e on the edge, drift -V_e', sigma = sqrt 2, equal
  weights, reflecting leaves."""
import math

import numpy as np
import pytest

from paper_2512_02175_gb300 import workloads as W


@pytest.fixture(scope="module")
def vasc():
    pytest.importorskip("scipy")
    return W.vascular()


def test_vascular_topology(vasc):
    V, E = vasc["n_vertices"], len(vasc["src"])
    deg = np.bincount(np.concatenate([vasc["src"], vasc["dst"]]), minlength=V)
    assert deg.min() >= 1 and deg.max() <= 4
    frac = np.bincount(deg, minlength=5) / V
    assert frac[3] + frac[4] > 0.8 and frac[3] > 0.35
    assert 45_000 <= V <= 50_000 and 70_000 <= E <= 90_000
    # one connected component
    import scipy.sparse as sp
    import scipy.sparse.csgraph as csg
    A = sp.coo_matrix((np.ones(E), (vasc["src"], vasc["dst"])), shape=(V, V))
    assert csg.connected_components(A, directed=False)[0] == 1


def test_vascular_lengths_and_flow(vasc):
    L = vasc["length"]
    assert abs(np.median(L) / 50.0 - 1.0) < 0.02
    assert abs(np.std(np.log(L)) / 0.6 - 1.0) < 0.02
    V = vasc["n_vertices"]
    src, dst, Q = vasc["src"], vasc["dst"], vasc["flow"]
    net = np.zeros(V)
    np.add.at(net, src, -Q)
    np.add.at(net, dst, Q)
    deg = np.bincount(np.concatenate([src, dst]), minlength=V)
    interior = deg > 1
    scale = np.abs(Q).max()
    assert np.abs(net[interior]).max() <= 1e-9 * scale  # Kirchhoff
    u = vasc["c0"]
    assert abs(np.median(np.abs(u)) - 1000.0) < 1e-6 * 1000.0
    assert np.all(vasc["c1"] == 0.0)
    area = vasc["w_init"]
    assert np.array_equal(area, vasc["w_term"]) and np.all(area > 0)
    moving = Q != 0.0  # u = Q / A up to the one scale factor
    ratio = np.abs(u[moving]) * area[moving] / np.abs(Q[moving])
    assert np.allclose(ratio, np.median(ratio)) and np.all(u[~moving] == 0.0)


def test_vascular_boundary_and_step(vasc):
    V = vasc["n_vertices"]
    deg = np.bincount(np.concatenate([vasc["src"], vasc["dst"]]), minlength=V)
    kind = vasc["kind"]
    inlet, outlet = vasc["inlet"], vasc["outlet"]
    assert np.all(deg[inlet] == 1) and np.all(deg[outlet] == 1)
    assert len(inlet) + len(outlet) == int((deg == 1).sum()) and len(inlet) > 0
    assert np.all(kind[inlet] == 0) and np.all(kind[outlet] == 1)
    assert np.count_nonzero(kind) == len(outlet)
    # the flow enters the network at every inlet
    assert np.all(vasc["inflow"][inlet] > 0)
    D = vasc["D"]
    assert np.allclose(vasc["sigma"], math.sqrt(2.0 * D))
    L, u = vasc["length"], vasc["c0"]
    assert vasc["dt"] == pytest.approx(10.0 * np.min(1.0 / (np.abs(u) / L + 2.0 * D / L ** 2)),
                                       rel=1e-12)


def test_star_langevin():
    d = W.star_langevin(16)
    L, a, c = d["length"], d["potential_a"], d["potential_c"]
    assert len(L) == 16 and np.all((L >= 0.5) & (L <= 2.0))
    assert np.all((a >= 0.5) & (a <= 4.0)) and np.all((c >= 0.0) & (c <= L))
    # mu = -V' for V = a (x - c)^2, at a few points of every edge
    for xs in (0.0, 0.3, 1.0):
        x = xs * L
        assert np.allclose(d["c0"] + d["c1"] * x, -2.0 * a * (x - c))
    assert np.allclose(d["sigma"], math.sqrt(2.0))
    assert np.all(d["src"] == 0) and np.array_equal(d["dst"], np.arange(1, 17))
    assert np.all(d["w_init"] == 1.0) and np.all(d["w_term"] == 1.0)
    assert "kind" not in d or not np.any(d["kind"])


def test_batch_instances():
    """512 uneven instances: half stars of 3..64 edges, half random trees of
    100..10^4 edges (lognormal lengths, quadratic potentials), N from 2^12 to
    2^22, steps from 100 to 5000, dt = 1e-3, M = 16; the totals the batched
    benchmark reports."""
    insts = W.batch_instances(512)
    assert len(insts) == 512 and [it["instance"] for it in insts] == list(range(512))
    stars, trees = insts[0::2], insts[1::2]
    ks = [len(it["graph"]["src"]) for it in stars]
    es = [len(it["graph"]["src"]) for it in trees]
    assert min(ks) >= 3 and max(ks) <= 64 and len(set(ks)) > 30
    assert min(es) >= 100 and max(es) <= 10_000 and max(es) > 5_000
    for it in trees[:8]:
        g = it["graph"]
        assert len(g["src"]) == g["n_vertices"] - 1  # a tree
    n = np.array([it["n"] for it in insts])
    steps = np.array([it["steps"] for it in insts])
    assert n.min() >= 2**12 and n.max() <= 2**22
    assert steps.min() >= 100 and steps.max() <= 5000
    assert all(it["dt"] == 1e-3 and it["M"] == 16 for it in insts)
    assert int(n.sum()) == 326_674_086 and int((n * steps).sum()) == 889_336_178_611
