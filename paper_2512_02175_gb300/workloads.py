"""Seeded synthetic inputs: metric graphs and initial particle states.

This module is shared by the CUDA path, the benchmark and the oracle tests.
It holds none of the method's arithmetic: it only draws graphs, edge
parameters and starting positions with ``numpy.random.Generator(PCG64)`` at
stated seeds.  A graph description is a dict with

    n_vertices             int
    src, dst               int32[E]  init / term vertex of each edge (dst = -1:
                                      semi-infinite edge, length = +inf)
    length                 float64[E]
    c0, c1                 float64[E] drift mu_e(x) = c0 + c1 x (x from e_init)
    sigma                  float64[E] diffusion, > 0
    w_init, w_term         float64[E] unnormalised jump weights b_ve per end
    hist_range (optional)  float64[E] histogram range (default: length)
    kind (optional)        uint8[V]   0 standard, 1 absorbing

Workloads (sizes as in the paper's experiments and the configurations the
benchmark measures):

* ``star_brownian``   3-edge star of unit edges, standard Brownian motion.
* ``star_langevin``   16-edge star, lengths U[0.5, 2], quadratic potentials
                       V_e = a_e (x - c_e)^2, a_e ~ U[0.5, 4], c_e ~ U[0, L_e],
                       sigma = sqrt(2), equal weights, reflecting leaves.
* ``paper_star``      the paper's 5-edge semi-infinite star with linear
                       (mu_i = -10 i) or quadratic (mu_i = -10 i x) drift.
* ``vascular``        random-geometric stand-in for the paper's cortical
                       vascular network (not available here): degree <= 4,
                       lognormal lengths and radii, Poiseuille flow from a
                       Kirchhoff pressure solve, drift u_e = Q_e / A_e,
                       absorbing outlets.
* ``random_tree`` / ``random_mixed``  small graphs that reach every branch of
                       the path (cycles, self-loops, semi-infinite edges,
                       absorbing vertices, zero jump weights).
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _desc(V, src, dst, length, c0, c1, sigma, w_init, w_term, hist_range=None, kind=None):
    E = len(src)
    d = dict(
        n_vertices=int(V),
        src=np.asarray(src, np.int32), dst=np.asarray(dst, np.int32),
        length=np.asarray(length, np.float64),
        c0=np.broadcast_to(np.asarray(c0, np.float64), (E,)).copy(),
        c1=np.broadcast_to(np.asarray(c1, np.float64), (E,)).copy(),
        sigma=np.broadcast_to(np.asarray(sigma, np.float64), (E,)).copy(),
        w_init=np.broadcast_to(np.asarray(w_init, np.float64), (E,)).copy(),
        w_term=np.broadcast_to(np.asarray(w_term, np.float64), (E,)).copy(),
    )
    if hist_range is not None:
        d["hist_range"] = np.asarray(hist_range, np.float64)
    if kind is not None:
        d["kind"] = np.asarray(kind, np.uint8)
    return d


# ------------------------------------------------------------------ graphs

def star_brownian(k: int = 3, length: float = 1.0, sigma: float = 1.0):
    """Star of k finite edges (centre 0 -> leaf i), mu = 0, equal weights."""
    src = np.zeros(k, np.int32)
    dst = np.arange(1, k + 1, dtype=np.int32)
    return _desc(k + 1, src, dst, np.full(k, length), 0.0, 0.0, sigma, 1.0, 1.0)


def star_langevin(k: int = 16, seed: int = 2, sigma: float = math.sqrt(2.0)):
    """Star of k finite edges with quadratic potentials V_e = a_e (x - c_e)^2:
    mu_e(x) = -V_e'(x) = 2 a_e c_e - 2 a_e x.  Reflecting leaves, equal b."""
    r = _rng(seed)
    L = r.uniform(0.5, 2.0, k)
    a = r.uniform(0.5, 4.0, k)
    c = r.uniform(0.0, 1.0, k) * L
    src = np.zeros(k, np.int32)
    dst = np.arange(1, k + 1, dtype=np.int32)
    d = _desc(k + 1, src, dst, L, 2.0 * a * c, -2.0 * a, sigma, 1.0, 1.0)
    d["potential_a"], d["potential_c"] = a, c
    return d


def paper_star(kind: str = "linear", k: int = 5, sigma: float = 1.0, hist_range=None):
    """The paper's star experiment: k semi-infinite edges, b = 1/k, drift
    mu_i = -10 i (linear potential) or mu_i = -10 i x (quadratic)."""
    i = np.arange(1, k + 1, dtype=np.float64)
    if kind == "linear":
        c0, c1 = -10.0 * i, 0.0
    elif kind == "quadratic":
        c0, c1 = 0.0, -10.0 * i
    else:
        raise ValueError(kind)
    hr = np.full(k, 1.0) if hist_range is None else np.broadcast_to(hist_range, (k,))
    return _desc(1, np.zeros(k, np.int32), np.full(k, -1, np.int32), np.full(k, np.inf),
                 c0, c1, sigma, 1.0, 0.0, hist_range=hr)


def line_as_star(half_length: float = 10.0, sigma: float = 1.0):
    """Two edges glued at vertex 0 with b = 1/2: Brownian motion on
    [-half_length, half_length] folded at 0 (reflecting far ends)."""
    return _desc(3, [0, 0], [1, 2], [half_length, half_length], 0.0, 0.0, sigma, 1.0, 1.0)


def line_affine_sigma(slopes=(1.0, 0.5), length: float = 1.0, sigma0: float = 1.0):
    """Two edges of length ``length`` glued at vertex 0 with b = 1/2, no
    drift, position-dependent diffusion sigma_e(x) = sigma0 + slopes[e] x
    (the same sigma0 at the shared vertex), reflecting far ends."""
    k = len(slopes)
    d = _desc(k + 1, np.zeros(k, np.int32), np.arange(1, k + 1, dtype=np.int32),
              np.full(k, length), 0.0, 0.0, sigma0, 1.0, 1.0)
    d["sigma1"] = np.asarray(slopes, np.float64)
    return d


def random_tree(n_edges: int, seed: int, sigma_range=(0.5, 1.5)):
    """Uniform random labelled tree (Pruefer sequence), lognormal lengths
    (median 1, sigma_log 0.5), quadratic potentials as in ``star_langevin``,
    random positive jump weights."""
    r = _rng(seed)
    n = n_edges + 1
    if n == 2:
        src, dst = np.array([0]), np.array([1])
    else:
        seq = r.integers(0, n, n - 2)
        degree = np.ones(n, np.int64)
        for s in seq:
            degree[s] += 1
        src, dst = [], []
        import heapq
        leaves = [i for i in range(n) if degree[i] == 1]
        heapq.heapify(leaves)
        for s in seq:
            leaf = heapq.heappop(leaves)
            src.append(int(s)); dst.append(leaf)
            degree[s] -= 1
            if degree[s] == 1:
                heapq.heappush(leaves, int(s))
        u, v = heapq.heappop(leaves), heapq.heappop(leaves)
        src.append(u); dst.append(v)
        src, dst = np.array(src), np.array(dst)
    E = n_edges
    L = np.exp(r.normal(0.0, 0.5, E))
    a = r.uniform(0.5, 4.0, E)
    c = r.uniform(0.0, 1.0, E) * L
    sig = r.uniform(*sigma_range, E)
    return _desc(n, src, dst, L, 2.0 * a * c, -2.0 * a, sig, r.uniform(0.2, 2.0, E),
                 r.uniform(0.2, 2.0, E))


def random_mixed(seed: int = 7):
    """A small graph that reaches every branch: a cycle, a self-loop, a
    semi-infinite edge, a zero jump weight, two absorbing vertices, affine
    drifts of both signs and per-edge sigma."""
    r = _rng(seed)
    # vertices 0..6; 5 and 6 absorbing
    src = np.array([0, 1, 2, 0, 3, 3, 4, 2, 1, 0], np.int32)
    dst = np.array([1, 2, 0, 3, 3, 4, 5, 6, -1, 4], np.int32)
    E = len(src)
    L = r.uniform(0.3, 1.5, E)
    L[dst == -1] = np.inf
    c0 = r.uniform(-2.0, 2.0, E)
    c1 = r.uniform(-1.5, 1.5, E)
    c1[dst == -1] = -abs(c1[dst == -1]) - 0.5  # confine the semi-infinite edge
    c0[dst == -1] = -1.0
    sig = r.uniform(0.4, 1.2, E)
    wi = r.uniform(0.2, 2.0, E)
    wt = r.uniform(0.2, 2.0, E)
    wi[3] = 0.0  # edge 3 is never entered from vertex 0
    kind = np.zeros(7, np.uint8)
    kind[5] = kind[6] = 1
    hr = np.where(np.isfinite(L), L, 3.0)
    return _desc(7, src, dst, L, c0, c1, sig, wi, wt, hist_range=hr, kind=kind)


def vascular(seed: int = 3, n_points: int = 50_000, knn: int = 3, max_degree: int = 4,
             length_median: float = 50.0, length_sigma_log: float = 0.6,
             radius_median: float = 5.0, radius_sigma_log: float = 0.3,
             u_median: float = 1000.0, D: float = 1000.0, cfl_factor: float = 10.0):
    """Synthetic vascular-like network (units: um, s).

    Points uniform in a unit cube; symmetric k-nearest-neighbour graph;
    degrees above ``max_degree`` pruned by dropping the geometrically longest
    edges; largest connected component kept.  Edge lengths and radii are
    lognormal and independent of the geometry.  Poiseuille conductance
    g = pi r^4 / (8 L); degree-1 vertices in the upper half (z > 1/2) are
    inlets (pressure U[60, 80], reflecting), the others outlets (pressure
    U[10, 20], absorbing).  A Kirchhoff solve gives the flows Q_e; the drift is
    u_e = Q_e / A_e, A_e = pi r^2, rescaled to median |u| = ``u_median``.
    sigma = sqrt(2 D); b_ve proportional to A_e at both ends.  The step is
    ``cfl_factor`` times the explicit finite-volume limit with one cell per
    edge, min_e 1 / (|u_e| / L_e + 2 D / L_e^2)."""
    import scipy.sparse as sp
    import scipy.sparse.csgraph as csg
    import scipy.sparse.linalg as spl
    from scipy.spatial import cKDTree

    r = _rng(seed)
    P = r.uniform(0.0, 1.0, (n_points, 3))
    _, nb = cKDTree(P).query(P, k=knn + 1)
    a = np.repeat(np.arange(n_points), knn)
    b = nb[:, 1:].reshape(-1)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    pairs = np.unique(lo.astype(np.int64) * n_points + hi)
    u_, v_ = pairs // n_points, pairs % n_points
    geo = np.linalg.norm(P[u_] - P[v_], axis=1)
    order = np.argsort(-geo, kind="stable")
    deg = np.bincount(np.concatenate([u_, v_]), minlength=n_points)
    keep = np.ones(len(u_), bool)
    for e in order:  # drop longest edges at over-full vertices
        if deg[u_[e]] > max_degree or deg[v_[e]] > max_degree:
            keep[e] = False
            deg[u_[e]] -= 1
            deg[v_[e]] -= 1
    u_, v_ = u_[keep], v_[keep]
    A = sp.coo_matrix((np.ones(len(u_)), (u_, v_)), shape=(n_points, n_points))
    _, lab = csg.connected_components(A, directed=False)
    big = np.argmax(np.bincount(lab))
    vmask = lab == big
    newid = -np.ones(n_points, np.int64)
    newid[vmask] = np.arange(vmask.sum())
    emask = vmask[u_] & vmask[v_]
    src, dst = newid[u_[emask]], newid[v_[emask]]
    V, E = int(vmask.sum()), int(emask.sum())
    z = P[vmask, 2]

    L = length_median * np.exp(length_sigma_log * r.normal(size=E))
    rad = radius_median * np.exp(radius_sigma_log * r.normal(size=E))
    g = math.pi * rad ** 4 / (8.0 * L)
    deg = np.bincount(np.concatenate([src, dst]), minlength=V)
    bnd = deg == 1
    high = bnd & (z > 0.5)
    p_fix = np.zeros(V)
    p_fix[high] = r.uniform(60.0, 80.0, high.sum())
    p_fix[bnd & ~high] = r.uniform(10.0, 20.0, (bnd & ~high).sum())
    # Kirchhoff: sum_e g_e (p_v - p_w) = 0 at interior vertices
    Lap = sp.coo_matrix((np.concatenate([g, g, -g, -g]),
                         (np.concatenate([src, dst, src, dst]),
                          np.concatenate([src, dst, dst, src]))), shape=(V, V)).tocsr()
    free = ~bnd
    rhs = -Lap[free][:, bnd] @ p_fix[bnd]
    p = p_fix.copy()
    p[free] = spl.spsolve(Lap[free][:, free].tocsc(), rhs)
    Q = g * (p[src] - p[dst])  # positive: flow from src to dst
    # boundary vertices by the solved flow: where it enters the network an
    # inlet (reflecting), where it leaves an outlet (absorbing) -- a
    # reflecting wall that the flow runs into would trap particles at it
    net_in = np.zeros(V)
    np.add.at(net_in, src, -Q)
    np.add.at(net_in, dst, Q)
    inlet = bnd & (net_in < 0)   # flow leaves the vertex into its edge
    outlet = bnd & ~inlet
    area = math.pi * rad ** 2
    u = Q / area
    u *= u_median / np.median(np.abs(u))
    sigma = math.sqrt(2.0 * D)
    dt = cfl_factor * float(np.min(1.0 / (np.abs(u) / L + 2.0 * D / L ** 2)))
    kind = outlet.astype(np.uint8)
    d = _desc(V, src, dst, L, u, 0.0, sigma, area, area, kind=kind)
    # inflow at inlets (flow entering the network through the inlet's edge)
    inflow = np.zeros(V)
    np.add.at(inflow, src, np.where(inlet[src], np.maximum(Q, 0.0), 0.0))
    np.add.at(inflow, dst, np.where(inlet[dst], np.maximum(-Q, 0.0), 0.0))
    d.update(dt=dt, D=D, inlet=np.flatnonzero(inlet), outlet=np.flatnonzero(outlet),
             inflow=inflow, pressure=p, flow=Q)
    return d


# -------------------------------------------------------- initial states

def uniform_on_edges(d, n: int, seed: int, by_length: bool = True):
    """n particles: edge ~ length-weighted (finite edges) or uniform, position
    uniform on [0, L_e) (on [0, hist_range) for semi-infinite edges)."""
    r = _rng(seed)
    L = np.asarray(d["length"])
    span = np.where(np.isfinite(L), L, d.get("hist_range", np.ones_like(L)))
    p = span / span.sum() if by_length else np.full(len(L), 1.0 / len(L))
    edge = r.choice(len(L), size=n, p=p).astype(np.int32)
    x = r.uniform(0.0, 1.0, n) * span[edge]
    return edge, x


def round_robin_uniform(d, n: int, seed: int):
    """Particle i on edge i mod E at a uniform position on [0, L_e)."""
    r = _rng(seed)
    E = len(d["src"])
    edge = (np.arange(n) % E).astype(np.int32)
    x = r.uniform(0.0, 1.0, n) * np.asarray(d["length"])[edge]
    return edge, x


def at_vertex(d, n: int, edge_ids, end: int = 0):
    """n particles at an end (0: init, 1: term) of the given edges, cycling."""
    edge_ids = np.asarray(edge_ids, np.int32)
    edge = edge_ids[np.arange(n) % len(edge_ids)]
    x = np.zeros(n) if end == 0 else np.asarray(d["length"])[edge].astype(np.float64)
    return edge, x


def inject_at_inlets(d, n: int, seed: int):
    """Tracer particles started at the inlet vertices of a ``vascular`` graph,
    in proportion to the inflow, at the inlet end of the inlet's edge."""
    r = _rng(seed)
    inl = d["inlet"]
    w = d["inflow"][inl]
    if w.sum() <= 0:
        w = np.ones(len(inl))
    v = r.choice(inl, size=n, p=w / w.sum())
    src, dst = d["src"], d["dst"]
    # each inlet has exactly one incident edge
    inc_edge = np.full(d["n_vertices"], -1, np.int64)
    inc_end = np.zeros(d["n_vertices"], np.int64)
    inc_edge[src] = np.arange(len(src)); inc_end[src] = 0
    term_mask = np.zeros(d["n_vertices"], bool)
    term_mask[dst] = True
    inc_edge[dst] = np.arange(len(dst)); inc_end[dst] = 1
    edge = inc_edge[v].astype(np.int32)
    x = np.where(inc_end[v] == 0, 0.0, np.asarray(d["length"])[edge])
    return edge, x.astype(np.float64)


def star_quadratic(k: int, seed: int):
    """Star of k edges, lognormal lengths (median 1, sigma_log 0.5), quadratic
    potentials as in ``star_langevin``, sigma = sqrt(2), equal b."""
    r = _rng(seed)
    L = np.exp(r.normal(0.0, 0.5, k))
    a = r.uniform(0.5, 4.0, k)
    c = r.uniform(0.0, 1.0, k) * L
    return _desc(k + 1, np.zeros(k, np.int32), np.arange(1, k + 1), L, 2.0 * a * c, -2.0 * a,
                 math.sqrt(2.0), 1.0, 1.0)


def batch_instances(n_inst: int = 512, seed: int = 4, n_scale: float = 1.0,
                    steps_scale: float = 1.0, max_tree_edges: int = 10_000):
    """Uneven instances for one batched launch: half stars with K ~ U{3..64}
    edges, half uniform random trees with E ~ log-U[100, max_tree_edges]; each
    with N ~ 2^U[12, 22] particles (times n_scale), steps ~ U{100..5000}
    (times steps_scale), dt = 1e-3, M = 16.  Returns a list of dicts with the
    graph description, n, steps, dt, M and a graph seed."""
    r = _rng(seed)
    out = []
    for i in range(n_inst):
        if i % 2 == 0:
            g = star_quadratic(int(r.integers(3, 65)), seed=1000 + i)
        else:
            E = int(round(math.exp(r.uniform(math.log(100), math.log(max_tree_edges)))))
            g = random_tree(E, seed=1000 + i)
        n = max(32, int(round(2.0 ** r.uniform(12, 22) * n_scale)))
        steps = max(1, int(round(r.integers(100, 5001) * steps_scale)))
        out.append(dict(graph=g, n=n, steps=steps, dt=1e-3, M=16, instance=i))
    return out


CONFIGS = {
    "star3_brownian": dict(graph=lambda: star_brownian(3), n=10_000, dt=1e-3, steps=1000, M=8,
                           bins=32, seed=0, init="round_robin"),
    "star16_langevin": dict(graph=lambda: star_langevin(16), n=1 << 24, dt=1e-3, steps=10_000,
                            M=16, bins=32, seed=0, init="uniform"),
    "vascular": dict(graph=lambda: vascular(), n=1 << 26, dt=None, steps=2000, M=32, bins=16,
                     seed=0, init="inlets"),
}


def initial_state(name: str, d, n: int | None = None, seed: int = 11):
    cfg = CONFIGS[name]
    n = cfg["n"] if n is None else n
    if cfg["init"] == "round_robin":
        return round_robin_uniform(d, n, seed)
    if cfg["init"] == "uniform":
        return uniform_on_edges(d, n, seed)
    return inject_at_inlets(d, n, seed)
