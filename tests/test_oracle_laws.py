"""Law-level pins of the oracle against what the paper and the mathematics fix.

* Corollary 1 / standard Brownian motion: on a star with mu = 0 a sub-step
  from the vertex never returns to it, so the exit frequencies equal b
  exactly at every dt (multinomial test), one split per vertex visit.
* Renewal recursion: for constant drift toward the vertex on semi-infinite
  edges the exit law of one step and its truncation probability follow from
  q_e(h) = P(|W| > |mu_e| sqrt(h) / sigma_e) and h' = h - sigma_e^2 W^2 /
  mu_e^2 (Algorithm 1's alpha); computed here by quadrature, independently.
* Theorem 1: P(crossings <= k) >= 1 - exp(-(k - gamma)^2 / (4k)).
* Corollary 1: the exit law tends to b as dt -> 0.
* Reflection principle: two edges with b = 1/2 are Brownian motion on a
  line; the first-hit fraction matches 2 Phi(-(x0 + beta sigma sqrt(dt)) /
  (sigma sqrt(T))) with the discrete-monitoring shift beta = -zeta(1/2) /
  sqrt(2 pi) (Broadie, Glasserman, Kou 1997), and edge occupancy is half of it.
* Stationary density on a star with quadratic potentials and unequal b:
  rho_e(x) proportional to b_e exp(-(V_e(x) - V_e(0)) / D) (zero flux per
  edge, rho_e(v) proportional to b_ve, the cross-sectional-area reading of
  the vertex condition); the O(sqrt(dt)) bias of the scheme is removed by
  Richardson extrapolation over two step sizes.
"""
import math

import numpy as np
from scipy import integrate, special, stats

from paper_2512_02175_gb300 import workloads as W

BETA_BGK = 0.5825971579390106  # -zeta(1/2) / sqrt(2 pi)


def _sim(oracle, d, edge, x, seed, dt, steps, M):
    g = oracle.Graph.from_desc(d)
    st = oracle.State(edge, x)
    cnt = oracle.Counters(g)
    oracle.simulate(g, st, cnt, seed=seed, instance=0, dt=dt, steps=steps, M=M)
    return g, st, cnt


def test_exit_law_equals_b_for_brownian_star(oracle):
    d = W.star_brownian(3)
    e, x = W.round_robin_uniform(d, 10_000, 11)
    g, st, cnt = _sim(oracle, d, e, x, 0, 1e-3, 1000, 8)
    off, se, send, T = g.slots()
    centre = cnt.exits[off[0]:off[1]].astype(float)
    n = centre.sum()
    assert n > 50_000
    assert stats.chisquare(centre).pvalue > 1e-4
    # every hit is followed by exactly one exit (mu = 0, |W| into the edge)
    assert cnt.exits.sum() == st.hits.sum()
    assert int(cnt.truncations[0]) == 0


def _exit_law_quadrature(mu, sigma, b, dt, M, ns=3000, nq=96):
    """P(the step ends inside edge i) for a particle that has just reached the
    vertex (edge drawn from b) with time dt left and at most M splits."""
    K = len(mu)
    s = np.linspace(0.0, math.sqrt(dt), ns + 1)  # grid uniform in sqrt(h)
    h = s * s
    xg, wg = np.polynomial.legendre.leggauss(nq)
    G_next = None
    for k in range(M - 1, -1, -1):
        G = np.zeros((K, ns + 1, K))
        for e in range(K):
            c = abs(mu[e]) * np.sqrt(h) / sigma[e]
            G[e, :, e] += special.erfc(c / math.sqrt(2.0))  # P(|W| > c)
            if k + 1 < M:
                w = 0.5 * c[:, None] * (xg[None, :] + 1.0)
                ww = 0.5 * c[:, None] * wg[None, :]
                hp = h[:, None] - (sigma[e] / mu[e]) ** 2 * w * w
                sp = np.sqrt(np.clip(hp, 0.0, None))
                mix = np.tensordot(b, G_next, axes=(0, 0))
                interp = np.stack([np.interp(sp, s, mix[:, i]) for i in range(K)], -1)
                phi = np.exp(-0.5 * w * w) / math.sqrt(2 * math.pi)
                G[e] += 2.0 * np.einsum("ij,ijk->ik", phi * ww, interp)
        G_next = G
    return np.tensordot(b, G_next[:, -1, :], axes=(0, 0))


def _one_step_from_vertex(oracle, mu, sigma, b, dt, M, n, seed):
    K = len(mu)
    d = W._desc(1, np.zeros(K, np.int32), np.full(K, -1), np.full(K, np.inf), mu, 0.0, sigma,
                b, 0.0)
    e0 = np.random.default_rng(seed).choice(K, n, p=b).astype(np.int32)
    g, st, cnt = _sim(oracle, d, e0, np.zeros(n), seed + 1, dt, 1, M)
    f = np.array([((st.edge == i) & (st.x > 0)).sum() for i in range(K)]) / n
    return f, st, cnt


def test_exit_law_matches_renewal_quadrature(oracle):
    K = 5
    mu = -10.0 * np.arange(1, K + 1)  # the paper's linear-potential drifts
    sigma = np.array([1.0, 0.8, 1.2, 1.0, 0.9])
    b = np.array([1, 2, 3, 2, 2.0])
    b /= b.sum()
    n = 400_000
    for dt, M in [(2e-4, 4), (1e-3, 6)]:
        p = _exit_law_quadrature(mu, sigma, b, dt, M)
        f, st, cnt = _one_step_from_vertex(oracle, mu, sigma, b, dt, M, n, 17)
        se = np.sqrt(p * (1 - p) / n)
        assert np.all(np.abs(f - p) < 4 * se + 1e-6), (f, p)
        p_trunc = 1 - p.sum()
        assert abs(cnt.truncations[0] / n - p_trunc) < 4 * math.sqrt(p_trunc / n) + 1e-6
        # exits are the counted events of the same law
        assert np.array_equal(cnt.exits.astype(np.int64),
                              np.round(f * n).astype(np.int64))


def test_theorem1_bound_on_crossings(oracle):
    K = 5
    mu = -10.0 * np.arange(1, K + 1)
    sigma = np.ones(K)
    b = np.full(K, 0.2)
    n = 100_000
    for dt in (4e-4, 2e-3):
        gamma = dt * np.max(mu ** 2 / sigma ** 2)
        f, st, cnt = _one_step_from_vertex(oracle, mu, sigma, b, dt, 64, n, 5)
        assert int(cnt.truncations[0]) == 0
        crossings = st.hits.astype(np.int64) + 1  # sub-steps from the vertex
        for k in range(1, 12):
            if k <= gamma:
                continue
            bound = 1 - math.exp(-(k - gamma) ** 2 / (4 * k))
            emp = (crossings <= k).mean()
            assert emp >= bound - 4 * math.sqrt(max(bound * (1 - bound), 1e-12) / n)


def test_exit_law_tends_to_b(oracle):
    K = 5
    mu = -10.0 * np.arange(1, K + 1)
    sigma = np.ones(K)
    b = np.array([0.1, 0.3, 0.2, 0.25, 0.15])
    errs = []
    for dt in (1e-3, 1e-4, 1e-5, 1e-6):
        p = _exit_law_quadrature(mu, sigma, b, dt, 8, ns=800, nq=48)
        errs.append(np.abs(p - b).max())
    # the deviation shrinks like sqrt(dt) (the chance of returning to the vertex)
    for e1, e2 in zip(errs, errs[1:]):
        assert e2 < 0.45 * e1
    assert errs[-1] < 3e-3
    n = 200_000
    f, _, _ = _one_step_from_vertex(oracle, mu, sigma, b, 1e-6, 8, n, 23)
    assert np.all(np.abs(f - b) < 4 * np.sqrt(b * (1 - b) / n) + errs[-1])


def test_reflection_principle_two_edge_star(oracle):
    d = W.line_as_star(10.0)
    n, dt, steps, x0 = 20_000, 1e-3, 1000, 1.0
    g, st, cnt = _sim(oracle, d, np.zeros(n, np.int32), np.full(n, x0), 3, dt, steps, 8)
    T = dt * steps
    p_hit = 2 * stats.norm.cdf(-(x0 + BETA_BGK * math.sqrt(dt)) / math.sqrt(T))
    fh = (st.first_hits > 0).mean()
    assert abs(fh - p_hit) < 4 * math.sqrt(p_hit * (1 - p_hit) / n)
    # after the first hit both edges are equally likely: occupancy of edge 1 = p_hit / 2
    e1 = (st.edge == 1).mean()
    assert abs(e1 - p_hit / 2) < 4 * math.sqrt(0.25 * p_hit / n)
    # continuous monitoring is further away than the shifted barrier
    assert abs(fh - 2 * stats.norm.cdf(-x0 / math.sqrt(T))) > abs(fh - p_hit) - 1e-12


def _langevin_star():
    L = np.array([0.6, 1.4, 0.9, 1.2])
    a = np.array([0.7, 1.8, 1.2, 0.5])
    c = np.array([0.2, 0.9, 0.1, 0.8]) * L
    b = np.array([1.0, 2.0, 3.0, 4.0])
    k = len(L)
    d = W._desc(k + 1, np.zeros(k, np.int32), np.arange(1, k + 1), L, 2 * a * c, -2 * a,
                math.sqrt(2.0), b, 1.0)
    m = np.array([b[e] * integrate.quad(
        lambda x: math.exp(-(a[e] * (x - c[e]) ** 2 - a[e] * c[e] ** 2)), 0, L[e])[0]
        for e in range(k)])
    return d, m / m.sum()


def test_stationary_masses_langevin_star(oracle):
    d, m = _langevin_star()
    n, T = 30_000, 4.0
    f = {}
    for dt in (8e-3, 2e-3):
        e, x = W.uniform_on_edges(d, n, 1)
        g, st, cnt = _sim(oracle, d, e, x, 4, dt, int(round(T / dt)), 16)
        f[dt] = np.bincount(st.edge, minlength=4) / n
    se = np.sqrt(m * (1 - m) / n)
    # O(sqrt(dt)) bias: Richardson extrapolation to dt = 0 (weights 2, -1)
    f0 = 2 * f[2e-3] - f[8e-3]
    assert np.all(np.abs(f0 - m) < 4 * math.sqrt(5) * se), (f0, m)
    # and the error shrinks with dt on the dominant edge
    assert abs(f[2e-3][1] - m[1]) < abs(f[8e-3][1] - m[1])
