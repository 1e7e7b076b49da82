"""Pins of the oracle's position-dependent diffusion sigma_e(x) = sigma_e +
sigma1_e x (the edge generator of Section 2.2 allows any C^1 sigma_e;
Algorithm 1 evaluates it at the sub-step's starting point, reading R15).

* One Euler-Maruyama step far from any vertex has mean mu_e(x) h and
  variance sigma_e(x)^2 h at three starting points (a slope measured from
  the wrong end, a multiplicative slope or sigma squared twice fail).
* The stationary density of dX = sigma(X) dW (Ito, zero flux) is
  proportional to 1 / sigma_e(x)^2; on two edges glued with b = 1/2 and the
  same sigma at the vertex it is continuous there, so the edge masses are
  int_0^1 dx / (1 + k_e x)^2 = 1 / (1 + k_e) normalised, and each bin's mass
  follows in closed form.  Particles start from that law and must stay in it
  (bins within 4 standard errors, masses within 3).
* Hand-worked steps with injected draws: an interior step, and a split
  whose quadratic uses sigma at the starting point, followed by the
  sub-step from the vertex with sigma at that end.
* Zero slope leaves every result unchanged (the stored golden values of the
  constant-sigma oracle are checked elsewhere; here a run with an explicit
  zero slope equals one without).
"""
import math

import numpy as np
import pytest

from paper_2512_02175_gb300 import workloads as W
from tests import oracle_pool


def test_step_moments_follow_sigma_at_start(oracle):
    L, c0, c1, s0, s1, h = 100.0, 0.3, -0.002, 0.5, 0.02, 0.01
    d = dict(n_vertices=2, src=np.array([0], np.int32), dst=np.array([1], np.int32),
             length=np.array([L]), c0=np.array([c0]), c1=np.array([c1]), sigma=np.array([s0]),
             w_init=np.array([1.0]), w_term=np.array([1.0]), sigma1=np.array([s1]))
    n = 40_000
    for x0 in (10.0, 40.0, 70.0):
        g = oracle.Graph.from_desc(d)
        st = oracle.State(np.zeros(n, np.int32), np.full(n, x0))
        cnt = oracle.Counters(g)
        oracle.simulate(g, st, cnt, seed=4, instance=0, dt=h, steps=1, M=8)
        dx = st.x - x0
        mu, sig = c0 + c1 * x0, s0 + s1 * x0
        assert abs(dx.mean() - mu * h) <= 4 * sig * math.sqrt(h / n)
        assert abs(dx.var() / (sig * sig * h) - 1.0) <= 4 * math.sqrt(2.0 / n)


def test_invalid_slope_rejected(oracle):
    d = W.line_affine_sigma((1.0, -1.5))  # sigma(1) = -0.5 on the second edge
    with pytest.raises(ValueError):
        oracle.Graph.from_desc(d)


def _stationary(slopes, bins):
    k = np.asarray(slopes)
    mass = 1.0 / (1.0 + k)  # int_0^1 (1 + k x)^-2 dx
    mass = mass / mass.sum()
    edges = np.linspace(0.0, 1.0, bins + 1)
    out = np.zeros((len(k), bins))
    for e in range(len(k)):
        F = (1.0 - 1.0 / (1.0 + k[e] * edges)) / k[e]  # int_0^x (1 + k t)^-2 dt
        out[e] = np.diff(F) / F[-1] * mass[e]
    return mass, out


def _sample(slopes, n, seed):
    k = np.asarray(slopes)
    mass, _ = _stationary(slopes, 1)
    r = np.random.Generator(np.random.PCG64(seed))
    e = r.choice(len(k), size=n, p=mass).astype(np.int32)
    u = r.uniform(0.0, 1.0, n)
    Fe = 1.0 / (1.0 + k[e])  # F(1) k = 1 - 1/(1 + k)... solve F(x) = u F(1)
    tot = (1.0 - Fe) / k[e]
    x = (1.0 / (1.0 - k[e] * u * tot) - 1.0) / k[e]
    return e, np.clip(x, 0.0, 1.0)


def test_stationary_density_inverse_sigma_squared(oracle):
    slopes, bins, n = (1.0, 0.5), 16, 1 << 16
    d = W.line_affine_sigma(slopes)
    e, x = _sample(slopes, n, 7)
    mass, pb = _stationary(slopes, bins)
    o = oracle_pool.run(d, e, x, seed=3, dt=1e-3, steps=2000, M=32, bins=bins)
    ph = o["hist"].reshape(2, bins) / n
    se = np.sqrt(pb * (1 - pb) / n)
    assert np.all(np.abs(ph - pb) <= 4 * se), (ph - pb) / se
    pm = ph.sum(1)
    assert np.all(np.abs(pm - mass) <= 3 * np.sqrt(mass * (1 - mass) / n)), (pm, mass)
    # the density is far from uniform: the test can tell 1/sigma^2 from 1/sigma
    assert pb[0, 0] / pb[0, -1] > 3.5


def test_injected_steps_with_affine_sigma(oracle):
    # edge 0: l = 2, mu = 0.3 - 0.1 x, sigma = 0.5 + 0.25 x; edge 1: l = 1,
    # mu = 0, sigma = 0.4 + 0.6 x; both start at vertex 0 (b: 1/2 each)
    d = dict(n_vertices=3, src=np.array([0, 0], np.int32), dst=np.array([1, 2], np.int32),
             length=np.array([2.0, 1.0]), c0=np.array([0.3, 0.0]), c1=np.array([-0.1, 0.0]),
             sigma=np.array([0.5, 0.4]), w_init=np.array([1.0, 1.0]), w_term=np.array([1.0, 1.0]),
             sigma1=np.array([0.25, 0.6]))
    g = oracle.Graph.from_desc(d)
    h = 0.04
    # interior: x = 1.2 -> 1.2 + 0.18 * 0.04 + 0.8 * 0.2 * 0.7
    r = oracle.em_step_injected(g, 0, 1.2, h, 8, [0.7], [])
    assert r["edge"] == 0 and r["splits"] == 0
    assert abs(r["x"] - 1.3192) <= 1e-15
    # split at the init end: x = 0.05, W = -2: a = 0.295 * 0.04 = 0.0118,
    # b = 0.5125 * 0.2 * -2 = -0.205; s = 2C / (-B + sqrt(B^2 - 4AC));
    # u = 2^31 + 5 picks the second slot (edge 1 at its init end); the rest
    # of the step from vertex 0 with |W| = 1.5 and sigma_1(0) = 0.4
    A, Bq, Cq = 0.0118, -0.205, 0.05
    s = 2 * Cq / (-Bq + math.sqrt(Bq * Bq - 4 * A * Cq))
    assert abs(s - 0.24742631) < 1e-8
    h2 = (1 - s * s) * h
    r = oracle.em_step_injected(g, 0, 0.05, h, 8, [-2.0, -1.5], [2**31 + 5])
    assert r["edge"] == 1 and r["splits"] == 1
    assert abs(r["x"] - 0.4 * math.sqrt(h2) * 1.5) <= 1e-15


def test_zero_slope_changes_nothing(oracle):
    d = W.star_langevin(4)
    e, x = W.uniform_on_edges(d, 500, 2)
    a = oracle_pool.run(d, e, x, seed=1, dt=1e-3, steps=300, M=16, bins=8)
    b = oracle_pool.run(dict(d, sigma1=np.zeros(4)), e, x, seed=1, dt=1e-3, steps=300, M=16, bins=8)
    for k in ("edge", "x", "hits", "n_draw"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["exits"], b["exits"]) and np.array_equal(a["hist"], b["hist"])
