"""Pins of the oracle's hitting-fraction root (the partial step of
Algorithms 1 and 2).

* numpy.roots (a library routine) on random crossing sub-steps: the oracle
  returns the first root in [0, 1].
* Algorithm 1's closed form for a sub-step that starts at the vertex:
  alpha = W^2 sigma^2 / (mu^2 h).
* Brownian motion (mu = 0): alpha = x^2 / (sigma^2 h W^2).
* Degenerate cases: no movement, tangency, rounding past the ends.
"""
import math

import numpy as np


def _first_root_in_unit(A, B, C):
    if A == 0.0:
        rts = [-C / B] if B != 0 else []
    else:
        rts = [r.real for r in np.roots([A, B, C]) if abs(r.imag) <= 1e-9 * max(1.0, abs(r))]
    rts = sorted(r for r in rts if -1e-12 <= r <= 1 + 1e-12)
    return rts[0] if rts else None


def test_root_matches_numpy_roots(oracle):
    rng = np.random.default_rng(7)
    n_checked = 0
    for _ in range(20000):
        A, B = rng.uniform(-3, 3, 2)
        C = rng.uniform(0, 2)
        if rng.random() < 0.1:
            A = 0.0
        if A + B + C > 0:  # the sub-step must end beyond the vertex
            continue
        ref = _first_root_in_unit(A, B, C)
        assert ref is not None
        s = oracle.root(A, B, C)
        assert abs(s - ref) <= 1e-10 * max(1.0, ref), (A, B, C, s, ref)
        n_checked += 1
    assert n_checked > 2000


def test_return_to_vertex_matches_algorithm1(oracle):
    # sub-step from the vertex into the edge (|W|) with drift back toward it
    rng = np.random.default_rng(8)
    for _ in range(2000):
        mu = -rng.uniform(0.5, 50)
        sigma = rng.uniform(0.2, 3)
        h = 10 ** rng.uniform(-5, -1)
        W = abs(rng.normal())
        A, B = mu * h, sigma * math.sqrt(h) * W
        if A + B > 0:
            continue  # no return within the sub-step
        alpha_alg1 = W * W * sigma * sigma / (mu * mu * h)
        s = oracle.root(A, B, 0.0)
        assert abs(s * s - alpha_alg1) <= 1e-12 * max(1.0, alpha_alg1)


def test_brownian_alpha(oracle):
    rng = np.random.default_rng(9)
    for _ in range(2000):
        x = rng.uniform(1e-4, 1)
        sigma = rng.uniform(0.2, 3)
        h = 10 ** rng.uniform(-5, -1)
        W = -rng.uniform(x / (sigma * math.sqrt(h)), 10 * x / (sigma * math.sqrt(h)))
        s = oracle.root(0.0, sigma * math.sqrt(h) * W, x)
        alpha = x * x / (sigma * sigma * h * W * W)
        assert abs(s * s - alpha) <= 1e-12 * max(1.0, alpha)


def test_degenerate_roots(oracle):
    assert oracle.root(0.0, 0.0, 0.0) == 0.0          # no movement
    assert oracle.root(-1.0, 0.0, 0.0) == 0.0         # from the vertex, W = 0
    assert oracle.root(0.0, -2.0, 0.0) == 0.0         # already at the vertex
    assert oracle.root(0.0, -1.0, 1.0) == 1.0         # lands exactly on it
    assert oracle.root(0.0, -0.5, 1.0) == 1.0         # rounding past the end: clamped
    assert oracle.root(1.0, -2.0, 1.0) == 1.0         # tangent double root at s = 1
    assert 0.0 <= oracle.root(1.0, 1e-300, 1e-300) <= 1.0
    # -s^2 + s/2 + 1/4 = 0: the positive root (1/2 + sqrt(5/4)) / 2
    assert abs(oracle.root(-1.0, 0.5, 0.25) - (0.5 + math.sqrt(1.25)) / 2) < 1e-15
