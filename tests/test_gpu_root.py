"""The hitting fraction of a split on the GPU (mg_hit_root) against the
oracle's or_root, on the coefficients the binary32 modes form.

The partial sub-step of Algorithms 1 and 2 reaches the vertex after the
fraction alpha = s^2 of the time left, s the first root in [0, 1] of
A s^2 + B s + C = 0.  The kernels form A, B, C in binary32; the FP32-mixed
mode solves for s to binary64 accuracy (the precision stated for the hitting
fraction: a binary32 root refined by Newton steps whose residuals are carried
exactly in binary32 error-free arithmetic, summed in binary64), the FP32
mode in binary32.  Here:

* the FP64 mode's closed form equals or_root bit for bit (both compute the
  same binary64 operations, correctly rounded square root and quotient);
* the FP32-mixed root agrees with or_root to binary64 accuracy: within a
  few binary64 ulps scaled by the root's condition number
  (|A| s^2 + |B| s + |C|) / |2 A s + B|;
* the FP32 root is within binary32 accuracy, and the relative error of its
  alpha against the binary64 alpha is printed (the figure quoted for the
  FP32 mode).

Coefficients: sub-steps of the 16-edge Langevin star (dt = 1e-3) that end
beyond a vertex -- starting points within six diffusion lengths of either
end, the first sub-step of a step (h = dt) and sub-steps after a split
(h uniform in (0, dt], from the vertex with |W| into the edge) -- plus
generic triples (A, B uniform in [-3, 3], C in [0, 2], A + B + C <= 0).
"""
import math

import numpy as np
import pytest

from paper_2512_02175_gb300 import workloads as W

pytestmark = pytest.mark.gpu

F = np.float32


def star_split_coefficients(n, seed=5, dt=1e-3):
    """(A, B, C) in binary32 of sub-steps of the 16-edge star that end
    beyond a vertex, formed as the binary32 kernels form them."""
    d = W.star_langevin(16)
    rng = np.random.default_rng(seed)
    L = d["length"].astype(F)
    c0 = d["c0"].astype(F)
    c1 = d["c1"].astype(F)
    sig = d["sigma"].astype(F)
    out = []
    got = 0
    while got < n:
        m = 4 * n
        e = rng.integers(0, 16, m)
        at_vertex = rng.random(m) < 0.25
        h = np.where(at_vertex, rng.uniform(0, dt, m), dt).astype(F)
        S = (sig[e] * np.sqrt(h)).astype(F)
        near = (rng.uniform(0, 6, m).astype(F) * S).astype(F)
        init = rng.random(m) < 0.5
        xs = np.where(init, near, (L[e] - near).astype(F)).astype(F)
        xs = np.where(at_vertex, np.where(init, F(0), L[e]), xs).astype(F)
        z = rng.standard_normal(m).astype(F)
        z = np.where(at_vertex, np.where(init, np.abs(z), -np.abs(z)), z).astype(F)
        a = ((c0[e] + c1[e] * xs).astype(F) * h).astype(F)
        b = (S * z).astype(F)
        xt = (xs.astype(np.float64) + a + b)
        hit_init = xt <= 0
        hit = hit_init | (xt >= L[e])
        A = np.where(hit_init, a, -a).astype(F)
        Bc = np.where(hit_init, b, -b).astype(F)
        C = np.where(hit_init, xs, (L[e] - xs).astype(F)).astype(F)
        keep = hit & (C >= 0)
        out.append(np.stack([A[keep], Bc[keep], C[keep]], 1))
        got += int(keep.sum())
    return np.concatenate(out)[:n]


def generic_coefficients(n, seed=6):
    rng = np.random.default_rng(seed)
    A = rng.uniform(-3, 3, 4 * n).astype(F)
    A[rng.random(4 * n) < 0.1] = 0
    Bc = rng.uniform(-3, 3, 4 * n).astype(F)
    C = rng.uniform(0, 2, 4 * n).astype(F)
    keep = (A.astype(np.float64) + Bc + C) <= 0
    return np.stack([A[keep], Bc[keep], C[keep]], 1)[:n]


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2512_02175_gb300 import binding as B
    B.load()
    return B


def gpu_roots(B, mode, abc):
    import torch
    t = [torch.from_numpy(np.ascontiguousarray(abc[:, k])).cuda() for k in range(3)]
    s = torch.empty(len(abc), dtype=torch.float64, device="cuda")
    B.mg_hit_root(mode, t[0], t[1], t[2], s)
    torch.cuda.synchronize()
    return s.cpu().numpy()


def oracle_roots(oracle, abc):
    return np.array([oracle.root(float(a), float(b), float(c)) for a, b, c in abc])


def condition(abc, s):
    A, Bc, C = (abc[:, k].astype(np.float64) for k in range(3))
    scale = np.abs(A) * s * s + np.abs(Bc) * s + np.abs(C)
    slope = np.abs(2 * A * s + Bc)
    return scale, slope


@pytest.mark.parametrize("kind", ["star16", "generic"])
def test_hit_root_against_oracle(B, oracle, kind):
    abc = star_split_coefficients(60_000) if kind == "star16" else generic_coefficients(30_000)
    ref = oracle_roots(oracle, abc)
    assert np.all((ref >= 0) & (ref <= 1))
    # FP64: the same closed form in binary64, bit for bit
    s64 = gpu_roots(B, B.MG_FP64, abc)
    assert np.array_equal(s64, ref), np.flatnonzero(s64 != ref)[:5]
    # FP32-mixed: binary64 accuracy, within a few ulps scaled by the condition
    smx = gpu_roots(B, B.MG_FP32_MIXED, abc)
    scale, slope = condition(abc, ref)
    eps = 2.0 ** -52
    bound = 8 * eps * (ref + scale / np.maximum(slope, 1e-300))
    err = np.abs(smx - ref)
    bad = err > bound
    assert not bad.any(), (abc[bad][:3], smx[bad][:3], ref[bad][:3])
    well = slope > 1e-3 * scale  # well-conditioned roots: relative accuracy
    rel = err[well] / np.maximum(ref[well], 1e-300)
    assert rel.max() <= 64 * eps, rel.max()
    # FP32: binary32 accuracy; the error of its alpha against binary64
    s32 = gpu_roots(B, B.MG_FP32, abc)
    e32 = np.abs(s32 - ref)
    assert np.all(e32 <= 2e-5 * np.maximum(ref, 1e-3) + 64 * 2.0 ** -24 * scale / np.maximum(slope, 1e-30))
    pos = ref > 0
    ra = np.abs(s32[pos] ** 2 - ref[pos] ** 2) / ref[pos] ** 2
    print(f"\n{kind}: {len(abc)} splits; FP32-mixed root vs oracle max rel "
          f"{rel.max():.2e} (well-conditioned {well.mean():.4f}); binary32 alpha vs binary64 "
          f"alpha: max rel {ra.max():.2e}, mean {ra.mean():.2e}, median {np.median(ra):.2e}")


def test_hit_root_degenerate_cases(B, oracle):
    abc = np.array([
        [0.0, -1.0, 0.5],   # no drift: s = C / -B
        [0.0, 0.0, 0.0],    # no movement
        [1.0, -2.0, 1.0],   # double root at 1
        [-1.0, 0.0, 0.0],   # C = 0: root 0
        [0.5, -0.5, 1e-30], # tiny C
        [-2.0, 0.5, 0.25],  # drift toward the vertex, B > 0
        [1e-30, -1.0, 0.3],
    ], dtype=F)
    ref = oracle_roots(oracle, abc)
    for mode in (B.MG_FP64, B.MG_FP32_MIXED):
        s = gpu_roots(B, mode, abc)
        assert np.allclose(s, ref, rtol=1e-7, atol=1e-15), (mode, s, ref)
    assert np.array_equal(gpu_roots(B, B.MG_FP64, abc), ref)


def test_hit_root_rejects_bad_arguments(B):
    import torch
    a = torch.zeros(4, dtype=torch.float32, device="cuda")
    s = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(B.MGError):
        B.mg_hit_root(7, a, a, a, s)
    with pytest.raises(ValueError):
        B.mg_hit_root(B.MG_FP64, a, a, a, torch.zeros(3, dtype=torch.float64, device="cuda"))
