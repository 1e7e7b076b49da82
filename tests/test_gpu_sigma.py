"""Position-dependent diffusion sigma_e(x) = sigma_e + k_e x on the GPU
(mg_graph_desc.sigma_slope; the kVarSigma kernels) against the FP64 oracle.

* FP64: trajectory by trajectory on a 16-edge Langevin star with random
  slopes and on two edges glued at a vertex (edge ids, counters identical,
  positions within 1e-12).
* FP32-mixed and FP32: the stationary density 1/sigma_e(x)^2 of two edges
  with a common sigma at the vertex (zero drift, b = 1/2), 2^20 particles
  started from it, 8000 steps of 2.5e-4: the 32 bins pass a chi-square test
  against the closed form (p > 1e-3; the oracle, run on the same particles
  and streams, shows the same sample's fluctuations bin for bin), edge masses
  within 3 standard errors; against the oracle on the first 2^18 particles,
  per-edge occupancy within 3 standard errors and the coupled total-variation
  distance under a quarter of the independent-sample noise floor.
* A graph with constant diffusion run inside a batch that needs the
  position-dependent kernel gives the same bits as alone.
* Slopes that let sigma_e(x) reach zero are rejected.
"""
import numpy as np
import pytest

from paper_2512_02175_gb300 import workloads as W
from tests import oracle_pool
from tests.test_gpu_parity import assert_fp64_parity, gpu_run
from tests.test_oracle_sigma import _sample, _stationary

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2512_02175_gb300 import binding as B
    B.load()
    return B


def star16_sloped():
    d = W.star_langevin(16)
    r = np.random.Generator(np.random.PCG64(9))
    # sigma_e(x) = sqrt(2) + k_e x with k_e in [-0.5, 0.5] / L_e: stays in [0.9, 1.9]
    d["sigma1"] = r.uniform(-0.5, 0.5, 16) / d["length"]
    return d


@pytest.mark.parametrize("graph", ["star16", "line"])
def test_sigma_slope_fp64_trajectories(B, graph):
    d = star16_sloped() if graph == "star16" else W.line_affine_sigma((1.0, 0.5))
    n = 8192
    e, x = W.uniform_on_edges(d, n, 4)
    gs, gc, gh = gpu_run(B, d, e, x, seed=6, dt=1e-3, steps=600, M=16, prec=B.MG_FP64, bins=8)
    o = oracle_pool.run(d, e, x, seed=6, dt=1e-3, steps=600, M=16, bins=8)
    assert_fp64_parity(gs, gc, o, ghist=gh)
    assert gc["exits"].sum() > 0


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_sigma_slope_stationary_density(B, prec):
    import torch
    from scipy import stats
    slopes, bins, n = (1.0, 0.5), 16, 1 << 20
    d = W.line_affine_sigma(slopes)
    e, x = _sample(slopes, n, 7)
    mass, pb = _stationary(slopes, bins)
    P = {"mixed": B.MG_FP32_MIXED, "fp32": B.MG_FP32}[prec]

    def gpu_hist(k):
        g = B.Graph(d)
        p = B.Particles(g, e[:k], x[:k], seed=3, precision=P)
        h = torch.zeros(2 * bins, dtype=torch.int32, device="cuda")
        p.simulate(2.5e-4, 8000, 32, hist_bins=bins, hist_out=h)
        p.synchronize()
        p.close()
        g.close()
        return h.cpu().numpy().view(np.uint32).astype(np.int64)

    # against the closed form: chi-square over the 32 bins, edge masses at 3 SE
    counts = gpu_hist(n)
    ph = counts.reshape(2, bins) / n
    z = (ph - pb) / np.sqrt(pb * (1 - pb) / n)
    chi2 = stats.chisquare(counts, pb.reshape(-1) * n)
    pm = ph.sum(1)
    zm = (pm - mass) / np.sqrt(mass * (1 - mass) / n)
    # against the oracle on the first 2^18 particles (same streams: coupled)
    ns = 1 << 18
    o = oracle_pool.run(d, e[:ns], x[:ns], seed=3, dt=2.5e-4, steps=8000, M=32, bins=bins,
                        chunks=64, keep_state=False)
    hs = gpu_hist(ns)
    tv = 0.5 * np.abs(hs - o["hist"]).sum() / ns
    floor = np.sqrt(2 * bins / (np.pi * ns))
    po, pg = o["occupancy"] / ns, hs.reshape(2, bins).sum(1) / ns
    print(f"\nsigma slope {prec}: chi-square p {chi2.pvalue:.3f} (max |z| of a bin "
          f"{np.abs(z).max():.2f}), edge masses max |z| {np.abs(zm).max():.2f}; coupled TV vs "
          f"oracle {tv:.2e} (independent noise floor {floor:.1e})")
    assert chi2.pvalue > 1e-3, (chi2, z)
    assert np.all(np.abs(zm) <= 3), zm
    assert np.all(np.abs(pg - po) <= 3 * np.sqrt(po * (1 - po) / ns)), (pg, po)
    assert tv <= 0.25 * floor, (tv, floor)


def test_constant_sigma_in_sloped_batch_is_bit_identical(B):
    import torch
    dc = W.star_langevin(16)
    ds = star16_sloped()
    n = 4096
    ec, xc = W.uniform_on_edges(dc, n, 1)
    es, xs = W.uniform_on_edges(ds, n, 2)
    for P in (B.MG_FP64, B.MG_FP32_MIXED, B.MG_FP32):
        alone, _, _ = gpu_run(B, dc, ec, xc, seed=5, dt=1e-3, steps=300, M=16, prec=P)
        gc_, gs_ = B.Graph(dc), B.Graph(ds)
        pc = B.Particles(gc_, ec, xc, seed=5, instance=0, precision=P)
        ps = B.Particles(gs_, es, xs, seed=5, instance=1, precision=P)
        b = B.Batch()
        b.add(pc, 1e-3, 300, 16)
        b.add(ps, 1e-3, 300, 16)
        s = torch.cuda.Stream()
        b.run(use_graph=False, stream=s)
        s.synchronize()
        got = pc.state()
        for k in ("edge", "x", "n_draw", "hits", "first_hits", "flags"):
            assert np.array_equal(got[k], alone[k]), (P, k)
        b.close()
        pc.close()
        ps.close()
        gc_.close()
        gs_.close()


def test_sigma_slope_validation(B):
    d = W.line_affine_sigma((1.0, -1.5))  # sigma(1) = -0.5 on the second edge
    with pytest.raises(B.MGError) as ei:
        B.Graph(d)
    assert ei.value.status == B.MG_ERR_INVALID_ARG
    d = W.paper_star("linear", k=2)
    d["sigma1"] = np.array([0.1, -0.1])  # a negative slope on a semi-infinite edge
    with pytest.raises(B.MGError):
        B.Graph(d)
