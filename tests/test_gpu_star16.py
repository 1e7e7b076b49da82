"""The benchmark's configuration -- the 16-edge Langevin star (lengths
U[0.5, 2], V_e = a_e (x - c_e)^2, sigma = sqrt(2), equal b, reflecting
leaves, M = 16) in FP32-mixed (and, for the first comparison, FP32) --
against the FP64 oracle itself and against its stationary density.

* Against the oracle at N = 2^24 (the benchmark's launch: 10^4 EM-Steps, the
  fused 32-bin histogram): per-edge occupancy and per-slot exit frequencies
  of the whole population within 3 standard errors of an oracle sample of
  2^18 particles (the first 2^18 ids, run for the same 10^4 steps; standard
  errors by batch means over 64 groups of particles, since a particle's
  exits are correlated in time), and the coupled total-variation distance
  between the histogram of those 2^18 particles on the GPU and the oracle's,
  printed beside the independent-sample noise floor sqrt(B / (pi N)).
* Coupled total variation at N = 2^24 over 1000 EM-Steps against the oracle
  run on all 2^24 particles: <= 1e-3.
* The stationary density.  On a tree with the standard gluing conditions
  the zero-flux density of the diffusion L_e f = mu_e f' + (sigma^2/2) f''
  with mu_e = -V_e' is rho_e(x) = K b_e exp(-(V_e(x) - V_e(0)) / D), D =
  sigma^2 / 2 (reading R11: rho_e(v) proportional to b_ve at the vertex,
  the "cross-sectional area" weighting of the paper's finite-volume
  appendix).  Particles start from that density (edge by mass, position by
  inverse CDF of the truncated Gaussian), 2^24 of them run 20 time units,
  and the occupancy averaged over the last 10 (100 snapshots,
  mg_simulate_sampled) is compared
  bin by bin with the exact bin masses (closed form, erf) along
  dt = 4e-3, 2e-3, 1e-3, 5e-4: the error must fall with dt.
"""
import math

import numpy as np
import pytest
from scipy.special import erf, erfinv

from paper_2512_02175_gb300 import workloads as W
from tests import oracle_pool

pytestmark = pytest.mark.gpu

E, BINS, DT, M = 16, 32, 1e-3, 16


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2512_02175_gb300 import binding as B
    B.load()
    return B


def gpu_hist(B, d, e, x, steps, prec=None, bins=BINS, dt=DT):
    import torch
    g = B.Graph(d)
    p = B.Particles(g, e, x, seed=0, precision=B.MG_FP32_MIXED if prec is None else prec)
    h = torch.zeros(E * bins, dtype=torch.int32, device="cuda")
    p.simulate(dt, steps, M, hist_bins=bins, hist_out=h)
    p.synchronize()
    cnt = p.counts()
    st = p.state()
    p.close()
    g.close()
    return h.cpu().numpy().view(np.uint32).astype(np.int64), cnt, st


def batch_se(parts, key, norm):
    """Standard error of a per-particle mean by batch means over the groups
    of particles the oracle ran (equal sizes): the spread of the groups'
    estimates / sqrt(groups)."""
    est = np.array([norm(q[key]) for q in parts])
    return est.std(axis=0, ddof=1) / math.sqrt(len(parts))


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_star16_full_size_against_oracle(B, prec):
    d = W.star_langevin(E)
    n = 1 << 24
    e, x = W.uniform_on_edges(d, n, 11)
    P = {"mixed": B.MG_FP32_MIXED, "fp32": B.MG_FP32}[prec]
    hist, cnt, st = gpu_hist(B, d, e, x, 10_000, prec=P)
    assert hist.sum() == n and cnt["particle_steps"] == n * 10_000
    ns = 1 << 18
    o = oracle_pool.run(d, e[:ns], x[:ns], seed=0, dt=DT, steps=10_000, M=M, bins=BINS,
                        chunks=64, keep_state=False)
    # per-edge occupancy: the population (2^24) against the oracle's sample
    pg = np.bincount(st["edge"], minlength=E) / n
    po = o["occupancy"] / ns
    se = np.sqrt(po * (1 - po) / ns + pg * (1 - pg) / n)
    z_occ = (pg - po) / se
    # exit frequencies per slot (16 at the centre, 16 at the leaves)
    fg = cnt["exits"] / cnt["exits"].sum()
    fo = o["exits"] / o["exits"].sum()
    se_f = batch_se(o["parts"], "exits", lambda v: v / v.sum())
    z_exit = (fg - fo) / np.maximum(se_f, 1e-300)
    # coupled histogram of the same 2^18 particles (the GPU result of a
    # particle does not depend on the set it runs in)
    hs, _, _ = gpu_hist(B, d, e[:ns], x[:ns], 10_000, prec=P)
    tv = 0.5 * np.abs(hs - o["hist"]).sum() / ns
    floor = math.sqrt(E * BINS / (math.pi * ns))
    print(f"\nstar16 2^24 x 10^4 {prec} vs oracle 2^18: max |z| occupancy "
          f"{np.abs(z_occ).max():.2f}, exits {np.abs(z_exit).max():.2f}; coupled TV of 2^18 "
          f"{tv:.2e} (independent noise floor {floor:.2e})")
    assert np.all(np.abs(z_occ) <= 3), z_occ
    assert np.all(np.abs(z_exit) <= 3), z_exit
    assert tv <= 0.25 * floor, (tv, floor)


def test_star16_coupled_tv_vs_oracle_full_n(B):
    """TV <= 1e-3 at N = 2^24 between the FP32-mixed histogram and the
    oracle's, both over all 2^24 particles (1000 EM-Steps; same random
    streams, so the two differ only where a binary32 rounding turned a
    branch)."""
    d = W.star_langevin(E)
    n = 1 << 24
    e, x = W.uniform_on_edges(d, n, 11)
    hist, cnt, _ = gpu_hist(B, d, e, x, 1000)
    o = oracle_pool.run(d, e, x, seed=0, dt=DT, steps=1000, M=M, bins=BINS, chunks=64,
                        keep_state=False)
    tv = 0.5 * np.abs(hist - o["hist"]).sum() / n
    floor = math.sqrt(E * BINS / (math.pi * n))
    print(f"\nstar16 2^24 x 1000: coupled TV vs oracle {tv:.2e} (independent noise floor "
          f"{floor:.2e})")
    assert tv <= 1e-3, tv
    assert cnt["truncations"] == o["truncations"] or abs(cnt["truncations"] - o["truncations"]) <= 3


# ------------------------------------------------------ stationary density

def stationary_law(d):
    """Edge masses and the per-edge truncated-Gaussian parameters of
    rho_e(x) = K b_e exp(-(V_e(x) - V_e(0)) / D) (equal b, D = 1)."""
    a, c, L = d["potential_a"], d["potential_c"], np.asarray(d["length"])
    D = d["sigma"][0] ** 2 / 2.0
    s = np.sqrt(a / D)  # exp(-a (x - c)^2 / D) = exp(-(s (x - c))^2)
    F = lambda e, y: math.sqrt(math.pi) / (2 * s[e]) * erf(s[e] * (y - c[e]))
    Z = np.array([math.exp(a[e] * c[e] ** 2 / D) * (F(e, L[e]) - F(e, 0.0)) for e in range(E)])
    return Z / Z.sum(), a, c, L, s, F


def sample_stationary(d, n, seed):
    mass, a, c, L, s, F = stationary_law(d)
    r = np.random.Generator(np.random.PCG64(seed))
    e = r.choice(E, size=n, p=mass).astype(np.int32)
    u = r.uniform(0.0, 1.0, n)
    lo = erf(s[e] * (0.0 - c[e]))
    hi = erf(s[e] * (L[e] - c[e]))
    x = c[e] + erfinv(lo + u * (hi - lo)) / s[e]
    return e, np.clip(x, 0.0, L[e])


def exact_bin_mass(d):
    mass, a, c, L, s, F = stationary_law(d)
    out = np.zeros((E, BINS))
    for e in range(E):
        xs = np.linspace(0.0, L[e], BINS + 1)
        cdf = np.array([F(e, y) for y in xs])
        out[e] = mass[e] * np.diff(cdf) / (cdf[-1] - cdf[0])
    return out


T_RUN, T_AVG, N_SNAP = 20.0, 10.0, 100


def stationary_error(B, n, dt, seed=3):
    import torch
    d = W.star_langevin(E)
    e, x = sample_stationary(d, n, seed)
    g = B.Graph(d)
    p = B.Particles(g, e, x, seed=seed, precision=B.MG_FP32_MIXED)
    h = torch.zeros(E * BINS, dtype=torch.int32, device="cuda")
    every = int(round(T_AVG / dt / N_SNAP))
    burn = int(round(T_RUN / dt)) - every * N_SNAP
    p.simulate(dt, burn, M)
    p.simulate_sampled(dt, every * N_SNAP, M, every, BINS, h)
    p.synchronize()
    c = p.counts()
    p.close()
    g.close()
    ph = h.cpu().numpy().view(np.uint32).astype(np.float64).reshape(E, BINS) / (n * N_SNAP)
    pe = exact_bin_mass(d)
    tv = 0.5 * np.abs(ph - pe).sum()
    mass_err = np.abs(ph.sum(1) - pe.sum(1)).max()
    return tv, mass_err, int(c["truncations"])


def test_star16_stationary_density_dt_sweep(B):
    n = 1 << 24
    rows = []
    for dt in (4e-3, 2e-3, 1e-3, 5e-4):
        tv, me, tr = stationary_error(B, n, dt)
        rows.append((dt, tv, me, tr))
    floor = math.sqrt(E * BINS / (math.pi * n * N_SNAP))
    print("\nstar16 stationary density, N = 2^24, T = 20, averaged over the last 10 "
          f"(noise floor of a TV from {N_SNAP} independent snapshots: {floor:.1e})")
    for dt, tv, me, tr in rows:
        print(f"  dt {dt:.0e}: TV {tv:.3e}  max |edge mass error| {me:.3e}  truncations {tr}")
    tvs = [r[1] for r in rows]
    assert all(a > b for a, b in zip(tvs, tvs[1:])), tvs
    assert tvs[-1] < 0.5 * tvs[0], tvs
    assert tvs[-1] < 3e-3, tvs
