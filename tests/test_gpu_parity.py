"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
* FP64 mode: trajectory by trajectory -- edge ids, hit counters and exit /
  absorption / truncation counts identical; |x_gpu - x_oracle| <=
  1e-12 max(1, |x|); particles whose trajectory passed within 1e-9 of a
  branch (flag bit 0 on either side) are excluded, and counted.  The only
  allowed differences are the ulp-level results of log / sin / cos on the two
  sides (test_fp64_normals_match_oracle), which a 1e-9 branch margin cannot
  turn into a different decision.
* FP32-mixed mode: statistical -- per-edge occupancy and per-slot exit
  frequencies within 3 standard errors of the oracle's (same Philox streams),
  coupled final-edge agreement, and the histogram total-variation distance.
"""
import math

import numpy as np
import pytest

from paper_2512_02175_gb300 import workloads as W
from tests import oracle_pool

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2512_02175_gb300 import binding as B
    B.load()
    return B


def gpu_run(B, desc, edge, x, *, seed, dt, steps, M, prec, pid_base=0, instance=0, chunks=None,
            bins=0):
    g = B.Graph(desc)
    p = B.Particles(g, edge, x, pid_base=pid_base, seed=seed, instance=instance, precision=prec)
    for c in (chunks or [steps]):
        p.simulate(dt, c, M)
    p.synchronize()
    st = p.state()
    cnt = p.counts()
    hist = p.histogram(bins) if bins else None
    p.close()
    g.close()
    return st, cnt, hist


def assert_fp64_parity(gs, gc, o, *, max_flag_frac=0.01, ghist=None):
    flagged = ((gs["flags"] & 1) | (o["flags"] & 1)) != 0
    ok = ~flagged
    assert flagged.mean() <= max_flag_frac, flagged.mean()
    assert np.array_equal(gs["edge"][ok], o["edge"][ok])
    assert np.array_equal(gs["n_draw"][ok], o["n_draw"][ok])
    assert np.array_equal(gs["hits"][ok], o["hits"][ok])
    assert np.array_equal(gs["first_hits"][ok], o["first_hits"][ok])
    dx = np.abs(gs["x"][ok] - o["x"][ok])
    tol = REL * np.maximum(1.0, np.abs(o["x"][ok]))
    assert np.all(dx <= tol), (dx.max(), np.argmax(dx - tol))
    if not flagged.any():
        assert np.array_equal(gc["exits"], o["exits"])
        assert np.array_equal(gc["absorbed"], o["absorbed"])
        assert gc["truncations"] == o["truncations"]
        assert gc["particle_steps"] == o["particle_steps"]
        if ghist is not None:
            assert np.array_equal(ghist.astype(np.uint64), o["hist"])
    else:
        slack = int(gs["hits"][flagged].sum() + o["hits"][flagged].sum()) + int(flagged.sum())
        assert np.abs(gc["exits"].astype(np.int64) - o["exits"].astype(np.int64)).sum() <= 2 * slack
    return int(flagged.sum())


# ------------------------------------------------------------ FP64 parity

def test_star3_brownian_fp64_trajectories(B):
    """The 3-edge Brownian star in full: N = 10^4, 1000 steps, M = 8."""
    d = W.star_brownian(3)
    e, x = W.round_robin_uniform(d, 10_000, 11)
    gs, gc, gh = gpu_run(B, d, e, x, seed=0, dt=1e-3, steps=1000, M=8, prec=B.MG_FP64, bins=32)
    o = oracle_pool.run(d, e, x, seed=0, dt=1e-3, steps=1000, M=8, bins=32)
    assert_fp64_parity(gs, gc, o, ghist=gh)
    assert gc["exits"].sum() > 100_000


def test_star3_fp64_matches_golden_values(B):
    """The FP64 kernel against the stored oracle values of tests/golden/
    (the 3-edge Brownian star, 48 particles, 400 steps): same edges, draw and
    hit counters, histogram and exit counts; positions within 1e-12."""
    import json
    import os
    from tests.golden import make_golden
    with open(os.path.join(os.path.dirname(__file__), "golden", "star3_brownian.json")) as f:
        gold = json.load(f)
    c = gold["case"]
    e, x = make_golden.initial(c["n"])
    g = B.Graph(make_golden.star3())
    p = B.Particles(g, e, x, seed=c["seed"], instance=c["instance"], precision=B.MG_FP64)
    p.simulate(c["dt"], c["steps"], c["M"])
    p.synchronize()
    st, cn = p.state(), p.counts()
    hist = p.histogram(c["bins"])
    p.close()
    g.close()
    assert not np.any(st["flags"] & 1)
    assert st["edge"].tolist() == gold["edge"]
    assert st["n_draw"].tolist() == gold["n_draw"]
    assert st["hits"].tolist() == gold["hits"]
    assert st["first_hits"].tolist() == gold["first_hits"]
    xg = np.array([float.fromhex(v) for v in gold["x"]])
    assert np.max(np.abs(st["x"] - xg)) <= 1e-12
    assert hist.tolist() == gold["histogram"]
    assert cn["exits"].tolist() == gold["exits"]
    assert cn["particle_steps"] == gold["particle_steps"]



def test_fp64_normals_match_oracle(B):
    """The binary64 mode's normals against the oracle's (both Box-Muller in
    binary64: the kernel's correctly rounded logarithm of its uniforms and
    CUDA's sqrt / sin / cos, the host's libm): four drift-free steps of length h
    from x0 = 1/2 on long edges move a particle by
    sigma sqrt(h) (z0 + z1 + z2 + z3), so the position difference bounds the
    normals' difference.  262 144 particles, 2^20 normals covering all four
    words of a Philox block: every position within 1e-15, i.e. the normals
    agree to a few ulps -- the accuracy the 1e-12 trajectory bound needs, as
    a near-grazing split (time left a few 1e-9 dt) amplifies a normal's
    error by up to ~1e4.  The largest difference is printed."""
    d = W.star_brownian(3, length=1000.0)  # mu = 0, sigma = 1
    n, dt, steps = 1 << 18, 2.5e-3, 4
    e = (np.arange(n) % 3).astype(np.int32)
    x = np.full(n, 0.5)
    gs, gc, _ = gpu_run(B, d, e, x, seed=9, dt=dt, steps=steps, M=8, prec=B.MG_FP64)
    o = oracle_pool.run(d, e, x, seed=9, dt=dt, steps=steps, M=8)
    ok = (gs["hits"] == 0) & (o["hits"] == 0)
    assert ok.mean() > 0.999
    assert np.array_equal(gs["n_draw"], o["n_draw"]) and int(gs["n_draw"][0]) == steps
    dx = np.abs(gs["x"][ok] - o["x"][ok])
    disp = np.abs(o["x"][ok] - 0.5).max()
    print(f"\nmax |x_gpu - x_oracle| after {steps} steps: {dx.max():.2e} "
          f"(largest displacement {disp:.3f})")
    assert dx.max() <= 1e-15

def test_mixed_graph_fp64_unaligned_chunks(B):
    """Cycles, a self-loop, a semi-infinite edge, zero weights, absorbing
    vertices, a small split cap (truncations), ids offset, steps in chunks
    that start off a multiple of four."""
    d = W.random_mixed(7)
    e, x = W.uniform_on_edges(d, 4096, 3)
    x[:64] = 0.0  # start at init vertices
    kw = dict(seed=5, dt=5e-3, steps=300, M=3, pid_base=1000, instance=3)
    gs, gc, gh = gpu_run(B, d, e, x, prec=B.MG_FP64, chunks=[7, 1, 290, 2], bins=8, **kw)
    o = oracle_pool.run(d, e, x, np.arange(1000, 1000 + 4096), seed=5, instance=3, dt=5e-3,
                        steps=300, M=3, bins=8)
    assert_fp64_parity(gs, gc, o, ghist=gh)
    assert gc["truncations"] > 0 and gc["absorbed"].sum() > 0


def test_random_tree_fp64_from_vertices(B):
    d = W.random_tree(300, seed=4)
    e, x = W.uniform_on_edges(d, 8192, 8)
    x[::5] = 0.0
    x[1::5] = d["length"][e[1::5]]  # start at term vertices
    gs, gc, gh = gpu_run(B, d, e, x, seed=9, dt=2e-3, steps=200, M=16, prec=B.MG_FP64, bins=4)
    o = oracle_pool.run(d, e, x, seed=9, dt=2e-3, steps=200, M=16, bins=4)
    assert_fp64_parity(gs, gc, o, ghist=gh)


def test_large_graph_global_tables_fp64(B):
    """A graph too large for shared-memory staging: tables read through L2,
    counters with global atomics."""
    d = W.random_tree(6000, seed=12)
    e, x = W.uniform_on_edges(d, 8192, 2)
    gs, gc, gh = gpu_run(B, d, e, x, seed=1, dt=4e-3, steps=150, M=8, prec=B.MG_FP64, bins=2)
    o = oracle_pool.run(d, e, x, seed=1, dt=4e-3, steps=150, M=8, bins=2)
    assert_fp64_parity(gs, gc, o, ghist=gh)


def test_paper_star_semi_infinite_fp64(B):
    """The paper's 5-edge semi-infinite star, linear potential mu_i = -10 i."""
    d = W.paper_star("linear")
    n = 4096
    e = (np.arange(n) % 5).astype(np.int32)
    x = np.random.default_rng(0).exponential(0.05, n)
    gs, gc, gh = gpu_run(B, d, e, x, seed=3, dt=1e-4, steps=500, M=16, prec=B.MG_FP64, bins=16)
    o = oracle_pool.run(d, e, x, seed=3, dt=1e-4, steps=500, M=16, bins=16)
    assert_fp64_parity(gs, gc, o, ghist=gh)


def test_edge_cases_fp64(B):
    d = W.star_brownian(3)
    # one particle; zero steps leaves it untouched
    gs, gc, _ = gpu_run(B, d, [1], [0.25], seed=0, dt=1e-3, steps=0, M=8, prec=B.MG_FP64)
    assert gs["edge"][0] == 1 and gs["x"][0] == 0.25 and gc["particle_steps"] == 0
    o = oracle_pool.run(d, [1], [0.25], seed=0, dt=1e-3, steps=57, M=8)
    gs, gc, _ = gpu_run(B, d, [1], [0.25], seed=0, dt=1e-3, steps=57, M=8, prec=B.MG_FP64)
    assert_fp64_parity(gs, gc, o)
    # M = 1 with steps far larger than the edges: truncation on nearly every step
    e, x = W.round_robin_uniform(d, 999, 1)
    o = oracle_pool.run(d, e, x, seed=2, dt=0.5, steps=40, M=1)
    gs, gc, _ = gpu_run(B, d, e, x, seed=2, dt=0.5, steps=40, M=1, prec=B.MG_FP64)
    assert_fp64_parity(gs, gc, o)
    assert gc["truncations"] > 999 * 10
    # every particle absorbed
    da = dict(d, kind=np.array([0, 1, 1, 1], np.uint8))
    o = oracle_pool.run(da, e, x, seed=2, dt=0.05, steps=400, M=32)
    gs, gc, _ = gpu_run(B, da, e, x, seed=2, dt=0.05, steps=400, M=32, prec=B.MG_FP64, bins=4)
    assert_fp64_parity(gs, gc, o)
    assert np.all(gs["edge"] == -1) and gc["absorbed"].sum() == 999


def test_largest_particle_ids_fp64(B):
    """Particle ids at the top of the 32-bit range (pid_base + n = 2^32): the
    random streams are keyed by the global id, so these particles follow the
    oracle's trajectories like any others (FP64), and in the binary32 modes
    equal the same particles inside a larger set; a set whose ids would wrap
    is rejected."""
    d = W.random_mixed(7)
    e, x = W.uniform_on_edges(d, 4096, 9)
    base = (1 << 32) - 4096
    pid = np.arange(base, base + 4096, dtype=np.uint64).astype(np.uint32)
    o = oracle_pool.run(d, e, x, pid, seed=11, dt=2e-3, steps=150, M=8)
    gs, gc, _ = gpu_run(B, d, e, x, seed=11, dt=2e-3, steps=150, M=8, prec=B.MG_FP64,
                        pid_base=base)
    assert_fp64_parity(gs, gc, o)
    # binary32 modes: the same particles alone at the top ids and as the upper
    # half of a set starting 4096 ids lower give bit-identical results
    e2 = np.concatenate([e, e])
    x2 = np.concatenate([x, x])
    for prec in (B.MG_FP32_MIXED, B.MG_FP32):
        a, _, _ = gpu_run(B, d, e, x, seed=11, dt=2e-3, steps=150, M=8, prec=prec, pid_base=base)
        b, _, _ = gpu_run(B, d, e2, x2, seed=11, dt=2e-3, steps=150, M=8, prec=prec,
                          pid_base=base - 4096)
        for k in ("edge", "x", "n_draw", "hits", "first_hits", "flags"):
            assert np.array_equal(a[k], b[k][4096:]), k
    g = B.Graph(d)
    with pytest.raises(B.MGError) as ei:
        B.Particles(g, e, x, pid_base=base + 1, seed=11)
    assert ei.value.status == B.MG_ERR_INVALID_ARG
    g.close()


# ------------------------------------------------------------ invariances

MODES = {"fp64": 0, "mixed": 1, "fp32": 2}


@pytest.mark.parametrize("prec", list(MODES))
def test_chunking_sharding_resume_bit_exact(B, prec):
    P = MODES[prec]
    d = W.random_mixed(3)
    n = 6000
    e, x = W.uniform_on_edges(d, n, 4)
    kw = dict(seed=77, dt=3e-3, M=6, prec=P)
    a, ca, ha = gpu_run(B, d, e, x, steps=600, bins=8, **kw)
    b, cb, hb = gpu_run(B, d, e, x, steps=600, chunks=[200, 200, 200], bins=8, **kw)
    c, cc, hc = gpu_run(B, d, e, x, steps=600, chunks=[1, 598, 1], bins=8, **kw)
    for other, co, ho in [(b, cb, hb), (c, cc, hc)]:
        for k in ("edge", "x", "n_draw", "hits", "first_hits", "flags"):
            assert np.array_equal(a[k], other[k]), k
        for k in ("exits", "absorbed"):
            assert np.array_equal(ca[k], co[k])
        assert ca["truncations"] == co["truncations"]
        assert ca["particle_steps"] == co["particle_steps"]
        assert np.array_equal(ha, ho)
    # two shards by particle id sum to the whole
    s1, c1, h1 = gpu_run(B, d, e[:2500], x[:2500], steps=600, bins=8, **kw)
    s2, c2, h2 = gpu_run(B, d, e[2500:], x[2500:], steps=600, pid_base=2500, bins=8, **kw)
    assert np.array_equal(a["x"], np.concatenate([s1["x"], s2["x"]]))
    assert np.array_equal(ca["exits"], c1["exits"] + c2["exits"])
    assert np.array_equal(ha, h1 + h2)
    # checkpoint after 250 steps, resume in a fresh set
    g = B.Graph(d)
    p = B.Particles(g, e, x, seed=77, precision=P)
    p.simulate(3e-3, 250, 6)
    ck = p.state()
    q = B.Particles(g, e, x, seed=77, precision=P)
    q.set_state(ck)
    q.simulate(3e-3, 350, 6)
    r = q.state()
    assert r["step"] == 600
    for k in ("edge", "x", "n_draw", "hits", "first_hits", "flags"):
        assert np.array_equal(a[k], r[k]), k
    p.close(); q.close(); g.close()


@pytest.mark.parametrize("prec", list(MODES))
def test_split_batching_does_not_change_results(B, prec):
    """How many pending vertex hits a warp collects before resolving them is
    a launch choice: every setting gives bit-identical results."""
    d = W.star_langevin(16)
    e, x = W.uniform_on_edges(d, 20_000, 2)
    g = B.Graph(d)
    outs = []
    for sb in (1, 5, 32):
        p = B.Particles(g, e, x, seed=3, precision=MODES[prec])
        p.set_tuning(split_batch=sb)
        p.simulate(2e-3, 300, 16)
        p.synchronize()
        outs.append((p.state(), p.counts()))
        p.close()
    g.close()
    for st, cn in outs[1:]:
        for k in ("edge", "x", "n_draw", "hits", "first_hits", "flags"):
            assert np.array_equal(outs[0][0][k], st[k]), k
        assert np.array_equal(outs[0][1]["exits"], cn["exits"])


@pytest.mark.parametrize("prec", list(MODES))
def test_binned_histogram_matches_oracle_rule(B, oracle, prec):
    """Variable-width bins: the GPU's counts equal the oracle's rule applied
    to the GPU's own final state, bit for bit, in every precision -- with
    boundaries placed exactly on particle positions and one binary64 ulp on
    either side of them (the binary32 boundaries are rounded up so that the
    binary32 comparison decides as the binary64 one), edges without bins and
    dead particles included."""
    O = oracle
    d = W.random_mixed(7)
    E = len(d["src"])
    e, x = W.uniform_on_edges(d, 30_000, 6)
    g = B.Graph(d)
    p = B.Particles(g, e, x, seed=2, precision=MODES[prec])
    p.simulate(2e-3, 100, 8)
    st = p.state()
    es, xs = st["edge"], st["x"]
    rng = np.random.Generator(np.random.PCG64(1))
    off, up = [0], []
    for k in range(E):
        if k % 4 == 3:
            off.append(off[-1])
            continue
        L = d["length"][k] if np.isfinite(d["length"][k]) else 4.0
        b = list(rng.uniform(0.0, L, int(rng.integers(1, 10))))
        on = xs[es == k][:3]
        for v in on:
            b += [v, np.nextafter(v, np.inf), np.nextafter(v, -np.inf)]
        b = np.unique(np.array([v for v in b if v > 0.0]))
        up += list(b)
        off.append(off[-1] + len(b))
    off = np.array(off, np.int32)
    up = np.array(up)
    h = p.histogram_binned(off, up)
    ref = O.histogram_binned(O.Graph.from_desc(d), O.State(es, xs), off, up)
    assert np.array_equal(h.astype(np.uint64), ref)
    assert ref.sum() > 0 and np.count_nonzero(es < 0) > 0
    import torch
    hd = torch.zeros(int(off[-1]), dtype=torch.int32, device="cuda")
    p.histogram_binned(off, up, hd)
    assert np.array_equal(hd.cpu().numpy().astype(np.uint64), ref)
    p.close()
    g.close()


def test_binned_histogram_validation(B):
    d = W.star_brownian(3)
    e, x = W.uniform_on_edges(d, 1000, 1)
    g = B.Graph(d)
    p = B.Particles(g, e, x, seed=1, precision=B.MG_FP32_MIXED)
    for off, up in (([1, 2, 3, 4], [0.5, 0.5, 0.5, 0.5]),       # offsets[0] != 0
                    ([0, 2, 1, 3], [0.5, 1.0, 0.5]),             # decreasing offsets
                    ([0, 2, 2, 2], [0.5, 0.5]),                  # not increasing
                    ([0, 1, 1, 1], [0.0]),                       # not > 0
                    ([0, 1, 1, 1], [np.inf])):                   # not finite
        with pytest.raises(B.MGError):
            p.histogram_binned(np.array(off, np.int32), np.array(up, float))
    h = p.histogram_binned(np.array([0, 0, 0, 0], np.int32), np.zeros(0))
    assert h.sum() == 0
    p.close()
    g.close()


@pytest.mark.parametrize("prec", list(MODES))
def test_particles_per_block_do_not_change_results(B, prec):
    """A graph with absorbing vertices runs a set larger than the resident
    blocks with lanes that take the next particle when theirs dies or
    finishes: bit for bit the same results as one particle per thread (here
    forced with few blocks), including particles already dead at the second
    launch, split batches above one and the fused histogram."""
    import torch
    d = W.random_mixed(7)
    assert np.any(np.asarray(d["kind"]) == 1)
    e, x = W.uniform_on_edges(d, 20_000, 4)
    g = B.Graph(d)
    outs = []
    for blocks, sb in ((0, 1), (1, 1), (3, 5), (7, 32)):
        p = B.Particles(g, e, x, seed=8, precision=MODES[prec])
        p.set_tuning(split_batch=sb, max_blocks=blocks)
        h = torch.zeros(g.n_edges * 8, dtype=torch.int32, device="cuda")
        p.simulate(3e-3, 150, 8, hist_bins=8, hist_out=h)
        p.simulate(3e-3, 70, 8)
        p.synchronize()
        outs.append((p.state(), p.counts(), h.cpu().numpy()))
        p.close()
    g.close()
    ref_state, ref_counts, ref_hist = outs[0]
    assert ref_counts["absorbed"].sum() > 0
    for st, cn, hist in outs[1:]:
        for k in ("edge", "x", "n_draw", "hits", "first_hits", "flags"):
            assert np.array_equal(ref_state[k], st[k]), k
        for k in ("exits", "absorbed", "truncations", "particle_steps"):
            assert np.array_equal(np.asarray(ref_counts[k]), np.asarray(cn[k])), k
        assert np.array_equal(ref_hist, hist)



@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
def test_small_set_spread_over_more_blocks(B, prec):
    """A set too small to fill the GPU runs with fewer particles per block
    (down to 32; the rest of each block idles): every particle's trajectory
    and the counters are bit for bit those of the same particles inside a
    large set, which runs 256 per block."""
    import torch
    d = W.star_langevin(16)
    n_big, n_small = 1 << 19, 5000
    e, x = W.uniform_on_edges(d, n_big, 6)
    g = B.Graph(d)
    runs = []
    for n in (n_small, n_big, 33, 1):
        p = B.Particles(g, e[:n], x[:n], seed=2, precision=MODES[prec])
        h = torch.zeros(g.n_edges * 4, dtype=torch.int32, device="cuda")
        p.simulate(1e-3, 120, 16, 4, h)
        p.synchronize()
        runs.append((p.state(), p.counts(), h.cpu().numpy()))
        p.close()
    g.close()
    small, big = runs[0][0], runs[1][0]
    for k in ("edge", "x", "n_draw", "hits", "first_hits", "flags"):
        assert np.array_equal(small[k], big[k][:n_small]), k
        assert np.array_equal(runs[2][0][k], big[k][:33]), k
        assert np.array_equal(runs[3][0][k], big[k][:1]), k
    assert runs[0][1]["particle_steps"] == n_small * 120
    assert runs[0][2].sum() == n_small and runs[2][2].sum() == 33

def test_fused_histogram_matches_standalone(B):
    import torch
    d = W.star_langevin(16)
    e, x = W.uniform_on_edges(d, 50_000, 1)
    for P in (B.MG_FP32, B.MG_FP32_MIXED, B.MG_FP64):
        g = B.Graph(d)
        p = B.Particles(g, e, x, seed=4, precision=P)
        h = torch.zeros(16 * 32, dtype=torch.int32, device="cuda")
        p.simulate(1e-3, 500, 16, hist_bins=32, hist_out=h)
        p.synchronize()
        alone = p.histogram(32)
        assert np.array_equal(h.cpu().numpy().view(np.uint32), alone)
        assert alone.sum() == 50_000
        p.close(); g.close()


def test_device_inputs_and_validation(B):
    import torch
    d = W.random_tree(50, seed=1)
    e, x = W.uniform_on_edges(d, 3000, 5)
    a, ca, _ = gpu_run(B, d, e, x, seed=3, dt=2e-3, steps=100, M=8, prec=B.MG_FP64)
    g = B.Graph(d)
    et = torch.from_numpy(e).cuda()
    xt = torch.from_numpy(x).cuda()
    p = B.Particles(g, et, xt, seed=3, precision=B.MG_FP64)
    p.simulate(2e-3, 100, 8)
    p.synchronize()
    s = p.state()
    assert np.array_equal(s["x"], a["x"]) and np.array_equal(s["edge"], a["edge"])
    p.close()
    # an out-of-range edge in device input is reported, not trapped
    bad = et.clone()
    bad[17] = 10_000
    p = B.Particles(g, bad, xt, seed=3, precision=B.MG_FP64)
    with pytest.raises(B.MGError) as ei:
        p.synchronize()
    assert ei.value.status == B.MG_ERR_DEVICE_FAULT
    p.close()
    # host input is validated on the host
    with pytest.raises(B.MGError) as ei:
        B.Particles(g, np.array([0, 99], np.int32), np.array([0.1, 0.1]), seed=3)
    assert ei.value.status == B.MG_ERR_INVALID_ARG
    # a rejected reset leaves the set as it was: state and counters
    p = B.Particles(g, e, x, seed=3, precision=B.MG_FP64)
    p.simulate(2e-3, 50, 8)
    st0, c0 = p.state(), p.counts()
    bad_e = e.copy()
    bad_e[5] = 10_000
    with pytest.raises(B.MGError) as ei:
        p.reset(bad_e, x)
    assert ei.value.status == B.MG_ERR_INVALID_ARG
    st1, c1 = p.state(), p.counts()
    for k in ("edge", "x", "n_draw", "hits", "step"):
        assert np.array_equal(st0[k], st1[k]), k
    assert np.array_equal(c0["exits"], c1["exits"]) and c0["particle_steps"] == c1["particle_steps"]
    p.close()
    g.close()
    # a position at +inf on a semi-infinite edge (x <= l_e = inf holds) is
    # rejected: on the host, and as a device error for device input, in
    # every mode
    d = W.paper_star("linear")
    g = B.Graph(d)
    with pytest.raises(B.MGError) as ei:
        B.Particles(g, np.array([0, 1], np.int32), np.array([0.1, np.inf]), seed=3)
    assert ei.value.status == B.MG_ERR_INVALID_ARG
    for prec in (B.MG_FP64, B.MG_FP32_MIXED, B.MG_FP32):
        p = B.Particles(g, torch.tensor([0, 1], dtype=torch.int32, device="cuda"),
                        torch.tensor([0.1, np.inf], dtype=torch.float64, device="cuda"),
                        seed=3, precision=prec)
        with pytest.raises(B.MGError) as ei:
            p.simulate(1e-3, 10, 8)
            p.synchronize()
        assert ei.value.status == B.MG_ERR_DEVICE_FAULT
        p.close()
    g.close()


def test_buffers_checked_before_any_launch(B):
    """Caller buffers the library would read or write out of bounds, or in the
    wrong memory, are refused before anything runs: by the binding (lengths,
    dtypes, placement) and, for raw pointers, by the C library (host memory
    where device memory is required and the reverse).  The set stays usable."""
    import ctypes as C
    import torch
    L = B.load()
    d = W.random_tree(20, seed=2)
    g = B.Graph(d)
    E = g.n_edges
    e, x = W.uniform_on_edges(d, 1000, 4)
    with pytest.raises(ValueError):                       # lengths differ
        B.Particles(g, e[:-1], x, seed=1)
    with pytest.raises(ValueError):                       # float32 device positions
        B.Particles(g, torch.from_numpy(e).cuda(), torch.from_numpy(x).float().cuda(), seed=1)
    with pytest.raises(ValueError):                       # host edges, device positions
        B.Particles(g, e, torch.from_numpy(x).cuda(), seed=1)
    p = B.Particles(g, e, x, seed=1, precision=B.MG_FP32_MIXED)
    with pytest.raises(ValueError):
        p.reset(e[:10], x[:10])
    with pytest.raises(ValueError):                       # host histogram for a kernel
        p.simulate(1e-3, 10, 8, 4, np.zeros(E * 4, np.uint32))
    with pytest.raises(ValueError):                       # one entry short
        p.simulate(1e-3, 10, 8, 4, torch.zeros(E * 4 - 1, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        p.simulate(1e-3, 10, 8, 4, torch.zeros(E * 4, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        p.histogram(4, np.zeros(E * 4 - 1, np.uint32))
    with pytest.raises(ValueError):                       # offsets for fewer edges
        p.histogram_binned(np.arange(E, dtype=np.int32), np.ones(E - 1))
    with pytest.raises(ValueError):
        st = p.state()
        st["x"] = st["x"][:-1]
        p.set_state(st)
    # the C library on raw pointers
    host = np.zeros(E * 4, np.uint32)
    assert L.mg_simulate(p.h, 1e-3, 10, 8, 4, C.c_void_p(host.ctypes.data), None) == \
        B.MG_ERR_INVALID_ARG
    assert L.mg_histogram(p.h, 4, C.c_void_p(host.ctypes.data), 1, None) == B.MG_ERR_INVALID_ARG
    dev = torch.zeros(E * 4, dtype=torch.int32, device="cuda")
    assert L.mg_histogram(p.h, 4, C.c_void_p(dev.data_ptr()), 0, None) == B.MG_ERR_INVALID_ARG
    assert L.mg_histogram_static(p.h, 4, C.c_void_p(dev.data_ptr()), None) == B.MG_ERR_INVALID_ARG
    xd = torch.zeros(len(x), dtype=torch.float64, device="cuda")
    assert L.mg_state_get(p.h, None, C.c_void_p(xd.data_ptr()), None, None, None, None, None,
                          None) == B.MG_ERR_INVALID_ARG
    h = C.c_void_p()
    assert L.mg_particles_init(g.h, len(x), C.c_void_p(e.ctypes.data), C.c_void_p(x.ctypes.data),
                               1, 0, 1, 0, B.MG_FP32_MIXED, None, C.byref(h)) == \
        B.MG_ERR_INVALID_ARG
    s, keep = B._desc_struct(d)
    src = torch.from_numpy(np.asarray(d["src"], np.int32)).cuda()
    s.edge_src = C.cast(C.c_void_p(src.data_ptr()), C.POINTER(C.c_int32))
    assert L.mg_graph_create(C.byref(s), C.byref(h)) == B.MG_ERR_INVALID_ARG
    assert "device memory" in B.mg_last_error()
    # nothing ran; the set still works and matches a fresh one
    p.simulate(1e-3, 10, 8, 4, dev)
    q = B.Particles(g, e, x, seed=1, precision=B.MG_FP32_MIXED)
    q.simulate(1e-3, 10, 8)
    p.synchronize()
    q.synchronize()
    sp = p.state()
    assert np.array_equal(sp["x"], q.state()["x"])
    assert int(dev.sum()) == int(np.count_nonzero(sp["edge"] >= 0))
    p.close()
    q.close()
    g.close()



def test_large_host_inputs_checked_on_all_cores(B):
    """Starting positions of a large set are checked on several host threads;
    the error still names the first bad particle, and the set is unchanged by
    a rejected reset.  Results read back to the host through the library's
    pinned buffer are the same from several host threads at once."""
    import threading
    d = W.star_langevin(16)
    n = 1 << 21
    e, x = W.uniform_on_edges(d, n, 12)
    g = B.Graph(d)
    for bad in ([1_500_000, 1_900_000], [700_001], [n - 1]):
        xb = x.copy()
        xb[bad] = -1.0
        with pytest.raises(B.MGError) as ei:
            B.Particles(g, e, xb, seed=1, precision=B.MG_FP32_MIXED)
        assert ei.value.status == B.MG_ERR_INVALID_ARG
        assert f"particle {min(bad)}:" in str(ei.value), str(ei.value)
    eb = e.copy()
    eb[123_456] = 99
    with pytest.raises(B.MGError) as ei:
        B.Particles(g, eb, x, seed=1, precision=B.MG_FP32_MIXED)
    assert "particle 123456: edge 99" in str(ei.value)
    sets = [B.Particles(g, e, x, seed=s, precision=B.MG_FP32_MIXED) for s in range(4)]
    for p in sets:
        p.simulate(1e-3, 20, 16)
        p.synchronize()
    ref = [(p.counts(), p.histogram(8)) for p in sets]
    got = [None] * len(sets)

    def read(k):
        for _ in range(5):
            got[k] = (sets[k].counts(), sets[k].histogram(8))

    threads = [threading.Thread(target=read, args=(k,)) for k in range(len(sets))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for (c0, h0), (c1, h1) in zip(ref, got):
        assert np.array_equal(c0["exits"], c1["exits"]) and c0["particle_steps"] == c1["particle_steps"]
        assert np.array_equal(h0, h1)
    for p in sets:
        p.close()
    g.close()

def test_overflow_to_infinity_is_reported(B):
    """A drift that pushes particles off to infinity on a semi-infinite edge
    (mu = +50 x: x grows by 5% a step) overflows binary32 within ~1800 steps:
    the kernel stops those particles and reports a device error instead of
    treating the overflow as a hit at the edge's missing far end."""
    d = W.paper_star("quadratic", k=2)
    d = dict(d, c1=np.array([50.0, -10.0]))
    g = B.Graph(d)
    e = np.array([0] * 64 + [1] * 64, np.int32)
    x = np.full(128, 1.0)
    for prec in (B.MG_FP32_MIXED, B.MG_FP32):
        p = B.Particles(g, e, x, seed=1, precision=prec)
        with pytest.raises(B.MGError) as ei:
            p.simulate(1e-3, 4000, 8)
            p.synchronize()
        assert ei.value.status == B.MG_ERR_DEVICE_FAULT
        p.close()
    g.close()


def test_torch_allocator_same_results(B):
    d = W.star_brownian(3)
    e, x = W.round_robin_uniform(d, 2000, 3)
    a, ca, _ = gpu_run(B, d, e, x, seed=1, dt=1e-3, steps=300, M=8, prec=B.MG_FP32_MIXED)
    B.use_torch_allocator()
    try:
        b, cb, _ = gpu_run(B, d, e, x, seed=1, dt=1e-3, steps=300, M=8, prec=B.MG_FP32_MIXED)
    finally:
        B.use_cuda_allocator()
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(ca["exits"], cb["exits"])


# ------------------------------------------------------ FP32-mixed parity

def _occupancy(edge, E):
    alive = edge >= 0
    return np.bincount(edge[alive], minlength=E) / len(edge)


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_star16_langevin_fp32_statistics(B, prec):
    """binary32 modes vs the FP64 oracle on the 16-edge Langevin star: same
    streams, N = 2^16, 2000 steps."""
    d = W.star_langevin(16)
    n = 1 << 16
    e, x = W.uniform_on_edges(d, n, 11)
    gs, gc, gh = gpu_run(B, d, e, x, seed=0, dt=1e-3, steps=2000, M=16, prec=MODES[prec],
                         bins=32)
    o = oracle_pool.run(d, e, x, seed=0, dt=1e-3, steps=2000, M=16, bins=32)
    po, pg = _occupancy(o["edge"], 16), _occupancy(gs["edge"], 16)
    se = np.sqrt(po * (1 - po) / n)
    assert np.all(np.abs(pg - po) <= 3 * se + 1e-12), (pg - po) / se
    eo = o["exits"].astype(float)
    eg = gc["exits"].astype(float)
    fo, fg = eo / eo.sum(), eg / eg.sum()
    assert np.all(np.abs(fg - fo) <= 3 * np.sqrt(fo * (1 - fo) / eo.sum()) + 1e-12)
    # coupled streams: almost every particle ends on the same edge, nearby
    same = gs["edge"] == o["edge"]
    assert same.mean() > 0.95
    assert np.median(np.abs(gs["x"][same] - o["x"][same])) < 1e-4
    tv = 0.5 * np.abs(gh / n - o["hist"] / n).sum()
    assert tv < 0.02, tv


def test_star16_full_size_sampled(B):
    """The benchmark's configuration (N = 2^24, 10^4 steps, M = 16, FP32-mixed)
    against oracle trajectories of 1024 sampled particles, plus FP64 mode at
    full N on 200 steps, trajectory by trajectory on the same sample."""
    import torch
    d = W.star_langevin(16)
    n = 1 << 24
    e, x = W.uniform_on_edges(d, n, 11)
    idx = np.sort(np.random.default_rng(5).choice(n, 1024, replace=False))
    h = torch.zeros(16 * 32, dtype=torch.int32, device="cuda")
    g = B.Graph(d)
    p = B.Particles(g, e, x, seed=0, precision=B.MG_FP32_MIXED)
    p.simulate(1e-3, 10_000, 16, hist_bins=32, hist_out=h)
    p.synchronize()
    st = p.state()
    cnt = p.counts()
    p.close()
    hist = h.cpu().numpy().view(np.uint32).astype(np.int64)
    assert hist.sum() == n and cnt["particle_steps"] == n * 10_000
    o = oracle_pool.run(d, e[idx], x[idx], idx, seed=0, dt=1e-3, steps=10_000, M=16)
    same = st["edge"][idx] == o["edge"]
    assert same.mean() > 0.85, same.mean()
    # occupancy of the whole population (N = 2^24: its own error is negligible)
    # against the oracle's sample of 1024; 16 edges, so 4 standard errors
    po = _occupancy(o["edge"], 16)
    pg = np.bincount(st["edge"], minlength=16) / n
    assert np.all(np.abs(pg - po) <= 4 * np.sqrt(pg * (1 - pg) / len(idx)) + 1e-9)
    # FP64 at full N: sampled trajectories exact
    p = B.Particles(g, e, x, seed=0, precision=B.MG_FP64)
    p.simulate(1e-3, 200, 16)
    p.synchronize()
    s64 = p.state()
    p.close()
    g.close()
    o64 = oracle_pool.run(d, e[idx], x[idx], idx, seed=0, dt=1e-3, steps=200, M=16)
    sub = {k: s64[k][idx] for k in ("edge", "x", "n_draw", "hits", "first_hits", "flags")}
    flagged = ((sub["flags"] | o64["flags"]) & 1) != 0
    ok = ~flagged
    assert np.array_equal(sub["edge"][ok], o64["edge"][ok])
    assert np.array_equal(sub["n_draw"][ok], o64["n_draw"][ok])
    assert np.all(np.abs(sub["x"][ok] - o64["x"][ok]) <= REL * np.maximum(1, np.abs(o64["x"][ok])))


def test_star16_coupled_tv_fp32_vs_fp64_full_n(B):
    """Coupled total-variation distance between the FP32-mixed and FP64
    histograms at N = 2^24 (both GPU; the FP64 mode is the oracle's
    trajectories, as the tests above show).  Two independent histograms of
    N particles over 512 bins would differ by about sqrt(512 / (pi N)) =
    3.1e-3; shared random streams bring the coupled distance under 1e-3."""
    import torch
    d = W.star_langevin(16)
    n = 1 << 24
    e, x = W.uniform_on_edges(d, n, 11)
    hs = []
    g = B.Graph(d)
    for P in (B.MG_FP32_MIXED, B.MG_FP64):
        h = torch.zeros(16 * 32, dtype=torch.int32, device="cuda")
        p = B.Particles(g, e, x, seed=0, precision=P)
        p.simulate(1e-3, 1000, 16, hist_bins=32, hist_out=h)
        p.synchronize()
        hs.append(h.cpu().numpy().view(np.uint32).astype(np.int64))
        p.close()
    g.close()
    tv = 0.5 * np.abs(hs[0] - hs[1]).sum() / n
    assert tv <= 1e-3, tv


# ------------------------------------------------ synthetic vascular graph

def test_vascular_fp64_trajectories(B):
    """The vascular stand-in (5000 points): drift-dominated edges, many
    splits per step, absorbing outlets, tracer injected at the inlets."""
    d = W.vascular(n_points=5000)
    n = 4096
    e, x = W.inject_at_inlets(d, n, 3)
    gs, gc, gh = gpu_run(B, d, e, x, seed=2, dt=d["dt"], steps=300, M=32, prec=B.MG_FP64, bins=4)
    o = oracle_pool.run(d, e, x, seed=2, dt=d["dt"], steps=300, M=32, bins=4)
    assert_fp64_parity(gs, gc, o, ghist=gh)
    assert gc["absorbed"].sum() > 0


def test_vascular_full_size_sampled(B):
    """The vascular configuration at full size (2^26 tracers, 2000 steps,
    M = 32, FP32-mixed: the range kernel): every tracer counted once (alive
    in the histogram or absorbed), positions inside their edges, and the
    absorbed fraction equal to an oracle sample's within 4 standard errors;
    then FP64 at full N over 800 steps (also the range kernel) against
    oracle trajectories of 512 sampled tracers."""
    import torch
    d = W.vascular()
    n = 1 << 26
    e, x = W.inject_at_inlets(d, n, 11)
    g = B.Graph(d)
    h = torch.zeros(g.n_edges * 16, dtype=torch.int32, device="cuda")
    p = B.Particles(g, e, x, seed=0, precision=B.MG_FP32_MIXED)
    p.simulate(d["dt"], 2000, 32, hist_bins=16, hist_out=h)
    p.synchronize()
    st, cnt = p.state(), p.counts()
    p.close()
    alive = st["edge"] >= 0
    hist = h.cpu().numpy().view(np.uint32).astype(np.int64)
    assert hist.sum() == alive.sum()
    assert hist.sum() + cnt["absorbed"].sum() == n
    # binary32 state: an edge's length is its binary32 rounding (a tracer at
    # the far vertex sits at float(l_e), which may exceed l_e)
    L = np.asarray(d["length"]).astype(np.float32).astype(np.float64)[st["edge"][alive]]
    assert np.all((st["x"][alive] >= 0) & (st["x"][alive] <= L))
    idx = np.sort(np.random.default_rng(7).choice(n, 1024, replace=False))
    o = oracle_pool.run(d, e[idx], x[idx], idx, seed=0, dt=d["dt"], steps=2000, M=32)
    pg = 1.0 - alive.mean()
    po = np.mean(o["edge"] < 0)
    assert abs(pg - po) <= 4 * np.sqrt(pg * (1 - pg) / len(idx)) + 1e-9, (pg, po)
    # FP64 at full N over 800 steps: the sampled trajectories exactly
    p = B.Particles(g, e, x, seed=0, precision=B.MG_FP64)
    p.simulate(d["dt"], 800, 32)
    p.synchronize()
    s64 = p.state()
    p.close()
    g.close()
    idx = idx[:512]
    o64 = oracle_pool.run(d, e[idx], x[idx], idx, seed=0, dt=d["dt"], steps=800, M=32)
    sub = {k: s64[k][idx] for k in ("edge", "x", "n_draw", "hits", "flags")}
    ok = ((sub["flags"] | o64["flags"]) & 1) == 0
    assert ok.mean() > 0.9
    assert np.array_equal(sub["edge"][ok], o64["edge"][ok])
    assert np.array_equal(sub["n_draw"][ok], o64["n_draw"][ok])
    assert np.array_equal(sub["hits"][ok], o64["hits"][ok])
    live = ok & (o64["edge"] >= 0)
    assert np.all(np.abs(sub["x"][live] - o64["x"][live]) <= REL * np.maximum(1, np.abs(o64["x"][live])))


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_vascular_fp32_statistics(B, prec):
    d = W.vascular(n_points=5000)
    n = 1 << 15
    e, x = W.inject_at_inlets(d, n, 5)
    gs, gc, _ = gpu_run(B, d, e, x, seed=4, dt=d["dt"], steps=400, M=32, prec=MODES[prec])
    o = oracle_pool.run(d, e, x, seed=4, dt=d["dt"], steps=400, M=32)
    # absorbed fraction and the coupled per-particle fate
    fa_g, fa_o = (gs["edge"] < 0).mean(), (o["edge"] < 0).mean()
    assert abs(fa_g - fa_o) <= 3 * np.sqrt(fa_o * (1 - fa_o) / n) + 1e-9
    assert (gs["edge"] == o["edge"]).mean() > 0.8
    ao, ag = o["absorbed"].astype(float), gc["absorbed"].astype(float)
    top = np.argsort(-ao)[:10]  # the busiest outlets
    assert np.all(np.abs(ag[top] - ao[top]) <= 4 * np.sqrt(ao[top]) + 3)
    # exit frequency of every slot within 3 standard errors (multinomial over
    # the exits of each run, both runs' errors; one count of slack for
    # slots that see a handful of exits)
    eo, eg = o["exits"].astype(float), gc["exits"].astype(float)
    fo, fg = eo / eo.sum(), eg / eg.sum()
    se = np.sqrt(fo * (1 - fo) / eo.sum() + fg * (1 - fg) / eg.sum())
    dev = np.abs(fg - fo)
    print(f"\nvascular {prec}: {len(eo)} slots, {int(eo.sum())} exits; max |z| "
          f"{np.max(dev / np.maximum(se, 1e-300)):.2f} (slots with exits)")
    assert np.all(dev <= 3 * se + 1.0 / eo.sum()), np.argmax(dev - 3 * se)
