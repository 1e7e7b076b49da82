"""The batched persistent kernel: many uneven particle sets in one launch.

* alone == in mix: every instance's state, counters and fused histogram are
  bit-identical whether it runs alone (mg_simulate) or inside a batch, with
  or without CUDA-graph capture, in every precision mode -- the random
  streams are keyed by (seed, instance, particle id) and each particle is
  computed by the same device function either way.
* graph replay: a captured batch replayed twice equals two direct runs.
* FP64 through the batch matches the CPU oracle trajectory by trajectory.
"""
import numpy as np
import pytest

from paper_2512_02175_gb300 import workloads as W
from tests import oracle_pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available()
    from paper_2512_02175_gb300 import binding as B
    B.load()
    return B


def _instances(n_inst=14, seed=9):
    insts = W.batch_instances(n_inst, seed=seed, n_scale=1 / 256, steps_scale=0.1,
                              max_tree_edges=3000)
    for k, it in enumerate(insts):
        it["x0"] = W.uniform_on_edges(it["graph"], it["n"], 100 + k)
    return insts


def _make(B, insts, prec, seed=5):
    import torch
    objs = []
    for it in insts:
        g = B.Graph(it["graph"])
        e, x = it["x0"]
        p = B.Particles(g, e, x, pid_base=0, seed=seed, instance=it["instance"], precision=prec)
        h = torch.zeros(g.n_edges * 8, dtype=torch.int32, device="cuda")
        objs.append((g, p, h))
    return objs


def _collect(objs):
    out = []
    for g, p, h in objs:
        p.synchronize()
        out.append((p.state(), p.counts(), h.cpu().numpy().copy()))
    return out


def _same(a, b):
    for (sa, ca, ha), (sb, cb, hb) in zip(a, b):
        for k in ("edge", "x", "n_draw", "hits", "first_hits", "flags", "step"):
            assert np.array_equal(sa[k], sb[k]), k
        for k in ("exits", "absorbed"):
            assert np.array_equal(ca[k], cb[k]), k
        assert ca["truncations"] == cb["truncations"]
        assert ca["particle_steps"] == cb["particle_steps"]
        assert np.array_equal(ha, hb)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("graph", [False, True])
def test_alone_equals_in_batch(B, prec, graph):
    import torch
    insts = _instances()
    alone = _make(B, insts, prec)
    for (g, p, h), it in zip(alone, insts):
        p.simulate(it["dt"], it["steps"], it["M"], 8, h)
    ra = _collect(alone)
    mixed = _make(B, insts, prec)
    b = B.Batch()
    for (g, p, h), it in zip(mixed, insts):
        b.add(p, it["dt"], it["steps"], it["M"], 8, h)
    s = torch.cuda.Stream()
    b.run(use_graph=graph, stream=s)
    s.synchronize()
    n_members, n_items, blocks = b.info()
    assert n_members == len(insts) and n_items == sum((it["n"] + 255) // 256 for it in insts)
    _same(ra, _collect(mixed))
    b.close()


def test_graph_replay_equals_direct_runs(B):
    import torch
    insts = _instances(8, seed=3)
    runs = []
    for graph in (False, True):
        objs = _make(B, insts, 1)
        b = B.Batch()
        b.set_tuning(split_batch=2, stage_limit_bytes=4096, blocks_per_sm=2)
        for (g, p, h), it in zip(objs, insts):
            b.add(p, it["dt"], it["steps"], it["M"], 8, h)
        s = torch.cuda.Stream()
        b.run(use_graph=graph, stream=s)
        b.run(use_graph=graph, stream=s)
        s.synchronize()
        runs.append(_collect(objs))
        b.close()
    _same(runs[0], runs[1])


def test_batch_fp64_matches_oracle(B):
    import torch
    insts = _instances(6, seed=21)
    objs = _make(B, insts, 0)
    b = B.Batch()
    for (g, p, h), it in zip(objs, insts):
        b.add(p, it["dt"], it["steps"], it["M"], 8, h)
    s = torch.cuda.Stream()
    b.run(use_graph=True, stream=s)
    s.synchronize()
    for ((g, p, h), it) in zip(objs, insts):
        st = p.state()
        e, x = it["x0"]
        o = oracle_pool.run(it["graph"], e, x, seed=5, instance=it["instance"], dt=it["dt"],
                            steps=it["steps"], M=it["M"])
        ok = ((st["flags"] | o["flags"]) & 1) == 0
        assert ok.mean() > 0.99
        assert np.array_equal(st["edge"][ok], o["edge"][ok])
        assert np.array_equal(st["n_draw"][ok], o["n_draw"][ok])
        assert np.all(np.abs(st["x"][ok] - o["x"][ok]) <= 1e-12 * np.maximum(1, np.abs(o["x"][ok])))
    b.close()


def test_batch_rejects_mixed_seeds_and_precisions(B):
    d = W.star_brownian(3)
    g = B.Graph(d)
    e, x = W.round_robin_uniform(d, 100, 1)
    p1 = B.Particles(g, e, x, seed=1, precision=1)
    p2 = B.Particles(g, e, x, seed=2, precision=1)
    p3 = B.Particles(g, e, x, seed=1, precision=0)
    b = B.Batch()
    b.add(p1, 1e-3, 10, 8)
    with pytest.raises(B.MGError):
        b.add(p2, 1e-3, 10, 8)
    with pytest.raises(B.MGError):
        b.add(p3, 1e-3, 10, 8)
    with pytest.raises(B.MGError):
        b.add(p1, 1e-3, 10, 8)
    b.close()


def test_full_size_batch_sampled(B):
    """The batched configuration at full size, in the launch the benchmark
    times: all 512 instances (3.3e8 particles, 100..5000 steps each) in one
    graph-replayed persistent launch, FP32-mixed -- every instance takes all
    its particle-steps (no vertex absorbs) and stays on its edges; then the
    same 512 instances in FP64 over a tenth of their steps, 8 sampled
    particles of every 32nd instance against the oracle, trajectory by
    trajectory."""
    import torch
    insts = W.batch_instances(512)
    s = torch.cuda.Stream()
    graphs, parts = [], []
    for k, it in enumerate(insts):
        g = B.Graph(it["graph"])
        e, x = W.uniform_on_edges(it["graph"], it["n"], 100 + k)
        it["x0"] = (e, x)
        graphs.append(g)
        parts.append(B.Particles(g, e, x, seed=0, instance=k, precision=B.MG_FP32_MIXED))
    b = B.Batch()
    for p, it in zip(parts, insts):
        b.add(p, it["dt"], it["steps"], it["M"])
    b.run(use_graph=True, stream=s)
    s.synchronize()
    for p, it, g in zip(parts, insts, graphs):
        c = p.counts()
        assert c["particle_steps"] == it["n"] * it["steps"]
        if it["instance"] % 64 == 0:
            st = p.state()
            L = np.asarray(it["graph"]["length"]).astype(np.float32).astype(np.float64)
            assert np.all((st["x"] >= 0) & (st["x"] <= L[st["edge"]]))
        p.close()
    b.close()
    # FP64, a tenth of the steps, full particle counts
    parts = [B.Particles(g, *it["x0"], seed=0, instance=k, precision=B.MG_FP64)
             for k, (g, it) in enumerate(zip(graphs, insts))]
    b = B.Batch()
    for p, it in zip(parts, insts):
        b.add(p, it["dt"], max(1, it["steps"] // 10), it["M"])
    b.run(use_graph=True, stream=s)
    s.synchronize()
    rng = np.random.default_rng(3)
    for k in range(0, 512, 32):
        it, p = insts[k], parts[k]
        st = p.state()
        idx = np.sort(rng.choice(it["n"], 8, replace=False))
        e, x = it["x0"]
        o = oracle_pool.run(it["graph"], e[idx], x[idx], idx, seed=0, instance=k, dt=it["dt"],
                            steps=max(1, it["steps"] // 10), M=it["M"])
        ok = ((st["flags"][idx] | o["flags"]) & 1) == 0
        assert np.array_equal(st["edge"][idx][ok], o["edge"][ok])
        assert np.array_equal(st["n_draw"][idx][ok], o["n_draw"][ok])
        assert np.all(np.abs(st["x"][idx][ok] - o["x"][ok])
                      <= 1e-12 * np.maximum(1.0, np.abs(o["x"][ok])))
    for p in parts:
        p.close()
    b.close()
    for g in graphs:
        g.close()
