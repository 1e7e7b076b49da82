"""The served request loop on the GPU: a Poisson stream of requests of
different graphs, sizes, horizons and dt, admitted under a memory budget,
advanced in continuous-batching rounds on two streams.  Each request's final
state, counters and histogram are bit-identical to running it alone."""
import numpy as np
import pytest

from paper_2512_02175_gb300 import serve
from paper_2512_02175_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _graphs():
    return {"star3": W.star_brownian(3), "star16": W.star_langevin(16),
            "vascular": W.vascular(n_points=3000)}


@pytest.mark.parametrize("prec", [1, 0])
def test_served_equals_alone(prec):
    import torch
    from paper_2512_02175_gb300 import binding as B
    B.load()
    graphs = _graphs()
    reqs = serve.poisson_trace(400.0, 0.08, 3, graphs, n_range=(9, 13), steps_range=(20, 400),
                               init=serve.default_init)
    assert len(reqs) >= 12
    be = serve.GpuBackend(graphs, prec, seed=7, n_lanes=2)
    total = sum(be.bytes_of(r) for r in reqs)
    srv = serve.Server(be, mem_budget=max(total // 3, max(be.bytes_of(r) for r in reqs)),
                       n_lanes=2, chunk_steps=64, keep_state=True)
    res = srv.run_trace(reqs, time_limit=300)
    assert sorted(r.rid for r in res) == [q.rid for q in sorted(reqs, key=lambda q: q.rid)]
    assert srv.peak_reserved <= srv.mem_budget
    by = {r.rid: r for r in res}
    G = {k: B.Graph(d) for k, d in graphs.items()}
    for q in reqs:
        p = B.Particles(G[q.graph], q.edge0, q.x0, seed=7, instance=q.rid, precision=prec)
        p.simulate(q.dt, q.steps, q.M)
        st, cn, h = p.state(), p.counts(), p.histogram(q.bins)
        p.close()
        r = by[q.rid]
        for k in ("edge", "x", "n_draw", "hits", "first_hits", "flags"):
            assert np.array_equal(st[k], r.state[k]), (q.rid, k)
        assert np.array_equal(cn["exits"], r.counts["exits"])
        assert np.array_equal(cn["absorbed"], r.counts["absorbed"])
        assert cn["truncations"] == r.counts["truncations"]
        assert np.array_equal(h, r.hist)
    s = serve.latency_summary(res)
    assert s["p99_s"] >= s["p50_s"] > 0
    be.close()


def test_failed_request_is_isolated():
    """One request with a starting position off its edge (refused at
    admission) and one whose drift carries its particles off to infinity on a
    semi-infinite edge (a device error of its own set, found at collection)
    fail alone: their results carry the error, every other request completes
    and equals its run alone."""
    from paper_2512_02175_gb300 import binding as B
    B.load()
    graphs = {"star3": W.star_brownian(3),
              "runaway": dict(W.paper_star("quadratic", k=2), c1=np.array([50.0, -10.0]))}
    reqs = []
    for i in range(8):
        key = "runaway" if i == 5 else "star3"
        n = 256 + 64 * i
        if key == "runaway":
            e0, x0 = np.zeros(n, np.int32), np.full(n, 1.0)
            steps = 4000
        else:
            e0, x0 = W.uniform_on_edges(graphs[key], n, 50 + i)
            steps = 300
        if i == 2:
            x0 = x0.copy()
            x0[7] = 1.5  # the edges have length 1
        reqs.append(serve.Request(i, key, n, steps, 1e-3, 8, 16, e0, x0, 0.001 * i))
    be = serve.GpuBackend(graphs, B.MG_FP32_MIXED, seed=7, n_lanes=2)
    srv = serve.Server(be, mem_budget=1 << 30, n_lanes=2, chunk_steps=100, keep_state=True)
    res = srv.run_trace(reqs, time_limit=300)
    by = {r.rid: r for r in res}
    assert sorted(by) == list(range(8)) and srv.reserved == 0
    assert by[2].error and "INVALID_ARG" in by[2].error
    assert by[5].error and "DEVICE_FAULT" in by[5].error
    G = {k: B.Graph(d) for k, d in graphs.items()}
    for q in reqs:
        if q.rid in (2, 5):
            continue
        assert by[q.rid].error is None
        p = B.Particles(G[q.graph], q.edge0, q.x0, seed=7, instance=q.rid,
                        precision=B.MG_FP32_MIXED)
        p.simulate(q.dt, q.steps, q.M)
        st = p.state()
        p.close()
        assert np.array_equal(st["x"], by[q.rid].state["x"])
        assert np.array_equal(st["edge"], by[q.rid].state["edge"])
    s = serve.latency_summary(res)
    assert s["requests"] == 6 and s["failed"] == 2
    be.close()
    for g in G.values():
        g.close()

def test_plain_path_runs():
    graphs = _graphs()
    reqs = serve.poisson_trace(200.0, 0.03, 5, graphs, n_range=(8, 10), steps_range=(10, 50),
                               init=serve.default_init)
    res = serve.serve_plain(reqs, graphs, 0, seed=7)
    assert len(res) == len(reqs)
    assert all(r.particle_steps > 0 for r in res)


def test_full_size_trace_sampled():
    """The served configuration at full size, as the benchmark runs it: 634
    requests in 3 s over the 3-edge star, the 16-edge star and the full
    vascular network (n = 2^U[12, 18]), 32 GB admission budget, rounds of 500
    steps on two streams -- every request completes, and a dozen sampled
    requests are bit-identical to running them alone."""
    import torch
    from paper_2512_02175_gb300 import binding as B
    B.load()
    graphs = {"star3": W.star_brownian(3), "star16": W.star_langevin(16),
              "vascular": W.vascular()}
    reqs = serve.poisson_trace(200.0, 3.0, 17, graphs, n_range=(12, 18),
                               init=serve.default_init)
    assert len(reqs) > 500
    sample = set(np.random.default_rng(1).choice(len(reqs), 12, replace=False).tolist())
    be = serve.GpuBackend(graphs, B.MG_FP32_MIXED, seed=0, n_lanes=2)
    srv = serve.Server(be, mem_budget=32 << 30, n_lanes=2, chunk_steps=500, keep_state=sample)
    res = srv.run_trace(reqs, time_limit=600)
    be.close()
    assert sorted(r.rid for r in res) == list(range(len(reqs)))
    by = {r.rid: r for r in res}
    G = {k: B.Graph(d) for k, d in graphs.items()}
    for rid in sorted(sample):
        q = reqs[rid]
        p = B.Particles(G[q.graph], q.edge0, q.x0, seed=0, instance=q.rid,
                        precision=B.MG_FP32_MIXED)
        p.simulate(q.dt, q.steps, q.M)
        st, cn, h = p.state(), p.counts(), p.histogram(q.bins)
        p.close()
        r = by[rid]
        assert r.state is not None
        for k in ("edge", "x", "n_draw", "hits", "first_hits", "flags"):
            assert np.array_equal(st[k], r.state[k]), (rid, k)
        assert np.array_equal(cn["exits"], r.counts["exits"])
        assert np.array_equal(h, r.hist)
    assert all(r.state is None for r in res if r.rid not in sample)
    for g in G.values():
        g.close()
