"""Admission and scheduling of the served request loop, on the CPU with a
fake backend (no GPU): memory budget respected, FIFO admission, continuous
batching in rounds of at most chunk_steps, several lanes in flight, every
request completed exactly once with all its steps."""
import numpy as np
import pytest

from paper_2512_02175_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    """Rounds complete after a fixed number of polls; records every launch."""

    def __init__(self, delay_polls=2):
        self.delay = delay_polls
        self.launches = []
        self.live = {}
        self.steps_done = {}

    def bytes_of(self, req):
        return req.n * 24

    def admit(self, req):
        self.live[req.rid] = req
        self.steps_done[req.rid] = 0
        return req.rid

    def launch(self, lane, members):
        for rid, s in members:
            assert rid in self.live
            self.steps_done[rid] += s
        tok = {"polls": 0, "lane": lane, "members": list(members)}
        self.launches.append(tok)
        return tok

    def poll(self, tok):
        tok["polls"] += 1
        return tok["polls"] > self.delay

    def collect(self, rid, keep_state):
        req = self.live[rid]
        return np.zeros(4, np.uint32), {"particle_steps": req.n * req.steps}, None

    def release(self, rid):
        del self.live[rid]


def _reqs(k, seed=0):
    r = np.random.default_rng(seed)
    return [serve.Request(i, "g", int(r.integers(100, 2000)), int(r.integers(1, 3000)), 1e-3)
            for i in range(k)]


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_all_requests_complete_within_budget(lanes):
    be = FakeBackend()
    clk = FakeClock()
    srv = serve.Server(be, mem_budget=60_000, n_lanes=lanes, chunk_steps=500, clock=clk)
    reqs = _reqs(40)
    for q in reqs:
        srv.submit(q)
    for _ in range(100_000):
        if srv.idle():
            break
        srv.step()
        clk.t += 1.0
        assert srv.reserved <= 60_000
        assert sum(1 for l in srv.lanes if l is not None) <= lanes
    assert srv.idle()
    assert sorted(r.rid for r in srv.results) == list(range(40))
    for q in reqs:
        assert be.steps_done[q.rid] == q.steps
    assert srv.peak_reserved <= 60_000
    # no round gives a request more than chunk_steps, and a request is never
    # in two rounds at once
    for tok in be.launches:
        assert all(s <= 500 for _, s in tok["members"])
    assert not be.live


def test_fifo_admission_blocks_behind_large_request():
    be = FakeBackend()
    clk = FakeClock()
    srv = serve.Server(be, mem_budget=10_000, n_lanes=2, chunk_steps=100, clock=clk)
    big = serve.Request(0, "g", 400, 300, 1e-3)      # 9600 bytes
    small = serve.Request(1, "g", 10, 10, 1e-3)      # 240 bytes: would fit, but waits its turn
    big2 = serve.Request(2, "g", 300, 10, 1e-3)
    for q in (big, big2, small):
        srv.submit(q)
    srv.step()
    assert [a.req.rid for a in srv.active] == [0]
    assert [q.rid for q in srv.queue] == [2, 1]


def test_request_larger_than_budget_rejected():
    srv = serve.Server(FakeBackend(), mem_budget=100, clock=FakeClock())
    with pytest.raises(ValueError):
        srv.submit(serve.Request(0, "g", 1000, 10, 1e-3))


def test_new_arrivals_join_next_round():
    be = FakeBackend(delay_polls=0)
    clk = FakeClock()
    srv = serve.Server(be, mem_budget=10**9, n_lanes=1, chunk_steps=100, clock=clk)
    srv.submit(serve.Request(0, "g", 10, 1000, 1e-3))
    srv.step()  # the first server round: request 0 alone
    srv.submit(serve.Request(1, "g", 10, 1000, 1e-3))
    for _ in range(3):
        srv.step()
    members = [[rid for rid, _ in t["members"]] for t in be.launches]
    assert members[0] == [0]
    assert any(m == [0, 1] for m in members[1:])


def test_latency_summary():
    res = [serve.Result(i, np.zeros(1), {}, None, 0.0, 0.0, float(i + 1), 100) for i in range(100)]
    s = serve.latency_summary(res, 0.0, 100.0)
    assert s["requests"] == 100 and abs(s["p50_s"] - 50.5) < 1e-9 and s["p99_s"] > 98.9
    assert s["served_particle_steps_per_s"] == 100.0


def test_poisson_trace_shape():
    tr = serve.poisson_trace(200.0, 5.0, 1, {"a": None, "b": None})
    assert 800 < len(tr) < 1200
    arr = np.array([q.arrival for q in tr])
    assert np.all(np.diff(arr) > 0) and arr[-1] <= 5.0
    assert all(2 ** 14 - 1 <= q.n <= 2 ** 24 + 1 for q in tr)
    assert all(100 <= q.steps <= 5000 for q in tr)


class FailingBackend(FakeBackend):
    """Admission of some requests raises (invalid input), collection of
    others raises (a device error of their own particle set)."""

    def __init__(self, bad_admit, bad_collect):
        super().__init__()
        self.bad_admit, self.bad_collect = set(bad_admit), set(bad_collect)
        self.released = []

    def admit(self, req):
        if req.rid in self.bad_admit:
            raise ValueError(f"request {req.rid}: starting position off its edge")
        return super().admit(req)

    def collect(self, rid, keep_state):
        if rid in self.bad_collect:
            raise RuntimeError(f"request {rid}: device error bits 0x2")
        return super().collect(rid, keep_state)

    def release(self, rid):
        self.released.append(rid)
        super().release(rid)


def test_failed_request_does_not_stop_the_others():
    be = FailingBackend(bad_admit=[3, 17], bad_collect=[5, 30])
    clk = FakeClock()
    srv = serve.Server(be, mem_budget=60_000, n_lanes=2, chunk_steps=500, clock=clk)
    reqs = _reqs(40, seed=4)
    for q in reqs:
        srv.submit(q)
    for _ in range(100_000):
        if srv.idle():
            break
        srv.step()
        clk.t += 1.0
    assert srv.idle() and srv.reserved == 0 and not be.live
    by = {r.rid: r for r in srv.results}
    assert sorted(by) == list(range(40))          # every request answered once
    for rid in (3, 17, 5, 30):
        assert by[rid].error and by[rid].hist is None
    assert "off its edge" in by[3].error and "device error" in by[5].error
    assert 3 not in be.released and 5 in be.released   # admitted sets are freed
    for q in reqs:
        if q.rid not in (3, 17, 5, 30):
            assert by[q.rid].error is None and be.steps_done[q.rid] == q.steps
    s = serve.latency_summary(srv.results)
    assert s["requests"] == 36 and s["failed"] == 4


def test_rounds_sized_by_work():
    """With round_work, a member takes max(chunk_steps, round_work // n)
    of its remaining steps per round: a small request is done in one round, a
    large one in several, and every request still gets all its steps."""
    be = FakeBackend(delay_polls=1)
    clk = FakeClock()
    srv = serve.Server(be, mem_budget=10**9, n_lanes=2, chunk_steps=100, clock=clk,
                       round_work=1_000_000)
    small = serve.Request(0, "g", 1000, 900, 1e-3)      # quota 1000 steps: one round
    large = serve.Request(1, "g", 100_000, 900, 1e-3)   # quota 100 steps: nine rounds
    for q in (small, large):
        srv.submit(q)
    for _ in range(10_000):
        if srv.idle():
            break
        srv.step()
        clk.t += 1.0
    assert srv.idle()
    rounds = {0: [], 1: []}
    for tok in be.launches:
        for rid, s in tok["members"]:
            rounds[rid].append(s)
    assert rounds[0] == [900]
    assert rounds[1] == [100] * 9
    assert be.steps_done == {0: 900, 1: 900}


def test_zero_step_request_completes_at_admission():
    """A request of zero steps needs no round: it is answered as soon as it
    is admitted (before, it waited for a round that never came)."""
    be = FakeBackend()
    clk = FakeClock()
    srv = serve.Server(be, mem_budget=10**9, n_lanes=1, chunk_steps=100, clock=clk)
    srv.submit(serve.Request(0, "g", 50, 0, 1e-3))
    srv.submit(serve.Request(1, "g", 50, 120, 1e-3))
    done = srv.step()
    assert [r.rid for r in done] == [0] and done[0].error is None
    for _ in range(100):
        if srv.idle():
            break
        clk.t += 1.0
        srv.step()
    assert srv.idle() and sorted(r.rid for r in srv.results) == [0, 1]
    assert all(rid != 0 for tok in be.launches for rid, _ in tok["members"])


def test_trace_cut_off_abandons_open_requests():
    """A trace cut off at its time limit (partial=True) returns the answered
    requests, releases every admitted one and leaves nothing queued; without
    partial it raises."""
    be = FakeBackend(delay_polls=3)
    clk = FakeClock()

    class TickingServer(serve.Server):
        def step(self):
            clk.t += 1.0  # every pass costs a second of the fake clock
            return super().step()

    reqs = _reqs(30, seed=4)
    for q in reqs:
        q.arrival = 0.0
    srv = TickingServer(be, mem_budget=60_000, n_lanes=2, chunk_steps=200, clock=clk)
    res = srv.run_trace(reqs, time_limit=300.0, poll=0.0, partial=True)
    assert 0 < len(res) < len(reqs)
    assert srv.idle() and srv.reserved == 0 and not be.live
    assert all(l is None for l in srv.lanes)
    srv2 = TickingServer(FakeBackend(delay_polls=3), mem_budget=60_000, n_lanes=2,
                         chunk_steps=200, clock=clk)
    for q in reqs:
        q.arrival = 0.0
    with pytest.raises(TimeoutError):
        srv2.run_trace(reqs, time_limit=40.0, poll=0.0)
