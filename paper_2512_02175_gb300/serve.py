"""Served simulation requests with continuous batching.

A request asks for ``steps`` EM-Steps of ``n`` particles on one of the
server's resident graphs.  The server

* admits requests in arrival order while their device memory (particle state
  and histogram) fits a budget; later ones wait;
* keeps admitted requests resident and advances them in rounds: each round is
  one batched launch (``mg_batch``) over the admitted requests that are not
  already in flight, each taking the next part of its remaining steps --
  ``chunk_steps``, or more for a small request, up to ``round_work``
  particle-steps -- so requests that arrive while others run join at the
  next round, and a small request is done in one round;
* runs rounds on several streams at once, so the work of different rounds
  overlaps on the device;
* returns a request's histogram and counters when its last round completes,
  and records arrival, admission and completion times for p50/p99 latency;
* fails a single request -- one whose admission or collection raises, e.g.
  on invalid starting positions or a device error of its own particle set --
  with its error in the result, and keeps serving the others.

Every particle's draws depend only on (seed, instance = request id, particle
id) and chunking a run into rounds is bit-exact, so a request's result is the
same alone and in any mix.  The scheduling policy is host logic over a small
backend interface: ``GpuBackend`` drives the CUDA library; tests also use a
fake backend to check admission and scheduling without a GPU.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    graph: str
    n: int
    steps: int
    dt: float
    M: int = 16
    bins: int = 16
    edge0: np.ndarray | None = None
    x0: np.ndarray | None = None
    arrival: float = 0.0


@dataclass
class Result:
    rid: int
    hist: np.ndarray
    counts: dict
    state: dict | None
    arrival: float
    admitted: float
    finished: float
    particle_steps: int
    error: str | None = None  # set when the request failed (then hist is None)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Active:
    req: Request
    handle: object
    remaining: int
    admitted: float
    in_flight: bool = False


class Server:
    def __init__(self, backend, mem_budget: int, n_lanes: int = 2, chunk_steps: int = 500,
                 max_members: int = 512, clock=time.perf_counter, keep_state=False,
                 round_work: int = 0):
        """keep_state: return every request's final particle state (True), none
        (False), or those of the request ids in a given set.  A member takes
        max(chunk_steps, round_work // n) of its remaining steps per round
        (round_work = 0: chunk_steps)."""
        self.backend = backend
        self.mem_budget = int(mem_budget)
        self.n_lanes = n_lanes
        self.chunk_steps = int(chunk_steps)
        self.round_work = int(round_work)
        self.max_members = max_members
        self.clock = clock
        self.keep_state = keep_state
        self.queue: collections.deque[Request] = collections.deque()
        self.active: list[_Active] = []
        self.reserved = 0
        self.lanes: list[tuple[object, list[tuple[_Active, int]]] | None] = [None] * n_lanes
        self.results: list[Result] = []
        self.peak_reserved = 0

    # ------------------------------------------------------------ intake
    def submit(self, req: Request):
        if self.backend.bytes_of(req) > self.mem_budget:
            raise ValueError(f"request {req.rid} needs more memory than the whole budget")
        self.queue.append(req)

    def idle(self) -> bool:
        return not self.queue and not self.active

    # ---------------------------------------------------------- one pass
    def step(self) -> list[Result]:
        done = self._complete()
        done += self._admit()
        self._launch()
        return done

    def _failed(self, req: Request, admitted: float, ex: Exception) -> Result:
        res = Result(req.rid, None, {}, None, req.arrival, admitted, self.clock(), 0,
                     error=f"{type(ex).__name__}: {ex}")
        self.results.append(res)
        return res

    def _complete(self) -> list[Result]:
        out = []
        for k, lane in enumerate(self.lanes):
            if lane is None:
                continue
            token, members = lane
            if not self.backend.poll(token):
                continue
            self.lanes[k] = None
            for act, _ in members:
                act.in_flight = False
                if act.remaining == 0:
                    out.extend(self._finish(act))
        return out

    def _finish(self, act: _Active) -> list[Result]:
        """Collect a request whose steps are all done, and release it."""
        keep = (act.req.rid in self.keep_state
                if isinstance(self.keep_state, (set, frozenset)) else bool(self.keep_state))
        r = act.req
        try:
            hist, counts, state = self.backend.collect(act.handle, keep)
        except Exception as ex:  # this request's failure, not the server's
            return [self._failed(r, act.admitted, ex)]
        else:
            res = Result(r.rid, hist, counts, state, r.arrival, act.admitted,
                         self.clock(), int(counts.get("particle_steps", r.n * r.steps)))
            self.results.append(res)
            return [res]
        finally:
            self.backend.release(act.handle)
            self.reserved -= self.backend.bytes_of(r)
            self.active.remove(act)

    def _admit(self) -> list[Result]:
        failed = []
        while self.queue:
            req = self.queue[0]
            need = self.backend.bytes_of(req)
            if self.reserved + need > self.mem_budget:
                break
            self.queue.popleft()
            try:
                handle = self.backend.admit(req)
            except Exception as ex:  # e.g. starting positions off their edges
                failed.append(self._failed(req, self.clock(), ex))
                continue
            self.reserved += need
            self.peak_reserved = max(self.peak_reserved, self.reserved)
            self.active.append(_Active(req, handle, req.steps, self.clock()))
        # a request of zero steps is done as admitted
        for act in [a for a in self.active if a.remaining == 0 and not a.in_flight]:
            failed.extend(self._finish(act))
        return failed

    def _launch(self):
        for k in range(self.n_lanes):
            if self.lanes[k] is not None:
                continue
            ready = [a for a in self.active if not a.in_flight and a.remaining > 0]
            if not ready:
                return
            members = []
            for a in ready[: self.max_members]:
                quota = max(self.chunk_steps, self.round_work // max(1, a.req.n))
                now = min(quota, a.remaining)
                a.remaining -= now
                a.in_flight = True
                members.append((a, now))
            token = self.backend.launch(k, [(a.handle, s) for a, s in members])
            self.lanes[k] = (token, members)

    # ------------------------------------------------------- trace replay
    def abandon(self):
        """Waits for the rounds in flight, then releases every admitted
        request unanswered and drops the queue (a trace cut off at its time
        limit)."""
        for k, lane in enumerate(self.lanes):
            if lane is not None:
                token, _ = lane
                while not self.backend.poll(token):
                    time.sleep(1e-4)
                self.lanes[k] = None
        for act in list(self.active):
            self.backend.release(act.handle)
            self.reserved -= self.backend.bytes_of(act.req)
            self.active.remove(act)
        self.queue.clear()

    def run_trace(self, requests: list[Request], time_limit: float = 600.0, poll: float = 5e-5,
                  partial: bool = False):
        """Replays requests whose ``arrival`` is in seconds from the start,
        in real time, until every request has completed; a pass that finds
        nothing to do sleeps ``poll`` seconds (a round's completion is seen
        that much later at most: 50 us against 200 us took the benchmark
        trace's p50 from 1.6 to 1.3 ms).  Past ``time_limit`` seconds it
        raises TimeoutError, or with ``partial`` abandons the requests still
        open and returns the answered ones."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = self.clock()
        i = 0
        while i < len(reqs) or not self.idle():
            now = self.clock() - t0
            if now > time_limit:
                if partial:
                    self.abandon()
                    break
                raise TimeoutError("serving trace did not finish in time")
            while i < len(reqs) and reqs[i].arrival <= now:
                r = reqs[i]
                r.arrival = t0 + r.arrival
                self.submit(r)
                i += 1
            if not self.step():
                time.sleep(poll)
        return self.results


def latency_summary(results: list[Result], t_start: float | None = None,
                    t_end: float | None = None) -> dict:
    """Latency percentiles and throughput of the requests that succeeded
    (failed ones are counted apart)."""
    failed = sum(1 for r in results if r.error is not None)
    results = [r for r in results if r.error is None]
    if not results:
        return dict(requests=0, failed=failed, p50_s=None, p99_s=None, mean_s=None,
                    particle_steps=0, served_particle_steps_per_s=0.0)
    lat = np.array([r.latency for r in results])
    ps = sum(r.particle_steps for r in results)
    if t_start is None:
        t_start = min(r.arrival for r in results)
    if t_end is None:
        t_end = max(r.finished for r in results)
    return dict(requests=len(results), failed=failed, p50_s=float(np.percentile(lat, 50)),
                p99_s=float(np.percentile(lat, 99)), mean_s=float(lat.mean()),
                particle_steps=int(ps), served_particle_steps_per_s=ps / max(t_end - t_start, 1e-9))


# --------------------------------------------------------------- backends

class GpuBackend:
    """Requests on the CUDA library: one particle set per admitted request;
    one reusable mg_batch and stream per lane (a round whose members and step
    counts repeat the lane's previous round replays its captured CUDA graph);
    a request's histogram is the snapshot of its final positions, fused into
    its last round (device memory, read back through pinned host memory)."""

    def __init__(self, graphs: dict, precision: int, seed: int = 0, n_lanes: int = 2,
                 use_graph: bool = True, tuning=None):
        import torch

        from . import binding as B
        self.B = B
        self.torch = torch
        B.load()
        self.graphs = {k: B.Graph(d) for k, d in graphs.items()}
        self.precision = precision
        self.seed = seed
        self.use_graph = use_graph
        self.streams = [torch.cuda.Stream() for _ in range(n_lanes)]
        self.batches = [B.Batch() for _ in range(n_lanes)]
        self.last = [None] * n_lanes
        if tuning is not None:
            for b in self.batches:
                b.set_tuning(**tuning.as_dict())
        self.state_bytes = 28 if precision == B.MG_FP64 else 24

    def bytes_of(self, req: Request) -> int:
        g = self.graphs[req.graph]
        return req.n * self.state_bytes + g.n_edges * req.bins * 4 + 8 * (g.n_slots + g.n_vertices)

    def admit(self, req: Request):
        g = self.graphs[req.graph]
        p = self.B.Particles(g, req.edge0, req.x0, seed=self.seed, instance=req.rid,
                             precision=self.precision)
        return dict(req=req, p=p, graph=g, done=0, hist=None)

    def launch(self, lane: int, members):
        b = self.batches[lane]
        st = self.streams[lane]
        torch = self.torch
        plan = []
        for h, s in members:
            r = h["req"]
            last = r.bins > 0 and h["done"] + s == r.steps
            if last and h["hist"] is None:
                with torch.cuda.stream(st):  # zeroed in order before the round
                    h["hist"] = torch.zeros(h["graph"].n_edges * r.bins, dtype=torch.int32,
                                            device="cuda")
            plan.append((h, s, h["hist"] if last else None))
        sig = [(id(h["p"]), s, 0 if hb is None else hb.data_ptr()) for h, s, hb in plan]
        if sig != self.last[lane]:  # else: replay the lane's captured graph
            b.clear()
            for h, s, hb in plan:
                r = h["req"]
                b.add(h["p"], r.dt, s, r.M, r.bins if hb is not None else 0, hb)
            self.last[lane] = sig
        b.run(use_graph=self.use_graph, stream=st)
        for h, s, _ in plan:
            h["done"] += s
        ev = self.torch.cuda.Event()
        ev.record(st)
        return ev

    def poll(self, token) -> bool:
        return token.query()

    def collect(self, handle, keep_state: bool):
        p, r = handle["p"], handle["req"]
        p.synchronize()
        counts = p.counts()
        if handle["hist"] is not None:  # fused into the last round
            hp = self.torch.empty(handle["hist"].numel(), dtype=self.torch.int32, pin_memory=True)
            hp.copy_(handle["hist"])
            hist = hp.numpy().view(np.uint32)
        else:  # no round ran (zero steps) or no bins
            hist = p.histogram(r.bins) if r.bins > 0 else np.zeros(0, np.uint32)
        state = p.state() if keep_state else None
        return hist, counts, state

    def release(self, handle):
        for k, lane_sig in enumerate(self.last):
            if lane_sig and any(sg[0] == id(handle["p"]) for sg in lane_sig):
                self.last[k] = None
                self.batches[k].clear()
        handle["hist"] = None
        handle["p"].close()

    def close(self):
        for b in self.batches:
            b.close()
        for g in self.graphs.values():
            g.close()


def serve_plain(requests: list[Request], graphs: dict, precision: int, seed: int = 0,
                time_limit: float = 600.0, keep_state: bool = False) -> list[Result]:
    """The plain path: each request, in arrival order, as its own particle set
    and one mg_simulate launch on the default stream; requests that arrive
    while one runs wait."""
    import torch

    from . import binding as B
    B.load()
    G = {k: B.Graph(d) for k, d in graphs.items()}
    reqs = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    out = []
    for r in reqs:
        now = time.perf_counter() - t0
        if now < r.arrival:
            time.sleep(r.arrival - now)
        g = G[r.graph]
        start = time.perf_counter()
        p = B.Particles(g, r.edge0, r.x0, seed=seed, instance=r.rid, precision=precision)
        p.simulate(r.dt, r.steps, r.M)
        hist = p.histogram(r.bins)
        counts = p.counts()
        state = p.state() if keep_state else None
        p.close()
        fin = time.perf_counter()
        out.append(Result(r.rid, hist, counts, state, t0 + r.arrival, start, fin,
                          int(counts["particle_steps"])))
        if fin - t0 > time_limit:
            break
    for g in G.values():
        g.close()
    return out


def default_init(desc, n, seed):
    """Starting positions of a request: tracer injection at the inlets of a
    vascular graph, else uniform on the edges (length-weighted)."""
    from . import workloads as W
    if "inlet" in desc:
        return W.inject_at_inlets(desc, n, seed)
    return W.uniform_on_edges(desc, n, seed)


def poisson_trace(rate: float, window: float, seed: int, graphs: dict, n_range=(14, 24),
                  steps_range=(100, 5000), dt_range=(1e-4, 1e-2), bins: int = 16, M: int = 16,
                  init=None) -> list[Request]:
    """Requests arriving as a Poisson process of ``rate`` per second over
    ``window`` seconds: graph uniform over ``graphs``, n = 2^U[n_range],
    steps log-uniform in steps_range, dt log-uniform in dt_range; starting
    positions from ``init(graph_desc, n, seed)``."""
    r = np.random.Generator(np.random.PCG64(seed))
    t, out, keys = 0.0, [], sorted(graphs)
    while True:
        t += r.exponential(1.0 / rate)
        if t > window:
            break
        key = keys[int(r.integers(0, len(keys)))]
        n = int(round(2.0 ** r.uniform(*n_range)))
        steps = int(round(math.exp(r.uniform(math.log(steps_range[0]), math.log(steps_range[1])))))
        dt = float(math.exp(r.uniform(math.log(dt_range[0]), math.log(dt_range[1]))))
        rid = len(out)
        e0, x0 = init(graphs[key], n, 10_000 + rid) if init else (None, None)
        out.append(Request(rid, key, n, steps, dt, M, bins, e0, x0, t))
    return out
