"""Runs the CPU oracle over particle ranges in a process pool (test helper).

Processes are started with ``spawn`` so that a test process that already
holds a CUDA context never forks.  Each worker builds its own oracle graph
from the (picklable) graph description.
"""
from __future__ import annotations

import atexit
import multiprocessing as mp
import os

import numpy as np

_POOL = None


def _worker(args):
    desc, edge, x, pid, seed, instance, dt, steps, M, bins, keep_state = args
    from oracle import oracle as O
    g = O.Graph.from_desc(desc)
    st = O.State(edge, x, pid)
    cnt = O.Counters(g)
    O.simulate(g, st, cnt, seed=seed, instance=instance, dt=dt, steps=steps, M=M)
    hist = O.histogram(g, st, bins) if bins else None
    if not keep_state:  # counters and histogram only (large runs)
        alive = st.edge >= 0
        occ = np.bincount(st.edge[alive], minlength=len(desc["src"]))
        return (occ, None, None, None, None, cnt.exits, cnt.absorbed,
                int(cnt.truncations[0]), int(cnt.particle_steps[0]), hist, None)
    return (st.edge, st.x, st.hits, st.first_hits, st.flags, cnt.exits, cnt.absorbed,
            int(cnt.truncations[0]), int(cnt.particle_steps[0]), hist, st.n_draw)


def _pool():
    global _POOL
    if _POOL is None:
        ctx = mp.get_context("spawn")
        _POOL = ctx.Pool(max(1, min(16, os.cpu_count() or 1)))
        atexit.register(_close)
    return _POOL


def _close():
    global _POOL
    if _POOL is not None:
        _POOL.terminate()
        _POOL.join()
        _POOL = None


def run(desc, edge, x, pid=None, *, seed, instance=0, dt, steps, M, bins=0, chunks=None,
        keep_state=True):
    """Oracle over all particles; returns a dict of state, counters, histogram
    (keep_state=False: no per-particle state; "occupancy" = living particles
    per edge, and the results of each chunk under "parts")."""
    from oracle import oracle as O
    O.build()  # once here, not racing in every worker
    n = len(edge)
    pid = np.arange(n, dtype=np.uint32) if pid is None else np.asarray(pid, np.uint32)
    desc = {k: (np.asarray(v) if not isinstance(v, (int, float)) else v) for k, v in desc.items()
            if k in ("n_vertices", "src", "dst", "length", "c0", "c1", "sigma", "w_init",
                     "w_term", "hist_range", "kind", "sigma1")}
    edge = np.asarray(edge, np.int32)
    x = np.asarray(x, np.float64)
    work = n * max(steps, 1)
    if chunks is None:
        chunks = 1 if work < 2_000_000 else min(64, max(2, work // 2_000_000))
    bounds = np.linspace(0, n, chunks + 1).astype(np.int64)
    jobs = [(desc, edge[a:b], x[a:b], pid[a:b], seed, instance, dt, steps, M, bins, keep_state)
            for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    res = [_worker(jobs[0])] if len(jobs) == 1 else _pool().map(_worker, jobs)
    if not keep_state:
        out = dict(occupancy=sum(r[0] for r in res), exits=sum(r[5] for r in res),
                   absorbed=sum(r[6] for r in res), truncations=sum(r[7] for r in res),
                   particle_steps=sum(r[8] for r in res))
        out["hist"] = sum(r[9] for r in res) if bins else None
        out["parts"] = [dict(occupancy=r[0], exits=r[5], n=int(b - a))
                        for r, (a, b) in zip(res, [(a, b) for a, b in zip(bounds[:-1], bounds[1:])
                                                   if b > a])]
        return out
    cat = lambda k: np.concatenate([r[k] for r in res])
    out = dict(edge=cat(0), x=cat(1), hits=cat(2), first_hits=cat(3), flags=cat(4),
               exits=sum(r[5] for r in res), absorbed=sum(r[6] for r in res),
               truncations=sum(r[7] for r in res), particle_steps=sum(r[8] for r in res))
    out["hist"] = sum(r[9] for r in res) if bins else None
    out["n_draw"] = cat(10)
    return out
