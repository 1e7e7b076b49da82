"""Autotuner for batched launches.

Picks the launch tuning of a batch -- split batch (pending vertex hits a
warp collects before resolving them), the size limit under which a member's
graph tables are staged in shared memory, and persistent blocks per SM -- by
timing short trial runs of the batch itself, and remembers the choice in a
JSON cache keyed by (GPU name, precision, size class of the batch).  The
results of a run never depend on the tuning (tested), only its speed does.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import threading
from dataclasses import dataclass

DEFAULT_CANDIDATES = dict(
    # 0: the precision's own default (5 pending lanes for FP32-mixed, 3 for
    # FP32, 2 for FP64)
    split_batch=(0, 1, 2, 4),
    stage_limit_bytes=(0, 16 * 1024, -1),
    blocks_per_sm=(0, 3),
)

_lock = threading.Lock()


@dataclass(frozen=True)
class Tuning:
    split_batch: int = 0
    stage_limit_bytes: int = -1
    blocks_per_sm: int = 0

    def as_dict(self):
        return dict(split_batch=self.split_batch, stage_limit_bytes=self.stage_limit_bytes,
                    blocks_per_sm=self.blocks_per_sm)


def cache_path() -> str:
    base = os.environ.get("MG_TUNING_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "metricgraph", "tuning.json")


def size_class(n_particles: int, n_edges_max: int, n_members: int) -> str:
    """Coarse key: powers of two of the particle count, the largest graph and
    the member count."""
    lg = lambda v: int(math.log2(max(1, v)))
    return f"n2^{lg(n_particles)}-e2^{lg(n_edges_max)}-m2^{lg(n_members)}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(key: str, tuning: Tuning, seconds: float, path: str | None = None):
    path = path or cache_path()
    with _lock:
        data = load_cache(path)
        data[key] = dict(tuning.as_dict(), seconds=seconds)
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def lookup(key: str, path: str | None = None) -> Tuning | None:
    rec = load_cache(path).get(key)
    if not rec:
        return None
    return Tuning(rec["split_batch"], rec["stage_limit_bytes"], rec["blocks_per_sm"])


def search(trial, candidates: dict | None = None, repeats: int = 1):
    """Times ``trial(tuning) -> seconds`` for every candidate combination
    and returns (best tuning, its time, all timings).  ``trial`` must run the
    same work each time."""
    cand = dict(DEFAULT_CANDIDATES)
    cand.update(candidates or {})
    timings = []
    for sb, sl, bps in itertools.product(cand["split_batch"], cand["stage_limit_bytes"],
                                         cand["blocks_per_sm"]):
        t = Tuning(sb, sl, bps)
        best = min(trial(t) for _ in range(max(1, repeats)))
        timings.append((t, best))
    tbest, sbest = min(timings, key=lambda kv: kv[1])
    return tbest, sbest, timings


def tune(key: str, trial, candidates: dict | None = None, refresh: bool = False,
         path: str | None = None) -> Tuning:
    """Cached search: returns the stored tuning for ``key`` unless ``refresh``."""
    if not refresh:
        t = lookup(key, path)
        if t is not None:
            return t
    tbest, sbest, _ = search(trial, candidates)
    store(key, tbest, sbest, path)
    return tbest
