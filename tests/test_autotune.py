"""The autotuner's search and cache on the CPU (timing function injected)."""
from paper_2512_02175_gb300 import autotune as A


def test_search_picks_fastest_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    calls = []

    def trial(t):
        calls.append(t)
        # a made-up cost surface with its minimum at (2, 16 KiB, 3)
        return abs(t.split_batch - 2) + (0 if t.stage_limit_bytes == 16384 else 1) + \
            (0 if t.blocks_per_sm == 3 else 0.5) + 1.0

    best = A.tune("k", trial, path=path)
    assert best == A.Tuning(2, 16384, 3)
    n = len(calls)
    assert n == len(A.DEFAULT_CANDIDATES["split_batch"]) * 3 * 2
    again = A.tune("k", trial, path=path)  # from the cache: no new trials
    assert again == best and len(calls) == n
    fresh = A.tune("k", trial, path=path, refresh=True)
    assert fresh == best and len(calls) == 2 * n


def test_size_class():
    assert A.size_class(1 << 20, 5000, 512) == "n2^20-e2^12-m2^9"
