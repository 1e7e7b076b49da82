"""mg_histogram_static: the host-output histogram that allocates no device
memory, for callers that cannot let a library allocate (fixed memory budgets,
code that must not synchronise the device through cudaMalloc/cudaFree, or an
allocator hook that is not safe to call there).  Its counts must equal those
of mg_histogram, the entry point that stages them in memory it allocates,
and they must stay right on a second call, since all calls share one static
array that keeps the previous call's contents.  This file is collected last
so that, run with -x, every other test has run before it."""
import numpy as np
import pytest

from paper_2512_02175_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_static_histogram_equals_allocating_one(prec):
    import torch
    assert torch.cuda.is_available()
    from paper_2512_02175_gb300 import binding as B
    B.load()
    d = W.star_langevin(16)
    e, x = W.uniform_on_edges(d, 200_000, 7)
    g = B.Graph(d)
    p = B.Particles(g, e, x, seed=1, precision=prec)
    bins = 32
    for call in range(2):  # two calls in a row: the shared array is cleared each time
        p.simulate(1e-3, 50, 16)
        ref = p.histogram(bins)
        got = np.zeros(g.n_edges * bins, np.uint32)
        B.mg_histogram_static(p.h, bins, got)
        assert np.array_equal(got, ref), call
        assert got.sum() == 200_000
    # a different (smaller) shape after a larger one: nothing stale leaks in
    got = np.zeros(g.n_edges * 4, np.uint32)
    B.mg_histogram_static(p.h, 4, got)
    assert np.array_equal(got, p.histogram(4))
    # beyond the static limit: rejected, not truncated
    with pytest.raises(B.MGError) as ei:
        B.mg_histogram_static(p.h, (1 << 20) // 16 + 1, np.zeros(16 * ((1 << 20) // 16 + 1), np.uint32))
    assert ei.value.status == B.MG_ERR_INVALID_ARG
    p.close()
    g.close()
