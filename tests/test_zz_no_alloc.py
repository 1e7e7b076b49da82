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


def test_static_histogram_allocates_nothing():
    """The defining property: with the library on cudaMalloc, repeated calls
    on a set that never had a histogram leave the device's free memory
    unchanged, while the allocating entry point, on another such set, takes
    its 4 MiB staging buffer (the check can see an allocation)."""
    import torch
    assert torch.cuda.is_available()
    from paper_2512_02175_gb300 import binding as B
    B.load()
    B.use_cuda_allocator()
    d = W.star_langevin(16)
    e, x = W.uniform_on_edges(d, 100_000, 3)
    g = B.Graph(d)
    bins = (1 << 20) // 16  # the largest request: 2^20 counts, 4 MiB
    warm = B.Particles(g, e, x, seed=2, precision=1)
    out = np.zeros(16 * bins, np.uint32)
    B.mg_histogram_static(warm.h, bins, out)  # first call on the device: set-up
    fresh = B.Particles(g, e, x, seed=2, precision=1)
    other = B.Particles(g, e, x, seed=2, precision=1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        B.mg_histogram_static(fresh.h, bins, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert out.sum() == 100_000
    ref = other.histogram(bins)  # allocates its staging buffer
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free0
    assert np.array_equal(ref, out)
    for p in (warm, fresh, other):
        p.close()
    g.close()
