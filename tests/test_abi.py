"""The C ABI library builds for sm_103a, loads, exports every entry point that
include/mg.h declares, and rejects invalid graph descriptions before touching
the GPU (no compute call is made here)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "mg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z_]+)\s*\(", txt)) - {"mg_alloc_fn", "mg_free_fn"})


def test_library_exports_declared_symbols():
    from paper_2512_02175_gb300 import binding as B
    lib = B.load()
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(B.SYMBOLS) == declared
    assert "sm_103a" in B.mg_version()


def _desc(**over):
    d = dict(n_vertices=2, src=[0], dst=[1], length=[1.0], c0=[0.0], c1=[0.0], sigma=[1.0],
             w_init=[1.0], w_term=[1.0])
    d.update(over)
    return d


@pytest.mark.parametrize("bad", [
    dict(src=[2]), dict(dst=[5]), dict(length=[0.0]), dict(length=[float("nan")]),
    dict(length=[float("inf")]), dict(sigma=[-1.0]), dict(c0=[float("inf")]),
    dict(w_init=[-0.5]), dict(w_init=[0.0]), dict(hist_range=[0.0]), dict(kind=[0, 3]),
    dict(n_vertices=0),
])
def test_invalid_graph_rejected_on_host(bad):
    from paper_2512_02175_gb300 import binding as B
    with pytest.raises(B.MGError) as ei:
        B.mg_graph_create(_desc(**bad))
    assert ei.value.status == B.MG_ERR_INVALID_ARG
    assert B.mg_last_error()


def test_null_handles_rejected():
    from paper_2512_02175_gb300 import binding as B
    with pytest.raises(B.MGError):
        B.mg_simulate(None, 1e-3, 10, 4)
    with pytest.raises(B.MGError):
        B.mg_synchronize(None)
