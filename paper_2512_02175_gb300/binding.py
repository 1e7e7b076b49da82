"""ctypes binding of libmetricgraph (C ABI in ``include/mg.h``).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  Functions keep the C names (``mg_graph_create``, ``mg_simulate``,
...); a failing call raises ``MGError`` with the library's message.  If the
library cannot be loaded the import of this module raises: there is no CPU
fallback.

Device arrays may be passed as torch CUDA tensors (their data pointers are
handed to the library); host arrays as numpy arrays or CPU tensors.  Device
memory the library allocates comes from torch's caching allocator once
``use_torch_allocator()`` has been called (PyTorch provides device memory and
streams; the library does the work).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

MG_OK, MG_ERR_INVALID_ARG, MG_ERR_OUT_OF_MEMORY, MG_ERR_CUDA = 0, 1, 2, 3
MG_ERR_TIMEOUT, MG_ERR_CANCELLED, MG_ERR_BUSY, MG_ERR_DEVICE_FAULT = 4, 5, 6, 7
MG_FP64, MG_FP32_MIXED, MG_FP32 = 0, 1, 2
MG_VERTEX_STANDARD, MG_VERTEX_ABSORBING = 0, 1
_NAMES = {0: "MG_OK", 1: "MG_ERR_INVALID_ARG", 2: "MG_ERR_OUT_OF_MEMORY", 3: "MG_ERR_CUDA",
          4: "MG_ERR_TIMEOUT", 5: "MG_ERR_CANCELLED", 6: "MG_ERR_BUSY",
          7: "MG_ERR_DEVICE_FAULT"}


class MGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_NAMES.get(status, status)}: {msg}")
        self.status = status


class mg_graph_desc(C.Structure):
    _fields_ = [
        ("n_vertices", C.c_int32), ("n_edges", C.c_int32),
        ("edge_src", C.POINTER(C.c_int32)), ("edge_dst", C.POINTER(C.c_int32)),
        ("length", C.POINTER(C.c_double)), ("drift_c0", C.POINTER(C.c_double)),
        ("drift_c1", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
        ("weight_init", C.POINTER(C.c_double)), ("weight_term", C.POINTER(C.c_double)),
        ("hist_range", C.POINTER(C.c_double)), ("vertex_kind", C.POINTER(C.c_uint8)),
        ("sigma_slope", C.POINTER(C.c_double)),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

# every symbol the C ABI declares (checked against include/mg.h by the tests)
SYMBOLS = [
    "mg_set_allocator", "mg_graph_create", "mg_graph_destroy", "mg_graph_info", "mg_graph_slots",
    "mg_particles_init", "mg_particles_reset", "mg_particles_destroy", "mg_particles_set_tuning",
    "mg_simulate_sampled", "mg_histogram_binned",
    "mg_simulate",
    "mg_synchronize", "mg_histogram", "mg_histogram_static", "mg_exit_counts", "mg_counters_reset", "mg_state_get",
    "mg_state_set", "mg_particles_info", "mg_hit_root", "mg_last_error", "mg_version",
    "mg_batch_create", "mg_batch_add", "mg_batch_clear", "mg_batch_set_tuning", "mg_batch_run",
    "mg_batch_info", "mg_batch_destroy",
]

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library; raises if impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libmetricgraph not built at {path}")
        lib = C.CDLL(path)
        _declare(lib)
        _lib = lib
        return lib


def _declare(L):
    vp, i32, i64, u32, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
    st = C.c_int
    sig = {
        "mg_set_allocator": ([ALLOC_FN, FREE_FN, vp], st),
        "mg_graph_create": ([C.POINTER(mg_graph_desc), C.POINTER(vp)], st),
        "mg_graph_destroy": ([vp], st),
        "mg_graph_info": ([vp, vp, vp, vp], st),
        "mg_graph_slots": ([vp, vp, vp, vp, vp], st),
        "mg_particles_init": ([vp, i64, vp, vp, C.c_int, u32, u64, u32, C.c_int, vp, C.POINTER(vp)], st),
        "mg_particles_reset": ([vp, vp, vp, C.c_int, vp], st),
        "mg_particles_destroy": ([vp], st),
        "mg_particles_set_tuning": ([vp, i32, i64, i32], st),
        "mg_simulate": ([vp, dbl, i64, i32, i32, vp, vp], st),
        "mg_simulate_sampled": ([vp, dbl, i64, i32, i64, i32, vp, vp], st),
        "mg_histogram_binned": ([vp, vp, vp, vp, C.c_int, vp], st),
        "mg_synchronize": ([vp], st),
        "mg_histogram": ([vp, i32, vp, C.c_int, vp], st),
        "mg_histogram_static": ([vp, i32, vp, vp], st),
        "mg_exit_counts": ([vp, vp, vp, vp, vp, vp], st),
        "mg_counters_reset": ([vp, vp], st),
        "mg_state_get": ([vp, vp, vp, vp, vp, vp, vp, vp, vp], st),
        "mg_state_set": ([vp, vp, vp, vp, vp, vp, vp, u64, vp], st),
        "mg_particles_info": ([vp, vp, vp, vp], st),
        "mg_batch_create": ([C.POINTER(vp)], st),
        "mg_batch_add": ([vp, vp, dbl, i64, i32, i32, vp], st),
        "mg_batch_clear": ([vp], st),
        "mg_batch_set_tuning": ([vp, i32, i64, i32], st),
        "mg_batch_run": ([vp, C.c_int, vp], st),
        "mg_batch_info": ([vp, vp, vp, vp], st),
        "mg_batch_destroy": ([vp], st),
        "mg_last_error": ([], C.c_char_p),
        "mg_hit_root": ([i32, i64, vp, vp, vp, vp, vp], st),
        "mg_version": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res


def _check(status: int):
    if status != MG_OK:
        raise MGError(status, load().mg_last_error().decode(errors="replace"))


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _on_device(a) -> int:
    return int(bool(getattr(a, "is_cuda", False)))


# Sizes the library reads or writes through caller pointers are checked here,
# where the arrays' lengths are known (the C ABI sees bare pointers).  The
# graph sizes (V, E, S) of every particle set created through this module:
_set_sizes: dict[int, tuple[int, int, int]] = {}


def _sizes(p):
    """(V, E, S) of particle set p's graph, or None if it was not created here."""
    return _set_sizes.get(getattr(p, "value", None))


def _host_in(a, dtype, n, what):
    """A C-contiguous host array of `dtype` with exactly n entries."""
    if _on_device(a):
        raise ValueError(f"{what} must be a host array")
    a = np.ascontiguousarray(a, dtype=dtype)
    if a.ndim != 1 or (n is not None and a.size != n):
        raise ValueError(f"{what} must be 1-D with {n} entries (got shape {a.shape})")
    return a


def _host_out(a, dtype, n, what):
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"] \
            or not a.flags["WRITEABLE"]:
        raise ValueError(f"{what} must be a writeable C-contiguous {np.dtype(dtype).name} host array")
    if n is not None and a.size < n:
        raise ValueError(f"{what} needs at least {n} entries (got {a.size})")
    return a


def _device_arr(t, dtypes, n, what, exact=False):
    """A contiguous CUDA tensor on the current device, of one of `dtypes`
    (names), with n entries (at least n unless exact)."""
    import torch
    if not _on_device(t):
        raise ValueError(f"{what} must be a CUDA tensor")
    if str(t.dtype).replace("torch.", "") not in dtypes:
        raise ValueError(f"{what} must have dtype {' or '.join(dtypes)} (got {t.dtype})")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{what} is on {t.device}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")
    if n is not None and (t.numel() != n if exact else t.numel() < n):
        raise ValueError(f"{what} needs {'exactly' if exact else 'at least'} {n} entries "
                         f"(got {t.numel()})")
    return t


_U32 = ("int32", "uint32")


def _hist_dev(p, bins, out, what="hist_out"):
    sz = _sizes(p)
    return _device_arr(out, _U32, None if sz is None else sz[1] * int(bins), what)


def _positions(edge0, x0, n):
    """edge0 (int32) and x0 (float64) with n entries each, both host or both
    device; returns (edge0, x0, on_device)."""
    on_dev = _on_device(x0)
    if _on_device(edge0) != on_dev:
        raise ValueError("edge0 and x0 must both be host or both be device arrays")
    if on_dev:
        return (_device_arr(edge0, ("int32",), n, "edge0", exact=True),
                _device_arr(x0, ("float64",), n, "x0", exact=True), 1)
    return _host_in(edge0, np.int32, n, "edge0"), _host_in(x0, np.float64, n, "x0"), 0


# -------------------------------------------------------------- allocator

_torch_hooks = None


def use_torch_allocator():
    """Route the library's device allocations to torch's caching allocator."""
    global _torch_hooks
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream or 0)
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(load().mg_set_allocator(hooks[0], hooks[1], None))
    _torch_hooks = hooks  # keep the callbacks alive


def use_cuda_allocator():
    global _torch_hooks
    _check(load().mg_set_allocator(ALLOC_FN(), FREE_FN(), None))
    _torch_hooks = None


# ------------------------------------------------------------------ graph

def _desc_struct(d):
    keep = []

    def arr(key, dtype, ctype, optional=False):
        v = d.get(key)
        if v is None:
            if optional:
                return None
            raise ValueError(f"graph description lacks {key}")
        a = np.ascontiguousarray(v, dtype=dtype)
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(ctype))

    s = mg_graph_desc()
    s.n_vertices = int(d["n_vertices"])
    s.n_edges = int(len(d["src"]))
    s.edge_src = arr("src", np.int32, C.c_int32)
    s.edge_dst = arr("dst", np.int32, C.c_int32)
    s.length = arr("length", np.float64, C.c_double)
    s.drift_c0 = arr("c0", np.float64, C.c_double)
    s.drift_c1 = arr("c1", np.float64, C.c_double)
    s.sigma = arr("sigma", np.float64, C.c_double)
    s.weight_init = arr("w_init", np.float64, C.c_double)
    s.weight_term = arr("w_term", np.float64, C.c_double)
    s.hist_range = arr("hist_range", np.float64, C.c_double, optional=True)
    s.vertex_kind = arr("kind", np.uint8, C.c_uint8, optional=True)
    if d.get("sigma1") is not None:  # position-dependent diffusion sigma + sigma1 x
        d = dict(d, sigma1=np.broadcast_to(np.asarray(d["sigma1"], np.float64), (s.n_edges,)))
    s.sigma_slope = arr("sigma1", np.float64, C.c_double, optional=True)
    return s, keep


def mg_graph_create(desc: dict):
    s, keep = _desc_struct(desc)
    h = C.c_void_p()
    _check(load().mg_graph_create(C.byref(s), C.byref(h)))
    return h


def mg_graph_destroy(g):
    _check(load().mg_graph_destroy(g))


def mg_graph_info(g):
    V, E, S = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().mg_graph_info(g, C.byref(V), C.byref(E), C.byref(S)))
    return V.value, E.value, S.value


def mg_graph_slots(g):
    V, E, S = mg_graph_info(g)
    off = np.zeros(V + 1, np.int32)
    se = np.zeros(S, np.int32)
    send = np.zeros(S, np.uint8)
    T = np.zeros(S, np.uint64)
    _check(load().mg_graph_slots(g, _ptr(off), _ptr(se), _ptr(send), _ptr(T)))
    return off, se, send, T


# -------------------------------------------------------------- particles

def mg_particles_init(g, edge0, x0, *, pid_base=0, seed=0, instance=0, precision=MG_FP64,
                      stream=None):
    """edge0 (int32) and x0 (float64): numpy/CPU arrays or CUDA tensors."""
    edge0, x0, on_dev = _positions(edge0, x0, len(x0))
    sizes = mg_graph_info(g)
    h = C.c_void_p()
    _check(load().mg_particles_init(g, len(x0), _ptr(edge0), _ptr(x0), on_dev, pid_base, seed,
                                    instance, precision, _stream_ptr(stream), C.byref(h)))
    _set_sizes[h.value] = sizes
    return h


def mg_particles_reset(p, edge0, x0, stream=None):
    n = mg_particles_info(p)[0]
    edge0, x0, on_dev = _positions(edge0, x0, n)
    _check(load().mg_particles_reset(p, _ptr(edge0), _ptr(x0), on_dev, _stream_ptr(stream)))


def mg_particles_destroy(p):
    _check(load().mg_particles_destroy(p))
    _set_sizes.pop(getattr(p, "value", None), None)


def mg_particles_set_tuning(p, split_batch=0, steps_per_launch=0, max_blocks=0):
    _check(load().mg_particles_set_tuning(p, int(split_batch), int(steps_per_launch),
                                          int(max_blocks)))


def mg_particles_info(p):
    n, prec, step = C.c_int64(), C.c_int32(), C.c_uint64()
    _check(load().mg_particles_info(p, C.byref(n), C.byref(prec), C.byref(step)))
    return n.value, prec.value, step.value


def mg_simulate(p, dt, steps, M, hist_bins=0, hist_out=None, stream=None):
    if int(hist_bins) > 0:
        _hist_dev(p, hist_bins, hist_out)
    _check(load().mg_simulate(p, float(dt), int(steps), int(M), int(hist_bins), _ptr(hist_out),
                              _stream_ptr(stream)))


def mg_simulate_sampled(p, dt, steps, M, every, hist_bins, hist_out, stream=None):
    if int(hist_bins) > 0:
        _hist_dev(p, hist_bins, hist_out)
    _check(load().mg_simulate_sampled(p, float(dt), int(steps), int(M), int(every),
                                      int(hist_bins), _ptr(hist_out), _stream_ptr(stream)))


def mg_synchronize(p):
    _check(load().mg_synchronize(p))


def mg_histogram(p, bins, out=None, stream=None):
    """Returns a numpy uint32 [E * bins] histogram, or fills the CUDA tensor
    ``out`` (stream-ordered)."""
    if out is not None and _on_device(out):
        _hist_dev(p, bins, out, "out")
        _check(load().mg_histogram(p, int(bins), _ptr(out), 1, _stream_ptr(stream)))
        return out
    if out is None:
        raise ValueError("pass a host output array (numpy uint32 [E * bins]) or a CUDA tensor")
    sz = _sizes(p)
    _host_out(out, np.uint32, None if sz is None else sz[1] * int(bins), "out")
    _check(load().mg_histogram(p, int(bins), _ptr(out), 0, _stream_ptr(stream)))
    return out


def mg_histogram_binned(p, bin_offsets, bin_upper, out, stream=None):
    """Variable-width bins: bin_offsets int32 [E + 1], bin_upper float64
    [bin_offsets[-1]]; fills ``out`` (numpy uint32 or a CUDA tensor) with the
    counts (see include/mg.h)."""
    sz = _sizes(p)
    off = _host_in(bin_offsets, np.int32, None if sz is None else sz[1] + 1, "bin_offsets")
    if off.size < 1:
        raise ValueError("bin_offsets must have n_edges + 1 entries")
    up = _host_in(bin_upper, np.float64, None, "bin_upper")
    if len(up) != int(off[-1]):
        raise ValueError("bin_upper must have bin_offsets[-1] entries")
    dev = 1 if _on_device(out) else 0
    if dev:
        _device_arr(out, _U32, max(0, int(off[-1])), "out")
    else:
        _host_out(out, np.uint32, max(0, int(off[-1])), "out")
    _check(load().mg_histogram_binned(p, _ptr(off), _ptr(up), _ptr(out), dev, _stream_ptr(stream)))
    return out


def mg_histogram_static(p, bins, out, stream=None):
    """The snapshot histogram into the host array ``out`` (uint32 [E * bins])
    without any device allocation by the library (see include/mg.h)."""
    sz = _sizes(p)
    _host_out(out, np.uint32, None if sz is None else sz[1] * int(bins), "out")
    _check(load().mg_histogram_static(p, int(bins), _ptr(out), _stream_ptr(stream)))
    return out


def mg_hit_root(mode, A, B, C, s, stream=None):
    """Hitting-fraction roots of the coefficient triples (A, B, C) (CUDA
    float32 tensors of one length) into ``s`` (CUDA float64 tensor) by the
    device function of precision mode ``mode`` (see include/mg.h)."""
    n = int(A.numel())
    for t, what in ((A, "A"), (B, "B"), (C, "C")):
        _device_arr(t, ("float32",), n, what, exact=True)
    _device_arr(s, ("float64",), n, "s", exact=True)
    _check(load().mg_hit_root(int(mode), n, _ptr(A), _ptr(B), _ptr(C), _ptr(s),
                              _stream_ptr(stream)))
    return s


def mg_exit_counts(p, n_slots, n_vertices, stream=None):
    sz = _sizes(p)
    if sz is not None and (int(n_slots), int(n_vertices)) != (sz[2], sz[0]):
        raise ValueError(f"the set's graph has {sz[2]} slots and {sz[0]} vertices")
    ex = np.zeros(n_slots, np.uint64)
    ab = np.zeros(n_vertices, np.uint64)
    tr = np.zeros(1, np.uint64)
    ps = np.zeros(1, np.uint64)
    _check(load().mg_exit_counts(p, _ptr(ex), _ptr(ab), _ptr(tr), _ptr(ps), _stream_ptr(stream)))
    return dict(exits=ex, absorbed=ab, truncations=int(tr[0]), particle_steps=int(ps[0]))


def mg_counters_reset(p, stream=None):
    _check(load().mg_counters_reset(p, _stream_ptr(stream)))


def mg_state_get(p, stream=None):
    n, _, _ = mg_particles_info(p)
    edge = np.zeros(n, np.int32)
    x = np.zeros(n, np.float64)
    nd = np.zeros(n, np.uint32)
    hits = np.zeros(n, np.uint32)
    fh = np.zeros(n, np.uint32)
    fl = np.zeros(n, np.uint32)
    step = C.c_uint64()
    _check(load().mg_state_get(p, _ptr(edge), _ptr(x), _ptr(nd), _ptr(hits), _ptr(fh), _ptr(fl),
                               C.byref(step), _stream_ptr(stream)))
    return dict(edge=edge, x=x, n_draw=nd, hits=hits, first_hits=fh, flags=fl, step=step.value)


def mg_state_set(p, state, stream=None):
    n = mg_particles_info(p)[0]
    a = {k: _host_in(state[k], dt, n, k) for k, dt in
         [("edge", np.int32), ("x", np.float64), ("n_draw", np.uint32), ("hits", np.uint32),
          ("first_hits", np.uint32), ("flags", np.uint32)]}
    _check(load().mg_state_set(p, _ptr(a["edge"]), _ptr(a["x"]), _ptr(a["n_draw"]), _ptr(a["hits"]),
                               _ptr(a["first_hits"]), _ptr(a["flags"]), int(state["step"]),
                               _stream_ptr(stream)))


# ---------------------------------------------------------------- batches

def mg_batch_create():
    h = C.c_void_p()
    _check(load().mg_batch_create(C.byref(h)))
    return h


def mg_batch_add(b, p, dt, steps, M, hist_bins=0, hist_out=None):
    if int(hist_bins) > 0:
        _hist_dev(p, hist_bins, hist_out)
    _check(load().mg_batch_add(b, p, float(dt), int(steps), int(M), int(hist_bins),
                               _ptr(hist_out)))


def mg_batch_clear(b):
    _check(load().mg_batch_clear(b))


def mg_batch_set_tuning(b, split_batch=0, stage_limit_bytes=-1, blocks_per_sm=0):
    _check(load().mg_batch_set_tuning(b, int(split_batch), int(stage_limit_bytes),
                                      int(blocks_per_sm)))


def mg_batch_run(b, use_graph=False, stream=None):
    _check(load().mg_batch_run(b, int(bool(use_graph)), _stream_ptr(stream)))


def mg_batch_info(b):
    m, it, bl = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().mg_batch_info(b, C.byref(m), C.byref(it), C.byref(bl)))
    return m.value, it.value, bl.value


def mg_batch_destroy(b):
    _check(load().mg_batch_destroy(b))


class Batch:
    """Owns an mg_batch handle; keeps its members (Particles) alive."""

    def __init__(self):
        self.h = mg_batch_create()
        self.members = []

    def add(self, parts, dt, steps, M, hist_bins=0, hist_out=None):
        mg_batch_add(self.h, parts.h, dt, steps, M, hist_bins, hist_out)
        self.members.append((parts, hist_out))

    def clear(self):
        mg_batch_clear(self.h)
        self.members = []

    def set_tuning(self, split_batch=0, stage_limit_bytes=-1, blocks_per_sm=0):
        mg_batch_set_tuning(self.h, split_batch, stage_limit_bytes, blocks_per_sm)

    def run(self, use_graph=False, stream=None):
        mg_batch_run(self.h, use_graph, stream)

    def info(self):
        return mg_batch_info(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            mg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mg_version() -> str:
    return load().mg_version().decode()


def mg_last_error() -> str:
    return load().mg_last_error().decode(errors="replace")


# ----------------------------------------------------- convenience classes

class Graph:
    """Owns an mg_graph handle."""

    def __init__(self, desc: dict):
        self.desc = desc
        self.h = mg_graph_create(desc)
        self.n_vertices, self.n_edges, self.n_slots = mg_graph_info(self.h)

    def slots(self):
        return mg_graph_slots(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            mg_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Particles:
    """Owns an mg_particles handle on a Graph."""

    def __init__(self, graph: Graph, edge0, x0, *, pid_base=0, seed=0, instance=0,
                 precision=MG_FP64, stream=None):
        self.graph = graph
        self.n = len(x0)
        self.precision = precision
        self.h = mg_particles_init(graph.h, edge0, x0, pid_base=pid_base, seed=seed,
                                   instance=instance, precision=precision, stream=stream)

    def set_tuning(self, split_batch=0, steps_per_launch=0, max_blocks=0):
        mg_particles_set_tuning(self.h, split_batch, steps_per_launch, max_blocks)

    def simulate(self, dt, steps, M, hist_bins=0, hist_out=None, stream=None):
        mg_simulate(self.h, dt, steps, M, hist_bins, hist_out, stream)

    def simulate_sampled(self, dt, steps, M, every, hist_bins, hist_out, stream=None):
        mg_simulate_sampled(self.h, dt, steps, M, every, hist_bins, hist_out, stream)

    def synchronize(self):
        mg_synchronize(self.h)

    def histogram(self, bins, out=None, stream=None):
        if out is None:
            out = np.zeros(self.graph.n_edges * bins, np.uint32)
        return mg_histogram(self.h, bins, out, stream)

    def histogram_binned(self, bin_offsets, bin_upper, out=None, stream=None):
        if out is None:
            out = np.zeros(max(1, int(np.asarray(bin_offsets)[-1])), np.uint32)
        return mg_histogram_binned(self.h, bin_offsets, bin_upper, out, stream)

    def counts(self, stream=None):
        return mg_exit_counts(self.h, self.graph.n_slots, self.graph.n_vertices, stream)

    def state(self, stream=None):
        return mg_state_get(self.h, stream)

    def set_state(self, state, stream=None):
        mg_state_set(self.h, state, stream)

    def reset(self, edge0, x0, stream=None):
        mg_particles_reset(self.h, edge0, x0, stream)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            mg_particles_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
