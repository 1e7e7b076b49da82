"""Python handle on the FP64 CPU oracle (``mg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` use it; the
library never does.  This module compiles the plain C oracle with gcc
(``-O2 -ffp-contract=off``: no fused multiply-adds, so every FP64 operation
rounds as written) and marshals numpy arrays into it.  It holds none of the
method's arithmetic itself.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_HDR = os.path.join(_HERE, "mg_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmgoracle.so")
_lock = threading.Lock()
_lib = None

DEAD = -1
END_INIT, END_TERM = 0, 1
FLAG_NEAR = 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libmgoracle.so`` (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest_src = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest_src:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


def _p(t):
    return C.POINTER(t)


def _declare(L):
    u32, i32, u64, i64, dbl, u8 = C.c_uint32, C.c_int32, C.c_uint64, C.c_int64, C.c_double, C.c_uint8
    L.or_philox4x32_10.argtypes = [_p(u32), _p(u32), _p(u32)]
    L.or_philox4x32_10.restype = None
    L.or_u01.argtypes = [u32]
    L.or_u01.restype = dbl
    L.or_box_muller.argtypes = [u32, u32, _p(dbl), _p(dbl)]
    L.or_box_muller.restype = None
    L.or_normal.argtypes = [u64, u32, u32, u32]
    L.or_normal.restype = dbl
    L.or_split_draw.argtypes = [u64, u32, u32, u32]
    L.or_split_draw.restype = u32
    L.or_graph_build.argtypes = [i32, i32, _p(i32), _p(i32), _p(dbl), _p(dbl), _p(dbl), _p(dbl),
                                 _p(dbl), _p(dbl), _p(dbl), _p(u8), C.POINTER(C.c_void_p)]
    L.or_graph_build.restype = C.c_int
    L.or_graph_set_sigma1.argtypes = [C.c_void_p, _p(dbl)]
    L.or_graph_set_sigma1.restype = C.c_int
    L.or_graph_free.argtypes = [C.c_void_p]
    L.or_graph_free.restype = None
    L.or_graph_n_slots.argtypes = [C.c_void_p]
    L.or_graph_n_slots.restype = i32
    L.or_graph_slots.argtypes = [C.c_void_p, _p(i32), _p(i32), _p(u8), _p(u64)]
    L.or_graph_slots.restype = None
    L.or_choose_slot.argtypes = [C.c_void_p, i32, u32]
    L.or_choose_slot.restype = i32
    L.or_root.argtypes = [dbl, dbl, dbl]
    L.or_root.restype = dbl
    L.or_simulate.argtypes = [C.c_void_p, i64, _p(u32), _p(i32), _p(dbl), _p(u32), _p(u32),
                              _p(u32), _p(u32), u64, u32, dbl, i64, i32, _p(u64), _p(u64),
                              _p(u64), _p(i64)]
    L.or_simulate.restype = None
    L.or_histogram.argtypes = [C.c_void_p, i64, _p(i32), _p(dbl), i32, _p(u64)]
    L.or_histogram.restype = None
    L.or_histogram_binned.argtypes = [C.c_void_p, i64, _p(i32), _p(dbl), _p(i32), _p(dbl),
                                      _p(u64)]
    L.or_histogram_binned.restype = None
    L.or_em_step_injected.argtypes = [C.c_void_p, _p(i32), _p(dbl), _p(u32), _p(u32), _p(u32),
                                      _p(u32), dbl, i32, _p(dbl), i32, _p(u32), i32, _p(u64),
                                      _p(u64), _p(u64)]
    L.or_em_step_injected.restype = C.c_int


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


# ------------------------------------------------------------------ random

def philox4x32_10(ctr, key):
    """Philox-4x32-10 of one counter block: ctr (4 u32), key (2 u32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def u01(w: int) -> float:
    return lib().or_u01(int(w))


def box_muller(wa: int, wb: int):
    zc, zs = C.c_double(), C.c_double()
    lib().or_box_muller(int(wa), int(wb), C.byref(zc), C.byref(zs))
    return zc.value, zs.value


def normal(seed: int, instance: int, pid: int, n: int) -> float:
    """The n-th normal of particle pid."""
    return lib().or_normal(seed, instance, pid, n)


def split_draw(seed: int, instance: int, pid: int, j: int) -> int:
    """The u32 of the j-th vertex hit of particle pid."""
    return lib().or_split_draw(seed, instance, pid, j)


def root(A: float, B: float, Cc: float) -> float:
    return lib().or_root(float(A), float(B), float(Cc))


# ------------------------------------------------------------------- graph

class Graph:
    """Oracle copy of a metric graph (arrays as in the library's description)."""

    def __init__(self, n_vertices, src, dst, length, c0, c1, sigma, w_init, w_term,
                 hist_range=None, kind=None, sigma1=None):
        E = len(src)
        self.n_vertices = int(n_vertices)
        self.n_edges = E
        self._arrs = dict(
            src=np.ascontiguousarray(src, dtype=np.int32),
            dst=np.ascontiguousarray(dst, dtype=np.int32),
            length=np.ascontiguousarray(length, dtype=np.float64),
            c0=np.ascontiguousarray(c0, dtype=np.float64),
            c1=np.ascontiguousarray(c1, dtype=np.float64),
            sigma=np.ascontiguousarray(sigma, dtype=np.float64),
            w_init=np.ascontiguousarray(w_init, dtype=np.float64),
            w_term=np.ascontiguousarray(w_term, dtype=np.float64),
        )
        a = self._arrs
        hr = None if hist_range is None else np.ascontiguousarray(hist_range, dtype=np.float64)
        kd = None if kind is None else np.ascontiguousarray(kind, dtype=np.uint8)
        self._hr, self._kd = hr, kd
        h = C.c_void_p()
        rc = lib().or_graph_build(
            self.n_vertices, E, _ptr(a["src"], C.c_int32), _ptr(a["dst"], C.c_int32),
            _ptr(a["length"], C.c_double), _ptr(a["c0"], C.c_double), _ptr(a["c1"], C.c_double),
            _ptr(a["sigma"], C.c_double), _ptr(a["w_init"], C.c_double),
            _ptr(a["w_term"], C.c_double),
            None if hr is None else _ptr(hr, C.c_double),
            None if kd is None else _ptr(kd, C.c_uint8), C.byref(h))
        if rc != 0:
            raise ValueError("oracle: invalid graph description")
        self._h = h
        if sigma1 is not None:
            self._s1 = np.ascontiguousarray(np.broadcast_to(sigma1, (E,)), dtype=np.float64)
            if lib().or_graph_set_sigma1(h, _ptr(self._s1, C.c_double)) != 0:
                raise ValueError("oracle: invalid diffusion slope")
        self.n_slots = lib().or_graph_n_slots(h)

    @classmethod
    def from_desc(cls, d):
        """Build from a dict with the keys of a workload graph description."""
        return cls(d["n_vertices"], d["src"], d["dst"], d["length"], d["c0"], d["c1"],
                   d["sigma"], d["w_init"], d["w_term"], d.get("hist_range"), d.get("kind"),
                   d.get("sigma1"))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().or_graph_free(h)
            except Exception:
                pass
            self._h = None

    def slots(self):
        V, S = self.n_vertices, self.n_slots
        off = np.zeros(V + 1, np.int32)
        se = np.zeros(S, np.int32)
        send = np.zeros(S, np.uint8)
        T = np.zeros(S, np.uint64)
        lib().or_graph_slots(self._h, _ptr(off, C.c_int32), _ptr(se, C.c_int32),
                             _ptr(send, C.c_uint8), _ptr(T, C.c_uint64))
        return off, se, send, T

    def choose_slot(self, v: int, u: int) -> int:
        return lib().or_choose_slot(self._h, int(v), int(u))


class State:
    """Particle state arrays (structure of arrays), all host numpy."""

    def __init__(self, edge, x, pid=None):
        n = len(edge)
        self.edge = np.ascontiguousarray(edge, dtype=np.int32).copy()
        self.x = np.ascontiguousarray(x, dtype=np.float64).copy()
        self.n_draw = np.zeros(n, np.uint32)
        self.hits = np.zeros(n, np.uint32)
        self.first_hits = np.zeros(n, np.uint32)
        self.flags = np.zeros(n, np.uint32)
        self.pid = (np.arange(n, dtype=np.uint32) if pid is None
                    else np.ascontiguousarray(pid, dtype=np.uint32).copy())

    def __len__(self):
        return len(self.edge)


class Counters:
    def __init__(self, g: Graph):
        self.exits = np.zeros(g.n_slots, np.uint64)
        self.absorbed = np.zeros(g.n_vertices, np.uint64)
        self.truncations = np.zeros(1, np.uint64)
        self.particle_steps = np.zeros(1, np.int64)


def simulate(g: Graph, st: State, cnt: Counters, *, seed: int, instance: int, dt: float,
             steps: int, M: int):
    """Advance every particle of ``st`` by ``steps`` EM-Steps."""
    if not (dt > 0) or M < 1 or steps < 0:
        raise ValueError("oracle: dt > 0, M >= 1, steps >= 0 required")
    n = len(st)
    lib().or_simulate(g._h, n, _ptr(st.pid, C.c_uint32), _ptr(st.edge, C.c_int32),
                      _ptr(st.x, C.c_double), _ptr(st.n_draw, C.c_uint32),
                      _ptr(st.hits, C.c_uint32), _ptr(st.first_hits, C.c_uint32),
                      _ptr(st.flags, C.c_uint32), int(seed), int(instance), float(dt),
                      int(steps), int(M),
                      _ptr(cnt.exits, C.c_uint64), _ptr(cnt.absorbed, C.c_uint64),
                      _ptr(cnt.truncations, C.c_uint64), _ptr(cnt.particle_steps, C.c_int64))


def histogram(g: Graph, st: State, bins: int) -> np.ndarray:
    h = np.zeros(g.n_edges * bins, np.uint64)
    lib().or_histogram(g._h, len(st), _ptr(st.edge, C.c_int32), _ptr(st.x, C.c_double),
                       int(bins), _ptr(h, C.c_uint64))
    return h


def histogram_binned(g: Graph, st: State, offsets, upper) -> np.ndarray:
    """Counts per variable-width bin: offsets[E+1] (int32), upper[offsets[E]]
    (binary64 upper boundaries, increasing within an edge)."""
    off = np.ascontiguousarray(offsets, np.int32)
    up = np.ascontiguousarray(upper, np.float64)
    h = np.zeros(int(off[-1]), np.uint64)
    lib().or_histogram_binned(g._h, len(st), _ptr(st.edge, C.c_int32), _ptr(st.x, C.c_double),
                              _ptr(off, C.c_int32), _ptr(up, C.c_double), _ptr(h, C.c_uint64))
    return h


def em_step_injected(g: Graph, edge: int, x: float, dt: float, M: int, zs, us,
                     n_draw: int = 0, hits: int = 0, first_hits: int = 0, flags: int = 0):
    """One EM-Step of one particle with its draws injected: ``zs`` the normals
    of its sub-steps in order, ``us`` the u32s of its vertex hits.  Returns
    (edge, x, n_draw, hits, first_hits, flags, splits, exits, absorbed,
    truncations) as a dict."""
    e_, x_ = C.c_int32(edge), C.c_double(x)
    nd_, h_ = C.c_uint32(n_draw), C.c_uint32(hits)
    f_, fl_ = C.c_uint32(first_hits), C.c_uint32(flags)
    zs = np.ascontiguousarray(list(zs) if len(zs) else [0.0], dtype=np.float64)
    us = np.ascontiguousarray(list(us) if len(us) else [0], dtype=np.uint32)
    exits = np.zeros(g.n_slots, np.uint64)
    absorbed = np.zeros(g.n_vertices, np.uint64)
    tr = np.zeros(1, np.uint64)
    k = lib().or_em_step_injected(g._h, C.byref(e_), C.byref(x_), C.byref(nd_), C.byref(h_),
                                  C.byref(f_), C.byref(fl_), float(dt), int(M),
                                  _ptr(zs, C.c_double), len(zs), _ptr(us, C.c_uint32), len(us),
                                  _ptr(exits, C.c_uint64), _ptr(absorbed, C.c_uint64),
                                  _ptr(tr, C.c_uint64))
    return dict(edge=e_.value, x=x_.value, n_draw=nd_.value, hits=h_.value,
                first_hits=f_.value, flags=fl_.value, splits=k, exits=exits,
                absorbed=absorbed, truncations=int(tr[0]))
