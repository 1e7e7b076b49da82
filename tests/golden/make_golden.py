"""Writes the stored expected values under tests/golden/ -- computed by the
plain FP64 CPU oracle only (oracle/), never by the CUDA path.

star3_brownian.json: the 3-edge Brownian star (three edges of length 1,
mu = 0, sigma = 1, equal b; Algorithms 1-2 under the readings of the oracle)
with 48 particles, particle i on edge i mod 3 at x_i = (i + 0.5) / 48 of the
edge; seed 5, instance 2, dt = 1e-3, 400 EM-Steps, M = 8.  Stored: the final
state of every particle (positions as exact hexadecimal binary64), the
8-bin histogram, the exit counts per slot and the particle-step count.

Run from the repository root: python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402

CASE = dict(n=48, seed=5, instance=2, dt=1e-3, steps=400, M=8, bins=8)


def star3():
    """The 3-edge Brownian star as an oracle graph description (no CUDA code)."""
    return dict(n_vertices=4, src=np.zeros(3, np.int32), dst=np.arange(1, 4, dtype=np.int32),
                length=np.ones(3), c0=np.zeros(3), c1=np.zeros(3), sigma=np.ones(3),
                w_init=np.ones(3), w_term=np.ones(3))


def initial(n):
    edge = (np.arange(n) % 3).astype(np.int32)
    x = (np.arange(n) + 0.5) / n
    return edge, x


def compute():
    c = CASE
    d = star3()
    g = O.Graph(d["n_vertices"], d["src"], d["dst"], d["length"], d["c0"], d["c1"], d["sigma"],
                d["w_init"], d["w_term"])
    e, x = initial(c["n"])
    st = O.State(e, x)
    cnt = O.Counters(g)
    O.simulate(g, st, cnt, seed=c["seed"], instance=c["instance"], dt=c["dt"], steps=c["steps"],
               M=c["M"])
    return dict(case=c,
                edge=[int(v) for v in st.edge], x=[float(v).hex() for v in st.x],
                n_draw=[int(v) for v in st.n_draw], hits=[int(v) for v in st.hits],
                first_hits=[int(v) for v in st.first_hits],
                histogram=[int(v) for v in O.histogram(g, st, c["bins"])],
                exits=[int(v) for v in cnt.exits],
                particle_steps=int(np.asarray(cnt.particle_steps).reshape(-1)[0]))


if __name__ == "__main__":
    out = compute()
    with open(os.path.join(HERE, "star3_brownian.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("wrote star3_brownian.json")
