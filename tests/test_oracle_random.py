"""Pins of the oracle's random streams against things other than itself.

* Philox-4x32-10: Triton's own Philox implementation (``tl.philox``), run on
  the CPU by Triton's interpreter, over random counters and 64-bit keys.
* u = (2w+1) 2^-33: exact end points and exact arithmetic.
* Box-Muller: the normals pass a Kolmogorov-Smirnov test against scipy's
  normal CDF; r^2 is exponential with mean 2 (a dropped factor 2 in
  -2 ln u fails); the angle is uniform; cos/sin partners are uncorrelated.
* The split draws: every byte of the u32 uniform (chi-square over 256 cells).
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy import stats

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_TRITON_SCRIPT = textwrap.dedent(r"""
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(cp, sp, op, n, BLOCK: tl.constexpr):
        i = tl.arange(0, BLOCK)
        m = i < n
        c0 = tl.load(cp + 4 * i + 0, mask=m); c1 = tl.load(cp + 4 * i + 1, mask=m)
        c2 = tl.load(cp + 4 * i + 2, mask=m); c3 = tl.load(cp + 4 * i + 3, mask=m)
        s = tl.load(sp + i, mask=m)
        r0, r1, r2, r3 = tl.philox(s, c0, c1, c2, c3, 10)
        tl.store(op + 4 * i + 0, r0, mask=m); tl.store(op + 4 * i + 1, r1, mask=m)
        tl.store(op + 4 * i + 2, r2, mask=m); tl.store(op + 4 * i + 3, r3, mask=m)

    d = np.load(sys.argv[1])
    ctr, seed = d["ctr"], d["seed"]
    n = len(seed)
    out = torch.zeros(n * 4, dtype=torch.int32)
    k[(1,)](torch.from_numpy(ctr.view(np.int32).reshape(-1).copy()),
            torch.from_numpy(seed.copy()), out, n, BLOCK=n)
    np.save(sys.argv[2], out.numpy().view(np.uint32).reshape(n, 4))
""")


def test_philox_matches_triton_reference(oracle, tmp_path):
    pytest.importorskip("triton")
    rng = np.random.default_rng(1234)
    n = 512
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    # include structured counters like the ones the scheme uses
    ctr[:8] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1],
               [0xffffffff] * 4, [7, 123456, 1, 3], [0x40000000, 99, 0, 0]]
    seed = rng.integers(0, 2 ** 63, n, dtype=np.int64)
    seed[:4] = [0, 1, 0x7fffffff, 0x123456789]
    inp, outp = tmp_path / "in.npz", tmp_path / "out.npy"
    np.savez(inp, ctr=ctr, seed=seed)
    script = tmp_path / "tri.py"
    script.write_text(_TRITON_SCRIPT)
    subprocess.run([sys.executable, str(script), str(inp), str(outp)], check=True,
                   timeout=600, env={**os.environ, "TRITON_INTERPRET": "1"})
    ref = np.load(outp)
    got = np.array([oracle.philox4x32_10(ctr[i], [int(seed[i]) & 0xffffffff, int(seed[i]) >> 32])
                    for i in range(n)])
    assert np.array_equal(got, ref)


def test_u01_exact(oracle):
    assert oracle.u01(0) == 2.0 ** -33
    assert oracle.u01(0xffffffff) == 1.0 - 2.0 ** -33
    for w in [1, 2, 12345, 2 ** 31, 2 ** 32 - 2]:
        assert oracle.u01(w) == (2 * w + 1) / 2.0 ** 33  # exact in binary64


def _many_normals(oracle, n_pid=64, n_t=2048, seed=5, instance=2):
    z = np.empty(n_pid * n_t)
    i = 0
    for pid in range(n_pid):
        for t in range(n_t):
            z[i] = oracle.normal(seed, instance, pid, t)
            i += 1
    return z.reshape(n_pid, n_t)


def test_main_normals_are_standard_normal(oracle):
    z = _many_normals(oracle)
    flat = z.reshape(-1)
    ks = stats.kstest(flat, "norm")
    assert ks.pvalue > 1e-3, ks
    n = flat.size
    assert abs(flat.mean()) < 4.0 / np.sqrt(n)
    assert abs(flat.var() - 1.0) < 4.0 * np.sqrt(2.0 / n)
    # Box-Muller partners (t = 4j, 4j+1): r^2 ~ Exp(mean 2), angle uniform, uncorrelated
    zc, zs = z[:, 0::4].reshape(-1), z[:, 1::4].reshape(-1)
    r2 = zc * zc + zs * zs
    assert stats.kstest(r2, "expon", args=(0, 2.0)).pvalue > 1e-3
    ang = np.arctan2(zs, zc)
    assert stats.kstest(ang, "uniform", args=(-np.pi, 2 * np.pi)).pvalue > 1e-3
    assert abs(np.corrcoef(zc, zs)[0, 1]) < 4.0 / np.sqrt(zc.size)
    # consecutive steps of one particle are uncorrelated
    assert abs(np.corrcoef(z[:, :-1].reshape(-1), z[:, 1:].reshape(-1))[0, 1]) < 4.0 / np.sqrt(z.size)


def test_split_draws(oracle):
    us = np.array([oracle.split_draw(9, 1, pid, j) for pid in range(32) for j in range(1024)],
                  dtype=np.uint64)
    for shift in (0, 8, 16, 24):  # every byte of the word is uniform (4 tests: 1e-4 each)
        counts = np.bincount(((us >> shift) & 255).astype(np.int64), minlength=256)
        assert stats.chisquare(counts).pvalue > 1e-4


def test_split_draws_of_one_block_are_independent(oracle):
    """Four consecutive hits share a Philox block (one word each): the pairs
    (u_j, u_j+1) -- within a block (j mod 4 = 0, 1, 2) and across a block
    boundary (j mod 4 = 3) -- are uniform on the 16 x 16 grid of their top 4
    bits, and the four words of a block differ."""
    us = np.array([[oracle.split_draw(3, 0, pid, j) for j in range(64)] for pid in range(256)],
                  dtype=np.uint64)
    hi = (us >> 28).astype(np.int64)
    for r in range(4):
        a, b = hi[:, r:63:4].reshape(-1), hi[:, r + 1:64:4].reshape(-1)
        counts = np.bincount(a * 16 + b, minlength=256)
        assert stats.chisquare(counts).pvalue > 1e-4, r
    for r in range(3):
        assert np.all(us[:, r::4] != us[:, r + 1::4])


def test_streams_are_distinct(oracle):
    # tag, pid, instance and seed each change the stream
    a = oracle.normal(1, 0, 0, 0)
    assert a != oracle.normal(2, 0, 0, 0)
    assert a != oracle.normal(1, 1, 0, 0)
    assert a != oracle.normal(1, 0, 1, 0)
    assert a != oracle.normal(1, 0, 0, 4)
    assert oracle.split_draw(1, 0, 0, 0) != oracle.split_draw(1, 0, 0, 1)
