"""The binary64 mode's logarithm of its uniforms (ln_u01 in mg_em_step.cuh,
tables in mg_log_table.h written by gen_log_table.py), checked on the CPU:

* every table entry against a 40-digit logarithm: c_j is the binary64
  nearest 64 / (64 + j), and hi + lo equals -k ln 2 - ln(c_j) to within
  2^-100 relative (hi the nearest binary64);
* the kernel's steps, emulated in binary64 (fused multiply-adds exactly
  rounded through fractions), give the correctly rounded ln u on the ends of
  the range, on both sides of the fold at f = 2 - 2^-7 and of every table
  interval, and on random words.

The compiled kernel's normals are compared with the oracle's on the GPU
(test_fp64_normals_match_oracle)."""
import math
import os
import re
import struct
from fractions import Fraction

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

HEADER = os.path.join(os.path.dirname(__file__), "..", "paper_2512_02175_gb300", "csrc",
                      "mg_log_table.h")
K, J = 34, 64


def _tables():
    src = open(HEADER).read()
    body = re.search(r"const double kLogC\[\d+\] = \{(.*?)\};", src, re.S).group(1)
    c = [float.fromhex(v.strip()) for v in body.split(",") if v.strip()]
    body = re.search(r"const double2 kLogKJ\[\d+\] = \{(.*?)\};\n", src, re.S).group(1)
    kj = [(float.fromhex(h), float.fromhex(l))
          for h, l in re.findall(r"\{\s*([-0-9a-fx.p+]+)\s*,\s*([-0-9a-fx.p+]+)\s*\}", body)]
    return c, kj


C, KJ = _tables()


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _d(bits):
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def ln_u01(w):
    """The kernel's steps, one binary64 operation at a time."""
    m = 2 * w + 1
    t = m.bit_length() - 1
    frac = (m << (52 - t)) & ((1 << 52) - 1)
    k, j = 33 - t, 0
    if frac >= 0x000FE00000000000:
        f = _d((1022 << 52) | frac)
        k -= 1
    else:
        f = _d((1023 << 52) | frac)
        j = (frac + (1 << 45)) >> 46
    c = C[j]
    ph = f * c
    pl = _fma(f, c, -ph)
    r = ph - 1.0
    q = _fma(r, -0.125, 1.0 / 7.0)
    for coef in (-1.0 / 6.0, 0.2, -0.25, 1.0 / 3.0, -0.5):
        q = _fma(q, r, coef)
    vh, vl = KJ[J * k + j]
    t1 = vh + r
    e1 = r - (t1 - vh)
    small = (vl + e1) + _fma(-pl, r, pl)
    return t1 + _fma(r * r, q, small)


def test_table_entries():
    mpmath.mp.dps = 40
    assert len(C) == 65 and len(KJ) == K * J
    for j in range(65):
        assert C[j] == float(mpmath.mpf(64) / (64 + j))
    assert C[0] == 1.0 and KJ[0] == (0.0, 0.0)
    for k in range(K):
        for j in range(J):
            exact = -k * mpmath.log(2) - mpmath.log(mpmath.mpf(C[j]))
            hi, lo = KJ[J * k + j]
            assert hi == float(exact)
            assert abs(mpmath.mpf(hi) + mpmath.mpf(lo) - exact) <= abs(exact) * mpmath.mpf(2) ** -100


def _words():
    ws = {0, 1, 2, 3, 2**31 - 1, 2**31, 2**32 - 2, 2**32 - 1}
    ws |= {2**p for p in range(32)} | {2**p - 1 for p in range(1, 33)}
    # both sides of the fold (f = 2 - 2^-7) and of every table interval, at
    # several binades
    for top in (8, 20, 31, 32):
        for j in range(65):
            edge = ((1 << 52) + (2 * j + 1) * (1 << 45)) >> (52 - top)
            for dm in (-2, -1, 0, 1, 2):
                m = edge + dm
                if m % 2 == 1 and 0 < m < 2**33:
                    ws.add((m - 1) // 2)
    rng = np.random.default_rng(2512)
    ws |= {int(v) for v in rng.integers(0, 2**32, 1500)}
    return sorted(ws)


def test_correctly_rounded():
    mpmath.mp.dps = 40
    bad = []
    for w in _words():
        got = ln_u01(w)
        exact = mpmath.log(mpmath.mpf(2 * w + 1) / mpmath.mpf(2) ** 33)
        err = abs(mpmath.mpf(got) - exact) / mpmath.mpf(math.ulp(float(exact)))
        if err > 0.5 + 1e-9:
            bad.append((w, float(err)))
    assert not bad, bad[:5]


def test_header_is_the_generators_output():
    """mg_log_table.h is exactly what gen_log_table.py writes (no hand edits)."""
    import contextlib
    import importlib.util
    import io
    gen = os.path.join(os.path.dirname(HEADER), "gen_log_table.py")
    spec = importlib.util.spec_from_file_location("gen_log_table", gen)
    mod = importlib.util.module_from_spec(spec)
    dps = mpmath.mp.dps
    spec.loader.exec_module(mod)
    buf = io.StringIO()
    try:
        with contextlib.redirect_stdout(buf):
            mod.main()
    finally:
        mpmath.mp.dps = dps
    assert buf.getvalue() == open(HEADER).read()
