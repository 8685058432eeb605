"""Double-float arithmetic of the MIXED solver (csrc/dfloat.cuh), checked on the host.

The header's inline functions are compiled for the host by nvcc and evaluated on random operands
spanning many binades; every result is compared with the exact rational value.  Bars: the
Dekker-style addition errs by at most 2^-45 (|a| + |b|), products by 2^-45 |a b|, the band
accumulation acc + b x by 2^-45 (|acc| + |b x|), the fused a b + c d of the complex products by
2^-45 (|a b| + |c d|), a 343-term lazily normalised band sum by
2^-40 sum |b x| (343 terms of at most ~2^-48 each), and the conversion from a double by
2^-48 |v|; every result is normalised (hi = fl(hi + lo))."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2101_11751_gb300", "csrc")


def _f32(v):
    return float(np.float32(v))


def _split(v):
    h = _f32(v)
    return h, _f32(v - h)


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("dfl") / "dfloat_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "dfloat_check.cu"), "-o", out],
                   check=True, capture_output=True)
    return out


def _run(driver, lines):
    r = subprocess.run([driver], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return [tuple(float.fromhex(t) for t in ln.split()) for ln in r.stdout.strip().splitlines()]


def _normalised(h, l):
    return _f32(h + l) == h and abs(l) <= abs(h) * 2.0 ** -24


def _operands(rng, k):
    e = rng.integers(-30, 30, size=k)
    v = rng.uniform(-1, 1, size=k) * 2.0 ** e
    return [_split(x) for x in v]


def test_add_sub_mul(driver):
    rng = np.random.default_rng(0)
    A, B = _operands(rng, 400), _operands(rng, 400)
    # cancellation cases: b close to -a
    for i in range(0, 400, 5):
        B[i] = (-A[i][0], _f32(A[i][1] * 0.5))
    lines = []
    for op in "asm":
        lines += [f"{op} {a[0].hex()} {a[1].hex()} {b[0].hex()} {b[1].hex()}" for a, b in zip(A, B)]
    res = _run(driver, lines)
    k = 0
    for op in "asm":
        for a, b in zip(A, B):
            fa = Fraction(a[0]) + Fraction(a[1])
            fb = Fraction(b[0]) + Fraction(b[1])
            h, l = res[k]
            k += 1
            got = Fraction(h) + Fraction(l)
            assert _normalised(h, l)
            if op == "m":
                exact, scale = fa * fb, abs(fa * fb)
            else:
                exact = fa + fb if op == "a" else fa - fb
                scale = abs(fa) + abs(fb)
            assert abs(got - exact) <= Fraction(2) ** -45 * scale, (op, a, b)


def test_mul_f32_and_band_accumulation(driver):
    rng = np.random.default_rng(1)
    A, X = _operands(rng, 300), _operands(rng, 300)
    bs = [_f32(v) for v in rng.uniform(-2, 2, 300) * 2.0 ** rng.integers(-10, 10, 300)]
    lines = [f"f {a[0].hex()} {a[1].hex()} {b.hex()}" for a, b in zip(A, bs)]
    lines += [f"x {a[0].hex()} {a[1].hex()} {b.hex()} {x[0].hex()} {x[1].hex()}" for a, b, x in zip(A, bs, X)]
    res = _run(driver, lines)
    for i, (a, b) in enumerate(zip(A, bs)):
        fa = Fraction(a[0]) + Fraction(a[1])
        h, l = res[i]
        assert _normalised(h, l)
        assert abs(Fraction(h) + Fraction(l) - fa * Fraction(b)) <= Fraction(2) ** -45 * abs(fa * Fraction(b))
    for i, (a, b, x) in enumerate(zip(A, bs, X)):
        fa = Fraction(a[0]) + Fraction(a[1])
        bx = Fraction(b) * (Fraction(x[0]) + Fraction(x[1]))
        h, l = res[300 + i]
        assert _normalised(h, l)
        assert abs(Fraction(h) + Fraction(l) - (fa + bx)) <= Fraction(2) ** -45 * (abs(fa) + abs(bx))


def test_from_double(driver):
    rng = np.random.default_rng(2)
    vs = list(rng.uniform(-1, 1, 200) * 2.0 ** rng.integers(-40, 40, 200)) + [0.0, 1.0, -3.0, 1.0 / 3.0]
    res = _run(driver, [f"c {float(v).hex()}" for v in vs])
    for v, (h, l) in zip(vs, res):
        assert _normalised(h, l)
        assert abs(Fraction(h) + Fraction(l) - Fraction(v)) <= Fraction(2) ** -48 * abs(Fraction(v))


def test_lazy_band_sum(driver):
    rng = np.random.default_rng(3)
    lines, terms = [], []
    for case in range(40):
        k = 343
        bs = [_f32(v) for v in rng.uniform(-1, 1, k) * 2.0 ** rng.integers(-6, 6, k)]
        xs = _operands(rng, k)
        if case % 4 == 0:  # heavy cancellation: the sum is far below its terms
            xs[-1] = (_f32(-sum(b * (x[0] + x[1]) for b, x in zip(bs[:-1], xs[:-1])) / bs[-1]), 0.0)
            xs[-1] = _split(xs[-1][0])
        terms.append((bs, xs))
        lines.append(f"A {k} " + " ".join(f"{b.hex()} {x[0].hex()} {x[1].hex()}" for b, x in zip(bs, xs)))
    res = _run(driver, lines)
    for (bs, xs), (h, l) in zip(terms, res):
        prods = [Fraction(b) * (Fraction(x[0]) + Fraction(x[1])) for b, x in zip(bs, xs)]
        exact = sum(prods)
        mag = sum(abs(p) for p in prods)
        assert _normalised(h, l)
        assert abs(Fraction(h) + Fraction(l) - exact) <= Fraction(2) ** -40 * mag


def test_dot2(driver):
    """a b + c d with one normalisation (the K_G butterflies' complex products), including
    near-cancelling pairs (c d close to -a b)."""
    rng = np.random.default_rng(4)
    A, B, C, D = (_operands(rng, 300) for _ in range(4))
    for i in range(0, 300, 4):  # c d = -(a b) up to the low parts
        C[i] = (-A[i][0], _f32(A[i][1] * 0.5))
        D[i] = (B[i][0], _f32(B[i][1] * 0.25))
    lines = [f"d {a[0].hex()} {a[1].hex()} {b[0].hex()} {b[1].hex()} {c[0].hex()} {c[1].hex()} "
             f"{d[0].hex()} {d[1].hex()}" for a, b, c, d in zip(A, B, C, D)]
    res = _run(driver, lines)
    fr = lambda t: Fraction(t[0]) + Fraction(t[1])  # noqa: E731
    for (a, b, c, d), (h, l) in zip(zip(A, B, C, D), res):
        ab, cd = fr(a) * fr(b), fr(c) * fr(d)
        assert _normalised(h, l)
        assert abs(Fraction(h) + Fraction(l) - (ab + cd)) <= Fraction(2) ** -45 * (abs(ab) + abs(cd)), (a, b, c, d)
