"""Host checks of the integer-based FP64 <-> FP32-pair conversions and the double-float
arithmetic used by the FP32-refined solve (csrc/fpconv.cuh), against exact rationals."""
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("fpconv") / "fpconv_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", os.path.join(HERE, "host", "fpconv_check.cpp"),
                    "-o", out], check=True)
    return out


def d2h(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def h2f(h):
    return struct.unpack("<f", struct.pack("<I", int(h, 16)))[0]


def h2d(h):
    return struct.unpack("<d", struct.pack("<Q", int(h, 16)))[0]


def run(prog, lines):
    r = subprocess.run([prog], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return r.stdout.split("\n")[:-1]


def sample_doubles(n, seed):
    rng = np.random.default_rng(seed)
    mags = 10.0 ** rng.uniform(-30, 30, n)
    vals = mags * rng.choice([-1.0, 1.0], n) * (1 + rng.random(n))
    special = [0.0, -0.0, 1.0, -1.0, 1.5, 2.0 ** -126, 2.0 ** -127, 2.0 ** 127, 3.4e38, 1e-45, 1e300, -1e-300,
               np.pi, np.e, 1.0 + 2.0 ** -30, 1.0 - 2.0 ** -40]
    return list(vals) + special


def trunc_ref(x):
    if x == 0 or abs(x) < 2.0 ** -126:
        return 0.0
    if abs(x) >= 2.0 ** 128:
        return np.copysign(np.inf, x)
    f = np.float32(x)
    if abs(float(f)) > abs(x):
        f = np.nextafter(f, np.float32(0))
    if np.isinf(f):
        f = np.copysign(np.float32(3.4028234663852886e38), x)
    return float(f)


def test_truncation_to_fp32(prog):
    xs = sample_doubles(3000, 1)
    outs = run(prog, [f"trunc {d2h(x):016x} 0" for x in xs])
    for x, o in zip(xs, outs):
        got = h2f(o)
        assert got == trunc_ref(x) or (got == 0 and trunc_ref(x) == 0), (x, got, trunc_ref(x))


def test_split_is_accurate_to_47_bits(prog):
    xs = [x for x in sample_doubles(3000, 2) if 2.0 ** -70 < abs(x) < 2.0 ** 127]
    outs = run(prog, [f"split {d2h(x):016x} 0" for x in xs])
    for x, o in zip(xs, outs):
        hi, lo = (h2f(t) for t in o.split())
        err = abs(Fraction(x) - Fraction(hi) - Fraction(lo))
        assert err <= Fraction(abs(x)) * Fraction(1, 2 ** 46), (x, hi, lo)
        assert abs(hi) <= abs(x)


def test_sum_to_double_is_correctly_rounded(prog):
    """f32_add_to_f64: the exact sum rounded to nearest FP64 (half an ulp), including cancellation,
    operands of very different size and the two parts of normalised pairs (exact there); FP32
    subnormal operands are flushed, so the bound adds 2^-126 for them."""
    rng = np.random.default_rng(6)
    a = (rng.standard_normal(4000) * 10.0 ** rng.uniform(-20, 20, 4000)).astype(np.float32)
    rel = 10.0 ** rng.uniform(-14, 3, 4000)
    b = (a * rng.choice([-1.0, 1.0], 4000) * rel).astype(np.float32)
    pairs = list(zip(a, b)) + [(np.float32(1), np.float32(-2 ** -30)), (np.float32(2 ** 10), np.float32(-2 ** -20)),
                              (np.float32(1), np.float32(-1)), (np.float32(0), np.float32(0)),
                              (np.float32(3), np.float32(2 ** -40)), (np.float32(-1), np.float32(2 ** -25)),
                              (np.float32(1.5), np.float32(-1.25)), (np.float32(1e-30), np.float32(1e-38))]
    outs = run(prog, [f"sum {d2h(float(x)):016x} {d2h(float(y)):016x}" for x, y in pairs])
    for (x, y), o in zip(pairs, outs):
        got = h2d(o)
        exact = Fraction(float(x)) + Fraction(float(y))
        if exact == 0:
            assert got == 0.0
            continue
        ulp = Fraction(np.spacing(abs(float(exact))))
        assert abs(Fraction(got) - exact) <= ulp / 2 + Fraction(1, 2 ** 126), (x, y, got, float(exact))


def test_widening_to_double_is_exact(prog):
    """f32_to_f64_exact: the FP64 value of every normal FP32 input (and of zeros, infinities and a
    NaN) bit for bit; FP32 subnormals become signed zeros."""
    rng = np.random.default_rng(8)
    bits = rng.integers(0, 2 ** 32, 20000, dtype=np.uint64).astype(np.uint32)
    vals = list(bits.view(np.float32)) + [np.float32(v) for v in (0.0, -0.0, 1.0, -2.5, 3.4e38, -1.2e-38)]
    vals += [np.float32(np.inf), np.float32(-np.inf), np.float32(1e-40), np.float32(-1e-45)]
    outs = run(prog, [f"widen {d2h(float(v)):016x} 0000000000000000" for v in vals])
    for v, o in zip(vals, outs):
        got = h2d(o)
        if np.isnan(v):
            assert np.isnan(got)
        elif v != 0 and abs(float(v)) < 2.0 ** -126:
            assert got == 0.0 and np.signbit(got) == np.signbit(v)
        else:
            assert d2h(got) == d2h(float(v)), (v, o)


@pytest.mark.parametrize("op", ["dfadd", "dfmul"])
def test_double_float_arithmetic(prog, op):
    rng = np.random.default_rng(4)
    x = rng.standard_normal(2000) * 10.0 ** rng.uniform(-5, 5, 2000)
    y = rng.standard_normal(2000) * 10.0 ** rng.uniform(-5, 5, 2000)
    outs = run(prog, [f"{op} {d2h(a):016x} {d2h(b):016x}" for a, b in zip(x, y)])
    for a, b, o in zip(x, y, outs):
        hi, lo = (h2f(t) for t in o.split())
        exact = Fraction(a) + Fraction(b) if op == "dfadd" else Fraction(a) * Fraction(b)
        bound = (abs(Fraction(a)) + abs(Fraction(b))) if op == "dfadd" else abs(exact)
        assert abs(Fraction(hi) + Fraction(lo) - exact) <= bound * Fraction(1, 2 ** 43), (a, b)


def test_two_diff_is_exact(prog):
    rng = np.random.default_rng(5)
    a = rng.standard_normal(2000).astype(np.float32)
    b = (a * (1 + rng.standard_normal(2000) * 10.0 ** rng.uniform(-8, 1, 2000))).astype(np.float32)
    outs = run(prog, [f"twodiff {d2h(float(x)):016x} {d2h(float(y)):016x}" for x, y in zip(a, b)])
    for x, y, o in zip(a, b, outs):
        hi, lo = (h2f(t) for t in o.split())
        assert Fraction(hi) + Fraction(lo) == Fraction(float(x)) - Fraction(float(y))
