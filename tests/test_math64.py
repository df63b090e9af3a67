"""Pins of the table-driven FP64 exp and log of the FP64 path (the FP64
integrands and the grid refinement): the tables against their definitions
recomputed in 300-bit arithmetic, and a step-by-step emulation of the device
functions (each fma rounded once, from exact rationals) within one ulp of
the exact exp and, for ln, of max(1, |ln x|), on samples across their
ranges."""
import math
import random
import re
import struct
from fractions import Fraction
from pathlib import Path

import pytest

mp = pytest.importorskip("mpmath")

HEADER = Path(__file__).resolve().parents[1] / "paper_1503_06182_gb300" / "csrc" / "gv_math64.cuh"


def table(name):
    text = HEADER.read_text()
    body = re.search(name + r"\[\d+\] = \{(.*?)\};", text, re.S).group(1)
    return [float.fromhex(t) for t in re.findall(r"-?0x[0-9a-fA-F.]+p[-+]?\d+", body)]


def rn(x):
    return float(x)  # an mpf or Fraction to the nearest double


def fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def from_bits(b):
    return struct.unpack("<d", struct.pack("<q", b))[0]


def ulp_err(y, exact):
    """|y - exact| in units of the last place of the exact value."""
    e = math.frexp(float(exact))[1]
    return float(abs(mp.mpf(y) - exact) / mp.ldexp(1, e - 53))


def test_exp_table_is_2_to_the_j_over_64():
    mp.mp.prec = 300
    t = table("gv_exp2j_tab")
    assert len(t) == 128
    for j in range(64):
        v = mp.power(2, mp.mpf(j) / 64)
        assert t[2 * j] == rn(v)
        assert t[2 * j + 1] == rn(v - mp.mpf(t[2 * j]))


def test_log_table_is_its_definition():
    mp.mp.prec = 300
    t = table("gv_log_tab")
    assert len(t) == 258
    for j in range(128):
        R = 1.0 / (1.0 + (j + 0.5) / 128.0)
        assert t[2 * j] == R
        assert t[2 * j + 1] == rn(-mp.log(mp.mpf(R)))
    ln2 = mp.log(2)
    assert t[256] == math.floor(float(ln2) * 2.0**42) / 2.0**42
    assert Fraction(t[256]).denominator <= 2**42
    assert t[257] == rn(ln2 - mp.mpf(t[256]))


# ---- step-by-step emulation of the device functions
def emu_log1p_series(r):
    p = 1.0 / 9.0
    for c in (-1.0 / 8.0, 1.0 / 7.0, -1.0 / 6.0, 1.0 / 5.0, -1.0 / 4.0, 1.0 / 3.0, -0.5):
        p = fma(p, r, c)
    return fma(r * r, p, r)


def emu_log(x, t):
    if abs(x - 1.0) <= 2.0**-7:
        return emu_log1p_series(x - 1.0)
    b, k = bits(x), 0
    if b < (1 << 52):
        x *= 2.0**54
        b, k = bits(x), -54
    k += (b >> 52) - 1023
    j = (b >> 45) & 127
    m = from_bits((b & 0xFFFFFFFFFFFFF) | 0x3FF0000000000000)
    p = emu_log1p_series(fma(m, t[2 * j], -1.0))
    kd = float(k)
    return fma(kd, t[256], t[2 * j + 1]) + fma(kd, t[257], p)


def emu_exp(x, t):
    assert abs(x) < 707.0
    tt = fma(x, float.fromhex("0x1.71547652b82fep+6"), float.fromhex("0x1.8p52"))
    N = bits(tt) & 0xFFFFFFFF
    N = N - (1 << 32) if N >= 1 << 31 else N
    Nd = tt - float.fromhex("0x1.8p52")
    r = fma(-Nd, float.fromhex("0x1.cf79abc9e3b3ap-46"),
            fma(-Nd, float.fromhex("0x1.62e42fefa0000p-7"), x))
    q = fma(r, float.fromhex("0x1.6c16c16c16c17p-10"), float.fromhex("0x1.1111111111111p-7"))
    q = fma(q, r, float.fromhex("0x1.5555555555555p-5"))
    q = fma(q, r, float.fromhex("0x1.5555555555555p-3"))
    q = fma(q, r, 0.5)
    p = fma(r * r, q, r)
    j = N & 63
    y = t[2 * j] + fma(t[2 * j], p, t[2 * j + 1])
    return from_bits(bits(y) + ((N >> 6) << 52))


def test_emulated_exp_within_one_ulp():
    mp.mp.prec = 200
    t = table("gv_exp2j_tab")
    rng = random.Random(11)
    xs = [rng.uniform(-707, 707) for _ in range(3000)]
    xs += [rng.uniform(-1, 1) * 10.0 ** rng.randint(-20, 0) for _ in range(2000)]
    xs += [0.0, -0.0, 706.999, -706.999, math.log(2) / 128, -math.log(2) / 128]
    xs += [k * math.log(2) / 64 for k in range(-64, 65)]  # the table's own points
    worst = 0.0
    for x in xs:
        y = emu_exp(x, t)
        worst = max(worst, ulp_err(y, mp.exp(mp.mpf(x))))
    assert worst < 0.75, worst


def test_emulated_log_within_one_ulp_of_max_1_abs_log():
    mp.mp.prec = 200
    t = table("gv_log_tab")
    rng = random.Random(12)
    xs = [math.ldexp(rng.uniform(1, 2), rng.randint(-1074 + 60, 1023)) for _ in range(3000)]
    xs += [1.0 + rng.uniform(-1, 1) * 2.0**-7 for _ in range(1000)]  # the series branch
    xs += [1.0 + rng.uniform(-1, 1) * 2.0**-6 for _ in range(1000)]  # just outside it
    xs += [rng.uniform(0, 1) * 2.0**-1022 for _ in range(300)]  # subnormal
    xs += [5e-324, 2.0**-1022, 0.5, 2.0, 1.7976931348623157e308]
    worst, series_worst = 0.0, [0.0]
    for x in xs:
        if x <= 0.0:
            continue
        y = emu_log(x, t)
        exact = mp.log(mp.mpf(x))
        # in ulps of max(1, |ln x|): relative away from 1, absolute near it
        worst = max(worst, ulp_err(y, exact) if abs(exact) >= 1 else
                    float(abs(mp.mpf(y) - exact) / mp.mpf(2) ** -52))
        if 2.0**-8 <= x - 1.0 <= 2.0**-7 or -(2.0**-7) <= x - 1.0 <= -(2.0**-8):
            series_worst[0] = max(series_worst[0], ulp_err(y, exact))
    assert worst < 1.0, worst
    assert series_worst[0] < 1.0, series_worst[0]  # the series branch: relative


def test_emulated_exp_of_a_mutated_table_fails():
    """The check above has teeth: a table head two units off moves the
    results that use it by more than an ulp."""
    mp.mp.prec = 200
    t = table("gv_exp2j_tab")
    bad = list(t)
    bad[2 * 37] = from_bits(bits(bad[2 * 37]) + 2)  # two ulps off in one head
    x = 37 * math.log(2) / 64
    assert ulp_err(emu_exp(x, bad), mp.exp(mp.mpf(x))) > 1.0
