"""The fixed-point tables and integer steps behind the library's FP64 angles
and square roots, checked on the CPU against 120-bit arithmetic.

The CUDA code evaluates sin/cos(2 pi k 2^-53) from a 256-entry table scaled
by 2^62 and the Taylor series of the remainder in Q64, and sqrt(x) from a
float seed refined by two Newton steps in 64-bit fixed point.  Here the
generated table and constants are compared with mpmath, and the same integer
steps, written again in Python (the high half of a 128-bit product is
(a * b) >> 64), are run on random and edge inputs: the angles must be within
2^-59 absolute, the square roots within 0.51 ulp.  On the GPU the same
functions are compared with CUDA's sincospi and sqrt (test_gpu_fp64_math)."""
import math
import os
import random
import re
import struct

import pytest

mpmath = pytest.importorskip("mpmath")

TABLES = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_1009_2768_gb300", "csrc", "fp64_tables.inc")
M64 = (1 << 64) - 1


def load():
    src = open(TABLES).read()
    body = src[src.index("kSinCos256Q62"):]
    tab = [(int(a), int(b)) for a, b in re.findall(r"\{(-?\d+)ll, (-?\d+)ll\}", body)]
    consts = {n: int(v) for n, v in re.findall(r"kQ(\w+) = (\d+)ull", src)}
    return tab, consts


def umulhi(a, b):
    assert 0 <= a <= M64 and 0 <= b <= M64
    return (a * b) >> 64


def mulhi(a, b):
    assert -(1 << 63) <= a < (1 << 63) and -(1 << 63) <= b < (1 << 63)
    return (a * b) >> 64


def sincos_q62(k, tab, K):
    i = k >> 45
    T = umulhi(((k & ((1 << 45) - 1)) << 16) & M64, K["2Pi59"])
    T2 = umulhi(T, T)
    p = (K["Inv120"] - umulhi(T2, K["Inv5040"])) & M64
    p = (K["Inv6"] - umulhi(T2, p)) & M64
    SN = (T - umulhi(umulhi(T2, T), p)) & M64
    q = (K["Inv720"] - umulhi(T2, K["Inv40320"])) & M64
    q = (K["Inv24"] - umulhi(T2, q)) & M64
    q = ((1 << 63) - umulhi(T2, q)) & M64
    CM = umulhi(T2, q)
    assert SN < (1 << 63) and CM < (1 << 63)
    S, C = tab[i]
    return S - mulhi(S, CM) + mulhi(C, SN), C - mulhi(C, CM) - mulhi(S, SN)


def f32(x):
    return struct.unpack("<f", struct.pack("<f", x))[0]


def sqrt_fx(x, seed_ulps=0):
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    ef = b >> 52
    assert 0 < ef < 0x7FF
    E = ef - 1075
    m = (b & ((1 << 52) - 1)) | (1 << 52)
    if E & 1:
        m <<= 1
        E -= 1
    X = m << 10
    assert (1 << 62) <= X <= M64
    y0 = f32(1.0 / math.sqrt(f32((X >> 40) * 2.0 ** -24)))          # the float unit's seed
    yb = struct.unpack("<I", struct.pack("<f", y0))[0] + seed_ulps    # ... give or take a few ulp
    Y = ((yb & 0x7FFFFF) | 0x800000) << (39 + (yb >> 23) - 127)
    for _ in range(2):
        zy2 = umulhi(X, umulhi(Y, Y))
        Y = umulhi(Y, (((3 << 60) - zy2) << 2) & M64) << 1
        assert Y <= M64
    S = umulhi(X, Y)
    bits = ((1023 + 26 + (E >> 1) - 1) << 52) + ((S + 256) >> 9)
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def test_tables_and_constants_are_correctly_rounded():
    tab, K = load()
    mpmath.mp.prec = 200
    assert len(tab) == 256
    for i, (s, c) in enumerate(tab):
        a = 2 * mpmath.pi * i / 256
        assert abs(s - mpmath.sin(a) * 2 ** 62) <= 0.5 + 1e-9
        assert abs(c - mpmath.cos(a) * 2 ** 62) <= 0.5 + 1e-9
    assert abs(K["2Pi59"] - 2 * mpmath.pi * 2 ** 59) <= 0.5
    for n in (6, 24, 120, 720, 5040, 40320):
        assert abs(K[f"Inv{n}"] - mpmath.mpf(2) ** 64 / n) <= 0.5


def test_fixed_point_angles_within_2_to_minus_59():
    tab, K = load()
    mpmath.mp.prec = 120
    rnd = random.Random(11)
    ks = [rnd.randrange(1 << 53) for _ in range(3000)]
    ks += [(i << 45) + d for i in range(256) for d in (-1, 0, 1) if 0 <= (i << 45) + d < (1 << 53)]
    ks += [0, 1, (1 << 45) - 1, (1 << 53) - 1, 1 << 51, 3 << 51]
    worst = mpmath.mpf(0)
    for k in ks:
        s, c = sincos_q62(k, tab, K)
        a = 2 * mpmath.pi * k / mpmath.mpf(2) ** 53
        worst = max(worst, abs(mpmath.mpf(s) / 2 ** 62 - mpmath.sin(a)), abs(mpmath.mpf(c) / 2 ** 62 - mpmath.cos(a)))
    assert worst < mpmath.mpf(2) ** -59, float(worst)


def test_fixed_point_sqrt_faithful_with_a_perturbed_seed():
    mpmath.mp.prec = 160
    rnd = random.Random(12)
    xs = [(1.0 + rnd.random()) * 2.0 ** rnd.randint(-1020, 1020) for _ in range(1500)]
    xs += [2.0 ** e for e in range(-1022, 1023, 13)] + [4.0, 0.25, 2.0, 1 - 2 ** -53, math.nextafter(4.0, 0)]
    xs += [float(k) ** 2 for k in range(1, 200)] + [math.nextafter(float(k) ** 2, 0) for k in range(2, 200)]
    for seed in (0, -3, 3):
        worst = 0.0
        for x in xs:
            r = sqrt_fx(x, seed)
            ex = mpmath.sqrt(mpmath.mpf(x))
            worst = max(worst, float(abs(mpmath.mpf(r) - ex) / mpmath.mpf(math.ulp(float(ex)))))
        assert worst <= 0.51, (seed, worst)
