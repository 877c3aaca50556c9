"""Writes csrc/fp64_tables.inc: the correctly rounded constants of the FP64
angle and logarithm evaluations of the collision kernel (collide.cu), computed
here in 60-digit decimal arithmetic from their series (pi by Machin's formula,
sin/cos by Taylor series, ln by the atanh series).  Run by build.py when the
file is missing; the file is committed, so the build normally only reads it.

The evaluations are table-driven in the manner of P. T. P. Tang ("Table-driven
implementation of the exponential function in IEEE floating-point
arithmetic", ACM TOMS 15, 1989, and its logarithm companion, TOMS 16, 1990):
the argument picks a breakpoint whose function value is tabulated to full
precision, and a short series evaluates the function of the small remainder;
the addition formulas (sin, cos) or a sum of logarithms (ln) combine the two.

  kSinCos256[i] = { sin(2 pi i / 256), cos(2 pi i / 256) },  i = 0..255
  kLnT128[j]    = { ln((1 + j/128) / 2), 2^-52 / (1 + j/128) }, j = 0..127
  kTwoPi53      = { hi, lo }: 2 pi 2^-53 as an unevaluated sum of doubles
  kLn2          = { hi, lo }: ln 2 as an unevaluated sum of doubles
  kSinCos256Q62[i] = the same sines and cosines in fixed point, round(x 2^62)
  kQ2Pi59       = round(2 pi 2^59)
  kQInvN        = round(2^64 / N) for N = 6, 24, 120, 720, 5040, 40320
"""
import os
from decimal import Decimal, getcontext

getcontext().prec = 60
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "fp64_tables.inc")


def arctan_inv(x):
    """arctan(1/x) for an integer x > 1 (alternating series)."""
    x = Decimal(x)
    x2 = x * x
    term = 1 / x
    s, k, sign = Decimal(0), 1, 1
    eps = Decimal(10) ** -(getcontext().prec + 2)
    while abs(term) > eps:
        s += sign * term / k
        term /= x2
        k += 2
        sign = -sign
    return s


PI = 16 * arctan_inv(5) - 4 * arctan_inv(239)      # Machin


def sincos(a):
    eps = Decimal(10) ** -(getcontext().prec + 2)
    s = Decimal(0)
    c = Decimal(0)
    term = Decimal(1)                               # a^k / k!
    k = 0
    while True:
        if k % 4 == 0:
            c += term
        elif k % 4 == 1:
            s += term
        elif k % 4 == 2:
            c -= term
        else:
            s -= term
        k += 1
        term = term * a / k
        if abs(term) < eps and k > 2:
            break
    return s, c


def ln1p(x):
    """ln(1 + x) = 2 atanh(x / (2 + x))."""
    y = x / (2 + x)
    y2 = y * y
    eps = Decimal(10) ** -(getcontext().prec + 2)
    s, term, k = Decimal(0), y, 1
    while abs(term) > eps:
        s += term / k
        term *= y2
        k += 2
    return 2 * s


def dbl(x):
    """Decimal -> nearest double (the exact zeros of sin and cos at multiples of
    pi/2 come out of the series as residues near 1e-60: they are zero)."""
    return 0.0 if abs(x) < Decimal(10) ** -40 else float(x)


def split(x):
    hi = float(x)
    lo = float(x - Decimal(hi))
    return hi, lo


def lit(v):
    return repr(v) if v != 0 else "0.0"


def main():
    lines = ["// Generated by gen_tables.py; do not edit.", "static __device__ const double kSinCos256[256][2] = {"]
    for i in range(256):
        s, c = sincos(2 * PI * i / 256)
        lines.append(f"    {{{lit(dbl(s))}, {lit(dbl(c))}}},")
    lines.append("};")
    lines.append("static __device__ const double kLnT128[128][2] = {")
    for j in range(128):
        T = 1 + Decimal(j) / 128
        lines.append(f"    {{{lit(dbl(ln1p(Decimal(j) / 128) - ln1p(Decimal(1))))}, {lit(dbl(Decimal(2) ** -52 / T))}}},")
    lines.append("};")
    h, l = split(2 * PI * Decimal(2) ** -53)
    lines.append(f"static __device__ const double kTwoPi53[2] = {{{lit(h)}, {lit(l)}}};")
    h, l = split(ln1p(Decimal(1)))
    lines.append(f"static __device__ const double kLn2[2] = {{{lit(h)}, {lit(l)}}};")
    lines.append("static __device__ const long long kSinCos256Q62[256][2] = {")
    for i in range(256):
        sn, cs = sincos(2 * PI * i / 256)
        q = [0 if abs(x) < Decimal(10) ** -40 else int((x * 2 ** 62).to_integral_value()) for x in (sn, cs)]
        lines.append(f"    {{{q[0]}ll, {q[1]}ll}},")
    lines.append("};")
    lines.append(f"static __device__ const unsigned long long kQ2Pi59 = {int((2 * PI * 2 ** 59).to_integral_value())}ull;")
    for n in (6, 24, 120, 720, 5040, 40320):
        lines.append(f"static __device__ const unsigned long long kQInv{n} = "
                     f"{int((Decimal(2) ** 64 / n).to_integral_value())}ull;")
    text = "\n".join(lines) + "\n"
    with open(OUT, "w") as f:
        f.write(text)
    return OUT


if __name__ == "__main__":
    print(main())
