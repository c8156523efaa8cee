"""Generate the elementary-function tables of the float-float kernels (a build step).

Writes ``_build/gvx_tables.inc``: values computed here with Python's ``decimal`` module at 60
significant digits (Taylor series; pi by Machin's formula, ln 2 by the atanh series), each
split into a float pair hi + lo:

  kExpTab[j]  = {tm1.hi, tm1.lo, um1.hi, um1.lo},  tm1 = 2^(j/N) - 1, um1 = 1 - 2^(-j/N),
                j = 0 .. N-1, N = 1024 (so c = ln2 / N is the exp reduction step);
  kTrigTab[j] = {sin.hi, sin.lo, cos.hi, cos.lo} of j d, d = pi / 2048, j = 0 .. 1024;

and the Cody-Waite splits of c and d (c0 with 9 significant bits, so n c0 is exact for
|n| < 2^15; d0 with 13 bits, exact for j <= 2^11), 1/c, 1/d and pi as a float pair.

Two tables at a power-of-two step h = 2^-8 serve the light-cone pair mass (mass_lc.cuh), whose
argument reduction x = n h + r is then exact in float arithmetic:

  kHypTab[n] = {cosh.hi, cosh.lo, sinh.hi, sinh.lo} of n h, n = 0 .. 2048 (x <= 8);
  kSinTab[j] = {sin.hi, sin.lo, cos.hi, cos.lo} of j h, j = 0 .. 896 (x <= 3.5).
"""
from __future__ import annotations

import os
import struct
import sys
from decimal import Decimal, getcontext

getcontext().prec = 60
EXP_N = 1024
TRIG_STEPS = 2048  # d = pi / TRIG_STEPS; the table covers [0, pi/2]
LC_STEP_LOG2 = 8   # the light-cone tables' step is 2^-8
HYP_N = 2048       # kHypTab covers [0, 8]
SIN_N = 896        # kSinTab covers [0, 3.5]


def _atan_inv(k: int) -> Decimal:
    """atan(1/k) by its alternating series."""
    x = Decimal(1) / k
    x2 = x * x
    term, total, n = x, Decimal(0), 1
    eps = Decimal(10) ** -65
    while abs(term) > eps:
        total += term / n
        term = -term * x2
        n += 2
    return total


def _pi() -> Decimal:
    return 16 * _atan_inv(5) - 4 * _atan_inv(239)


def _ln2() -> Decimal:
    # ln 2 = 2 atanh(1/3) = 2 sum x^(2k+1)/(2k+1), x = 1/3
    x = Decimal(1) / 3
    x2 = x * x
    term, total, n = x, Decimal(0), 1
    while term > Decimal(10) ** -65:
        total += term / n
        term *= x2
        n += 2
    return 2 * total


def _exp(x: Decimal) -> Decimal:
    term, total, n = Decimal(1), Decimal(1), 1
    while abs(term) > Decimal(10) ** -65:
        term = term * x / n
        total += term
        n += 1
    return total


def _sin_cos(x: Decimal):
    s, c = Decimal(0), Decimal(0)
    term, n = Decimal(1), 0
    while abs(term) > Decimal(10) ** -65 or n < 2:
        if n % 4 == 0:
            c += term
        elif n % 4 == 1:
            s += term
        elif n % 4 == 2:
            c -= term
        else:
            s -= term
        n += 1
        term = term * x / n
    return s, c


def _f32(x: float) -> float:
    return struct.unpack("f", struct.pack("f", x))[0]


def _split(v: Decimal):
    hi = _f32(float(v))
    lo = _f32(float(v - Decimal(hi)))
    return hi, lo


def _trunc_bits(v: Decimal, bits: int) -> float:
    """v truncated to `bits` significant bits (exact in float for bits <= 24)."""
    e = 0
    a = abs(v)
    while a >= 1:
        a /= 2
        e += 1
    while a < Decimal("0.5"):
        a *= 2
        e -= 1
    m = int(a * (1 << bits))  # a in [0.5, 1)
    val = Decimal(m) / (1 << bits) * (Decimal(2) ** e)
    return float(val) if v > 0 else -float(val)


def _lit(x: float) -> str:
    return "%.9ef" % x


def generate() -> str:
    pi, ln2 = _pi(), _ln2()
    c = ln2 / EXP_N
    d = pi / TRIG_STEPS
    out = ["// Generated by paper_2312_02756_gb300/gen_tables.py (decimal arithmetic, 60 digits).",
           "// Do not edit; rebuilt with the library.",
           "#pragma once",
           "#define GVX_EXP_N %d" % EXP_N,
           "#define GVX_TRIG_N %d" % (TRIG_STEPS // 2),
           "GVX_TABLE const gvx_f4 kExpTab[%d] = {" % EXP_N]
    for j in range(EXP_N):
        tm1 = _exp(j * c) - 1
        um1 = 1 - _exp(-j * c)
        a, b = _split(tm1)
        e, f = _split(um1)
        out.append("  {%s, %s, %s, %s}," % (_lit(a), _lit(b), _lit(e), _lit(f)))
    out.append("};")
    out.append("GVX_TABLE const gvx_f4 kTrigTab[%d] = {" % (TRIG_STEPS // 2 + 1))
    for j in range(TRIG_STEPS // 2 + 1):
        s, co = _sin_cos(j * d)
        a, b = _split(s)
        e, f = _split(co)
        out.append("  {%s, %s, %s, %s}," % (_lit(a), _lit(b), _lit(e), _lit(f)))
    out.append("};")
    step = Decimal(1) / (1 << LC_STEP_LOG2)
    out.append("#define GVX_HYP_N %d" % HYP_N)
    out.append("#define GVX_SIN_N %d" % SIN_N)
    out.append("GVX_TABLE const gvx_f4 kHypTab[%d] = {" % (HYP_N + 1))
    for n in range(HYP_N + 1):
        ep, em = _exp(n * step), _exp(-n * step)
        a, b = _split((ep + em) / 2)
        e, f = _split((ep - em) / 2)
        out.append("  {%s, %s, %s, %s}," % (_lit(a), _lit(b), _lit(e), _lit(f)))
    out.append("};")
    out.append("GVX_TABLE const gvx_f4 kSinTab[%d] = {" % (SIN_N + 1))
    for j in range(SIN_N + 1):
        s_, co = _sin_cos(j * step)
        a, b = _split(s_)
        e, f = _split(co)
        out.append("  {%s, %s, %s, %s}," % (_lit(a), _lit(b), _lit(e), _lit(f)))
    out.append("};")
    c0 = _trunc_bits(c, 9)
    c1 = _f32(float(c - Decimal(c0)))
    c2 = _f32(float(c - Decimal(c0) - Decimal(c1)))
    d0 = _trunc_bits(d, 13)
    d1 = _f32(float(d - Decimal(d0)))
    d2 = _f32(float(d - Decimal(d0) - Decimal(d1)))
    pih, pil = _split(pi)
    for name, val in (("kExpC0", c0), ("kExpC1", c1), ("kExpC2", c2),
                      ("kExpInvC", _f32(float(1 / c))), ("kTrigD0", d0), ("kTrigD1", d1),
                      ("kTrigD2", d2), ("kTrigInvD", _f32(float(1 / d))), ("kPiHi", pih),
                      ("kPiLo", pil)):
        out.append("constexpr float %s = %s;" % (name, _lit(val)))
    return "\n".join(out) + "\n"


def write(path: str) -> str:
    text = generate()
    if os.path.exists(path) and open(path).read() == text:
        return path
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        f.write(text)
    os.replace(tmp, path)
    return path


if __name__ == "__main__":
    print(write(sys.argv[1] if len(sys.argv) > 1 else os.path.join(
        os.path.dirname(os.path.abspath(__file__)), "_build", "gvx_tables.inc")))
