"""Writes special_tables.inc: coefficients of the FP64 erfc / exp evaluation
used by the real-space kernel.

erfc(t) = exp(-t^2) * erfcx(t).  erfcx(t) = exp(t^2) erfc(t) is smooth and
slowly varying on [0, 12); it is approximated on intervals of width 1/4 by the
Chebyshev interpolant of degree 10 (nodes cos(pi (k + 1/2)/11)), rewritten as a
polynomial in the local variable u = 8 (t - centre) in [-1, 1].  The values come
from mpmath at 40 digits; the interpolation error is below 4e-16 relative.

exp(-x) uses the Cody-Waite argument reduction x * log2(e) = n + f with ln 2 split
into a head of 40 significant bits (so n * head is exact for |n| < 2^13) and a
tail, then the Taylor polynomial of e^r to degree 13 on |r| <= ln(2)/2.

Run: python gen_special_tables.py  (needs mpmath)
"""
import os

import mpmath as mp

mp.mp.dps = 40
WIDTH = mp.mpf(1) / 4
DEG = 10
NINT = 48  # [0, 12)


def erfcx(t):
    return mp.exp(t * t) * mp.erfc(t)


def interval_coeffs(a, b):
    c, w = (a + b) / 2, (b - a) / 2
    nodes = [mp.cos(mp.pi * (k + mp.mpf(1) / 2) / (DEG + 1)) for k in range(DEG + 1)]
    V = mp.matrix([[u ** j for j in range(DEG + 1)] for u in nodes])
    y = mp.matrix([erfcx(c + w * u) for u in nodes])
    return [x for x in mp.lu_solve(V, y)]


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "special_tables.inc")
    lines = ["// generated by gen_special_tables.py -- do not edit",
             f"// erfcx on [0, {NINT}/4): {NINT} intervals of width 1/4, degree {DEG} in u = 8 (t - centre)",
             f"#define HSE_ERFCX_NINT {NINT}", f"#define HSE_ERFCX_DEG {DEG}",
             "#define HSE_ERFCX_COEFS \\"]
    for i in range(NINT):
        a = WIDTH * i
        co = interval_coeffs(a, a + WIDTH)
        lines.append("    " + ", ".join(mp.nstr(x, 20, strip_zeros=False) for x in co) +
                     (", \\" if i < NINT - 1 else ""))
    ln2 = mp.log(2)
    head = mp.mpf(float(mp.floor(ln2 * 2 ** 40))) / 2 ** 40
    tail = ln2 - head
    lines.append(f"constexpr double kLn2Head = {mp.nstr(head, 25)};")
    lines.append(f"constexpr double kLn2Tail = {mp.nstr(tail, 25)};")
    lines.append(f"constexpr double kLog2e = {mp.nstr(1 / ln2, 25)};")
    lines.append("#define HSE_EXP_TAYLOR_COEFS " + ", ".join(mp.nstr(1 / mp.factorial(k), 25) for k in range(14)))
    open(out, "w").write("\n".join(lines) + "\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
