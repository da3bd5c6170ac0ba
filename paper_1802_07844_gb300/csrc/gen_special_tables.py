"""Writes special_tables.inc: coefficients of the FP64 erfc / exp evaluation
used by the real-space kernel.

erfc(t) = exp(-t^2) * erfcx(t).  erfcx(t) = exp(t^2) erfc(t) is smooth and
slowly varying on [0, 12); it is approximated on intervals of width 1/8 by the
Chebyshev interpolant of degree 8 (nodes cos(pi (k + 1/2)/9)), rewritten as a
polynomial in the local variable u = 16 (t - centre) in [-1, 1].  The values come
from mpmath at 40 digits; the interpolation error is below 1e-15 relative.

exp(-x) uses Tang's table-driven reduction (P. T. P. Tang, ACM TOMS 15, 1989):
-x = m ln2/64 + r with m = round(-x 64/ln2), |r| <= ln2/128, ln2/64 split into a
head of 36 significant bits (m * head is exact for |m| < 2^17) and a tail; then
e^{-x} = 2^n 2^{j/64} e^r with m = 64 n + j, 2^{j/64} from a 64-entry table and
e^r from its Taylor polynomial of degree 5 (remainder < 4e-17 relative).

Run: python gen_special_tables.py  (needs mpmath)
"""
import os

import mpmath as mp

mp.mp.dps = 40
WIDTH = mp.mpf(1) / 8
DEG = 8
NINT = 96  # [0, 12)


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
             f"// erfcx on [0, 12): {NINT} intervals of width 1/{int(1 / WIDTH)}, degree {DEG} in"
             f" u = {int(2 / WIDTH)} (t - centre)",
             f"#define HSE_ERFCX_NINT {NINT}", f"#define HSE_ERFCX_DEG {DEG}",
             f"#define HSE_ERFCX_INV_WIDTH {int(1 / WIDTH)}",
             "#define HSE_ERFCX_COEFS \\"]
    for i in range(NINT):
        a = WIDTH * i
        co = interval_coeffs(a, a + WIDTH)
        lines.append("    " + ", ".join(mp.nstr(x, 20, strip_zeros=False) for x in co) +
                     (", \\" if i < NINT - 1 else ""))
    ln2 = mp.log(2)
    c = ln2 / 64
    e = mp.floor(mp.log(c, 2))
    head = mp.floor(c / mp.mpf(2) ** (e - 35)) * mp.mpf(2) ** (e - 35)  # 36 significant bits
    lines.append(f"constexpr double kLn2By64Head = {mp.nstr(head, 25)};")
    lines.append(f"constexpr double kLn2By64Tail = {mp.nstr(c - head, 25)};")
    lines.append(f"constexpr double k64Log2e = {mp.nstr(64 / ln2, 25)};")
    lines.append("#define HSE_EXP_TAYLOR5_COEFS " + ", ".join(mp.nstr(1 / mp.factorial(k), 25) for k in range(6)))
    lines.append("#define HSE_EXP2_J64 " + ", ".join(mp.nstr(mp.mpf(2) ** (mp.mpf(j) / 64), 25) for j in range(64)))
    open(out, "w").write("\n".join(lines) + "\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
