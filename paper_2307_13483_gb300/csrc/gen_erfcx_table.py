"""Writes vbk_erfcx_table.h: piecewise polynomial coefficients of the scaled complementary
error function erfcx(y) = exp(y^2) erfc(y) on [0, 16).

Each interval [k/2, (k+1)/2) carries the degree-12 polynomial that interpolates erfcx at the
13 Chebyshev points of the interval, written in the local variable t = 4 y - (2 k + 1)
(t in [-1, 1]) with monomial coefficients.  Values and the interpolation are computed with
mpmath at 40 significant digits, then rounded to double; the maximum relative error of the
rounded polynomials on the interval is about 1e-15 (printed by this script).  Above 16 the
library uses the asymptotic series of erfcx.

Run from this directory:  python gen_erfcx_table.py > vbk_erfcx_table.h
"""

import mpmath as mp

mp.mp.dps = 40
WIDTH = mp.mpf(1) / 2
NINT = 32
DEG = 12


def erfcx(y):
    return mp.exp(y * y) * mp.erfc(y)


def interval_coefficients(k):
    a = k * WIDTH
    c, h = a + WIDTH / 2, WIDTH / 2
    n = DEG + 1
    nodes = [mp.cos(mp.pi * (j + mp.mpf(1) / 2) / n) for j in range(n)]
    V = mp.matrix([[t ** p for p in range(n)] for t in nodes])
    coef = mp.lu_solve(V, mp.matrix([erfcx(c + h * t) for t in nodes]))
    return [float(coef[p]) for p in range(n)]


def horner(coef, t):
    r = coef[-1]
    for p in range(len(coef) - 2, -1, -1):
        r = r * t + coef[p]
    return r


def main():
    rows, worst = [], 0.0
    for k in range(NINT):
        coef = interval_coefficients(k)
        rows.append(coef)
        for j in range(65):
            y = mp.mpf(k) / 2 + mp.mpf(j) / 128
            got = horner(coef, float(4 * y - (2 * k + 1)))
            ref = erfcx(y)
            worst = max(worst, float(abs((got - ref) / ref)))
    import sys

    print(f"max relative error of the rounded polynomials: {worst:.3e}", file=sys.stderr)
    print("// Generated by gen_erfcx_table.py (mpmath, 40 digits): erfcx(y) on [k/2, (k+1)/2),")
    print("// k = 0..31, as sum_p c[k][p] t^p with t = 4 y - (2 k + 1).  Do not edit.")
    print("#pragma once")
    print(f"#define VBK_ERFCX_NINT {NINT}")
    print(f"#define VBK_ERFCX_DEG {DEG}")
    print("#define VBK_ERFCX_COEFFS \\")
    for k, coef in enumerate(rows):
        tail = ", \\" if k < NINT - 1 else ""
        print("    " + ", ".join(f"{c:.17e}" for c in coef) + tail)


if __name__ == "__main__":
    main()
