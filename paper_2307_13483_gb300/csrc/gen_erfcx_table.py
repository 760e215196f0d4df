"""Writes vbk_erfcx_table.h: piecewise polynomial coefficients of the scaled complementary
error function erfcx(y) = exp(y^2) erfc(y) and of Dawson's integral
D(x) = exp(-x^2) int_0^x exp(t^2) dt on [0, 16).

Each interval [k/2, (k+1)/2) carries the degree-12 polynomial that interpolates the function at
the 13 Chebyshev points of the interval, written in the local variable t = 4 y - (2 k + 1)
(t in [-1, 1]) with monomial coefficients.  Values and the interpolation are computed with
mpmath at 40 significant digits, then rounded to double; the maximum relative errors of the
rounded polynomials are printed by this script (about 1e-15 for erfcx, 3e-15 for Dawson's
integral on [1/2, 16); the library evaluates D by its Taylor series below 1/2).  Above 16 the
library uses the asymptotic series of both functions.

Run from this directory:  python gen_erfcx_table.py > vbk_erfcx_table.h
"""

import mpmath as mp

mp.mp.dps = 40
WIDTH = mp.mpf(1) / 2
NINT = 32
DEG = 12


def erfcx(y):
    return mp.exp(y * y) * mp.erfc(y)


def dawson(x):
    return mp.sqrt(mp.pi) / 2 * mp.exp(-x * x) * mp.erfi(x)


def interval_coefficients(k, f=erfcx):
    a = k * WIDTH
    c, h = a + WIDTH / 2, WIDTH / 2
    n = DEG + 1
    nodes = [mp.cos(mp.pi * (j + mp.mpf(1) / 2) / n) for j in range(n)]
    V = mp.matrix([[t ** p for p in range(n)] for t in nodes])
    coef = mp.lu_solve(V, mp.matrix([f(c + h * t) for t in nodes]))
    return [float(coef[p]) for p in range(n)]


def horner(coef, t):
    r = coef[-1]
    for p in range(len(coef) - 2, -1, -1):
        r = r * t + coef[p]
    return r


def table(f, first):
    rows, worst = [], 0.0
    for k in range(NINT):
        if k < first:
            rows.append([0.0] * (DEG + 1))
            continue
        coef = interval_coefficients(k, f)
        rows.append(coef)
        for j in range(65):
            y = mp.mpf(k) / 2 + mp.mpf(j) / 128
            got = horner(coef, float(4 * y - (2 * k + 1)))
            ref = f(y)
            worst = max(worst, float(abs((got - ref) / ref)))
    return rows, worst


def emit(name, rows):
    print(f"#define {name} \\")
    for k, coef in enumerate(rows):
        tail = ", \\" if k < NINT - 1 else ""
        print("    " + ", ".join(f"{c:.17e}" for c in coef) + tail)


def main():
    import sys

    erows, ew = table(erfcx, 0)
    drows, dw = table(dawson, 1)
    print(f"max relative error: erfcx {ew:.3e}, Dawson (from 1/2) {dw:.3e}", file=sys.stderr)
    print("// Generated by gen_erfcx_table.py (mpmath, 40 digits): erfcx(y) and Dawson's integral on")
    print("// [k/2, (k+1)/2), k = 0..31 (Dawson: k >= 1; row 0 unused), as sum_p c[k][p] t^p with")
    print("// t = 4 y - (2 k + 1).  Do not edit.")
    print("#pragma once")
    print(f"#define VBK_ERFCX_NINT {NINT}")
    print(f"#define VBK_ERFCX_DEG {DEG}")
    emit("VBK_ERFCX_COEFFS", erows)
    emit("VBK_DAWSON_COEFFS", drows)


if __name__ == "__main__":
    main()
