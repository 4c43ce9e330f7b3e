"""Writes fabf_fp64_tables.h: the coefficient tables of the library's own
binary64 erfcx and exp (fabf_device.cuh, `erfcx_fp64`, `exp_fp64`).

erfcx(x) = exp(x^2) erfc(x), x >= 0:
  * x < 12: 384 intervals [i/32, (i+1)/32); on each, the Chebyshev
    interpolant of degree 7 at the Chebyshev points (computed with mpmath at
    50 digits), rewritten as a polynomial in t = 64x - 2i - 1 in [-1, 1) and
    rounded to binary64.  Its truncation error is below 2e-18 relative
    (measured against mpmath on every interval).
  * x >= 12: erfcx(x) = g(u) / x with u = 1/x^2 in (0, 1/144] and
    g(u) = x erfcx(x) (g(0) = 1/sqrt(pi), the asymptotic expansion's limit),
    the Chebyshev interpolant of g of degree 7 on [0, 1/144] in
    t = 288u - 1 (truncation below 2e-18).
  The constant coefficient of each piece is also written as hi + lo.
exp: Tang's table-driven method (ACM TOMS 15(2), 1989): 2^(j/1024),
  j = 0..1023, correctly rounded, and the reduction constant ln2/1024 split in
  two parts (|r| <= ln2/2048: a degree-4 polynomial truncates below 4e-20).

Run with: python gen_fp64_tables.py > fabf_fp64_tables.h  (mpmath needed; the
header is committed, so building the library does not run this script)."""
from __future__ import annotations

import struct
import sys

import mpmath as mp

mp.mp.dps = 50

DEG = 7                  # polynomial degree of every erfcx piece
PER_UNIT = 32            # erfcx pieces per unit of x
XL = 12                  # erfcx pieces on [0, XL); the large-x polynomial beyond
NSEG = PER_UNIT * XL
EXP_BITS = 10
EXP_J = 1 << EXP_BITS    # table entries of exp
NCOEF = DEG + 1


def erfcx(x):
    return mp.exp(x * x) * mp.erfc(x)


def g_large(u):
    if u == 0:
        return 1 / mp.sqrt(mp.pi)
    x = 1 / mp.sqrt(u)
    return x * erfcx(x)


def cheb_interp_power(f, a, b, n):
    """Power-basis coefficients p_0..p_n in t in [-1, 1] (x = mid + half t) of
    the degree-n interpolant of f at the Chebyshev points of [a, b]."""
    a, b = mp.mpf(a), mp.mpf(b)
    mid, half = (a + b) / 2, (b - a) / 2
    pts = [mp.cos(mp.pi * (k + mp.mpf(1) / 2) / (n + 1)) for k in range(n + 1)]
    vals = [f(mid + half * t) for t in pts]
    c = []
    for j in range(n + 1):
        s = mp.fsum(vals[k] * mp.cos(mp.pi * j * (k + mp.mpf(1) / 2) / (n + 1)) for k in range(n + 1))
        c.append(2 * s / (n + 1) if j else s / (n + 1))
    # Chebyshev series -> power basis: T_0 = 1, T_1 = t, T_{j+1} = 2t T_j - T_{j-1}
    T = [[mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]]
    for j in range(2, n + 1):
        nxt = [mp.mpf(0)] * (j + 1)
        for k, v in enumerate(T[j - 1]):
            nxt[k + 1] += 2 * v
        for k, v in enumerate(T[j - 2]):
            nxt[k] -= v
        T.append(nxt)
    p = [mp.mpf(0)] * (n + 1)
    for j in range(n + 1):
        for k, v in enumerate(T[j]):
            p[k] += c[j] * v
    return p


def hexd(v) -> str:
    return float(v).hex()


def main(out=sys.stdout):
    pieces = [cheb_interp_power(erfcx, mp.mpf(i) / PER_UNIT, mp.mpf(i + 1) / PER_UNIT, DEG) for i in range(NSEG)]
    pieces.append(cheb_interp_power(g_large, 0, mp.mpf(1) / (XL * XL), DEG))
    nrow = NSEG + 1
    w = out.write
    w("// Generated by gen_fp64_tables.py (mpmath, 50 digits); do not edit.\n")
    w("// erfcx pieces: coefficient k of piece i at [k * %d + i]; pieces 0..%d are\n" % (nrow, NSEG - 1))
    w("// polynomials in t = %dx - 2i - 1 on [i/%d, (i+1)/%d), piece %d the large-x\n"
      % (2 * PER_UNIT, PER_UNIT, PER_UNIT, NSEG))
    w("// polynomial in t = %d/x^2 - 1 of x erfcx(x).\n" % (2 * XL * XL))
    w("#pragma once\n\n")
    w("#define FABF_ERFCX_DEG %d\n" % DEG)
    w("#define FABF_ERFCX_NSEG %d\n" % NSEG)
    w("#define FABF_ERFCX_PER_UNIT %d.0\n" % PER_UNIT)
    w("#define FABF_ERFCX_LARGE_T %d.0      // t = LARGE_T / x^2 - 1 beyond XL\n" % (2 * XL * XL))
    w("#define FABF_ERFCX_XL_HIGH_WORD 0x%08X   // high word of %d.0 (low word 0)\n"
      % (struct.unpack("<Q", struct.pack("<d", float(XL)))[0] >> 32, XL))
    w("#define FABF_ERFCX_TABLE \\\n")
    rows = []
    for k in range(NCOEF):
        rows.append("    " + ", ".join(hexd(pieces[i][k]) for i in range(nrow)))
    w(", \\\n".join(rows) + "\n\n")
    # the low parts of the constant coefficients (p_0 = hi + lo): the final
    # addition of each evaluation is then one rounding of a value accurate
    # well beyond binary64
    w("#define FABF_ERFCX_P0_LO \\\n")
    lo = [hexd(pieces[i][0] - mp.mpf(float(pieces[i][0]))) for i in range(nrow)]
    w(", \\\n".join("    " + ", ".join(lo[r:r + 4]) for r in range(0, nrow, 4)) + "\n\n")
    # exp: 2^(j/EXP_J) correctly rounded, and ln2/EXP_J = L1 + L2
    w("#define FABF_EXP_TABLE_BITS %d\n" % EXP_BITS)
    w("#define FABF_EXP2_TABLE \\\n")
    vals = [hexd(mp.mpf(2) ** (mp.mpf(j) / EXP_J)) for j in range(EXP_J)]
    w(", \\\n".join("    " + ", ".join(vals[r:r + 4]) for r in range(0, EXP_J, 4)) + "\n\n")
    ln2_j = mp.log(2) / EXP_J
    L1 = mp.mpf(float(ln2_j))
    L2 = mp.mpf(float(ln2_j - L1))
    w("#define FABF_EXP_INV_L %s   // %d / ln 2\n" % (hexd(EXP_J / mp.log(2)), EXP_J))
    w("#define FABF_EXP_L1 %s      // ln 2 / %d, leading part\n" % (hexd(L1), EXP_J))
    w("#define FABF_EXP_L2 %s      // ln 2 / %d - L1\n" % (hexd(L2), EXP_J))


if __name__ == "__main__":
    main()
