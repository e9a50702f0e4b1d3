"""Generate expint_cheb.inc: Chebyshev coefficients of A(z) = e^z E1(z) and
B(z) = e^z E2(z) on [1, 16); the Horner coefficients of the Ein series; the
constants and 2^{-j/256} table of the table-driven e^{-x}.

FP64: eight intervals [a_k, a_{k+1}], a_k the double nearest 2^{k/2}
(ratio sqrt 2).  The device maps z to t = fma(z, s_k, o_k) with the double
constants s_k = 2 / (a_{k+1} - a_k), o_k = -(a_k + a_{k+1}) / (a_{k+1} - a_k);
the coefficients are fitted through that same map, z = (t - o_k) / s_k, at
the Chebyshev points of the first kind, in 40-digit arithmetic (mpmath):
    f = c_0 / 2 + sum_{k>=1} c_k T_k(t).
On each interval the nearest singularity of A and B is the log branch point
at z = 0, (1 + sqrt 2) / (sqrt 2 - 1) = 5.83 half-widths from the centre, so
the coefficients decay like 11.66^{-k}: 18 terms reach ~1e-19.
The device evaluates 16-term fits (Chebyshev coefficients beyond the 15th
are below 1e-17 of c_0) in the monomial basis of t with Horner's rule: the
Chebyshev series is converted exactly (in 40 digits) to powers of t; since
sum |a_j| / |f| <= 1.4 on every interval, Horner's rounding stays near one
ulp -- 15 fused multiply-adds instead of 17 Clenshaw steps of two
operations.
FP32: the leading 12 coefficients on the four intervals [1,2], [2,4], [4,8],
[8,16] (26-point fits).

Run from the repository root:  python paper_1811_05224_gb300/csrc/gen_expint_tables.py
"""
import os

import mpmath as mp

mp.mp.dps = 40
NC = 18
NH = 16
NC_F32_FIT = 26
NCF = 12
NEIN = 18
INTERVALS = [(1, 2), (2, 4), (4, 8), (8, 16)]
N_INT64 = 8


def f64_intervals():
    """Endpoints a_k (doubles nearest 2^{k/2}) and the device's map constants."""
    a = [float(mp.power(2, mp.mpf(k) / 2)) for k in range(N_INT64 + 1)]
    out = []
    for k in range(N_INT64):
        lo, hi = a[k], a[k + 1]
        s = 2.0 / (hi - lo)
        o = -(lo + hi) / (hi - lo)
        out.append((lo, hi, s, o))
    return out


def cheb_coeffs_map(f, s, o, n=NC):
    """Chebyshev coefficients in t of f((t - o) / s) on t in [-1, 1]."""
    s, o = mp.mpf(s), mp.mpf(o)
    nodes = [mp.cos(mp.pi * (j + mp.mpf(1) / 2) / n) for j in range(n)]
    vals = [f((t - o) / s) for t in nodes]
    out = []
    for k in range(n):
        acc = mp.fsum(v * mp.cos(k * mp.pi * (j + mp.mpf(1) / 2) / n) for j, v in enumerate(vals))
        out.append(2 * acc / n)
    return out


def cheb_to_monomial(c):
    """Exact coefficients a_j of c_0 / 2 + sum_{k>=1} c_k T_k(t) = sum_j a_j t^j
    (T_0 = 1, T_1 = t, T_{k+1} = 2 t T_k - T_{k-1})."""
    n = len(c)
    T = [[mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]]
    for k in range(2, n):
        t = [mp.mpf(0)] * (k + 1)
        for j, v in enumerate(T[k - 1]):
            t[j + 1] += 2 * v
        for j, v in enumerate(T[k - 2]):
            t[j] -= v
        T.append(t)
    a = [mp.mpf(0)] * n
    for k in range(n):
        ck = c[k] / 2 if k == 0 else c[k]
        for j, v in enumerate(T[k]):
            a[j] += ck * v
    return a


def cheb_coeffs(f, a, b, n=NC_F32_FIT):
    nodes = [mp.cos(mp.pi * (j + mp.mpf(1) / 2) / n) for j in range(n)]
    vals = [f((b - a) / mp.mpf(2) * t + (a + b) / mp.mpf(2)) for t in nodes]
    out = []
    for k in range(n):
        s = mp.fsum(v * mp.cos(k * mp.pi * (j + mp.mpf(1) / 2) / n) for j, v in enumerate(vals))
        out.append(2 * s / n)
    return out


def main():
    A = lambda z: mp.e ** z * mp.e1(z)            # noqa: E731
    B = lambda z: mp.e ** z * mp.expint(2, z)     # noqa: E731
    iv = f64_intervals()
    lines = ["// Generated by gen_expint_tables.py: polynomial fits of",
             "// A(z) = e^z E1(z) and B(z) = e^z E2(z) on [1, 16): FP64 %d powers of t on each of" % NH,
             "// %d intervals [a_k, a_{k+1}] (a_k = 2^{k/2}), t = fma(z, kChebS[k], kChebO[k]),"  % N_INT64,
             "// f = sum_j a_j t^j (a %d-term Chebyshev fit converted exactly);" % NH,
             "// FP32 %d Chebyshev terms on [1,2], [2,4], [4,8], [8,16]; f = c0/2 + sum_k c_k T_k(t)." % NCF,
             "#pragma once", "namespace stbem {",
             "constexpr int kChebN = %d;" % NC,
             "constexpr int kChebIntervals = %d;" % N_INT64]
    r = lambda x: repr(float(x))               # noqa: E731  shortest round-trip double literal
    lines.append("static __constant__ const double kChebSplit[4] = {%s};" % ", ".join(r(iv[2 * e][1]) for e in range(4)))
    lines.append("static __constant__ const double kChebS[%d] = {%s};" % (N_INT64, ", ".join(r(x[2]) for x in iv)))
    lines.append("static __constant__ const double kChebO[%d] = {%s};" % (N_INT64, ", ".join(r(x[3]) for x in iv)))
    # the 18-term fits as powers of t, a_0 .. a_{NH-1}, for Horner's rule
    tails, drop = [], []
    lines.append("constexpr int kHornN = %d;" % NH)
    for name, f in (("kHornE1", A), ("kHornE2", B)):
        lines.append("static __constant__ const double %s[%d][%d] = {" % (name, N_INT64, NH))
        for lo, hi, sk, ok in iv:
            c = cheb_coeffs_map(f, sk, ok)                 # 18 terms: the size of the tail
            tails.append(abs(c[-1] / c[0]))
            c16 = cheb_coeffs_map(f, sk, ok, NH)           # the fit that is converted
            drop.append(max(abs(x) for x in c[NH:]) / abs(c[0]))
            a = cheb_to_monomial(c16)
            lines.append("  {" + ", ".join(mp.nstr(x, 20, min_fixed=0, max_fixed=0) for x in a) + "},")
        lines.append("};")
    print("largest |c_17 / c_0|: %.2e; largest dropped |c_k / c_0|, k >= %d: %.2e" % (max(tails), NH, max(drop)))
    # FP32 copies: the leading 12 coefficients (the tail is below 2e-9 of c0)
    for name, f in (("kChebE1f", A), ("kChebE2f", B)):
        lines.append("static __constant__ const float %s[%d][%d] = {" % (name, len(INTERVALS), NCF))
        for a, b in INTERVALS:
            c = cheb_coeffs(f, mp.mpf(a), mp.mpf(b))[:NCF]
            lines.append("  {" + ", ".join(mp.nstr(x, 10, min_fixed=0, max_fixed=0) + "f" for x in c) + "},")
        lines.append("};")
    lines.append("constexpr int kChebNf = %d;" % NCF)
    # Ein(z) = sum_{k>=1} (-1)^{k+1} z^k / (k k!): Horner coefficients, k = 1..18
    # (the dropped tail is below 1e-17 for |z| <= 1)
    coef = [(-1) ** (k + 1) / (mp.mpf(k) * mp.factorial(k)) for k in range(1, NEIN + 1)]
    lines.append("constexpr int kEinTerms = %d;" % NEIN)
    lines.append("static __constant__ const double kEinCoef[%d] = {%s};" % (
        NEIN, ", ".join(mp.nstr(c, 20, min_fixed=0, max_fixed=0) for c in coef)))
    # e^{-x} by reduction to r = x - n ln2/256: table 2^{-j/256}, j = 0..255,
    # 256/ln2 and a two-part ln2/256 whose leading part has 34 significant
    # bits (n ln2_hi is exact for n < 2^19, i.e. x < 1.4e3)
    l = mp.log(2) / 256
    e = int(mp.floor(mp.log(l, 2)))            # l = 1.xx * 2^e
    hi = mp.ldexp(mp.floor(mp.ldexp(l, 33 - e)), -(33 - e))
    lo = l - hi
    tab = [mp.power(2, -mp.mpf(j) / 256) for j in range(256)]
    lines.append("constexpr double kInvLn2x256 = %s;" % mp.nstr(256 / mp.log(2), 20, min_fixed=0, max_fixed=0))
    lines.append("constexpr double kLn2by256Hi = %s;" % mp.nstr(hi, 25, min_fixed=0, max_fixed=0))
    lines.append("constexpr double kLn2by256Lo = %s;" % mp.nstr(lo, 20, min_fixed=0, max_fixed=0))
    lines.append("static __constant__ const double kExp2Tab[256] = {%s};" % ", ".join(
        mp.nstr(t, 20, min_fixed=0, max_fixed=0) for t in tab))
    # e^{-c k} with k = sigma 2048/ln2 for the hot loops: c k = n + r by a fused
    # multiply-add rounding, table 2^{-j/2048}, j = 0..2047, and Taylor
    # coefficients (-l)^k / k!, k = 1..3, l = ln2/2048 (remainder
    # (l/2)^4 / 24 < 4e-17)
    l11 = mp.log(2) / 2048
    tab11 = [mp.power(2, -mp.mpf(j) / 2048) for j in range(2048)]
    lines.append("constexpr double kInvLn2x2048 = %s;" % mp.nstr(2048 / mp.log(2), 20, min_fixed=0, max_fixed=0))
    for k in range(1, 4):
        lines.append("constexpr double kExpProdC%d = %s;" % (
            k, mp.nstr((-l11) ** k / mp.factorial(k), 21, min_fixed=0, max_fixed=0)))
    lines.append("static __constant__ const double kExp2Tab2048[2048] = {%s};" % ", ".join(
        mp.nstr(t, 20, min_fixed=0, max_fixed=0) for t in tab11))
    lines.append("}  // namespace stbem")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "expint_cheb.inc")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(out)


if __name__ == "__main__":
    main()
