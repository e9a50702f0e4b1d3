"""The CUDA path's device numerics compiled for the host (same headers) and
checked on the CPU against the C library / scipy / numpy: the table-driven
e^{-x}, E1 and E2 in FP64 and FP32, the Ein series, Gauss-Legendre tables,
and the double time integrals of every branch (timeint.cuh) against the
oracle's (oracle.timeint, the same rule written independently)."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest
from scipy.special import exp1, expn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1811_05224_gb300", "csrc")


@pytest.fixture(scope="module")
def lib():
    out = os.path.join(tempfile.mkdtemp(), "libnumerics_host.so")
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I" + CSRC,
           "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "hostcheck", "numerics_shim.cpp"),
           os.path.join(CSRC, "rules_host.cpp"), "-o", out]
    subprocess.run(cmd, check=True)
    L = ctypes.CDLL(out)
    L.nc_init()
    return L


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def test_exp_neg_within_two_ulp(lib):
    x = np.concatenate([np.linspace(0.0, 1.0, 20001), np.linspace(1.0, 707.9, 200001),
                        np.logspace(-300, 0, 2001)])
    out = np.zeros_like(x)
    lib.nc_exp_neg(_d(x), len(x), _d(out))
    ref = np.exp(-x)
    ulp = np.spacing(ref)
    assert np.max(np.abs(out - ref) / ulp) <= 2.0


def test_exp_prod_within_two_ulp(lib):
    """e^{-c k ln2/2048} of the hot loops (k = sigma 2048/ln2 from a node
    table) against extended-precision numpy for the same c and k: the product
    c k is rounded to its integer part by a fused multiply-add and the
    remainder is exact, so the errors are the table, the cubic and the final
    product."""
    rng = np.random.default_rng(4)
    kmax = 700.0 * 2048 / np.log(2.0)
    y = np.concatenate([np.linspace(0.0, 3.0, 20001), np.linspace(3.0, kmax, 300001)[:-1],
                        np.logspace(-300, 0, 2001)])
    k = np.exp(rng.uniform(np.log(1e-3), np.log(1e6), y.size))      # node values over a wide range
    c = y / k
    out = np.zeros_like(y)
    lib.nc_exp_prod(_d(c), _d(k), len(y), _d(out))
    l = np.log(np.longdouble(2)) / np.longdouble(2048)
    ref = np.exp(-(c.astype(np.longdouble) * k.astype(np.longdouble)) * l)
    ulp = np.spacing(ref.astype(np.float64))
    err = np.abs(out.astype(np.longdouble) - ref) / ulp.astype(np.longdouble)
    assert float(err.max()) <= 2.5, float(err.max())


def test_e1_e2_fp64_and_fp32(lib):
    z = np.concatenate([np.logspace(-12, 0, 400), np.linspace(1.0, 16.5, 2000), np.logspace(1.2, 2.85, 300)])
    e1, e2 = np.zeros_like(z), np.zeros_like(z)
    lib.nc_e1e2(_d(z), len(z), _d(e1), _d(e2))
    assert np.max(np.abs(e1 / exp1(z) - 1)) < 4e-15
    assert np.max(np.abs(e2 / expn(2, z) - 1)) < 4e-15
    # E1 alone: the same operations as the E1 half of e1e2, bitwise
    zz = np.concatenate([z, np.linspace(690.0, 760.0, 301)])
    a, b, c = np.zeros_like(zz), np.zeros_like(zz), np.zeros_like(zz)
    lib.nc_e1e2(_d(zz), len(zz), _d(a), _d(b))
    lib.nc_e1only(_d(zz), len(zz), _d(c))
    assert np.array_equal(a, c)
    zf = z[z < 85].astype(np.float32)
    f1, f2 = np.zeros_like(zf), np.zeros_like(zf)
    P = ctypes.POINTER(ctypes.c_float)
    lib.nc_e1e2f(zf.ctypes.data_as(P), len(zf), f1.ctypes.data_as(P), f2.ctypes.data_as(P))
    zd = zf.astype(np.float64)
    assert np.max(np.abs(f1 / exp1(zd) - 1)) < 1e-6
    assert np.max(np.abs(f2 / expn(2, zd) - 1)) < 1e-6


def test_ein_and_gauss_tables(lib):
    z = np.linspace(1e-6, 1.0, 1001)
    out = np.zeros_like(z)
    lib.nc_ein(_d(z), len(z), _d(out))
    ref = exp1(z) + np.euler_gamma + np.log(z)     # Ein = E1 + gamma + ln z
    assert np.max(np.abs(out - ref)) < 4e-16 * 4
    for n in (3, 4, 6, 8, 12, 16):
        x, w = np.zeros(n), np.zeros(n)
        lib.nc_gauss(n, _d(x), _d(w))
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.allclose(x, 0.5 * (xr + 1), atol=2e-16) and np.allclose(w, 0.5 * wr, atol=4e-16)


def test_time_integrals_match_oracle(lib):
    """lag_kernel (d = 0; d = 1 series and closed; d >= 2 closed and Peano)
    against oracle.timeint over c spanning both sides of every switch.  Both
    evaluate the same formulas with their own E1/E2 (within 2e-15 of each
    other); the closed second differences amplify that by at most their
    cancellation, bounded here by 1e-12 relative."""
    from oracle import timeint
    from oracle.rules import DEFAULT_RULES as R
    ht, alpha = 1.0 / 64.0, 0.7
    c = np.logspace(-9, 3, 241)
    for d in (0, 1, 2, 3, 7, 8, 31, 32, 100, 300):
        for kind, ref_fn in ((0, timeint.lag_V), (1, timeint.lag_Kq), (2, timeint.lag_1)):
            out = np.zeros_like(c)
            lib.nc_lag(kind, _d(c), len(c), d, ctypes.c_double(ht), ctypes.c_double(alpha), _d(out))
            ref = ref_fn(c, d, ht, alpha, R)
            big = np.abs(ref) > 1e-280
            assert np.all(np.abs(out[big] - ref[big]) <= 1e-12 * np.abs(ref[big])), (d, kind)


def test_time_integral_c_derivatives_match_oracle(lib):
    """dtimeint.cuh (the gradient kernels' values and d/dc: lags 0 and 1, and
    the closed second difference at lags >= 2 where c / (d ht) > d / 2)
    against oracle.timeint's dlag_V / dlag_Kq."""
    from oracle import timeint
    from oracle.rules import DEFAULT_RULES as R
    ht, alpha = 1.0 / 64.0, 0.7
    for d in (0, 1, 2, 5, 40):
        c = np.logspace(-9, 3, 241)
        if d >= 2:
            c = c[c / (d * ht) > 0.5 * d]
        for kind, vf, df in ((0, timeint.lag_V, timeint.dlag_V), (1, timeint.lag_Kq, timeint.dlag_Kq)):
            k, dk = np.zeros_like(c), np.zeros_like(c)
            lib.nc_dlag(kind, _d(c), len(c), d, ctypes.c_double(ht), ctypes.c_double(alpha), _d(k), _d(dk))
            rv, rd = vf(c, d, ht, alpha, R), df(c, d, ht, alpha, R)
            for got, ref in ((k, rv), (dk, rd)):
                big = np.abs(ref) > 1e-280
                assert np.all(np.abs(got[big] - ref[big]) <= 1e-12 * np.abs(ref[big])), (d, kind)


def test_nonuniform_time_integrals_match_oracle(lib):
    """nonuniform_time.cuh (the device form of the non-uniform grids' time
    integrals: d = 0; d = 1 series and closed; d >= 2 closed and Peano with
    up to three pieces) against oracle.nonuniform on a graded grid and on a
    uniform one, over c spanning every switch."""
    from oracle import nonuniform as NU
    alpha = 0.7
    grids = [np.array([0.0, 0.02, 0.05, 0.07, 0.11, 0.16, 0.19, 0.26, 0.30, 0.37, 0.41]),
             np.arange(11) / 64.0]
    c = np.logspace(-9, 1, 161)
    for t in grids:
        for m in range(10):
            for n in range(m + 1):
                s = (t[m + 1] - t[n], t[m + 1] - t[n + 1], t[m] - t[n], t[m] - t[n + 1])
                for kind, name in ((0, "V"), (1, "K"), (2, "1")):
                    out = np.zeros_like(c)
                    lib.nc_nu_time(kind, _d(c), len(c), m - n, *[ctypes.c_double(x) for x in s],
                                   ctypes.c_double(alpha), _d(out))
                    ref = NU.time_integral(name, c, t, m, n, alpha)
                    big = np.abs(ref) > 1e-280
                    assert np.all(np.abs(out[big] - ref[big]) <= 1e-12 * np.abs(ref[big])), (m, n, name)
