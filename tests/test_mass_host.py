"""Host numerics of the consistent mixed mass (stbem_mixed_mass_inverse),
compiled from the library's own header for the CPU: the matrix against the
oracle's mixed_mass_matrix, the Gauss-Jordan inverse against numpy's."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import workloads as W
from oracle import assembly
from oracle.geometry import BoundaryMesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1811_05224_gb300", "csrc")


@pytest.fixture(scope="module")
def lib():
    out = os.path.join(tempfile.mkdtemp(), "libmass_host.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I" + CSRC,
                    os.path.join(ROOT, "tests", "hostcheck", "mass_shim.cpp"), "-o", out], check=True)
    return ctypes.CDLL(out)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@pytest.mark.parametrize("X", [W.unit_square(4), W.l_shape(64, seed=3), W.star(8, 4, seed=5)],
                         ids=["square16", "lshape64", "star32"])
def test_mixed_mass_and_inverse(lib, X):
    m = BoundaryMesh(X, 1.0, 7, 0.9)
    N = m.N
    h = np.ascontiguousarray(m.h)
    A = np.zeros((N, N))
    lib.mh_matrix(_dp(h), N, ctypes.c_double(m.ht), _dp(A))
    ref = assembly.mixed_mass_matrix(m)
    assert np.abs(A - ref).max() <= 1e-15 * np.abs(ref).max()
    Inv = np.zeros((N, N))
    assert lib.mh_inverse(_dp(h), N, ctypes.c_double(m.ht), _dp(Inv)) == 1
    R = np.linalg.inv(ref)
    assert np.abs(Inv - R).max() <= 1e-12 * np.abs(R).max()
    assert np.abs(Inv @ ref - np.eye(N)).max() <= 1e-12
