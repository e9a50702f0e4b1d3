"""Host logic of the triangulation handle (stbem_domain_create), compiled
from the library's own header for the CPU: boundary-vertex matching against
the oracle's nearest-node map, and the node-disjoint colouring that lets the
M_h^0 assembly launch one colour at a time without write conflicts."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import workloads as W
from oracle import initial as OI
from oracle.geometry import BoundaryMesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1811_05224_gb300", "csrc")


@pytest.fixture(scope="module")
def lib():
    out = os.path.join(tempfile.mkdtemp(), "libdomain_host.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I" + CSRC,
                    os.path.join(ROOT, "tests", "hostcheck", "domain_shim.cpp"), "-o", out], check=True)
    return ctypes.CDLL(out)


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


CASES = [
    ("square8", lambda: W.unit_square(8), lambda: W.square_triangulation(8)),
    ("jitter16", lambda: W.unit_square(16), lambda: W.square_triangulation(16, jitter=0.3, seed=4)),
    ("lshape", lambda: W.l_shape(32, jitter=(1.0, 1.0)), lambda: W.lshape_triangulation(8)),
]


@pytest.mark.parametrize("name,mkX,mkT", CASES)
def test_matching_equals_oracle_and_colouring_is_node_disjoint(lib, name, mkX, mkT):
    X = mkX()
    nodes, tris = mkT()
    M, K, N = nodes.shape[0], tris.shape[0], X.shape[0]
    nd = np.ascontiguousarray(nodes, dtype=np.float64)
    xy = np.ascontiguousarray(X, dtype=np.float64)
    bnode = np.zeros(N, dtype=np.int32)
    tol = 1e-12 * float(np.ptp(nodes, axis=0).max())
    assert lib.dh_match(_dp(nd), M, _dp(xy), N, ctypes.c_double(tol), _ip(bnode)) == -1
    od = OI.DomainMesh(nodes, tris, BoundaryMesh(X, 1.0, 2, 1.0))
    assert np.array_equal(bnode, od.bnode)
    tr = np.ascontiguousarray(tris, dtype=np.int32)
    col = np.zeros(K, dtype=np.int32)
    nc = lib.dh_colour(M, K, _ip(tr), _ip(col))
    assert col.min() == 0 and col.max() == nc - 1
    for c in range(nc):
        used = tris[col == c].ravel()
        assert np.unique(used).size == used.size, (name, c)     # no node twice in one colour
    # greedy bound: at most 1 + the largest number of node-sharing neighbours
    share = [len(set(np.nonzero(np.isin(tris, t).any(1))[0]) - {k}) for k, t in enumerate(tris)]
    assert nc <= 1 + max(share)
    col2 = np.zeros(K, dtype=np.int32)
    assert lib.dh_colour(M, K, _ip(tr), _ip(col2)) == nc and np.array_equal(col, col2)


def test_matching_reports_the_first_unmatched_vertex(lib):
    X = W.unit_square(4)
    nodes, _ = W.square_triangulation(4)
    nd = np.ascontiguousarray(nodes * 1.01, dtype=np.float64)
    xy = np.ascontiguousarray(X, dtype=np.float64)
    bnode = np.zeros(X.shape[0], dtype=np.int32)
    # vertex 0 = (0, 0) still matches, vertex 1 = (0.25, 0) does not
    assert lib.dh_match(_dp(nd), nd.shape[0], _dp(xy), X.shape[0], ctypes.c_double(1e-12), _ip(bnode)) == 1
