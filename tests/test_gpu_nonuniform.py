"""Non-uniform time grids on the GPU (NEXT-4; Section 1 allows any
decomposition of (0, T)) against the oracle's oracle/nonuniform.py: packed
block assembly of V, K and D on graded grids t_j = T (j / N_t)^q, the
reduction to the Toeplitz lag blocks on a uniform grid, the block lower
triangular product, the right-hand side and the preconditioned solve.

Bounds as for the uniform path: V within 1e-12 of max(|a|, 1e-6 max|A[p]|)
per block; K with its structural zeros compared absolutely; D against the
oracle's exactly summed entries within 1e-12 max(|a|, floor) + 1e-14 S (S the
sum of the magnitudes of the entry's terms)."""
import numpy as np
import pytest

import workloads as W
from oracle import assembly as OA
from oracle import nonuniform as ON
from oracle import solve as OS
from oracle.geometry import BoundaryMesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "square8_q1.5": (W.unit_square(2), 1.0, 6, 1.0, 1.5),
    "lshape16_q1.5": (W.l_shape(16, seed=3), 0.8, 5, 0.5, 1.5),
    "star16_q2": (W.star(8, 2, seed=5), 1.0, 5, 1.3, 2.0),
}


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_05224_gb300 as P
    return P.Context(0)


def _grid(T, nt, q):
    return T * (np.arange(nt + 1) / nt) ** q


def _blocks(A_packed, nt):
    """packed -> (m, n, N, N) with zeros above the block diagonal"""
    a = A_packed.cpu().numpy()
    N = a.shape[1]
    out = np.zeros((nt, nt, N, N))
    for m in range(nt):
        for n in range(m + 1):
            out[m, n] = a[m * (m + 1) // 2 + n]
    return out


def _oracle_D(om, t, exact=False, magnitude=False):
    nt = t.size - 1
    N = om.N
    I, J = np.triu_indices(N)
    out = np.zeros((nt, nt, N, N))
    for m in range(nt):
        for n in range(m + 1):
            tf = (lambda kind, c, m=m, n=n: ON.time_integral(kind, c, t, m, n, om.alpha))
            v = OA.D_entries(om, m - n, I, J, tfun=tf, exact=exact, magnitude=magnitude)
            out[m, n, I, J] = v
            out[m, n, J, I] = v
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_nu_assembly_matches_oracle(ctx, name):
    import paper_1811_05224_gb300 as P
    from tests.parity import k_structural_zeros
    X, T, nt, al, q = CASES[name]
    t = _grid(T, nt, q)
    m = P.GradedMesh(ctx, X, t, al)
    om = BoundaryMesh(X, T, nt, al)
    zeros = k_structural_zeros(om)
    for op in "VKD":
        got = _blocks(P.nu_assemble(ctx, m, op), nt)
        if op == "D":
            ref, S = _oracle_D(om, t, exact=True), _oracle_D(om, t, magnitude=True)
        else:
            ref, S = ON.assemble(op, om, t), None
        for mm in range(nt):
            for n in range(mm + 1):
                a, b = got[mm, n], ref[mm, n]
                scale = np.abs(b).max()
                den = 1e-12 * np.maximum(np.abs(b), 1e-6 * scale)
                if op == "D":
                    den = den + 1e-14 * S[mm, n]
                err = np.abs(a - b) / np.where(den > 0, den, 1.0)
                if op == "K":
                    assert np.abs(a[zeros]).max(initial=0.0) <= 1e-14 * scale
                    err[zeros] = 0.0
                assert err.max() <= 1.0, (name, op, mm, n, err.max())


def test_nu_uniform_grid_equals_toeplitz_blocks(ctx):
    """On a uniform grid every block equals the Toeplitz lag block (two code
    paths: per-block time tables against per-lag ones), to rounding."""
    import paper_1811_05224_gb300 as P
    X, T, nt, al = W.l_shape(16, seed=3), 1.0, 12, 0.7
    m = P.Mesh(ctx, X, T, nt, al)
    for op in "VKD":
        U = P.assemble(ctx, m, op).cpu().numpy()
        G = _blocks(P.nu_assemble(ctx, m, op), nt)
        for mm in range(nt):
            for n in range(mm + 1):
                b = U[mm - n]
                scale = np.abs(b).max()
                assert np.abs(G[mm, n] - b).max() <= 1e-12 * scale, (op, mm, n)


def test_nu_apply_matches_oracle(ctx):
    import paper_1811_05224_gb300 as P
    rng = np.random.default_rng(9)
    for nt, nx in [(7, 33), (1, 5), (20, 64)]:
        A = torch.as_tensor(rng.standard_normal((nt * (nt + 1) // 2, nx, nx))).cuda()
        x = torch.as_tensor(rng.standard_normal((nt, nx))).cuda()
        y = P.nu_apply(ctx, A, nt, x).cpu().numpy()
        Ab = _blocks(A, nt)
        ref = ON.block_apply(Ab, x.cpu().numpy())
        mag = ON.block_apply(np.abs(Ab), np.abs(x.cpu().numpy()))
        assert np.all(np.abs(y - ref) <= 1e-13 * mag + 1e-300), (nt, nx)


@pytest.mark.parametrize("name", ["square8_q1.5", "lshape16_q1.5"])
def test_nu_rhs_and_preconditioned_solve_against_oracle(ctx, name):
    """g, f = 1/2 M_h g + K_h g and the GMRES solution (Section 2
    preconditioner with the lumped mass of each step) against the oracle's
    g_vec, f_vec and block forward substitution on the same graded grid."""
    import paper_1811_05224_gb300 as P
    X, T, nt, al, q = CASES[name]
    t = _grid(T, nt, q)
    m = P.GradedMesh(ctx, X, t, al)
    om = BoundaryMesh(X, T, nt, al)
    ys = (1.5, 1.5)
    V, K, D = (P.nu_assemble(ctx, m, o) for o in "VKD")
    g, f = P.nu_rhs(ctx, m, K, ys)
    g_ref = ON.g_vec(om, t, ys)
    f_ref = ON.f_vec(om, t, ON.assemble("K", om, t), g_ref)
    assert np.abs(g.cpu().numpy() - g_ref).max() <= 1e-13 * np.abs(g_ref).max()
    assert np.abs(f.cpu().numpy() - f_ref).max() <= 1e-12 * np.abs(f_ref).max()
    L = P.nu_lumped_mass(ctx, m).cpu().numpy()
    h = np.diff(t)
    hm, h0, hp = np.roll(om.h, 1), om.h, np.roll(om.h, -1)
    assert np.allclose(L, h[:, None] * (hm + 2 * h0 + hp)[None, :] / 4, rtol=1e-15, atol=0)
    w_ref = ON.forward_substitution(ON.assemble("V", om, t), f.cpu().numpy())
    for prec in (True, False):
        w, info = P.nu_solve(ctx, V, f, D if prec else None, P.nu_lumped_mass(ctx, m) if prec else None, tol=1e-11)
        assert info["status"] == 0 and info["rel_residual"] <= 1e-11
        assert np.linalg.norm(w.cpu().numpy() - w_ref) <= 1e-8 * np.linalg.norm(w_ref), (name, prec)


def test_nu_rejects_graded_mesh_in_uniform_calls(ctx):
    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import capi
    m = P.GradedMesh(ctx, W.unit_square(2), _grid(1.0, 4, 1.5), 1.0)
    with pytest.raises(capi.StbemError) as e:
        P.assemble(ctx, m, "V")
    assert e.value.code == capi.STBEM_ERR_ARG
    with pytest.raises(capi.StbemError):
        P.GradedMesh(ctx, W.unit_square(2), np.array([0.0, 0.5, 0.4, 1.0]), 1.0)
