"""Parity at the full sizes of the named workloads, in the launch
configuration the library uses for them: lag ranges of the full operators
assembled on the GPU (stbem_assemble_lags into the full n_t x N_x x N_x
arrays), sampled entries of every pair class and lag regime checked one by one
against the oracle.

Bounds per entry (as for the small meshes): V within 1e-12 of max(|v|, 1e-6
max|V^(d)|) in FP64 and 1e-5 in FP32; K and D within
tol max(|a|, 1e-6 max|A^(d)|) + term_tol S, S the sum of the magnitudes of the
entry's quadrature terms from the oracle (tol, term_tol = 1e-12, 1e-14 in
FP64 and 1e-5, 2e-6 in FP32).  FP64 D entries are compared with the oracle's
exactly summed entries (math.fsum over all point terms): the GPU's own
rounding measured there is at most 19.5 eps S (square512), 11.7 (lshape1024)
and 9.3 (star256), eps = 2^-52, so 1e-14 S (45 eps) leaves a margin of 2.3 or
more.  The max over the lag block is taken from the
GPU block.  K entries that vanish identically (all trial segments collinear
with the test segment) are compared absolutely, |k| <= 1e-14 (FP64) or 1e-6
(FP32) of the block's largest entry.

The precision workload (L-shape, N_x = N_t = 1024, alpha = 0.5, FP32 operators
of 4.3 GB each) is also solved end to end in mixed precision and checked by its
FP64 residual, computed with the FP64 operator."""
import numpy as np
import pytest

import workloads as W
from oracle import assembly as OA
from oracle.geometry import BoundaryMesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_05224_gb300 as P
    return P.Context(0)


def _lag_ranges(nt):
    r = [(0, 2), (2, 4), (7, 10), (31, 34), (nt // 2, nt // 2 + 2), (nt - 2, nt)]
    return [(a, b) for a, b in r if 0 <= a < b <= nt]


def _k_zero(om, I, P, tol=1e-12):
    """K[i][p] whose trial segments (p - 1, p, minus i) are collinear with
    segment i: q = (x - y) . n_y vanishes identically there (a structural
    zero), and both sides return rounding noise."""
    cr = lambda a, b: a[0] * b[1] - a[1] * b[0]     # noqa: E731
    out = []
    for i, p in zip(I, P):
        js = [j for j in (p % om.N, (p - 1) % om.N) if j != i]
        out.append(all(abs(cr(om.t[i], om.t[j])) < tol and abs(cr(om.t[i], om.a[j] - om.a[i])) < tol * om.h[i]
                       for j in js))
    return np.array(out, dtype=bool)


def _pairs(N, rng):
    fixed = [(0, 0), (0, 1), (1, 0), (0, 2), (N // 4, N // 4 + 1), (N // 2, N // 2 - 2), (0, N - 1),
             (N - 1, 0), (3, N // 2), (N // 3, N // 3 + 3)]
    return fixed + [tuple(x) for x in rng.integers(0, N, size=(6, 2))]


@pytest.mark.parametrize("name", ["lshape1024", "square512", "star256"])
def test_sampled_entries_full_size(ctx, name):
    import paper_1811_05224_gb300 as P
    p = W.config(name)
    m = P.Mesh(ctx, p.vertices, p.T, p.n_t, p.alpha)
    om = BoundaryMesh(p.vertices, p.T, p.n_t, p.alpha)
    rng = np.random.default_rng(11)
    fn = {"V": OA.V_entries, "K": OA.K_entries, "D": OA.D_entries}
    for op in "VKD":
        for prec, tol, term_tol in (("f64", 1e-12, 1e-14), ("f32", 1e-5, 2e-6)):
            A = None
            for a, b in _lag_ranges(p.n_t):
                A = P.assemble_lags(ctx, m, op, a, b, prec, out=A)
            for a, b in _lag_ranges(p.n_t):
                for d in range(a, b):
                    pairs = _pairs(p.n_x, rng)
                    I = np.array([x for x, _ in pairs])
                    J = np.array([y for _, y in pairs])
                    got = A[d, torch.as_tensor(I), torch.as_tensor(J)].double().cpu().numpy()
                    exact = op == "D" and prec == "f64"
                    ref = fn[op](om, d, I, J, exact=True) if exact else fn[op](om, d, I, J)
                    scale = float(A[d].abs().max())
                    den = tol * np.maximum(np.abs(ref), 1e-6 * scale)
                    if op != "V":
                        den = den + term_tol * fn[op](om, d, I, J, magnitude=True)
                    err = np.abs(got - ref) / den
                    if op == "K":
                        z = _k_zero(om, I, J)
                        zero_tol = 1e-14 if prec == "f64" else 1e-6
                        assert np.all(np.abs(got[z]) <= zero_tol * scale), (name, prec, d)
                        err[z] = 0.0
                    assert err.max() <= 1.0, (name, op, prec, d, pairs[int(err.argmax())], err.max())
            del A
            torch.cuda.empty_cache()


def test_precision_workload_mixed_solve(ctx):
    """lshape1024: FP64 V and K (8.6 GB each), FP32 D (4.3 GB), FP32 V for the
    inner GMRES; mixed solve to 1e-8 checked by its FP64 residual."""
    import paper_1811_05224_gb300 as P
    p = W.config("lshape1024")
    m = P.Mesh(ctx, p.vertices, p.T, p.n_t, p.alpha)
    V = P.assemble(ctx, m, "V")
    K = P.assemble(ctx, m, "K")
    g, f = P.rhs(ctx, m, K, p.y_star)
    del K
    torch.cuda.empty_cache()
    D32 = P.assemble(ctx, m, "D", "f32")
    V32 = P.round_f32(ctx, V)
    Minv = P.mixed_mass_inverse(ctx, m)       # consistent mixed mass: bounded iterations on this mesh
    w, info = P.solve_mixed(ctx, V, V32, f, D32, Minv, tol=1e-8, inner_tol=1e-4, max_iter=400, restart=60)
    assert info["status"] == 0
    r = f - P.apply(ctx, V, w)
    assert float(r.norm() / f.norm()) <= 1e-8
    # the same solve with exact-slice outer residuals (one step tile per 128
    # steps, 1024 x 1024 lag blocks: the full-size case of that product)
    Vx = P.exact_slices(ctx, V, 7)
    wx, infox = P.solve_mixed(ctx, Vx, V32, f, D32, Minv, tol=1e-8, inner_tol=1e-4, max_iter=400, restart=60)
    assert infox["status"] == 0
    r = f - P.apply(ctx, V, wx)
    assert float(r.norm() / f.norm()) <= 1.01e-8
    assert float((wx - w).norm() / w.norm()) <= 1e-6
    # and with the inner GMRES on the tensor cores (three-slice V and D; the
    # D slices from the FP32 D: only the preconditioner)
    V3, D3 = P.bf16_split3(ctx, V), P.bf16_split3(ctx, D32.double())
    wt, infot = P.solve_mixed(ctx, Vx, V3, f, D3, Minv, tol=1e-8, inner_tol=1e-4, max_iter=400, restart=60)
    assert infot["status"] == 0
    r = f - P.apply(ctx, V, wt)
    assert float(r.norm() / f.norm()) <= 1.01e-8
    assert float((wt - w).norm() / w.norm()) <= 1e-6
