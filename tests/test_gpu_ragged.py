"""Ragged batches: problems of different N_x, N_t, T, alpha and shapes through
one persistent launch per step.

* assembly of V, K, D for every problem against the single-problem assembly
  (FP64: same rule, summation order may differ, 1e-13 of the lag block's
  largest entry; FP32: error against the FP64 blocks no worse than the
  single-problem FP32 path's);
* the ragged product against the oracle's Toeplitz product (FP64, within
  1e-13 of |A||x|), before and after autotuning;
* right-hand sides and lumped masses against the single-problem calls;
* the lockstep GMRES against the single-problem solves and, for one problem,
  the oracle's exact forward substitution.
"""
import numpy as np
import pytest

import workloads as W
from oracle import solve as OS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_05224_gb300 as P
    return P.Context(0)


def _problems():
    return [
        (W.unit_square(5), 1.0, 17, 1.0),       # N_x 20
        (W.l_shape(40, seed=3), 0.7, 40, 0.5),  # N_x 40, ragged lengths
        (W.unit_square(2), 1.0, 3, 2.0),        # N_x 8, three steps
        (W.star(8, 2, seed=5), 1.3, 33, 0.9),   # N_x 16
        (W.unit_square(3), 0.5, 1, 1.0),        # one step
    ]


@pytest.fixture(scope="module")
def batch(ctx):
    import paper_1811_05224_gb300 as P
    probs = _problems()
    R = P.Ragged(ctx, probs)
    meshes = [P.Mesh(ctx, v, T, nt, a) for v, T, nt, a in probs]
    return R, meshes, probs


@pytest.mark.parametrize("op", ["V", "K", "D"])
def test_ragged_assembly_matches_single(ctx, batch, op):
    import paper_1811_05224_gb300 as P
    R, meshes, _ = batch
    A = R.assemble(op)
    A32 = R.assemble(op, "f32")
    for p, m in enumerate(meshes):
        ref = P.assemble(ctx, m, op)
        got = R.view_op(A, p)
        scale = ref.abs().amax(dim=(1, 2), keepdim=True)
        assert bool(((got - ref).abs() <= 1e-13 * scale + 1e-300).all()), (op, p)
        # FP32: the ragged launch runs one lag per tile, the single-problem
        # assembly several lags per tile, so their FP32 sums round
        # differently; D and K entries are signed sums whose terms cancel, so
        # the check is accuracy against the FP64 blocks: no worse than the
        # single-problem FP32 path (itself parity-tested against the oracle)
        ref32 = P.assemble(ctx, m, op, "f32").double()
        got32 = R.view_op(A32, p).double()
        e_single = (ref32 - ref).abs().amax(dim=(1, 2), keepdim=True)
        e_ragged = (got32 - ref).abs().amax(dim=(1, 2), keepdim=True)
        assert bool((e_ragged <= 2.0 * e_single + 1e-7 * scale).all()), (op, p)


def test_ragged_apply_matches_oracle_and_tuner(ctx, batch):
    R, _, _ = batch
    V = R.assemble("V")
    x = torch.as_tensor(np.random.default_rng(9).standard_normal(R.vec_elems)).cuda()

    def check(y):
        for p in range(R.P):
            A = R.view_op(V, p).cpu().numpy()
            xp = R.view_vec(x, p).cpu().numpy()
            ref = OS.toeplitz_apply(A, xp)
            mag = OS.toeplitz_apply(np.abs(A), np.abs(xp))
            assert np.all(np.abs(R.view_vec(y, p).cpu().numpy() - ref) <= 1e-13 * mag + 1e-300), p

    check(R.apply(V, x))
    y = torch.empty_like(x)
    import paper_1811_05224_gb300 as P
    P.tune_cache_clear()
    best, report = R.tune(V, x, y)
    assert not best["from_cache"] and len(report) >= 1
    assert "tiles32=%d lpc=%d" % (best["tiles32"], best["lags_per_chunk"]) in report
    assert all(ms > 0 for ms in report.values())
    check(R.apply(V, x))
    # the same shapes again: the recorded choice, no timing
    best2, report2 = R.tune(V, x, y)
    assert best2["from_cache"] and report2 == {}
    assert (best2["tiles32"], best2["lags_per_chunk"]) == (best["tiles32"], best["lags_per_chunk"])
    check(R.apply(V, x))
    # FP32 operators: both tile families are candidates
    V32 = R.assemble("V", "f32")
    best3, report3 = R.tune(V32, x, y)
    assert {k.split()[0] for k in report3} == {"tiles32=0", "tiles32=1"}


def test_ragged_rhs_and_mass_match_single(ctx, batch):
    import paper_1811_05224_gb300 as P
    R, meshes, _ = batch
    K = R.assemble("K")
    ys = [(1.5, 1.5), (1.3, 1.4), (1.8, -0.2), (2.0, 0.4), (-0.7, 0.5)]
    g, f = R.rhs(K, ys)
    L = R.lumped_mass()
    for p, m in enumerate(meshes):
        Kp = P.assemble(ctx, m, "K")
        g1, f1 = P.rhs(ctx, m, Kp, ys[p])
        assert float((R.view_vec(g, p) - g1).abs().max()) <= 1e-15 * float(g1.abs().max())
        assert float((R.view_vec(f, p) - f1).abs().max()) <= 1e-13 * float(f1.abs().max())
        L1 = P.lumped_mass(ctx, m)
        assert torch.equal(R.view_mass(L, p), L1)


@pytest.mark.parametrize("precondition", [True, False])
def test_ragged_solve_matches_single_and_oracle(ctx, batch, precondition):
    import paper_1811_05224_gb300 as P
    R, meshes, _ = batch
    V, K, D = R.assemble("V"), R.assemble("K"), R.assemble("D")
    L = R.lumped_mass()
    ys = [(1.5, 1.5), (1.3, 1.4), (1.8, -0.2), (2.0, 0.4), (-0.7, 0.5)]
    _, f = R.rhs(K, ys)
    w, infos = R.solve(V, f, D if precondition else None, L if precondition else None, tol=1e-11, restart=30,
                       max_iter=800)
    assert all(i["status"] == 0 for i in infos), infos
    assert all(i["rel_residual"] <= 1e-11 for i in infos), infos
    for p, m in enumerate(meshes):
        Vp = R.view_op(V, p)
        fp = R.view_vec(f, p)
        w1, _ = P.solve(ctx, Vp, fp, R.view_op(D, p), R.view_mass(L, p), tol=1e-11)
        assert float((R.view_vec(w, p) - w1).norm() / w1.norm()) < 1e-8, p
        # true residual of the batch's solution
        r = fp - P.apply(ctx, Vp, R.view_vec(w, p))
        assert float(r.norm() / fp.norm()) <= 1.01e-11, p
    # one problem against the oracle's exact block forward substitution with the oracle's V
    from oracle import assembly as OA
    from oracle.geometry import BoundaryMesh
    Vn = OA.assemble("V", BoundaryMesh(*_problems()[1]))
    wref = OS.forward_substitution(Vn, R.view_vec(f, 1).cpu().numpy())
    assert float(np.linalg.norm(R.view_vec(w, 1).cpu().numpy() - wref) / np.linalg.norm(wref)) < 1e-8


def test_ragged_rejects_bad_arguments(ctx, batch):
    from paper_1811_05224_gb300 import capi
    R, _, _ = batch
    out = torch.empty(R.op_elems, dtype=torch.float64, device="cuda")
    code = ctx.lib.stbem_ragged_assemble(ctx.h, R.h, 7, capi.F64, out.data_ptr())
    assert code == capi.STBEM_ERR_ARG
    code = ctx.lib.stbem_ragged_assemble(ctx.h, R.h, capi.OP_V, 5, out.data_ptr())
    assert code == capi.STBEM_ERR_ARG


def test_ragged_solve_fp32_operators(ctx, batch):
    """FP32 operators (FP64 singular pairs), FP64 vectors: the product sums
    FP32 terms over one lag block's columns and flushes into FP64 per lag, so
    the residual reaches 1e-7; the batch's solutions agree with the
    single-problem FP32 solves to the solver tolerance times kappa (~100)."""
    import paper_1811_05224_gb300 as P
    R, meshes, _ = batch
    V, K, D = R.assemble("V", "f32"), R.assemble("K"), R.assemble("D", "f32")
    L = R.lumped_mass()
    ys = [(1.5, 1.5), (1.3, 1.4), (1.8, -0.2), (2.0, 0.4), (-0.7, 0.5)]
    _, f = R.rhs(K, ys)
    w, infos = R.solve(V, f, D, L, tol=1e-7, restart=30, max_iter=400)
    assert all(i["status"] == 0 and i["rel_residual"] <= 1e-7 for i in infos), infos
    for p, m in enumerate(meshes):
        w1, _ = P.solve(ctx, R.view_op(V, p), R.view_vec(f, p), R.view_op(D, p), R.view_mass(L, p), tol=1e-7)
        assert float((R.view_vec(w, p) - w1).norm() / w1.norm()) < 2e-5, p


def test_ragged_mixed_solve_reaches_fp64_accuracy(ctx, batch):
    """FP32 lockstep solves inside FP64 refinement (residuals with the FP64
    V): every problem's FP64 residual <= 1e-10 and w within 1e-8 of the
    oracle's block forward substitution (oracle V, same f) for the L-shape,
    and within 1e-8 of the single-problem FP64 solves for the others."""
    import paper_1811_05224_gb300 as P
    from oracle import assembly as OA
    from oracle.geometry import BoundaryMesh
    R, meshes, probs = batch
    V64 = R.assemble("V")
    V32, D32 = R.assemble("V", "f32"), R.assemble("D", "f32")
    K = R.assemble("K")
    L = R.lumped_mass()
    ys = [(1.5, 1.5), (1.3, 1.4), (1.8, -0.2), (2.0, 0.4), (-0.7, 0.5)]
    _, f = R.rhs(K, ys)
    w, infos = R.solve_mixed(V64, V32, f, D32, L, tol=1e-10, inner_tol=1e-3, restart=30, max_iter=800)
    assert all(i["status"] == 0 and i["rel_residual"] <= 1e-10 for i in infos), infos
    D64 = R.assemble("D")
    for p, m in enumerate(meshes):
        fp = R.view_vec(f, p)
        r = fp - P.apply(ctx, R.view_op(V64, p), R.view_vec(w, p))
        assert float(r.norm() / fp.norm()) <= 1.01e-10, p
        w1, _ = P.solve(ctx, R.view_op(V64, p), fp, R.view_op(D64, p), R.view_mass(L, p), tol=1e-12)
        assert float((R.view_vec(w, p) - w1).norm() / w1.norm()) < 1e-8, p
    Vo = OA.assemble("V", BoundaryMesh(*probs[1]))
    wref = OS.forward_substitution(Vo, R.view_vec(f, 1).cpu().numpy())
    assert float(np.linalg.norm(R.view_vec(w, 1).cpu().numpy() - wref) / np.linalg.norm(wref)) < 1e-8
