"""Lag sharding on the GPU: compact lag-block assembly, lag-range products,
and the sharded GMRES.  Two ranks are emulated by two host threads, each with
its own context and stream on the one GPU; their all-reduce is done on the
host side (each thread synchronises its stream, a host barrier with a timeout,
the sum of the two partial results), so no kernel waits on another."""
import threading

import numpy as np
import pytest

import workloads as W
from oracle import assembly as OA
from oracle import rhs as OR
from oracle import solve as OS
from oracle.geometry import BoundaryMesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

X, T, NT, ALPHA = W.l_shape(48, seed=3), 1.0, 40, 0.5


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_05224_gb300 as P
    return P.Context(0)


def test_lag_blocks_and_range_products(ctx):
    """Compact blocks equal the full assembly's (bitwise); the range
    products of a partition sum to the full product (per element, FP64 and
    FP32, forward and transposed) against the oracle."""
    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import shard
    m = P.Mesh(ctx, X, T, NT, ALPHA)
    for op in "VKD":
        full = P.assemble(ctx, m, op)
        for r in range(3):
            S = shard.ShardedOperator(ctx, m, op, shard.lag_ranges(NT, 3, r, 8))
            for (a, b), off in zip(S.ranges, S.offsets()):
                assert torch.equal(S.blocks[off:off + b - a], full[a:b]), (op, r, a, b)
    rng = np.random.default_rng(6)
    for prec, tol in (("f64", 1e-13), ("f32", None)):
        dt = torch.float64 if prec == "f64" else torch.float32
        nt, nx, nb = 70, 64, 2
        A = torch.as_tensor(rng.standard_normal((nt, nx, nx))).to(dt).cuda()
        x = torch.as_tensor(rng.standard_normal((nb, nt, nx))).cuda()
        Ae = A.double().cpu().numpy()
        for tr in (False, True):
            y = torch.zeros_like(x)
            for r in range(3):
                for a, b in shard.lag_ranges(nt, 3, r, 16):
                    y += P.api.apply_lags(ctx, A[a:b], a, b, nt, x, transpose=tr)
            yh = y.cpu().numpy()
            for k in range(nb):
                ref = OS.toeplitz_apply(Ae, x[k].cpu().numpy(), transpose=tr)
                mag = OS.toeplitz_apply(np.abs(Ae), np.abs(x[k].cpu().numpy()), transpose=tr)
                t = tol if tol is not None else (nx + 2) * 2.0 ** -24 + 3e-16
                assert np.all(np.abs(yh[k] - ref) <= t * mag + 1e-300), (prec, tr)


def test_sharded_solve_one_rank_equals_plain_solve(ctx):
    """One rank holding every lag, identity reduction: the same iterations and
    the same w, bit for bit, as stbem_solve."""
    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import shard
    m = P.Mesh(ctx, X, T, NT, ALPHA)
    V, K, D = (P.assemble(ctx, m, o) for o in "VKD")
    L = P.lumped_mass(ctx, m)
    g, f = P.rhs(ctx, m, K, (1.5, 1.5))
    w, info = P.solve(ctx, V, f, D, L, tol=1e-10)
    Vs = shard.ShardedOperator(ctx, m, "V", [(0, NT)])
    Ds = shard.ShardedOperator(ctx, m, "D", [(0, NT)])
    w1, info1 = shard.solve_sharded(ctx, Vs, f, Ds, L, tol=1e-10, reducer=lambda t: None)
    assert info1["iterations"] == info["iterations"]
    assert torch.equal(w1, w)


def _host_allreduce(n_ranks, stream, slots, barrier, rank):
    def red(t):
        stream.synchronize()                 # this rank's partial product is complete
        slots[rank] = t.clone()
        barrier.wait()
        with torch.cuda.stream(stream):
            total = slots[0].clone()
            for k in range(1, n_ranks):
                total += slots[k]
            t.copy_(total)
        stream.synchronize()
        barrier.wait()                       # nobody overwrites a slot before all have read
    return red


def test_sharded_solve_two_ranks_against_oracle():
    """Two ranks (threads), lags dealt in chunks of 8 in snake order: the
    sharded right-hand side and preconditioned GMRES give the same w on both
    ranks, within 1e-8 of the oracle's block forward substitution with the
    oracle's V and f."""
    import paper_1811_05224_gb300 as P
    from paper_1811_05224_gb300 import shard
    n_ranks = 2
    barrier = threading.Barrier(n_ranks, timeout=120)
    slots = [None] * n_ranks
    out = [None] * n_ranks

    def run(rank):
        try:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                c = P.Context(0, stream)
                m = P.Mesh(c, X, T, NT, ALPHA)
                ranges = shard.lag_ranges(NT, n_ranks, rank, 8)
                Vs, Ks, Ds = (shard.ShardedOperator(c, m, o, ranges) for o in "VKD")
                L = P.lumped_mass(c, m)
                red = _host_allreduce(n_ranks, stream, slots, barrier, rank)
                g, f = shard.rhs_sharded(c, m, Ks, (1.5, 1.5), reducer=red)
                w, info = shard.solve_sharded(c, Vs, f, Ds, L, tol=1e-10, reducer=red)
                stream.synchronize()
                out[rank] = (ranges, f.cpu().numpy(), w.cpu().numpy(), info)
        except Exception as e:               # surfaced by the main thread
            barrier.abort()
            out[rank] = e

    threads = [threading.Thread(target=run, args=(r,)) for r in range(n_ranks)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    for r in range(n_ranks):
        assert not isinstance(out[r], Exception), out[r]
        assert out[r] is not None, r
    assert all(out[r][0] for r in range(n_ranks))          # both ranks hold lags
    assert np.array_equal(out[0][2], out[1][2])             # identical solutions
    assert out[0][3]["iterations"] == out[1][3]["iterations"]
    om = BoundaryMesh(X, T, NT, ALPHA)
    Vo = OA.assemble("V", om)
    f_ref = OR.f_vec(om, OA.assemble("K", om), OR.g_vec(om, (1.5, 1.5)))
    assert np.linalg.norm(out[0][1] - f_ref) <= 1e-12 * np.linalg.norm(f_ref)
    w_ref = OS.forward_substitution(Vo, f_ref)
    assert np.linalg.norm(out[0][2] - w_ref) <= 1e-8 * np.linalg.norm(w_ref)
