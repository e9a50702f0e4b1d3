"""Lag sharding of one problem across ranks (stbem_lag_shard and friends).

Section 3 distributes the blocks of the block-lower-triangular matrices over
processes; on a uniform time grid the blocks of one lag coincide, so a rank
holds the blocks of some lags (chunks dealt in snake order), computes its part
of every product and one all-reduce of the n_t x n_x result completes it.
Vectors and the GMRES recurrences are replicated.  Argument marshalling only:
the products and the solver run in the library; the all-reduce is the
caller's (torch.distributed by default: NCCL on GPUs, gloo on CPUs).
"""
import ctypes

import torch

from . import capi
from .api import Context, Mesh, _ptr, OPS, PRECS, apply_lags


def lag_ranges(n_t: int, n_ranks: int, rank: int, chunk: int = 16):
    """[(begin, end), ...] of the lags held by `rank` (host only)."""
    lib = capi.load()
    cap = (n_t + chunk - 1) // chunk + 1
    buf = (ctypes.c_int * (2 * cap))()
    n = ctypes.c_int()
    code = lib.stbem_lag_shard(n_t, n_ranks, rank, chunk, cap, buf, ctypes.byref(n))
    if code != capi.STBEM_OK:
        raise capi.StbemError(code, "stbem_lag_shard(%d, %d, %d, %d)" % (n_t, n_ranks, rank, chunk))
    return [(buf[2 * k], buf[2 * k + 1]) for k in range(n.value)]


def _ranges_array(ranges):
    arr = (ctypes.c_int * max(1, 2 * len(ranges)))()
    for k, (a, b) in enumerate(ranges):
        arr[2 * k], arr[2 * k + 1] = a, b
    return arr


def default_reducer(group=None):
    """In-place sum over the ranks of `group` (torch.distributed.all_reduce)."""
    import torch.distributed as dist

    def red(t):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return red


def make_allreduce_callback(buffer, reducer):
    """The C callback of stbem_solve_sharded: maps the device pointer it
    receives (inside `buffer`, the solve's workspace) to a float64 view and
    applies `reducer` to it in place.  Returns the ctypes function object,
    which the caller keeps alive for the duration of the solve."""
    base = buffer.data_ptr()
    nbytes = buffer.numel() * buffer.element_size()
    flat = buffer.view(torch.uint8).reshape(-1)

    def cb(ptr, n, _user):
        try:
            off = int(ptr) - base
            if off < 0 or off % 8 or off + 8 * int(n) > nbytes:
                return 1
            reducer(flat[off:off + 8 * int(n)].view(torch.float64))
            return 0
        except Exception:       # reported to the solver as STBEM_ERR_REDUCE
            return 2
    return capi.ALLREDUCE_FN(cb)


class ShardedOperator:
    """This rank's lag blocks of one operator (compact: the ranges' blocks in
    order), with the full problem's sizes."""

    def __init__(self, ctx: Context, mesh: Mesh, op: str, ranges, prec: str = "f64"):
        self.ctx, self.n_t, self.n_x, self.prec, self.op = ctx, mesh.n_t, mesh.n_x, prec, op
        self.ranges = list(ranges)
        n_lags = sum(b - a for a, b in self.ranges)
        dt = torch.float64 if prec == "f64" else torch.float32
        self.blocks = torch.empty((max(1, n_lags), mesh.n_x, mesh.n_x), dtype=dt, device=ctx.device)
        self.assemble(mesh)

    def assemble(self, mesh: Mesh):
        """(Re)assemble this rank's blocks on `mesh` (same sizes) in place."""
        ctx = self.ctx
        k = 0
        for a, b in self.ranges:
            ctx.check(ctx.lib.stbem_assemble_lag_blocks(ctx.h, mesh.h, OPS[self.op], PRECS[self.prec], a, b,
                                                        _ptr(self.blocks[k:k + (b - a)])))
            k += b - a
        return self

    def offsets(self):
        out, k = [], 0
        for a, b in self.ranges:
            out.append(k)
            k += b - a
        return out

    def apply_local(self, x, transpose: bool = False, out=None):
        """This rank's partial product (zero when it holds no lags)."""
        ctx = self.ctx
        xb = x if x.dim() == 3 else x.unsqueeze(0)
        y = torch.zeros_like(xb) if out is None else out.view_as(xb)
        if not self.ranges:
            y.zero_()
            return y if x.dim() == 3 else y[0]
        longest = max(b - a for a, b in self.ranges)
        nb = ctypes.c_size_t()
        ctx.check(ctx.lib.stbem_apply_lags_workspace_bytes(self.n_t, self.n_x, longest, xb.shape[0],
                                                           ctypes.byref(nb)))
        work = torch.empty(nb.value, dtype=torch.uint8, device=ctx.device)
        for k, ((a, b), off) in enumerate(zip(self.ranges, self.offsets())):
            apply_lags(ctx, self.blocks[off:off + (b - a)], a, b, self.n_t, xb, transpose=transpose, out=y,
                       accumulate=k > 0, work=work)
        return y if x.dim() == 3 else y[0]

    def apply(self, x, transpose: bool = False, reducer=None):
        """The full product: partial product, then the all-reduce."""
        y = self.apply_local(x, transpose)
        (reducer or default_reducer())(y)
        return y


def rhs_sharded(ctx: Context, mesh: Mesh, K: ShardedOperator, y_star, reducer=None):
    """(g, f) of eq. (4) for g = U*(x - y*, t): f = 1/2 M_h g + K_h g with the
    K product sharded (partial product, all-reduce), the mass term added
    once after the reduction."""
    ys = (ctypes.c_double * 2)(float(y_star[0]), float(y_star[1]))
    g = ctx.empty((mesh.n_t, mesh.n_x))
    ctx.check(ctx.lib.stbem_rhs_g_batched(ctx.h, mesh.h, 1, ys, _ptr(g)))
    f = K.apply(g, reducer=reducer)
    ctx.check(ctx.lib.stbem_half_mass_add(ctx.h, mesh.h, 1, _ptr(g), _ptr(f)))
    return g, f


def solve_sharded(ctx: Context, V: ShardedOperator, f, D: ShardedOperator = None, L=None, tol: float = 1e-8,
                  max_iter: int = 500, restart: int = 200, reducer=None, out=None, raise_on_fail: bool = True):
    """Right-preconditioned GMRES (stbem_solve_sharded) whose V and D
    products are this rank's lag ranges followed by `reducer` (default: a
    torch.distributed all-reduce); every rank calls it with the same f."""
    n_t, n_x = f.shape
    if D is not None and D.ranges != V.ranges:
        raise ValueError("V and D must hold the same lag ranges")
    mode = 0 if D is None else (2 if L is not None and L.dim() == 2 else 1)
    opts = capi.SolveOpts(tol, max_iter, restart, mode)
    info = capi.SolveInfo()
    if out is None:
        out = ctx.empty((n_t, n_x))
    nb = ctypes.c_size_t()
    ctx.check(ctx.lib.stbem_solve_sharded_workspace_bytes(n_t, n_x, restart, ctypes.byref(nb)))
    work = torch.empty(nb.value, dtype=torch.uint8, device=ctx.device)
    cb = make_allreduce_callback(work, reducer or default_reducer())
    ranges = _ranges_array(V.ranges)
    p = PRECS[V.prec]
    code = ctx.lib.stbem_solve_sharded(ctx.h, n_t, n_x, p, _ptr(V.blocks), _ptr(D.blocks) if D is not None else None,
                                       len(V.ranges), ranges, cb, None, _ptr(L), _ptr(f), _ptr(out),
                                       ctypes.byref(opts), ctypes.byref(info), _ptr(work), work.numel())
    res = {"iterations": info.iterations, "status": info.status, "rel_residual": info.rel_residual}
    if code != capi.STBEM_OK and raise_on_fail:
        ctx.check(code)
    return out, res
