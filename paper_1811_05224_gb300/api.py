"""Torch-facing wrappers of the C ABI (argument marshalling only).

PyTorch provides device memory (outputs and workspaces are torch tensors) and
the CUDA stream; every computation runs in libstbem's kernels.  Nothing here
falls back to the CPU: without a CUDA device or the built library the calls
raise.
"""
import ctypes

import numpy as np
import torch

from . import capi

OPS = {"V": capi.OP_V, "K": capi.OP_K, "D": capi.OP_D}
PRECS = {"f64": capi.F64, "f32": capi.F32}
DTYPES = {capi.F64: torch.float64, capi.F32: torch.float32}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Context:
    """A library context on one CUDA device, bound to a CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("stbem needs a CUDA device (no CPU fallback)")
        self.lib = capi.load()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        code = self.lib.stbem_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream))
        if code != capi.STBEM_OK:
            raise capi.StbemError(code, "stbem_create failed on device %d" % device)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.stbem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, code):
        return capi.check(self.h, code)

    def empty(self, shape, dtype=torch.float64):
        return torch.empty(shape, dtype=dtype, device=self.device)


class Mesh:
    """Polygon boundary mesh x uniform time grid (vertices counter-clockwise)."""

    def __init__(self, ctx: Context, vertices, T: float, n_t: int, alpha: float):
        xy = np.ascontiguousarray(np.asarray(vertices, dtype=np.float64).reshape(-1))
        self.ctx = ctx
        self.n_x = xy.size // 2
        self.n_t = int(n_t)
        self.T = float(T)
        self.alpha = float(alpha)
        self.vertices = xy.reshape(-1, 2).copy()
        h = ctypes.c_void_p()
        ctx.check(ctx.lib.stbem_mesh_create(ctx.h, xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            self.n_x, self.T, self.n_t, self.alpha, ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.stbem_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GradedMesh(Mesh):
    """Polygon boundary mesh x the non-uniform time grid t (n_t + 1 nodes,
    t_0 = 0, increasing): operators are the packed blocks of the nu_* calls."""

    def __init__(self, ctx: Context, vertices, t, alpha: float):
        xy = np.ascontiguousarray(np.asarray(vertices, dtype=np.float64).reshape(-1))
        tn = np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(-1))
        self.ctx = ctx
        self.n_x = xy.size // 2
        self.n_t = tn.size - 1
        self.T = float(tn[-1])
        self.alpha = float(alpha)
        self.vertices = xy.reshape(-1, 2).copy()
        self.t = tn.copy()
        h = ctypes.c_void_p()
        P = ctypes.POINTER(ctypes.c_double)
        ctx.check(ctx.lib.stbem_mesh_create_graded(ctx.h, xy.ctypes.data_as(P), self.n_x, tn.ctypes.data_as(P),
                                                   self.n_t, self.alpha, ctypes.byref(h)))
        self.h = h


def nu_assemble(ctx: Context, mesh: Mesh, op: str, out=None):
    """Packed blocks A[p] (p = m (m + 1) / 2 + n, n <= m) of op on mesh's time grid."""
    nt, nx = mesh.n_t, mesh.n_x
    if out is None:
        out = ctx.empty((nt * (nt + 1) // 2, nx, nx))
    ctx.check(ctx.lib.stbem_nu_assemble(ctx.h, mesh.h, OPS[op], _ptr(out)))
    return out


def nu_apply(ctx: Context, A, n_t: int, x, out=None):
    """y[m] = sum_{n <= m} A[p(m, n)] x[n] (x: n_t x n_x)."""
    if out is None:
        out = torch.empty_like(x)
    ctx.check(ctx.lib.stbem_nu_apply(ctx.h, n_t, x.shape[-1], _ptr(A), _ptr(x), _ptr(out)))
    return out


def nu_rhs(ctx: Context, mesh: Mesh, K, y_star):
    """(g, f) of eq. (4) on mesh's time grid for g = U*(x - y*, t)."""
    g = ctx.empty((mesh.n_t, mesh.n_x))
    f = ctx.empty((mesh.n_t, mesh.n_x))
    ctx.check(ctx.lib.stbem_nu_rhs(ctx.h, mesh.h, _ptr(K), float(y_star[0]), float(y_star[1]), _ptr(g), _ptr(f)))
    return g, f


def nu_lumped_mass(ctx: Context, mesh: Mesh):
    """L[m][l] = h_m (h_{l-1} + 2 h_l + h_{l+1}) / 4."""
    L = ctx.empty((mesh.n_t, mesh.n_x))
    ctx.check(ctx.lib.stbem_nu_lumped_mass(ctx.h, mesh.h, _ptr(L)))
    return L


def nu_solve(ctx: Context, V, f, D=None, L=None, tol: float = 1e-8, max_iter: int = 500, restart: int = 200,
             work=None, out=None, raise_on_fail: bool = True):
    """GMRES for the packed V (and preconditioner D, L) on a non-uniform grid."""
    n_t, n_x = f.shape
    opts = capi.SolveOpts(tol, max_iter, restart, int(D is not None))
    info = capi.SolveInfo()
    if out is None:
        out = ctx.empty((n_t, n_x))
    if work is None:
        work = solve_workspace(ctx, n_t, n_x, restart)
    code = ctx.lib.stbem_nu_solve(ctx.h, n_t, n_x, _ptr(V), _ptr(D), _ptr(L), _ptr(f), _ptr(out),
                                  ctypes.byref(opts), ctypes.byref(info), _ptr(work), work.numel())
    res = {"iterations": info.iterations, "status": info.status, "rel_residual": info.rel_residual}
    if code != capi.STBEM_OK and raise_on_fail:
        ctx.check(code)
    return out, res


class Domain:
    """Triangulation Omega_h of the domain bounded by ``mesh`` (nodes (M, 2),
    triangles (K, 3) counter-clockwise, boundary vertices among the nodes)."""

    def __init__(self, ctx: Context, mesh: Mesh, nodes, tris):
        nd = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1))
        tr = np.ascontiguousarray(np.asarray(tris, dtype=np.int32).reshape(-1))
        self.ctx, self.mesh = ctx, mesh
        self.n_nodes = nd.size // 2
        self.n_tris = tr.size // 3
        h = ctypes.c_void_p()
        ctx.check(ctx.lib.stbem_domain_create(ctx.h, mesh.h, nd.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                              self.n_nodes, tr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                              self.n_tris, ctypes.byref(h)))
        self.h = h

    def info(self):
        """(n_nodes, n_tris, n_colors, bnode) with bnode[p] the node of vertex p."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        bn = np.zeros(self.mesh.n_x, dtype=np.int32)
        self.ctx.check(self.ctx.lib.stbem_domain_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                                      bn.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return a.value, b.value, c.value, bn

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.stbem_domain_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def m0_assemble(ctx: Context, dom: Domain, out=None):
    """M_h^0 as M0[m][i][j] (n_t x n_x x n_nodes, FP64)."""
    if out is None:
        out = ctx.empty((dom.mesh.n_t, dom.mesh.n_x, dom.n_nodes))
    ctx.check(ctx.lib.stbem_m0_assemble(ctx.h, dom.h, _ptr(out)))
    return out


def m0_workspace(ctx: Context, dom: Domain):
    nb = ctypes.c_size_t()
    ctx.check(ctx.lib.stbem_m0_apply_workspace_bytes(dom.h, ctypes.byref(nb)))
    return torch.empty(max(nb.value, 8), dtype=torch.uint8, device=ctx.device)


def m0_apply(ctx: Context, dom: Domain, u0, scale: float = 1.0, out=None, work=None):
    """out += scale * M_h^0 u0, matrix-free (u0: [n_rhs,] n_nodes; out: [n_rhs,]
    n_t x n_x, zeros when not given)."""
    ub = u0 if u0.dim() == 2 else u0.unsqueeze(0)
    n_rhs = ub.shape[0]
    if out is None:
        out = torch.zeros((n_rhs, dom.mesh.n_t, dom.mesh.n_x), dtype=torch.float64, device=ctx.device)
        ret = out if u0.dim() == 2 else out[0]
    else:
        ret = out
    if work is None:
        work = m0_workspace(ctx, dom)
    ctx.check(ctx.lib.stbem_m0_apply(ctx.h, dom.h, n_rhs, _ptr(ub), float(scale), _ptr(out), _ptr(work),
                                     work.numel()))
    return ret


def planewave_data(ctx: Context, dom: Domain, theta: float = np.pi / 8):
    """(g, u0) of the Section 4 example u = exp(-t/alpha) sin(x . d)."""
    g = ctx.empty((dom.mesh.n_t, dom.mesh.n_x))
    u0 = ctx.empty((dom.n_nodes,))
    ctx.check(ctx.lib.stbem_planewave_data(ctx.h, dom.h, float(theta), _ptr(g), _ptr(u0)))
    return g, u0


def evaluate(ctx: Context, mesh: Mesh, points, times, w, g, dom: Domain = None, u0=None):
    """u_h at interior points (P x 2) and times (P,) by the representation
    formula, eq. (2), from w (n_t x n_x), g (n_t x n_x) and, with a domain,
    the nodal initial datum u0.  points and times may be host arrays."""
    pts = torch.as_tensor(np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 2)) if not
                          torch.is_tensor(points) else points, dtype=torch.float64).to(ctx.device).contiguous()
    ts = torch.as_tensor(np.ascontiguousarray(np.asarray(times, dtype=np.float64).reshape(-1)) if not
                         torch.is_tensor(times) else times, dtype=torch.float64).to(ctx.device).contiguous()
    out = ctx.empty((ts.numel(),))
    ctx.check(ctx.lib.stbem_evaluate(ctx.h, mesh.h, dom.h if dom is not None else None, ts.numel(), _ptr(pts),
                                     _ptr(ts), _ptr(w), _ptr(g), _ptr(u0), _ptr(out)))
    return out


def rhs_initial(ctx: Context, dom: Domain, K, g, u0, work=None):
    """f = 1/2 M_h g + K_h g - M_h^0 u0 (eq. (4)), M_h^0 u0 matrix-free."""
    mesh = dom.mesh
    f = apply(ctx, K, g)
    ctx.check(ctx.lib.stbem_half_mass_add(ctx.h, mesh.h, 1, _ptr(g), _ptr(f)))
    m0_apply(ctx, dom, u0, -1.0, out=f, work=work)
    return f


def assemble(ctx: Context, mesh: Mesh, op: str, prec: str = "f64", out=None):
    """Lag blocks A[d][i][j] of op in {'V','K','D'} (n_t x n_x x n_x)."""
    p = PRECS[prec]
    if out is None:
        out = ctx.empty((mesh.n_t, mesh.n_x, mesh.n_x), DTYPES[p])
    ctx.check(ctx.lib.stbem_assemble(ctx.h, mesh.h, OPS[op], p, _ptr(out)))
    return out


def assemble_ops(ctx: Context, mesh: Mesh, prec="f64", ops: str = "VKD", out=None):
    """The lag blocks of each operator in ops, assembled concurrently on the
    context's stream and two side streams; returns {op: array}.  prec is one
    precision for all, or a dict {op: precision}; out may map an operator to a
    preallocated array."""
    precs = {op: PRECS[prec[op] if isinstance(prec, dict) else prec] for op in "VKD" if op in ops}
    out = dict(out or {})
    for op in ops:
        if op not in out:
            out[op] = ctx.empty((mesh.n_t, mesh.n_x, mesh.n_x), DTYPES[precs[op]])
        elif out[op].dtype != DTYPES[precs[op]] or tuple(out[op].shape) != (mesh.n_t, mesh.n_x, mesh.n_x) \
                or not out[op].is_contiguous():
            raise ValueError("assemble_ops: out[%r] must be a contiguous %s array of shape %s"
                             % (op, DTYPES[precs[op]], (mesh.n_t, mesh.n_x, mesh.n_x)))
    ptrs = [_ptr(out[op]) if op in ops else None for op in "VKD"]
    pv = [precs.get(op, capi.F64) for op in "VKD"]
    ctx.check(ctx.lib.stbem_assemble_ops(ctx.h, mesh.h, *pv, *ptrs))
    return {op: out[op] for op in ops}


def assemble_lags(ctx: Context, mesh: Mesh, op: str, lag_begin: int, lag_end: int, prec: str = "f64", out=None):
    """Write only the lag blocks [lag_begin, lag_end) of op into out."""
    p = PRECS[prec]
    if out is None:
        out = ctx.empty((mesh.n_t, mesh.n_x, mesh.n_x), DTYPES[p])
    ctx.check(ctx.lib.stbem_assemble_lags(ctx.h, mesh.h, OPS[op], p, lag_begin, lag_end, _ptr(out)))
    return out


def apply_workspace(ctx: Context, n_t: int, n_x: int, n_rhs: int = 1, prec: str = "f64"):
    nb = ctypes.c_size_t()
    ctx.check(ctx.lib.stbem_apply_workspace_bytes(n_t, n_x, n_rhs, PRECS[prec], ctypes.byref(nb)))
    return torch.empty(max(nb.value, 8), dtype=torch.uint8, device=ctx.device)


def apply(ctx: Context, A, x, transpose: bool = False, work=None, out=None):
    """Block-Toeplitz product with the lag blocks A (x: [n_rhs,] n_t x n_x, FP64)."""
    prec = capi.F64 if A.dtype == torch.float64 else capi.F32
    n_t, n_x = A.shape[0], A.shape[1]
    xb = x if x.dim() == 3 else x.unsqueeze(0)
    n_rhs = xb.shape[0]
    if out is None:
        out = torch.empty_like(xb)
    if work is None:
        work = apply_workspace(ctx, n_t, n_x, n_rhs, "f64" if prec == capi.F64 else "f32")
    ctx.check(ctx.lib.stbem_apply(ctx.h, prec, int(transpose), n_t, n_x, _ptr(A), n_rhs, _ptr(xb),
                                  _ptr(out), _ptr(work), work.numel()))
    return out if x.dim() == 3 else out[0]


def apply_lags(ctx: Context, A_blocks, lag_begin: int, lag_end: int, n_t: int, x, transpose: bool = False,
               out=None, accumulate: bool = False, work=None):
    """Block-Toeplitz product over the lags [lag_begin, lag_end) only, with
    A_blocks holding those blocks (block d at A_blocks[d - lag_begin])."""
    prec = capi.F64 if A_blocks.dtype == torch.float64 else capi.F32
    n_x = A_blocks.shape[1]
    xb = x if x.dim() == 3 else x.unsqueeze(0)
    n_rhs = xb.shape[0]
    if out is None:
        out = torch.empty_like(xb)
    if work is None:
        nb = ctypes.c_size_t()
        ctx.check(ctx.lib.stbem_apply_lags_workspace_bytes(n_t, n_x, lag_end - lag_begin, n_rhs, ctypes.byref(nb)))
        work = torch.empty(nb.value, dtype=torch.uint8, device=ctx.device)
    ctx.check(ctx.lib.stbem_apply_lags(ctx.h, prec, int(transpose), n_t, n_x, lag_begin, lag_end, _ptr(A_blocks),
                                       n_rhs, _ptr(xb), _ptr(out), int(accumulate), _ptr(work), work.numel()))
    return out if x.dim() == 3 else out[0]


def rhs(ctx: Context, mesh: Mesh, K, y_star, work=None):
    """(g, f): vertex time averages of g = U*(x - y*, t) and f = 1/2 M_h g + K_h g."""
    g = ctx.empty((mesh.n_t, mesh.n_x))
    f = ctx.empty((mesh.n_t, mesh.n_x))
    if work is None:
        work = apply_workspace(ctx, mesh.n_t, mesh.n_x, 1)
    ctx.check(ctx.lib.stbem_rhs(ctx.h, mesh.h, _ptr(K), float(y_star[0]), float(y_star[1]), _ptr(g),
                                _ptr(f), _ptr(work), work.numel()))
    return g, f


def mixed_mass_inverse(ctx: Context, mesh: Mesh):
    """M_h^{-1} (n_x x n_x) of the consistent mixed mass; passing it as L to a
    solver selects the preconditioner M_h^{-1} D_h M_h^{-T}."""
    out = ctx.empty((mesh.n_x, mesh.n_x))
    ctx.check(ctx.lib.stbem_mixed_mass_inverse(ctx.h, mesh.h, _ptr(out)))
    return out


def _prec_mode(D, L):
    if D is None:
        return 0
    return 2 if (L is not None and L.dim() == 2) else 1


def lumped_mass(ctx: Context, mesh: Mesh):
    L = ctx.empty((mesh.n_x,))
    ctx.check(ctx.lib.stbem_lumped_mass(ctx.h, mesh.h, _ptr(L)))
    return L


def solve_workspace(ctx: Context, n_t: int, n_x: int, restart: int):
    nb = ctypes.c_size_t()
    ctx.check(ctx.lib.stbem_solve_workspace_bytes(n_t, n_x, restart, ctypes.byref(nb)))
    return torch.empty(nb.value, dtype=torch.uint8, device=ctx.device)


def solve(ctx: Context, V, f, D=None, L=None, tol: float = 1e-8, max_iter: int = 500,
          restart: int = 200, work=None, out=None, raise_on_fail: bool = True):
    """Right-preconditioned GMRES for V_h w = f; returns (w, info dict)."""
    n_t, n_x = V.shape[0], V.shape[1]
    prec = capi.F64 if V.dtype == torch.float64 else capi.F32
    if D is not None and D.dtype != V.dtype:
        raise ValueError("V and D must share a precision")
    opts = capi.SolveOpts(tol, max_iter, restart, _prec_mode(D, L))
    info = capi.SolveInfo()
    if out is None:
        out = ctx.empty((n_t, n_x))
    if work is None:
        work = solve_workspace(ctx, n_t, n_x, restart)
    code = ctx.lib.stbem_solve(ctx.h, n_t, n_x, prec, _ptr(V), _ptr(D), _ptr(L), _ptr(f), _ptr(out),
                               ctypes.byref(opts), ctypes.byref(info), _ptr(work), work.numel())
    res = {"iterations": info.iterations, "status": info.status, "rel_residual": info.rel_residual}
    if code != capi.STBEM_OK and raise_on_fail:
        ctx.check(code)
    return out, res


def solve_adjoint(ctx: Context, V, b, D=None, L=None, tol: float = 1e-8, max_iter: int = 500,
                  restart: int = 200, work=None, out=None, raise_on_fail: bool = True):
    """GMRES for the adjoint V_h^T lam = b (backward in time); returns (lam, info)."""
    n_t, n_x = V.shape[0], V.shape[1]
    prec = capi.F64 if V.dtype == torch.float64 else capi.F32
    opts = capi.SolveOpts(tol, max_iter, restart, _prec_mode(D, L))
    info = capi.SolveInfo()
    if out is None:
        out = ctx.empty((n_t, n_x))
    if work is None:
        work = solve_workspace(ctx, n_t, n_x, restart)
    code = ctx.lib.stbem_solve_adjoint(ctx.h, n_t, n_x, prec, _ptr(V), _ptr(D), _ptr(L), _ptr(b), _ptr(out),
                                       ctypes.byref(opts), ctypes.byref(info), _ptr(work), work.numel())
    res = {"iterations": info.iterations, "status": info.status, "rel_residual": info.rel_residual}
    if code != capi.STBEM_OK and raise_on_fail:
        ctx.check(code)
    return out, res


class FFTOperator:
    """Frequency blocks Ahat_k = sum_d A_d w^{d k}, k = 0 .. L/2, of an
    n_t x n_x x n_x lag-block operator (stbem_fft_operator): `data` is a
    complex128 array (L/2 + 1) x n_x x n_x."""

    def __init__(self, data, n_t: int, n_x: int):
        self.data, self.n_t, self.n_x = data, n_t, n_x


def fft_operator(ctx: Context, A, out=None) -> FFTOperator:
    """The frequency blocks of the lag blocks A (FP64 or FP32, n_t x n_x x n_x)."""
    n_t, n_x = A.shape[0], A.shape[1]
    prec = capi.F64 if A.dtype == torch.float64 else capi.F32
    nf, nb = ctypes.c_int(), ctypes.c_size_t()
    ctx.check(ctx.lib.stbem_fft_operator_bytes(n_t, n_x, ctypes.byref(nf), ctypes.byref(nb)))
    if out is None:
        out = torch.empty((nf.value, n_x, n_x), dtype=torch.complex128, device=ctx.device)
    elif out.dtype != torch.complex128 or tuple(out.shape) != (nf.value, n_x, n_x) or not out.is_contiguous():
        raise ValueError("fft_operator: out must be a contiguous complex128 array of shape %s"
                         % ((nf.value, n_x, n_x),))
    ctx.check(ctx.lib.stbem_fft_operator(ctx.h, n_t, n_x, prec, _ptr(A.contiguous()), _ptr(out)))
    return FFTOperator(out, n_t, n_x)


def apply_fft_workspace(ctx: Context, n_t: int, n_x: int, n_rhs: int = 1):
    nb = ctypes.c_size_t()
    ctx.check(ctx.lib.stbem_apply_fft_workspace_bytes(n_t, n_x, n_rhs, ctypes.byref(nb)))
    return torch.empty(nb.value, dtype=torch.uint8, device=ctx.device)


def apply_fft(ctx: Context, Ah: FFTOperator, x, transpose: bool = False, work=None, out=None):
    """y = A x (or A^T x) through the frequency blocks (x: [n_rhs,] n_t x n_x, FP64)."""
    xb = x if x.dim() == 3 else x.unsqueeze(0)
    n_rhs = xb.shape[0]
    if out is None:
        out = torch.empty_like(x)
    if work is None:
        work = apply_fft_workspace(ctx, Ah.n_t, Ah.n_x, n_rhs)
    ctx.check(ctx.lib.stbem_apply_fft(ctx.h, int(transpose), Ah.n_t, Ah.n_x, n_rhs, _ptr(Ah.data), _ptr(x),
                                      _ptr(out), _ptr(work), work.numel()))
    return out


def solve_fft_workspace(ctx: Context, n_t: int, n_x: int, restart: int):
    nb = ctypes.c_size_t()
    ctx.check(ctx.lib.stbem_solve_fft_workspace_bytes(n_t, n_x, restart, ctypes.byref(nb)))
    return torch.empty(nb.value, dtype=torch.uint8, device=ctx.device)


def solve_fft(ctx: Context, Vh: FFTOperator, f, Dh: FFTOperator = None, L=None, tol: float = 1e-8,
              max_iter: int = 500, restart: int = 200, transpose: bool = False, work=None, out=None,
              raise_on_fail: bool = True):
    """solve (or solve_adjoint with transpose) with the products of V_h and
    D_h through their frequency blocks; returns (w, info dict)."""
    n_t, n_x = Vh.n_t, Vh.n_x
    opts = capi.SolveOpts(tol, max_iter, restart, _prec_mode(Dh, L))
    info = capi.SolveInfo()
    if out is None:
        out = ctx.empty((n_t, n_x))
    if work is None:
        work = solve_fft_workspace(ctx, n_t, n_x, restart)
    code = ctx.lib.stbem_solve_fft(ctx.h, int(transpose), n_t, n_x, _ptr(Vh.data),
                                   _ptr(Dh.data) if Dh is not None else None, _ptr(L), _ptr(f), _ptr(out),
                                   ctypes.byref(opts), ctypes.byref(info), _ptr(work), work.numel())
    res = {"iterations": info.iterations, "status": info.status, "rel_residual": info.rel_residual}
    if code != capi.STBEM_OK and raise_on_fail:
        ctx.check(code)
    return out, res


def grad_workspace(ctx: Context, n_t: int, n_x: int):
    nb = ctypes.c_size_t()
    ctx.check(ctx.lib.stbem_grad_workspace_bytes(n_t, n_x, ctypes.byref(nb)))
    return torch.empty(nb.value, dtype=torch.uint8, device=ctx.device)


def grad(ctx: Context, mesh: Mesh, K, y_star, g, w, lam, work=None):
    """lam^T (df/dtheta - dV_h/dtheta w) for the vertices (n_x, 2) and alpha
    (0-dim tensor), f = 1/2 M_h g + K_h g with g the datum of source y_star."""
    dxy = ctx.empty((mesh.n_x, 2))
    dal = ctx.empty((1,))
    if work is None:
        work = grad_workspace(ctx, mesh.n_t, mesh.n_x)
    ctx.check(ctx.lib.stbem_grad(ctx.h, mesh.h, _ptr(K), float(y_star[0]), float(y_star[1]), _ptr(g), _ptr(w),
                                 _ptr(lam), _ptr(dxy), _ptr(dal), _ptr(work), work.numel()))
    return dxy, dal[0]


def pipe_peaks(ctx: Context):
    """Measured pipe rates of the context's GPU (stbem_pipe_peaks): FP64 and
    FP32 FMA TFLOP/s and MUFU ex2 results per second (1e12)."""
    out = (ctypes.c_double * 3)()
    ctx.check(ctx.lib.stbem_pipe_peaks(ctx.h, out))
    return {"fp64_tflops": out[0], "fp32_tflops": out[1], "ex2_tera_per_s": out[2]}


def round_f32(ctx: Context, A):
    """FP32 copy of an FP64 operator (rounded by a library kernel)."""
    out = torch.empty(A.shape, dtype=torch.float32, device=A.device)
    ctx.check(ctx.lib.stbem_round_f32(ctx.h, A.numel(), _ptr(A), _ptr(out)))
    return out


def solve_mixed(ctx: Context, V64, V32, f, D32=None, L=None, tol: float = 1e-8, inner_tol: float = 1e-4,
                max_iter: int = 500, restart: int = 200, work=None, out=None, raise_on_fail: bool = True):
    """FP64 iterative refinement around preconditioned GMRES on FP32 operators.
    V64 gives the outer residuals: the FP64 lag blocks (an FP64 CUDA-core
    product) or their ExactOperand (the exact-slice tensor-core product).
    With V32 and D32 given as the three BF16 slices of V and D
    (bf16_split3) and V64 an ExactOperand, the inner GMRES runs on the
    tensor cores (three-slice products, FP32-grade accuracy)."""
    n_t, n_x = V64.shape[0], V64.shape[1]
    exact = isinstance(V64, ExactOperand)
    if isinstance(V32, (tuple, list)):
        if not exact:
            raise ValueError("solve_mixed: tensor-core inner operators need an ExactOperand V64")
        Vs = list(V32) + [None] * (3 - len(V32))
        Ds = list(D32) + [None] * (3 - len(D32)) if D32 is not None else [None] * 3
        opts = capi.SolveOpts(tol, max_iter, restart, _prec_mode(D32, L))
        info = capi.SolveInfo()
        if out is None:
            out = ctx.empty((n_t, n_x))
        if work is None:
            nb = ctypes.c_size_t()
            ctx.check(ctx.lib.stbem_solve_mixed_tc_workspace_bytes(n_t, n_x, restart, V64.n_slices,
                                                                   ctypes.byref(nb)))
            work = torch.empty(nb.value, dtype=torch.uint8, device=ctx.device)
        sv = V64.c_struct()
        code = ctx.lib.stbem_solve_mixed_tc(ctx.h, n_t, n_x, ctypes.byref(sv), _ptr(Vs[0]), _ptr(Vs[1]), _ptr(Vs[2]),
                                            _ptr(Ds[0]), _ptr(Ds[1]), _ptr(Ds[2]), _ptr(L), _ptr(f), _ptr(out),
                                            ctypes.byref(opts), float(inner_tol), ctypes.byref(info), _ptr(work),
                                            work.numel())
        res = {"iterations": info.iterations, "status": info.status, "rel_residual": info.rel_residual}
        if code != capi.STBEM_OK and raise_on_fail:
            ctx.check(code)
        return out, res
    opts = capi.SolveOpts(tol, max_iter, restart, _prec_mode(D32, L))
    info = capi.SolveInfo()
    if out is None:
        out = ctx.empty((n_t, n_x))
    if work is None:
        nb = ctypes.c_size_t()
        if exact:
            ctx.check(ctx.lib.stbem_solve_mixed_exact_workspace_bytes(n_t, n_x, restart, V64.n_slices,
                                                                      ctypes.byref(nb)))
        else:
            ctx.check(ctx.lib.stbem_solve_mixed_workspace_bytes(n_t, n_x, restart, ctypes.byref(nb)))
        work = torch.empty(nb.value, dtype=torch.uint8, device=ctx.device)
    if exact:
        sv = V64.c_struct()
        code = ctx.lib.stbem_solve_mixed_exact(ctx.h, n_t, n_x, ctypes.byref(sv), _ptr(V32), _ptr(D32), _ptr(L),
                                               _ptr(f), _ptr(out), ctypes.byref(opts), float(inner_tol),
                                               ctypes.byref(info), _ptr(work), work.numel())
    else:
        code = ctx.lib.stbem_solve_mixed(ctx.h, n_t, n_x, _ptr(V64), _ptr(V32), _ptr(D32), _ptr(L), _ptr(f),
                                         _ptr(out), ctypes.byref(opts), float(inner_tol), ctypes.byref(info),
                                         _ptr(work), work.numel())
    res = {"iterations": info.iterations, "status": info.status, "rel_residual": info.rel_residual}
    if code != capi.STBEM_OK and raise_on_fail:
        ctx.check(code)
    return out, res


def to_bf16(ctx: Context, src):
    """BF16 copy (round to nearest even) of an FP64 or FP32 tensor."""
    out = torch.empty(src.shape, dtype=torch.bfloat16, device=src.device)
    prec = capi.F64 if src.dtype == torch.float64 else capi.F32
    ctx.check(ctx.lib.stbem_to_bf16(ctx.h, prec, src.numel(), _ptr(src), _ptr(out)))
    return out


def apply_tc(ctx: Context, A_bf16, x_bf16, out=None, chunk=0):
    """Tensor-core block-Toeplitz product: BF16 A (n_t, n_x, n_x) times BF16 x
    (n_rhs, n_t, n_x), FP32 accumulation, FP64 result (n_rhs, n_t, n_x).
    chunk > 0 selects the compensated accumulation (FP32 partials of `chunk`
    64-wide K steps, Kahan-summed)."""
    n_t, n_x = A_bf16.shape[0], A_bf16.shape[1]
    xb = x_bf16 if x_bf16.dim() == 3 else x_bf16.unsqueeze(0)
    if out is None:
        out = torch.empty(xb.shape, dtype=torch.float64, device=xb.device)
    if chunk:
        ctx.check(ctx.lib.stbem_apply_tc_comp(ctx.h, n_t, n_x, _ptr(A_bf16), xb.shape[0], _ptr(xb), _ptr(out),
                                              int(chunk)))
    else:
        ctx.check(ctx.lib.stbem_apply_tc(ctx.h, n_t, n_x, _ptr(A_bf16), xb.shape[0], _ptr(xb), _ptr(out)))
    return out if x_bf16.dim() == 3 else out[0]


def bf16_split3(ctx: Context, src):
    """Three BF16 slices (hi, mid, lo) of an FP64 tensor."""
    outs = [torch.empty(src.shape, dtype=torch.bfloat16, device=src.device) for _ in range(3)]
    ctx.check(ctx.lib.stbem_bf16_split3(ctx.h, src.numel(), _ptr(src), _ptr(outs[0]), _ptr(outs[1]), _ptr(outs[2])))
    return outs


def apply_tc3(ctx: Context, A_slices, x, out=None, work=None):
    """Accurate tensor-core product with a three-slice BF16 operator and FP64 x."""
    n_t, n_x = A_slices[0].shape[0], A_slices[0].shape[1]
    xb = x if x.dim() == 3 else x.unsqueeze(0)
    if out is None:
        out = torch.empty_like(xb)
    if work is None:
        nb = ctypes.c_size_t()
        ctx.check(ctx.lib.stbem_apply_tc3_workspace_bytes(n_t, n_x, xb.shape[0], ctypes.byref(nb)))
        work = torch.empty(nb.value, dtype=torch.uint8, device=xb.device)
    A = list(A_slices) + [None] * (3 - len(A_slices))
    ctx.check(ctx.lib.stbem_apply_tc3(ctx.h, n_t, n_x, _ptr(A[0]), _ptr(A[1]), _ptr(A[2]), xb.shape[0], _ptr(xb),
                                      _ptr(out), _ptr(work), work.numel()))
    return out if x.dim() == 3 else out[0]


class ExactOperand:
    """Exact-slice form of an FP64 tensor whose last axis is a row: ``slices``
    (BF16, (n_slices,) + shape) and ``row_exp`` (int32, shape[:-1]), with
    row = 2^row_exp sum_s slices[s] 2^(-6 (s + 1)) to 6 n_slices bits."""

    def __init__(self, ctx: Context, src, n_slices: int = 7):
        if src.dtype != torch.float64 or not src.is_contiguous():
            raise ValueError("ExactOperand: a contiguous FP64 tensor is required")
        self.shape = tuple(src.shape)
        self.n_slices = int(n_slices)
        cols = src.shape[-1]
        rows = src.numel() // cols
        self.slices = torch.empty((self.n_slices,) + self.shape, dtype=torch.bfloat16, device=src.device)
        self.row_exp = torch.empty(self.shape[:-1], dtype=torch.int32, device=src.device)
        ctx.check(ctx.lib.stbem_exact_slices(ctx.h, rows, cols, self.n_slices, _ptr(src), _ptr(self.slices),
                                             _ptr(self.row_exp)))

    def c_struct(self):
        return capi.ExactOperand(self.n_slices, self.slices.data_ptr(), self.row_exp.data_ptr())


def exact_slices(ctx: Context, src, n_slices: int = 7):
    """The exact-slice form (ExactOperand) of FP64 lag blocks (n_t, n_x, n_x)
    or right-hand sides (n_rhs, n_t, n_x)."""
    return ExactOperand(ctx, src, n_slices)


def apply_exact(ctx: Context, A, x, out=None, work=None):
    """Block-Toeplitz product on the tensor cores to FP64-grade accuracy
    relative to the row scales (at most 2^(-6 n_slices) (1 + n_slices / 4)
    n_x sum_d 2^(eA[d][i] + eX[b][m - d])): A an ExactOperand of lag blocks,
    x FP64 (n_rhs, n_t, n_x) or (n_t, n_x), or an ExactOperand of it."""
    n_t, n_x = A.shape[0], A.shape[1]
    sa = A.c_struct()
    if isinstance(x, ExactOperand):
        B = x.shape[0] if len(x.shape) == 3 else 1
        if out is None:
            out = torch.empty((B, n_t, n_x), dtype=torch.float64, device=A.slices.device)
        sx = x.c_struct()
        ctx.check(ctx.lib.stbem_apply_tc_exact(ctx.h, n_t, n_x, ctypes.byref(sa), B, ctypes.byref(sx), _ptr(out)))
        return out if len(x.shape) == 3 else out[0]
    xb = x if x.dim() == 3 else x.unsqueeze(0)
    if out is None:
        out = torch.empty_like(xb)
    if work is None:
        nb = ctypes.c_size_t()
        ctx.check(ctx.lib.stbem_apply_exact_workspace_bytes(n_t, n_x, xb.shape[0], A.n_slices, ctypes.byref(nb)))
        work = torch.empty(nb.value, dtype=torch.uint8, device=xb.device)
    ctx.check(ctx.lib.stbem_apply_exact(ctx.h, n_t, n_x, ctypes.byref(sa), xb.shape[0], _ptr(xb), _ptr(out),
                                        _ptr(work), work.numel()))
    return out if x.dim() == 3 else out[0]


def rhs_batched(ctx: Context, mesh: Mesh, K, y_stars):
    """(G, F) for many sources: G[k] vertex time averages of U*(x - y_k, t),
    F = 1/2 M_h G + K_h G.  K is the FP64 operator (an FP64 CUDA-core product
    of all right-hand sides: F to FP64 accuracy), its ExactOperand (the
    exact-slice tensor-core product, normwise a few 1e-13 at 7 slices), its
    FFTOperator (the product through time FFTs, FP64, normwise) or a tuple of
    its three BF16 slices (the compensated tensor-core product, a few 1e-7 of
    |K||G|)."""
    ys = np.ascontiguousarray(np.asarray(y_stars, dtype=np.float64).reshape(-1))
    B = ys.size // 2
    G = ctx.empty((B, mesh.n_t, mesh.n_x))
    ctx.check(ctx.lib.stbem_rhs_g_batched(ctx.h, mesh.h, B, ys.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          _ptr(G)))
    if isinstance(K, ExactOperand):
        F = apply_exact(ctx, K, G)
    elif isinstance(K, FFTOperator):
        F = apply_fft(ctx, K, G)
    elif isinstance(K, (tuple, list)):
        F = apply_tc3(ctx, K, G)
    else:
        F = apply(ctx, K, G)
    ctx.check(ctx.lib.stbem_half_mass_add(ctx.h, mesh.h, B, _ptr(G), _ptr(F)))
    return G, F


def solve_batched(ctx: Context, V_slices, F, D_bf16=None, L=None, tol: float = 1e-6, inner_tol: float = 1e-2,
                  max_iter: int = 400, restart: int = 40, work=None, out=None, raise_on_fail: bool = True,
                  V64=None):
    """Many-right-hand-side solve on the tensor cores; returns (W, infos).
    With V64 the refinement finishes on residuals of that operator: the FP64
    lag blocks (an FP64 CUDA-core product), their ExactOperand (the
    exact-slice tensor-core product) or their FFTOperator (the FP64 product
    through time FFTs); each gives FP64-solve accuracy for tol down to 1e-8
    and below."""
    B, n_t, n_x = F.shape
    opts = capi.SolveOpts(tol, max_iter, restart, int(D_bf16 is not None))
    infos = (capi.SolveInfo * B)()
    if out is None:
        out = torch.empty_like(F)
    exact = isinstance(V64, ExactOperand)
    fft = isinstance(V64, FFTOperator)
    if work is None:
        nb = ctypes.c_size_t()
        if fft:
            ctx.check(ctx.lib.stbem_solve_batched_fft_workspace_bytes(n_t, n_x, B, restart, ctypes.byref(nb)))
        elif exact:
            ctx.check(ctx.lib.stbem_solve_batched_exact_workspace_bytes(n_t, n_x, B, restart, V64.n_slices,
                                                                        ctypes.byref(nb)))
        else:
            ctx.check(ctx.lib.stbem_solve_batched_workspace_bytes(n_t, n_x, B, restart, int(V64 is not None),
                                                                  ctypes.byref(nb)))
        work = torch.empty(nb.value, dtype=torch.uint8, device=F.device)
    Vs = list(V_slices) + [None] * (3 - len(V_slices))
    if fft:
        code = ctx.lib.stbem_solve_batched_fft(ctx.h, n_t, n_x, B, _ptr(Vs[0]), _ptr(Vs[1]), _ptr(Vs[2]),
                                               _ptr(D_bf16), _ptr(L), _ptr(V64.data), _ptr(F), _ptr(out),
                                               ctypes.byref(opts), float(inner_tol), infos, _ptr(work), work.numel())
    elif exact:
        sv = V64.c_struct()
        code = ctx.lib.stbem_solve_batched_exact(ctx.h, n_t, n_x, B, _ptr(Vs[0]), _ptr(Vs[1]), _ptr(Vs[2]),
                                                 _ptr(D_bf16), _ptr(L), ctypes.byref(sv), _ptr(F), _ptr(out),
                                                 ctypes.byref(opts), float(inner_tol), infos, _ptr(work), work.numel())
    else:
        code = ctx.lib.stbem_solve_batched(ctx.h, n_t, n_x, B, _ptr(Vs[0]), _ptr(Vs[1]), _ptr(Vs[2]), _ptr(D_bf16),
                                           _ptr(L), _ptr(V64), _ptr(F), _ptr(out), ctypes.byref(opts),
                                           float(inner_tol), infos, _ptr(work), work.numel())
    res = [{"iterations": i.iterations, "status": i.status, "rel_residual": i.rel_residual} for i in infos]
    if code != capi.STBEM_OK and raise_on_fail:
        ctx.check(code)
    return out, res


def tune_cache(path):
    """Back the tuned-launch-parameter cache with a text file (None: memory
    only); entries already in the file are loaded.  The STBEM_TUNE_CACHE
    environment variable sets the default file."""
    code = capi.load().stbem_tune_cache_path(None if path is None else str(path).encode())
    if code != capi.STBEM_OK:
        raise capi.StbemError(code, "tune cache file %s cannot be read" % path)


def tune_cache_get(key: str):
    """The cached value for key, or None."""
    buf = ctypes.create_string_buffer(512)
    code = capi.load().stbem_tune_cache_get(key.encode(), buf, len(buf))
    return buf.value.decode() if code == capi.STBEM_OK else None


def tune_cache_put(key: str, value: str):
    code = capi.load().stbem_tune_cache_put(key.encode(), value.encode())
    if code != capi.STBEM_OK:
        raise capi.StbemError(code, "tune cache: bad entry or unwritable file")


def tune_cache_clear():
    """Forget every in-process entry (the backing file is kept)."""
    capi.load().stbem_tune_cache_clear()


def tc_tune(ctx: Context, A_bf16, x_bf16, out=None):
    """Pick the plain tensor-core product's tile width (128 or 256 steps) for
    this shape by timing both (or take the cached choice); later products of
    the shape use it.  Returns (tile_n, from_cache)."""
    n_t, n_x = A_bf16.shape[0], A_bf16.shape[1]
    xb = x_bf16 if x_bf16.dim() == 3 else x_bf16.unsqueeze(0)
    if out is None:
        out = torch.empty(xb.shape, dtype=torch.float64, device=xb.device)
    tn, cached = ctypes.c_int(), ctypes.c_int()
    ctx.check(ctx.lib.stbem_tc_tune(ctx.h, n_t, n_x, _ptr(A_bf16), xb.shape[0], _ptr(xb), _ptr(out),
                                    ctypes.byref(tn), ctypes.byref(cached)))
    return tn.value, bool(cached.value)


class Ragged:
    """A ragged batch: independent problems of different sizes handled by one
    persistent launch per step (stbem_ragged_*).  ``problems`` is a list of
    (vertices (n_x, 2), T, n_t, alpha).  Batch arrays are the problems' arrays
    concatenated; ``view_op`` / ``view_vec`` return one problem's part."""

    def __init__(self, ctx: Context, problems):
        self.ctx = ctx
        self._xy = [np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1)) for v, _, _, _ in problems]
        arr = (capi.Problem * len(problems))()
        for k, (v, T, n_t, alpha) in enumerate(problems):
            arr[k].xy = self._xy[k].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            arr[k].n_x = self._xy[k].size // 2
            arr[k].n_t = int(n_t)
            arr[k].T = float(T)
            arr[k].alpha = float(alpha)
        self.P = len(problems)
        self.n_x = [self._xy[k].size // 2 for k in range(self.P)]
        self.n_t = [int(p[2]) for p in problems]
        h = ctypes.c_void_p()
        ctx.check(ctx.lib.stbem_ragged_create(ctx.h, self.P, arr, ctypes.byref(h)))
        self.h = h
        ll = ctypes.c_longlong
        a, b, c = ll(), ll(), ll()
        ctx.check(ctx.lib.stbem_ragged_sizes(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        self.op_elems, self.vec_elems, self.mass_elems = a.value, b.value, c.value
        oo, vo, mo = (ll * self.P)(), (ll * self.P)(), (ll * self.P)()
        ctx.check(ctx.lib.stbem_ragged_offsets(self.h, oo, vo, mo))
        self.op_off, self.vec_off, self.mass_off = list(oo), list(vo), list(mo)
        self._awork = None

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.stbem_ragged_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # views of one problem's part of a batch array
    def view_op(self, A, p):
        n, t = self.n_x[p], self.n_t[p]
        return A[self.op_off[p]:self.op_off[p] + t * n * n].view(t, n, n)

    def view_vec(self, x, p):
        n, t = self.n_x[p], self.n_t[p]
        return x[self.vec_off[p]:self.vec_off[p] + t * n].view(t, n)

    def view_mass(self, L, p):
        return L[self.mass_off[p]:self.mass_off[p] + self.n_x[p]]

    def apply_workspace(self):
        if self._awork is None:
            nb = ctypes.c_size_t()
            self.ctx.check(self.ctx.lib.stbem_ragged_apply_workspace_bytes(self.h, ctypes.byref(nb)))
            self._awork = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=self.ctx.device)
        return self._awork

    def assemble(self, op: str, prec: str = "f64", out=None):
        p = PRECS[prec]
        if out is None:
            out = torch.empty(self.op_elems, dtype=torch.float64 if p == capi.F64 else torch.float32,
                              device=self.ctx.device)
        self.ctx.check(self.ctx.lib.stbem_ragged_assemble(self.ctx.h, self.h, OPS[op], p, _ptr(out)))
        return out

    def lumped_mass(self):
        L = self.ctx.empty((self.mass_elems,))
        self.ctx.check(self.ctx.lib.stbem_ragged_lumped_mass(self.ctx.h, self.h, _ptr(L)))
        return L

    def apply(self, A, x, out=None):
        p = capi.F64 if A.dtype == torch.float64 else capi.F32
        if out is None:
            out = self.ctx.empty((self.vec_elems,))
        w = self.apply_workspace()
        self.ctx.check(self.ctx.lib.stbem_ragged_apply(self.ctx.h, self.h, p, _ptr(A), _ptr(x), _ptr(out), _ptr(w),
                                                        w.numel()))
        return out

    def tune(self, A, x, y):
        """Autotune the product on A over the tile family (FP32 register tiles
        or generic tiles) and the lag-chunk length, or take the choice the
        tune cache holds for these shapes on this device.  Returns (choice,
        report): choice = {"tiles32", "lags_per_chunk", "from_cache"},
        report = {"tiles32=T lpc=C": ms} of the candidates timed (empty when
        the choice came from the cache)."""
        p = capi.F64 if A.dtype == torch.float64 else capi.F32
        w = self.apply_workspace()
        best, t32b = ctypes.c_int(), ctypes.c_int()
        self.ctx.check(self.ctx.lib.stbem_ragged_tune(self.ctx.h, self.h, p, _ptr(A), _ptr(x), _ptr(y), _ptr(w),
                                                       w.numel(), ctypes.byref(best), ctypes.byref(t32b)))
        cand, t32, ms = (ctypes.c_int * 32)(), (ctypes.c_int * 32)(), (ctypes.c_float * 32)()
        n, cached = ctypes.c_int(), ctypes.c_int()
        self.ctx.check(self.ctx.lib.stbem_ragged_tune_report(self.h, 32, cand, t32, ms, ctypes.byref(n),
                                                              ctypes.byref(cached)))
        report = {"tiles32=%d lpc=%d" % (t32[k], cand[k]): ms[k] for k in range(min(n.value, 32))}
        return {"tiles32": t32b.value, "lags_per_chunk": best.value, "from_cache": bool(cached.value)}, report

    def rhs(self, K, y_stars):
        p = capi.F64 if K.dtype == torch.float64 else capi.F32
        ys = np.ascontiguousarray(np.asarray(y_stars, dtype=np.float64).reshape(-1))
        g = self.ctx.empty((self.vec_elems,))
        f = self.ctx.empty((self.vec_elems,))
        aw = self.apply_workspace()
        work = torch.empty(aw.numel() + 256 + ((16 * self.P + 255) // 256) * 256, dtype=torch.uint8,
                           device=self.ctx.device)
        self.ctx.check(self.ctx.lib.stbem_ragged_rhs(self.ctx.h, self.h, p, _ptr(K),
                                                      ys.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(g),
                                                      _ptr(f), _ptr(work), work.numel()))
        return g, f

    def solve_workspace(self, restart: int):
        nb = ctypes.c_size_t()
        self.ctx.check(self.ctx.lib.stbem_ragged_solve_workspace_bytes(self.h, restart, ctypes.byref(nb)))
        return torch.empty(nb.value, dtype=torch.uint8, device=self.ctx.device)

    def solve(self, V, f, D=None, L=None, tol: float = 1e-8, max_iter: int = 500, restart: int = 60, work=None,
              out=None, raise_on_fail: bool = True):
        p = capi.F64 if V.dtype == torch.float64 else capi.F32
        opts = capi.SolveOpts(tol, max_iter, restart, int(D is not None))
        infos = (capi.SolveInfo * self.P)()
        if out is None:
            out = self.ctx.empty((self.vec_elems,))
        if work is None:
            work = self.solve_workspace(restart)
        code = self.ctx.lib.stbem_ragged_solve(self.ctx.h, self.h, p, _ptr(V), _ptr(D), _ptr(L), _ptr(f), _ptr(out),
                                               ctypes.byref(opts), infos, _ptr(work), work.numel())
        res = [{"iterations": x.iterations, "status": x.status, "rel_residual": x.rel_residual} for x in infos]
        if code != capi.STBEM_OK and raise_on_fail:
            self.ctx.check(code)
        return out, res

    def solve_mixed_workspace(self, restart: int):
        nb = ctypes.c_size_t()
        self.ctx.check(self.ctx.lib.stbem_ragged_solve_mixed_workspace_bytes(self.h, restart, ctypes.byref(nb)))
        return torch.empty(nb.value, dtype=torch.uint8, device=self.ctx.device)

    def solve_mixed(self, V64, V32, f, D32=None, L=None, tol: float = 1e-8, inner_tol: float = 1e-4,
                    max_iter: int = 500, restart: int = 60, work=None, out=None, raise_on_fail: bool = True):
        """FP64 refinement (residuals with the FP64 V64) around lockstep FP32
        solves (V32, D32): every problem to an FP64 residual <= tol."""
        opts = capi.SolveOpts(tol, max_iter, restart, int(D32 is not None))
        infos = (capi.SolveInfo * self.P)()
        if out is None:
            out = self.ctx.empty((self.vec_elems,))
        if work is None:
            work = self.solve_mixed_workspace(restart)
        code = self.ctx.lib.stbem_ragged_solve_mixed(self.ctx.h, self.h, _ptr(V64), _ptr(V32), _ptr(D32), _ptr(L),
                                                     _ptr(f), _ptr(out), ctypes.byref(opts), float(inner_tol),
                                                     infos, _ptr(work), work.numel())
        res = [{"iterations": x.iterations, "status": x.status, "rel_residual": x.rel_residual} for x in infos]
        if code != capi.STBEM_OK and raise_on_fail:
            self.ctx.check(code)
        return out, res
