"""torch.autograd around the space-time BEM solve.

``neumann_solve(ctx, vertices, alpha, y_star, T, n_t)`` returns the Galerkin
solution w_h (n_t x n_x, FP64, on the context's device) of V_h w = f,
f = (1/2 M_h + K_h) g, for the polygon ``vertices`` (n_x x 2, counter-clockwise)
and the manufactured datum g = U*(x - y*, t) (Section 1, eq. (4) with u_0 = 0).
It is differentiable in ``vertices`` and ``alpha``: the backward pass solves the
adjoint system V_h^T lambda = dL/dw with the transposed (backward-in-time)
products and calls the assembly-derivative kernels, which recompute the
quadrature of every pair and contract it with C(d) = sum_m lambda_m x_{m-d}^T
(stbem_grad).  Everything after the vertex upload runs in the library's
kernels; the vertices themselves go to the host once per call, as the mesh
handle is built from a host array.
"""
import torch

from . import api


class _NeumannSolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, vertices, alpha, ctx, y_star, T, n_t, tol, restart):
        X = vertices.detach().to("cpu", torch.float64).numpy()
        al = float(alpha.detach())
        mesh = api.Mesh(ctx, X, T, n_t, al)
        V = api.assemble(ctx, mesh, "V")
        K = api.assemble(ctx, mesh, "K")
        D = api.assemble(ctx, mesh, "D")
        L = api.lumped_mass(ctx, mesh)
        g, f = api.rhs(ctx, mesh, K, y_star)
        w, info = api.solve(ctx, V, f, D, L, tol=tol, restart=restart, max_iter=20 * restart)
        fctx.state = (ctx, mesh, V, K, D, L, g, w, tuple(float(v) for v in y_star), tol, restart)
        fctx.dev = (vertices.device, alpha.device)
        fctx.info = info
        return w

    @staticmethod
    def backward(fctx, grad_w):
        ctx, mesh, V, K, D, L, g, w, y_star, tol, restart = fctx.state
        b = grad_w.detach().to(ctx.device, torch.float64).contiguous()
        lam, _ = api.solve_adjoint(ctx, V, b, D, L, tol=tol, restart=restart, max_iter=20 * restart)
        dxy, dal = api.grad(ctx, mesh, K, y_star, g, w, lam)
        vdev, adev = fctx.dev
        return dxy.to(vdev), dal.to(adev), None, None, None, None, None, None


def neumann_solve(ctx, vertices, alpha, y_star, T: float, n_t: int, tol: float = 1e-12, restart: int = 100):
    """w_h(vertices, alpha) for the datum of source ``y_star``; differentiable
    in ``vertices`` ((n_x, 2) float64 tensor) and ``alpha`` (0-dim float64 tensor)."""
    if not torch.is_tensor(alpha):
        alpha = torch.tensor(float(alpha), dtype=torch.float64)
    return _NeumannSolve.apply(vertices, alpha, ctx, tuple(y_star), float(T), int(n_t), float(tol), int(restart))
