"""torch.autograd around the space-time BEM solve.

``neumann_solve(ctx, vertices, alpha, y_star, T, n_t)`` returns the Galerkin
solution w_h (n_t x n_x, FP64, on the context's device) of V_h w = f,
f = (1/2 M_h + K_h) g, for the polygon ``vertices`` (n_x x 2, counter-clockwise)
and the manufactured datum g = U*(x - y*, t) (Section 1, eq. (4) with u_0 = 0).
It is differentiable in ``vertices`` and ``alpha``: the backward pass solves the
adjoint system V_h^T lambda = dL/dw with the transposed (backward-in-time)
products and calls the assembly-derivative kernels, which recompute the
quadrature of every pair and contract it with C(d) = sum_m lambda_m x_{m-d}^T
(stbem_grad).  With ``products="fft"`` the forward and adjoint GMRES take
their products of V_h and D_h through the frequency blocks of the lag blocks
(time FFTs, stbem_solve_fft); ``"direct"`` uses the block sums.  Everything
after the vertex upload runs in the library's kernels; the vertices
themselves go to the host once per call, as the mesh handle is built from a
host array.
"""
import torch

from . import api


class _NeumannSolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, vertices, alpha, ctx, y_star, T, n_t, tol, restart, products):
        X = vertices.detach().to("cpu", torch.float64).numpy()
        al = float(alpha.detach())
        mesh = api.Mesh(ctx, X, T, n_t, al)
        ops = api.assemble_ops(ctx, mesh, "f64")
        V, K, D = ops["V"], ops["K"], ops["D"]
        L = api.lumped_mass(ctx, mesh)
        g, f = api.rhs(ctx, mesh, K, y_star)
        if products == "fft":
            # the frequency blocks replace V and D for both solves
            V, D = api.fft_operator(ctx, V), api.fft_operator(ctx, D)
            del ops
            w, info = api.solve_fft(ctx, V, f, D, L, tol=tol, restart=restart, max_iter=20 * restart)
        else:
            w, info = api.solve(ctx, V, f, D, L, tol=tol, restart=restart, max_iter=20 * restart)
        fctx.state = (ctx, mesh, V, K, D, L, g, w, tuple(float(v) for v in y_star), tol, restart, products)
        fctx.dev = (vertices.device, alpha.device)
        fctx.info = info
        return w

    @staticmethod
    def backward(fctx, grad_w):
        ctx, mesh, V, K, D, L, g, w, y_star, tol, restart, products = fctx.state
        b = grad_w.detach().to(ctx.device, torch.float64).contiguous()
        if products == "fft":
            lam, _ = api.solve_fft(ctx, V, b, D, L, tol=tol, restart=restart, max_iter=20 * restart, transpose=True)
        else:
            lam, _ = api.solve_adjoint(ctx, V, b, D, L, tol=tol, restart=restart, max_iter=20 * restart)
        dxy, dal = api.grad(ctx, mesh, K, y_star, g, w, lam)
        vdev, adev = fctx.dev
        return dxy.to(vdev), dal.to(adev), None, None, None, None, None, None, None


def neumann_solve(ctx, vertices, alpha, y_star, T: float, n_t: int, tol: float = 1e-12, restart: int = 100,
                  products: str = "direct"):
    """w_h(vertices, alpha) for the datum of source ``y_star``; differentiable
    in ``vertices`` ((n_x, 2) float64 tensor) and ``alpha`` (0-dim float64 tensor).
    products: "direct" (block sums) or "fft" (through time FFTs) inside the
    forward and adjoint GMRES."""
    if products not in ("direct", "fft"):
        raise ValueError("products must be 'direct' or 'fft'")
    if not torch.is_tensor(alpha):
        alpha = torch.tensor(float(alpha), dtype=torch.float64)
    return _NeumannSolve.apply(vertices, alpha, ctx, tuple(y_star), float(T), int(n_t), float(tol), int(restart),
                               products)
