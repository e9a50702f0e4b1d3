"""Block-Toeplitz products and solvers for the oracle (FP64, numpy).

Section 3: the matrices are block lower triangular in time; on a uniform grid
the block (m, n) is the lag block A^(m-n).  Vectors are (N_t, N_x) arrays,
x[n][j].

* ``toeplitz_apply``: y[m] = sum_{d=0}^{m} A^(d) x[m-d]  (one library matmul
  per lag);  transpose: y[n] = sum_d A^(d)^T x[n+d] (backward in time).
* ``forward_substitution``: the exact solution of V_h w = f, solving the
  lag-0 block once per step: w_m = V^(0)^{-1} (f_m - sum_{d>=1} V^(d) w_{m-d}).
  V_h is positive definite (Section 1), so V^(0) is invertible.
* ``gmres``: right-preconditioned GMRES (Section 2; the paper fixes only the
  relative precision 1e-8, Section 4), x0 = 0, modified Gram-Schmidt and Givens
  rotations, restarted after ``restart`` steps; stops when the true relative
  residual ||f - A x|| / ||f|| (which right preconditioning minimises) is below
  ``tol``.

Pins: tests/test_oracle_solve.py (Toeplitz product against the dense block
matrix, forward substitution against a dense solve, GMRES against both).
"""
import numpy as np
import scipy.linalg as sla


def toeplitz_apply(A, x, transpose=False):
    A = np.asarray(A)
    x = np.asarray(x)
    nt = x.shape[0]
    y = np.zeros((nt, A.shape[1] if not transpose else A.shape[2]))
    for d in range(min(nt, A.shape[0])):
        if not transpose:
            y[d:] += x[:nt - d] @ A[d].T
        else:
            y[:nt - d] += x[d:] @ A[d]
    return y


def dense(A, nt=None):
    """The full block lower-triangular matrix (time-major unknowns)."""
    nt = A.shape[0] if nt is None else nt
    n1, n2 = A.shape[1], A.shape[2]
    M = np.zeros((nt * n1, nt * n2))
    for m in range(nt):
        for n in range(m + 1):
            M[m * n1:(m + 1) * n1, n * n2:(n + 1) * n2] = A[m - n]
    return M


def forward_substitution(V, f):
    nt = f.shape[0]
    lu = sla.lu_factor(V[0])
    w = np.zeros_like(f)
    for m in range(nt):
        rhs = f[m].copy()
        for d in range(1, m + 1):
            rhs -= V[d] @ w[m - d]
        w[m] = sla.lu_solve(lu, rhs)
    return w


def gmres(apply_A, f, apply_M=None, tol=1e-8, maxit=500, restart=200):
    """Right-preconditioned GMRES for A x = f; returns (x, iters, res_hist)."""
    shape = f.shape
    b = f.ravel()
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    A = lambda v: apply_A(v.reshape(shape)).ravel()                    # noqa: E731
    M = (lambda v: v) if apply_M is None else (lambda v: apply_M(v.reshape(shape)).ravel())  # noqa: E731
    hist = [1.0]
    it = 0
    if nb == 0:
        return x.reshape(shape), 0, hist
    while it < maxit:
        r = b - A(x)
        beta = np.linalg.norm(r)
        if beta / nb <= tol:
            break
        m = restart
        Q = np.zeros((m + 1, b.size))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        Q[0] = r / beta
        k_done = 0
        for k in range(m):
            z = M(Q[k])
            v = A(z)
            for i in range(k + 1):
                H[i, k] = Q[i] @ v
                v = v - H[i, k] * Q[i]
            H[k + 1, k] = np.linalg.norm(v)
            if H[k + 1, k] > 0:
                Q[k + 1] = v / H[k + 1, k]
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            k_done = k + 1
            hist.append(abs(g[k + 1]) / nb)
            if abs(g[k + 1]) / nb <= tol or it >= maxit:
                break
        y = sla.solve_triangular(H[:k_done, :k_done], g[:k_done])
        x = x + M(Q[:k_done].T @ y)
        if hist[-1] <= tol:
            break
    return x.reshape(shape), it, hist
