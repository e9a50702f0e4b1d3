"""Non-uniform time grids (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 1 allows any decomposition I_h = {tau_k} of (0, T).  With time nodes
0 = t_0 < t_1 < ... < t_{N_t} = T (steps h_k = t_{k+1} - t_k) the Galerkin
blocks A[m][n] (test step m, trial step n <= m) depend on (m, n), not on the
lag m - n alone: the matrices stay block lower triangular (the kernel vanishes
for tau > t) but are no longer block Toeplitz, so all N_t (N_t + 1) / 2 blocks
are assembled and stored.

Time.  For a kernel G with second antiderivative F (oracle.timeint: F_V, F_Kq,
F_1; F = 0 for s <= 0)

    int_{tau_m} int_{tau_n} G(t - tau) dtau dt = F(s1) - F(s2) - F(s3) + F(s4),
    s1 = t_{m+1} - t_n, s2 = t_{m+1} - t_{n+1}, s3 = t_m - t_n, s4 = t_m - t_{n+1},

which on a uniform grid is the second difference of oracle.timeint.  The
evaluation branches reduce to oracle.timeint's there (d = m - n, and the
centre separation s_c = (s1 + s4) / 2 = d ht):
* d = 0: F(h_m);
* d = 1: with z = c / s_c < 1, the closed form with its ln c terms cancelled
  analytically (E1 = -gamma - ln z + Ein(z), E2 = e^{-z} - z E1, and
  s1 - s2 - s3 = 0 exactly); z >= 1: the closed form;
* d >= 2: the closed form when c / s_c > d / 2, else the Peano form
  int w(s) G(s) ds, w(s) = |tau_m cap (tau_n + s)| the overlap length, a
  trapezoid on [s4, s1] with breaks at min(s2, s3) and max(s2, s3): up to
  three linear pieces, each with peano_order(k) Gauss nodes,
  k = round(start / length) (the interval index on a uniform grid).
Space: the uniform rule with the lag d = m - n (classes and orders).

The rule assumes neighbouring steps within a modest ratio (graded grids):
against nested quadrature it is exact to rounding (2e-14) for step ratios up
to 4 and 2e-9 at ratio 8, where a piece starts much closer to s = 0 than its
length and would need more nodes than peano_order gives.

Pins (tests/test_oracle_nonuniform.py): on a uniform grid every block equals
the Toeplitz lag block; every branch against nested adaptive quadrature
(mpmath) of G over two unequal steps; the manufactured solution converges on
graded grids.
"""
import numpy as np

from . import assembly
from .geometry import BoundaryMesh
from .quadrature import gauss01
from .rules import DEFAULT_RULES
from .special import EULER_GAMMA, e1, ein
from .timeint import F_1, F_Kq, F_V, G_1, G_Kq, G_V

FOUR_PI = 4.0 * np.pi


def check_grid(t):
    t = np.asarray(t, dtype=np.float64)
    if t.ndim != 1 or t.size < 2 or t[0] != 0.0 or np.any(np.diff(t) <= 0):
        raise ValueError("need time nodes 0 = t_0 < t_1 < ... < t_N")
    return t


def _args(t, m, n):
    return (t[m + 1] - t[n], t[m + 1] - t[n + 1], t[m] - t[n], t[m] - t[n + 1])


def _closed(Ffun, c, s):
    out = Ffun(c, s[0])
    for sign, sk in ((-1.0, s[1]), (-1.0, s[2]), (1.0, s[3])):
        if sk > 0.0:
            out = out + sign * Ffun(c, sk)
    return out


def _peano(Gfun, c, s, rules):
    """int w(s) G(s) ds over the trapezoid of the overlap length."""
    s1, s2, s3, s4 = s
    p = [s4, min(s2, s3), max(s2, s3), s1]
    plateau = p[1] - p[0]
    c_ = np.asarray(c)[..., None]
    out = np.zeros(np.shape(c))
    for piece in range(3):
        lo, hi = p[piece], p[piece + 1]
        L = hi - lo
        if L <= 0.0:
            continue
        x, w = gauss01(rules.peano_order(int(round(lo / L))))
        if piece == 0:
            wt = x * L                    # rising: s - s4
        elif piece == 1:
            wt = np.full_like(x, plateau)
        else:
            wt = (1.0 - x) * L            # falling: s1 - s
        out = out + L * (w * wt * Gfun(c_, lo + x * L)).sum(-1)
    return out


def _d1_small(kind, c, s, alpha):
    """d = 1 (s4 = 0, s1 = s2 + s3), z = c / s_c < 1: the closed form with the
    ln c terms combined analytically."""
    s1, s2, s3 = s[0], s[1], s[2]
    sig = ((1.0, s1), (-1.0, s2), (-1.0, s3))
    if kind == 'V':
        acc = c * (EULER_GAMMA + np.log(c))
        for sg, sk in sig:
            acc = acc + sg * ((sk + c) * (np.log(sk) + ein(c / sk)) - sk * np.expm1(-c / sk))
        return acc / FOUR_PI
    if kind == 'K':
        acc = -(EULER_GAMMA + np.log(c))
        for sg, sk in sig:
            acc = acc + sg * (sk * np.expm1(-c / sk) / c - np.log(sk) - ein(c / sk))
        return alpha / (2.0 * FOUR_PI) * acc
    acc = EULER_GAMMA + np.log(c)
    for sg, sk in sig:
        acc = acc + sg * (np.log(sk) + ein(c / sk))
    return alpha / FOUR_PI * acc


def time_integral(kind, c, t, m, n, alpha, rules=DEFAULT_RULES):
    """int_{tau_m} int_{tau_n} G(t - tau) dtau dt for an array of
    c = alpha r^2 / 4 (K: divided by q), kind in {'V', 'K', '1'}."""
    if n > m:
        raise ValueError("blocks above the diagonal vanish")
    c = np.asarray(c, dtype=np.float64)
    s = _args(t, m, n)
    F = {'V': F_V, 'K': lambda cc, ss: F_Kq(cc, ss, alpha), '1': lambda cc, ss: F_1(cc, ss, alpha)}[kind]
    G = {'V': G_V, 'K': lambda cc, ss: G_Kq(cc, ss, alpha), '1': lambda cc, ss: G_1(cc, ss, alpha)}[kind]
    d = m - n
    if d == 0:
        return F(c, s[0])
    sc = 0.5 * (s[0] + s[3])
    z = c / sc
    out = np.empty_like(c)
    if d == 1:
        sm = z < 1.0
        if np.any(sm):
            out[sm] = _d1_small(kind, c[sm], s, alpha)
        if np.any(~sm):
            out[~sm] = _closed(F, c[~sm], s)
        return out
    closed = z > 0.5 * d
    if np.any(closed):
        out[closed] = _closed(F, c[closed], s)
    if np.any(~closed):
        out[~closed] = _peano(G, c[~closed], s, rules)
    return out


def assemble(op, mesh: BoundaryMesh, t, rules=DEFAULT_RULES):
    """Blocks A[m][n][i][j] (N_t x N_t x N_x x N_x, zero above the block
    diagonal) of op in {'V', 'K', 'D'} on the time grid t (N_t + 1 nodes;
    mesh.ht and mesh.n_t are not used)."""
    t = check_grid(t)
    nt = t.size - 1
    N = mesh.N
    sym = op in ('V', 'D')
    I, J = (np.triu_indices(N) if sym else tuple(x.ravel() for x in np.indices((N, N))))
    fn = {'V': assembly.V_entries, 'K': assembly.K_entries, 'D': assembly.D_entries}[op]
    out = np.zeros((nt, nt, N, N))
    for m in range(nt):
        for n in range(m + 1):
            tf = (lambda kind, c, m=m, n=n: time_integral(kind, c, t, m, n, mesh.alpha, rules))
            vals = fn(mesh, m - n, I, J, rules, tfun=tf)
            out[m, n, I, J] = vals
            if sym:
                out[m, n, J, I] = vals
    return out


def block_apply(A, x):
    """y[m] = sum_{n <= m} A[m][n] x[n]."""
    nt = A.shape[0]
    y = np.zeros((nt, A.shape[2]))
    for m in range(nt):
        for n in range(m + 1):
            y[m] += A[m, n] @ x[n]
    return y


def forward_substitution(V, f):
    """The exact solution of the block lower triangular system, step by step."""
    nt = V.shape[0]
    w = np.zeros_like(f)
    for m in range(nt):
        r = f[m] - sum(V[m, n] @ w[n] for n in range(m))
        w[m] = np.linalg.solve(V[m, m], r)
    return w


# ---- manufactured data on the grid t (u = U*(x - y*, t), u_0 = 0) ----------

def g_vec(mesh: BoundaryMesh, t, y_star):
    """g[n][p] = (1/h_n) int_{tau_n} U*(x_p - y*, t) dt (vertex time averages)."""
    t = check_grid(t)
    ys = np.asarray(y_star, dtype=np.float64)
    a = mesh.alpha * ((mesh.X - ys) ** 2).sum(1) / 4.0
    E = np.zeros((t.size, mesh.N))
    E[1:] = e1(a[None, :] / t[1:, None])
    h = np.diff(t)
    return (E[1:] - E[:-1]) * mesh.alpha / FOUR_PI / h[:, None]


def f_vec(mesh: BoundaryMesh, t, K, g):
    """f = 1/2 M_h g + K_h g with M_h block diagonal, h_m h_i / 2 per touching
    vertex on step m."""
    h = np.diff(check_grid(t))
    half_mass = 0.5 * h[:, None] * 0.5 * mesh.h[None, :] * (g + np.roll(g, -1, axis=-1))
    return half_mass + block_apply(K, g)


def w_projection(mesh: BoundaryMesh, t, y_star, n_gauss: int = 8):
    """Element averages of the exact Neumann datum over gamma_i x tau_m."""
    t = check_grid(t)
    ys = np.asarray(y_star, dtype=np.float64)
    xg, wg = gauss01(n_gauss)
    x = mesh.a[:, None, :] + xg[None, :, None] * (mesh.b - mesh.a)[:, None, :]
    dx = x - ys
    r2 = (dx * dx).sum(-1)
    qn = (dx * mesh.n[:, None, :]).sum(-1)
    a = mesh.alpha * r2 / 4.0
    ex = np.zeros((t.size,) + a.shape)
    ex[1:] = np.exp(-a[None] / t[1:, None, None])
    tint = -(mesh.alpha / (2.0 * np.pi * r2))[None] * qn[None] * (ex[1:] - ex[:-1])
    return (tint * wg[None, None, :]).sum(-1) / np.diff(t)[:, None]


def l2_rel_error(mesh: BoundaryMesh, t, w_h, w_ref):
    wt = mesh.h[None, :] * np.diff(t)[:, None]
    return np.sqrt((wt * (w_h - w_ref) ** 2).sum() / (wt * w_ref ** 2).sum())
