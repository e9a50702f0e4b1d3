"""Shape and alpha derivatives of the discrete system, and the gradient of a
loss on w_h by the adjoint method (oracle, FP64, test infrastructure).

The paper solves V_h w = f, f = (1/2 M_h + K_h) g (Section 1, eq. (4)), for one
boundary Gamma_h; it does not differentiate.  The parameters here are the
polygon vertices x_k (2 N_x coordinates) and the diffusion coefficient alpha.
For L(theta) = ||w_h - w_target||^2 (sum over all coefficients):

    V_h^T lambda = dL/dw = 2 (w_h - w_target)              (adjoint; V_h^T is
                                                            block upper triangular,
                                                            so it runs backward in time)
    dL/dtheta = lambda^T (df/dtheta - (dV_h/dtheta) w_h),
    lambda^T (dA/dtheta) x = sum_d sum_ij C_ij(d) dA^(d)_ij/dtheta,
    C_ij(d) = sum_m lambda[m][i] x[m-d][j]                  (A = V_h with x = w_h,
                                                            A = K_h with x = g).

Every entry of V_h and K_h is a fixed quadrature rule in the local parameters
(xi, eta) of two segments (oracle.assembly), so its derivative is the same rule
applied to the derivative of the integrand.  Per rule point x - y is linear in
the four segment endpoints P_r, x - y = sum_r c_r P_r with fixed c_r(xi, eta)
(for the singular rules written from the rule's own offsets, so that shared
endpoints combine exactly), hence

    d r^2 / dP_r = 2 c_r (x - y),   dc/dP_r = (alpha/2) c_r (x - y),
    dc/dalpha = r^2 / 4,            d h_a / dA1 = -d h_a / dA0 = t_a,
    q = (x - y) . n_b:  dq/dP_r = c_r n_b + (P_r = B0: +, B1: -) ((x - y) . t_b / h_b) n_b,

and the lag kernels enter through their c-derivatives (oracle.timeint.dlag_*);
lag_Kq is proportional to alpha at fixed c.  f adds the derivatives of the
mass matrix (h_i) and of the manufactured datum g (x_p and alpha).

Pins: tests/test_oracle_gradient.py -- every entry derivative against central
differences of the oracle's own entries, and the loss gradient against central
differences of the oracle's loss (exact forward substitution) in random
directions.
"""
import numpy as np
import scipy.linalg as sla

from .assembly import assemble, half_mass_apply
from .geometry import BoundaryMesh, classify
from .rhs import g_vec
from .rules import DEFAULT_RULES
from .solve import forward_substitution, toeplitz_apply
from .timeint import dlag_Kq, dlag_V, lag_Kq, lag_V
from .assembly import _rule

FOUR_PI = 4.0 * np.pi


def _coefficients(mode, xi, eta, p, q):
    """(x - y, as a function of the endpoints) coefficients c_r for the roles
    A0, A1, B0, B1, shape (4, n_points)."""
    z = np.zeros_like(xi)
    if mode == 'T':          # x - y = (A0 - B0) + xi (A1 - A0) - eta (B1 - B0)
        return np.stack([1.0 - xi, xi, -(1.0 - eta), -eta])
    if mode == 'S':          # x - y = p (A1 - A0), p = xi - eta (same segment)
        return np.stack([-p, p, z, z])
    if mode == 'N':          # x - y = -p (A1 - A0) - q (B1 - B0)
        return np.stack([p, -p, q, -q])
    return np.stack([-p, p, -q, q])      # 'P': x - y = p (A1 - A0) + q (B1 - B0)


def pair_grad(kind, d, mesh, ia, jb, cls, W0, W1, rules=DEFAULT_RULES):
    """Derivatives of  sum over pairs of  int_a int_b k_d (W0 (1 - eta) + W1 eta)
    ds_y ds_x  for segment pairs (ia[k], jb[k]) with per-pair weights.

    kind 'V': k = D2_d F_V; kind 'K': k = q D2_d F_Kq.  Returns
    (G, Ga): G[k, r, :] the derivative of pair k's term with respect to its
    endpoint r in (A0, A1, B0, B1) = (x_ia, x_ia+1, x_jb, x_jb+1), Ga[k] the
    derivative with respect to alpha."""
    N = mesh.N
    ia, jb = np.asarray(ia), np.asarray(jb)
    A0, A1 = mesh.a[ia], mesh.b[ia]
    B0, B1 = mesh.a[jb], mesh.b[jb]
    LA, LB = mesh.h[ia], mesh.h[jb]
    tA, tB, NB = mesh.t[ia], mesh.t[jb], mesh.n[jb]
    ht, alpha = mesh.ht, mesh.alpha
    n = ia.size
    G = np.zeros((n, 4, 2))
    Ga = np.zeros(n)
    codes = np.unique(cls) if d < 2 else np.array([-1])
    for code in codes:
        sel = np.where(cls == code)[0] if code >= 0 else np.arange(n)
        if sel.size == 0:
            continue
        xi, eta, w, mode, p, q = _rule(code if code >= 0 else 0, d, rules)
        ea = (A1 - A0)[sel, None, :]
        eb = (B1 - B0)[sel, None, :]
        if mode == 'T':
            dx = (A0 - B0)[sel, None, :] + p[None, :, None] * ea - q[None, :, None] * eb
        elif mode == 'S':
            dx = p[None, :, None] * ea
        elif mode == 'N':
            dx = -p[None, :, None] * ea - q[None, :, None] * eb
        else:
            dx = p[None, :, None] * ea + q[None, :, None] * eb
        cr = _coefficients(mode, xi, eta, p, q)                     # (4, P)
        r2 = (dx * dx).sum(-1)
        c = 0.25 * alpha * r2
        phi = W0[sel, None] * (1.0 - eta[None, :]) + W1[sel, None] * eta[None, :]
        LL = (LA * LB)[sel, None]
        if kind == 'V':
            k = lag_V(c, d, ht, alpha, rules)
            dk = dlag_V(c, d, ht, alpha, rules)
            val = (w[None, :] * phi * k).sum(-1)                      # int k phi (no lengths)
            gc = w[None, :] * phi * dk * LL                            # d/dc weight per point
            for r in range(4):
                G[sel, r, :] += 0.5 * alpha * (gc[..., None] * cr[r][None, :, None] * dx).sum(1)
            Ga[sel] += (gc * r2 * 0.25).sum(-1)
        else:
            qn = (dx * NB[sel, None, :]).sum(-1)
            k = lag_Kq(c, d, ht, alpha, rules)
            dk = dlag_Kq(c, d, ht, alpha, rules)
            val = (w[None, :] * phi * qn * k).sum(-1)
            gc = w[None, :] * phi * qn * dk * LL
            gq = w[None, :] * phi * k * LL                              # d/dq weight per point
            tau = (dx * tB[sel, None, :]).sum(-1) / LB[sel, None]        # (x - y) . t_b / h_b
            for r in range(4):
                G[sel, r, :] += 0.5 * alpha * (gc[..., None] * cr[r][None, :, None] * dx).sum(1)
                coef_q = cr[r][None, :].copy() * np.ones_like(tau)
                if r == 2:
                    coef_q = coef_q + tau
                elif r == 3:
                    coef_q = coef_q - tau
                G[sel, r, :] += (gq * coef_q).sum(-1)[:, None] * NB[sel]
            Ga[sel] += (gc * r2 * 0.25).sum(-1) + (w[None, :] * phi * qn * k * LL).sum(-1) / alpha
        # lengths: d(LA LB)
        G[sel, 0, :] -= (val * LB[sel])[:, None] * tA[sel]
        G[sel, 1, :] += (val * LB[sel])[:, None] * tA[sel]
        G[sel, 2, :] -= (val * LA[sel])[:, None] * tB[sel]
        G[sel, 3, :] += (val * LA[sel])[:, None] * tB[sel]
    return G, Ga


def _scatter(N, ia, jb, G):
    """Endpoint roles -> vertex gradient (N, 2)."""
    out = np.zeros((N, 2))
    for r, nodes in enumerate((ia, (ia + 1) % N, jb, (jb + 1) % N)):
        np.add.at(out, nodes, G[:, r, :])
    return out


def V_entry_grad(mesh, d, i, j, rules=DEFAULT_RULES):
    """Gradient of the single entry V^(d)[i][j] (vertices (N, 2), alpha)."""
    a, b = min(i, j), max(i, j)
    ia, jb = np.array([a]), np.array([b])
    cls = classify(mesh.N, ia, jb, mesh.a, mesh.b, mesh.h, rules.near_gap_ratio)
    G, Ga = pair_grad('V', d, mesh, ia, jb, cls, np.ones(1), np.ones(1), rules)
    return _scatter(mesh.N, ia, jb, G), Ga[0]


def K_entry_grad(mesh, d, i, p, rules=DEFAULT_RULES):
    """Gradient of the single entry K^(d)[i][p]."""
    N = mesh.N
    gx, ga = np.zeros((N, 2)), 0.0
    for j, w0, w1 in ((p % N, 1.0, 0.0), ((p - 1) % N, 0.0, 1.0)):
        if j == i:
            continue
        ia, jb = np.array([i]), np.array([j])
        cls = classify(N, ia, jb, mesh.a, mesh.b, mesh.h, rules.near_gap_ratio)
        G, Ga = pair_grad('K', d, mesh, ia, jb, cls, np.array([w0]), np.array([w1]), rules)
        gx += _scatter(N, ia, jb, G)
        ga += Ga[0]
    return gx, ga


def correlation(lam, x, n_lags):
    """C[d] = sum_m lam[m] x[m-d]^T (N_t x N x N)."""
    nt = lam.shape[0]
    return np.stack([lam[d:].T @ x[:nt - d] for d in range(n_lags)])


def dV_contract(mesh, C, rules=DEFAULT_RULES):
    """sum_d sum_ij C[d][i][j] dV^(d)_ij/dtheta -> (vertices (N, 2), alpha)."""
    N = mesh.N
    I, J = np.triu_indices(N)
    cls = classify(N, I, J, mesh.a, mesh.b, mesh.h, rules.near_gap_ratio)
    gx, ga = np.zeros((N, 2)), 0.0
    for d in range(C.shape[0]):
        S = np.where(I == J, C[d][I, J], C[d][I, J] + C[d][J, I])   # V^(d) is symmetric
        G, Ga = pair_grad('V', d, mesh, I, J, cls, S, S, rules)
        gx += _scatter(N, I, J, G)
        ga += Ga.sum()
    return gx, ga


def dK_contract(mesh, C, rules=DEFAULT_RULES):
    """sum_d sum_ip C[d][i][p] dK^(d)_ip/dtheta (K_ip sums the trial segments
    p (hat falling) and p - 1 (hat rising); the pair (i, i) is identically 0)."""
    N = mesh.N
    I, J = np.indices((N, N))
    I, J = I.ravel(), J.ravel()
    keep = I != J
    I, J = I[keep], J[keep]
    cls = classify(N, I, J, mesh.a, mesh.b, mesh.h, rules.near_gap_ratio)
    gx, ga = np.zeros((N, 2)), 0.0
    for d in range(C.shape[0]):
        G, Ga = pair_grad('K', d, mesh, I, J, cls, C[d][I, J], C[d][I, (J + 1) % N], rules)
        gx += _scatter(N, I, J, G)
        ga += Ga.sum()
    return gx, ga


def g_grad(mesh, y_star, gbar):
    """sum_{n,p} gbar[n][p] dg[n][p]/dtheta for the time averages of
    U*(x_p - y*, t) (oracle.rhs.g_vec): with a_p = alpha |x_p - y*|^2 / 4,
    dg/da = alpha/(4 pi ht) (e^{-a/t_n} - e^{-a/t_{n+1}}) / a."""
    ys = np.asarray(y_star, dtype=np.float64)
    rho = mesh.X - ys
    a = mesh.alpha * (rho * rho).sum(1) / 4.0
    t = np.arange(mesh.n_t + 1) * mesh.ht
    with np.errstate(divide='ignore', over='ignore'):
        ex = np.where(t[:, None] > 0, np.exp(-a[None, :] / np.where(t[:, None] > 0, t[:, None], 1.0)), 0.0)
    dg_da = mesh.alpha / (FOUR_PI * mesh.ht) * (ex[:-1] - ex[1:]) / a[None, :]
    s = (gbar * dg_da).sum(0)                                          # per vertex
    gx = (s * 0.5 * mesh.alpha)[:, None] * rho
    g = g_vec(mesh, ys)
    ga = (gbar * g).sum() / mesh.alpha + (s * (rho * rho).sum(1) / 4.0).sum()
    return gx, ga


def mass_grad(mesh, lam, g):
    """lambda^T (1/2 dM_h/dtheta) g with (1/2 M_h g)[m][i] = ht h_i (g_i + g_{i+1}) / 4."""
    N = mesh.N
    s = (lam * 0.25 * mesh.ht * (g + np.roll(g, -1, axis=-1))).sum(0)  # per segment, times dh_i
    gx = np.zeros((N, 2))
    np.add.at(gx, (np.arange(N) + 1) % N, s[:, None] * mesh.t)
    np.add.at(gx, np.arange(N), -s[:, None] * mesh.t)
    return gx


def half_mass_transpose(mesh, lam):
    """(1/2 M_h)^T lambda: [m][p] = ht (h_p lam_p + h_{p-1} lam_{p-1}) / 4."""
    hl = mesh.h * lam
    return 0.25 * mesh.ht * (hl + np.roll(hl, 1, axis=-1))


def backward_substitution(V, b):
    """Solve V_h^T lam = b: lam_m = V^(0)^{-T} (b_m - sum_{d>=1} V^(d)^T lam_{m+d}),
    m from the last step down (V_h^T is block upper triangular)."""
    nt = b.shape[0]
    lu = sla.lu_factor(V[0].T)
    lam = np.zeros_like(b)
    for m in range(nt - 1, -1, -1):
        rhs = b[m].copy()
        for d in range(1, nt - m):
            rhs -= V[d].T @ lam[m + d]
        lam[m] = sla.lu_solve(lu, rhs)
    return lam


def solve_w(mesh, y_star, rules=DEFAULT_RULES):
    """(w_h, V, K, g) for the manufactured datum at source y*."""
    V = assemble('V', mesh, rules)
    K = assemble('K', mesh, rules)
    g = g_vec(mesh, y_star)
    f = half_mass_apply(mesh, g) + toeplitz_apply(K, g)
    return forward_substitution(V, f), V, K, g


def loss(vertices, T, n_t, alpha, y_star, w_target, rules=DEFAULT_RULES):
    mesh = BoundaryMesh(vertices, T, n_t, alpha)
    w = solve_w(mesh, y_star, rules)[0]
    return float(((w - w_target) ** 2).sum())


def loss_grad(vertices, T, n_t, alpha, y_star, w_target, rules=DEFAULT_RULES):
    """(L, dL/dvertices (N, 2), dL/dalpha) by the adjoint method."""
    mesh = BoundaryMesh(vertices, T, n_t, alpha)
    w, V, K, g = solve_w(mesh, y_star, rules)
    r = w - w_target
    lam = backward_substitution(V, 2.0 * r)
    CV = correlation(lam, w, n_t)
    CK = correlation(lam, g, n_t)
    gv, av = dV_contract(mesh, CV, rules)
    gk, ak = dK_contract(mesh, CK, rules)
    gbar = half_mass_transpose(mesh, lam) + toeplitz_apply(K, lam, transpose=True)
    gg, ag = g_grad(mesh, y_star, gbar)
    gm = mass_grad(mesh, lam, g)
    return float((r * r).sum()), gk + gg + gm - gv, ak + ag - av
