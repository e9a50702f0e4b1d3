"""Galerkin lag blocks of V_h, K_h, D_h and the mass matrices (oracle, FP64).

Section 1 eq. (4): with piecewise constant test/trial functions phi^0 on the
space-time elements gamma_i x tau_m and the P1-in-space / P0-in-time functions
phi^{10},

    V_h[(i,m),(j,n)] = <V phi^0_{j,n}, phi^0_{i,m}>,
    K_h[(i,m),(p,n)] = <K phi^{10}_{p,n}, phi^0_{i,m}>,
    M_h[(i,m),(p,n)] = <phi^{10}_{p,n}, phi^0_{i,m}>.

On a uniform time grid every block depends only on the lag d = m - n >= 0 (the
kernel depends on t - tau and vanishes for tau > t, which also makes the
matrices block lower triangular, Section 3).  This module returns the lag
blocks A^(d)[i][j], d = 0..N_t-1 (time-major unknowns l = m N_x + i).

Section 2 (Theorem and the choice of Y_h): D_h[l,k] = <D psi_k, psi_l> on the
dual P1 space.  Its bilinear form after integration by parts in space (the
paper cites Costabel 1990, Thm 6.1; written out here from
-d_{n_x} d_{n_y} E = (n_x . n_y) alpha d_t E + d_{t_x} d_{t_y} E for a heat
kernel E = U*/alpha, then twice integrating by parts along the closed curve):

    <D psi_k, psi_l>_d = sum_{pieces a, b} psi_l'(a) psi_k'(b) int_a int_b D2_d F_V
                       + (n_a . n_b) int_a int_b psi_l(x) psi_k(y) D2_d F_1

with psi' = d psi / ds (piecewise constant) and pieces the half-segments.

Every entry is sum over the rule's points of (weight x kernel x basis
functions), evaluated entry by entry in plain numpy (vectorised over entries of
one lag).  V^(d) and D^(d) are symmetric: entries are evaluated with the
smaller index first, so both triangles hold the identical number.

Pins: tests/test_oracle_assembly.py (brute-force adaptive quadrature of the
space integrals on tiny meshes, symmetry, invariances, K = 0 on collinear
pairs, the D_h form against the non-integrated kernel on separated supports,
positive definiteness of V_h).
"""
import math

import numpy as np

from .geometry import (ADJ_NEXT, ADJ_PREV, IDENTICAL, NEAR, REGULAR,
                       BoundaryMesh, classify)
from .quadrature import adjacent_rule, identical_rule, tensor_rule
from .rules import DEFAULT_RULES
from .timeint import lag_1, lag_Kq, lag_V


def _rule(code, d, rules):
    if d >= 2:
        return tensor_rule(rules.space_order(d))
    if code == REGULAR:
        return tensor_rule(rules.n_regular01)
    if code == NEAR:
        return tensor_rule(rules.n_near01)
    if code == IDENTICAL:
        return identical_rule(rules)
    if code == ADJ_NEXT:          # end of piece a == start of piece b
        return adjacent_rule(rules, 1.0, 0.0)
    if code == ADJ_PREV:          # start of piece a == end of piece b
        return adjacent_rule(rules, 0.0, 1.0)
    raise ValueError(code)


def pair_integrals(kind, d, mesh, A0, A1, LA, B0, B1, LB, NB, cls,
                   wa0, wa1, wb0, wb1, rules=DEFAULT_RULES, chunk=2048, magnitude=False, tfun=None,
                   keep_terms=False):
    """int_a int_b k_d(x, y) wa(x) wb(y) ds_y ds_x for arrays of piece pairs.

    kind: 'V' (D2_d F_V), 'K' (D2_d F_K, uses the trial normal NB) or '1'
    (D2_d F_1).  Pieces a: A0 -> A1 (length LA), b: B0 -> B1 (length LB).
    wa, wb are linear in the local parameters xi, eta in [0,1]:
    wa(xi) = wa0 + (wa1 - wa0) xi.
    With magnitude=True the sum of the absolute values of the point terms is
    returned instead (the scale of the rounding error of the sum).
    tfun(kind, c), if given, replaces the uniform-grid time integrals at lag
    d (lag_V, lag_Kq / q, lag_1) by another pair of time steps' integrals
    (non-uniform grids); d still selects the spatial rule.
    With keep_terms=True an object array is returned instead whose entry k
    holds pair k's point terms (times LA LB), unsummed.
    """
    n = len(cls)
    out = np.empty(n, dtype=object) if keep_terms else np.zeros(n)
    ht, alpha = mesh.ht, mesh.alpha
    codes = np.unique(cls) if d < 2 else np.array([-1])
    for code in codes:
        sel_all = np.where(cls == code)[0] if code >= 0 else np.arange(n)
        xi, eta, w, mode, p, q = _rule(code if code >= 0 else REGULAR, d, rules)
        for s in range(0, sel_all.size, chunk):
            sel = sel_all[s:s + chunk]
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
            r2 = (dx * dx).sum(-1)
            c = 0.25 * alpha * r2
            if kind not in ('V', 'K', '1'):
                raise ValueError(kind)
            if tfun is not None:
                k = tfun(kind, c)
            elif kind == 'V':
                k = lag_V(c, d, ht, alpha, rules)
            elif kind == 'K':
                k = lag_Kq(c, d, ht, alpha, rules)
            else:
                k = lag_1(c, d, ht, alpha, rules)
            if kind == 'K':
                k = (dx * NB[sel, None, :]).sum(-1) * k
            fa = wa0[sel, None] + (wa1 - wa0)[sel, None] * xi[None, :]
            fb = wb0[sel, None] + (wb1 - wb0)[sel, None] * eta[None, :]
            terms = w[None, :] * k * fa * fb
            if magnitude:
                terms = np.abs(terms)
            if keep_terms:
                for r, e in enumerate(sel):
                    out[e] = terms[r] * (LA[e] * LB[e])
            else:
                out[sel] = terms.sum(-1) * LA[sel] * LB[sel]
    return out


# --- V_h ----------------------------------------------------------------------

def V_entries(mesh: BoundaryMesh, d, I, J, rules=DEFAULT_RULES, tfun=None):
    """V^(d)[i][j] = int_{gamma_i} int_{gamma_j} D2_d F_V ds_y ds_x."""
    I, J = np.asarray(I), np.asarray(J)
    a, b = np.minimum(I, J), np.maximum(I, J)
    cls = classify(mesh.N, a, b, mesh.a, mesh.b, mesh.h, rules.near_gap_ratio)
    one = np.ones(a.shape)
    return pair_integrals('V', d, mesh, mesh.a[a], mesh.b[a], mesh.h[a],
                          mesh.a[b], mesh.b[b], mesh.h[b],
                          mesh.n[b], cls, one, one, one, one, rules, tfun=tfun)


# --- K_h ----------------------------------------------------------------------

def K_entries(mesh: BoundaryMesh, d, I, P, rules=DEFAULT_RULES, magnitude=False, tfun=None):
    """K^(d)[i][p] = sum_{j in {p-1, p}} int_{gamma_i} int_{gamma_j}
    D2_d F_K(x, y) phi_p(y) ds_y ds_x, phi_p the P1 hat at vertex p.

    magnitude=True returns the sum of the absolute values of the quadrature
    terms instead (q changes sign inside some pairs near re-entrant corners).

    On gamma_p the hat falls 1 -> 0, on gamma_{p-1} it rises 0 -> 1.  The
    identical pair (i == j) contributes exactly 0: x - y is tangential there,
    so q = (x - y) . n_y vanishes.
    """
    I, P = np.asarray(I), np.asarray(P)
    N = mesh.N
    total = np.zeros(I.shape, dtype=np.float64)
    for j, w0, w1 in (((P) % N, 1.0, 0.0), ((P - 1) % N, 0.0, 1.0)):
        keep = j != I
        ii, jj = I[keep], j[keep]
        cls = classify(N, ii, jj, mesh.a, mesh.b, mesh.h, rules.near_gap_ratio)
        one = np.ones(ii.shape)
        val = pair_integrals('K', d, mesh, mesh.a[ii], mesh.b[ii], mesh.h[ii],
                             mesh.a[jj], mesh.b[jj], mesh.h[jj], mesh.n[jj], cls,
                             one, one, w0 * one, w1 * one, rules, magnitude=magnitude, tfun=tfun)
        total[keep] += val
    return total


# --- D_h ----------------------------------------------------------------------

def _dual_tables(mesh):
    N = mesh.N
    idx = np.zeros((N, 4), dtype=np.int64)
    v0 = np.zeros((N, 4))
    v1 = np.zeros((N, 4))
    dp = np.zeros((N, 4))
    for l in range(N):
        for k, (p, a, b, s) in enumerate(mesh.dual_pieces(l)):
            idx[l, k], v0[l, k], v1[l, k], dp[l, k] = p, a, b, s
    return idx, v0, v1, dp


def D_entries(mesh: BoundaryMesh, d, L, K, rules=DEFAULT_RULES, magnitude=False, tfun=None, exact=False):
    """D^(d)[l][k] = <D psi_k, psi_l> at lag d (form written above).

    magnitude=True returns S = sum over pieces and quadrature points of the
    absolute values of the terms of the sum, the scale against which rounding
    in any evaluation order of this signed sum is measured.  exact=True sums
    all point terms of each entry (both terms of the form, all 16 piece pairs)
    with math.fsum, i.e. exactly rounded: only the rounding of the terms
    themselves remains, so any other evaluation order can be measured against
    it in units of eps S."""
    L, K = np.asarray(L), np.asarray(K)
    lo, hi = np.minimum(L, K), np.maximum(L, K)
    idx, v0, v1, dp = _dual_tables(mesh)
    E = lo.size
    rows_a, rows_b, e_of = [], [], []
    for ia in range(4):
        for ib in range(4):
            rows_a.append(np.stack([lo, np.full(E, ia)], 1))
            rows_b.append(np.stack([hi, np.full(E, ib)], 1))
            e_of.append(np.arange(E))
    ra = np.concatenate(rows_a)
    rb = np.concatenate(rows_b)
    eo = np.concatenate(e_of)
    pa = idx[ra[:, 0], ra[:, 1]]
    pb = idx[rb[:, 0], rb[:, 1]]
    cls = classify(2 * mesh.N, pa, pb, mesh.hs0, mesh.hs1, mesh.hs_len,
                   rules.near_gap_ratio)
    one = np.ones(pa.shape)
    A0, A1, LA = mesh.hs0[pa], mesh.hs1[pa], mesh.hs_len[pa]
    B0, B1, LB = mesh.hs0[pb], mesh.hs1[pb], mesh.hs_len[pb]
    NB = mesh.hs_n[pb]
    IV = pair_integrals('V', d, mesh, A0, A1, LA, B0, B1, LB, NB, cls,
                        one, one, one, one, rules, magnitude=magnitude, tfun=tfun, keep_terms=exact)
    I1 = pair_integrals('1', d, mesh, A0, A1, LA, B0, B1, LB, NB, cls,
                        v0[ra[:, 0], ra[:, 1]], v1[ra[:, 0], ra[:, 1]],
                        v0[rb[:, 0], rb[:, 1]], v1[rb[:, 0], rb[:, 1]], rules, magnitude=magnitude,
                        tfun=tfun, keep_terms=exact)
    curl = dp[ra[:, 0], ra[:, 1]] * dp[rb[:, 0], rb[:, 1]]
    nn = (mesh.hs_n[pa] * mesh.hs_n[pb]).sum(-1)
    if magnitude:
        curl, nn = np.abs(curl), np.abs(nn)
    if exact:
        parts = [[] for _ in range(E)]
        for r in range(eo.size):
            parts[eo[r]].append(curl[r] * IV[r])
            parts[eo[r]].append(nn[r] * I1[r])
        return np.array([math.fsum(np.concatenate(p)) for p in parts])
    contrib = curl * IV + nn * I1
    out = np.zeros(E)
    np.add.at(out, eo, contrib)
    return out


# --- whole operators ------------------------------------------------------------

def _all_pairs(N, symmetric):
    if symmetric:
        I, J = np.triu_indices(N)
    else:
        I, J = np.indices((N, N))
        I, J = I.ravel(), J.ravel()
    return I, J


def assemble(op: str, mesh: BoundaryMesh, rules=DEFAULT_RULES, lags=None, magnitude=False, exact=False):
    """Lag blocks A[d][i][j] (N_t x N_x x N_x) of op in {'V', 'K', 'D'}.

    magnitude=True (K and D) returns the term-magnitude sums S instead;
    exact=True (D) the exactly summed entries of D_entries."""
    N = mesh.N
    lags = range(mesh.n_t) if lags is None else lags
    sym = op in ('V', 'D')
    I, J = _all_pairs(N, sym)
    fn = {'V': V_entries, 'K': K_entries, 'D': D_entries}[op]
    out = np.zeros((len(list(lags)), N, N))
    for k, d in enumerate(lags):
        if magnitude:
            vals = fn(mesh, d, I, J, rules, magnitude=True)
        elif exact:
            vals = fn(mesh, d, I, J, rules, exact=True)
        else:
            vals = fn(mesh, d, I, J, rules)
        out[k, I, J] = vals
        if sym:
            out[k, J, I] = vals
    return out


# --- mass matrices --------------------------------------------------------------

def half_mass_apply(mesh: BoundaryMesh, g):
    """(1/2 M_h g)[m][i] with M_h[(i,m),(p,m)] = ht h_i / 2 for p in {i, i+1}.

    M_h = <phi^{10}_p, phi^0_i> (Section 1) is block diagonal in time; each P1
    hat integrates to h_i / 2 over either segment it touches.
    """
    g = np.asarray(g)
    return 0.5 * mesh.ht * 0.5 * mesh.h * (g + np.roll(g, -1, axis=-1))


def lumped_dual_mass(mesh: BoundaryMesh):
    """Row sums of the mixed mass M_h[l,k] = <phi^0_k, psi_l> (Section 2),
    L_l = ht int psi_l ds = ht (h_{l-1} + 2 h_l + h_{l+1}) / 4 (Section 4,
    "lumped mass matrix")."""
    h = mesh.h
    return mesh.ht * (np.roll(h, 1) + 2.0 * h + np.roll(h, -1)) / 4.0


def mixed_mass_matrix(mesh: BoundaryMesh):
    """The consistent mixed mass M_h[l, k] = <phi0_k, psi_l> of one time step
    (Section 2; the time factor is ht): psi_l is linear on each of its four
    half-segments (dual_pieces), so its integral over the part of gamma_k it
    covers is the trapezoid (value at start + value at end) / 2 x length.
    Row l has entries at k = l - 1, l, l + 1 (cyclic); its row sums are the
    lumped masses of lumped_dual_mass."""
    N = mesh.N
    M = np.zeros((N, N))
    for l in range(N):
        for piece, v0, v1, _ in mesh.dual_pieces(l):
            k = mesh.hs_seg[piece]
            M[l, k] += 0.5 * (v0 + v1) * mesh.hs_len[piece]
    return mesh.ht * M
