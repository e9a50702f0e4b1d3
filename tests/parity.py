"""Shared comparison helpers for GPU-vs-oracle parity tests."""
import numpy as np


def lag_rel_err(A, B, floor=1e-6):
    """max over entries of |A - B| / max(|B|, floor * max|B^(d)|), per lag block.

    The floor keeps entries that underflow or sit at a zero of the kernel from
    dominating: far pairs at small lags are e^{-z}-small (z up to ~700)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = []
    for d in range(B.shape[0]):
        den = np.maximum(np.abs(B[d]), floor * np.abs(B[d]).max())
        den = np.where(den > 0, den, 1.0)
        out.append((np.abs(A[d] - B[d]) / den).max())
    return np.array(out)


def k_structural_zeros(om, tol=1e-12):
    """(i, p) of K whose trial support (segments p-1, p, minus i itself) is
    collinear with the test segment i: there q = (x - y) . n_y vanishes
    identically, so both sides compute rounding noise (|K| ~ eps max|K|)."""
    N = om.N
    cr = lambda a, b: a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]   # noqa: E731
    mask = np.zeros((N, N), dtype=bool)
    for i in range(N):
        for p in range(N):
            js = [j for j in (p, (p - 1) % N) if j != i]
            mask[i, p] = all(abs(cr(om.t[i], om.t[j])) < tol and
                             abs(cr(om.t[i], om.a[j] - om.a[i])) < tol * om.h[i] for j in js)
    return mask


def k_rel_err(A, B, om, floor=1e-6, zero_tol=1e-14):
    """lag_rel_err for K with the structural zeros compared in absolute terms
    (|value| <= zero_tol * max|K^(d)| on both sides)."""
    mask = k_structural_zeros(om)
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = []
    for d in range(B.shape[0]):
        scale = np.abs(B[d]).max()
        if mask.any():
            assert np.abs(A[d][mask]).max() <= zero_tol * scale
            assert np.abs(B[d][mask]).max() <= zero_tol * scale
        den = np.maximum(np.abs(B[d]), floor * scale)
        den = np.where(den > 0, den, 1.0)
        e = np.abs(A[d] - B[d]) / den
        e[mask] = 0.0
        out.append(e.max())
    return np.array(out)


def d_rel_err(A, B, S, floor=1e-6, tol=1e-12, term_tol=4e-15):
    """Normalised D error: |A - B| / (tol max(|B|, floor max|B^(d)|) + term_tol S).

    A D_h entry (Section 2, integrated-by-parts form) is a signed sum of curl
    and time terms; S, the sum of the magnitudes of all its quadrature terms,
    exceeds |D| by up to ~1e6 far from the diagonal.  Any evaluation order
    rounds by ~eps S.  B is the oracle's exactly summed entry
    (assembly.D_entries(exact=True)), so |A - B| is A's own rounding: measured
    at most 4.3 eps S on the small parity meshes and 9.3 eps S on sampled
    square256 entries (eps = 2^-52), hence term_tol = 4e-15 (18 eps).  The
    entry is required to 1e-12 relative where it is well conditioned and to
    term_tol S elsewhere; the returned value is <= 1 when both hold jointly."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    out = []
    for d in range(B.shape[0]):
        den = tol * np.maximum(np.abs(B[d]), floor * np.abs(B[d]).max()) + term_tol * S[d]
        den = np.where(den > 0, den, 1.0)
        out.append((np.abs(A[d] - B[d]) / den).max())
    return np.array(out)
