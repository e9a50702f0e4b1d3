"""Boundary mesh Gamma_h, dual pieces and pair classes (oracle).

Section 1 (tensor-product decomposition): Gamma_h = {gamma_i}, i = 0..N_x-1,
segment gamma_i runs from vertex x_i to x_{i+1} (indices mod N_x, vertices
counter-clockwise) with length h_i, unit tangent t_i and outward unit normal
n_i = (t_i,y, -t_i,x).

Section 2 (dual mesh, space Y_h): each dual basis function psi_l is the
piecewise linear hat, in arc length, with value 1 at the midpoint m_l of
gamma_l and support [m_{l-1}, m_{l+1}].  It is linear on each of its four
half-segments: the ring of half-segments has piece 2i = [x_i, m_i] and piece
2i+1 = [m_i, x_{i+1}]; psi_l lives on pieces 2l-1 .. 2l+2.

Pair classes (the rule's switch): identical, adjacent through the next /
previous shared endpoint, near (ring distance 2, or a gap below
``near_gap_ratio`` times the longer piece), regular.
"""
import numpy as np

REGULAR, NEAR, IDENTICAL, ADJ_NEXT, ADJ_PREV = 0, 1, 2, 3, 4


class BoundaryMesh:
    """Polygon boundary mesh plus its half-segment ring (all float64)."""

    def __init__(self, vertices, T: float, n_t: int, alpha: float):
        X = np.asarray(vertices, dtype=np.float64)
        if X.ndim != 2 or X.shape[1] != 2 or X.shape[0] < 3:
            raise ValueError("need an (N_x >= 3, 2) vertex array")
        if not (T > 0 and n_t >= 1 and alpha > 0):
            raise ValueError("need T > 0, n_t >= 1, alpha > 0")
        self.X = X
        self.N = X.shape[0]
        self.a = X
        self.b = np.roll(X, -1, axis=0)
        e = self.b - self.a
        self.h = np.sqrt((e * e).sum(1))
        if np.any(self.h <= 0):
            raise ValueError("zero-length segment")
        area2 = np.sum(self.a[:, 0] * self.b[:, 1] - self.b[:, 0] * self.a[:, 1])
        if area2 <= 0:
            raise ValueError("vertices must be counter-clockwise")
        self.t = e / self.h[:, None]
        self.n = np.stack([self.t[:, 1], -self.t[:, 0]], axis=1)
        self.mid = 0.5 * (self.a + self.b)
        self.T = float(T)
        self.n_t = int(n_t)
        self.ht = self.T / self.n_t
        self.alpha = float(alpha)
        # half-segment ring
        N = self.N
        hs0 = np.empty((2 * N, 2))
        hs1 = np.empty((2 * N, 2))
        hs0[0::2], hs1[0::2] = self.a, self.mid
        hs0[1::2], hs1[1::2] = self.mid, self.b
        self.hs0, self.hs1 = hs0, hs1
        self.hs_len = np.repeat(0.5 * self.h, 2)
        self.hs_seg = np.repeat(np.arange(N), 2)
        self.hs_n = self.n[self.hs_seg]

    # ---- dual basis data (Section 2) --------------------------------------
    def dual_pieces(self, l: int):
        """Pieces of psi_l: list of (half-segment index, value at start,
        value at end, d psi / ds) for the four half-segments 2l-1 .. 2l+2."""
        N = self.N
        hm, h0, hp = self.h[(l - 1) % N], self.h[l], self.h[(l + 1) % N]
        a_l = hm / (hm + h0)
        b_l = hp / (h0 + hp)
        up = 2.0 / (hm + h0)
        dn = -2.0 / (h0 + hp)
        M = 2 * N
        return [((2 * l - 1) % M, 0.0, a_l, up),
                ((2 * l) % M, a_l, 1.0, up),
                ((2 * l + 1) % M, 1.0, b_l, dn),
                ((2 * l + 2) % M, b_l, 0.0, dn)]


def _point_seg_dist(p, s0, s1):
    e = s1 - s0
    L2 = (e * e).sum(-1)
    tt = np.clip(((p - s0) * e).sum(-1) / L2, 0.0, 1.0)
    q = s0 + tt[..., None] * e
    return np.sqrt(((p - q) ** 2).sum(-1))


def classify(ring_len, ia, ib, p0, p1, lens, near_gap_ratio):
    """Pair classes for pieces ia, ib of a closed ring of ``ring_len`` pieces.

    Piece k runs p0[k] -> p1[k] and p1[k] == p0[k+1].  Identical and adjacent
    classes follow the ring topology; near = ring distance 2 or a geometric gap
    below ``near_gap_ratio`` times the longer piece (ring distance >= 3).
    """
    ia = np.asarray(ia)
    ib = np.asarray(ib)
    cls = np.full(ia.shape, REGULAR, dtype=np.int64)
    diff = (ib - ia) % ring_len
    cls[diff == 0] = IDENTICAL
    cls[(diff == 1) & (diff != 0)] = ADJ_NEXT
    cls[(diff == ring_len - 1) & (diff != 0) & (diff != 1)] = ADJ_PREV
    ringd = np.minimum(diff, ring_len - diff)
    cls[(ringd == 2) & (cls == REGULAR)] = NEAR
    far = (ringd >= 3)
    if np.any(far):
        A0, A1, B0, B1 = p0[ia[far]], p1[ia[far]], p0[ib[far]], p1[ib[far]]
        gap = np.minimum.reduce([_point_seg_dist(A0, B0, B1), _point_seg_dist(A1, B0, B1),
                                 _point_seg_dist(B0, A0, A1), _point_seg_dist(B1, A0, A1)])
        lmax = np.maximum(lens[ia[far]], lens[ib[far]])
        sub = np.where(far)[0]
        cls[sub[gap < near_gap_ratio * lmax]] = NEAR
    return cls
