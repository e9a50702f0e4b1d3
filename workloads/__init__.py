"""Seeded synthetic workloads for the space-time BEM of the 2D heat equation.

This module only produces *inputs*: closed polygons (counter-clockwise vertex
lists), time-grid parameters and source points for the manufactured Dirichlet
datum.  It holds none of the method's arithmetic (no kernels, no quadrature, no
operators), so both the CPU oracle and the CUDA path may use it.

The domains follow the paper's setting of a bounded Lipschitz domain Omega in
R^2 with a polygonal boundary mesh Gamma_h and a uniform time decomposition I_h
(Section 1, the tensor-product decomposition of Sigma).  The concrete shapes and
sizes are the workloads this repository is measured on:

* ``unit_square``   -- [0,1]^2 with ``n_per_side`` equal segments per side;
* ``l_shape``       -- [0,1]^2 minus [0.5,1]^2 with seeded segment lengths;
* ``star``          -- a star polygon with seeded radii, every edge subdivided;
* ``annulus_sources`` -- seeded source points y_k outside the domain;
* ``ragged_squares``  -- seeded (N_x, N_t) pairs for a ragged batch;
* ``square_triangulation`` -- a P1 triangulation Omega_h of [0,1]^2 whose
  boundary nodes are the vertices of ``unit_square`` (for the initial datum);
* ``lshape_triangulation``  -- the same grid on the L-shape, conforming with
  ``l_shape(4 n, jitter=(1, 1))`` (equal segments).

All random draws use ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem",
    "unit_square",
    "l_shape",
    "star_corners",
    "subdivision_matrix",
    "star",
    "annulus_sources",
    "ragged_squares",
    "square_triangulation",
    "lshape_triangulation",
    "config",
    "CONFIG_NAMES",
]


@dataclass
class Problem:
    """One space-time problem: polygon vertices plus time grid and data.

    ``vertices`` is an (N_x, 2) float64 array of the polygon's vertices in
    counter-clockwise order; segment i runs from vertex i to vertex i+1 (mod
    N_x).  ``n_t`` uniform steps cover (0, T).  ``alpha`` is the heat capacity
    constant of the model problem.  ``y_star`` is the source point of the
    manufactured Dirichlet datum g = U*(x - y*, t) (u_0 = 0).
    """

    name: str
    vertices: np.ndarray
    T: float
    n_t: int
    alpha: float
    y_star: np.ndarray = field(default_factory=lambda: np.array([1.5, 1.5]))

    @property
    def n_x(self) -> int:
        return int(self.vertices.shape[0])


def _subdivide(corners: np.ndarray, counts, lengths_per_side=None) -> np.ndarray:
    """Vertices along a closed polygon given by ``corners`` (CCW).

    Side s (corner s -> corner s+1) gets ``counts[s]`` segments.  With
    ``lengths_per_side`` None the segments are equal; otherwise
    ``lengths_per_side[s]`` holds relative segment lengths (positive), which are
    rescaled so that the side keeps its exact length.
    """
    out = []
    nc = corners.shape[0]
    for s in range(nc):
        a = corners[s]
        b = corners[(s + 1) % nc]
        n = int(counts[s])
        if lengths_per_side is None:
            frac = np.arange(n, dtype=np.float64) / n
        else:
            rel = np.asarray(lengths_per_side[s], dtype=np.float64)
            cum = np.concatenate([[0.0], np.cumsum(rel)[:-1]])
            frac = cum / rel.sum()
        for f in frac:
            out.append(a + f * (b - a))
    return np.asarray(out, dtype=np.float64)


def unit_square(n_per_side: int) -> np.ndarray:
    """Vertices of [0,1]^2 with ``n_per_side`` equal segments per side (CCW)."""
    corners = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    return _subdivide(corners, [n_per_side] * 4)


def l_shape(n_x: int, seed: int = 3, jitter=(0.5, 1.5)) -> np.ndarray:
    """[0,1]^2 minus [0.5,1]^2 with ``n_x`` segments of seeded lengths.

    Sides of length 1 get n_x/4 segments and sides of length 0.5 get n_x/8
    (n_x must be a multiple of 8).  Relative lengths are drawn uniformly in
    ``jitter`` times the nominal length, then each side is rescaled to its
    exact length.
    """
    if n_x % 8:
        raise ValueError("l_shape needs n_x divisible by 8")
    corners = np.array(
        [[0.0, 0.0], [1.0, 0.0], [1.0, 0.5], [0.5, 0.5], [0.5, 1.0], [0.0, 1.0]]
    )
    side_len = [1.0, 0.5, 0.5, 0.5, 0.5, 1.0]
    counts = [n_x // 4 if L == 1.0 else n_x // 8 for L in side_len]
    rng = np.random.default_rng(seed)
    rel = [rng.uniform(jitter[0], jitter[1], size=c) for c in counts]
    return _subdivide(corners, counts, rel)


def star(n_vertices: int = 16, seg_per_edge: int = 16, seed: int = 5,
         radii_range=(0.6, 1.0), center=(0.5, 0.5), radii=None) -> np.ndarray:
    """Star polygon: vertex k at angle 2*pi*k/n_vertices and a seeded radius.

    Every edge between consecutive star vertices is split into
    ``seg_per_edge`` equal segments.  ``radii`` overrides the seeded draw.
    """
    if radii is None:
        rng = np.random.default_rng(seed)
        radii = rng.uniform(radii_range[0], radii_range[1], size=n_vertices)
    radii = np.asarray(radii, dtype=np.float64)
    ang = 2.0 * np.pi * np.arange(n_vertices) / n_vertices
    c = np.asarray(center, dtype=np.float64)
    corners = c + radii[:, None] * np.stack([np.cos(ang), np.sin(ang)], axis=1)
    return _subdivide(corners, [seg_per_edge] * n_vertices)


def star_corners(n_vertices: int = 16, seed: int = 5, radii_range=(0.6, 1.0), center=(0.5, 0.5),
                 radii=None) -> np.ndarray:
    """The ``n_vertices`` corners of ``star`` (same seeded radii)."""
    if radii is None:
        rng = np.random.default_rng(seed)
        radii = rng.uniform(radii_range[0], radii_range[1], size=n_vertices)
    radii = np.asarray(radii, dtype=np.float64)
    ang = 2.0 * np.pi * np.arange(n_vertices) / n_vertices
    c = np.asarray(center, dtype=np.float64)
    return c + radii[:, None] * np.stack([np.cos(ang), np.sin(ang)], axis=1)


def subdivision_matrix(n_corners: int, seg_per_edge: int) -> np.ndarray:
    """S (n_corners seg_per_edge x n_corners) with vertices = S @ corners for
    the equal subdivision of every edge (as ``star``)."""
    S = np.zeros((n_corners * seg_per_edge, n_corners))
    for s in range(n_corners):
        for k in range(seg_per_edge):
            f = k / seg_per_edge
            S[s * seg_per_edge + k, s] += 1.0 - f
            S[s * seg_per_edge + k, (s + 1) % n_corners] += f
    return S


def annulus_sources(n: int, seed: int = 4, r_in: float = 1.2, r_out: float = 3.0,
                    center=(0.5, 0.5)) -> np.ndarray:
    """``n`` source points uniform (in area) on r_in < |y - center| < r_out."""
    rng = np.random.default_rng(seed)
    rad = np.sqrt(rng.uniform(r_in * r_in, r_out * r_out, size=n))
    th = rng.uniform(0.0, 2.0 * np.pi, size=n)
    c = np.asarray(center, dtype=np.float64)
    return c + rad[:, None] * np.stack([np.cos(th), np.sin(th)], axis=1)


def ragged_squares(n_problems: int = 64, seed: int = 41, k_range=(16, 128),
                   nt_range=(64, 512)):
    """Seeded (N_x, N_t) pairs: N_x = 4k with k uniform in ``k_range``."""
    rng = np.random.default_rng(seed)
    ks = rng.integers(k_range[0], k_range[1] + 1, size=n_problems)
    nts = rng.integers(nt_range[0], nt_range[1] + 1, size=n_problems)
    return [(int(4 * k), int(nt)) for k, nt in zip(ks, nts)]


def square_triangulation(n_per_side: int, jitter: float = 0.0, seed: int = 7):
    """Triangulation of [0,1]^2: (n+1)^2 grid nodes, 2 n^2 triangles.

    Node (k, l) sits at (k/n, l/n), index l (n+1) + k.  Cell (k, l) is split
    along its diagonal from (k, l) to (k+1, l+1); both triangles are listed
    counter-clockwise.  With ``jitter`` > 0 every interior node moves by a
    seeded uniform offset of at most ``jitter`` / n per coordinate (jitter <
    0.5 keeps every triangle positively oriented).  The boundary nodes are the
    vertices of ``unit_square(n)`` (equal up to rounding of the side
    parametrisation).  Returns (nodes (M, 2) float64, tris (2 n^2, 3) int64).
    """
    n = int(n_per_side)
    g = np.arange(n + 1, dtype=np.float64) / n
    X, Y = np.meshgrid(g, g)            # X[l, k] = k/n, Y[l, k] = l/n
    nodes = np.stack([X.ravel(), Y.ravel()], axis=1)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        inner = (X.ravel() > 0) & (X.ravel() < 1) & (Y.ravel() > 0) & (Y.ravel() < 1)
        off = rng.uniform(-jitter / n, jitter / n, size=(int(inner.sum()), 2))
        nodes[inner] += off
    tris = []
    for l in range(n):
        for k in range(n):
            p00 = l * (n + 1) + k
            p10, p01, p11 = p00 + 1, p00 + n + 1, p00 + n + 2
            tris.append((p00, p10, p11))
            tris.append((p00, p11, p01))
    return nodes, np.asarray(tris, dtype=np.int64)


def lshape_triangulation(n_per_unit: int):
    """Triangulation of [0,1]^2 minus [0.5,1]^2 on the grid of spacing 1/n
    (n even): the cells of ``square_triangulation(n)`` outside the removed
    quadrant, with the unused nodes dropped.  Its boundary nodes are the
    vertices of ``l_shape(4 n, jitter=(1, 1))``.  Returns (nodes, tris)."""
    n = int(n_per_unit)
    if n % 2:
        raise ValueError("lshape_triangulation needs an even n")
    nodes, tris = square_triangulation(n)
    keep = []
    for l in range(n):
        for k in range(n):
            if not (k >= n // 2 and l >= n // 2):
                c = 2 * (l * n + k)
                keep += [c, c + 1]
    tris = tris[keep]
    used = np.unique(tris)
    remap = -np.ones(nodes.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.size)
    return nodes[used], remap[tris]


CONFIG_NAMES = ("square32", "square64", "square256", "lshape1024", "square512", "star256")


def config(name: str) -> Problem:
    """Named workloads (sizes of the measured configurations).

    * ``square32``   unit square, N_x = 32 (8 per side), N_t = 32, T = 1, alpha = 1
    * ``square64``   unit square, N_x = 64, N_t = 64 (small profiling case)
    * ``square256``  unit square, N_x = 256, N_t = 256, T = 1, alpha = 1
    * ``lshape1024`` L-shape, N_x = 1024 (seeded lengths, seed 3), N_t = 1024, alpha = 0.5
    * ``square512``  unit square, N_x = 512, N_t = 512, alpha = 1
    * ``star256``    16-vertex star (seed 5), N_x = 256, N_t = 256, alpha = 1
    Tiny variants for tests are built directly with the generators above.
    """
    if name == "square32":
        return Problem(name, unit_square(8), 1.0, 32, 1.0)
    if name == "square64":
        return Problem(name, unit_square(16), 1.0, 64, 1.0)
    if name == "square256":
        return Problem(name, unit_square(64), 1.0, 256, 1.0)
    if name == "lshape1024":
        return Problem(name, l_shape(1024, seed=3), 1.0, 1024, 0.5)
    if name == "square512":
        return Problem(name, unit_square(128), 1.0, 512, 1.0)
    if name == "star256":
        return Problem(name, star(16, 16, seed=5), 1.0, 256, 1.0)
    raise KeyError(name)
