"""Quadrature orders and switching thresholds of the reference discretisation.

The paper prints no quadrature rule (it refers the assembly to companion
papers), so the discretisation both the oracle and the CUDA path implement is
fixed here, in the paper's notation: Galerkin entries over a pair of boundary
pieces (segments of Gamma_h, or half-segments for the dual space Y_h of
Section 2) and a pair of time steps of I_h at lag d.

* lags 0 and 1 (the kernel keeps a log r or r^2 log r singularity):
  - regular pairs: tensor Gauss-Legendre, ``n_regular01`` points per piece;
  - near pairs (ring distance 2, or gap < ``near_gap_ratio`` * longer piece):
    ``n_near01`` points per piece;
  - identical pieces: split at the diagonal, graded Gauss in |xi - eta|;
  - adjacent pieces: Duffy split at the shared vertex, graded Gauss radially.
* lags d >= 2 (integrands analytic in space): tensor Gauss with
  ``space_order(d)`` points per piece for every pair class.
* time: lag 0 and lag 1 in closed form (series-rearranged for z < 1 at lag 1);
  lags d >= 2 in closed form when z_d = alpha r^2 / (4 d ht) > d / 2, else in
  the Peano form with ``peano_order(k)`` Gauss nodes on time interval k.

Orders were chosen by measuring against brute-force adaptive quadrature;
tests/test_oracle_assembly.py pins the result in every regime: lags 0-2 on
tiny meshes, and lags 8, 9, 31, 32, 33, 100 (and 255) on the meshes where one
step's diffusion length is shortest against the pieces (unit square with
h = 1/16 and N_t = 512, the seeded L-shape at its shortest and longest
segments, the alpha = 10 example at level 4, the star).
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class Rules:
    n_regular01: int = 12
    n_near01: int = 16
    graded_sigma: float = 0.2
    graded_levels: int = 18
    graded_points: int = 16
    singular_inner: int = 4
    duffy_angular: int = 16
    lag_space_orders: tuple = ((2, 8), (8, 6), (32, 4))
    peano_orders: tuple = ((1, 16), (2, 8), (32, 6))
    near_gap_ratio: float = 0.5

    def space_order(self, d: int) -> int:
        """Gauss points per piece for every pair at lag d >= 2."""
        n = self.lag_space_orders[0][1]
        for start, order in self.lag_space_orders:
            if d >= start:
                n = order
        return n

    def peano_order(self, k: int) -> int:
        """Gauss nodes on time interval [k ht, (k+1) ht], k >= 1."""
        n = self.peano_orders[0][1]
        for start, order in self.peano_orders:
            if k >= start:
                n = order
        return n


DEFAULT_RULES = Rules()
