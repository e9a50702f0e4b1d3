// Host logic of the triangulation handle (initial datum, Section 1 eq. (4)):
// matching the boundary vertices to nodes and the node-disjoint colouring of
// the triangles that lets the M_h^0 assembly write without conflicts.  Plain
// C++ (no CUDA), also compiled into the CPU tests.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

namespace stbem {

// bnode[p] = the node nearest to boundary vertex p (xy[2p], xy[2p+1]); ties
// go to the lower index.  Returns -1, or the first p whose nearest node is
// farther than tol.
inline int match_boundary_nodes(const std::vector<double>& x, const std::vector<double>& y, const double* xy,
                                int N, double tol, int* bnode) {
  const int M = (int)x.size();
  std::vector<int> byx(M);
  for (int j = 0; j < M; ++j) byx[j] = j;
  std::sort(byx.begin(), byx.end(), [&](int a, int b) { return x[a] < x[b] || (x[a] == x[b] && a < b); });
  for (int p = 0; p < N; ++p) {
    const double px = xy[2 * p], py = xy[2 * p + 1];
    auto it = std::lower_bound(byx.begin(), byx.end(), px - tol, [&](int a, double v) { return x[a] < v; });
    int best = -1;
    double bd = 1e300;
    for (; it != byx.end() && x[*it] <= px + tol; ++it) {
      const double dx = x[*it] - px, dy = y[*it] - py;
      const double d = std::sqrt(dx * dx + dy * dy);
      if (d < bd || (d == bd && *it < best)) {
        bd = d;
        best = *it;
      }
    }
    if (best < 0 || bd > tol) return p;
    bnode[p] = best;
  }
  return -1;
}

// Greedy colouring: each triangle (in index order) takes the smallest colour
// not used by a triangle that shares one of its nodes.  tri: 3 K node indices
// below M.  Returns the colour of every triangle; *n_colors the count.
inline std::vector<int> colour_triangles(int M, int K, const std::vector<int>& tri, int* n_colors) {
  std::vector<int> off(M + 1, 0), adj(3 * (size_t)K);
  for (int t = 0; t < 3 * K; ++t) ++off[tri[t] + 1];
  for (int j = 0; j < M; ++j) off[j + 1] += off[j];
  std::vector<int> fill(off.begin(), off.end() - 1);
  for (int k = 0; k < K; ++k)
    for (int c = 0; c < 3; ++c) adj[fill[tri[3 * k + c]]++] = k;
  std::vector<int> col(K, -1);
  std::vector<int> used;
  int nc = 0;
  for (int k = 0; k < K; ++k) {
    used.assign(nc + 1, 0);
    for (int c = 0; c < 3; ++c) {
      const int j = tri[3 * k + c];
      for (int a = off[j]; a < off[j + 1]; ++a) {
        const int o = col[adj[a]];
        if (o >= 0) used[o] = 1;
      }
    }
    int pick = 0;
    while (pick < nc && used[pick]) ++pick;
    col[k] = pick;
    nc = std::max(nc, pick + 1);
  }
  *n_colors = nc;
  return col;
}

}  // namespace stbem
