// Host build of the triangulation handle's host logic (domain_host.h) for CPU tests.
#include "domain_host.h"
extern "C" {
int dh_match(const double* nodes, int M, const double* xy, int N, double tol, int* bnode) {
  std::vector<double> x(M), y(M);
  for (int j = 0; j < M; ++j) {
    x[j] = nodes[2 * j];
    y[j] = nodes[2 * j + 1];
  }
  return stbem::match_boundary_nodes(x, y, xy, N, tol, bnode);
}
int dh_colour(int M, int K, const int* tri, int* col) {
  std::vector<int> t(tri, tri + 3 * K);
  int nc = 0;
  const std::vector<int> c = stbem::colour_triangles(M, K, t, &nc);
  for (int k = 0; k < K; ++k) col[k] = c[k];
  return nc;
}
}
