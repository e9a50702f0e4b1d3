// Initial-data operator M_h^0 (Section 1, eq. (4)) on a triangulation of the
// domain: device view of the triangulation and the launches.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

#include "assemble.h"

namespace stbem {

// Triangulation Omega_h, conforming with the boundary mesh: node bnode[p] is
// boundary vertex p (its coordinates equal the vertex's).
struct DevDomain {
  int M, K;                  // nodes, triangles
  const double *nx, *ny;     // node coordinates (M)
  const int* tri;            // 3 K node indices, counter-clockwise
  const double *area, *diam; // per triangle (K): area, longest edge
  const int* bnode;          // N
};

// The kernels' own copy of the Gauss tables.
cudaError_t upload_m0_rule_tables(const RuleTables& t, cudaStream_t s);

// M0[m][i][j] += the contributions of the n_tris triangles listed in tris
// (no two of them share a node, so no two threads write one entry).
cudaError_t m0_assemble_launch(const DevMesh& M, const DevDomain& D, const int* tris, int n_tris, double* M0,
                               cudaStream_t s);

// y[m][i] += scale (M0 u0)[m][i], matrix-free: per-block partial sums in work,
// then a fixed-order reduction.
size_t m0_apply_workspace_bytes(int nt, int N, int K);
cudaError_t m0_apply_launch(const DevMesh& M, const DevDomain& D, const double* u0, double scale, double* y,
                            void* work, cudaStream_t s);

// u_h at n_points points (xy: 2 n_points) and times t (n_points) by the
// representation formula, eq. (2); D and u0 may be NULL (u_0 = 0).
cudaError_t evaluate_launch(const DevMesh& M, const DevDomain* D, int n_points, const double* xy, const double* t,
                            const double* w, const double* g, const double* u0, double* u, cudaStream_t s);

// Section 4 example u = exp(-t/alpha) sin(x . d), d = (cos theta, sin theta):
// g[n][p] time averages at the vertices, u0[j] nodal values.
cudaError_t planewave_launch(const DevMesh& M, const DevDomain& D, double theta, double* g, double* u0,
                             cudaStream_t s);

}  // namespace stbem
