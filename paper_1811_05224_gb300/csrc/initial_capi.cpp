// C ABI of the initial-data operator M_h^0 (Section 1, eq. (4)): the
// triangulation handle (validation, boundary-vertex matching, node-disjoint
// colouring of the triangles), assembly, the matrix-free product and the
// Section 4 example data.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "capi_internal.h"
#include "domain_host.h"
#include "initial.h"
#include "stbem.h"

using stbem_internal::cuda_fail;
using stbem_internal::fail;

struct stbem_domain {
  int device = 0;
  const stbem_mesh* mesh = nullptr;
  int M = 0, K = 0;
  double* dbuf = nullptr;        // nx | ny | area | diam
  int* ibuf = nullptr;           // tri (3K) | bnode (N) | colour lists (K)
  std::vector<int> color_off;    // colour c: entries color_off[c] .. color_off[c+1] of the lists
  stbem::DevDomain dev{};
};


extern "C" {

int stbem_domain_create(stbem_ctx* ctx, const stbem_mesh* mesh, const double* host_nodes, int n_nodes,
                        const int* host_tris, int n_tris, stbem_domain** out) {
  if (!ctx || !out) return STBEM_ERR_ARG;
  *out = nullptr;
  if (!mesh || !host_nodes || !host_tris) return fail(ctx, STBEM_ERR_ARG, "domain: NULL argument");
  if (n_nodes < 3 || n_tris < 1) return fail(ctx, STBEM_ERR_ARG, "domain: need n_nodes >= 3, n_tris >= 1");
  const int M = n_nodes, K = n_tris, N = mesh->N;
  std::vector<double> x(M), y(M);
  double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
  for (int j = 0; j < M; ++j) {
    x[j] = host_nodes[2 * j];
    y[j] = host_nodes[2 * j + 1];
    if (!std::isfinite(x[j]) || !std::isfinite(y[j])) return fail(ctx, STBEM_ERR_ARG, "domain: non-finite node %d", j);
    lo[0] = std::min(lo[0], x[j]);
    hi[0] = std::max(hi[0], x[j]);
    lo[1] = std::min(lo[1], y[j]);
    hi[1] = std::max(hi[1], y[j]);
  }
  std::vector<int> tri(host_tris, host_tris + 3 * K);
  for (int t = 0; t < 3 * K; ++t)
    if (tri[t] < 0 || tri[t] >= M) return fail(ctx, STBEM_ERR_ARG, "domain: triangle index out of range");
  // boundary vertex p -> the nearest node, which must lie within 1e-12 x diameter
  const double diam = std::max(hi[0] - lo[0], hi[1] - lo[1]);
  std::vector<int> bnode(N);
  const int bad = stbem::match_boundary_nodes(x, y, mesh->xy.data(), N, 1e-12 * diam, bnode.data());
  if (bad >= 0) return fail(ctx, STBEM_ERR_ARG, "domain: boundary vertex %d is not a node", bad);
  for (int p = 0; p < N; ++p) {
    x[bnode[p]] = mesh->xy[2 * p];
    y[bnode[p]] = mesh->xy[2 * p + 1];
  }
  std::vector<double> area(K), dmax(K);
  for (int k = 0; k < K; ++k) {
    const int a = tri[3 * k], b = tri[3 * k + 1], c = tri[3 * k + 2];
    const double a2 = (x[b] - x[a]) * (y[c] - y[a]) - (y[b] - y[a]) * (x[c] - x[a]);
    if (!(a2 > 0)) return fail(ctx, STBEM_ERR_ARG, "domain: triangle %d is not counter-clockwise", k);
    area[k] = 0.5 * a2;
    double dm = 0.0;
    for (int e = 0; e < 3; ++e) {
      const int u = tri[3 * k + e], v = tri[3 * k + (e + 1) % 3];
      const double dx = x[u] - x[v], dy = y[u] - y[v];
      dm = std::max(dm, std::sqrt(dx * dx + dy * dy));
    }
    dmax[k] = dm;
  }
  int nc = 0;
  const std::vector<int> col = stbem::colour_triangles(M, K, tri, &nc);
  std::vector<int> lists;
  lists.reserve(K);
  stbem_domain* d = new stbem_domain();
  d->color_off.assign(1, 0);
  for (int c = 0; c < nc; ++c) {
    for (int k = 0; k < K; ++k)
      if (col[k] == c) lists.push_back(k);
    d->color_off.push_back((int)lists.size());
  }
  std::vector<double> hd;
  hd.reserve(2 * (size_t)M + 2 * (size_t)K);
  hd.insert(hd.end(), x.begin(), x.end());
  hd.insert(hd.end(), y.begin(), y.end());
  hd.insert(hd.end(), area.begin(), area.end());
  hd.insert(hd.end(), dmax.begin(), dmax.end());
  std::vector<int> hi_;
  hi_.reserve(3 * (size_t)K + N + K);
  hi_.insert(hi_.end(), tri.begin(), tri.end());
  hi_.insert(hi_.end(), bnode.begin(), bnode.end());
  hi_.insert(hi_.end(), lists.begin(), lists.end());
  d->device = ctx->device;
  d->mesh = mesh;
  d->M = M;
  d->K = K;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&d->dbuf, hd.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d->ibuf, hi_.size() * sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d->dbuf, hd.data(), hd.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d->ibuf, hi_.data(), hi_.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    if (d->dbuf) cudaFree(d->dbuf);
    if (d->ibuf) cudaFree(d->ibuf);
    delete d;
    return cuda_fail(ctx, e, "domain upload");
  }
  stbem::DevDomain& D = d->dev;
  D.M = M;
  D.K = K;
  D.nx = d->dbuf;
  D.ny = d->dbuf + M;
  D.area = d->dbuf + 2 * (size_t)M;
  D.diam = d->dbuf + 2 * (size_t)M + K;
  D.tri = d->ibuf;
  D.bnode = d->ibuf + 3 * (size_t)K;
  *out = d;
  return STBEM_OK;
}

void stbem_domain_destroy(stbem_domain* d) {
  if (!d) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(d->device);
  if (d->dbuf) cudaFree(d->dbuf);
  if (d->ibuf) cudaFree(d->ibuf);
  cudaSetDevice(prev);
  delete d;
}

int stbem_domain_info(const stbem_domain* d, int* n_nodes, int* n_tris, int* n_colors, int* host_bnode) {
  if (!d) return STBEM_ERR_ARG;
  if (n_nodes) *n_nodes = d->M;
  if (n_tris) *n_tris = d->K;
  if (n_colors) *n_colors = (int)d->color_off.size() - 1;
  if (host_bnode) {
    cudaError_t e = cudaMemcpy(host_bnode, d->dev.bnode, sizeof(int) * d->mesh->N, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return STBEM_ERR_CUDA;
  }
  return STBEM_OK;
}

int stbem_m0_bytes(const stbem_domain* d, size_t* bytes) {
  if (!d || !bytes) return STBEM_ERR_ARG;
  *bytes = (size_t)d->mesh->n_t * d->mesh->N * d->M * sizeof(double);
  return STBEM_OK;
}

int stbem_m0_assemble(stbem_ctx* ctx, const stbem_domain* d, double* dev_M0) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!d || !dev_M0) return fail(ctx, STBEM_ERR_ARG, "m0_assemble: NULL argument");
  size_t bytes = 0;
  stbem_m0_bytes(d, &bytes);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "m0_assemble");
  CUDA_TRY(ctx, cudaMemsetAsync(dev_M0, 0, bytes, ctx->stream), "m0_assemble memset");
  const int* lists = d->dev.bnode + d->mesh->N;
  for (size_t c = 0; c + 1 < d->color_off.size(); ++c) {
    const int b = d->color_off[c], n = d->color_off[c + 1] - b;
    CUDA_TRY(ctx, stbem::m0_assemble_launch(d->mesh->dev, d->dev, lists + b, n, dev_M0, ctx->stream),
             "m0_assemble launch");
  }
  return STBEM_OK;
}

int stbem_m0_apply_workspace_bytes(const stbem_domain* d, size_t* bytes) {
  if (!d || !bytes) return STBEM_ERR_ARG;
  *bytes = stbem::m0_apply_workspace_bytes(d->mesh->n_t, d->mesh->N, d->K);
  return STBEM_OK;
}

int stbem_m0_apply(stbem_ctx* ctx, const stbem_domain* d, int n_rhs, const double* dev_u0, double scale,
                   double* dev_y, void* dev_work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!d || !dev_u0 || !dev_y || !dev_work) return fail(ctx, STBEM_ERR_ARG, "m0_apply: NULL argument");
  if (n_rhs < 1) return fail(ctx, STBEM_ERR_ARG, "m0_apply: need n_rhs >= 1");
  if (d->mesh->n_t > 6144) return fail(ctx, STBEM_ERR_ARG, "m0_apply: n_t above 6144");
  if (d->mesh->N > 65535) return fail(ctx, STBEM_ERR_ARG, "m0_apply: n_x above 65535");
  const size_t need = stbem::m0_apply_workspace_bytes(d->mesh->n_t, d->mesh->N, d->K);
  if (work_bytes < need) return fail(ctx, STBEM_ERR_NOMEM, "m0_apply: workspace %zu < %zu bytes", work_bytes, need);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "m0_apply");
  const size_t vec = (size_t)d->mesh->n_t * d->mesh->N;
  for (int b = 0; b < n_rhs; ++b)
    CUDA_TRY(ctx, stbem::m0_apply_launch(d->mesh->dev, d->dev, dev_u0 + (size_t)b * d->M, scale, dev_y + b * vec,
                                         dev_work, ctx->stream),
             "m0_apply launch");
  return STBEM_OK;
}

int stbem_evaluate(stbem_ctx* ctx, const stbem_mesh* mesh, const stbem_domain* d, int n_points,
                   const double* dev_xy, const double* dev_t, const double* dev_w, const double* dev_g,
                   const double* dev_u0, double* dev_u) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!mesh) return fail(ctx, STBEM_ERR_ARG, "evaluate: NULL mesh");
  if (n_points < 0) return fail(ctx, STBEM_ERR_ARG, "evaluate: n_points < 0");
  if (n_points == 0) return STBEM_OK;
  if (!dev_xy || !dev_t || !dev_w || !dev_g || !dev_u) return fail(ctx, STBEM_ERR_ARG, "evaluate: NULL array");
  if (dev_u0 && !d) return fail(ctx, STBEM_ERR_ARG, "evaluate: u0 given without a domain");
  if (d && d->mesh != mesh) return fail(ctx, STBEM_ERR_ARG, "evaluate: domain built on another mesh");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "evaluate");
  CUDA_TRY(ctx, stbem::evaluate_launch(mesh->dev, d ? &d->dev : nullptr, n_points, dev_xy, dev_t, dev_w, dev_g,
                                       dev_u0, dev_u, ctx->stream),
           "evaluate launch");
  return STBEM_OK;
}

int stbem_planewave_data(stbem_ctx* ctx, const stbem_domain* d, double theta, double* dev_g, double* dev_u0) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!d) return fail(ctx, STBEM_ERR_ARG, "planewave_data: NULL domain");
  if (!std::isfinite(theta)) return fail(ctx, STBEM_ERR_ARG, "planewave_data: non-finite theta");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "planewave_data");
  CUDA_TRY(ctx, stbem::planewave_launch(d->mesh->dev, d->dev, theta, dev_g, dev_u0, ctx->stream),
           "planewave_data launch");
  return STBEM_OK;
}

}  // extern "C"
