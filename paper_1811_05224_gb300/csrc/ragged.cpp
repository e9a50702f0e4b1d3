// Ragged batches: many independent problems of different sizes (N_x, N_t)
// through the same hot path.
//
//   * assembly: one persistent launch per operator (plus one for the lag-0/1
//     singular pairs) over the (problem, lag, tile) work items of every
//     problem, largest problems first, taken from an atomic counter;
//   * products: one persistent launch over the (problem, lag chunk, time tile,
//     row tile) units of every problem, then one reduction; the tile family
//     (FP32 register tiles or generic tiles) and the lag-chunk length are
//     picked by an autotuner that times the candidates on the batch itself
//     (stbem_ragged_tune), keeps the fastest and records it in the tune cache
//     under the device and the batch's shape, so that a later batch of the
//     same shapes (in this process, or in another one with the same cache
//     file) skips the timing;
//   * GMRES: all problems in lockstep, per-problem Hessenberg / Givens on the
//     host, masks for converged problems.  The device work of one Arnoldi step
//     (preconditioner, product, two Gram-Schmidt passes, norm, normalisation,
//     copies of the coefficients to pinned host memory) is captured once per
//     Krylov index as a CUDA graph and replayed, so an iteration costs one
//     graph launch and one synchronisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>
#include <numeric>
#include <vector>

#include "assemble.h"
#include "capi_internal.h"
#include "stbem.h"
#include "toeplitz.h"
#include "tune_cache.h"
#include "vec.h"

using stbem_internal::cuda_fail;
using stbem_internal::fail;

struct stbem_ragged {
  int device = 0;
  int P = 0;
  std::vector<stbem_mesh*> meshes;
  std::vector<int> nx, nt;
  std::vector<long long> op_off, vec_off, mass_off;
  long long op_elems = 0, vec_elems = 0, mass_elems = 0;
  int max_nx = 0;
  std::vector<int> order;                       // problems by decreasing work
  stbem::RaggedProblem* d_probs = nullptr;
  int* d_order = nullptr;
  long long* d_sing_prefix = nullptr;           // 3 ops x (P + 1)
  long long* d_tile_prefix = nullptr;           // 2 precisions x 3 ops x (P + 1)
  long long* d_vprefix = nullptr;               // P + 1, natural order
  unsigned long long* d_counters = nullptr;     // 4 words
  // products
  int lags_per_chunk = 0;                       // 0: not tuned yet
  std::vector<stbem::RaggedApplyPlan> plans;
  stbem::RaggedApplyPlan* d_plans = nullptr;    // generic tiles (FP64, and FP32 when N_x % 4 != 0)
  long long* d_aprefix = nullptr;               // P + 1 (problem order)
  bool fp32_tiles = false;                      // every N_x % 4 == 0: register-tiled FP32 kernel possible
  bool use_tiles32 = true;                      // FP32 products use it (tuned)
  bool tuned_from_cache = false;
  stbem::RaggedApplyPlan* d_plans32 = nullptr;
  long long* d_aprefix32 = nullptr;
  long long part_elems = 0;                     // max over both plan sets
  std::vector<int> tuned_candidates;            // lag-chunk lengths tried
  std::vector<int> tuned_tiles;                 // 1: register tiles, 0: generic
  std::vector<float> tuned_ms;
  // solve: pinned host buffers and captured graphs
  double* h_buf = nullptr;                      // 2 (restart + 1) P + P doubles
  int* h_mask = nullptr;                        // P
  int graph_restart = 0;
  const void* graph_key[6] = {};
  int graph_prec = -1;
  std::vector<cudaGraphExec_t> graphs;
  std::vector<unsigned> graph_kernels;
  cudaStream_t gs = nullptr;                    // solve stream (capturable; the caller's may be the legacy one)
};

namespace {

constexpr int kTuneCandidates[] = {32, 64, 128, 256, 512};

void free_graphs(stbem_ragged* R) {
  for (auto g : R->graphs)
    if (g) cudaGraphExecDestroy(g);
  R->graphs.clear();
  R->graph_kernels.clear();
}

// plans for a lag-chunk length; returns the partial-sum elements needed
long long build_plans(stbem_ragged* R, int lpc, bool fp32_tiles, std::vector<stbem::RaggedApplyPlan>* out,
                      std::vector<long long>* aprefix) {
  const int P = R->P;
  out->assign(P, {});
  long long part = 0;
  for (int p = 0; p < P; ++p) {
    stbem::RaggedApplyPlan& pl = (*out)[p];
    stbem::ragged_apply_plan(R->nt[p], R->nx[p], lpc, fp32_tiles, &pl);
    pl.a_off = R->op_off[p];
    pl.v_off = R->vec_off[p];
    pl.part_off = part;
    part += pl.part_elems;
  }
  aprefix->assign(P + 1, 0);
  for (int s = 0; s < P; ++s) (*aprefix)[s + 1] = (*aprefix)[s] + (*out)[R->order[s]].units;
  return part;
}

cudaError_t upload_plans(const std::vector<stbem::RaggedApplyPlan>& plans, const std::vector<long long>& aprefix,
                         stbem::RaggedApplyPlan* d_plans, long long* d_aprefix, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(d_plans, plans.data(), plans.size() * sizeof(plans[0]), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_aprefix, aprefix.data(), aprefix.size() * sizeof(long long), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

long long part_elems_for(stbem_ragged* R, int lpc) {
  std::vector<stbem::RaggedApplyPlan> pl;
  std::vector<long long> pre;
  long long n = build_plans(R, lpc, false, &pl, &pre);
  if (R->fp32_tiles) n = std::max(n, build_plans(R, lpc, true, &pl, &pre));
  return n;
}

int set_chunk(stbem_ctx* ctx, stbem_ragged* R, int lpc) {
  std::vector<long long> pre;
  R->part_elems = build_plans(R, lpc, false, &R->plans, &pre);
  CUDA_TRY(ctx, upload_plans(R->plans, pre, R->d_plans, R->d_aprefix, ctx->stream), "ragged: upload product plans");
  if (R->fp32_tiles) {
    std::vector<stbem::RaggedApplyPlan> p32;
    R->part_elems = std::max(R->part_elems, build_plans(R, lpc, true, &p32, &pre));
    CUDA_TRY(ctx, upload_plans(p32, pre, R->d_plans32, R->d_aprefix32, ctx->stream), "ragged: upload FP32 plans");
  }
  R->lags_per_chunk = lpc;
  free_graphs(R);   // captured steps refer to the old plans' partial layout
  return STBEM_OK;
}

cudaError_t rapply(stbem_ragged* R, int prec, const void* A, const double* x, double* y, double* part,
                   cudaStream_t s) {
  const bool t32 = prec == STBEM_F32 && R->fp32_tiles && R->use_tiles32;
  return stbem::ragged_apply_launch(prec, t32, t32 ? R->d_plans32 : R->d_plans,
                                    {R->d_order, t32 ? R->d_aprefix32 : R->d_aprefix}, R->d_vprefix, R->P,
                                    R->d_counters + 2, A, x, y, part, s);
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// tune-cache key: device, precision and the (N_x, N_t) list (FNV-1a 64)
std::string ragged_tune_key(const stbem_ragged* R, int prec) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](long long v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (unsigned long long)((v >> (8 * b)) & 0xff);
      h *= 1099511628211ull;
    }
  };
  for (int p = 0; p < R->P; ++p) {
    mix(R->nx[p]);
    mix(R->nt[p]);
  }
  char buf[64];
  std::snprintf(buf, sizeof(buf), "%016llx", h);
  return stbem::tune_device_key(R->device) + "|ragged_apply|prec=" + (prec == STBEM_F64 ? "f64" : "f32") +
         "|P=" + std::to_string(R->P) + "|shapes=" + buf;
}

}  // namespace

extern "C" {

int stbem_ragged_create(stbem_ctx* ctx, int n, const stbem_problem* probs, stbem_ragged** out) {
  if (!ctx || !out) return STBEM_ERR_ARG;
  *out = nullptr;
  if (n < 1 || !probs) return fail(ctx, STBEM_ERR_ARG, "ragged: need at least one problem");
  stbem_ragged* R = new stbem_ragged();
  R->device = ctx->device;
  R->P = n;
  auto bail = [&](int code) {
    stbem_ragged_destroy(R);
    return code;
  };
  for (int p = 0; p < n; ++p) {
    stbem_mesh* m = nullptr;
    const int rc = stbem_mesh_create(ctx, probs[p].xy, probs[p].n_x, probs[p].T, probs[p].n_t, probs[p].alpha, &m);
    if (rc != STBEM_OK) return bail(rc);
    R->meshes.push_back(m);
    R->nx.push_back(m->N);
    R->nt.push_back(m->n_t);
    R->op_off.push_back(R->op_elems);
    R->vec_off.push_back(R->vec_elems);
    R->mass_off.push_back(R->mass_elems);
    R->op_elems += (long long)m->n_t * m->N * m->N;
    R->vec_elems += (long long)m->n_t * m->N;
    R->mass_elems += m->N;
    R->max_nx = std::max(R->max_nx, m->N);
  }
  R->fp32_tiles = true;
  for (int v : R->nx) R->fp32_tiles = R->fp32_tiles && stbem::ragged_fp32_tiles_ok(v);
  // largest problems first (work ~ n_t N_x^2)
  R->order.resize(n);
  std::iota(R->order.begin(), R->order.end(), 0);
  std::stable_sort(R->order.begin(), R->order.end(), [&](int a, int b) {
    return (double)R->nt[a] * R->nx[a] * R->nx[a] > (double)R->nt[b] * R->nx[b] * R->nx[b];
  });
  std::vector<stbem::RaggedProblem> hp(n);
  for (int p = 0; p < n; ++p) hp[p] = {R->meshes[p]->dev, R->op_off[p], R->vec_off[p], R->mass_off[p]};
  std::vector<long long> sp(3 * (n + 1), 0), tp(6 * (n + 1), 0), vp(n + 1, 0);
  for (int op = 0; op < 3; ++op)
    for (int s = 0; s < n; ++s) {
      const int p = R->order[s];
      const int Rl = op == STBEM_OP_D ? 2 * R->nx[p] : R->nx[p];
      const int l01 = R->nt[p] < 2 ? R->nt[p] : 2;
      sp[op * (n + 1) + s + 1] = sp[op * (n + 1) + s] + (long long)l01 * 3 * Rl;
      for (int pi = 0; pi < 2; ++pi) {
        const int prec = pi == 0 ? STBEM_F64 : STBEM_F32;
        long long* t = tp.data() + (size_t)(pi * 3 + op) * (n + 1);
        t[s + 1] = t[s] + (long long)stbem::assembly_lag_groups(op, prec, R->nt[p]) *
                              stbem::assembly_tiles_per_lag(op, R->nx[p]);
      }
    }
  for (int p = 0; p < n; ++p) vp[p + 1] = vp[p] + (long long)R->nt[p] * R->nx[p];
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&R->d_probs, n * sizeof(stbem::RaggedProblem));
  if (e == cudaSuccess) e = cudaMalloc(&R->d_order, n * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&R->d_sing_prefix, sp.size() * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&R->d_tile_prefix, tp.size() * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&R->d_vprefix, vp.size() * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&R->d_counters, 4 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&R->d_plans, n * sizeof(stbem::RaggedApplyPlan));
  if (e == cudaSuccess) e = cudaMalloc(&R->d_aprefix, (n + 1) * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&R->d_plans32, n * sizeof(stbem::RaggedApplyPlan));
  if (e == cudaSuccess) e = cudaMalloc(&R->d_aprefix32, (n + 1) * sizeof(long long));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&R->gs, cudaStreamNonBlocking);
  cudaStream_t s = ctx->stream;
  if (e == cudaSuccess) e = cudaMemcpyAsync(R->d_probs, hp.data(), n * sizeof(hp[0]), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(R->d_order, R->order.data(), n * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(R->d_sing_prefix, sp.data(), sp.size() * sizeof(long long), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(R->d_tile_prefix, tp.data(), tp.size() * sizeof(long long), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(R->d_vprefix, vp.data(), vp.size() * sizeof(long long), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "ragged: upload"));
  const int rc = set_chunk(ctx, R, 64);   // default until tuned
  if (rc != STBEM_OK) return bail(rc);
  R->lags_per_chunk = 0;
  *out = R;
  return STBEM_OK;
}

void stbem_ragged_destroy(stbem_ragged* R) {
  if (!R) return;
  cudaSetDevice(R->device);
  free_graphs(R);
  for (auto* m : R->meshes) stbem_mesh_destroy(m);
  for (void* p : {(void*)R->d_probs, (void*)R->d_order, (void*)R->d_sing_prefix, (void*)R->d_tile_prefix,
                  (void*)R->d_vprefix, (void*)R->d_counters, (void*)R->d_plans, (void*)R->d_aprefix,
                  (void*)R->d_plans32, (void*)R->d_aprefix32})
    if (p) cudaFree(p);
  if (R->h_buf) cudaFreeHost(R->h_buf);
  if (R->h_mask) cudaFreeHost(R->h_mask);
  if (R->gs) cudaStreamDestroy(R->gs);
  delete R;
}

int stbem_ragged_sizes(const stbem_ragged* R, long long* op_elems, long long* vec_elems, long long* mass_elems) {
  if (!R) return STBEM_ERR_ARG;
  if (op_elems) *op_elems = R->op_elems;
  if (vec_elems) *vec_elems = R->vec_elems;
  if (mass_elems) *mass_elems = R->mass_elems;
  return STBEM_OK;
}

int stbem_ragged_offsets(const stbem_ragged* R, long long* op_off, long long* vec_off, long long* mass_off) {
  if (!R) return STBEM_ERR_ARG;
  for (int p = 0; p < R->P; ++p) {
    if (op_off) op_off[p] = R->op_off[p];
    if (vec_off) vec_off[p] = R->vec_off[p];
    if (mass_off) mass_off[p] = R->mass_off[p];
  }
  return STBEM_OK;
}

int stbem_ragged_assemble(stbem_ctx* ctx, stbem_ragged* R, int op, int prec, void* out) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!R || !out) return fail(ctx, STBEM_ERR_ARG, "ragged_assemble: NULL argument");
  if (op < STBEM_OP_V || op > STBEM_OP_D) return fail(ctx, STBEM_ERR_ARG, "ragged_assemble: bad operator");
  if (prec != STBEM_F64 && prec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "ragged_assemble: bad precision");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "ragged_assemble: set device");
  const int P = R->P;
  stbem::RaggedItems si{R->d_order, R->d_sing_prefix + (size_t)op * (P + 1)};
  const int pi = prec == STBEM_F64 ? 0 : 1;
  stbem::RaggedItems ti{R->d_order, R->d_tile_prefix + (size_t)(pi * 3 + op) * (P + 1)};
  CUDA_TRY(ctx, stbem::ragged_assemble_launch(op, prec, R->d_probs, P, si, ti, R->d_counters, out, ctx->stream),
           "ragged_assemble");
  return STBEM_OK;
}

int stbem_ragged_lumped_mass(stbem_ctx* ctx, stbem_ragged* R, double* L) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!R || !L) return fail(ctx, STBEM_ERR_ARG, "ragged_lumped_mass: NULL argument");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "ragged_lumped_mass: set device");
  CUDA_TRY(ctx, stbem::rlumped_launch(R->d_probs, R->P, R->max_nx, L, ctx->stream), "ragged_lumped_mass");
  return STBEM_OK;
}

int stbem_ragged_apply_workspace_bytes(const stbem_ragged* R, size_t* bytes) {
  if (!R || !bytes) return STBEM_ERR_ARG;
  long long need = 0;
  for (int c : kTuneCandidates) need = std::max(need, part_elems_for(const_cast<stbem_ragged*>(R), c));
  *bytes = (size_t)need * sizeof(double);
  return STBEM_OK;
}

int stbem_ragged_apply(stbem_ctx* ctx, stbem_ragged* R, int prec, const void* A, const double* x, double* y,
                       void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!R || !A || !x || !y || !work) return fail(ctx, STBEM_ERR_ARG, "ragged_apply: NULL argument");
  if (prec != STBEM_F64 && prec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "ragged_apply: bad precision");
  if (work_bytes < (size_t)R->part_elems * sizeof(double))
    return fail(ctx, STBEM_ERR_NOMEM, "ragged_apply: workspace %zu < %zu bytes", work_bytes,
                (size_t)R->part_elems * sizeof(double));
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "ragged_apply: set device");
  CUDA_TRY(ctx, rapply(R, prec, A, x, y, static_cast<double*>(work), ctx->stream), "ragged_apply");
  return STBEM_OK;
}

int stbem_ragged_tune(stbem_ctx* ctx, stbem_ragged* R, int prec, const void* A, const double* x, double* y,
                      void* work, size_t work_bytes, int* lags_per_chunk, int* tiles32) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!R || !A || !x || !y || !work) return fail(ctx, STBEM_ERR_ARG, "ragged_tune: NULL argument");
  if (prec != STBEM_F64 && prec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "ragged_tune: bad precision");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "ragged_tune: set device");
  cudaStream_t s = ctx->stream;
  int nt_max = 0;
  for (int v : R->nt) nt_max = std::max(nt_max, v);
  R->tuned_candidates.clear();
  R->tuned_tiles.clear();
  R->tuned_ms.clear();
  const bool try32 = prec == STBEM_F32 && R->fp32_tiles;
  // a recorded choice for these shapes on this device
  const std::string key = ragged_tune_key(R, prec);
  std::string v;
  int c_lpc = 0, c_t32 = -1;
  if (stbem::tune_cache_get(key, &v) && std::sscanf(v.c_str(), "tiles32=%d lpc=%d", &c_t32, &c_lpc) == 2 &&
      (c_t32 == 0 || (c_t32 == 1 && try32)) &&
      std::find(std::begin(kTuneCandidates), std::end(kTuneCandidates), c_lpc) != std::end(kTuneCandidates) &&
      (size_t)part_elems_for(R, c_lpc) * sizeof(double) <= work_bytes) {
    R->use_tiles32 = c_t32 == 1 || !try32;
    const int rc = set_chunk(ctx, R, c_lpc);
    if (rc != STBEM_OK) return rc;
    R->tuned_from_cache = true;
    if (lags_per_chunk) *lags_per_chunk = c_lpc;
    if (tiles32) *tiles32 = c_t32;
    return STBEM_OK;
  }
  cudaEvent_t e0, e1;
  CUDA_TRY(ctx, cudaEventCreate(&e0), "ragged_tune: event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(ctx, STBEM_ERR_CUDA, "ragged_tune: event");
  }
  int best = 0, best_t32 = 0;
  float best_ms = 0.f;
  // candidates: tile family (FP32 register tiles first when possible) x lag-chunk length
  for (int t32 = try32 ? 1 : 0; t32 >= 0; --t32) {
    R->use_tiles32 = t32 == 1;
    int tried = 0;
    for (int c : kTuneCandidates) {
      if (c > nt_max && tried > 0) break;   // longer chunks change nothing
      if ((size_t)part_elems_for(R, c) * sizeof(double) > work_bytes) continue;
      int rc = set_chunk(ctx, R, c);
      if (rc != STBEM_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc;
      }
      cudaError_t e = rapply(R, prec, A, x, y, static_cast<double*>(work), s);   // warm-up
      float ms = 0.f;
      for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = rapply(R, prec, A, x, y, static_cast<double*>(work), s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        ms = r == 0 ? t : std::min(ms, t);
      }
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(ctx, e, "ragged_tune: product");
      }
      ++tried;
      R->tuned_candidates.push_back(c);
      R->tuned_tiles.push_back(t32);
      R->tuned_ms.push_back(ms);
      if (best == 0 || ms < best_ms) {
        best = c;
        best_t32 = t32;
        best_ms = ms;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best == 0) return fail(ctx, STBEM_ERR_NOMEM, "ragged_tune: workspace too small for any candidate");
  R->use_tiles32 = best_t32 == 1 || !try32;
  const int rc = set_chunk(ctx, R, best);
  if (rc != STBEM_OK) return rc;
  R->tuned_from_cache = false;
  char val[64];
  std::snprintf(val, sizeof(val), "tiles32=%d lpc=%d", best_t32, best);
  if (!stbem::tune_cache_put(key, val))
    return fail(ctx, STBEM_ERR_ARG, "ragged_tune: cannot write the tune cache file %s",
                stbem::tune_cache_path().c_str());
  if (lags_per_chunk) *lags_per_chunk = best;
  if (tiles32) *tiles32 = best_t32;
  return STBEM_OK;
}

int stbem_ragged_tune_report(const stbem_ragged* R, int max_n, int* candidates, int* tiles32, float* ms, int* n_out,
                             int* from_cache) {
  if (!R || !n_out) return STBEM_ERR_ARG;
  const int n = (int)R->tuned_candidates.size();
  for (int i = 0; i < n && i < max_n; ++i) {
    if (candidates) candidates[i] = R->tuned_candidates[i];
    if (tiles32) tiles32[i] = R->tuned_tiles[i];
    if (ms) ms[i] = R->tuned_ms[i];
  }
  *n_out = n;
  if (from_cache) *from_cache = R->tuned_from_cache ? 1 : 0;
  return STBEM_OK;
}

int stbem_ragged_rhs(stbem_ctx* ctx, stbem_ragged* R, int kprec, const void* K, const double* ystar, double* g,
                     double* f, void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!R || !K || !ystar || !g || !f || !work) return fail(ctx, STBEM_ERR_ARG, "ragged_rhs: NULL argument");
  const size_t ybytes = align256((size_t)2 * R->P * sizeof(double));
  if (work_bytes < ybytes + (size_t)R->part_elems * sizeof(double))
    return fail(ctx, STBEM_ERR_NOMEM, "ragged_rhs: workspace too small");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "ragged_rhs: set device");
  cudaStream_t s = ctx->stream;
  double* dy = static_cast<double*>(work);
  double* part = reinterpret_cast<double*>(static_cast<char*>(work) + ybytes);
  CUDA_TRY(ctx, cudaMemcpyAsync(dy, ystar, 2 * R->P * sizeof(double), cudaMemcpyHostToDevice, s), "ragged_rhs: y*");
  CUDA_TRY(ctx, stbem::rrhs_g_launch(R->d_probs, R->d_vprefix, R->P, dy, g, R->vec_elems, s), "ragged_rhs: g");
  CUDA_TRY(ctx, rapply(R, kprec, K, g, f, part, s), "ragged_rhs: K g");
  CUDA_TRY(ctx, stbem::rhalf_mass_add_launch(R->d_probs, R->d_vprefix, R->P, g, f, R->vec_elems, s),
           "ragged_rhs: mass");
  CUDA_TRY(ctx, cudaStreamSynchronize(s), "ragged_rhs: sync");   // y* copy from the caller's host array
  return STBEM_OK;
}

}  // extern "C"

// ---- lockstep GMRES over a ragged batch --------------------------------------------
namespace {

struct RWork {
  double *Q, *Z, *U, *Rv, *W0, *h, *sq, *nrm, *inv, *Y, *part;
  int* mask;
};

size_t ragged_solve_bytes(const stbem_ragged* R, int m, long long part_elems) {
  const size_t n = (size_t)R->vec_elems, P = (size_t)R->P;
  size_t b = 0;
  b += align256((m + 1) * n * sizeof(double));   // Q
  b += 4 * align256(n * sizeof(double));          // Z, U, R, spare
  b += align256(2 * (m + 1) * P * sizeof(double));
  b += 3 * align256(P * sizeof(double));          // sq, nrm, inv
  b += align256((size_t)(m + 1) * P * sizeof(double));   // Y
  b += align256(P * sizeof(int));
  b += align256((size_t)part_elems * sizeof(double));
  return b;
}

void carve_ragged(void* base, const stbem_ragged* R, int m, RWork* w) {
  const size_t n = (size_t)R->vec_elems, P = (size_t)R->P;
  char* p = static_cast<char*>(base);
  auto take = [&](size_t bytes) {
    char* q = p;
    p += align256(bytes);
    return q;
  };
  w->Q = reinterpret_cast<double*>(take((m + 1) * n * sizeof(double)));
  w->Z = reinterpret_cast<double*>(take(n * sizeof(double)));
  w->U = reinterpret_cast<double*>(take(n * sizeof(double)));
  w->Rv = reinterpret_cast<double*>(take(n * sizeof(double)));
  w->W0 = reinterpret_cast<double*>(take(n * sizeof(double)));
  w->h = reinterpret_cast<double*>(take(2 * (m + 1) * P * sizeof(double)));
  w->sq = reinterpret_cast<double*>(take(P * sizeof(double)));
  w->nrm = reinterpret_cast<double*>(take(P * sizeof(double)));
  w->inv = reinterpret_cast<double*>(take(P * sizeof(double)));
  w->Y = reinterpret_cast<double*>(take((size_t)(m + 1) * P * sizeof(double)));
  w->mask = reinterpret_cast<int*>(take(P * sizeof(int)));
  w->part = reinterpret_cast<double*>(p);
}

struct ROps {
  stbem_ragged* R;
  int prec;
  const void *V, *D;
  const double* L;
  RWork W;
  cudaStream_t s;
  cudaError_t applyP(const double* x, double* y) const {
    if (!D) return cudaMemcpyAsync(y, x, (size_t)R->vec_elems * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaError_t e = stbem::rdiag_div_launch(R->d_probs, R->d_vprefix, R->P, x, L, W.W0, R->vec_elems, s);
    if (e == cudaSuccess) e = rapply(R, prec, D, W.W0, y, W.part, s);
    if (e == cudaSuccess) e = stbem::rdiag_div_launch(R->d_probs, R->d_vprefix, R->P, y, L, y, R->vec_elems, s);
    return e;
  }
  // the device part of Arnoldi step k (basis vectors 0..k given)
  cudaError_t step(int k, double* h_host) const {
    const size_t n = (size_t)R->vec_elems;
    const int P = R->P;
    double* qk = W.Q + (size_t)k * n;
    double* qk1 = W.Q + (size_t)(k + 1) * n;
    cudaError_t e = applyP(qk, W.Z);
    if (e == cudaSuccess) e = rapply(R, prec, V, W.Z, W.U, W.part, s);
    if (e == cudaSuccess) e = stbem::rdots_launch(W.Q, n, k + 1, W.U, R->d_vprefix, P, W.h, s);
    if (e == cudaSuccess) e = stbem::rcomb_launch(W.Q, n, k + 1, W.h, R->d_vprefix, P, true, W.U, (long long)n, s);
    if (e == cudaSuccess) e = stbem::rdots_launch(W.Q, n, k + 1, W.U, R->d_vprefix, P, W.h + (size_t)(k + 1) * P, s);
    if (e == cudaSuccess)
      e = stbem::rcomb_launch(W.Q, n, k + 1, W.h + (size_t)(k + 1) * P, R->d_vprefix, P, true, W.U, (long long)n, s);
    if (e == cudaSuccess) e = stbem::rdots_launch(W.U, n, 1, W.U, R->d_vprefix, P, W.sq, s);
    if (e == cudaSuccess) e = stbem::rinv_launch(W.sq, W.mask, P, W.nrm, W.inv, s);
    if (e == cudaSuccess) e = stbem::rscale_launch(W.U, W.inv, R->d_vprefix, P, qk1, (long long)n, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_host, W.h, 2 * (size_t)(k + 1) * P * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_host + 2 * (size_t)(k + 1) * P, W.nrm, P * sizeof(double), cudaMemcpyDeviceToHost, s);
    return e;
  }
};

}  // namespace

extern "C" {

int stbem_ragged_solve_workspace_bytes(const stbem_ragged* R, int restart, size_t* bytes) {
  if (!R || !bytes || restart < 1) return STBEM_ERR_ARG;
  size_t ab = 0;
  stbem_ragged_apply_workspace_bytes(R, &ab);
  *bytes = ragged_solve_bytes(R, restart, (long long)(ab / sizeof(double)));
  return STBEM_OK;
}

int stbem_ragged_solve(stbem_ctx* ctx, stbem_ragged* R, int prec, const void* V, const void* D, const double* L,
                       const double* f, double* w, const stbem_solve_opts* opts, stbem_solve_info* infos,
                       void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!R || !V || !f || !w || !opts || !infos || !work) return fail(ctx, STBEM_ERR_ARG, "ragged_solve: NULL argument");
  if (prec != STBEM_F64 && prec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "ragged_solve: bad precision");
  const int m = opts->restart, maxit = opts->max_iter;
  if (m < 1 || maxit < 1 || !(opts->tol > 0)) return fail(ctx, STBEM_ERR_ARG, "ragged_solve: bad options");
  const bool prec_on = opts->precondition != 0;
  if (prec_on && (!D || !L)) return fail(ctx, STBEM_ERR_ARG, "ragged_solve: preconditioner needs D and L");
  if (opts->precondition == 2)
    return fail(ctx, STBEM_ERR_ARG, "ragged_solve: the lumped mass (precondition = 1) only");
  if (work_bytes < ragged_solve_bytes(R, m, R->part_elems))
    return fail(ctx, STBEM_ERR_NOMEM, "ragged_solve: workspace too small");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "ragged_solve: set device");
  // the solve runs on the batch's own stream, which graph capture accepts;
  // inputs are complete once the caller's stream has drained
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "ragged_solve: caller stream");
  cudaStream_t s = R->gs;
  const int P = R->P;
  const size_t n = (size_t)R->vec_elems;
  RWork W;
  carve_ragged(work, R, m, &W);
  const ROps ops{R, prec, V, prec_on ? D : nullptr, prec_on ? L : nullptr, W, s};
  // pinned host buffers and the captured steps
  if (R->graph_restart != m || !R->h_buf) {
    if (R->h_buf) cudaFreeHost(R->h_buf);
    if (R->h_mask) cudaFreeHost(R->h_mask);
    R->h_buf = nullptr;
    R->h_mask = nullptr;
    CUDA_TRY(ctx, cudaHostAlloc(&R->h_buf, (2 * (size_t)(m + 1) * P + P) * sizeof(double), cudaHostAllocDefault),
             "ragged_solve: pinned buffer");
    CUDA_TRY(ctx, cudaHostAlloc(&R->h_mask, P * sizeof(int), cudaHostAllocDefault), "ragged_solve: pinned mask");
    free_graphs(R);
    R->graph_restart = m;
  }
  const void* key[6] = {V, ops.D, ops.L, work, reinterpret_cast<const void*>((uintptr_t)prec),
                        reinterpret_cast<const void*>((uintptr_t)R->lags_per_chunk)};
  if (!std::equal(key, key + 6, R->graph_key)) {
    free_graphs(R);
    std::copy(key, key + 6, R->graph_key);
  }
  if (R->graphs.empty()) {
    R->graphs.assign(m, nullptr);
    R->graph_kernels.assign(m, 0);
  }
  double* hh = R->h_buf;
  int* hmask = R->h_mask;

  auto norms = [&](const double* x, std::vector<double>& out) -> cudaError_t {
    cudaError_t e = stbem::rdots_launch(x, n, 1, x, R->d_vprefix, P, W.sq, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hh, W.sq, P * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    out.resize(P);
    for (int p = 0; p < P; ++p) out[p] = std::sqrt(hh[p]);
    return e;
  };

  std::vector<double> normF, rn;
  CUDA_TRY(ctx, norms(f, normF), "ragged_solve: norm f");
  CUDA_TRY(ctx, cudaMemsetAsync(w, 0, n * sizeof(double), s), "ragged_solve: w = 0");
  CUDA_TRY(ctx, cudaMemcpyAsync(W.Rv, f, n * sizeof(double), cudaMemcpyDeviceToDevice, s), "ragged_solve: r = f");
  for (int p = 0; p < P; ++p) {
    infos[p].iterations = 0;
    infos[p].rel_residual = 0.0;
    infos[p].status = std::isfinite(normF[p]) ? STBEM_OK : STBEM_ERR_NAN;
  }
  int total = 0;
  std::vector<double> inv(P);
  for (int cycle = 0; cycle < 1000; ++cycle) {
    CUDA_TRY(ctx, norms(W.Rv, rn), "ragged_solve: norm r");
    bool any = false;
    std::vector<char> active(P, 0);
    for (int p = 0; p < P; ++p) {
      const double rel = normF[p] > 0 ? rn[p] / normF[p] : 0.0;
      if (!std::isfinite(rel)) infos[p].status = STBEM_ERR_NAN;
      infos[p].rel_residual = rel;
      active[p] = infos[p].status == STBEM_OK && rel > opts->tol;
      any = any || active[p];
    }
    if (!any) break;
    if (total >= maxit) {
      for (int p = 0; p < P; ++p)
        if (active[p]) infos[p].status = STBEM_ERR_NOCONV;
      break;
    }
    for (int p = 0; p < P; ++p) inv[p] = (active[p] && rn[p] > 0) ? 1.0 / rn[p] : 0.0;
    CUDA_TRY(ctx, cudaMemcpyAsync(W.inv, inv.data(), P * sizeof(double), cudaMemcpyHostToDevice, s), "inv");
    CUDA_TRY(ctx, stbem::rscale_launch(W.Rv, W.inv, R->d_vprefix, P, W.Q, (long long)n, s), "q0");
    std::vector<double> H((size_t)P * (m + 1) * m, 0.0), cs((size_t)P * m), sn((size_t)P * m),
        g((size_t)P * (m + 1), 0.0);
    std::vector<int> kb(P, 0);
    std::vector<char> done(P, 0);
    for (int p = 0; p < P; ++p) {
      g[(size_t)p * (m + 1)] = active[p] ? rn[p] : 0.0;
      done[p] = !active[p];
    }
    int kmax = 0;
    for (int k = 0; k < m; ++k) {
      for (int p = 0; p < P; ++p) hmask[p] = !done[p];
      CUDA_TRY(ctx, cudaMemcpyAsync(W.mask, hmask, P * sizeof(int), cudaMemcpyHostToDevice, s), "mask");
      if (!R->graphs[k]) {
        // capture step k once; replays read and write the same buffers
        cudaGraph_t graph = nullptr;
        const unsigned long long c0 = stbem_launch_count();
        CUDA_TRY(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "ragged_solve: capture");
        const cudaError_t es = ops.step(k, hh);
        cudaError_t ee = cudaStreamEndCapture(s, &graph);
        if (es != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          return cuda_fail(ctx, es, "ragged_solve: capture step");
        }
        CUDA_TRY(ctx, ee, "ragged_solve: end capture");
        cudaGraphExec_t exec = nullptr;
        ee = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CUDA_TRY(ctx, ee, "ragged_solve: instantiate");
        R->graphs[k] = exec;
        R->graph_kernels[k] = (unsigned)(stbem_launch_count() - c0);
      }
      CUDA_TRY(ctx, cudaGraphLaunch(R->graphs[k], s), "ragged_solve: graph launch");
      stbem::count_launches(R->graph_kernels[k]);
      CUDA_TRY(ctx, cudaStreamSynchronize(s), "ragged_solve: step");
      ++total;
      kmax = k + 1;
      bool all_done = true;
      const double* h1 = hh;
      const double* h2 = hh + (size_t)(k + 1) * P;
      const double* nr = hh + 2 * (size_t)(k + 1) * P;
      for (int p = 0; p < P; ++p) {
        if (done[p]) continue;
        double* Hp = H.data() + (size_t)p * (m + 1) * m;
        double* gp = g.data() + (size_t)p * (m + 1);
        double* cp = cs.data() + (size_t)p * m;
        double* sp = sn.data() + (size_t)p * m;
        std::vector<double> col(k + 2);
        for (int t = 0; t <= k; ++t) col[t] = h1[(size_t)t * P + p] + h2[(size_t)t * P + p];
        const double hk1 = nr[p];
        bool bad = !std::isfinite(hk1);
        for (int t = 0; t <= k; ++t) bad = bad || !std::isfinite(col[t]);
        if (bad) {
          infos[p].status = STBEM_ERR_NAN;
          done[p] = 1;
          kb[p] = 0;
          continue;
        }
        for (int t = 0; t < k; ++t) {
          const double a = cp[t] * col[t] + sp[t] * col[t + 1];
          col[t + 1] = -sp[t] * col[t] + cp[t] * col[t + 1];
          col[t] = a;
        }
        const double den = std::hypot(col[k], hk1);
        if (!(den > 0.0)) {        // zero pivot: singular preconditioned operator
          infos[p].status = STBEM_ERR_BREAKDOWN;
          infos[p].iterations = total;
          done[p] = 1;
          kb[p] = k;
          continue;
        }
        cp[k] = den > 0 ? col[k] / den : 1.0;
        sp[k] = den > 0 ? hk1 / den : 0.0;
        col[k] = den;
        gp[k + 1] = -sp[k] * gp[k];
        gp[k] = cp[k] * gp[k];
        for (int t = 0; t <= k; ++t) Hp[(size_t)t * m + k] = col[t];
        kb[p] = k + 1;
        infos[p].iterations = total;
        if (std::fabs(gp[k + 1]) <= opts->tol * normF[p] || hk1 == 0.0) done[p] = 1;
        all_done = all_done && done[p];
      }
      if (all_done || total >= maxit) break;
    }
    // w += P (Q y) per problem
    std::vector<double> Y((size_t)kmax * P, 0.0);
    for (int p = 0; p < P; ++p) {
      const int kk = kb[p];
      const double* Hp = H.data() + (size_t)p * (m + 1) * m;
      const double* gp = g.data() + (size_t)p * (m + 1);
      std::vector<double> y(kk, 0.0);
      for (int t = kk - 1; t >= 0; --t) {
        double acc = gp[t];
        for (int u = t + 1; u < kk; ++u) acc -= Hp[(size_t)t * m + u] * y[u];
        y[t] = Hp[(size_t)t * m + t] != 0.0 ? acc / Hp[(size_t)t * m + t] : 0.0;
      }
      for (int t = 0; t < kk; ++t) Y[(size_t)t * P + p] = y[t];
    }
    if (kmax > 0) {
      CUDA_TRY(ctx, cudaMemcpyAsync(W.Y, Y.data(), Y.size() * sizeof(double), cudaMemcpyHostToDevice, s), "Y");
      CUDA_TRY(ctx, stbem::rcomb_launch(W.Q, n, kmax, W.Y, R->d_vprefix, P, false, W.U, (long long)n, s), "QY");
      CUDA_TRY(ctx, ops.applyP(W.U, W.Z), "P QY");
      CUDA_TRY(ctx, stbem::axpy_launch(1.0, W.Z, w, n, s), "w += dw");
      CUDA_TRY(ctx, cudaStreamSynchronize(s), "ragged_solve: Y copy");
    }
    // true residual
    CUDA_TRY(ctx, rapply(R, prec, V, w, W.U, W.part, s), "ragged_solve: V w");
    CUDA_TRY(ctx, stbem::sub_launch(f, W.U, W.Rv, n, s), "ragged_solve: r");
  }
  CUDA_TRY(ctx, cudaStreamSynchronize(s), "ragged_solve: finish");
  int worst = STBEM_OK;
  for (int p = 0; p < P; ++p)
    if (infos[p].status != STBEM_OK) worst = infos[p].status;
  if (worst != STBEM_OK) return fail(ctx, worst, "ragged_solve: some problems did not converge");
  return STBEM_OK;
}


int stbem_ragged_solve_mixed_workspace_bytes(const stbem_ragged* R, int restart, size_t* bytes) {
  if (!R || !bytes || restart < 1) return STBEM_ERR_ARG;
  size_t inner = 0;
  const int rc = stbem_ragged_solve_workspace_bytes(R, restart, &inner);
  if (rc != STBEM_OK) return rc;
  const size_t n = (size_t)R->vec_elems, P = (size_t)R->P;
  *bytes = align256(inner) + 2 * align256(n * sizeof(double)) + 2 * align256(P * sizeof(double));
  return STBEM_OK;
}

// FP64 iterative refinement around the lockstep solve: r = f - V64 w with the
// FP64 operators, inner lockstep GMRES on the FP32 operators (V32, D32) for
// the corrections; converged problems get a zero right-hand side, so they
// stop iterating.
int stbem_ragged_solve_mixed(stbem_ctx* ctx, stbem_ragged* R, const double* V64, const float* V32, const float* D32,
                             const double* L, const double* f, double* w, const stbem_solve_opts* opts,
                             double inner_tol, stbem_solve_info* infos, void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!R || !V64 || !V32 || !f || !w || !opts || !infos || !work)
    return fail(ctx, STBEM_ERR_ARG, "ragged_solve_mixed: NULL argument");
  const int m = opts->restart, maxit = opts->max_iter;
  if (m < 1 || maxit < 1 || !(opts->tol > 0) || !(inner_tol > 0) || !(inner_tol < 1))
    return fail(ctx, STBEM_ERR_ARG, "ragged_solve_mixed: bad options");
  size_t need = 0, inner = 0;
  stbem_ragged_solve_mixed_workspace_bytes(R, m, &need);
  stbem_ragged_solve_workspace_bytes(R, m, &inner);
  if (work_bytes < need) return fail(ctx, STBEM_ERR_NOMEM, "ragged_solve_mixed: workspace too small");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "ragged_solve_mixed: set device");
  const int P = R->P;
  const size_t n = (size_t)R->vec_elems;
  char* base = static_cast<char*>(work);
  double* r = reinterpret_cast<double*>(base + align256(inner));
  double* dw = r + align256(n * sizeof(double)) / sizeof(double);
  double* sq = dw + align256(n * sizeof(double)) / sizeof(double);
  double* msk = sq + align256(P * sizeof(double)) / sizeof(double);
  // the FP64 product's partial sums share the inner solve's product scratch
  RWork Wi;
  carve_ragged(work, R, m, &Wi);
  cudaStream_t s = ctx->stream;
  std::vector<double> hv(P);
  auto norms = [&](const double* x, std::vector<double>& out) -> cudaError_t {
    cudaError_t e = stbem::rdots_launch(x, n, 1, x, R->d_vprefix, P, sq, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hv.data(), sq, P * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    out.resize(P);
    for (int p = 0; p < P; ++p) out[p] = std::sqrt(hv[p]);
    return e;
  };
  std::vector<double> normF, rn;
  CUDA_TRY(ctx, norms(f, normF), "ragged_solve_mixed: norm f");
  CUDA_TRY(ctx, cudaMemsetAsync(w, 0, n * sizeof(double), s), "ragged_solve_mixed: w = 0");
  CUDA_TRY(ctx, cudaMemcpyAsync(r, f, n * sizeof(double), cudaMemcpyDeviceToDevice, s), "ragged_solve_mixed: r");
  for (int p = 0; p < P; ++p) {
    infos[p].iterations = 0;
    infos[p].rel_residual = 0.0;
    infos[p].status = std::isfinite(normF[p]) ? STBEM_OK : STBEM_ERR_NAN;
  }
  std::vector<stbem_solve_info> ii(P);
  int total = 0;
  for (int outer = 0; outer < 30; ++outer) {
    CUDA_TRY(ctx, norms(r, rn), "ragged_solve_mixed: norm r");
    bool any = false;
    std::vector<double> keep(P, 0.0);
    for (int p = 0; p < P; ++p) {
      const double rel = normF[p] > 0 ? rn[p] / normF[p] : 0.0;
      if (!std::isfinite(rel) && infos[p].status == STBEM_OK) infos[p].status = STBEM_ERR_NAN;
      infos[p].rel_residual = rel;
      const bool active = infos[p].status == STBEM_OK && rel > opts->tol;
      keep[p] = active ? 1.0 : 0.0;
      any = any || active;
    }
    if (!any) break;
    if (total >= maxit) {
      for (int p = 0; p < P; ++p)
        if (keep[p] != 0.0) infos[p].status = STBEM_ERR_NOCONV;
      break;
    }
    // right-hand sides of the corrections: the active problems' residuals
    CUDA_TRY(ctx, cudaMemcpyAsync(msk, keep.data(), P * sizeof(double), cudaMemcpyHostToDevice, s), "mask");
    CUDA_TRY(ctx, stbem::rscale_launch(r, msk, R->d_vprefix, P, dw, (long long)n, s), "mask r");
    stbem_solve_opts io = *opts;
    io.tol = inner_tol;
    io.max_iter = maxit - total;
    // correction: V32 c = (masked r), right-hand side in dw, c into r
    const int rc = stbem_ragged_solve(ctx, R, STBEM_F32, V32, D32, L, dw, r, &io, ii.data(), base, inner);
    if (rc != STBEM_OK && rc != STBEM_ERR_NOCONV && rc != STBEM_ERR_NAN && rc != STBEM_ERR_BREAKDOWN) return rc;
    int it = 0;
    for (int p = 0; p < P; ++p) {
      if (keep[p] == 0.0) continue;
      it = std::max(it, ii[p].iterations);
      infos[p].iterations += ii[p].iterations;
      if (ii[p].status == STBEM_ERR_NAN || ii[p].status == STBEM_ERR_BREAKDOWN) infos[p].status = ii[p].status;
    }
    total += it;
    CUDA_TRY(ctx, stbem::axpy_launch(1.0, r, w, n, s), "ragged_solve_mixed: w += c");
    CUDA_TRY(ctx, rapply(R, STBEM_F64, V64, w, dw, Wi.part, s), "ragged_solve_mixed: V64 w");
    CUDA_TRY(ctx, stbem::sub_launch(f, dw, r, n, s), "ragged_solve_mixed: r = f - V64 w");
    if (it == 0) {
      for (int p = 0; p < P; ++p)
        if (keep[p] != 0.0 && infos[p].status == STBEM_OK) infos[p].status = STBEM_ERR_NOCONV;
      break;
    }
  }
  CUDA_TRY(ctx, cudaStreamSynchronize(s), "ragged_solve_mixed: finish");
  int worst = STBEM_OK;
  for (int p = 0; p < P; ++p)
    if (infos[p].status != STBEM_OK) worst = infos[p].status;
  if (worst != STBEM_OK) return fail(ctx, worst, "ragged_solve_mixed: some problems did not converge");
  return STBEM_OK;
}

}  // extern "C"
