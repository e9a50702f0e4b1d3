// Internal definitions shared by the translation units of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "assemble.h"
#include "stbem.h"

struct stbem_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  // stbem_assemble_ops: two side streams and three events, created on first use
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  ~stbem_ctx() {
    for (auto& st : side)
      if (st) cudaStreamDestroy(st);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};

struct stbem_mesh {
  int device = 0;
  int N = 0, n_t = 0;
  double T = 0, ht = 0, alpha = 0;
  std::vector<double> h;     // segment lengths (host copy)
  std::vector<double> xy;    // vertices (host copy, 2 N)
  double* dbuf = nullptr;    // device geometry
  int* ibuf = nullptr;
  double* sbuf = nullptr;    // lag-0/1 singular-pair moments, one slice per operator (V, K, D: 2 lags x 3 x 2N x 5)
  double* tbuf = nullptr;    // the n_t + 1 time nodes (uniform k T / n_t unless graded)
  std::vector<double> tnodes;  // host copy of a graded mesh's nodes
  bool graded = false;       // non-uniform time grid: only the stbem_nu_* calls apply
  stbem::DevMesh dev{};
};

namespace stbem_internal {

// doubles of one operator's slice of the singular-pair scratch
inline size_t sing_slice(int N) { return (size_t)2 * 3 * (2 * N) * 5; }

// the mesh's device view for assembling operator op: its own slice of the
// singular-pair scratch, so that the three operators may be assembled
// concurrently
inline stbem::DevMesh op_dev(const stbem_mesh* m, int op) {
  stbem::DevMesh d = m->dev;
  d.sing = m->sbuf + (size_t)op * sing_slice(m->N);
  return d;
}

inline int fail(stbem_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

inline int cuda_fail(stbem_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, STBEM_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// The uniform-grid calls (Toeplitz lag blocks) reject a mesh with a
// non-uniform time grid; its operators are the packed blocks of stbem_nu_*.
inline int reject_graded(stbem_ctx* ctx, const stbem_mesh* m, const char* name) {
  if (m && m->graded)
    return fail(ctx, STBEM_ERR_ARG, "%s: the mesh has a non-uniform time grid (use the stbem_nu_* calls)", name);
  return STBEM_OK;
}

}  // namespace stbem_internal

#define CUDA_TRY(ctx, call, where)                                                  \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return stbem_internal::cuda_fail(ctx, e_, where);        \
  } while (0)
