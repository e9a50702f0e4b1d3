// C ABI of the library (declared in include/stbem.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "assemble.h"
#include "capi_internal.h"
#include "shard_host.h"
#include "stbem.h"
#include "toeplitz.h"
#include "grad.h"
#include "initial.h"
#include "mass_host.h"
#include "toeplitz_fft.h"
#include "toeplitz_tc.h"
#include "tune_cache.h"
#include "vec.h"

using stbem_internal::cuda_fail;
using stbem_internal::fail;
using stbem_internal::reject_graded;

namespace {

size_t elt_size(int prec) { return prec == STBEM_F64 ? 8 : 4; }

}  // namespace

extern "C" {

const char* stbem_version(void) { return "stbem 0.1 (sm_103a)"; }

unsigned long long stbem_launch_count(void) { return stbem::launch_count(); }

int stbem_create(stbem_ctx** out, int device, void* stream) {
  if (!out) return STBEM_ERR_ARG;
  *out = nullptr;
  stbem_ctx* ctx = new stbem_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete ctx;
    return STBEM_ERR_CUDA;
  }
  stbem::RuleTables t;
  stbem::build_rule_tables(&t);
  e = stbem::upload_rule_tables(t, ctx->stream);
  if (e == cudaSuccess) e = stbem::upload_grad_rule_tables(t, ctx->stream);
  if (e == cudaSuccess) e = stbem::upload_m0_rule_tables(t, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    delete ctx;
    return STBEM_ERR_CUDA;
  }
  *out = ctx;
  return STBEM_OK;
}

void stbem_destroy(stbem_ctx* ctx) { delete ctx; }

const char* stbem_last_error(const stbem_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

int stbem_mesh_create(stbem_ctx* ctx, const double* xy, int n_x, double T, int n_t, double alpha,
                      stbem_mesh** out) {
  if (!ctx || !out) return STBEM_ERR_ARG;
  *out = nullptr;
  if (!xy) return fail(ctx, STBEM_ERR_ARG, "mesh: NULL vertex array");
  if (n_x < 3) return fail(ctx, STBEM_ERR_ARG, "mesh: need n_x >= 3 (got %d)", n_x);
  if (n_t < 1) return fail(ctx, STBEM_ERR_ARG, "mesh: need n_t >= 1 (got %d)", n_t);
  if (!(T > 0) || !std::isfinite(T)) return fail(ctx, STBEM_ERR_ARG, "mesh: need T > 0");
  if (!(alpha > 0) || !std::isfinite(alpha)) return fail(ctx, STBEM_ERR_ARG, "mesh: need alpha > 0");
  const int N = n_x;
  std::vector<double> ax(N), ay(N), bx(N), by(N), h(N), nx(N), ny(N);
  double area2 = 0.0;
  for (int i = 0; i < N; ++i) {
    const int k = (i + 1) % N;
    ax[i] = xy[2 * i];
    ay[i] = xy[2 * i + 1];
    bx[i] = xy[2 * k];
    by[i] = xy[2 * k + 1];
    if (!std::isfinite(ax[i]) || !std::isfinite(ay[i])) return fail(ctx, STBEM_ERR_ARG, "mesh: non-finite vertex %d", i);
    const double ex = bx[i] - ax[i], ey = by[i] - ay[i];
    h[i] = std::sqrt(ex * ex + ey * ey);
    if (!(h[i] > 0)) return fail(ctx, STBEM_ERR_ARG, "mesh: zero-length segment %d", i);
    const double tx = ex / h[i], ty = ey / h[i];
    nx[i] = ty;
    ny[i] = -tx;
    area2 += ax[i] * by[i] - bx[i] * ay[i];
  }
  if (!(area2 > 0)) return fail(ctx, STBEM_ERR_ARG, "mesh: vertices must be counter-clockwise");
  const int M2 = 2 * N;
  std::vector<double> hx0(M2), hy0(M2), hx1(M2), hy1(M2), hl(M2), hnx(M2), hny(M2);
  for (int i = 0; i < N; ++i) {
    const double mx = 0.5 * (ax[i] + bx[i]), my = 0.5 * (ay[i] + by[i]);
    hx0[2 * i] = ax[i]; hy0[2 * i] = ay[i]; hx1[2 * i] = mx; hy1[2 * i] = my;
    hx0[2 * i + 1] = mx; hy0[2 * i + 1] = my; hx1[2 * i + 1] = bx[i]; hy1[2 * i + 1] = by[i];
    hl[2 * i] = hl[2 * i + 1] = 0.5 * h[i];
    hnx[2 * i] = hnx[2 * i + 1] = nx[i];
    hny[2 * i] = hny[2 * i + 1] = ny[i];
  }
  std::vector<int> dp(4 * N);
  std::vector<double> dv0(4 * N), dv1(4 * N), dc(4 * N);
  for (int l = 0; l < N; ++l) {
    const double hm = h[(l - 1 + N) % N], h0 = h[l], hp = h[(l + 1) % N];
    const double al = hm / (hm + h0), bl = hp / (h0 + hp);
    const double up = 2.0 / (hm + h0), dn = -2.0 / (h0 + hp);
    const int p[4] = {(2 * l - 1 + M2) % M2, (2 * l) % M2, (2 * l + 1) % M2, (2 * l + 2) % M2};
    const double v0[4] = {0.0, al, 1.0, bl}, v1[4] = {al, 1.0, bl, 0.0}, c[4] = {up, up, dn, dn};
    for (int k = 0; k < 4; ++k) {
      dp[4 * l + k] = p[k];
      dv0[4 * l + k] = v0[k];
      dv1[4 * l + k] = v1[k];
      dc[4 * l + k] = c[k];
    }
  }
  // pack: seg 7N | half 7*2N | dual 3*4N | vertices 2N
  std::vector<double> host;
  host.reserve(7 * N + 14 * N + 12 * N + 2 * N);
  for (auto* v : {&ax, &ay, &bx, &by, &h, &nx, &ny}) host.insert(host.end(), v->begin(), v->end());
  for (auto* v : {&hx0, &hy0, &hx1, &hy1, &hl, &hnx, &hny}) host.insert(host.end(), v->begin(), v->end());
  for (auto* v : {&dv0, &dv1, &dc}) host.insert(host.end(), v->begin(), v->end());
  host.insert(host.end(), ax.begin(), ax.end());
  host.insert(host.end(), ay.begin(), ay.end());

  stbem_mesh* m = new stbem_mesh();
  m->device = ctx->device;
  m->N = N;
  m->n_t = n_t;
  m->T = T;
  m->ht = T / n_t;
  m->alpha = alpha;
  m->h = h;
  m->xy.assign(xy, xy + 2 * N);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&m->dbuf, host.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->ibuf, dp.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&m->sbuf, 3 * stbem_internal::sing_slice(N) * sizeof(double));
  std::vector<double> tn(n_t + 1);
  for (int k = 0; k <= n_t; ++k) tn[k] = k == n_t ? T : (double)k * m->ht;
  if (e == cudaSuccess) e = cudaMalloc(&m->tbuf, tn.size() * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->tbuf, tn.data(), tn.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->dbuf, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->ibuf, dp.data(), dp.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    if (m->dbuf) cudaFree(m->dbuf);
    if (m->ibuf) cudaFree(m->ibuf);
    if (m->sbuf) cudaFree(m->sbuf);
    if (m->tbuf) cudaFree(m->tbuf);
    delete m;
    return cuda_fail(ctx, e, "mesh upload");
  }
  const double* b = m->dbuf;
  stbem::DevMesh& D = m->dev;
  D.N = N; D.n_t = n_t; D.ht = m->ht; D.alpha = alpha;
  D.sx0 = b; D.sy0 = b + N; D.sx1 = b + 2 * N; D.sy1 = b + 3 * N; D.slen = b + 4 * N; D.snx = b + 5 * N; D.sny = b + 6 * N;
  b += 7 * N;
  D.hx0 = b; D.hy0 = b + M2; D.hx1 = b + 2 * M2; D.hy1 = b + 3 * M2; D.hlen = b + 4 * M2; D.hnx = b + 5 * M2; D.hny = b + 6 * M2;
  b += 7 * M2;
  D.dv0 = b; D.dv1 = b + 4 * N; D.dcurl = b + 8 * N;
  b += 12 * N;
  D.vx = b; D.vy = b + N;
  D.dpiece = m->ibuf;
  D.sing = m->sbuf;
  *out = m;
  return STBEM_OK;
}

void stbem_mesh_destroy(stbem_mesh* m) {
  if (!m) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(m->device);
  if (m->dbuf) cudaFree(m->dbuf);
  if (m->ibuf) cudaFree(m->ibuf);
  if (m->sbuf) cudaFree(m->sbuf);
  if (m->tbuf) cudaFree(m->tbuf);
  cudaSetDevice(prev);
  delete m;
}

int stbem_mesh_create_graded(stbem_ctx* ctx, const double* xy, int n_x, const double* t, int n_t, double alpha,
                             stbem_mesh** out) {
  if (!ctx || !out) return STBEM_ERR_ARG;
  *out = nullptr;
  if (!t) return fail(ctx, STBEM_ERR_ARG, "mesh_graded: NULL time nodes");
  if (n_t < 1) return fail(ctx, STBEM_ERR_ARG, "mesh_graded: need n_t >= 1 (got %d)", n_t);
  if (t[0] != 0.0) return fail(ctx, STBEM_ERR_ARG, "mesh_graded: t_0 must be 0");
  for (int k = 0; k < n_t; ++k)
    if (!(t[k + 1] > t[k]) || !std::isfinite(t[k + 1]))
      return fail(ctx, STBEM_ERR_ARG, "mesh_graded: time nodes must increase (t_%d = %g, t_%d = %g)", k, t[k],
                  k + 1, t[k + 1]);
  stbem_mesh* m = nullptr;
  const int rc = stbem_mesh_create(ctx, xy, n_x, t[n_t], n_t, alpha, &m);
  if (rc != STBEM_OK) return rc;
  const cudaError_t e = cudaMemcpyAsync(m->tbuf, t, (size_t)(n_t + 1) * sizeof(double), cudaMemcpyHostToDevice,
                                        ctx->stream);
  const cudaError_t e2 = e == cudaSuccess ? cudaStreamSynchronize(ctx->stream) : e;
  if (e2 != cudaSuccess) {
    stbem_mesh_destroy(m);
    return cuda_fail(ctx, e2, "mesh_graded: time nodes");
  }
  m->graded = true;
  m->tnodes.assign(t, t + n_t + 1);
  *out = m;
  return STBEM_OK;
}

int stbem_op_bytes(const stbem_mesh* m, int op, int prec, size_t* bytes) {
  if (!m || !bytes || op < 0 || op > 2 || (prec != STBEM_F64 && prec != STBEM_F32)) return STBEM_ERR_ARG;
  *bytes = (size_t)m->n_t * m->N * m->N * elt_size(prec);
  return STBEM_OK;
}

int stbem_assemble(stbem_ctx* ctx, const stbem_mesh* m, int op, int prec, void* out) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rg = reject_graded(ctx, m, "assemble")) return rg;
  if (!m || !out) return fail(ctx, STBEM_ERR_ARG, "assemble: NULL mesh or output");
  if (op < 0 || op > 2) return fail(ctx, STBEM_ERR_ARG, "assemble: unknown operator %d", op);
  if (prec != STBEM_F64 && prec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "assemble: unknown precision %d", prec);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "assemble: set device");
  CUDA_TRY(ctx, stbem::assemble_launch(stbem_internal::op_dev(m, op), op, prec, 0, m->n_t, out, ctx->stream),
           "assemble: launch");
  return STBEM_OK;
}

int stbem_assemble_ops(stbem_ctx* ctx, const stbem_mesh* m, int prec_V, int prec_K, int prec_D, void* V, void* K,
                       void* D) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rg = reject_graded(ctx, m, "assemble_ops")) return rg;
  if (!m || (!V && !K && !D)) return fail(ctx, STBEM_ERR_ARG, "assemble_ops: NULL mesh or no output");
  const int precs[3] = {prec_V, prec_K, prec_D};
  for (int op = 0; op < 3; ++op)
    if (precs[op] != STBEM_F64 && precs[op] != STBEM_F32)
      return fail(ctx, STBEM_ERR_ARG, "assemble_ops: unknown precision %d", precs[op]);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "assemble_ops: set device");
  for (int k = 0; k < 2; ++k)
    if (!ctx->side[k]) CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking), "assemble_ops: stream");
  for (int k = 0; k < 3; ++k)
    if (!ctx->ev[k]) CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev[k], cudaEventDisableTiming), "assemble_ops: event");
  // D (the largest) on the caller's stream, K and V on the side streams, which
  // first wait for the caller's earlier work and are joined back at the end
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev[0], ctx->stream), "assemble_ops: fork");
  void* outs[3] = {V, K, D};
  const cudaStream_t streams[3] = {ctx->side[1], ctx->side[0], ctx->stream};
  for (int op = 2; op >= 0; --op) {
    if (!outs[op]) continue;
    if (streams[op] != ctx->stream) CUDA_TRY(ctx, cudaStreamWaitEvent(streams[op], ctx->ev[0], 0), "assemble_ops: wait");
    CUDA_TRY(ctx, stbem::assemble_launch(stbem_internal::op_dev(m, op), op, precs[op], 0, m->n_t, outs[op], streams[op]),
             "assemble_ops: launch");
  }
  for (int op = 0; op < 2; ++op) {
    if (!outs[op]) continue;
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev[1 + op], streams[op]), "assemble_ops: join");
    CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev[1 + op], 0), "assemble_ops: join");
  }
  return STBEM_OK;
}

int stbem_assemble_lags(stbem_ctx* ctx, const stbem_mesh* m, int op, int prec, int lag_begin, int lag_end,
                        void* out) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rg = reject_graded(ctx, m, "assemble_lags")) return rg;
  if (!m || !out) return fail(ctx, STBEM_ERR_ARG, "assemble_lags: NULL mesh or output");
  if (op < 0 || op > 2) return fail(ctx, STBEM_ERR_ARG, "assemble_lags: unknown operator %d", op);
  if (prec != STBEM_F64 && prec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "assemble_lags: unknown precision %d", prec);
  if (lag_begin < 0 || lag_end > m->n_t || lag_begin > lag_end)
    return fail(ctx, STBEM_ERR_ARG, "assemble_lags: lag range [%d, %d) outside [0, %d)", lag_begin, lag_end, m->n_t);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "assemble_lags: set device");
  CUDA_TRY(ctx, stbem::assemble_launch(stbem_internal::op_dev(m, op), op, prec, lag_begin, lag_end, out, ctx->stream),
           "assemble_lags");
  return STBEM_OK;
}

int stbem_apply_workspace_bytes(int n_t, int n_x, int n_rhs, int prec, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || n_rhs < 1 || (prec != STBEM_F64 && prec != STBEM_F32)) return STBEM_ERR_ARG;
  *bytes = stbem::apply_workspace_bytes(n_t, n_x, n_rhs);
  return STBEM_OK;
}

int stbem_apply(stbem_ctx* ctx, int prec, int transpose, int n_t, int n_x, const void* A, int n_rhs,
                const double* x, double* y, void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!A || !x || !y || !work) return fail(ctx, STBEM_ERR_ARG, "apply: NULL pointer");
  if (n_t < 1 || n_x < 1 || n_rhs < 1) return fail(ctx, STBEM_ERR_ARG, "apply: bad sizes");
  if (prec != STBEM_F64 && prec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "apply: bad precision");
  if ((const void*)x == (const void*)y) return fail(ctx, STBEM_ERR_ARG, "apply: x and y overlap");
  if (!stbem::apply_grid_fits(n_t, n_x, n_rhs))
    return fail(ctx, STBEM_ERR_ARG, "apply: n_rhs x time tiles exceeds the grid limit 65535; split the right-hand sides");
  const size_t need = stbem::apply_workspace_bytes(n_t, n_x, n_rhs);
  if (work_bytes < need) return fail(ctx, STBEM_ERR_NOMEM, "apply: workspace %zu < %zu bytes", work_bytes, need);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "apply: set device");
  CUDA_TRY(ctx, stbem::apply_launch(prec, transpose != 0, n_t, n_x, A, n_rhs, x, y, work, ctx->stream), "apply");
  return STBEM_OK;
}

int stbem_apply_noalloc(stbem_ctx* ctx, int prec, int transpose, int n_t, int n_x, const void* A,
                        int n_rhs, const double* x, double* y) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!A || !x || !y) return fail(ctx, STBEM_ERR_ARG, "apply_noalloc: NULL pointer");
  if (n_t < 1 || n_x < 1 || n_rhs < 1) return fail(ctx, STBEM_ERR_ARG, "apply_noalloc: bad sizes");
  if (prec != STBEM_F64 && prec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "apply_noalloc: bad precision");
  if ((const void*)x == (const void*)y) return fail(ctx, STBEM_ERR_ARG, "apply_noalloc: x and y overlap");
  if (!stbem::apply_grid_fits(n_t, n_x, n_rhs))
    return fail(ctx, STBEM_ERR_ARG,
                "apply_noalloc: n_rhs x time tiles exceeds the grid limit 65535; split the right-hand sides");
  const size_t need = stbem::apply_workspace_bytes(n_t, n_x, n_rhs);
  if (need > stbem::kNoAllocScratchBytes)
    return fail(ctx, STBEM_ERR_NOMEM,
                "apply_noalloc: this product needs %zu bytes of scratch but the fixed scratch holds %zu; "
                "use stbem_apply with a caller workspace", need, stbem::kNoAllocScratchBytes);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "apply_noalloc: set device");
  void* scratch = nullptr;
  CUDA_TRY(ctx, stbem::noalloc_scratch_ptr(ctx->device, &scratch), "apply_noalloc: scratch address");
  CUDA_TRY(ctx, stbem::apply_launch(prec, transpose != 0, n_t, n_x, A, n_rhs, x, y, scratch, ctx->stream),
           "apply_noalloc");
  return STBEM_OK;
}

int stbem_to_bf16(stbem_ctx* ctx, int src_prec, size_t n, const void* src, void* dst) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!src || !dst) return fail(ctx, STBEM_ERR_ARG, "to_bf16: NULL pointer");
  if (src_prec != STBEM_F64 && src_prec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "to_bf16: bad precision");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "to_bf16: set device");
  CUDA_TRY(ctx, stbem::to_bf16_launch(src_prec, src, dst, n, ctx->stream), "to_bf16");
  return STBEM_OK;
}

namespace {
int apply_tc_entry(stbem_ctx* ctx, const char* name, int n_t, int n_x, const void* A, int n_rhs, const void* x,
                   double* y, int chunk) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!A || !x || !y) return fail(ctx, STBEM_ERR_ARG, "%s: NULL pointer", name);
  if (!stbem::apply_tc_supported(n_t, n_x, n_rhs))
    return fail(ctx, STBEM_ERR_ARG, "%s: unsupported sizes n_t=%d n_x=%d n_rhs=%d (need n_x %% 8 == 0)", name, n_t,
                n_x, n_rhs);
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(x)) & 15)
    return fail(ctx, STBEM_ERR_ARG, "%s: A and x must be 16-byte aligned", name);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "apply_tc: set device");
  CUDA_TRY(ctx, stbem::tc_error_reset(ctx->stream), "apply_tc: reset error word");
  CUDA_TRY(ctx, stbem::apply_tc_launch(n_t, n_x, A, n_rhs, x, y, false, ctx->stream, chunk), "apply_tc");
  int flag = 0;
  CUDA_TRY(ctx, stbem::tc_error_read(&flag, ctx->stream), "apply_tc: read error word");
  if (flag) return fail(ctx, STBEM_ERR_TIMEOUT, "%s: a pipeline wait timed out", name);
  return STBEM_OK;
}
}  // namespace

int stbem_apply_tc(stbem_ctx* ctx, int n_t, int n_x, const void* A, int n_rhs, const void* x, double* y) {
  return apply_tc_entry(ctx, "apply_tc", n_t, n_x, A, n_rhs, x, y, 0);
}

int stbem_pipe_peaks(stbem_ctx* ctx, double* host_out) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!host_out) return fail(ctx, STBEM_ERR_ARG, "pipe_peaks: NULL pointer");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "pipe_peaks: set device");
  CUDA_TRY(ctx, stbem::pipe_peaks(host_out, ctx->stream), "pipe_peaks");
  return STBEM_OK;
}

int stbem_debug_tc_stall(int stall, long long wait_cycles) {
  if (stall && wait_cycles < 1024) return STBEM_ERR_ARG;
  stbem::tc_set_stall(stall ? wait_cycles : 0);
  return STBEM_OK;
}

int stbem_apply_tc_comp(stbem_ctx* ctx, int n_t, int n_x, const void* A, int n_rhs, const void* x, double* y,
                        int chunk) {
  if (ctx && chunk < 1) return fail(ctx, STBEM_ERR_ARG, "apply_tc_comp: chunk must be >= 1");
  return apply_tc_entry(ctx, "apply_tc_comp", n_t, n_x, A, n_rhs, x, y, chunk);
}


int stbem_bf16_split3(stbem_ctx* ctx, size_t n, const double* src, void* hi, void* mid, void* lo) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!src || !hi) return fail(ctx, STBEM_ERR_ARG, "bf16_split3: NULL pointer");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "bf16_split3: set device");
  CUDA_TRY(ctx, stbem::bf16_split3_launch(src, hi, mid, lo, n, ctx->stream), "bf16_split3");
  return STBEM_OK;
}

namespace {
// 64-wide K steps per FP32 partial in the accurate products.  Each K step is
// four MMAs, and each MMA adds about 0.7 u (u = 2^-24) of its partial's
// magnitude in error (measured on GB300: the error of one long FP32 chain
// grows linearly with its length), so the hi x hi product, which carries the
// whole magnitude, uses short partials and the five products that are 2^-8
// smaller or less use long ones.
constexpr int kTc3ChunkHi = 4;
constexpr int kTc3ChunkLo = 16;

// y = sum over slice pairs (s, t), s + t <= 2, of A_s x_t on the tensor cores,
// with x split into three BF16 slices in `xs` (3 n_rhs n_t n_x BF16), each
// product Kahan-accumulated over FP32 partials.
// part (optional, stbem::exact_part_bytes()): with few output tiles the
// products split each tile's lags into chunks, accumulated there and summed
// into y at the end.
cudaError_t apply_tc3(int nt, int nx, const void* const A[3], int B, const double* x, double* y, void* xs,
                      cudaStream_t s, double* part = nullptr) {
  const size_t n = (size_t)B * nt * nx;
  char* base = static_cast<char*>(xs);
  void* X[3] = {base, base + n * 2, base + 2 * n * 2};
  cudaError_t e = stbem::bf16_split3_launch(x, X[0], X[1], X[2], n, s);
  if (e != cudaSuccess) return e;
  bool first = true;
  for (int sa = 0; sa < 3; ++sa)
    for (int sx = 0; sx + sa < 3; ++sx) {
      if (!A[sa]) continue;
      e = stbem::apply_tc_launch(nt, nx, A[sa], B, X[sx], y, !first, s,
                                 sa + sx == 0 ? kTc3ChunkHi : kTc3ChunkLo, 0, part);
      if (e != cudaSuccess) return e;
      first = false;
    }
  return part ? stbem::tc_chunk_reduce_launch(nt, nx, B, part, y, s) : cudaSuccess;
}

// workspace of apply_tc3 with lag chunks: three slices of x, then the partials
size_t tc3_bytes(int nt, int nx, int B) {
  const size_t x3 = ((3 * (size_t)B * nt * nx * 2 + 255) & ~(size_t)255);
  return x3 + stbem::exact_part_bytes(nt, nx, B);
}
double* tc3_part(void* work, int nt, int nx, int B) {
  if (stbem::exact_part_bytes(nt, nx, B) == 0) return nullptr;
  return reinterpret_cast<double*>(static_cast<char*>(work) + ((3 * (size_t)B * nt * nx * 2 + 255) & ~(size_t)255));
}
}  // namespace

int stbem_apply_tc3_workspace_bytes(int n_t, int n_x, int n_rhs, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || n_rhs < 1) return STBEM_ERR_ARG;
  *bytes = tc3_bytes(n_t, n_x, n_rhs);
  return STBEM_OK;
}

int stbem_apply_tc3(stbem_ctx* ctx, int n_t, int n_x, const void* A_hi, const void* A_mid, const void* A_lo,
                    int n_rhs, const double* x, double* y, void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!A_hi || !x || !y || !work) return fail(ctx, STBEM_ERR_ARG, "apply_tc3: NULL pointer");
  if (!stbem::apply_tc_supported(n_t, n_x, n_rhs)) return fail(ctx, STBEM_ERR_ARG, "apply_tc3: unsupported sizes");
  if (work_bytes < tc3_bytes(n_t, n_x, n_rhs)) return fail(ctx, STBEM_ERR_NOMEM, "apply_tc3: workspace too small");
  if (reinterpret_cast<uintptr_t>(work) & 255) return fail(ctx, STBEM_ERR_ARG, "apply_tc3: workspace not 256-byte aligned");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "apply_tc3: set device");
  CUDA_TRY(ctx, stbem::tc_error_reset(ctx->stream), "apply_tc3: reset error word");
  const void* A[3] = {A_hi, A_mid, A_lo};
  CUDA_TRY(ctx, apply_tc3(n_t, n_x, A, n_rhs, x, y, work, ctx->stream, tc3_part(work, n_t, n_x, n_rhs)), "apply_tc3");
  int flag = 0;
  CUDA_TRY(ctx, stbem::tc_error_read(&flag, ctx->stream), "apply_tc3: read error word");
  if (flag) return fail(ctx, STBEM_ERR_TIMEOUT, "apply_tc3: a pipeline wait timed out");
  return STBEM_OK;
}

// ------------------------------------------------- tuned launch parameters ----
int stbem_tune_cache_path(const char* path) {
  return stbem::tune_cache_set_path(path) ? STBEM_OK : STBEM_ERR_ARG;
}

int stbem_tune_cache_get(const char* key, char* value, size_t cap) {
  if (!key || !value || cap == 0) return STBEM_ERR_ARG;
  std::string v;
  if (!stbem::tune_cache_get(key, &v)) return STBEM_ERR_ARG;
  if (v.size() + 1 > cap) return STBEM_ERR_NOMEM;
  std::memcpy(value, v.c_str(), v.size() + 1);
  return STBEM_OK;
}

int stbem_tune_cache_put(const char* key, const char* value) {
  if (!key || !value || !stbem::tune_cache_token_ok(key) || !stbem::tune_cache_token_ok(value)) return STBEM_ERR_ARG;
  return stbem::tune_cache_put(key, value) ? STBEM_OK : STBEM_ERR_ARG;   // the backing file cannot be written
}

int stbem_tune_cache_clear(void) {
  stbem::tune_cache_clear();
  return STBEM_OK;
}

int stbem_tc_tune(stbem_ctx* ctx, int n_t, int n_x, const void* A, int n_rhs, const void* x, double* y, int* tile_n,
                  int* from_cache) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!A || !x || !y) return fail(ctx, STBEM_ERR_ARG, "tc_tune: NULL pointer");
  if (!stbem::apply_tc_supported(n_t, n_x, n_rhs))
    return fail(ctx, STBEM_ERR_ARG, "tc_tune: unsupported sizes n_t=%d n_x=%d n_rhs=%d", n_t, n_x, n_rhs);
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(x)) & 15)
    return fail(ctx, STBEM_ERR_ARG, "tc_tune: A and x must be 16-byte aligned");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "tc_tune: set device");
  const std::string key = stbem::tc_plain_tune_key(n_t, n_x, n_rhs);
  std::string v;
  if (stbem::tune_cache_get(key, &v) && (v == "bn=128" || (v == "bn=256" && n_t > 128))) {
    if (tile_n) *tile_n = v == "bn=128" ? 128 : 256;
    if (from_cache) *from_cache = 1;
    return STBEM_OK;
  }
  cudaStream_t s = ctx->stream;
  CUDA_TRY(ctx, stbem::tc_error_reset(s), "tc_tune: reset error word");
  cudaEvent_t e0, e1;
  CUDA_TRY(ctx, cudaEventCreate(&e0), "tc_tune: event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(ctx, STBEM_ERR_CUDA, "tc_tune: event");
  }
  int best = 0;
  float best_ms = 0.f;
  cudaError_t e = cudaSuccess;
  for (int bn : {128, 256}) {
    if (bn == 256 && n_t <= 128) break;    // one tile covers every step
    float ms = 0.f;
    e = stbem::apply_tc_launch(n_t, n_x, A, n_rhs, x, y, false, s, 0, bn);   // warm-up
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = stbem::apply_tc_launch(n_t, n_x, A, n_rhs, x, y, false, s, 0, bn);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      ms = r == 0 ? t : std::min(ms, t);
    }
    if (e != cudaSuccess) break;
    if (best == 0 || ms < best_ms) {
      best = bn;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tc_tune: product");
  int flag = 0;
  CUDA_TRY(ctx, stbem::tc_error_read(&flag, s), "tc_tune: read error word");
  if (flag) return fail(ctx, STBEM_ERR_TIMEOUT, "tc_tune: a pipeline wait timed out");
  if (!stbem::tune_cache_put(key, best == 128 ? "bn=128" : "bn=256"))
    return fail(ctx, STBEM_ERR_ARG, "tc_tune: cannot write the tune cache file %s", stbem::tune_cache_path().c_str());
  if (tile_n) *tile_n = best;
  if (from_cache) *from_cache = 0;
  return STBEM_OK;
}

// ------------------------------------------------ exact-slice products ------
namespace {
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// workspace of the x side of an exact product: S slices of n values, n / n_x
// exponents, then (few output tiles) the lag-chunk partial products
size_t exact_x_bytes(int nt, int nx, int B, int S) {
  const size_t n = (size_t)B * nt * nx;
  return align256(align256((size_t)S * n * 2) + (size_t)B * nt * sizeof(int)) + stbem::exact_part_bytes(nt, nx, B);
}

int check_exact_operand(stbem_ctx* ctx, const char* name, const stbem_exact_operand* A) {
  if (!A || !A->slices || !A->row_exp) return fail(ctx, STBEM_ERR_ARG, "%s: NULL operand", name);
  if (A->n_slices < stbem::kExactMinSlices || A->n_slices > stbem::kExactMaxSlices)
    return fail(ctx, STBEM_ERR_ARG, "%s: n_slices must be in %d..%d", name, stbem::kExactMinSlices,
                stbem::kExactMaxSlices);
  if (reinterpret_cast<uintptr_t>(A->slices) & 15) return fail(ctx, STBEM_ERR_ARG, "%s: slices not 16-byte aligned", name);
  return STBEM_OK;
}

// y = A x with x in FP64: slice x into `work`, then the exact product
cudaError_t apply_exact(int nt, int nx, const stbem_exact_operand& A, int B, const double* x, double* y, void* work,
                        cudaStream_t s) {
  const int S = A.n_slices;
  const size_t n = (size_t)B * nt * nx;
  void* xs = work;
  int* xe = reinterpret_cast<int*>(static_cast<char*>(work) + align256((size_t)S * n * 2));
  double* part = stbem::exact_part_bytes(nt, nx, B) > 0
                     ? reinterpret_cast<double*>(static_cast<char*>(work) +
                                                 align256(align256((size_t)S * n * 2) + (size_t)B * nt * sizeof(int)))
                     : nullptr;
  cudaError_t e = stbem::exact_slices_launch(x, (long long)B * nt, nx, S, xs, xe, s);
  if (e == cudaSuccess) e = stbem::apply_tc_exact_launch(nt, nx, S, A.slices, A.row_exp, B, xs, xe, y, s, part);
  return e;
}
}  // namespace

int stbem_exact_slices(stbem_ctx* ctx, long long rows, int cols, int n_slices, const double* src, void* slices,
                       int* row_exp) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!src || !slices || !row_exp) return fail(ctx, STBEM_ERR_ARG, "exact_slices: NULL pointer");
  if (rows < 0 || cols < 1 || n_slices < stbem::kExactMinSlices || n_slices > stbem::kExactMaxSlices)
    return fail(ctx, STBEM_ERR_ARG, "exact_slices: bad sizes rows=%lld cols=%d n_slices=%d", rows, cols, n_slices);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "exact_slices: set device");
  CUDA_TRY(ctx, stbem::exact_slices_launch(src, rows, cols, n_slices, slices, row_exp, ctx->stream), "exact_slices");
  return STBEM_OK;
}

int stbem_apply_tc_exact(stbem_ctx* ctx, int n_t, int n_x, const stbem_exact_operand* A, int n_rhs,
                         const stbem_exact_operand* x, double* y) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int r = check_exact_operand(ctx, "apply_tc_exact", A)) return r;
  if (const int r = check_exact_operand(ctx, "apply_tc_exact", x)) return r;
  if (!y) return fail(ctx, STBEM_ERR_ARG, "apply_tc_exact: NULL pointer");
  if (x->n_slices != A->n_slices) return fail(ctx, STBEM_ERR_ARG, "apply_tc_exact: A and x differ in n_slices");
  if (!stbem::apply_tc_exact_supported(n_t, n_x, n_rhs, A->n_slices))
    return fail(ctx, STBEM_ERR_ARG, "apply_tc_exact: unsupported sizes n_t=%d n_x=%d n_rhs=%d", n_t, n_x, n_rhs);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "apply_tc_exact: set device");
  CUDA_TRY(ctx, stbem::tc_error_reset(ctx->stream), "apply_tc_exact: reset error word");
  CUDA_TRY(ctx, stbem::apply_tc_exact_launch(n_t, n_x, A->n_slices, A->slices, A->row_exp, n_rhs, x->slices,
                                             x->row_exp, y, ctx->stream),
           "apply_tc_exact");
  int flag = 0;
  CUDA_TRY(ctx, stbem::tc_error_read(&flag, ctx->stream), "apply_tc_exact: read error word");
  if (flag) return fail(ctx, STBEM_ERR_TIMEOUT, "apply_tc_exact: a pipeline wait timed out");
  return STBEM_OK;
}

int stbem_apply_exact_workspace_bytes(int n_t, int n_x, int n_rhs, int n_slices, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || n_rhs < 1 || n_slices < stbem::kExactMinSlices ||
      n_slices > stbem::kExactMaxSlices)
    return STBEM_ERR_ARG;
  *bytes = exact_x_bytes(n_t, n_x, n_rhs, n_slices);
  return STBEM_OK;
}

int stbem_apply_exact(stbem_ctx* ctx, int n_t, int n_x, const stbem_exact_operand* A, int n_rhs, const double* x,
                      double* y, void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int r = check_exact_operand(ctx, "apply_exact", A)) return r;
  if (!x || !y || !work) return fail(ctx, STBEM_ERR_ARG, "apply_exact: NULL pointer");
  if (!stbem::apply_tc_exact_supported(n_t, n_x, n_rhs, A->n_slices))
    return fail(ctx, STBEM_ERR_ARG, "apply_exact: unsupported sizes n_t=%d n_x=%d n_rhs=%d", n_t, n_x, n_rhs);
  if (reinterpret_cast<uintptr_t>(work) & 255) return fail(ctx, STBEM_ERR_ARG, "apply_exact: workspace not 256-byte aligned");
  const size_t need = exact_x_bytes(n_t, n_x, n_rhs, A->n_slices);
  if (work_bytes < need) return fail(ctx, STBEM_ERR_NOMEM, "apply_exact: workspace %zu < %zu bytes", work_bytes, need);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "apply_exact: set device");
  CUDA_TRY(ctx, stbem::tc_error_reset(ctx->stream), "apply_exact: reset error word");
  CUDA_TRY(ctx, apply_exact(n_t, n_x, *A, n_rhs, x, y, work, ctx->stream), "apply_exact");
  int flag = 0;
  CUDA_TRY(ctx, stbem::tc_error_read(&flag, ctx->stream), "apply_exact: read error word");
  if (flag) return fail(ctx, STBEM_ERR_TIMEOUT, "apply_exact: a pipeline wait timed out");
  return STBEM_OK;
}

int stbem_rhs_g_batched(stbem_ctx* ctx, const stbem_mesh* m, int n_src, const double* ys, double* G) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rg = reject_graded(ctx, m, "rhs_g_batched")) return rg;
  if (!m || !ys || !G || n_src < 1) return fail(ctx, STBEM_ERR_ARG, "rhs_g_batched: bad arguments");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "rhs_g_batched: set device");
  const size_t N = (size_t)m->n_t * m->N;
  for (int k = 0; k < n_src; ++k)
    CUDA_TRY(ctx, stbem::rhs_g_launch(m->dev, ys[2 * k], ys[2 * k + 1], G + k * N, ctx->stream), "rhs_g_batched");
  return STBEM_OK;
}

int stbem_half_mass_add(stbem_ctx* ctx, const stbem_mesh* m, int n_rhs, const double* G, double* F) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rg = reject_graded(ctx, m, "half_mass_add")) return rg;
  if (!m || !G || !F || n_rhs < 1) return fail(ctx, STBEM_ERR_ARG, "half_mass_add: bad arguments");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "half_mass_add: set device");
  CUDA_TRY(ctx, stbem::half_mass_add_launch(m->dev, G, F, ctx->stream, n_rhs), "half_mass_add");
  return STBEM_OK;
}

// ---------------------------------------------------------- batched GMRES ------
namespace {

struct BatchWork {
  double *Q, *Z, *U, *R, *DW, *h;   // h: device scratch for small batched results
  void* xb;                          // BF16 vector scratch (3 slices)
};

size_t batch_base_bytes(int nt, int nx, int B, int m) {
  const size_t n = (size_t)B * nt * nx;
  return ((size_t)(m + 1) * n + 4 * n + (size_t)(m + 4) * B) * sizeof(double) + 3 * n * 2 + 256;
}
// with an FP64 residual operator: + the FP64 product's lag-chunk partial sums;
// with an exact-slice one (exact_slices > 0): + the slices of W; with
// frequency blocks (fft): + the transforms of W and of the product
size_t batch_bytes(int nt, int nx, int B, int m, bool fp64_residual, int exact_slices = 0, bool fft = false) {
  size_t b = batch_base_bytes(nt, nx, B, m);
  if (fp64_residual) b = ((b + 255) & ~(size_t)255) + stbem::apply_workspace_bytes(nt, nx, B);
  else if (exact_slices > 0) b = ((b + 255) & ~(size_t)255) + exact_x_bytes(nt, nx, B, exact_slices);
  else if (fft) b = ((b + 255) & ~(size_t)255) + stbem::fft_apply_bytes(nt, nx, B);
  return b;
}

// The three-slice tensor-core residual is accurate to a few 1e-7 of |V||W|;
// refinement switches to the FP64 residual below this relative residual.
constexpr double kTc3ResidualFloor = 2e-6;

}  // namespace

int stbem_solve_batched_workspace_bytes(int n_t, int n_x, int n_rhs, int restart, int fp64_residual, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || n_rhs < 1 || restart < 1) return STBEM_ERR_ARG;
  *bytes = batch_bytes(n_t, n_x, n_rhs, restart, fp64_residual != 0);
  return STBEM_OK;
}

int stbem_solve_batched_exact_workspace_bytes(int n_t, int n_x, int n_rhs, int restart, int n_slices,
                                              size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || n_rhs < 1 || restart < 1 || n_slices < stbem::kExactMinSlices ||
      n_slices > stbem::kExactMaxSlices)
    return STBEM_ERR_ARG;
  *bytes = batch_bytes(n_t, n_x, n_rhs, restart, false, n_slices);
  return STBEM_OK;
}

int stbem_solve_batched_fft_workspace_bytes(int n_t, int n_x, int n_rhs, int restart, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || n_rhs < 1 || restart < 1 || n_t > stbem::kFftMaxSteps ||
      n_x > stbem::kFftMaxSpace)
    return STBEM_ERR_ARG;
  *bytes = batch_bytes(n_t, n_x, n_rhs, restart, false, 0, true);
  return STBEM_OK;
}

namespace {
// The batched solve; the refinement's final residual phase uses the FP64
// operator V64, the exact-slice operator Vx, the frequency blocks Vf, or
// none of them.
int solve_batched_impl(stbem_ctx* ctx, int nt, int nx, int B, const void* V_hi, const void* V_mid, const void* V_lo,
                       const void* D_bf16, const double* Lm, const double* V64, const stbem_exact_operand* Vx,
                       const void* Vf, const double* F, double* W, const stbem_solve_opts* opts, double inner_tol,
                       stbem_solve_info* infos, void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!V_hi || !F || !W || !opts || !infos || !work) return fail(ctx, STBEM_ERR_ARG, "solve_batched: NULL pointer");
  if (!stbem::apply_tc_supported(nt, nx, B)) return fail(ctx, STBEM_ERR_ARG, "solve_batched: unsupported sizes");
  const int m = opts->restart, maxit = opts->max_iter;
  if (m < 1 || maxit < 1 || !(opts->tol > 0) || !(inner_tol > 0) || !(inner_tol < 1))
    return fail(ctx, STBEM_ERR_ARG, "solve_batched: bad options");
  const bool prec = opts->precondition != 0;
  if (prec && (!D_bf16 || !Lm)) return fail(ctx, STBEM_ERR_ARG, "solve_batched: preconditioner needs D and L");
  if (opts->precondition == 2)
    return fail(ctx, STBEM_ERR_ARG, "solve_batched: the lumped mass (precondition = 1) only");
  if (V64 && !stbem::apply_grid_fits(nt, nx, B))
    return fail(ctx, STBEM_ERR_ARG, "solve_batched: too many right-hand sides for the FP64 residual product");
  if (Vx) {
    if (const int r = check_exact_operand(ctx, "solve_batched_exact", Vx)) return r;
    if (!stbem::apply_tc_exact_supported(nt, nx, B, Vx->n_slices))
      return fail(ctx, STBEM_ERR_ARG, "solve_batched_exact: unsupported sizes for the exact product");
    if (reinterpret_cast<uintptr_t>(work) & 255)
      return fail(ctx, STBEM_ERR_ARG, "solve_batched_exact: workspace not 256-byte aligned");
  }
  if (Vf) {
    if (nt > stbem::kFftMaxSteps || nx > stbem::kFftMaxSpace || B > 65535)
      return fail(ctx, STBEM_ERR_ARG, "solve_batched_fft: sizes beyond the FFT product's limits");
    if ((reinterpret_cast<uintptr_t>(Vf) & 15) || (reinterpret_cast<uintptr_t>(work) & 255))
      return fail(ctx, STBEM_ERR_ARG, "solve_batched_fft: frequency blocks or workspace misaligned");
  }
  if (work_bytes < batch_bytes(nt, nx, B, m, V64 != nullptr, Vx ? Vx->n_slices : 0, Vf != nullptr))
    return fail(ctx, STBEM_ERR_NOMEM, "solve_batched: workspace too small");
  const size_t N = (size_t)nt * nx, n = (size_t)B * N;
  BatchWork Wk;
  double* p = static_cast<double*>(work);
  Wk.Q = p; p += (size_t)(m + 1) * n;
  Wk.Z = p; p += n;
  Wk.U = p; p += n;
  Wk.R = p; p += n;
  Wk.DW = p; p += n;
  Wk.h = p; p += (size_t)(m + 4) * B;
  Wk.xb = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(p) + 255) & ~static_cast<uintptr_t>(255));
  // the final residual product's scratch after the base workspace (FP64
  // partial sums, or the slices of W)
  void* part64 = static_cast<char*>(work) + ((batch_base_bytes(nt, nx, B, m) + 255) & ~(size_t)255);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "solve_batched: set device");
  cudaStream_t s = ctx->stream;
  CUDA_TRY(ctx, stbem::tc_error_reset(s), "solve_batched: reset error word");
  const void* Vs[3] = {V_hi, V_mid, V_lo};

  std::vector<double> hbuf((size_t)(m + 1) * B), h2((size_t)(m + 1) * B), nrm(B), inv(B);
  auto bnorms = [&](const double* X, std::vector<double>& out) -> cudaError_t {
    cudaError_t e = stbem::bdots_launch(X, 1, X, B, N, Wk.h, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(out.data(), Wk.h, B * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int b = 0; b < B; ++b) out[b] = std::sqrt(out[b]);
    return e;
  };
  // preconditioner: y = L^{-1} D L^{-1} x on the tensor cores (or y = x)
  auto applyP = [&](const double* x, double* y) -> cudaError_t {
    if (!prec) return cudaMemcpyAsync(y, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaError_t e = stbem::diag_div_launch(x, Lm, Wk.Z, B * nt, nx, s);
    if (e == cudaSuccess) e = stbem::to_bf16_launch(STBEM_F64, Wk.Z, Wk.xb, n, s);
    if (e == cudaSuccess) e = stbem::apply_tc_launch(nt, nx, D_bf16, B, Wk.xb, y, false, s);
    if (e == cudaSuccess) e = stbem::diag_div_launch(y, Lm, y, B * nt, nx, s);
    return e;
  };

  std::vector<double> normF(B), rn(B);
  CUDA_TRY(ctx, bnorms(F, normF), "solve_batched: norm F");
  CUDA_TRY(ctx, cudaMemsetAsync(W, 0, n * sizeof(double), s), "solve_batched: zero W");
  CUDA_TRY(ctx, cudaMemcpyAsync(Wk.R, F, n * sizeof(double), cudaMemcpyDeviceToDevice, s), "solve_batched: R");
  for (int b = 0; b < B; ++b) {
    infos[b].iterations = 0;
    infos[b].status = std::isfinite(normF[b]) ? STBEM_OK : STBEM_ERR_NAN;
    infos[b].rel_residual = 0.0;
  }
  // refinement residual R = F - V W: the three-slice tensor-core product
  // first, then (with V64 or Vx) the FP64 or exact-slice product once that
  // one reaches its floor
  bool fp64_phase = false;
  const bool final_phase = V64 || Vx || Vf;
  const double tol_tc = final_phase ? std::max(opts->tol, kTc3ResidualFloor) : opts->tol;
  auto residual = [&]() -> cudaError_t {
    cudaError_t e = !fp64_phase ? apply_tc3(nt, nx, Vs, B, W, Wk.U, Wk.xb, s)
                    : Vx        ? apply_exact(nt, nx, *Vx, B, W, Wk.U, part64, s)
                    : Vf        ? stbem::fft_apply_launch(false, nt, nx, B, static_cast<const double2*>(Vf), W, Wk.U,
                                                          part64, s)
                                : stbem::apply_launch(STBEM_F64, false, nt, nx, V64, B, W, Wk.U, part64, s);
    if (e == cudaSuccess) e = stbem::sub_launch(F, Wk.U, Wk.R, n, s);
    return e;
  };
  int total = 0;
  bool any_active = true;
  for (int outer = 0; outer < 40 && any_active; ++outer) {
    CUDA_TRY(ctx, bnorms(Wk.R, rn), "solve_batched: norm R");
    std::vector<char> active(B, 0);
    any_active = false;
    const double target = fp64_phase ? opts->tol : tol_tc;
    for (int b = 0; b < B; ++b) {
      const double rel = normF[b] > 0 ? rn[b] / normF[b] : 0.0;
      if (!std::isfinite(rel)) infos[b].status = STBEM_ERR_NAN;
      infos[b].rel_residual = rel;
      active[b] = infos[b].status == STBEM_OK && rel > target;
      any_active = any_active || active[b];
    }
    if (!any_active && final_phase && !fp64_phase && opts->tol < tol_tc) {
      // the tensor-core residual is at its floor: continue on the FP64 residual
      fp64_phase = true;
      CUDA_TRY(ctx, residual(), "solve_batched: FP64 residual");
      any_active = true;
      continue;
    }
    if (!any_active) break;
    if (total >= maxit) {
      for (int b = 0; b < B; ++b)
        if (active[b]) infos[b].status = STBEM_ERR_NOCONV;
      break;
    }
    // inner: lockstep GMRES on the BF16 V for all right-hand sides
    for (int b = 0; b < B; ++b) inv[b] = (active[b] && rn[b] > 0) ? 1.0 / rn[b] : 0.0;
    CUDA_TRY(ctx, cudaMemcpyAsync(Wk.h, inv.data(), B * sizeof(double), cudaMemcpyHostToDevice, s), "inv");
    CUDA_TRY(ctx, stbem::bscale_launch(Wk.R, Wk.h, Wk.Q, B, N, s), "q0");
    std::vector<double> H((size_t)B * (m + 1) * m, 0.0), cs((size_t)B * m), sn((size_t)B * m),
        g((size_t)B * (m + 1), 0.0);
    std::vector<int> kb(B, 0);
    std::vector<char> done(B, 0);
    for (int b = 0; b < B; ++b) {
      g[(size_t)b * (m + 1)] = active[b] ? rn[b] : 0.0;
      done[b] = !active[b];
    }
    int kmax = 0;
    for (int k = 0; k < m; ++k) {
      double* qk = Wk.Q + (size_t)k * n;
      double* qk1 = Wk.Q + (size_t)(k + 1) * n;
      CUDA_TRY(ctx, applyP(qk, Wk.DW), "P q");
      CUDA_TRY(ctx, stbem::to_bf16_launch(STBEM_F64, Wk.DW, Wk.xb, n, s), "bf16 z");
      CUDA_TRY(ctx, stbem::apply_tc_launch(nt, nx, V_hi, B, Wk.xb, Wk.U, false, s), "V z");
      CUDA_TRY(ctx, stbem::bdots_launch(Wk.Q, k + 1, Wk.U, B, N, Wk.h, s), "dots");
      CUDA_TRY(ctx, stbem::bsub_comb_launch(Wk.Q, k + 1, Wk.h, Wk.U, B, N, s), "orth");
      CUDA_TRY(ctx, cudaMemcpyAsync(hbuf.data(), Wk.h, (size_t)(k + 1) * B * sizeof(double), cudaMemcpyDeviceToHost, s), "h");
      CUDA_TRY(ctx, stbem::bdots_launch(Wk.Q, k + 1, Wk.U, B, N, Wk.h, s), "dots2");
      CUDA_TRY(ctx, stbem::bsub_comb_launch(Wk.Q, k + 1, Wk.h, Wk.U, B, N, s), "orth2");
      CUDA_TRY(ctx, cudaMemcpyAsync(h2.data(), Wk.h, (size_t)(k + 1) * B * sizeof(double), cudaMemcpyDeviceToHost, s), "h2");
      CUDA_TRY(ctx, bnorms(Wk.U, nrm), "norm u");
      for (int b = 0; b < B; ++b) inv[b] = (!done[b] && nrm[b] > 0 && std::isfinite(nrm[b])) ? 1.0 / nrm[b] : 0.0;
      CUDA_TRY(ctx, cudaMemcpyAsync(Wk.h, inv.data(), B * sizeof(double), cudaMemcpyHostToDevice, s), "inv");
      CUDA_TRY(ctx, stbem::bscale_launch(Wk.U, Wk.h, qk1, B, N, s), "q");
      ++total;
      kmax = k + 1;
      bool all_done = true;
      for (int b = 0; b < B; ++b) {
        if (done[b]) continue;
        double* Hb = H.data() + (size_t)b * (m + 1) * m;
        double* gb = g.data() + (size_t)b * (m + 1);
        double* cb = cs.data() + (size_t)b * m;
        double* sb = sn.data() + (size_t)b * m;
        std::vector<double> col(k + 2);
        for (int t = 0; t <= k; ++t) col[t] = hbuf[(size_t)t * B + b] + h2[(size_t)t * B + b];
        const double hk1 = nrm[b];
        bool bad = !std::isfinite(hk1);
        for (int t = 0; t <= k; ++t) bad = bad || !std::isfinite(col[t]);
        if (bad) {
          infos[b].status = STBEM_ERR_NAN;
          done[b] = 1;
          kb[b] = 0;
          continue;
        }
        for (int t = 0; t < k; ++t) {
          const double a = cb[t] * col[t] + sb[t] * col[t + 1];
          col[t + 1] = -sb[t] * col[t] + cb[t] * col[t + 1];
          col[t] = a;
        }
        const double den = std::hypot(col[k], hk1);
        if (!(den > 0.0)) {        // zero pivot: singular preconditioned operator
          infos[b].status = STBEM_ERR_BREAKDOWN;
          done[b] = 1;
          kb[b] = k;
          continue;
        }
        cb[k] = den > 0 ? col[k] / den : 1.0;
        sb[k] = den > 0 ? hk1 / den : 0.0;
        col[k] = den;
        gb[k + 1] = -sb[k] * gb[k];
        gb[k] = cb[k] * gb[k];
        for (int t = 0; t <= k; ++t) Hb[(size_t)t * m + k] = col[t];
        kb[b] = k + 1;
        const double est = std::fabs(gb[k + 1]) / rn[b];
        if (est <= inner_tol || hk1 == 0.0) done[b] = 1;
        all_done = all_done && done[b];
      }
      if (all_done || total >= maxit) break;
    }
    // per right-hand side y_b = H_b^{-1} g_b, zero-padded to kmax
    std::vector<double> Y((size_t)kmax * B, 0.0);
    for (int b = 0; b < B; ++b) {
      const int kk = kb[b];
      const double* Hb = H.data() + (size_t)b * (m + 1) * m;
      const double* gb = g.data() + (size_t)b * (m + 1);
      std::vector<double> y(kk, 0.0);
      for (int t = kk - 1; t >= 0; --t) {
        double acc = gb[t];
        for (int u = t + 1; u < kk; ++u) acc -= Hb[(size_t)t * m + u] * y[u];
        y[t] = Hb[(size_t)t * m + t] != 0.0 ? acc / Hb[(size_t)t * m + t] : 0.0;
      }
      for (int t = 0; t < kk; ++t) Y[(size_t)t * B + b] = y[t];
      infos[b].iterations = total;
    }
    if (kmax > 0) {
      CUDA_TRY(ctx, cudaMemcpyAsync(Wk.h, Y.data(), Y.size() * sizeof(double), cudaMemcpyHostToDevice, s), "Y");
      CUDA_TRY(ctx, stbem::bcomb_launch(Wk.Q, kmax, Wk.h, Wk.U, B, N, s), "QY");
      CUDA_TRY(ctx, applyP(Wk.U, Wk.DW), "P QY");
      CUDA_TRY(ctx, stbem::axpy_launch(1.0, Wk.DW, W, n, s), "W += dW");
    }
    // refinement residual R = F - V W (the current phase's product)
    CUDA_TRY(ctx, residual(), "solve_batched: residual");
  }
  int flag = 0;
  CUDA_TRY(ctx, stbem::tc_error_read(&flag, s), "solve_batched: read error word");
  if (flag) return fail(ctx, STBEM_ERR_TIMEOUT, "solve_batched: a tensor-core pipeline wait timed out");
  int worst = STBEM_OK;
  for (int b = 0; b < B; ++b)
    if (infos[b].status != STBEM_OK) worst = infos[b].status;
  if (worst != STBEM_OK) return fail(ctx, worst, "solve_batched: some right-hand sides did not converge");
  return STBEM_OK;
}
}  // namespace

int stbem_solve_batched(stbem_ctx* ctx, int nt, int nx, int B, const void* V_hi, const void* V_mid,
                        const void* V_lo, const void* D_bf16, const double* Lm, const double* V64, const double* F,
                        double* W, const stbem_solve_opts* opts, double inner_tol, stbem_solve_info* infos,
                        void* work, size_t work_bytes) {
  return solve_batched_impl(ctx, nt, nx, B, V_hi, V_mid, V_lo, D_bf16, Lm, V64, nullptr, nullptr, F, W, opts,
                            inner_tol, infos, work, work_bytes);
}

int stbem_solve_batched_fft(stbem_ctx* ctx, int nt, int nx, int B, const void* V_hi, const void* V_mid,
                            const void* V_lo, const void* D_bf16, const double* Lm, const void* Vhat,
                            const double* F, double* W, const stbem_solve_opts* opts, double inner_tol,
                            stbem_solve_info* infos, void* work, size_t work_bytes) {
  if (ctx && !Vhat) return fail(ctx, STBEM_ERR_ARG, "solve_batched_fft: NULL frequency blocks");
  return solve_batched_impl(ctx, nt, nx, B, V_hi, V_mid, V_lo, D_bf16, Lm, nullptr, nullptr, Vhat, F, W, opts,
                            inner_tol, infos, work, work_bytes);
}

int stbem_solve_batched_exact(stbem_ctx* ctx, int nt, int nx, int B, const void* V_hi, const void* V_mid,
                              const void* V_lo, const void* D_bf16, const double* Lm, const stbem_exact_operand* Vx,
                              const double* F, double* W, const stbem_solve_opts* opts, double inner_tol,
                              stbem_solve_info* infos, void* work, size_t work_bytes) {
  if (ctx && !Vx) return fail(ctx, STBEM_ERR_ARG, "solve_batched_exact: NULL operand");
  return solve_batched_impl(ctx, nt, nx, B, V_hi, V_mid, V_lo, D_bf16, Lm, nullptr, Vx, nullptr, F, W, opts,
                            inner_tol, infos, work, work_bytes);
}

int stbem_rhs(stbem_ctx* ctx, const stbem_mesh* m, const double* K, double ysx, double ysy, double* g,
              double* f, void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rg = reject_graded(ctx, m, "rhs")) return rg;
  if (!m || !K || !g || !f || !work) return fail(ctx, STBEM_ERR_ARG, "rhs: NULL pointer");
  const size_t need = stbem::apply_workspace_bytes(m->n_t, m->N, 1);
  if (work_bytes < need) return fail(ctx, STBEM_ERR_NOMEM, "rhs: workspace %zu < %zu bytes", work_bytes, need);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "rhs: set device");
  CUDA_TRY(ctx, stbem::rhs_g_launch(m->dev, ysx, ysy, g, ctx->stream), "rhs: g");
  CUDA_TRY(ctx, stbem::apply_launch(STBEM_F64, false, m->n_t, m->N, K, 1, g, f, work, ctx->stream), "rhs: K g");
  CUDA_TRY(ctx, stbem::half_mass_add_launch(m->dev, g, f, ctx->stream), "rhs: mass");
  return STBEM_OK;
}

int stbem_lumped_mass(stbem_ctx* ctx, const stbem_mesh* m, double* L) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rg = reject_graded(ctx, m, "lumped_mass")) return rg;
  if (!m || !L) return fail(ctx, STBEM_ERR_ARG, "lumped: NULL pointer");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "lumped: set device");
  CUDA_TRY(ctx, stbem::lumped_mass_launch(m->dev, L, ctx->stream), "lumped");
  return STBEM_OK;
}

// ---------------------------------------------------------------- GMRES ------
namespace {

struct SolveWork {
  double *Q, *z, *v, *r, *u, *h;
  void* apply;
  size_t apply_bytes;
};

size_t solve_bytes(int nt, int nx, int restart) {
  const size_t N = (size_t)nt * nx;
  const size_t hn = (size_t)(restart + 2) * 65;
  return ((size_t)(restart + 1) * N + 4 * N + hn) * sizeof(double) + stbem::apply_workspace_bytes(nt, nx, 1);
}

bool carve(void* base, size_t bytes, int nt, int nx, int restart, SolveWork* w) {
  const size_t N = (size_t)nt * nx;
  double* p = static_cast<double*>(base);
  w->Q = p; p += (size_t)(restart + 1) * N;
  w->z = p; p += N;
  w->v = p; p += N;
  w->r = p; p += N;
  w->u = p; p += N;
  w->h = p; p += (size_t)(restart + 2) * 65;
  w->apply = p;
  w->apply_bytes = stbem::apply_workspace_bytes(nt, nx, 1);
  return (size_t)((char*)p - (char*)base) + w->apply_bytes <= bytes;
}

}  // namespace

int stbem_solve_workspace_bytes(int n_t, int n_x, int restart, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || restart < 1) return STBEM_ERR_ARG;
  *bytes = solve_bytes(n_t, n_x, restart);
  return STBEM_OK;
}

}  // extern "C"

namespace {

struct GmresOp {
  int nt, nx, prec;       // operator precision (F64 / F32 lag blocks)
  const void* V;
  const void* D;          // NULL: no preconditioner
  const double* L;
  bool transpose = false; // solve V^T x = f with the preconditioner L^-1 D^T L^-1
  int mass = 1;           // 1: L = lumped diagonal (N); 2: L = M_h^-1 (N x N), y = M^-1 D M^-T x
  // lag sharding: V and D hold only the lag ranges [ranges[2k], ranges[2k+1])
  // (blocks in range order); every product is this rank's partial sum
  // followed by the caller's all-reduce.  n_ranges < 0: full operators.
  int n_ranges = -1;
  const int* ranges = nullptr;
  stbem_allreduce_fn reduce = nullptr;
  void* reduce_user = nullptr;
  // non-uniform time grid: V and D are packed blocks (forward products only)
  // and L holds the lumped mass of every step (n_t x n_x)
  bool packed = false;
  // three-slice BF16 operators on the tensor cores (forward products of one
  // right-hand side): V3 / D3 the slices, V = V3[0] and D = D3[0] name them;
  // tcx the slices of x, tcpart the lag-chunk partial sums (may be NULL)
  const void* const* V3 = nullptr;
  const void* const* D3 = nullptr;
  void* tcx = nullptr;
  double* tcpart = nullptr;
  // frequency blocks (stbem_fft_operator): V and D name them; fftwork is the
  // product's scratch (stbem::fft_apply_bytes for one right-hand side)
  bool fft = false;
  void* fftwork = nullptr;
};

// y = A x with A one of op's operators (full, or this rank's lag ranges then
// the all-reduce).  A failing callback sets *reduce_rc and returns an error.
cudaError_t op_product(const GmresOp& op, const void* A, const double* x, double* y, void* work, cudaStream_t s,
                       int* reduce_rc) {
  if (op.packed) return stbem::nu_apply_launch(op.nt, op.nx, static_cast<const double*>(A), x, y, s);
  if (op.fft)
    return stbem::fft_apply_launch(op.transpose, op.nt, op.nx, 1, static_cast<const double2*>(A), x, y, op.fftwork, s);
  if (op.V3) return apply_tc3(op.nt, op.nx, A == op.V ? op.V3 : op.D3, 1, x, y, op.tcx, s, op.tcpart);
  if (op.n_ranges < 0) return stbem::apply_launch(op.prec, op.transpose, op.nt, op.nx, A, 1, x, y, work, s);
  const size_t N = (size_t)op.nt * op.nx;
  const size_t elt = op.prec == STBEM_F64 ? sizeof(double) : sizeof(float);
  cudaError_t e = cudaSuccess;
  if (op.n_ranges == 0) e = cudaMemsetAsync(y, 0, N * sizeof(double), s);
  size_t off = 0;
  for (int k = 0; k < op.n_ranges && e == cudaSuccess; ++k) {
    const int a = op.ranges[2 * k], b = op.ranges[2 * k + 1];
    const void* Ak = static_cast<const char*>(A) + off * op.nx * op.nx * elt;
    e = stbem::apply_range_launch(op.prec, op.transpose, op.nt, op.nx, a, b, Ak, 1, x, y, k > 0, work, s);
    off += (size_t)(b - a);
  }
  if (e != cudaSuccess) return e;
  const int rc = op.reduce(y, N, op.reduce_user);
  if (rc != 0) {
    *reduce_rc = rc;
    return cudaErrorUnknown;
  }
  return cudaSuccess;
}

// An operator product inside gmres_core: a failed all-reduce callback is
// reported as STBEM_ERR_REDUCE, other failures as CUDA errors.
#define OP_TRY(call, where)                                                                          \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      if (reduce_rc) return fail(ctx, STBEM_ERR_REDUCE, "%s: all-reduce callback returned %d", where, \
                                 reduce_rc);                                                        \
      return stbem_internal::cuda_fail(ctx, e_, where);                                             \
    }                                                                                               \
  } while (0)

// Right-preconditioned restarted GMRES for V x = f from x = 0 (see stbem_solve).
// Returns STBEM_OK, STBEM_ERR_NOCONV or STBEM_ERR_NAN (or a CUDA error code).
int gmres_core(stbem_ctx* ctx, const GmresOp& op, const double* f, double* w, double tol, int maxit,
               int restart, SolveWork& W, int* iters_out, double* relres_out) {
  cudaStream_t s = ctx->stream;
  const int nt = op.nt, nx = op.nx;
  const size_t N = (size_t)nt * nx;
  const bool prec = op.D != nullptr;
  *iters_out = 0;
  *relres_out = 0.0;
  int reduce_rc = 0;
  auto applyV = [&](const double* x, double* y) { return op_product(op, op.V, x, y, W.apply, s, &reduce_rc); };
  // right preconditioner: y = L^{-1} D L^{-1} x (lumped mixed mass), or
  // y = M^{-1} D M^{-T} x per time step (consistent mixed mass), or y = x
  auto applyP = [&](const double* x, double* y) -> cudaError_t {
    if (!prec) return cudaMemcpyAsync(y, x, N * sizeof(double), cudaMemcpyDeviceToDevice, s);
    // the lumped mass per step (packed) is divided elementwise over all n_t n_x
    const int dr = op.packed ? 1 : nt, dc = op.packed ? nt * nx : nx;
    cudaError_t e = op.mass == 2 ? stbem::blockmul_launch(nt, nx, op.L, true, x, W.u, s)
                                 : stbem::diag_div_launch(x, op.L, W.u, dr, dc, s);
    if (e != cudaSuccess) return e;
    if (op.mass == 2) {
      e = op_product(op, op.D, W.u, W.v, W.apply, s, &reduce_rc);
      if (e != cudaSuccess) return e;
      return stbem::blockmul_launch(nt, nx, op.L, false, W.v, y, s);
    }
    e = op_product(op, op.D, W.u, y, W.apply, s, &reduce_rc);
    if (e != cudaSuccess) return e;
    return stbem::diag_div_launch(y, op.L, y, dr, dc, s);
  };
  auto norm = [&](const double* x, double* out) -> cudaError_t {
    cudaError_t e = stbem::dots_launch(x, 1, x, N, W.h, s);
    if (e != cudaSuccess) return e;
    double v;
    e = cudaMemcpyAsync(&v, W.h, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *out = std::sqrt(v);
    return e;
  };

  double nf;
  CUDA_TRY(ctx, norm(f, &nf), "solve: norm f");
  CUDA_TRY(ctx, cudaMemsetAsync(w, 0, N * sizeof(double), s), "solve: zero w");
  if (!std::isfinite(nf)) return fail(ctx, STBEM_ERR_NAN, "solve: right-hand side is not finite");
  if (nf == 0.0) return STBEM_OK;

  std::vector<double> H((size_t)(restart + 1) * restart, 0.0), cs(restart), sn(restart), g(restart + 1);
  std::vector<double> hcol(restart + 2), h2(restart + 2);
  int iters = 0;
  double relres = 1.0;
  int status = STBEM_OK;
  bool first = true;
  while (true) {
    // true residual r = f - V w
    if (first) {
      CUDA_TRY(ctx, cudaMemcpyAsync(W.r, f, N * sizeof(double), cudaMemcpyDeviceToDevice, s), "solve: r");
    } else {
      OP_TRY(applyV(w, W.v), "solve: V w");
      CUDA_TRY(ctx, stbem::sub_launch(f, W.v, W.r, N, s), "solve: f - V w");
    }
    first = false;
    double beta;
    CUDA_TRY(ctx, norm(W.r, &beta), "solve: norm r");
    if (!std::isfinite(beta)) { status = STBEM_ERR_NAN; break; }
    relres = beta / nf;
    if (relres <= tol) break;
    if (iters >= maxit) { status = STBEM_ERR_NOCONV; break; }
    CUDA_TRY(ctx, stbem::scale_launch(W.r, 1.0 / beta, W.Q, N, s), "solve: q0");
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k_done = 0;
    for (int k = 0; k < restart; ++k) {
      double* qk = W.Q + (size_t)k * N;
      double* qk1 = W.Q + (size_t)(k + 1) * N;
      OP_TRY(applyP(qk, W.z), "solve: precondition");
      OP_TRY(applyV(W.z, W.v), "solve: V z");
      // classical Gram-Schmidt, twice
      CUDA_TRY(ctx, stbem::dots_launch(W.Q, k + 1, W.v, N, W.h, s), "solve: dots");
      CUDA_TRY(ctx, stbem::sub_combination_launch(W.Q, k + 1, W.h, W.v, N, s), "solve: orth");
      CUDA_TRY(ctx, cudaMemcpyAsync(hcol.data(), W.h, (k + 1) * sizeof(double), cudaMemcpyDeviceToHost, s), "solve: h");
      CUDA_TRY(ctx, stbem::dots_launch(W.Q, k + 1, W.v, N, W.h, s), "solve: dots2");
      CUDA_TRY(ctx, stbem::sub_combination_launch(W.Q, k + 1, W.h, W.v, N, s), "solve: orth2");
      CUDA_TRY(ctx, cudaMemcpyAsync(h2.data(), W.h, (k + 1) * sizeof(double), cudaMemcpyDeviceToHost, s), "solve: h2");
      double hk1;
      CUDA_TRY(ctx, norm(W.v, &hk1), "solve: norm v");
      for (int t = 0; t <= k; ++t) hcol[t] += h2[t];
      bool bad = !std::isfinite(hk1);
      for (int t = 0; t <= k; ++t) bad = bad || !std::isfinite(hcol[t]);
      if (bad) { status = STBEM_ERR_NAN; break; }
      if (hk1 > 0.0) CUDA_TRY(ctx, stbem::scale_launch(W.v, 1.0 / hk1, qk1, N, s), "solve: q");
      // Givens rotations on column k
      for (int t = 0; t < k; ++t) {
        const double a = cs[t] * hcol[t] + sn[t] * hcol[t + 1];
        hcol[t + 1] = -sn[t] * hcol[t] + cs[t] * hcol[t + 1];
        hcol[t] = a;
      }
      const double den = std::hypot(hcol[k], hk1);
      // a zero pivot: (V P) q_k has no component outside the earlier basis
      // and none along it, so the preconditioned operator is singular
      if (!(den > 0.0)) { status = STBEM_ERR_BREAKDOWN; break; }
      cs[k] = hcol[k] / den;
      sn[k] = hk1 / den;
      hcol[k] = den;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      for (int t = 0; t <= k; ++t) H[(size_t)t * restart + k] = hcol[t];
      ++iters;
      k_done = k + 1;
      const double est = std::fabs(g[k + 1]) / nf;
      if (est <= tol || iters >= maxit || hk1 == 0.0) break;
    }
    if (status != STBEM_OK) break;
    // y = H^{-1} g (upper triangular), w += P(Q y)
    std::vector<double> y(k_done, 0.0);
    for (int t = k_done - 1; t >= 0; --t) {
      double acc = g[t];
      for (int u = t + 1; u < k_done; ++u) acc -= H[(size_t)t * restart + u] * y[u];
      y[t] = acc / H[(size_t)t * restart + t];
    }
    CUDA_TRY(ctx, cudaMemcpyAsync(W.h, y.data(), k_done * sizeof(double), cudaMemcpyHostToDevice, s), "solve: y");
    CUDA_TRY(ctx, stbem::combination_launch(W.Q, k_done, W.h, W.r, N, s), "solve: Qy");
    OP_TRY(applyP(W.r, W.z), "solve: P Qy");
    CUDA_TRY(ctx, stbem::axpy_launch(1.0, W.z, w, N, s), "solve: update");
    CUDA_TRY(ctx, cudaStreamSynchronize(s), "solve: sync");
  }
  *iters_out = iters;
  *relres_out = relres;
  return status;
}

}  // namespace

extern "C" {

namespace {
int solve_impl(stbem_ctx* ctx, bool transpose, int nt, int nx, int vprec, const void* V, const void* D,
               const double* L, const double* f, double* w, const stbem_solve_opts* opts, stbem_solve_info* info,
               void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!V || !f || !w || !opts || !info || !work) return fail(ctx, STBEM_ERR_ARG, "solve: NULL pointer");
  if (nt < 1 || nx < 1) return fail(ctx, STBEM_ERR_ARG, "solve: bad sizes");
  if (vprec != STBEM_F64 && vprec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "solve: bad precision");
  const int restart = opts->restart, maxit = opts->max_iter;
  if (restart < 1 || maxit < 1 || !(opts->tol > 0)) return fail(ctx, STBEM_ERR_ARG, "solve: bad options");
  const bool prec = opts->precondition != 0;
  if (prec && (!D || !L)) return fail(ctx, STBEM_ERR_ARG, "solve: preconditioner needs D and L");
  SolveWork W;
  if (!carve(work, work_bytes, nt, nx, restart, &W))
    return fail(ctx, STBEM_ERR_NOMEM, "solve: workspace %zu < %zu bytes", work_bytes, solve_bytes(nt, nx, restart));
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "solve: set device");
  GmresOp op{nt, nx, vprec, V, prec ? D : nullptr, L};
  op.transpose = transpose;
  op.mass = opts->precondition == 2 ? 2 : 1;
  int iters = 0;
  double relres = 0.0;
  const int status = gmres_core(ctx, op, f, w, opts->tol, maxit, restart, W, &iters, &relres);
  info->iterations = iters;
  info->rel_residual = relres;
  info->status = status;
  if (status == STBEM_ERR_NAN || status == STBEM_ERR_NOCONV || status == STBEM_ERR_BREAKDOWN)
    return fail(ctx, status, "solve: %s after %d iterations (relres %.3e)",
                status == STBEM_ERR_NAN ? "NaN"
                : status == STBEM_ERR_NOCONV ? "no convergence" : "breakdown (singular operator)",
                iters, relres);
  return status;   // STBEM_OK, or a CUDA error already described
}
}  // namespace

int stbem_solve(stbem_ctx* ctx, int nt, int nx, int vprec, const void* V, const void* D, const double* L,
                const double* f, double* w, const stbem_solve_opts* opts, stbem_solve_info* info,
                void* work, size_t work_bytes) {
  return solve_impl(ctx, false, nt, nx, vprec, V, D, L, f, w, opts, info, work, work_bytes);
}

int stbem_solve_adjoint(stbem_ctx* ctx, int nt, int nx, int vprec, const void* V, const void* D, const double* L,
                        const double* b, double* lam, const stbem_solve_opts* opts, stbem_solve_info* info,
                        void* work, size_t work_bytes) {
  return solve_impl(ctx, true, nt, nx, vprec, V, D, L, b, lam, opts, info, work, work_bytes);
}

// ------------------------------------------ products through time FFTs ------

namespace {
size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

int fft_sizes_ok(stbem_ctx* ctx, int nt, int nx, const char* where) {
  if (nt < 1 || nx < 1 || nt > stbem::kFftMaxSteps || nx > stbem::kFftMaxSpace)
    return fail(ctx, STBEM_ERR_ARG, "%s: sizes n_t = %d, n_x = %d outside [1, %d] x [1, %d]", where, nt, nx,
                stbem::kFftMaxSteps, stbem::kFftMaxSpace);
  return STBEM_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

size_t solve_fft_bytes(int nt, int nx, int restart) {
  return align16(solve_bytes(nt, nx, restart)) + stbem::fft_apply_bytes(nt, nx, 1);
}
}  // namespace

int stbem_fft_operator_bytes(int n_t, int n_x, int* n_freq, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || n_t > stbem::kFftMaxSteps || n_x > stbem::kFftMaxSpace) return STBEM_ERR_ARG;
  if (n_freq) *n_freq = stbem::fft_freqs(n_t);
  *bytes = stbem::fft_operator_bytes(n_t, n_x);
  return STBEM_OK;
}

int stbem_fft_operator(stbem_ctx* ctx, int n_t, int n_x, int prec, const void* A, void* Ahat) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rc = fft_sizes_ok(ctx, n_t, n_x, "fft_operator")) return rc;
  if (!A || !Ahat) return fail(ctx, STBEM_ERR_ARG, "fft_operator: NULL pointer");
  if (prec != STBEM_F64 && prec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "fft_operator: bad precision %d", prec);
  if (!aligned16(Ahat)) return fail(ctx, STBEM_ERR_ARG, "fft_operator: frequency blocks not 16-byte aligned");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "fft_operator: set device");
  CUDA_TRY(ctx, stbem::fft_operator_launch(prec, n_t, n_x, A, static_cast<double2*>(Ahat), ctx->stream),
           "fft_operator");
  return STBEM_OK;
}

int stbem_apply_fft_workspace_bytes(int n_t, int n_x, int n_rhs, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || n_rhs < 1 || n_t > stbem::kFftMaxSteps || n_x > stbem::kFftMaxSpace)
    return STBEM_ERR_ARG;
  *bytes = stbem::fft_apply_bytes(n_t, n_x, n_rhs);
  return STBEM_OK;
}

int stbem_apply_fft(stbem_ctx* ctx, int transpose, int n_t, int n_x, int n_rhs, const void* Ahat, const double* x,
                    double* y, void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rc = fft_sizes_ok(ctx, n_t, n_x, "apply_fft")) return rc;
  if (n_rhs < 1 || n_rhs > 65535) return fail(ctx, STBEM_ERR_ARG, "apply_fft: n_rhs = %d outside [1, 65535]", n_rhs);
  if (!Ahat || !x || !y || !work) return fail(ctx, STBEM_ERR_ARG, "apply_fft: NULL pointer");
  if (!aligned16(Ahat) || !aligned16(work))
    return fail(ctx, STBEM_ERR_ARG, "apply_fft: frequency blocks or workspace not 16-byte aligned");
  const size_t need = stbem::fft_apply_bytes(n_t, n_x, n_rhs);
  if (work_bytes < need) return fail(ctx, STBEM_ERR_NOMEM, "apply_fft: workspace %zu < %zu bytes", work_bytes, need);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "apply_fft: set device");
  CUDA_TRY(ctx, stbem::fft_apply_launch(transpose != 0, n_t, n_x, n_rhs, static_cast<const double2*>(Ahat), x, y,
                                        work, ctx->stream),
           "apply_fft");
  return STBEM_OK;
}

int stbem_solve_fft_workspace_bytes(int n_t, int n_x, int restart, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || restart < 1 || n_t > stbem::kFftMaxSteps || n_x > stbem::kFftMaxSpace)
    return STBEM_ERR_ARG;
  *bytes = solve_fft_bytes(n_t, n_x, restart);
  return STBEM_OK;
}

int stbem_solve_fft(stbem_ctx* ctx, int transpose, int nt, int nx, const void* Vhat, const void* Dhat,
                    const double* L, const double* f, double* w, const stbem_solve_opts* opts, stbem_solve_info* info,
                    void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rc = fft_sizes_ok(ctx, nt, nx, "solve_fft")) return rc;
  if (!Vhat || !f || !w || !opts || !info || !work) return fail(ctx, STBEM_ERR_ARG, "solve_fft: NULL pointer");
  const int restart = opts->restart, maxit = opts->max_iter;
  if (restart < 1 || maxit < 1 || !(opts->tol > 0)) return fail(ctx, STBEM_ERR_ARG, "solve_fft: bad options");
  const bool prec = opts->precondition != 0;
  if (prec && (!Dhat || !L)) return fail(ctx, STBEM_ERR_ARG, "solve_fft: preconditioner needs D and L");
  if (!aligned16(Vhat) || (prec && !aligned16(Dhat)) || !aligned16(work))
    return fail(ctx, STBEM_ERR_ARG, "solve_fft: frequency blocks or workspace not 16-byte aligned");
  const size_t need = solve_fft_bytes(nt, nx, restart);
  if (work_bytes < need) return fail(ctx, STBEM_ERR_NOMEM, "solve_fft: workspace %zu < %zu bytes", work_bytes, need);
  SolveWork W;
  carve(work, work_bytes, nt, nx, restart, &W);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "solve_fft: set device");
  GmresOp op{nt, nx, STBEM_F64, Vhat, prec ? Dhat : nullptr, L};
  op.transpose = transpose != 0;
  op.mass = opts->precondition == 2 ? 2 : 1;
  op.fft = true;
  op.fftwork = static_cast<char*>(work) + align16(solve_bytes(nt, nx, restart));
  int iters = 0;
  double relres = 0.0;
  const int status = gmres_core(ctx, op, f, w, opts->tol, maxit, restart, W, &iters, &relres);
  info->iterations = iters;
  info->rel_residual = relres;
  info->status = status;
  if (status == STBEM_ERR_NAN || status == STBEM_ERR_NOCONV || status == STBEM_ERR_BREAKDOWN)
    return fail(ctx, status, "solve_fft: %s after %d iterations (relres %.3e)",
                status == STBEM_ERR_NAN ? "NaN"
                : status == STBEM_ERR_NOCONV ? "no convergence" : "breakdown (singular operator)",
                iters, relres);
  return status;
}

// ------------------------------------------------- non-uniform time grids ------

int stbem_nu_op_bytes(const stbem_mesh* m, size_t* bytes) {
  if (!m || !bytes) return STBEM_ERR_ARG;
  *bytes = (size_t)m->n_t * (m->n_t + 1) / 2 * m->N * m->N * sizeof(double);
  return STBEM_OK;
}

int stbem_nu_assemble(stbem_ctx* ctx, const stbem_mesh* m, int op, double* out) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!m || !out) return fail(ctx, STBEM_ERR_ARG, "nu_assemble: NULL mesh or output");
  if (op < 0 || op > 2) return fail(ctx, STBEM_ERR_ARG, "nu_assemble: unknown operator %d", op);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "nu_assemble: set device");
  CUDA_TRY(ctx, stbem::nu_assemble_launch(m->dev, m->tbuf, op, out, ctx->stream), "nu_assemble");
  return STBEM_OK;
}

int stbem_nu_apply(stbem_ctx* ctx, int n_t, int n_x, const double* A, const double* x, double* y) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!A || !x || !y) return fail(ctx, STBEM_ERR_ARG, "nu_apply: NULL pointer");
  if (n_t < 1 || n_x < 1) return fail(ctx, STBEM_ERR_ARG, "nu_apply: bad sizes");
  if (x == y) return fail(ctx, STBEM_ERR_ARG, "nu_apply: x and y overlap");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "nu_apply: set device");
  CUDA_TRY(ctx, stbem::nu_apply_launch(n_t, n_x, A, x, y, ctx->stream), "nu_apply");
  return STBEM_OK;
}

int stbem_nu_rhs(stbem_ctx* ctx, const stbem_mesh* m, const double* K, double ysx, double ysy, double* g,
                 double* f) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!m || !K || !g || !f) return fail(ctx, STBEM_ERR_ARG, "nu_rhs: NULL pointer");
  if (!std::isfinite(ysx) || !std::isfinite(ysy)) return fail(ctx, STBEM_ERR_ARG, "nu_rhs: non-finite source");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "nu_rhs: set device");
  CUDA_TRY(ctx, stbem::nu_rhs_launch(m->dev, m->tbuf, ysx, ysy, g, ctx->stream), "nu_rhs: g");
  CUDA_TRY(ctx, stbem::nu_apply_launch(m->n_t, m->N, K, g, f, ctx->stream), "nu_rhs: K g");
  CUDA_TRY(ctx, stbem::nu_half_mass_add_launch(m->dev, m->tbuf, g, f, ctx->stream), "nu_rhs: mass");
  return STBEM_OK;
}

int stbem_nu_lumped_mass(stbem_ctx* ctx, const stbem_mesh* m, double* L) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!m || !L) return fail(ctx, STBEM_ERR_ARG, "nu_lumped_mass: NULL pointer");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "nu_lumped_mass: set device");
  CUDA_TRY(ctx, stbem::nu_lumped_launch(m->dev, m->tbuf, L, ctx->stream), "nu_lumped_mass");
  return STBEM_OK;
}

int stbem_nu_solve(stbem_ctx* ctx, int nt, int nx, const double* V, const double* D, const double* L,
                   const double* f, double* w, const stbem_solve_opts* opts, stbem_solve_info* info, void* work,
                   size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!V || !f || !w || !opts || !info || !work) return fail(ctx, STBEM_ERR_ARG, "nu_solve: NULL pointer");
  if (nt < 1 || nx < 1) return fail(ctx, STBEM_ERR_ARG, "nu_solve: bad sizes");
  const int restart = opts->restart, maxit = opts->max_iter;
  if (restart < 1 || maxit < 1 || !(opts->tol > 0)) return fail(ctx, STBEM_ERR_ARG, "nu_solve: bad options");
  if (opts->precondition != 0 && opts->precondition != 1)
    return fail(ctx, STBEM_ERR_ARG, "nu_solve: precondition must be 0 or 1 (lumped mass per step)");
  const bool prec = opts->precondition != 0;
  if (prec && (!D || !L)) return fail(ctx, STBEM_ERR_ARG, "nu_solve: preconditioner needs D and L");
  SolveWork W;
  if (!carve(work, work_bytes, nt, nx, restart, &W))
    return fail(ctx, STBEM_ERR_NOMEM, "nu_solve: workspace %zu < %zu bytes", work_bytes, solve_bytes(nt, nx, restart));
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "nu_solve: set device");
  GmresOp op{nt, nx, STBEM_F64, V, prec ? D : nullptr, L};
  op.packed = true;
  int iters = 0;
  double relres = 0.0;
  const int status = gmres_core(ctx, op, f, w, opts->tol, maxit, restart, W, &iters, &relres);
  info->iterations = iters;
  info->rel_residual = relres;
  info->status = status;
  if (status == STBEM_ERR_NAN || status == STBEM_ERR_NOCONV || status == STBEM_ERR_BREAKDOWN)
    return fail(ctx, status, "nu_solve: %s after %d iterations (relres %.3e)",
                status == STBEM_ERR_NAN ? "NaN"
                : status == STBEM_ERR_NOCONV ? "no convergence" : "breakdown (singular operator)",
                iters, relres);
  return status;
}

// ---------------------------------------------------------- lag sharding ------

int stbem_lag_shard(int n_t, int n_ranks, int rank, int chunk, int max_ranges, int* host_ranges, int* n_ranges) {
  if (n_t < 1 || n_ranks < 1 || rank < 0 || rank >= n_ranks || chunk < 1 || max_ranges < 0 || !n_ranges)
    return STBEM_ERR_ARG;
  const std::vector<int> r = stbem::lag_ranges(n_t, n_ranks, rank, chunk);
  const int n = (int)r.size() / 2;
  *n_ranges = n;
  if (n > max_ranges || (n > 0 && !host_ranges)) return STBEM_ERR_NOMEM;
  std::copy(r.begin(), r.end(), host_ranges);
  return STBEM_OK;
}

int stbem_assemble_lag_blocks(stbem_ctx* ctx, const stbem_mesh* m, int op, int prec, int lag_begin, int lag_end,
                              void* dev_blocks) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rg = reject_graded(ctx, m, "assemble_lag_blocks")) return rg;
  if (!m || !dev_blocks) return fail(ctx, STBEM_ERR_ARG, "assemble_lag_blocks: NULL mesh or output");
  if (op < 0 || op > 2) return fail(ctx, STBEM_ERR_ARG, "assemble_lag_blocks: unknown operator %d", op);
  if (prec != STBEM_F64 && prec != STBEM_F32)
    return fail(ctx, STBEM_ERR_ARG, "assemble_lag_blocks: unknown precision %d", prec);
  if (lag_begin < 0 || lag_end > m->n_t || lag_begin > lag_end)
    return fail(ctx, STBEM_ERR_ARG, "assemble_lag_blocks: lag range [%d, %d) outside [0, %d)", lag_begin, lag_end,
                m->n_t);
  if (lag_begin == lag_end) return STBEM_OK;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "assemble_lag_blocks: set device");
  // The kernels write block d at base + d N^2 and only for d in the range;
  // with the base moved down by lag_begin blocks (integer address arithmetic)
  // block d lands at dev_blocks + (d - lag_begin) N^2, inside the caller's array.
  const size_t elt = prec == STBEM_F64 ? sizeof(double) : sizeof(float);
  const uintptr_t shifted = reinterpret_cast<uintptr_t>(dev_blocks) - (uintptr_t)lag_begin * m->N * m->N * elt;
  CUDA_TRY(ctx, stbem::assemble_launch(m->dev, op, prec, lag_begin, lag_end, reinterpret_cast<void*>(shifted),
                                       ctx->stream),
           "assemble_lag_blocks");
  return STBEM_OK;
}

int stbem_apply_lags_workspace_bytes(int n_t, int n_x, int n_lags, int n_rhs, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || n_lags < 1 || n_lags > n_t || n_rhs < 1) return STBEM_ERR_ARG;
  *bytes = stbem::apply_range_workspace_bytes(n_t, n_x, n_lags, n_rhs);
  return STBEM_OK;
}

int stbem_apply_lags(stbem_ctx* ctx, int prec, int transpose, int n_t, int n_x, int lag_begin, int lag_end,
                     const void* A_blocks, int n_rhs, const double* x, double* y, int accumulate, void* work,
                     size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!A_blocks || !x || !y || !work) return fail(ctx, STBEM_ERR_ARG, "apply_lags: NULL pointer");
  if (n_t < 1 || n_x < 1 || n_rhs < 1 || lag_begin < 0 || lag_end > n_t || lag_begin >= lag_end)
    return fail(ctx, STBEM_ERR_ARG, "apply_lags: bad sizes or lag range [%d, %d)", lag_begin, lag_end);
  if (prec != STBEM_F64 && prec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "apply_lags: bad precision");
  if ((const void*)x == (const void*)y) return fail(ctx, STBEM_ERR_ARG, "apply_lags: x and y overlap");
  if (!stbem::apply_grid_fits(n_t, n_x, n_rhs))
    return fail(ctx, STBEM_ERR_ARG, "apply_lags: n_rhs x time tiles exceeds the grid limit 65535");
  const size_t need = stbem::apply_range_workspace_bytes(n_t, n_x, lag_end - lag_begin, n_rhs);
  if (work_bytes < need) return fail(ctx, STBEM_ERR_NOMEM, "apply_lags: workspace %zu < %zu bytes", work_bytes, need);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "apply_lags: set device");
  CUDA_TRY(ctx, stbem::apply_range_launch(prec, transpose != 0, n_t, n_x, lag_begin, lag_end, A_blocks, n_rhs, x, y,
                                          accumulate != 0, work, ctx->stream),
           "apply_lags");
  return STBEM_OK;
}

namespace {
// the largest product workspace over every lag-range length
size_t any_range_apply_bytes(int nt, int nx) {
  size_t b = 0;
  for (int nl = 1; nl <= nt; ++nl) b = std::max(b, stbem::apply_range_workspace_bytes(nt, nx, nl, 1));
  return b;
}
}  // namespace

int stbem_solve_sharded_workspace_bytes(int n_t, int n_x, int restart, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || restart < 1) return STBEM_ERR_ARG;
  *bytes = solve_bytes(n_t, n_x, restart) - stbem::apply_workspace_bytes(n_t, n_x, 1) + any_range_apply_bytes(n_t, n_x);
  return STBEM_OK;
}

int stbem_solve_sharded(stbem_ctx* ctx, int nt, int nx, int vprec, const void* V_blocks, const void* D_blocks,
                        int n_ranges, const int* host_ranges, stbem_allreduce_fn allreduce, void* user,
                        const double* L, const double* f, double* w, const stbem_solve_opts* opts,
                        stbem_solve_info* info, void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!f || !w || !opts || !info || !work || !allreduce) return fail(ctx, STBEM_ERR_ARG, "solve_sharded: NULL pointer");
  if (nt < 1 || nx < 1 || n_ranges < 0 || (n_ranges > 0 && (!host_ranges || !V_blocks)))
    return fail(ctx, STBEM_ERR_ARG, "solve_sharded: bad sizes or ranges");
  for (int k = 0; k < n_ranges; ++k) {
    const int a = host_ranges[2 * k], b = host_ranges[2 * k + 1];
    if (a < 0 || b > nt || a >= b || (k > 0 && a < host_ranges[2 * k - 1]))
      return fail(ctx, STBEM_ERR_ARG, "solve_sharded: lag range %d [%d, %d) invalid", k, a, b);
  }
  if (vprec != STBEM_F64 && vprec != STBEM_F32) return fail(ctx, STBEM_ERR_ARG, "solve_sharded: bad precision");
  const int restart = opts->restart, maxit = opts->max_iter;
  if (restart < 1 || maxit < 1 || !(opts->tol > 0)) return fail(ctx, STBEM_ERR_ARG, "solve_sharded: bad options");
  const bool prec = opts->precondition != 0;
  if (prec && (!L || (n_ranges > 0 && !D_blocks)))
    return fail(ctx, STBEM_ERR_ARG, "solve_sharded: preconditioner needs D and L");
  size_t need = 0;
  stbem_solve_sharded_workspace_bytes(nt, nx, restart, &need);
  if (work_bytes < need) return fail(ctx, STBEM_ERR_NOMEM, "solve_sharded: workspace %zu < %zu bytes", work_bytes, need);
  SolveWork W;
  carve(work, work_bytes, nt, nx, restart, &W);
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "solve_sharded: set device");
  // D non-NULL signals the preconditioner to gmres_core; a rank without lags
  // never reads it
  GmresOp op{nt, nx, vprec, V_blocks ? V_blocks : work, prec ? (D_blocks ? D_blocks : work) : nullptr, L};
  op.mass = opts->precondition == 2 ? 2 : 1;
  op.n_ranges = n_ranges;
  op.ranges = host_ranges;
  op.reduce = allreduce;
  op.reduce_user = user;
  int iters = 0;
  double relres = 0.0;
  const int status = gmres_core(ctx, op, f, w, opts->tol, maxit, restart, W, &iters, &relres);
  info->iterations = iters;
  info->rel_residual = relres;
  info->status = status;
  if (status == STBEM_ERR_NAN || status == STBEM_ERR_NOCONV || status == STBEM_ERR_BREAKDOWN)
    return fail(ctx, status, "solve_sharded: %s after %d iterations (relres %.3e)",
                status == STBEM_ERR_NAN ? "NaN"
                : status == STBEM_ERR_NOCONV ? "no convergence" : "breakdown (singular operator)",
                iters, relres);
  return status;
}

int stbem_mixed_mass_inverse(stbem_ctx* ctx, const stbem_mesh* m, double* dev_Minv) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rg = reject_graded(ctx, m, "mixed_mass_inverse")) return rg;
  if (!m || !dev_Minv) return fail(ctx, STBEM_ERR_ARG, "mixed_mass_inverse: NULL pointer");
  // the cyclic tridiagonal mixed mass of one step, inverted on the host
  // (Gauss-Jordan with partial pivoting; M is not symmetric; N^3 host work,
  // once per mesh)
  std::vector<double> A = stbem::mixed_mass_matrix(m->h, m->ht), Inv;
  if (!stbem::gauss_jordan_inverse(A, m->N, Inv)) return fail(ctx, STBEM_ERR_ARG, "mixed_mass_inverse: singular");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "mixed_mass_inverse: set device");
  CUDA_TRY(ctx, cudaMemcpyAsync(dev_Minv, Inv.data(), Inv.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream),
           "mixed_mass_inverse: upload");
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "mixed_mass_inverse: sync");
  return STBEM_OK;
}

int stbem_grad_workspace_bytes(int n_t, int n_x, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 3) return STBEM_ERR_ARG;
  *bytes = stbem::grad_workspace_bytes(n_t, n_x);
  return STBEM_OK;
}

int stbem_grad(stbem_ctx* ctx, const stbem_mesh* m, const double* K, double ysx, double ysy, const double* g,
               const double* w, const double* lam, double* dxy, double* dalpha, void* work, size_t work_bytes) {
  if (!ctx) return STBEM_ERR_ARG;
  if (const int rg = reject_graded(ctx, m, "grad")) return rg;
  if (!m || !K || !g || !w || !lam || !dxy || !dalpha || !work) return fail(ctx, STBEM_ERR_ARG, "grad: NULL pointer");
  if (!std::isfinite(ysx) || !std::isfinite(ysy)) return fail(ctx, STBEM_ERR_ARG, "grad: non-finite source point");
  const size_t need = stbem::grad_workspace_bytes(m->n_t, m->N);
  if (work_bytes < need) return fail(ctx, STBEM_ERR_NOMEM, "grad: workspace %zu < %zu bytes", work_bytes, need);
  if (reinterpret_cast<uintptr_t>(work) & 255) return fail(ctx, STBEM_ERR_ARG, "grad: workspace must be 256-byte aligned");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "grad: set device");
  CUDA_TRY(ctx, stbem::grad_launch(m->dev, K, ysx, ysy, g, w, lam, dxy, dalpha, work, ctx->stream), "grad");
  return STBEM_OK;
}

int stbem_solve_mixed_workspace_bytes(int n_t, int n_x, int restart, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || restart < 1) return STBEM_ERR_ARG;
  *bytes = solve_bytes(n_t, n_x, restart) + 2 * (size_t)n_t * n_x * sizeof(double);
  return STBEM_OK;
}

namespace {
// The mixed solve; the outer residual f - V w uses the FP64 operator V64 or,
// when Vx is given, its exact-slice form on the tensor cores.
int solve_mixed_impl(stbem_ctx* ctx, int nt, int nx, const double* V64, const stbem_exact_operand* Vx,
                     const float* V32, const float* D32, const double* L, const double* f, double* w,
                     const stbem_solve_opts* opts, double inner_tol, stbem_solve_info* info, void* work,
                     size_t work_bytes, const void* const* V3 = nullptr, const void* const* D3 = nullptr) {
  if (!ctx) return STBEM_ERR_ARG;
  if ((!V64 && !Vx) || (!V32 && !(V3 && V3[0])) || !f || !w || !opts || !info || !work)
    return fail(ctx, STBEM_ERR_ARG, "solve_mixed: NULL pointer");
  if (V3 && !stbem::apply_tc_supported(nt, nx, 1))
    return fail(ctx, STBEM_ERR_ARG, "solve_mixed_tc: unsupported sizes (need n_x %% 8 == 0)");
  if (nt < 1 || nx < 1) return fail(ctx, STBEM_ERR_ARG, "solve_mixed: bad sizes");
  if (Vx) {
    if (const int r = check_exact_operand(ctx, "solve_mixed_exact", Vx)) return r;
    if (!stbem::apply_tc_exact_supported(nt, nx, 1, Vx->n_slices))
      return fail(ctx, STBEM_ERR_ARG, "solve_mixed_exact: unsupported sizes for the exact product");
    if (reinterpret_cast<uintptr_t>(work) & 255)
      return fail(ctx, STBEM_ERR_ARG, "solve_mixed_exact: workspace not 256-byte aligned");
  }
  const int restart = opts->restart, maxit = opts->max_iter;
  if (restart < 1 || maxit < 1 || !(opts->tol > 0) || !(inner_tol > 0) || !(inner_tol < 1))
    return fail(ctx, STBEM_ERR_ARG, "solve_mixed: bad options");
  const bool prec = opts->precondition != 0;
  const bool have_d = V3 ? (D3 && D3[0]) : D32 != nullptr;
  if (prec && (!have_d || !L)) return fail(ctx, STBEM_ERR_ARG, "solve_mixed: preconditioner needs D and L");
  const size_t N = (size_t)nt * nx;
  const size_t base = align256(solve_bytes(nt, nx, restart) + 2 * N * sizeof(double));
  const size_t xbytes = Vx ? align256(exact_x_bytes(nt, nx, 1, Vx->n_slices)) : 0;
  const size_t need = (Vx || V3) ? base + xbytes + (V3 ? tc3_bytes(nt, nx, 1) : 0)
                                 : solve_bytes(nt, nx, restart) + 2 * N * sizeof(double);
  if (work_bytes < need) return fail(ctx, STBEM_ERR_NOMEM, "solve_mixed: workspace %zu < %zu bytes", work_bytes, need);
  SolveWork W;
  carve(work, solve_bytes(nt, nx, restart), nt, nx, restart, &W);
  double* r = reinterpret_cast<double*>(static_cast<char*>(work) + solve_bytes(nt, nx, restart));
  double* dw = r + N;
  void* xwork = static_cast<char*>(work) + base;   // slices of w (exact residual)
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "solve_mixed: set device");
  cudaStream_t s = ctx->stream;
  auto norm = [&](const double* x, double* out) -> cudaError_t {
    cudaError_t e = stbem::dots_launch(x, 1, x, N, W.h, s);
    if (e != cudaSuccess) return e;
    double v;
    e = cudaMemcpyAsync(&v, W.h, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *out = std::sqrt(v);
    return e;
  };
  info->iterations = 0;
  info->status = STBEM_OK;
  info->rel_residual = 0.0;
  double nf;
  CUDA_TRY(ctx, norm(f, &nf), "solve_mixed: norm f");
  CUDA_TRY(ctx, cudaMemsetAsync(w, 0, N * sizeof(double), s), "solve_mixed: zero w");
  if (!std::isfinite(nf)) {
    info->status = STBEM_ERR_NAN;
    return fail(ctx, STBEM_ERR_NAN, "solve_mixed: right-hand side is not finite");
  }
  if (nf == 0.0) return STBEM_OK;
  GmresOp op{nt, nx, STBEM_F32, V32, prec ? (const void*)D32 : nullptr, L};
  op.mass = opts->precondition == 2 ? 2 : 1;
  if (V3) {   // the inner products: three-slice BF16 operators on the tensor cores
    op.V = V3[0];
    op.D = prec ? D3[0] : nullptr;
    op.V3 = V3;
    op.D3 = D3;
    op.tcx = static_cast<char*>(work) + base + xbytes;
    op.tcpart = tc3_part(op.tcx, nt, nx, 1);
  }
  // tensor-core pipeline time-outs of the inner products and the residuals
  if (V3 || Vx) CUDA_TRY(ctx, stbem::tc_error_reset(s), "solve_mixed: reset error word");
  CUDA_TRY(ctx, cudaMemcpyAsync(r, f, N * sizeof(double), cudaMemcpyDeviceToDevice, s), "solve_mixed: r");
  int total = 0, status = STBEM_OK;
  double relres = 1.0;
  for (int outer = 0; outer < 30; ++outer) {
    double nr;
    CUDA_TRY(ctx, norm(r, &nr), "solve_mixed: norm r");
    if (!std::isfinite(nr)) { status = STBEM_ERR_NAN; break; }
    relres = nr / nf;
    if (relres <= opts->tol) break;
    if (total >= maxit) { status = STBEM_ERR_NOCONV; break; }
    // inner: V32 dw = r to inner_tol (relative to r), FP64 Krylov vectors
    int it = 0;
    double rr = 0.0;
    const int st = gmres_core(ctx, op, r, dw, inner_tol, maxit - total, restart, W, &it, &rr);
    total += it;
    if (st == STBEM_ERR_NAN || st == STBEM_ERR_BREAKDOWN) { status = st; break; }
    if (st != STBEM_OK && st != STBEM_ERR_NOCONV) return st;
    CUDA_TRY(ctx, stbem::axpy_launch(1.0, dw, w, N, s), "solve_mixed: w += dw");
    // residual with the FP64 operator (or its exact slices)
    if (Vx) CUDA_TRY(ctx, apply_exact(nt, nx, *Vx, 1, w, W.v, xwork, s), "solve_mixed: exact V w");
    else CUDA_TRY(ctx, stbem::apply_launch(STBEM_F64, false, nt, nx, V64, 1, w, W.v, W.apply, s), "solve_mixed: V w");
    if (V3 || Vx) {
      int flag = 0;
      CUDA_TRY(ctx, stbem::tc_error_read(&flag, s), "solve_mixed: read error word");
      if (flag) return fail(ctx, STBEM_ERR_TIMEOUT, "solve_mixed: a tensor-core pipeline wait timed out");
    }
    CUDA_TRY(ctx, stbem::sub_launch(f, W.v, r, N, s), "solve_mixed: f - V w");
    if (it == 0) { status = STBEM_ERR_NOCONV; break; }
  }
  info->iterations = total;
  info->rel_residual = relres;
  info->status = status;
  if (status != STBEM_OK)
    return fail(ctx, status, "solve_mixed: %s after %d inner iterations (relres %.3e)",
                status == STBEM_ERR_NAN ? "NaN"
                : status == STBEM_ERR_NOCONV ? "no convergence" : "breakdown (singular operator)",
                total, relres);
  return STBEM_OK;
}
}  // namespace

int stbem_solve_mixed(stbem_ctx* ctx, int nt, int nx, const double* V64, const float* V32, const float* D32,
                      const double* L, const double* f, double* w, const stbem_solve_opts* opts,
                      double inner_tol, stbem_solve_info* info, void* work, size_t work_bytes) {
  if (ctx && !V64) return fail(ctx, STBEM_ERR_ARG, "solve_mixed: NULL pointer");
  return solve_mixed_impl(ctx, nt, nx, V64, nullptr, V32, D32, L, f, w, opts, inner_tol, info, work, work_bytes);
}

int stbem_solve_mixed_exact_workspace_bytes(int n_t, int n_x, int restart, int n_slices, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || restart < 1 || n_slices < stbem::kExactMinSlices ||
      n_slices > stbem::kExactMaxSlices)
    return STBEM_ERR_ARG;
  *bytes = align256(solve_bytes(n_t, n_x, restart) + 2 * (size_t)n_t * n_x * sizeof(double)) +
           exact_x_bytes(n_t, n_x, 1, n_slices);
  return STBEM_OK;
}

int stbem_solve_mixed_exact(stbem_ctx* ctx, int nt, int nx, const stbem_exact_operand* Vx, const float* V32,
                            const float* D32, const double* L, const double* f, double* w,
                            const stbem_solve_opts* opts, double inner_tol, stbem_solve_info* info, void* work,
                            size_t work_bytes) {
  if (ctx && !Vx) return fail(ctx, STBEM_ERR_ARG, "solve_mixed_exact: NULL operand");
  return solve_mixed_impl(ctx, nt, nx, nullptr, Vx, V32, D32, L, f, w, opts, inner_tol, info, work, work_bytes);
}

int stbem_solve_mixed_tc_workspace_bytes(int n_t, int n_x, int restart, int n_slices, size_t* bytes) {
  if (!bytes || n_t < 1 || n_x < 1 || restart < 1 || n_slices < stbem::kExactMinSlices ||
      n_slices > stbem::kExactMaxSlices)
    return STBEM_ERR_ARG;
  *bytes = align256(solve_bytes(n_t, n_x, restart) + 2 * (size_t)n_t * n_x * sizeof(double)) +
           align256(exact_x_bytes(n_t, n_x, 1, n_slices)) + tc3_bytes(n_t, n_x, 1);
  return STBEM_OK;
}

int stbem_solve_mixed_tc(stbem_ctx* ctx, int nt, int nx, const stbem_exact_operand* Vx, const void* V_hi,
                         const void* V_mid, const void* V_lo, const void* D_hi, const void* D_mid, const void* D_lo,
                         const double* L, const double* f, double* w, const stbem_solve_opts* opts, double inner_tol,
                         stbem_solve_info* info, void* work, size_t work_bytes) {
  if (ctx && (!Vx || !V_hi)) return fail(ctx, STBEM_ERR_ARG, "solve_mixed_tc: NULL operand");
  if (ctx && opts && opts->precondition && !D_hi) return fail(ctx, STBEM_ERR_ARG, "solve_mixed_tc: NULL D");
  const void* V3[3] = {V_hi, V_mid, V_lo};
  const void* D3[3] = {D_hi, D_mid, D_lo};
  return solve_mixed_impl(ctx, nt, nx, nullptr, Vx, nullptr, nullptr, L, f, w, opts, inner_tol, info, work,
                          work_bytes, V3, D3);
}

int stbem_round_f32(stbem_ctx* ctx, size_t n, const double* src, float* dst) {
  if (!ctx) return STBEM_ERR_ARG;
  if (!src || !dst) return fail(ctx, STBEM_ERR_ARG, "round_f32: NULL pointer");
  CUDA_TRY(ctx, cudaSetDevice(ctx->device), "round_f32: set device");
  CUDA_TRY(ctx, stbem::round_f32_launch(src, dst, n, ctx->stream), "round_f32");
  return STBEM_OK;
}

}  // extern "C"
