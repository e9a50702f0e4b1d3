// Initial-data operator M_h^0 of Section 1, eq. (4):
//
//   M0[m][i][j] = int_{tau_m} int_{gamma_i} int_Omega U*(x - y, t) phi_j(y) dy ds_x dt,
//
// phi_j the P1 hat functions of a triangulation Omega_h.  The time integral is
// exact, int_{tau_m} U*(r, t) dt = G(r, t_{m+1}) - G(r, t_m) with
// G(r, s) = alpha/(4 pi) E1(alpha r^2 / (4 s)), G(r, 0) = 0.  Space: per pair
// (segment i, triangle k) the rule of rule.cuh: at m = 0 a tensor rule whose
// order follows the pair class, or the polar rule for touching pairs; for
// m >= 1 a tensor rule whose order follows rho^2 = 4 m ht / (alpha s^2), the
// diffusion length over the pair size.  The m of one order range share the
// rule's points, so E1 is evaluated once per (point, time t_m).
//
// One warp per pair.  Full chunks of 31 steps of one order range: lanes over
// 31 consecutive times t_{m0} .. t_{m0+31}; the points are computed 32 at a
// time, one per lane, and broadcast by shuffles; lane l evaluates
// G(t_{m0+l}) and takes G(t_{m0+l-1}) from lane l - 1.  The remaining steps
// (and m = 0) in groups of up to 3: lanes over the rule's points, per-lane
// sums per step, one warp reduction per step; each point's G at the first
// time of the next group is carried in shared memory (ranges of at most 512
// points).
//
// Assembly writes M0[m][i][j] += for the three vertices of the triangle; it is
// launched once per colour of a node-disjoint colouring of the triangles, so
// no two threads of a launch write one entry and the order of the sums is
// fixed.  The matrix-free product y = M0 u0 contracts u0 at the points, sums
// a block's triangles per warp row in shared memory, then the blocks' partial
// sums in a fixed order.
#include <cuda_runtime.h>

#include "initial.h"
#include "rule.cuh"
#include "special.cuh"

namespace stbem {

namespace {

__constant__ RuleTables c_m0tab;

#ifndef STBEM_M0_MINB
#define STBEM_M0_MINB 5     // resident blocks per SM the pair kernels are compiled for
#endif
constexpr int kM0Warps = 4;
constexpr int kM0Threads = 32 * kM0Warps;
#ifndef STBEM_M0_SHORT
#define STBEM_M0_SHORT 3    // steps per chunk of the points-per-lane path
#endif
constexpr int kShortMax = STBEM_M0_SHORT;
constexpr int kApplyChunk = 64;     // triangles per block of the product
constexpr int kGCarry = 512;        // points whose G(t) a warp carries between step groups

enum { kClsR = 0, kClsN = 1, kClsT = 2 };

struct Seg {
  double ax, ay, bx, by, h;
};
struct Tri {
  double x[3], y[3], area, diam;
  int j[3];
};

__device__ __forceinline__ double pt_seg(double px, double py, double s0x, double s0y, double s1x, double s1y) {
  const double ex = s1x - s0x, ey = s1y - s0y;
  const double L2 = ex * ex + ey * ey;
  double tt = ((px - s0x) * ex + (py - s0y) * ey) / L2;
  tt = fmin(fmax(tt, 0.0), 1.0);
  const double dx = px - (s0x + tt * ex), dy = py - (s0y + tt * ey);
  return sqrt(dx * dx + dy * dy);
}

__device__ __forceinline__ void load_pair(const DevMesh& M, const DevDomain& D, int i, int k, Seg* S, Tri* T) {
  S->ax = M.sx0[i];
  S->ay = M.sy0[i];
  S->bx = M.sx1[i];
  S->by = M.sy1[i];
  S->h = M.slen[i];
  for (int c = 0; c < 3; ++c) {
    const int j = D.tri[3 * k + c];
    T->j[c] = j;
    T->x[c] = D.nx[j];
    T->y[c] = D.ny[j];
  }
  T->area = D.area[k];
  T->diam = D.diam[k];
}

// touching: a triangle vertex is an endpoint of gamma_i; near: the gap
// between segment and triangle below kM0NearRatio x max(h_i, diam).
__device__ __forceinline__ int pair_class(const DevMesh& M, const DevDomain& D, int i, const Seg& S, const Tri& T,
                                          bool* sh0, bool* sh1) {
  const int ba = D.bnode[i], bb = D.bnode[i + 1 == M.N ? 0 : i + 1];
  *sh0 = (T.j[0] == ba) || (T.j[1] == ba) || (T.j[2] == ba);
  *sh1 = (T.j[0] == bb) || (T.j[1] == bb) || (T.j[2] == bb);
  if (*sh0 || *sh1) return kClsT;
  double gap = 1e300;
  for (int c = 0; c < 3; ++c) {
    const int c1 = c == 2 ? 0 : c + 1;
    gap = fmin(gap, pt_seg(T.x[c], T.y[c], S.ax, S.ay, S.bx, S.by));
    gap = fmin(gap, pt_seg(S.ax, S.ay, T.x[c], T.y[c], T.x[c1], T.y[c1]));
    gap = fmin(gap, pt_seg(S.bx, S.by, T.x[c], T.y[c], T.x[c1], T.y[c1]));
  }
  return gap < kM0NearRatio * fmax(S.h, T.diam) ? kClsN : kClsR;
}

// Point q of the order-n tensor rule: n Gauss points on the segment (slowest
// index) times the collapsed n x n rule on the triangle, y = v0 + u ((1-v)
// (v1-v0) + v (v2-v0)), dy = 2|omega| u du dv.  Returns r^2 and the weight
// times the three barycentrics.
__device__ __forceinline__ void tensor_point(const Seg& S, const Tri& T, int n, int q, double* r2, double* wl) {
  const int go = gauss_offset(n);
  const int qo = q / (n * n), qt = q - qo * n * n;
  const int qu = qt / n, qv = qt - qu * n;
  const double g = c_m0tab.gx[go + qo], U = c_m0tab.gx[go + qu], V = c_m0tab.gx[go + qv];
  const double xx = S.ax + g * (S.bx - S.ax), xy = S.ay + g * (S.by - S.ay);
  const double yx = T.x[0] + U * ((1.0 - V) * (T.x[1] - T.x[0]) + V * (T.x[2] - T.x[0]));
  const double yy = T.y[0] + U * ((1.0 - V) * (T.y[1] - T.y[0]) + V * (T.y[2] - T.y[0]));
  const double dx = xx - yx, dy = xy - yy;
  *r2 = dx * dx + dy * dy;
  const double w = (S.h * c_m0tab.gw[go + qo]) * (2.0 * T.area * (c_m0tab.gw[go + qu] * c_m0tab.gw[go + qv] * U));
  wl[0] = w * (1.0 - U);
  wl[1] = w * (U * (1.0 - V));
  wl[2] = w * (U * V);
}

constexpr int kPolarPoints = 2 * kM0PolarOuter * 3 * kM0PolarAngular * kM0PolarRadial;

// Point q of the polar rule of a touching pair (see rule.cuh): returns false
// for points of a degenerate sub-triangle (skipped).
__device__ __forceinline__ bool polar_point(const Seg& S, const Tri& T, bool sh0, bool sh1, int q, double* r2,
                                            double* wl) {
  const int rr = q % kM0PolarRadial;
  q /= kM0PolarRadial;
  const int ta = q % kM0PolarAngular;
  q /= kM0PolarAngular;
  const int a = q % 3;
  const int o = q / 3;
  const int half = o / kM0PolarOuter, qo = o - half * kM0PolarOuter;
  // outer point x on gamma_i, distance rho from the half's end vertex
  const int go = gauss_offset(kM0PolarOuter);
  const double g = c_m0tab.gx[go + qo], gw = c_m0tab.gw[go + qo];
  const bool shared = half == 0 ? sh0 : sh1;
  double rho, wr;
  if (shared) {
    rho = 0.5 * S.h * (g * g * g);
    wr = 0.5 * S.h * (3.0 * (g * g)) * gw;
  } else {
    rho = 0.5 * S.h * g;
    wr = 0.5 * S.h * gw;
  }
  const double ex = half == 0 ? S.ax : S.bx, ey = half == 0 ? S.ay : S.by;
  const double ox = half == 0 ? S.bx : S.ax, oy = half == 0 ? S.by : S.ay;
  const double f = rho / S.h;
  const double xx = ex + f * (ox - ex), xy = ey + f * (oy - ey);
  // barycentrics of x (the linear extension outside the triangle)
  const double d0x = xx - T.x[0], d0y = xy - T.y[0];
  const double e1x = T.x[1] - T.x[0], e1y = T.y[1] - T.y[0];
  const double e2x = T.x[2] - T.x[0], e2y = T.y[2] - T.y[0];
  const double det = e1x * e2y - e1y * e2x;
  const double u1 = (d0x * e2y - d0y * e2x) / det;
  const double u2 = (e1x * d0y - e1y * d0x) / det;
  double lx[3] = {1.0 - u1 - u2, u1, u2};
  // sub-triangle (x, v_a, v_b)
  const int b = a == 2 ? 0 : a + 1;
  const double evx = T.x[b] - T.x[a], evy = T.y[b] - T.y[a];
  const double L = sqrt(evx * evx + evy * evy);
  const double A2 = (T.x[a] - xx) * (T.y[b] - xy) - (T.y[a] - xy) * (T.x[b] - xx);
  if (!(fabs(A2) > kM0Degenerate * L * L)) return false;
  const double p = fabs(A2) / L;
  const double t0 = ((xx - T.x[a]) * evx + (xy - T.y[a]) * evy) / L;
  const double m0 = asinh(-t0 / p), m1 = asinh((L - t0) / p);
  const int ga = gauss_offset(kM0PolarAngular), gr = gauss_offset(kM0PolarRadial);
  const double mu = m0 + (m1 - m0) * c_m0tab.gx[ga + ta];
  const double wmu = (m1 - m0) * c_m0tab.gw[ga + ta];
  const double rh = p * cosh(mu);
  const double sig = (t0 + p * sinh(mu)) / L;
  const double wv = c_m0tab.gx[gr + rr];
  const double s = wv * wv * wv;
  const double sw = 3.0 * (wv * wv) * c_m0tab.gw[gr + rr];
  const double sr = s * rh;
  *r2 = sr * sr;
  const double w = (A2 > 0.0 ? 1.0 : -1.0) * wr * wmu * (p * rh) * (sw * s);
  double le[3] = {0.0, 0.0, 0.0};
  le[a] = 1.0 - sig;
  le[b] = sig;
  for (int c = 0; c < 3; ++c) wl[c] = w * (lx[c] + s * (le[c] - lx[c]));
  return true;
}

struct Range {
  int b, e, n;
};
constexpr int kMaxRanges = 1 + kM0NSteps;

// rho^2 = 4 m ht / (alpha s^2), evaluated as a quotient of products (no sums)
__device__ __forceinline__ double m0_rho2(int m, double ht, double alpha, double s) {
  return (4.0 * (double)m * ht) / (alpha * s * s);
}

// first m >= 1 with rho^2(m) >= thr (monotone in m); at most nt
__device__ int first_step(double thr, double ht, double alpha, double s, int nt) {
  if (thr <= 0.0) return 1;
  const double guess = ceil(thr * alpha * s * s / (4.0 * ht));
  int m = guess < 1.0 ? 1 : (guess > (double)nt ? nt : (int)guess);
  for (int it = 0; it < 8 && m > 1 && m0_rho2(m - 1, ht, alpha, s) >= thr; ++it) --m;
  for (int it = 0; it < 8 && m < nt && m0_rho2(m, ht, alpha, s) < thr; ++it) ++m;
  while (m < nt && m0_rho2(m, ht, alpha, s) < thr) ++m;   // guess far off: walk (monotone)
  return m;
}

// m ranges and tensor orders of a pair: m = 0 (not for touching pairs, which
// take the polar rule there), then the rho steps for m >= 1
__device__ __forceinline__ int pair_ranges(int cls, double s, const DevMesh& M, Range* r) {
  const int nt = M.n_t;
  int nr = 0;
  if (cls != kClsT) r[nr++] = Range{0, 1, cls == kClsR ? kM0Order0Regular : kM0Order0Near};
  // steps in ascending threshold: [1, b(1.44)) order 12, [b(1.44), b(5)) 8, ...
  int lo = 1;
  for (int k = kM0NSteps - 1; k >= 0; --k) {
    const int hi = k == 0 ? nt : first_step(m0_step_threshold(k - 1), M.ht, M.alpha, s, nt);
    const int b = min(lo, nt), e = min(max(hi, b), nt);
    if (b < e) r[nr++] = Range{b, e, m0_step_order(k)};
    lo = max(lo, e);
  }
  return nr;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sink of one pair's sums: either the three matrix entries or, for the
// product, the warp's row of per-m sums in shared memory.
template <bool APPLY>
struct Sink {
  double* M0;       // assembly
  size_t rowN, rowM;
  int i;
  int j[3];
  double* ysm;      // product: this warp's row (n_t)
  double u[3];      // product: u0 at the vertices
  __device__ __forceinline__ void put(int m, const double* v) const {
    if (APPLY) {
      ysm[m] += v[0];
    } else {
      double* row = M0 + ((size_t)m * rowN + (size_t)i) * rowM;
      for (int c = 0; c < 3; ++c) row[j[c]] += v[c];
    }
  }
};

// gc: this warp's kGCarry doubles of shared memory (G at the first time of
// the next step group, per point, for ranges of at most kGCarry points)
template <bool APPLY>
__device__ void pair_unit(const DevMesh& M, const DevDomain& D, int i, int k, const Sink<APPLY>& sink,
                          double* gc) {
  constexpr int NV = APPLY ? 1 : 3;
  const int lane = threadIdx.x & 31;
  Seg S;
  Tri T;
  load_pair(M, D, i, k, &S, &T);
  bool sh0, sh1;
  const int cls = pair_class(M, D, i, S, T, &sh0, &sh1);
  const double ca = 0.25 * M.alpha;
  const double scale = M.alpha / kFourPi;
  const int nt = M.n_t;

  auto contract = [&](const double* wl, double* v) {
    if (APPLY) {
      v[0] = wl[0] * sink.u[0] + wl[1] * sink.u[1] + wl[2] * sink.u[2];
    } else {
      v[0] = wl[0];
      v[1] = wl[1];
      v[2] = wl[2];
    }
  };

  // touching pairs, m = 0: polar rule, G(., t_1) only
  if (cls == kClsT) {
    double acc[NV];
    for (int c = 0; c < NV; ++c) acc[c] = 0.0;
    const double inv_t1 = 1.0 / M.ht;
    for (int q = lane; q < kPolarPoints; q += 32) {
      double r2, wl[3], v[3];
      if (!polar_point(S, T, sh0, sh1, q, &r2, wl)) continue;
      contract(wl, v);
      const double G = e1_only(ca * r2 * inv_t1);
      for (int c = 0; c < NV; ++c) acc[c] = fma(G, v[c], acc[c]);
    }
    double out[3];
    for (int c = 0; c < NV; ++c) out[c] = scale * warp_sum(acc[c]);
    if (lane == 0) sink.put(0, out);
  }

  Range rg[kMaxRanges];
  const int nr = pair_ranges(cls, fmax(S.h, T.diam), M, rg);
  for (int r = 0; r < nr; ++r) {
    const int b = rg[r].b, e = rg[r].e, n = rg[r].n;
    const int nq = n * n * n;
    // full chunks of 31 steps: lanes over times t_{m0} .. t_{m0+31}; lane l
    // evaluates G(t_{m0+l}) and owns m = m0 + l - 1
    const int e_long = b + ((e - b) / 31) * 31;
    for (int m0 = b; m0 < e_long; m0 += 31) {
      const double inv_t = 1.0 / ((double)(m0 + lane) * M.ht);
      double acc[NV];
      for (int c = 0; c < NV; ++c) acc[c] = 0.0;
      for (int q0 = 0; q0 < nq; q0 += 32) {
        double r2 = 1.0, wl[3] = {0.0, 0.0, 0.0}, v[3] = {0.0, 0.0, 0.0};
        if (q0 + lane < nq) {
          tensor_point(S, T, n, q0 + lane, &r2, wl);
          contract(wl, v);
        }
        const int cnt = min(32, nq - q0);
        for (int jj = 0; jj < cnt; ++jj) {
          const double rj = __shfl_sync(0xffffffffu, r2, jj);
          double vj[NV];
          for (int c = 0; c < NV; ++c) vj[c] = __shfl_sync(0xffffffffu, v[c], jj);
          const double G = e1_only(ca * rj * inv_t);
          const double Gm = __shfl_up_sync(0xffffffffu, G, 1);
          const double d = G - Gm;
          for (int c = 0; c < NV; ++c) acc[c] = fma(d, vj[c], acc[c]);
        }
      }
      if (lane >= 1) {
        double out[3];
        for (int c = 0; c < NV; ++c) out[c] = scale * acc[c];
        sink.put(m0 + lane - 1, out);
      }
    }
    // the rest in chunks of up to kShortMax steps: lanes over points, all
    // steps of the chunk per lane, one warp reduction per step
    for (int c0 = e_long; c0 < e; c0 += kShortMax) {
      const int ce = min(c0 + kShortMax, e);
      double inv_t[kShortMax + 1];
#pragma unroll
      for (int mm = 0; mm <= kShortMax; ++mm) inv_t[mm] = 1.0 / ((double)(c0 + mm) * M.ht);
      double acc[kShortMax][NV];
#pragma unroll
      for (int mm = 0; mm < kShortMax; ++mm)
        for (int c = 0; c < NV; ++c) acc[mm][c] = 0.0;
      const bool carry = nq <= kGCarry;
      for (int q = lane; q < nq; q += 32) {
        double r2, wl[3], v[3];
        tensor_point(S, T, n, q, &r2, wl);
        contract(wl, v);
        const double c2 = ca * r2;
        // G(t_{c0}): 0 at t_0, carried from the previous group of this range
        // (same time, same value), else evaluated
        double Gp = c0 == 0 ? 0.0 : (carry && c0 > e_long ? gc[q] : e1_only(c2 * inv_t[0]));
#pragma unroll
        for (int mm = 0; mm < kShortMax; ++mm) {
          if (c0 + mm < ce) {
            const double Gn = e1_only(c2 * inv_t[mm + 1]);
            const double d = Gn - Gp;
            for (int c = 0; c < NV; ++c) acc[mm][c] = fma(d, v[c], acc[mm][c]);
            Gp = Gn;
          }
        }
        if (carry) gc[q] = Gp;
      }
#pragma unroll
      for (int mm = 0; mm < kShortMax; ++mm) {
        if (c0 + mm < ce) {
          double out[3];
          for (int c = 0; c < NV; ++c) out[c] = scale * warp_sum(acc[mm][c]);
          if (lane == 0) sink.put(c0 + mm, out);
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kM0Threads, STBEM_M0_MINB) k_m0_assemble(DevMesh M, DevDomain D, const int* __restrict__ tris,
                                                            int n_tris, double* __restrict__ M0) {
  __shared__ double gcache[kM0Warps * kGCarry];
  const long long unit = (long long)blockIdx.x * kM0Warps + (threadIdx.x >> 5);
  if (unit >= (long long)M.N * n_tris) return;
  const int i = (int)(unit / n_tris);
  const int k = tris[unit - (long long)i * n_tris];
  Sink<false> sink;
  sink.M0 = M0;
  sink.rowN = (size_t)M.N;
  sink.rowM = (size_t)D.M;
  sink.i = i;
  for (int c = 0; c < 3; ++c) sink.j[c] = D.tri[3 * k + c];
  sink.ysm = nullptr;
  pair_unit<false>(M, D, i, k, sink, gcache + (threadIdx.x >> 5) * kGCarry);
}

// block (chunk, i): triangles chunk*kApplyChunk .. +kApplyChunk, warp w takes
// every kM0Warps-th; per-warp rows of per-m sums, then the block's sum.
__global__ void __launch_bounds__(kM0Threads, STBEM_M0_MINB) k_m0_apply(DevMesh M, DevDomain D, const double* __restrict__ u0,
                                                         double* __restrict__ part, int n_chunks) {
  extern __shared__ double ysm[];    // kM0Warps x n_t
  __shared__ double gcache[kM0Warps * kGCarry];
  const int chunk = blockIdx.x, i = blockIdx.y;
  const int nt = M.n_t;
  for (int t = threadIdx.x; t < kM0Warps * nt; t += kM0Threads) ysm[t] = 0.0;
  __syncthreads();
  const int w = threadIdx.x >> 5;
  const int k0 = chunk * kApplyChunk, k1 = min(D.K, k0 + kApplyChunk);
  Sink<true> sink;
  sink.M0 = nullptr;
  sink.rowN = sink.rowM = 0;
  sink.i = i;
  sink.ysm = ysm + w * nt;
  for (int k = k0 + w; k < k1; k += kM0Warps) {
    for (int c = 0; c < 3; ++c) {
      sink.j[c] = D.tri[3 * k + c];
      sink.u[c] = u0[sink.j[c]];
    }
    pair_unit<true>(M, D, i, k, sink, gcache + w * kGCarry);
    __syncwarp();
  }
  __syncthreads();
  for (int m = threadIdx.x; m < nt; m += kM0Threads) {
    double s = 0.0;
    for (int ww = 0; ww < kM0Warps; ++ww) s += ysm[ww * nt + m];
    part[((size_t)i * n_chunks + chunk) * nt + m] = s;
  }
}

__global__ void k_m0_apply_reduce(int N, int nt, int n_chunks, const double* __restrict__ part, double scale,
                                  double* __restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * nt) return;
  const int m = (int)(t / N), i = (int)(t - (long long)m * N);
  double s = 0.0;
  for (int c = 0; c < n_chunks; ++c) s += part[((size_t)i * n_chunks + c) * nt + m];
  y[(size_t)m * N + i] += scale * s;
}

__global__ void k_planewave(DevMesh M, DevDomain D, double ct, double st, double* __restrict__ g,
                            double* __restrict__ u0) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = M.N;
  if (g && t < M.n_t * N) {
    const int n = t / N, p = t - n * N;
    const double al = M.alpha;
    const double tavg = al / M.ht * (exp(-((double)n * M.ht) / al) - exp(-((double)(n + 1) * M.ht) / al));
    g[t] = tavg * sin(M.vx[p] * ct + M.vy[p] * st);
  }
  if (u0 && t < D.M) u0[t] = sin(D.nx[t] * ct + D.ny[t] * st);
}

// ---- evaluation of u in Q by the representation formula, eq. (2) ----------
//
// u_h(x, t) = sum_j u0_j int_Omega U*(x - y, t) phi_j dy
//           + 1/alpha sum_{n, i} w[n][i] int_{gamma_i} [G(r, s_n) - G(r, s_{n+1})] ds
//           - 1/alpha sum_{n, p} g[n][p] int_Gamma phi_p [H(r, s_n) - H(r, s_{n+1})] ds,
// s_n = t - t_n, s_{n+1} = t - min(t_{n+1}, t) (the time integrals exactly),
// G(r, s) = alpha/(4 pi) E1(alpha r^2 / (4 s)), H(r, s) = alpha q / (2 pi r^2)
// e^{-alpha r^2 / (4 s)}, q = (x - y) . n_y, both 0 for s <= 0.  Rules: per
// segment 16 / 12 / 8 Gauss points for dist(x, gamma_i) < 2 h_i / < 4 h_i /
// beyond; per triangle the collapsed n x n rule with n from the step table at
// rho^2 = 4 t / (alpha diam^2).  One block per point; threads over segments,
// then over triangles; G and H are evaluated once per time s_k and shared by
// the two steps that meet there; fixed-order block reduction.

constexpr int kEvalThreads = 256;

__device__ __forceinline__ int boundary_order(double dist, double h) {
  return dist < 2.0 * h ? 16 : (dist < 4.0 * h ? 12 : 8);
}

__device__ __forceinline__ int volume_order(double t, double alpha, double diam) {
  const double r2 = (4.0 * t) / (alpha * diam * diam);
  for (int k = 0; k < kM0NSteps; ++k)
    if (r2 >= m0_step_threshold(k)) return m0_step_order(k);
  return m0_step_order(kM0NSteps - 1);
}

__global__ void __launch_bounds__(kEvalThreads) k_eval_points(DevMesh M, DevDomain D, int has_volume,
                                                              const double* __restrict__ xy,
                                                              const double* __restrict__ tp,
                                                              const double* __restrict__ w,
                                                              const double* __restrict__ g,
                                                              const double* __restrict__ u0,
                                                              double* __restrict__ u) {
  __shared__ double red[kEvalThreads / 32];
  const int p = blockIdx.x;
  const double x0 = xy[2 * p], x1 = xy[2 * p + 1], t = tp[p];
  const double al = M.alpha, ht = M.ht;
  const int N = M.N;
  int n_last = (int)ceil(t / ht);
  n_last = n_last < M.n_t ? n_last : M.n_t;
  const double cG = al / kFourPi, ca = 0.25 * al;
  double acc = 0.0;
  for (int i = threadIdx.x; i < N; i += kEvalThreads) {
    const double ax = M.sx0[i], ay = M.sy0[i], bx = M.sx1[i], by = M.sy1[i], h = M.slen[i];
    const double nx = M.snx[i], ny = M.sny[i];
    const int nb = boundary_order(pt_seg(x0, x1, ax, ay, bx, by), h);
    const int go = gauss_offset(nb);
    const int ip = i + 1 == N ? 0 : i + 1;
    double si = 0.0;
    for (int q = 0; q < nb; ++q) {
      const double xi = c_m0tab.gx[go + q], wq = c_m0tab.gw[go + q] * h;
      const double dx = x0 - (ax + xi * (bx - ax)), dy = x1 - (ay + xi * (by - ay));
      const double r2 = dx * dx + dy * dy;
      const double qn = dx * nx + dy * ny;
      const double c2 = ca * r2;
      const double hq = al * qn / (2.0 * kPi * r2);
      // s_0 = t
      double Gp = cG * e1_only(c2 / t);
      double Hp = hq * exp_neg_fast(c2 / t);
      double sw = 0.0, sg = 0.0;
      for (int n = 0; n < n_last; ++n) {
        const double tn1 = (double)(n + 1) * ht;
        const double s1 = n + 1 < n_last ? t - tn1 : t - (tn1 < t ? tn1 : t);
        double Gn = 0.0, Hn = 0.0;
        if (s1 > 0.0) {
          Gn = cG * e1_only(c2 / s1);
          Hn = hq * exp_neg_fast(c2 / s1);
        }
        sw = fma(w[(size_t)n * N + i], Gp - Gn, sw);
        const double gv = g[(size_t)n * N + i] * (1.0 - xi) + g[(size_t)n * N + ip] * xi;
        sg = fma(gv, Hp - Hn, sg);
        Gp = Gn;
        Hp = Hn;
      }
      si = fma(wq, sw - sg, si);
    }
    acc += si / al;
  }
  if (has_volume) {
    const double cU = al / (kFourPi * t);
    for (int k = threadIdx.x; k < D.K; k += kEvalThreads) {
      const int j0 = D.tri[3 * k], j1 = D.tri[3 * k + 1], j2 = D.tri[3 * k + 2];
      const double v0x = D.nx[j0], v0y = D.ny[j0];
      const double e1x = D.nx[j1] - v0x, e1y = D.ny[j1] - v0y, e2x = D.nx[j2] - v0x, e2y = D.ny[j2] - v0y;
      const double u00 = u0[j0], u01 = u0[j1], u02 = u0[j2];
      const int n = volume_order(t, al, D.diam[k]);
      const int go = gauss_offset(n);
      double sv = 0.0;
      for (int a = 0; a < n; ++a) {
        const double U = c_m0tab.gx[go + a], wu = c_m0tab.gw[go + a] * U;
        for (int b = 0; b < n; ++b) {
          const double V = c_m0tab.gx[go + b];
          const double yx = v0x + U * ((1.0 - V) * e1x + V * e2x);
          const double yy = v0y + U * ((1.0 - V) * e1y + V * e2y);
          const double dx = x0 - yx, dy = x1 - yy;
          const double r2 = dx * dx + dy * dy;
          const double uh = (1.0 - U) * u00 + U * (1.0 - V) * u01 + U * V * u02;
          sv = fma(wu * c_m0tab.gw[go + b], cU * exp_neg_fast(ca * r2 / t) * uh, sv);
        }
      }
      acc = fma(2.0 * D.area[k], sv, acc);
    }
  }
  const double ws = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ws;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kEvalThreads / 32; ++k) s += red[k];
    u[p] = s;
  }
}

}  // namespace

cudaError_t upload_m0_rule_tables(const RuleTables& t, cudaStream_t s) {
  cudaError_t e = cudaMemcpyToSymbolAsync(c_m0tab, &t, sizeof(RuleTables), 0, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

cudaError_t m0_assemble_launch(const DevMesh& M, const DevDomain& D, const int* tris, int n_tris, double* M0,
                               cudaStream_t s) {
  if (n_tris <= 0) return cudaSuccess;
  const long long units = (long long)M.N * n_tris;
  const long long blocks = (units + kM0Warps - 1) / kM0Warps;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  k_m0_assemble<<<(unsigned)blocks, kM0Threads, 0, s>>>(M, D, tris, n_tris, M0);
  count_launches(1);
  return cudaGetLastError();
}

static int apply_chunks(int K) { return (K + kApplyChunk - 1) / kApplyChunk; }

size_t m0_apply_workspace_bytes(int nt, int N, int K) {
  return (size_t)N * apply_chunks(K) * nt * sizeof(double);
}

cudaError_t m0_apply_launch(const DevMesh& M, const DevDomain& D, const double* u0, double scale, double* y,
                            void* work, cudaStream_t s) {
  const int nc = apply_chunks(D.K);
  const size_t smem = (size_t)kM0Warps * M.n_t * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_m0_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  double* part = static_cast<double*>(work);
  k_m0_apply<<<dim3(nc, M.N), kM0Threads, smem, s>>>(M, D, u0, part, nc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = (long long)M.N * M.n_t;
  k_m0_apply_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(M.N, M.n_t, nc, part, scale, y);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t evaluate_launch(const DevMesh& M, const DevDomain* D, int n_points, const double* xy, const double* t,
                            const double* w, const double* g, const double* u0, double* u, cudaStream_t s) {
  if (n_points <= 0) return cudaSuccess;
  DevDomain dd{};
  if (D) dd = *D;
  k_eval_points<<<n_points, kEvalThreads, 0, s>>>(M, dd, D && u0 ? 1 : 0, xy, t, w, g, u0, u);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t planewave_launch(const DevMesh& M, const DevDomain& D, double theta, double* g, double* u0,
                             cudaStream_t s) {
  const long long n = (long long)M.n_t * M.N > D.M ? (long long)M.n_t * M.N : D.M;
  k_planewave<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(M, D, cos(theta), sin(theta), g, u0);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace stbem
