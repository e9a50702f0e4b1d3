// Quadrature orders and switches of the discretisation rule (the paper prints
// none; they are fixed here and documented in the repository's design notes).
//
// Space, per pair of boundary pieces (segments, or half-segments for the dual
// space Y_h of Section 2):
//   lags 0 and 1: regular pairs  kRegular01 x kRegular01 Gauss-Legendre,
//                 near pairs     kNear01 x kNear01,
//                 identical      diagonal split, graded in |xi - eta|,
//                 sharing a vertex  Duffy split at the vertex, graded radially;
//   lags d >= 2:  space_order(d)^2 Gauss-Legendre for every pair.
// Time, per lag d: closed form at d = 0, 1 (series-rearranged for z < 1 at
// d = 1); d >= 2: closed form if z_d = c / (d ht) > d / 2, else the Peano form
// with peano_order(k) Gauss nodes on interval [k ht, (k+1) ht].
#pragma once
#include "hd.cuh"

namespace stbem {

constexpr int kRegular01 = 12;
constexpr int kNear01 = 16;
constexpr double kGradedSigma = 0.2;
constexpr int kGradedLevels = 18;
constexpr int kGradedPoints = 16;
constexpr int kGradedN = (kGradedLevels + 1) * kGradedPoints;   // 304 nodes
constexpr int kSingularInner = 4;
constexpr int kDuffyAngular = 16;
constexpr double kNearGapRatio = 0.5;

STB_HD int space_order(int d) { return d >= 32 ? 4 : (d >= 8 ? 6 : 8); }
STB_HD int peano_order(int k) { return k >= 32 ? 6 : (k >= 2 ? 8 : 16); }

// Initial-data operator M_h^0, per (segment, triangle) pair.  Classes:
// touching (the triangle has an endpoint of the segment as a vertex), near
// (gap < kM0NearRatio x max(h_i, diam)), regular.  Tensor rule of order n: n
// Gauss points on the segment times the n x n collapsed rule on the triangle.
// m = 0: order 8 (regular) or 12 (near); touching pairs use the polar rule
// (outer points graded (v^3) toward shared vertices, sinh transformation
// along each far edge, radial points graded (w^3)).  m >= 1, every class: the
// order follows rho^2 = 4 m ht / (alpha s^2), s = max(h_i, diam) (diffusion
// length over pair size): the first step of kM0Steps with rho^2 >= threshold.
constexpr int kM0Order0Regular = 8;
constexpr int kM0Order0Near = 12;
constexpr int kM0NSteps = 5;
STB_HD double m0_step_threshold(int k) { return k == 0 ? 1e4 : (k == 1 ? 144.0 : (k == 2 ? 5.0 : (k == 3 ? 1.44 : 0.0))); }
STB_HD int m0_step_order(int k) { return k == 0 ? 3 : (k == 1 ? 4 : (k == 2 ? 6 : (k == 3 ? 8 : 12))); }
constexpr double kM0NearRatio = 1.0;
constexpr int kM0PolarOuter = 8;       // per half of the segment
constexpr int kM0PolarRadial = 12;
constexpr int kM0PolarAngular = 12;
constexpr double kM0Degenerate = 1e-12;   // |A2| <= this x L^2: sub-triangle skipped

// Gauss-Legendre orders kept in the tables and their offsets.
constexpr int kGaussOrders[6] = {3, 4, 6, 8, 12, 16};
STB_HD int gauss_offset(int n) {
  return n == 3 ? 0 : n == 4 ? 3 : n == 6 ? 7 : n == 8 ? 13 : n == 12 ? 21 : 33;
}
constexpr int kGaussTotal = 49;

// Pair classes used at lags 0 and 1.
enum PairClass { kRegular = 0, kNear = 1, kIdentical = 2, kAdjNext = 3, kAdjPrev = 4 };

struct RuleTables {
  double gx[kGaussTotal];   // Gauss-Legendre nodes on [0,1], orders 4,6,8,12,16
  double gw[kGaussTotal];   // and weights
  double grx[kGradedN];     // composite Gauss graded toward 0
  double grw[kGradedN];
};

}  // namespace stbem
