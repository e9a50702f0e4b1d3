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

// Gauss-Legendre orders kept in the tables and their offsets.
constexpr int kGaussOrders[5] = {4, 6, 8, 12, 16};
STB_HD int gauss_offset(int n) {
  return n == 4 ? 0 : n == 6 ? 4 : n == 8 ? 10 : n == 12 ? 18 : 30;
}
constexpr int kGaussTotal = 46;

// Pair classes used at lags 0 and 1.
enum PairClass { kRegular = 0, kNear = 1, kIdentical = 2, kAdjNext = 3, kAdjPrev = 4 };

struct RuleTables {
  double gx[kGaussTotal];   // Gauss-Legendre nodes on [0,1], orders 4,6,8,12,16
  double gw[kGaussTotal];   // and weights
  double grx[kGradedN];     // composite Gauss graded toward 0
  double grw[kGradedN];
};

}  // namespace stbem
