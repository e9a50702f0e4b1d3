// Lag sharding of one problem across ranks (host logic, no CUDA).
//
// Section 3 distributes the blocks of the block-lower-triangular matrices
// over processes.  With a uniform time grid every block at one lag is the same
// (Toeplitz), so here the unit of distribution is a lag block: rank r holds
// the lags of some chunks and computes the part of every product that they
// contribute, y_r[m] = sum_{d held by r} A^(d) x[m - d]; one sum over ranks
// (an all-reduce) gives the product.  The work of lag d is proportional to
// n_t - d (the steps it multiplies), so chunks of `chunk` consecutive lags are
// dealt to ranks in snake order (0, 1, .., R-1, R-1, .., 1, 0, 0, 1, ..),
// which balances both the work and the number of blocks stored per rank.
#pragma once

#include <vector>

namespace stbem {

// Owner of chunk c among n_ranks ranks (snake order).
inline int lag_chunk_owner(int c, int n_ranks) {
  const int round = c / n_ranks, q = c % n_ranks;
  return (round % 2 == 0) ? q : n_ranks - 1 - q;
}

// The lag ranges [begin, end) held by `rank`, increasing, adjacent chunks of
// the same rank merged.  Empty when the rank owns no chunk (n_ranks larger
// than the number of chunks).
inline std::vector<int> lag_ranges(int n_t, int n_ranks, int rank, int chunk) {
  std::vector<int> out;
  const int nchunks = (n_t + chunk - 1) / chunk;
  for (int c = 0; c < nchunks; ++c) {
    if (lag_chunk_owner(c, n_ranks) != rank) continue;
    const int a = c * chunk, b = (c + 1) * chunk < n_t ? (c + 1) * chunk : n_t;
    if (!out.empty() && out.back() == a) out.back() = b;
    else {
      out.push_back(a);
      out.push_back(b);
    }
  }
  return out;
}

}  // namespace stbem
