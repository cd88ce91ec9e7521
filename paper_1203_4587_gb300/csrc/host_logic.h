// Host-side planning logic with no CUDA types, so that it also builds as
// plain C++ for the CPU checks in tests/host_logic_check.cpp.
//
//   fft_factor      the stage radices of the Stockham FFTs (every transform
//                   of the library: rows, columns and time)
//   lpt_work_lists  the per-CTA column lists of the column-inverse kernel
//   mask_rows       the sampled ky rows of each frame of a Cartesian mask
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <functional>
#include <queue>
#include <utility>
#include <vector>

namespace recon {

// Radices of an n-point FFT, at most max_stages of them: 4s first, then 2, 3,
// 5 and 7, then the remaining odd factors in increasing order (each done by
// the generic direct stage).  Returns the stage count; the radices multiply
// to n unless n needs more than max_stages stages.
inline int fft_factor(int n, int* radix, int max_stages) {
  int m = n, ns = 0;
  const int pref[] = {4, 2, 3, 5, 7};
  for (int r : pref) {
    while (m % r == 0 && ns < max_stages) { radix[ns++] = r; m /= r; }
  }
  for (int r = 11; m > 1 && ns < max_stages; r += 2) {
    while (m % r == 0) { radix[ns++] = r; m /= r; }
  }
  return ns;
}

// Column work lists: column c of slice q (ncols[q] columns, each streaming
// cost[q] bytes) becomes the item (q << 24) | c.  With one slice the columns
// are interleaved (CTA b takes b, b + grid, ...); otherwise they go out by
// longest-processing-time-first to the least-loaded CTA, and each CTA's list
// is then ordered by (slice, column).  CTA b's items are
// work[off[b] .. off[b+1]); work_max is the longest list.  q < 256 and
// c < 2^24.
inline void lpt_work_lists(const std::vector<long long>& cost, const std::vector<int>& ncols, int grid,
                           std::vector<unsigned>& work, std::vector<int>& off, int& work_max) {
  struct Col { long long cost; int q, c; };
  const int n = (int)ncols.size();
  std::vector<Col> cols;
  for (int q = 0; q < n; ++q)
    for (int c = 0; c < ncols[q]; ++c) cols.push_back({cost[q], q, c});
  std::vector<std::vector<std::pair<int, int>>> per(grid);
  if (n == 1) {
    for (size_t k = 0; k < cols.size(); ++k) per[k % grid].push_back({cols[k].q, cols[k].c});
  } else {
    std::stable_sort(cols.begin(), cols.end(), [](const Col& a, const Col& b) { return a.cost > b.cost; });
    using Load = std::pair<long long, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
    for (int b = 0; b < grid; ++b) pq.push({0, b});
    for (const Col& c : cols) {
      Load l = pq.top();
      pq.pop();
      per[l.second].push_back({c.q, c.c});
      pq.push({l.first + c.cost, l.second});
    }
    for (auto& v : per) std::sort(v.begin(), v.end());
  }
  work.clear();
  off.assign(grid + 1, 0);
  work_max = 0;
  for (int b = 0; b < grid; ++b) {
    off[b] = (int)work.size();
    for (const auto& w : per[b]) work.push_back(((unsigned)w.first << 24) | (unsigned)w.second);
    work_max = std::max(work_max, (int)per[b].size());
  }
  off[grid] = (int)work.size();
}

// Sampled ky rows of a Cartesian ky-t mask (Section II-A: every kx of a
// sampled row is sampled).  mask is [Nt][Ny] (full = false) or [Nt][Ny][Nx]
// (full = true, and then each row must be constant along kx).  Frame t's
// rows, in increasing ky, are rows[rowoff[t] .. rowoff[t+1]).  Returns the
// largest per-frame count, or -1 with (*bad_t, *bad_j) the first row that
// differs along kx.
inline int mask_rows(const uint8_t* mask, int Nt, int Ny, int Nx, bool full, std::vector<int>& rows,
                     std::vector<int>& rowoff, int* bad_t, int* bad_j) {
  rows.clear();
  rowoff.assign(Nt + 1, 0);
  int maxm = 0;
  for (int t = 0; t < Nt; ++t) {
    for (int j = 0; j < Ny; ++j) {
      bool on;
      if (full) {
        const uint8_t* rowp = &mask[((size_t)t * Ny + j) * Nx];
        on = rowp[0] != 0;
        for (int i = 1; i < Nx; ++i) {
          if ((rowp[i] != 0) != on) {
            *bad_t = t;
            *bad_j = j;
            return -1;
          }
        }
      } else {
        on = mask[(size_t)t * Ny + j] != 0;
      }
      if (on) rows.push_back(j);
    }
    rowoff[t + 1] = (int)rows.size();
    maxm = std::max(maxm, rowoff[t + 1] - rowoff[t]);
  }
  return maxm;
}

}  // namespace recon
