// CPU checks of the library's host-side planning logic (csrc/host_logic.h):
// FFT stage radices, mask row lists and batched column work lists,
// built with the host C++ compiler by tests/test_host_logic.py.  Prints one
// line per failed property and exits non-zero if any failed.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <set>
#include <vector>

#include "host_logic.h"

static int failures = 0;
#define CHECK(cond, ...)                      \
  do {                                        \
    if (!(cond)) {                            \
      std::printf("FAIL %s: ", #cond);        \
      std::printf(__VA_ARGS__);               \
      std::printf("\n");                      \
      ++failures;                             \
    }                                         \
  } while (0)

static bool is_prime(int r) {
  if (r < 2) return false;
  for (int d = 2; d * d <= r; ++d)
    if (r % d == 0) return false;
  return true;
}

// Every length the library transforms (1..1024 along x and y, 1..128 along t):
// the radices multiply to n, are 4, 2, 3, 5, 7 or a larger prime, come in the
// preferred order, and the plan fits its stage table.
static void check_fft_factor() {
  for (int n = 1; n <= 1024; ++n) {
    int radix[24];
    const int ns = recon::fft_factor(n, radix, 24);
    long long prod = 1;
    for (int s = 0; s < ns; ++s) prod *= radix[s];
    CHECK(prod == n, "n=%d product %lld", n, prod);
    CHECK(ns <= 24, "n=%d stages %d", n, ns);
    int rank_prev = -1, last_big = 0;
    for (int s = 0; s < ns; ++s) {
      const int r = radix[s];
      const int rank = r == 4 ? 0 : r == 2 ? 1 : r == 3 ? 2 : r == 5 ? 3 : r == 7 ? 4 : 5;
      CHECK(rank < 5 ? true : (is_prime(r) && r >= 11), "n=%d radix %d", n, r);
      CHECK(rank >= rank_prev, "n=%d radix order", n);
      if (rank == 5) {
        CHECK(r >= last_big, "n=%d large radices not increasing", n);
        last_big = r;
      }
      rank_prev = rank;
    }
    // a 4 is taken before any 2: at most one 2 remains
    int twos = 0;
    for (int s = 0; s < ns; ++s) twos += radix[s] == 2;
    CHECK(twos <= 1, "n=%d has %d radix-2 stages", n, twos);
  }
  // n = 1: no stage (the transform is the identity)
  int r[24];
  CHECK(recon::fft_factor(1, r, 24) == 0, "n=1");
}

// Work lists: every column of every slice exactly once, offsets consistent,
// each CTA's list ordered by (slice, column), the longest list reported, the
// single-slice interleave, and LPT's balance: no CTA carries more than the
// lightest one plus one column's cost.
static void check_work_lists(const std::vector<long long>& cost, const std::vector<int>& ncols, int grid) {
  std::vector<unsigned> work;
  std::vector<int> off;
  int work_max = -1;
  recon::lpt_work_lists(cost, ncols, grid, work, off, work_max);
  const int n = (int)ncols.size();
  long long total = 0;
  for (int c : ncols) total += c;
  CHECK((long long)work.size() == total, "items %zu of %lld", work.size(), total);
  CHECK((int)off.size() == grid + 1 && off[0] == 0 && off[grid] == (int)work.size(), "offsets");
  std::set<unsigned> seen(work.begin(), work.end());
  CHECK((long long)seen.size() == total, "duplicates");
  for (unsigned w : work) {
    const int q = (int)(w >> 24), c = (int)(w & 0xFFFFFFu);
    CHECK(q < n && c < ncols[q], "item (%d, %d) out of range", q, c);
  }
  int longest = 0;
  long long lo = -1, hi = -1, maxcost = 0;
  for (long long c : cost) maxcost = std::max(maxcost, c);
  for (int b = 0; b < grid; ++b) {
    CHECK(off[b] <= off[b + 1], "offsets not monotone at %d", b);
    longest = std::max(longest, off[b + 1] - off[b]);
    long long load = 0;
    for (int k = off[b]; k < off[b + 1]; ++k) {
      load += cost[work[k] >> 24];
      if (k > off[b]) CHECK(work[k - 1] < work[k], "CTA %d list not ordered", b);
    }
    lo = lo < 0 ? load : std::min(lo, load);
    hi = std::max(hi, load);
    if (n == 1)
      for (int k = off[b]; k < off[b + 1]; ++k)
        CHECK((int)(work[k] & 0xFFFFFFu) == b + (k - off[b]) * grid, "interleave at CTA %d", b);
  }
  CHECK(work_max == longest, "work_max %d, longest %d", work_max, longest);
  CHECK(hi - lo <= maxcost, "imbalance %lld above one column's cost %lld", hi - lo, maxcost);
}

// Row lists of random ky-t masks: the sampled rows of every frame in order,
// offsets and the largest count; a full [Nt][Ny][Nx] mask that is constant
// along kx gives the same lists, and one flipped entry is reported at its
// (frame, row) when it is the first row that differs.
static void check_mask_rows(std::mt19937& rng) {
  for (int trial = 0; trial < 30; ++trial) {
    const int Nt = 1 + (int)(rng() % 9), Ny = 1 + (int)(rng() % 40), Nx = 1 + (int)(rng() % 7);
    std::vector<uint8_t> m((size_t)Nt * Ny), full((size_t)Nt * Ny * Nx);
    for (auto& v : m) v = (uint8_t)(rng() % 3 == 0 ? (1 + rng() % 255) : 0);   // any nonzero means sampled
    for (int t = 0; t < Nt; ++t)
      for (int j = 0; j < Ny; ++j)
        for (int i = 0; i < Nx; ++i) full[((size_t)t * Ny + j) * Nx + i] = m[(size_t)t * Ny + j] ? 1 : 0;
    std::vector<int> rows, off, rows_f, off_f;
    int bt = -1, bj = -1;
    const int maxm = recon::mask_rows(m.data(), Nt, Ny, Nx, false, rows, off, &bt, &bj);
    int expect_max = 0;
    size_t k = 0;
    for (int t = 0; t < Nt; ++t) {
      CHECK(off[t] == (int)k, "trial %d offset of frame %d", trial, t);
      int cnt = 0;
      for (int j = 0; j < Ny; ++j)
        if (m[(size_t)t * Ny + j]) {
          CHECK(k < rows.size() && rows[k] == j, "trial %d frame %d row %d", trial, t, j);
          ++k;
          ++cnt;
        }
      expect_max = std::max(expect_max, cnt);
    }
    CHECK(k == rows.size() && off[Nt] == (int)k, "trial %d row count", trial);
    CHECK(maxm == expect_max, "trial %d maxm %d, expected %d", trial, maxm, expect_max);
    const int maxf = recon::mask_rows(full.data(), Nt, Ny, Nx, true, rows_f, off_f, &bt, &bj);
    CHECK(maxf == maxm && rows_f == rows && off_f == off, "trial %d full mask differs from the row mask", trial);
    if (Nx > 1) {
      const int t = (int)(rng() % Nt), j = (int)(rng() % Ny), i = 1 + (int)(rng() % (Nx - 1));
      full[((size_t)t * Ny + j) * Nx + i] ^= 1;
      bt = bj = -1;
      CHECK(recon::mask_rows(full.data(), Nt, Ny, Nx, true, rows_f, off_f, &bt, &bj) == -1 && bt == t && bj == j,
            "trial %d flipped (%d, %d, %d) reported at (%d, %d)", trial, t, j, i, bt, bj);
    }
  }
}

int main() {
  check_fft_factor();
  {
    std::mt19937 rng(7);
    check_mask_rows(rng);
  }
  // the cardiac plan alone, and a plan with fewer columns than CTAs
  check_work_lists({2206203904LL / 8192}, {8192}, 152);
  check_work_lists({1000}, {100}, 152);
  // seeded uneven batches (the batched workload's shape mix), up to 255 slices
  std::mt19937 rng(64);
  for (int trial = 0; trial < 10; ++trial) {
    const int n = 2 + (int)(rng() % (trial < 8 ? 70 : 254));
    std::vector<long long> cost(n);
    std::vector<int> ncols(n);
    const int ny[] = {128, 160, 192, 256}, nt[] = {16, 24, 32, 40};
    for (int q = 0; q < n; ++q) {
      const int Ny = ny[rng() % 4], Nx = ny[rng() % 4], Nt = nt[rng() % 4];
      cost[q] = 8LL * Ny * (Ny + 1) / 2 + 4096;
      ncols[q] = Nx * Nt;
    }
    check_work_lists(cost, ncols, 152);
  }
  if (failures == 0) std::printf("OK\n");
  return failures ? 1 : 0;
}
