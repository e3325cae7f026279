// Progressive sampling (host driver over pg_propagate_p and pg_metrics).
//
// Sec. 4.2 remarks that PROPAGATE-S can keep adding seeds until the
// estimates are good enough, and Sec. 6 names this progressive sampling as a
// use of the seed-by-seed variant; the paper fixes no stopping rule. Thm. 3
// bounds the sample a fixed accuracy needs by the order ln n / eps^2 (no
// constant given). This driver draws seeds uniformly without replacement in
// blocks, runs PROPAGATE-P on each block, appends the block's per-seed count
// columns (seeds never interact, Sec. 4, so the columns equal those of one
// call over every drawn seed) and stops at ceil(ln n / eps^2) seeds (constant
// 1, a reading), or earlier, once the average distance and the interpolated
// effective diameter both move by less than a relative tolerance over two
// consecutive blocks.
//
// Seed draws: value i of a SplitMix64 stream (Steele, Lea and Flood, OOPSLA
// 2014: state_i = key + (i + 1) * golden gamma, then the published output
// mix) mapped to [0, n) by a 128-bit multiply-high; a value already drawn is
// skipped, so the seeds are the stream's first distinct values and every
// smaller sample is a prefix of a larger one.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "propagate.h"

namespace {

uint64_t splitmix64_at(uint64_t key, uint64_t i) {
  uint64_t z = key + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" pg_status pg_progressive(pg_graph *g, double eps, int32_t block, double stable_tol,
                                    uint64_t rng_seed, int32_t *seeds, int32_t *s_drawn,
                                    pg_counts *out, pg_metrics_out *history,
                                    int32_t max_history, int32_t *blocks,
                                    const pg_options *opt, void *stream) {
  if (!g || !seeds || !s_drawn || !out || !out->counts || out->s < 1 || out->max_rounds < 0 ||
      !(eps > 0.0) || block < 1 || stable_tol < 0.0 || max_history < 0 ||
      (max_history > 0 && !history))
    return PG_EINVAL;
  int64_t n = 0, m = 0;
  pg_status rc = pg_graph_info(g, &n, &m);
  if (rc) return rc;
  const double want = std::ceil(std::log((double)(n > 2 ? n : 2)) / (eps * eps));
  const int64_t target = (int64_t)std::fmin((double)n, want);
  if (target > out->s) return PG_EINVAL;  // the caller's columns must hold the sample
  const int32_t cap = out->max_rounds;
  const size_t S = (size_t)out->s;
  std::memset(out->counts, 0, sizeof(uint32_t) * (size_t)(cap + 1) * S);
  if (out->m_active) std::memset(out->m_active, 0, sizeof(uint64_t) * (size_t)(cap + 2));
  std::vector<bool> taken((size_t)n, false);
  uint64_t draw = 0;
  int32_t drawn = 0, T = 0, nblk = 0, calm = 0;
  pg_metrics_out prev{};
  std::vector<uint32_t> bc, packed;
  std::vector<uint64_t> bm;
  while (drawn < target) {
    const int32_t b0 = drawn;
    const int32_t nb = (int32_t)std::min<int64_t>(block, target - drawn);
    for (int32_t k = 0; k < nb; ++k) {
      int64_t x;
      do {
        x = (int64_t)(((unsigned __int128)splitmix64_at(rng_seed, draw++) * (uint64_t)n) >> 64);
      } while (taken[(size_t)x]);
      taken[(size_t)x] = true;
      seeds[drawn++] = (int32_t)x;
    }
    bc.assign((size_t)(cap + 1) * nb, 0u);
    bm.assign((size_t)cap + 2, 0ULL);
    pg_counts c{};
    c.s = nb;
    c.max_rounds = cap;
    c.counts = bc.data();
    c.m_active = bm.data();
    rc = pg_propagate_p(g, seeds + b0, nb, &c, opt, stream);
    if (rc == PG_ERANGE) {
      out->rounds = cap + 1;
      *s_drawn = drawn;
      if (blocks) *blocks = nblk;
      return PG_ERANGE;
    }
    if (rc) return rc;
    for (int32_t t = 0; t <= c.rounds; ++t)
      std::memcpy(out->counts + (size_t)t * S + b0, bc.data() + (size_t)t * nb,
                  sizeof(uint32_t) * nb);
    if (out->m_active)  // the work each block's own run did
      for (int32_t t = 0; t <= std::min(c.rounds + 1, cap + 1); ++t) out->m_active[t] += bm[t];
    T = std::max(T, c.rounds);
    // metrics over every drawn seed so far (columns packed side by side)
    packed.assign((size_t)(T + 1) * drawn, 0u);
    for (int32_t t = 0; t <= T; ++t)
      std::memcpy(packed.data() + (size_t)t * drawn, out->counts + (size_t)t * S,
                  sizeof(uint32_t) * drawn);
    pg_counts all{};
    all.s = drawn;
    all.max_rounds = T;
    all.rounds = T;
    all.counts = packed.data();
    pg_metrics_out mo{};
    if ((rc = pg_metrics(&all, n, 9, 10, &mo))) return rc;
    if (nblk < max_history) history[nblk] = mo;
    if (nblk > 0 && stable_tol > 0.0) {
      const double d1 = std::fabs(mo.avg_distance - prev.avg_distance) /
                        std::fmax(prev.avg_distance, 1e-300);
      const double d2 = std::fabs(mo.eff_diameter_interp - prev.eff_diameter_interp) /
                        std::fmax(prev.eff_diameter_interp, 1e-300);
      calm = std::fmax(d1, d2) < stable_tol ? calm + 1 : 0;
    }
    prev = mo;
    ++nblk;
    if (calm >= 2) break;
  }
  out->rounds = T;
  *s_drawn = drawn;
  if (blocks) *blocks = nblk;
  return PG_OK;
}
