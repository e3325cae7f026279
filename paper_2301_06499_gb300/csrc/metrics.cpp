// Distance metrics from the per-round, per-seed counts (host, FP64 from exact
// 64-bit integer sums).
//
//   R[r]     = sum over seeds and hops k <= r of counts[k][i]: the sampled
//              neighbourhood function |N(r)| restricted to the seeds (Sec. 3;
//              Alg. 1 "R[r] = R[r-1] + CountAll[r]"), pairs (x_i, x_i)
//              included.
//   diameter = T, the last hop with a new pair (Alg. 1's Delta_LB).
//   eff_diameter = min k with R[k] >= tau R[T] (Sec. 3 definition, Alg. 1's
//              final step), tau = tau_num / tau_den compared by
//              cross-multiplication.
//   avg_distance = sum_r r (R[r] - R[r-1]) over pairs with u != v, i.e. divided
//              by R[T] - s (Sec. 3's sum over r in [Delta] counts no r = 0
//              term); avg_distance_incl_self divides by R[T] as Alg. 1 does.
//   connectivity_rate = (R[T] - s) / (s (n - 1)), Sec. 3's alpha on the sample.
//   reachable_pairs = (n / s) R[T], Alg. 1's last line.
#include <cstdint>
#include <vector>

#include "propagate.h"

extern "C" pg_status pg_metrics(const pg_counts *c, int64_t n, int32_t tau_num, int32_t tau_den,
                                pg_metrics_out *out) {
  if (!c || !out || !c->counts || c->s < 1 || c->rounds < 0 || c->rounds > c->max_rounds ||
      n < 1 || tau_den < 1 || tau_num < 1 || tau_num > tau_den)
    return PG_EINVAL;
  const int64_t s = c->s, T = c->rounds;
  std::vector<uint64_t> R((size_t)T + 1);
  uint64_t run = 0, dist_sum = 0;
  for (int64_t r = 0; r <= T; ++r) {
    uint64_t at = 0;
    const uint32_t *row = c->counts + (size_t)r * (size_t)s;
    for (int64_t i = 0; i < s; ++i) at += row[i];
    run += at;
    R[(size_t)r] = run;
    dist_sum += (uint64_t)r * at;
  }
  const uint64_t RT = R[(size_t)T];
  int64_t k = 0;
  while ((unsigned __int128)(uint64_t)tau_den * R[(size_t)k] <
         (unsigned __int128)(uint64_t)tau_num * RT)
    ++k;
  const double tau = (double)tau_num / (double)tau_den;
  double interp = 0.0;
  if (k > 0) {
    const double lo = (double)R[(size_t)k - 1], hi = (double)R[(size_t)k];
    interp = (double)(k - 1) + (tau * (double)RT - lo) / (hi - lo);
  }
  const uint64_t pairs = RT >= (uint64_t)s ? RT - (uint64_t)s : 0;
  out->diameter = (int32_t)T;
  out->eff_diameter = (int32_t)k;
  out->eff_diameter_interp = interp;
  out->avg_distance = pairs ? (double)dist_sum / (double)pairs : 0.0;
  out->avg_distance_incl_self = RT ? (double)dist_sum / (double)RT : 0.0;
  out->connectivity_rate = n > 1 ? (double)pairs / ((double)s * (double)(n - 1)) : 0.0;
  out->reachable_pairs = ((double)n / (double)s) * (double)RT;
  out->R_last = RT;
  out->dist_sum = dist_sum;
  return PG_OK;
}
