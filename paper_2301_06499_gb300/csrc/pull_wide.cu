// Pull kernel for wide signatures (many seeds per node): a warp per row
// piece, its 32 lanes spread over the row's words.
//
// Same round as k_pull (Alg. 1 inner loop on the deltas of round t-1): for
// each in-neighbour u of the piece, Sig_next(v) |= D_{t-1}(u). With W words
// per node, lane l holds words l, l + 32, l + 64, ... of the row, so the
// warp reads each gathered neighbour row as one contiguous 8·W-byte segment
// (256 bytes per 32 words) instead of W/8 separate 64-byte pieces; column
// indices are loaded 32 at a time (one per lane), their changed bits tested
// in parallel, and the surviving neighbours broadcast by shuffle. Dense rounds
// walk the row-major piece list of every unsaturated row, sparse rounds the
// pieces the post kernel claimed. Activity, statistics, frontier appends and
// the finish of split rows follow k_pull.
#include "kernels.cuh"

namespace pg {

// NW words per lane held in registers (rows of up to 32·NW words); NW = 0
// sweeps a longer row in passes of 128 words (4 per lane, so that 16 loads
// of four neighbours are in flight), re-reading the piece's columns (from
// L1) in each pass.
// Five resident blocks per SM (48 registers, no spills).
//
// PW: PROPAGATE-S passes as the words of one signature; m_active is counted
// per pass here, in dense and sparse rounds alike (see count_pass_words).
template <int NW, bool PW>
__global__ void __launch_bounds__(kBlock, 5) k_pull_wide(Params p) {
  constexpr int R = NW > 0 ? NW : 4;  // words per lane per pass
  Ctrl *ctrl = p.ctrl;
  if (*(volatile int32_t *)&ctrl->done) return;
  const int t = ctrl->t;
  const int mode = ctrl->mode;
  const uint64_t *Dprev = (t & 1) ? p.D0 : p.D1;
  const uint32_t *Cprev = (t & 1) ? p.C0 : p.C1;
  int32_t *F = (t & 1) ? p.F1 : p.F0;
  uint32_t *Ccur = (t & 1) ? p.C1 : p.C0;
  uint32_t *Kcur = (t & 1) ? p.K1 : p.K0;
  uint32_t *Knext = (t & 1) ? p.K0 : p.K1;
  uint32_t *Kwcur = (t & 1) ? p.Kw1 : p.Kw0;

  const int64_t gtid = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * kBlock;
  for (int64_t i = gtid; i < p.nbm; i += nthreads) Knext[i] = 0u;
  if constexpr (PW) {  // the per-pass claim bits of round t+1
    uint32_t *Kwnext = (t & 1) ? p.Kw0 : p.Kw1;
    for (int64_t i = gtid; i < p.nbm * p.Wp; i += nthreads) Kwnext[i] = 0u;
  }

  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid >> 5;
  const int64_t nwarps = nthreads >> 5;
  const int Wp = p.Wp;
  const int passes = NW > 0 ? 1 : (Wp + 32 * R - 1) / (32 * R);
  const bool tc = test_changed_now(p, ctrl);
  unsigned long long my_mact = 0, my_work = 0, my_scan = 0, my_gath = 0, my_items = 0,
                     my_rows = 0;
  // dense: every row's pieces; sparse: the claimed pieces; mixed (a packed
  // batch): the pieces of graphs that chose a full sweep, then the claimed ones
  const int64_t ndense = mode != kModeSparse ? p.nPall : 0;
  const int64_t nitems = ndense + (mode != kModeDense ? (int64_t)ctrl->nA : 0);

  for (int64_t item = warp; item < nitems; item += nwarps) {
    const bool dense = item < ndense;
    const ulonglong2 it = dense ? p.Pall[item] : p.A[item - ndense];
    const int64_t b = (int64_t)it.x;
    const int32_t v = (int32_t)(it.y >> 32);
    const bool whole = (it.y & 0x80000000ULL) != 0ULL;
    const int len = (int)(it.y & 0x7FFFFFFFULL);
    if (len == 0) continue;
    if (dense && test_bit(p.Sat, v)) continue;  // warp-uniform
    if (dense && p.gfsum) {  // a packed batch: only graphs in a full sweep
      const int gs = __ldg(p.node_graph + v);
      if (p.gfsum[(size_t)((t - 1) & 1) * (size_t)p.nseg + gs] <= __ldg(p.gthr + gs)) continue;
    }
    const uint64_t *xr = p.X + (size_t)v * Wp;
    uint64_t *yr = p.Y + (size_t)v * Wp;
    bool any_delta = false, row_changed = false;
    uint32_t pw_words = 0, pw_seeds = 0;  // PW: this lane's active passes
    for (int pass = 0; pass < passes; ++pass) {
      const int w0 = pass * 32 * R + lane;  // lane's first word of this pass
      uint64_t acc[R];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = 0ULL;
      for (int a0 = 0; a0 < len; a0 += 32) {
        int32_t u = a0 + lane < len ? __ldg(p.col + b + a0 + lane) : -1;
        if (u >= 0 && tc && !test_bit(Cprev, u)) u = -1;
        unsigned m = __ballot_sync(kFullMask, u >= 0);
        if (pass == 0 && lane == 0) my_gath += (unsigned long long)__popc(m);
        while (m) {  // four neighbours at a time: their loads are independent
          int32_t uu[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int src = m ? __ffs(m) - 1 : 0;
            uu[q] = m ? __shfl_sync(kFullMask, u, src) : -1;
            m &= m ? m - 1 : 0u;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (uu[q] >= 0) {
              const uint64_t *dr = Dprev + (size_t)uu[q] * Wp;
#pragma unroll
              for (int r = 0; r < R; ++r) {
                const int w = w0 + 32 * r;
                if (w < Wp && gather_ok(p, uu[q], w))
                  acc[r] |= __ldg(reinterpret_cast<const unsigned long long *>(dr) + w);
              }
            }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int w = w0 + 32 * r;
        if (w >= Wp) continue;
        any_delta |= acc[r] != 0ULL;
        uint64_t own = 0ULL;
        if (whole || (PW && acc[r]))
          own = __ldg(reinterpret_cast<const unsigned long long *>(xr) + w);
        if (PW && acc[r] && (whole || !set_bit(Kwcur + (size_t)w * (size_t)p.nbm, v))) {
          // pass w is active in this row unless the row already holds all its bits
          const uint64_t vm = valid_mask(w, p.s);
          if ((own | ~vm) != ~0ULL) {
            ++pw_words;
            pw_seeds += (uint32_t)__popcll(vm);
          }
        }
        if (whole) {
          const uint64_t nw = own | acc[r];
          if (nw != own) {
            yr[w] = nw;
            row_changed = true;
          }
        } else if (acc[r]) {
          const unsigned long long old =
              atomicOr(reinterpret_cast<unsigned long long *>(yr + w), (unsigned long long)acc[r]);
          row_changed |= (old | acc[r]) != old;
        }
      }
    }
    any_delta = __any_sync(kFullMask, any_delta);
    row_changed = __any_sync(kFullMask, row_changed);
    if constexpr (PW) {  // the row's active passes, summed over the lanes
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        pw_words += __shfl_xor_sync(kFullMask, pw_words, off);
        pw_seeds += __shfl_xor_sync(kFullMask, pw_seeds, off);
      }
      if (lane == 0 && pw_words) {
        const unsigned long long deg =
            whole ? (unsigned long long)len
                  : (unsigned long long)(__ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v));
        my_mact += deg * pw_words;
        my_work += deg * pw_seeds;
        my_rows += pw_words;
      }
    }
    bool app = false;
    if (lane == 0) {
      ++my_items;
      my_scan += (unsigned long long)len;
      if (!PW && dense && any_delta) {  // active in round t (sparse rounds count at the claim)
        unsigned long long deg = 0;
        if (whole) {
          deg = (unsigned long long)len;
          ++my_rows;
        } else if (!set_bit(Kcur, v)) {
          deg = (unsigned long long)(__ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v));
          ++my_rows;
        }
        my_mact += deg;
        my_work += deg * (unsigned long long)seeds_of(p, v);
        if (p.gmact && deg)  // a packed batch: the row's own graph
          atomicAdd(p.gmact + (size_t)(t - ctrl->row_base) * (size_t)p.nseg + __ldg(p.node_graph + v),
                    deg);
      }
      if (row_changed && (dense ? any_delta : true)) {
        if (whole) {
          atomicOr(Ccur + (v >> 5), 1u << (v & 31));
          app = true;
        } else {
          app = !set_bit(Ccur, v);
        }
      }
    }
    frontier_append(p, ctrl, F, v, app, lane);
  }
  RoundStats *r = p.rs + (t - ctrl->row_base);
  const unsigned long long vals[6] = {my_mact, my_work, my_scan, my_gath, my_items, my_rows};
  unsigned long long *const dsts[6] = {&r->m_active, &r->work,  &r->scanned,
                                       &r->gathered, &r->items, &r->rows};
  block_add<6>(vals, dsts);
}

template <bool PW>
static PullFn pick(int Wp) {
  if (Wp <= 32) return &k_pull_wide<1, PW>;
  if (Wp <= 64) return &k_pull_wide<2, PW>;
  if (Wp <= 96) return &k_pull_wide<3, PW>;
  if (Wp <= 128) return &k_pull_wide<4, PW>;
  return &k_pull_wide<0, PW>;
}

PullFn pull_fn_wide(int Wp, bool pw) { return pw ? pick<true>(Wp) : pick<false>(Wp); }

}  // namespace pg
