// Device helpers and the pull kernel of one PROPAGATE round.
//
// Round t (Alg. 1's do-while body; Alg. 2's inner loop for one pass) is two
// kernels:
//   pull(t): for every active node v,  new = X[v] | OR_{u in in(v)} X[u];
//            if new != X[v]: Y[v] = new, v joins the frontier F_t.
//   post(t): for v in F_t: per-seed popcount of X[v] ^ Y[v] (the new pairs at
//            distance t), then X[v] = Y[v]; build the work list of t+1.
// X holds the signatures of round t-1 and is only read by the pull, Y only
// written, so a round never sees its own updates (the synchronous diffusion
// of Alg. 1: Sig_next is built from Sig, then copied back).
#pragma once

#include "common.cuh"

namespace pg {

__device__ __forceinline__ bool test_bit(const uint32_t *bm, int64_t v) {
  return (__ldg(bm + (v >> 5)) >> (v & 31)) & 1u;
}
// Volatile read for bitmaps written by other blocks of the running kernel.
__device__ __forceinline__ bool test_bit_live(const uint32_t *bm, int64_t v) {
  return (*((volatile const uint32_t *)bm + (v >> 5)) >> (v & 31)) & 1u;
}
// Sets bit v, returns whether it was already set.
__device__ __forceinline__ bool set_bit(uint32_t *bm, int64_t v) {
  const uint32_t b = 1u << (v & 31);
  return (atomicOr(bm + (v >> 5), b) & b) != 0u;
}

// Bits of word w that belong to one of the s seeds of the pass.
__device__ __forceinline__ uint64_t valid_mask(int w, int s) {
  const int lo = w * 64;
  if (lo + 64 <= s) return ~0ULL;
  if (lo >= s) return 0ULL;
  return (1ULL << (s - lo)) - 1ULL;
}

template <int CW>
__device__ __forceinline__ void load_words(uint64_t (&a)[CW], const uint64_t *p) {
  if constexpr (CW == 1) {
    a[0] = __ldg(reinterpret_cast<const unsigned long long *>(p));
  } else {
#pragma unroll
    for (int k = 0; k < CW; k += 2) {
      const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p) + k / 2);
      a[k] = v.x;
      a[k + 1] = v.y;
    }
  }
}

template <int CW>
__device__ __forceinline__ void or_words(uint64_t (&a)[CW], const uint64_t *p) {
  if constexpr (CW == 1) {
    a[0] |= __ldg(reinterpret_cast<const unsigned long long *>(p));
  } else {
#pragma unroll
    for (int k = 0; k < CW; k += 2) {
      const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p) + k / 2);
      a[k] |= v.x;
      a[k + 1] |= v.y;
    }
  }
}

template <int CW>
__device__ __forceinline__ void store_words(uint64_t *p, const uint64_t (&a)[CW]) {
  if constexpr (CW == 1) {
    p[0] = a[0];
  } else {
#pragma unroll
    for (int k = 0; k < CW; k += 2)
      reinterpret_cast<ulonglong2 *>(p)[k / 2] = make_ulonglong2(a[k], a[k + 1]);
  }
}

// Block-wide sum of up to 4 counters, then one atomicAdd per counter.
__device__ __forceinline__ void block_add4(unsigned long long a, unsigned long long b,
                                           unsigned long long c, unsigned long long d,
                                           unsigned long long *pa, unsigned long long *pb,
                                           unsigned long long *pc, unsigned long long *pd) {
  __shared__ unsigned long long red[4][kBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(kFullMask, a, off);
    b += __shfl_xor_sync(kFullMask, b, off);
    c += __shfl_xor_sync(kFullMask, c, off);
    d += __shfl_xor_sync(kFullMask, d, off);
  }
  if (lane == 0) {
    red[0][w] = a;
    red[1][w] = b;
    red[2][w] = c;
    red[3][w] = d;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    unsigned long long s = 0;
    for (int k = 0; k < kBlock / 32; ++k) s += red[threadIdx.x][k];
    unsigned long long *dst = threadIdx.x == 0 ? pa : threadIdx.x == 1 ? pb : threadIdx.x == 2 ? pc : pd;
    if (s && dst) atomicAdd(dst, s);
  }
}

// Pull kernel of round t.
//
// Work items are row pieces (row v, piece k): arcs [row_ptr[v] + k L,
// min(row_ptr[v+1], row_ptr[v] + (k+1) L)). Dense rounds walk the static list
// of every piece and skip saturated rows; sparse rounds walk the pieces of
// the rows claimed by the previous post kernel. A group of G lanes takes one
// piece; each lane ORs whole neighbour signatures (CW words per load
// sequence, several loads in flight per lane), then the group reduces with
// shuffles. A row of a single piece is finished by the group leader (compare
// with X[v], write Y[v]); a row cut into pieces is combined with 64-bit
// atomicOr into Y[v], and the piece whose OR first changed it appends v.
//
//  CHG: OR only in-neighbours whose bit in C_{t-1} is set (they are the only
//       ones that can add bits: the others were ORed in the round before).
//       Dense rounds always test C_{t-1}: a node with no changed in-neighbour
//       is not active in round t.
//  EB:  PROPAGATE-S early exit: a lane stops scanning once X[v] | acc has
//       every valid bit of the pass set (Alg. 2's break at the first set
//       in-neighbour, for 1..64 planes at once).
template <int CW, int G, bool CHG, bool EB>
__global__ void __launch_bounds__(kBlock) k_pull(Params p) {
  static_assert(G >= 1 && G <= 32 && (32 % G) == 0, "group size");
  Ctrl *ctrl = p.ctrl;
  if (*(volatile int32_t *)&ctrl->done) return;
  const int t = ctrl->t;
  const bool dense = ctrl->mode == kModeDense;
  const uint32_t *Cprev = (t & 1) ? p.C0 : p.C1;
  uint32_t *Ccur = (t & 1) ? p.C1 : p.C0;
  uint32_t *Kcur = (t & 1) ? p.K1 : p.K0;
  uint32_t *Knext = (t & 1) ? p.K0 : p.K1;

  const int64_t gtid = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * kBlock;
  for (int64_t i = gtid; i < p.nbm; i += nthreads) Knext[i] = 0u;

  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1);
  const int gw = lane / G;
  constexpr int GPW = 32 / G;
  const int64_t warp = gtid >> 5;
  const int64_t nwarps = nthreads >> 5;
  const int64_t nitems = dense ? p.nPall : (int64_t)ctrl->nA;
  const unsigned long long *items = dense ? p.Pall : p.A;
  const int nch = p.Wp / CW;
  const size_t Wp = (size_t)p.Wp;
  unsigned long long my_mact = 0, my_scan = 0, my_gath = 0, my_items = 0;

  for (int64_t base = warp * GPW; base < nitems; base += nwarps * GPW) {
    const int64_t item = base + gw;
    bool act = false, whole = true;
    int32_t v = 0;
    int64_t b = 0, e = 0, indeg = 0;
    if (item < nitems) {
      const unsigned long long it = items[item];
      v = (int32_t)(it >> 32);
      const int64_t k = (int64_t)(it & 0xFFFFFFFFULL);
      const int64_t rb = __ldg(p.row_ptr + v), re = __ldg(p.row_ptr + v + 1);
      indeg = re - rb;
      b = rb + k * p.L;
      e = min(re, b + (int64_t)p.L);
      whole = indeg <= p.L;
      act = dense ? !test_bit(p.Sat, v) : true;
      if (!act) b = e = 0;
    }
    if (gl == 0 && act) ++my_items;
    bool any_chg = false, row_changed = false;
    const uint64_t *xv = p.X + (size_t)v * Wp;
    for (int c = 0; c < nch; ++c) {
      uint64_t acc[CW];
#pragma unroll
      for (int k = 0; k < CW; ++k) acc[k] = 0;
      uint64_t own[CW];
#pragma unroll
      for (int k = 0; k < CW; ++k) own[k] = 0;
      if (EB && act) load_words<CW>(own, xv + c * CW);
      for (int64_t j = b + gl; j < e; j += G) {
        const int32_t u = __ldg(p.col + j);
        ++my_scan;
        if (CHG || dense) {
          if (!test_bit(Cprev, u)) continue;
          any_chg = true;
        }
        or_words<CW>(acc, p.X + (size_t)u * Wp + c * CW);
        ++my_gath;
        if (EB) {
          bool full = true;
#pragma unroll
          for (int k = 0; k < CW; ++k)
            full &= ((acc[k] | own[k] | ~valid_mask(c * CW + k, p.s)) == ~0ULL);
          if (full) break;
        }
      }
#pragma unroll
      for (int off = G >> 1; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < CW; ++k) acc[k] |= __shfl_xor_sync(kFullMask, acc[k], off);
        any_chg |= (__shfl_xor_sync(kFullMask, (int)any_chg, off) != 0);
      }
      if (c == 0 && dense && !any_chg) {
        act = false;
        b = e = 0;
      }
      if (act && gl == 0) {
        if (whole) {
          if (!EB) load_words<CW>(own, xv + c * CW);
          uint64_t nw[CW];
          bool ch = false;
#pragma unroll
          for (int k = 0; k < CW; ++k) {
            nw[k] = own[k] | acc[k];
            ch |= nw[k] != own[k];
          }
          if (ch) store_words<CW>(p.Y + (size_t)v * Wp + c * CW, nw);
          row_changed |= ch;
        } else {
#pragma unroll
          for (int k = 0; k < CW; ++k)
            if (acc[k]) {
              const unsigned long long old = atomicOr(
                  reinterpret_cast<unsigned long long *>(p.Y + (size_t)v * Wp + c * CW + k),
                  (unsigned long long)acc[k]);
              row_changed |= (old | acc[k]) != old;
            }
        }
      }
    }
    if (dense && act && gl == 0) {
      // m_active counts each active row once; pieces of a long row race for it.
      if (whole || !set_bit(Kcur, v)) my_mact += (unsigned long long)indeg;
    }
    bool app = false;
    if (act && gl == 0 && row_changed) app = !set_bit(Ccur, v) || whole;
    const unsigned mask = __ballot_sync(kFullMask, app);
    if (mask) {
      unsigned long long od = 0;
      if (app) od = (unsigned long long)(__ldg(p.out_ptr + v + 1) - __ldg(p.out_ptr + v));
      unsigned long long incl = od;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFullMask, incl, off);
        if (lane >= off) incl += y;
      }
      const unsigned long long total = __shfl_sync(kFullMask, incl, 31);
      unsigned long long basep = 0;
      if (lane == 0)
        basep = atomicAdd(&ctrl->fpack, ((unsigned long long)__popc(mask) << kFsumBits) + total);
      basep = __shfl_sync(kFullMask, basep, 0);
      if (app) {
        const int rank = __popc(mask & ((1u << lane) - 1u));
        const int64_t pos = (int64_t)(basep >> kFsumBits) + rank;
        p.F[pos] = v;
        p.Fpre[pos] = (int64_t)(basep & kFsumMask) + (int64_t)(incl - od);
      }
    }
  }
  RoundStats *r = p.rs + (t - ctrl->row_base);
  block_add4(my_mact, my_scan, my_gath, my_items, &r->m_active, &r->scanned, &r->gathered,
             &r->items);
}

using PullFn = void (*)(Params);
PullFn pull_fn_cw1(int G, bool chg, bool eb);
PullFn pull_fn_cw2(int G, bool chg, bool eb);
PullFn pull_fn_cw4(int G, bool chg, bool eb);
PullFn pull_fn_cw8(int G, bool chg, bool eb);

}  // namespace pg
