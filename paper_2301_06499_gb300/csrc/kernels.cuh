// Device helpers and the pull kernel of one PROPAGATE round.
//
// Round t (Alg. 1's do-while body; Alg. 2's inner loop for one pass) is two
// kernels:
//   pull(t): for every active node v, new = X[v] | OR_{u in in(v)} D[u];
//            if new != X[v]: Y[v] = new, v joins the frontier F_t.
//   post(t): for v in F_t: per-seed popcount of X[v] ^ Y[v] (the new pairs at
//            distance t), then D[v] = X[v] ^ Y[v] and X[v] = Y[v]; build the
//            work list of round t+1.
// X holds the signatures of round t-1 and is only read by the pull, Y only
// written, so a round never sees its own updates (the synchronous diffusion
// of Alg. 1: Sig_next is built from Sig, then copied back).
//
// D[u] (the bits u gained in round t-1, zero when u did not change) replaces
// Sig(u) in Alg. 1's inner OR: Sig_{t-1}(u) = Sig_{t-2}(u) | D[u], and
// Sig_{t-2}(u) was already ORed into Sig_{t-1}(v) in round t-1, so both give
// the same Sig_t(v). It also marks the active nodes for free: v can change in
// round t only if some in-neighbour has D[u] != 0.
#pragma once

#include "common.cuh"

namespace pg {

// Whether round t tests an in-neighbour's changed bit before gathering its
// delta: fixed for the call, or decided per round by the post kernel.
__device__ __forceinline__ bool test_changed_now(const Params &p, const Ctrl *ctrl) {
  return p.test_adapt ? ctrl->test != 0 : p.test_changed != 0;
}

// Bounds of a gathered row u and word w. A build with -DPG_DEBUG_BOUNDS
// checks every gather (0 <= u < n, 0 <= w < Wp): an index out of range is
// recorded in the control block (the call then returns PG_EDEVICE) and the
// gather is skipped instead of faulting. Other builds check nothing.
__device__ __forceinline__ bool gather_ok(const Params &p, int64_t u, int w) {
#ifdef PG_DEBUG_BOUNDS
  if (u >= 0 && u < p.n && w >= 0 && w < p.Wp) return true;
  atomicExch(&p.ctrl->bad_index, 1);
  return false;
#else
  (void)p;
  (void)u;
  (void)w;
  return true;
#endif
}

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

// 32-byte read-only load (one 256-bit access; p is 32-byte aligned). Random
// gathers do not allocate in L1: they are almost never reused from there.
__device__ __forceinline__ void ld_nc_256(uint64_t *a, const uint64_t *p) {
  asm volatile("ld.global.nc.L1::no_allocate.v4.u64 {%0, %1, %2, %3}, [%4];"
               : "=l"(a[0]), "=l"(a[1]), "=l"(a[2]), "=l"(a[3])
               : "l"(p));
}

// CW consecutive signature words (CW in {1, 2, 4, 8}; rows of CW >= 4 words
// are 32-byte aligned, rows of 2 words 16-byte aligned).
template <int CW>
__device__ __forceinline__ void load_words(uint64_t (&a)[CW], const uint64_t *p) {
  if constexpr (CW == 1) {
    a[0] = __ldg(reinterpret_cast<const unsigned long long *>(p));
  } else if constexpr (CW == 2) {
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
    a[0] = v.x;
    a[1] = v.y;
  } else {
#pragma unroll
    for (int k = 0; k < CW; k += 4) ld_nc_256(a + k, p + k);
  }
}

template <int CW>
__device__ __forceinline__ void or_words(uint64_t (&a)[CW], const uint64_t *p) {
  uint64_t t[CW];
  load_words<CW>(t, p);
#pragma unroll
  for (int k = 0; k < CW; ++k) a[k] |= t[k];
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

// Block-wide sums of N counters, then one atomicAdd per nonzero counter.
template <int N>
__device__ __forceinline__ void block_add(const unsigned long long (&v)[N],
                                          unsigned long long *const (&dst)[N]) {
  __shared__ unsigned long long red[N][kBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    unsigned long long x = v[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(kFullMask, x, off);
    if (lane == 0) red[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    unsigned long long s = 0;
    for (int k = 0; k < kBlock / 32; ++k) s += red[threadIdx.x][k];
    if (s && dst[threadIdx.x]) atomicAdd(dst[threadIdx.x], s);
  }
}

// Out-arc pieces of the frontier of round t: one list, or (with push rounds,
// which read round t-1's while appending round t's) two by round parity.
__device__ __forceinline__ unsigned long long *E_of(const Params &p, int t) {
  return ((t & 1) && p.E1) ? p.E1 : p.E;
}

// Seeds of the graph node v belongs to (a batch of disjoint graphs), else s.
__device__ __forceinline__ int seeds_of(const Params &p, int32_t v) {
  return p.node_graph ? __ldg(p.graph_s + __ldg(p.node_graph + v)) : p.s;
}

__device__ __forceinline__ unsigned long long warp_excl_scan64(unsigned long long x, int lane,
                                                               unsigned long long *total) {
  unsigned long long incl = x;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long y = __shfl_up_sync(kFullMask, incl, off);
    if (lane >= off) incl += y;
  }
  *total = __shfl_sync(kFullMask, incl, 31);
  return incl - x;
}

// Appends `cnt` list entries (row << 32 | q), q < cnt, for every lane with
// cnt > 0, into list[] at an offset reserved with one atomicAdd on *counter.
__device__ __forceinline__ void warp_append_pieces(unsigned long long *list,
                                                   unsigned long long *counter, int32_t row,
                                                   unsigned long long cnt, int lane) {
  unsigned long long total;
  const unsigned long long ex = warp_excl_scan64(cnt, lane, &total);
  if (total == 0) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(counter, total);
  base = __shfl_sync(kFullMask, base, 0);
  const unsigned long long at = base + ex;
  const unsigned long long head = cnt < 4 ? cnt : 4;
  for (unsigned long long q = 0; q < head; ++q)
    list[at + q] = ((unsigned long long)(uint32_t)row << 32) | q;
  unsigned big = __ballot_sync(kFullMask, cnt > 4);
  while (big) {  // long lists are written by the whole warp
    const int src = __ffs(big) - 1;
    big &= big - 1;
    const unsigned long long c = __shfl_sync(kFullMask, cnt, src);
    const unsigned long long a = __shfl_sync(kFullMask, at, src);
    const int32_t r = __shfl_sync(kFullMask, row, src);
    for (unsigned long long q = 4 + lane; q < c; q += 32)
      list[a + q] = ((unsigned long long)(uint32_t)r << 32) | q;
  }
}

// Appends the in-arc pieces of `row` (cnt = ceil(indeg / L) of them, first
// arc rb) to the 16-byte work list, one atomicAdd per warp.
__device__ __forceinline__ void warp_append_items(ulonglong2 *list, unsigned long long *counter,
                                                  int32_t row, int64_t rb, int64_t indeg,
                                                  int L, unsigned long long cnt, int lane) {
  unsigned long long total;
  const unsigned long long ex = warp_excl_scan64(cnt, lane, &total);
  if (total == 0) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(counter, total);
  base = __shfl_sync(kFullMask, base, 0);
  const unsigned long long at = base + ex;
  const bool whole = cnt == 1;
  const unsigned long long head = cnt < 4 ? cnt : 4;
  for (unsigned long long q = 0; q < head; ++q) {
    const int64_t first = rb + (int64_t)q * L;
    list[at + q] = make_item(row, first, min((int64_t)L, indeg - (int64_t)q * L), whole);
  }
  unsigned big = __ballot_sync(kFullMask, cnt > 4);
  while (big) {  // long rows are written by the whole warp
    const int src = __ffs(big) - 1;
    big &= big - 1;
    const unsigned long long c = __shfl_sync(kFullMask, cnt, src);
    const unsigned long long a = __shfl_sync(kFullMask, at, src);
    const int32_t r = __shfl_sync(kFullMask, row, src);
    const int64_t b0 = __shfl_sync(kFullMask, rb, src);
    const int64_t d0 = __shfl_sync(kFullMask, indeg, src);
    for (unsigned long long q = 4 + lane; q < c; q += 32)
      list[a + q] = make_item(r, b0 + (int64_t)q * L, min((int64_t)L, d0 - (int64_t)q * L), false);
  }
}

// warp_append_items for N rows per lane at once (cnt[q] pieces of row[q],
// its arcs read from row_ptr again): one scan and one atomicAdd on *counter
// for all of them (the post kernel's claims of one step).
template <int N>
__device__ __forceinline__ void warp_append_items_n(ulonglong2 *list, unsigned long long *counter,
                                                    const int64_t *row_ptr,
                                                    const int32_t (&row)[N], int L,
                                                    const uint32_t (&cnt)[N], int lane) {
  unsigned long long mine = 0;
#pragma unroll
  for (int q = 0; q < N; ++q) mine += cnt[q];
  unsigned long long total;
  const unsigned long long ex = warp_excl_scan64(mine, lane, &total);
  if (total == 0) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(counter, total);
  base = __shfl_sync(kFullMask, base, 0);
  unsigned long long at = base + ex;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    const uint32_t c = cnt[q];
    int64_t rb = 0, indeg = 0;
    if (c) {
      rb = __ldg(row_ptr + row[q]);
      indeg = __ldg(row_ptr + row[q] + 1) - rb;
    }
    const bool whole = c == 1;
    const uint32_t head = c < 4 ? c : 4;
    for (uint32_t k = 0; k < head; ++k)
      list[at + k] = make_item(row[q], rb + (int64_t)k * L, min((int64_t)L, indeg - (int64_t)k * L),
                               whole);
    unsigned big = __ballot_sync(kFullMask, c > 4);
    while (big) {  // long rows are written by the whole warp
      const int src = __ffs(big) - 1;
      big &= big - 1;
      const uint32_t cc = __shfl_sync(kFullMask, c, src);
      const unsigned long long a = __shfl_sync(kFullMask, at, src);
      const int32_t r = __shfl_sync(kFullMask, row[q], src);
      const int64_t b0 = __shfl_sync(kFullMask, rb, src);
      const int64_t d0 = __shfl_sync(kFullMask, indeg, src);
      for (uint32_t k = 4 + lane; k < cc; k += 32)
        list[a + k] = make_item(r, b0 + (int64_t)k * L, min((int64_t)L, d0 - (int64_t)k * L), false);
    }
    at += c;
  }
}

// Frontier append of the rows whose lane has app set: F_t (rows; the packed
// counter also sums their out-degrees) and E (their out-arcs in pieces of LE).
__device__ __forceinline__ void frontier_append(const Params &p, Ctrl *ctrl, int32_t *F, int32_t v,
                                                bool app, int lane) {
  const unsigned mask = __ballot_sync(kFullMask, app);
  if (!mask) return;
  unsigned long long od = 0;
  if (app) od = (unsigned long long)(__ldg(p.out_ptr + v + 1) - __ldg(p.out_ptr + v));
  unsigned long long odt;
  warp_excl_scan64(od, lane, &odt);
  unsigned long long basep = 0;
  if (lane == 0)
    basep = atomicAdd(&ctrl->fpack, ((unsigned long long)__popc(mask) << kFsumBits) + odt);
  basep = __shfl_sync(kFullMask, basep, 0);
  if (p.gfsum) {  // a packed batch: each graph's own frontier out-arcs
    unsigned long long *gf = p.gfsum + (size_t)(ctrl->t & 1) * (size_t)p.nseg;
    const int gid = app ? __ldg(p.node_graph + v) : -1;
    const int g0 = __shfl_sync(kFullMask, gid, __ffs(mask) - 1);
    if (__all_sync(kFullMask, !app || gid == g0)) {
      if (lane == 0 && odt) atomicAdd(gf + g0, odt);
    } else if (app && od) {
      atomicAdd(gf + gid, od);
    }
  }
  if (app) {
    const int rank = __popc(mask & ((1u << lane) - 1u));
    F[(int64_t)(basep >> kFsumBits) + rank] = v;
  }
  const unsigned long long ne = app ? (od + p.LE - 1) / p.LE : 0ULL;
  warp_append_pieces(E_of(p, ctrl->t), &ctrl->nE, v, ne, lane);
}


// Finishes one row piece after its deltas are ORed into acc (words
// [c*CW, c*CW+CW) of the row): a row of one piece compares with X[v] and
// writes Y[v] if it changed; a row cut into pieces ORs acc into Y[v] with
// atomics and reports a change when its OR added a bit.
template <int CW>
__device__ __forceinline__ bool finish_piece(const Params &p, int32_t v, int c, bool whole,
                                             const uint64_t (&own)[CW],
                                             const uint64_t (&acc)[CW]) {
  const size_t Wp = (size_t)p.Wp;
  bool changed = false;
  if (whole) {
    uint64_t nw[CW];
#pragma unroll
    for (int k = 0; k < CW; ++k) {
      nw[k] = own[k] | acc[k];
      changed |= nw[k] != own[k];
    }
    if (changed) store_words<CW>(p.Y + (size_t)v * Wp + c * CW, nw);
  } else {
#pragma unroll
    for (int k = 0; k < CW; ++k)
      if (acc[k]) {
        const unsigned long long old =
            atomicOr(reinterpret_cast<unsigned long long *>(p.Y + (size_t)v * Wp + c * CW + k),
                     (unsigned long long)acc[k]);
        changed |= (old | acc[k]) != old;
      }
  }
  return changed;
}

// PROPAGATE-S with its passes as the words of one signature (p.pass_words):
// word w of a row holds pass w's 64 one-bit planes. A row is active in pass
// w in round t when an in-neighbour gained bits of that pass in round t-1
// (its OR of deltas, acc, is nonzero in word w) and the row still lacks one
// of the pass's bits (word w of X not full): the skip rule of Thm. 1 applied
// to each pass on its own, as if the passes ran one after another. Adds the
// active passes of one row piece to words (and their seeds to seeds); a row
// cut into pieces is counted once per pass, by the piece whose claim bit
// for that pass is set first.
template <int CW>
__device__ __forceinline__ void count_pass_words(const Params &p, int32_t v, int c, bool whole,
                                                 const uint64_t (&own)[CW],
                                                 const uint64_t (&acc)[CW], uint32_t *Kw,
                                                 uint32_t &words, uint32_t &seeds) {
#pragma unroll
  for (int k = 0; k < CW; ++k) {
    if (!acc[k]) continue;
    const int w = c * CW + k;
    if (!whole && set_bit(Kw + (size_t)w * (size_t)p.nbm, v)) continue;
    const uint64_t vm = valid_mask(w, p.s);
    const uint64_t x =
        whole ? own[k]
              : __ldg(reinterpret_cast<const unsigned long long *>(p.X) + (size_t)v * p.Wp + w);
    if ((x | ~vm) != ~0ULL) {
      ++words;
      seeds += (uint32_t)__popcll(vm);
    }
  }
}

// Staged frontier appends. Every warp of a pull or push keeps the rows it appends
// in a buffer of its own in shared memory and moves them to F_t (and their
// out-arc pieces to E_t) kStageRows at a time, with one atomicAdd on each of
// the two round counters per flush. Appending straight to F_t costs those two
// atomics per warp step: same-address atomics are serialised at one L2 slice
// (about 0.65 ns each measured on GB300), which at tens of thousands of warp
// steps per round, or millions on the largest graphs, became a queue that
// every appending warp waited in.
constexpr int kStageRows = 256;

// Writes list entries (row << 32 | q), q < cnt, at `at` for every lane with
// cnt > 0; long runs are written by the whole warp.
__device__ __forceinline__ void write_pieces(unsigned long long *list, unsigned long long at,
                                             int32_t row, unsigned long long cnt, int lane) {
  const unsigned long long head = cnt < 4 ? cnt : 4;
  for (unsigned long long q = 0; q < head; ++q)
    list[at + q] = ((unsigned long long)(uint32_t)row << 32) | q;
  unsigned big = __ballot_sync(kFullMask, cnt > 4);
  while (big) {
    const int src = __ffs(big) - 1;
    big &= big - 1;
    const unsigned long long c = __shfl_sync(kFullMask, cnt, src);
    const unsigned long long a = __shfl_sync(kFullMask, at, src);
    const int32_t r = __shfl_sync(kFullMask, row, src);
    for (unsigned long long q = 4 + lane; q < c; q += 32)
      list[a + q] = ((unsigned long long)(uint32_t)r << 32) | q;
  }
}

// Moves the warp's `cnt` staged rows to F_t and their pieces to E_t (and, in
// a packed batch, their out-degrees to their graphs' frontier sums). Returns
// the new stage count (0). Inlined: a call inside the sweeps' loops would
// spill the registers live across it.
__device__ __forceinline__ int stage_flush(const Params &p, Ctrl *ctrl, int32_t *F,
                                        const int32_t *stage, int cnt, int lane) {
  __syncwarp();
  unsigned long long od_l = 0, ne_l = 0;
  unsigned long long *gf = p.gfsum ? p.gfsum + (size_t)(ctrl->t & 1) * (size_t)p.nseg : nullptr;
  int gcur = -1;  // a packed batch: the lane's current graph and its out-degree sum
  unsigned long long gacc = 0;
  for (int i = lane; i < cnt; i += 32) {
    const int32_t v = stage[i];
    const unsigned long long od =
        (unsigned long long)(__ldg(p.out_ptr + v + 1) - __ldg(p.out_ptr + v));
    od_l += od;
    ne_l += (od + p.LE - 1) / p.LE;
    if (gf && od) {
      const int gq = __ldg(p.node_graph + v);
      if (gq != gcur) {
        if (gacc) atomicAdd(gf + gcur, gacc);
        gcur = gq;
        gacc = 0;
      }
      gacc += od;
    }
  }
  if (gf) {  // one atomic per warp when its lanes ended on one graph
    const unsigned has = __ballot_sync(kFullMask, gacc != 0);
    if (has) {
      const int g0 = __shfl_sync(kFullMask, gcur, __ffs(has) - 1);
      if (__all_sync(kFullMask, gacc == 0 || gcur == g0)) {
        unsigned long long gtot;
        warp_excl_scan64(gacc, lane, &gtot);
        if (lane == 0) atomicAdd(gf + g0, gtot);
      } else if (gacc) {
        atomicAdd(gf + gcur, gacc);
      }
    }
  }
  unsigned long long od_t, ne_t;
  warp_excl_scan64(od_l, lane, &od_t);
  warp_excl_scan64(ne_l, lane, &ne_t);
  unsigned long long basep = 0, basee = 0;
  if (lane == 0) {
    basep = atomicAdd(&ctrl->fpack, ((unsigned long long)cnt << kFsumBits) + od_t);
    if (ne_t) basee = atomicAdd(&ctrl->nE, ne_t);
  }
  basep = __shfl_sync(kFullMask, basep, 0) >> kFsumBits;
  basee = __shfl_sync(kFullMask, basee, 0);
  for (int i = lane; i < cnt; i += 32) F[basep + i] = stage[i];
  if (ne_t) {
    unsigned long long *E = E_of(p, ctrl->t);
    for (int j0 = 0; j0 < cnt; j0 += 32) {
      const int i = j0 + lane;
      int32_t v = 0;
      unsigned long long ne = 0;
      if (i < cnt) {
        v = stage[i];
        const unsigned long long od =
            (unsigned long long)(__ldg(p.out_ptr + v + 1) - __ldg(p.out_ptr + v));
        ne = (od + p.LE - 1) / p.LE;
      }
      unsigned long long tot;
      const unsigned long long ex = warp_excl_scan64(ne, lane, &tot);
      write_pieces(E, basee + ex, v, ne, lane);
      basee += tot;
    }
  }
  __syncwarp();
  return 0;
}

// Stages the rows whose lane has app set, without a flush (the caller made
// room for 32 more); returns the new stage count (warp-uniform).
__device__ __forceinline__ int stage_put(int32_t *stage, int cnt, int32_t v, bool app, int lane) {
  const unsigned mask = __ballot_sync(kFullMask, app);
  if (app) stage[cnt + __popc(mask & ((1u << lane) - 1u))] = v;
  return cnt + __popc(mask);
}

// Stages the rows whose lane has app set (flushing first when the buffer
// could overflow); returns the new stage count (warp-uniform).
__device__ __forceinline__ int stage_append(const Params &p, Ctrl *ctrl, int32_t *F,
                                            int32_t *stage, int cnt, int32_t v, bool app,
                                            int lane) {
  const unsigned mask = __ballot_sync(kFullMask, app);
  if (!mask) return cnt;
  if (cnt > kStageRows - 32) cnt = stage_flush(p, ctrl, F, stage, cnt, lane);
  if (app) stage[cnt + __popc(mask & ((1u << lane) - 1u))] = v;
  return cnt + __popc(mask);
}

// Tuning knobs (compile-time): minimum resident blocks per SM for the pull
// kernel (caps registers; the kernels are latency-bound, so occupancy pays:
// 4 blocks of 256 threads = 64 registers, measured 10% faster than 3 for
// 4-word rows on R-MAT 22, and 2.6% faster for 8-word rows on the scale-26
// R-MAT although those spill ~150 bytes at 64 registers) and arcs per lane
// per step of the dense sweep.
#ifndef PG_PULL_MIN_BLOCKS
#define PG_PULL_MIN_BLOCKS 4
#endif
#ifndef PG_PULL_MIN_BLOCKS_WIDE
#define PG_PULL_MIN_BLOCKS_WIDE 4
#endif
#ifndef PG_DENSE_UNROLL_NARROW
#define PG_DENSE_UNROLL_NARROW 4
#endif
#ifndef PG_DENSE_UNROLL_WIDE
#define PG_DENSE_UNROLL_WIDE 4
#endif

// A packed batch: adds a warp's m_active of round t (x on each lane whose
// row v is active) to the graph of those rows with one atomic. The rows of a
// sliced-ELL chunk are one graph's; every lane of the warp calls it.
__device__ __forceinline__ void gm_add_chunk(const Params &p, const Ctrl *ctrl, int32_t v,
                                             uint32_t x) {
  const unsigned am = __ballot_sync(kFullMask, x != 0u);
  if (!am) return;
  const int32_t va = __shfl_sync(kFullMask, v, __ffs(am) - 1);
  unsigned long long sum = x;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(kFullMask, sum, off);
  if ((threadIdx.x & 31) == 0)
    atomicAdd(p.gmact + (size_t)(ctrl->t - ctrl->row_base) * (size_t)p.nseg +
                  __ldg(p.node_graph + va),
              sum);
}

// Dense round over the sliced-ELL copy: a warp per chunk of 32 pieces, lane
// l owns piece l; step k reads arc k of all 32 pieces in one coalesced load,
// and the U deltas of a lane's U steps are gathered together. The sweep is
// software-pipelined so that column loads never wait behind gathers:
//  - within a chunk (rows of up to 4 words), the next U column indices are
//    loaded before the current U deltas are gathered;
//  - for narrow rows (1-2 words), the next chunk's descriptor is loaded when
//    a chunk starts and its first U column indices when the chunk ends
//    (before the frontier append), ahead of the saturation test: there the
//    latency matters more than the reads wasted on saturated rows.
template <int CW, bool PW>
__device__ __forceinline__ void pull_dense(const Params &p, Ctrl *ctrl, const uint64_t *Dprev,
                                           const uint32_t *Cprev, int32_t *F, uint32_t *Ccur,
                                           uint32_t *Kcur, uint32_t *Kwcur, int lane,
                                           int64_t warp, int64_t nwarps,
                                           uint32_t &my_mact,
                                           unsigned long long &my_work,
                                           uint32_t &my_scan,
                                           uint32_t &my_gath,
                                           uint32_t &my_items,
                                           uint32_t &my_rows, int32_t *stage, int &scnt) {
  constexpr int U = CW <= 2 ? PG_DENSE_UNROLL_NARROW : PG_DENSE_UNROLL_WIDE;
  const bool tc = test_changed_now(p, ctrl);
  constexpr bool kPrefetch = CW <= 2;
  constexpr bool kPipe = CW <= 4;  // at 8 words the registers are not there
  const size_t Wp = (size_t)p.Wp;
  const int nch = p.Wp / CW;
  // the chunks to sweep: all of them, or (a packed batch with a dense list)
  // those of the graphs in a full sweep; iteration i handles chunk_at(i)
  const int nd = p.dlist ? ctrl->ndense : 0;
  const int64_t nchunks = p.dlist ? p.dpref[nd] : p.sell_chunks;
  auto chunk_at = [&](int64_t i) -> int64_t {
    if (!p.dlist) return i;
    int lo = 0, hi = nd - 1;  // the last k with dpref[k] <= i
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.dpref[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return __ldg(p.seg_chunk0 + p.dlist[lo]) + (i - p.dpref[lo]);
  };
  int64_t ci = warp;
  ulonglong2 it_next = make_ulonglong2(0ULL, 0ULL);
  int clen_next = 0;
  int64_t off_next = 0;
  int32_t u0[U];  // first column batch of the chunk about to start
  auto first_batch = [&](int len_of, int64_t off) {
#pragma unroll
    for (int q = 0; q < U; ++q)
      u0[q] = q < len_of ? __ldg(p.sell_col + off + lane + 32LL * q) : -1;
  };
  if (kPrefetch && ci < nchunks) {
    const int64_t c = chunk_at(ci);
    it_next = p.sell_items[c * 32 + lane];
    clen_next = __ldg(p.sell_len + c);
    off_next = __ldg(p.sell_off + c);
    first_batch((int)(it_next.y & 0x7FFFFFFFULL), off_next);
  }
  for (; ci < nchunks; ci += nwarps) {
    const int64_t c = chunk_at(ci);
    if (!kPrefetch) {
      it_next = p.sell_items[c * 32 + lane];
      clen_next = __ldg(p.sell_len + c);
      off_next = __ldg(p.sell_off + c);
    }
    const ulonglong2 it = it_next;
    const int clen = clen_next;
    const int32_t *cc = p.sell_col + off_next + lane;
    const bool has_next = kPrefetch && ci + nwarps < nchunks;
    const int64_t cn = has_next ? chunk_at(ci + nwarps) : 0;
    if (has_next) {
      it_next = p.sell_items[cn * 32 + lane];
      clen_next = __ldg(p.sell_len + cn);
      off_next = __ldg(p.sell_off + cn);
    }
    // a packed batch: only the graphs whose own frontier chose a full sweep
    if (p.gfsum && !p.dlist) {
      const int gs = __ldg(p.sell_seg + c);
      if (p.gfsum[(size_t)((ctrl->t - 1) & 1) * (size_t)p.nseg + gs] <= __ldg(p.gthr + gs)) {
        if (has_next) first_batch((int)(it_next.y & 0x7FFFFFFFULL), off_next);
        continue;
      }
    }
    const int32_t v = (int32_t)(it.y >> 32);
    const bool whole = (it.y & 0x80000000ULL) != 0ULL;
    const int len = (int)(it.y & 0x7FFFFFFFULL);
    bool act = len > 0 && !test_bit(p.Sat, v);
    if (!kPrefetch) {
#pragma unroll
      for (int q = 0; q < U; ++q) u0[q] = act && q < len ? __ldg(cc + 32LL * q) : -1;
    }
    bool row_changed = false, any_delta = false;
    uint32_t pw_words = 0, pw_seeds = 0;
    for (int ch = 0; ch < nch; ++ch) {
      uint64_t own[CW], acc[CW];
#pragma unroll
      for (int k = 0; k < CW; ++k) own[k] = acc[k] = 0;
      if (act && whole) load_words<CW>(own, p.X + (size_t)v * Wp + ch * CW);
      int32_t u[U];
#pragma unroll
      for (int q = 0; q < U; ++q)
        u[q] = !act ? -1 : ch == 0 ? u0[q] : (q < len ? __ldg(cc + 32LL * q) : -1);
      for (int k0 = 0; k0 < clen; k0 += U) {
        const bool more = kPipe && k0 + U < clen;  // warp-uniform
        int32_t un[U];
        if (!kPipe && k0 > 0) {
#pragma unroll
          for (int q = 0; q < U; ++q)
            u[q] = (act && k0 + q < len) ? __ldg(cc + 32LL * (k0 + q)) : -1;
        }
        if (more) {
#pragma unroll
          for (int q = 0; q < U; ++q)
            un[q] = (act && k0 + U + q < len) ? __ldg(cc + 32LL * (k0 + U + q)) : -1;
        }
        if (tc) {
#pragma unroll
          for (int q = 0; q < U; ++q)
            if (u[q] >= 0 && !test_bit(Cprev, u[q])) u[q] = -1;
        }
#pragma unroll
        for (int q = 0; q < U; ++q)
          if (u[q] >= 0) {
            if (gather_ok(p, u[q], ch * CW + CW - 1))
              or_words<CW>(acc, Dprev + (size_t)u[q] * Wp + ch * CW);
            if (ch == 0) ++my_gath;
          }
        if (more) {
#pragma unroll
          for (int q = 0; q < U; ++q) u[q] = un[q];
        }
      }
#pragma unroll
      for (int k = 0; k < CW; ++k) any_delta |= acc[k] != 0ULL;
      if constexpr (PW)
        if (act) count_pass_words<CW>(p, v, ch, whole, own, acc, Kwcur, pw_words, pw_seeds);
      if (act) row_changed |= finish_piece<CW>(p, v, ch, whole, own, acc);
    }
    if (has_next) first_batch((int)(it_next.y & 0x7FFFFFFFULL), off_next);
    if (act) {
      ++my_items;
      my_scan += (uint32_t)len;
    }
    act = act && any_delta;  // no changed in-neighbour: not active in round t
    uint32_t gdeg = 0;       // this lane's m_active of the chunk
    if (PW && act) {
      if (pw_words) {
        const uint32_t deg =
            whole ? (uint32_t)len : (uint32_t)(__ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v));
        my_mact += deg * pw_words;
        my_work += (unsigned long long)deg * (unsigned long long)pw_seeds;
        my_rows += pw_words;
      }
    } else if (act) {
      uint32_t deg = 0;
      if (whole) {
        deg = (uint32_t)len;
        ++my_rows;
      } else if (!set_bit(Kcur, v)) {
        deg = (uint32_t)(__ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v));
        ++my_rows;
      }
      my_mact += deg;
      my_work += (unsigned long long)deg * (unsigned long long)seeds_of(p, v);
      gdeg = deg;
    }
    if (p.gmact) gm_add_chunk(p, ctrl, v, gdeg);  // a packed batch: per graph
    bool app = false;
    if (act && row_changed) {
      if (whole) {
        atomicOr(Ccur + (v >> 5), 1u << (v & 31));
        app = true;
      } else {
        app = !set_bit(Ccur, v);
      }
    }
    scnt = stage_append(p, ctrl, F, stage, scnt, v, app, lane);
  }
}

// Arcs per lane per piece of the sparse rounds: all of a lane's column loads
// and delta gathers of one piece are issued together.
template <int CW>
struct PullUnroll {
  static constexpr int value = CW <= 2 ? 8 : (CW == 4 ? 4 : 2);
};

// Buffers of round t, chosen by the round's parity, and the next round's
// claim bitmaps cleared by the pull (shared by every pull kernel).
struct RoundBufs {
  const uint64_t *Dprev;
  const uint32_t *Cprev;
  int32_t *F;
  uint32_t *Ccur, *Kcur, *Kwcur;
};

__device__ __forceinline__ RoundBufs pull_begin(const Params &p, int t, int64_t gtid,
                                                int64_t nthreads) {
  RoundBufs r;
  r.Dprev = (t & 1) ? p.D0 : p.D1;
  r.Cprev = (t & 1) ? p.C0 : p.C1;
  r.F = (t & 1) ? p.F1 : p.F0;
  r.Ccur = (t & 1) ? p.C1 : p.C0;
  r.Kcur = (t & 1) ? p.K1 : p.K0;
  r.Kwcur = (t & 1) ? p.Kw1 : p.Kw0;
  uint32_t *Knext = (t & 1) ? p.K0 : p.K1;
  for (int64_t i = gtid; i < p.nbm; i += nthreads) Knext[i] = 0u;
  if (p.pass_words) {  // the per-pass claim bits of round t+1
    uint32_t *Kwnext = (t & 1) ? p.Kw0 : p.Kw1;
    for (int64_t i = gtid; i < p.nbm * p.Wp; i += nthreads) Kwnext[i] = 0u;
  }
  return r;
}

// Sparse (and mixed) rounds: a group of G lanes per piece of the work list
// the previous post kernel built, UNR arcs per lane issued together.
template <int CW, int G, bool PW>
__device__ __forceinline__ void pull_sparse(const Params &p, Ctrl *ctrl, const RoundBufs &rb,
                                            int lane, int64_t warp, int64_t nwarps,
                                            uint32_t &my_mact, unsigned long long &my_work,
                                            uint32_t &my_scan, uint32_t &my_gath,
                                            uint32_t &my_items, uint32_t &my_rows,
                                            int32_t *stage, int &scnt) {
  constexpr int UNR = PullUnroll<CW>::value;
  constexpr int GPW = 32 / G;
  const bool tc = test_changed_now(p, ctrl);
  const uint64_t *Dprev = rb.Dprev;
  const uint32_t *Cprev = rb.Cprev;
  int32_t *F = rb.F;
  uint32_t *Ccur = rb.Ccur;
  uint32_t *Kwcur = rb.Kwcur;
  const int gl = lane & (G - 1);
  const int gw = lane / G;
  const int64_t nitems = (int64_t)ctrl->nA;
  const int nch = p.Wp / CW;
  const size_t Wp = (size_t)p.Wp;
  constexpr bool kPrefetch = CW <= 2;  // next item loaded during this one
  ulonglong2 it_next = make_ulonglong2(0ULL, 0ULL);
  if (kPrefetch && warp * GPW + gw < nitems) it_next = p.A[warp * GPW + gw];
  for (int64_t base = warp * GPW; base < nitems; base += nwarps * GPW) {
    const int64_t item = base + gw;
    bool act = false, whole = true;
    int32_t v = 0;
    int64_t b = 0;
    int len = 0;
    if (item < nitems) {
      const ulonglong2 it = kPrefetch ? it_next : p.A[item];
      if (kPrefetch && item + nwarps * GPW < nitems) it_next = p.A[item + nwarps * GPW];
      b = (int64_t)it.x;
      v = (int32_t)(it.y >> 32);
      whole = (it.y & 0x80000000ULL) != 0ULL;
      len = (int)(it.y & 0x7FFFFFFFULL);
      act = true;
    }
    if (gl == 0 && act) {
      ++my_items;
      my_scan += (uint32_t)len;
    }
    int32_t u[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) {
      const int j = gl + q * G;
      u[q] = (act && j < len) ? __ldg(p.col + b + j) : -1;
    }
    if (tc) {
#pragma unroll
      for (int q = 0; q < UNR; ++q)
        if (u[q] >= 0 && !test_bit(Cprev, u[q])) u[q] = -1;
    }
    bool row_changed = false;
    uint32_t pw_words = 0, pw_seeds = 0;
    for (int c = 0; c < nch; ++c) {
      uint64_t own[CW], acc[CW];
#pragma unroll
      for (int k = 0; k < CW; ++k) own[k] = acc[k] = 0;
      if (act && gl == 0 && whole) load_words<CW>(own, p.X + (size_t)v * Wp + c * CW);
#pragma unroll
      for (int q = 0; q < UNR; ++q)
        if (u[q] >= 0) {
          if (gather_ok(p, u[q], c * CW + CW - 1))
            or_words<CW>(acc, Dprev + (size_t)u[q] * Wp + c * CW);
          if (c == 0) ++my_gath;
        }
#pragma unroll
      for (int off = G >> 1; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < CW; ++k) acc[k] |= __shfl_xor_sync(kFullMask, acc[k], off);
      }
      if constexpr (PW)
        if (act && gl == 0) count_pass_words<CW>(p, v, c, whole, own, acc, Kwcur, pw_words, pw_seeds);
      if (act && gl == 0) row_changed |= finish_piece<CW>(p, v, c, whole, own, acc);
    }
    if (PW && pw_words) {  // passes as words: m_active here, not at the claim
      const uint32_t deg =
          whole ? (uint32_t)len : (uint32_t)(__ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v));
      my_mact += deg * pw_words;
      my_work += (unsigned long long)deg * (unsigned long long)pw_seeds;
      my_rows += pw_words;
    }
    bool app = false;
    if (act && gl == 0 && row_changed) {
      if (whole) {
        atomicOr(Ccur + (v >> 5), 1u << (v & 31));
        app = true;
      } else {
        app = !set_bit(Ccur, v);
      }
    }
    scnt = stage_append(p, ctrl, F, stage, scnt, v, app, lane);
  }
}

// Push round t (sparse rounds with p.push): every changed row u of round t-1
// ORs its delta D_{t-1}[u] into Y[v] of each unsaturated out-neighbour v
// with 64-bit atomics, over the out-arc pieces of F_{t-1} (E of round t-1).
// The result equals the pull's: Sig_t(v) = Sig_{t-1}(v) | OR of the deltas
// of v's changed in-neighbours. The pusher whose OR added a bit to v first
// puts v in the frontier. Activity for m_active is the same claim as the
// post kernel's for a pull round: the first pusher to reach an unsaturated v
// claims it and counts its in-degree.
//
// PW (PROPAGATE-S passes as words): a row is active in pass k when a pusher's
// delta has bits in word k and word k of the row's X is not full; the first
// pusher to set the row's claim bit of pass k (Kw) counts it, as the pull's
// count_pass_words does for a row cut into pieces.
template <int CW, bool PW = false>
__device__ __forceinline__ void pull_push(const Params &p, Ctrl *ctrl, const RoundBufs &rb, int t,
                                          int lane, int64_t warp, int64_t nwarps,
                                          uint32_t &my_mact, unsigned long long &my_work,
                                          uint32_t &my_scan, uint32_t &my_gath,
                                          uint32_t &my_items, uint32_t &my_rows,
                                          int32_t *stage, int &scnt) {
  constexpr int UNR = 4;
  const unsigned long long *Ep = E_of(p, t - 1);
  const int64_t nEp = (int64_t)ctrl->nE_prev;
  const size_t Wp = (size_t)p.Wp;
  for (int64_t base = warp * 32; base < nEp; base += nwarps * 32) {
    const int64_t i = base + lane;
    int64_t ob = 0, oe = 0;
    uint64_t d[CW];
#pragma unroll
    for (int k = 0; k < CW; ++k) d[k] = 0ULL;
    bool live = i < nEp;
    unsigned long long it = 0;
    if (live) {
      it = Ep[i];
      if (p.gfsum) {  // a packed batch: graphs swept whole this round take no push
        const int gu = __ldg(p.node_graph + (int32_t)(it >> 32));
        live = p.gfsum[(size_t)((t - 1) & 1) * (size_t)p.nseg + gu] <= __ldg(p.gthr + gu);
      }
    }
    if (live) {
      const int32_t u = (int32_t)(it >> 32);
      const int64_t k = (int64_t)(it & 0xFFFFFFFFULL);
      const int64_t o1 = __ldg(p.out_ptr + u + 1);
      ob = __ldg(p.out_ptr + u) + k * p.LE;
      oe = min(o1, ob + (int64_t)p.LE);
      if (gather_ok(p, u, CW - 1)) load_words<CW>(d, rb.Dprev + (size_t)u * Wp);
      ++my_items;
      ++my_gath;
      my_scan += (uint32_t)(oe - ob);
    }
    for (int h = 0; h < p.LE; h += UNR) {
      int32_t v[UNR];
#pragma unroll
      for (int q = 0; q < UNR; ++q) {
        const int64_t j = ob + h + q;
        v[q] = j < oe ? __ldg(p.out_col + j) : -1;
        if (v[q] >= 0 && (!gather_ok(p, v[q], CW - 1) || test_bit(p.Sat, v[q]))) v[q] = -1;
      }
      bool app[UNR];
#pragma unroll
      for (int q = 0; q < UNR; ++q) {
        app[q] = false;
        if (v[q] < 0) continue;
        if constexpr (PW) {
          uint32_t indeg = 0;
#pragma unroll
          for (int k = 0; k < CW; ++k) {
            if (!d[k]) continue;
            uint32_t *Kw = rb.Kwcur + (size_t)k * (size_t)p.nbm;
            if (test_bit_live(Kw, v[q]) || set_bit(Kw, v[q])) continue;
            const uint64_t vm = valid_mask(k, p.s);
            const uint64_t x =
                __ldg(reinterpret_cast<const unsigned long long *>(p.X) + (size_t)v[q] * Wp + k);
            if ((x | ~vm) != ~0ULL) {
              if (!indeg)
                indeg = (uint32_t)(__ldg(p.row_ptr + v[q] + 1) - __ldg(p.row_ptr + v[q]));
              my_mact += indeg;
              my_work += (unsigned long long)indeg * (unsigned long long)__popcll(vm);
              ++my_rows;
            }
          }
        } else if (!test_bit_live(rb.Kcur, v[q]) && !set_bit(rb.Kcur, v[q])) {
          const uint32_t indeg = (uint32_t)(__ldg(p.row_ptr + v[q] + 1) - __ldg(p.row_ptr + v[q]));
          my_mact += indeg;
          my_work += (unsigned long long)indeg * (unsigned long long)seeds_of(p, v[q]);
          ++my_rows;
          if (p.gmact)  // a packed batch: the claimed row's own graph
            atomicAdd(p.gmact + (size_t)(t - ctrl->row_base) * (size_t)p.nseg +
                          __ldg(p.node_graph + v[q]),
                      (unsigned long long)indeg);
        }
        bool changed = false;
#pragma unroll
        for (int k = 0; k < CW; ++k)
          if (d[k]) {
            const unsigned long long old = atomicOr(
                reinterpret_cast<unsigned long long *>(p.Y + (size_t)v[q] * Wp + k),
                (unsigned long long)d[k]);
            changed |= (old | d[k]) != old;
          }
        app[q] = changed && !set_bit(rb.Ccur, v[q]);
      }
      if (scnt > kStageRows - 32 * UNR) scnt = stage_flush(p, ctrl, rb.F, stage, scnt, lane);
#pragma unroll
      for (int q = 0; q < UNR; ++q) scnt = stage_put(stage, scnt, v[q], app[q], lane);
    }
  }
}

// Per-block sums of a pull launch's work counters into round t's slot.
__device__ __forceinline__ void pull_end(const Params &p, Ctrl *ctrl, int t, uint32_t my_mact,
                                         unsigned long long my_work, uint32_t my_scan,
                                         uint32_t my_gath, uint32_t my_items, uint32_t my_rows) {
  RoundStats *r = p.rs + (t - ctrl->row_base);
  const unsigned long long vals[6] = {my_mact, my_work, my_scan, my_gath, my_items, my_rows};
  unsigned long long *const dsts[6] = {&r->m_active, &r->work,  &r->scanned,
                                       &r->gathered, &r->items, &r->rows};
  block_add<6>(vals, dsts);
}

// Pull kernel of round t.
//
// Dense rounds (most nodes have a changed in-neighbour) sweep the sliced-ELL
// copy of every unsaturated row (pull_dense). Sparse rounds walk the pieces
// of the rows the previous post kernel claimed (rows with a changed
// in-neighbour and a zero bit); a group of G lanes takes one piece of at most
// L = G * UNR in-arcs and each lane handles UNR of them in one shot: UNR
// column loads, then UNR delta gathers, all independent. The group ORs its
// lanes with log2(G) shuffles and its leader finishes the piece.
//
// Activity (for m_active) follows the skip rule of the proof of Thm. 1: a
// node is revisited in round t when it still has a zero bit (not saturated)
// and some in-neighbour changed in round t-1 (a nonzero delta). Sparse rounds
// count it when the row is claimed (PW: here, per pass).
//
// With p.test_changed, an in-neighbour's changed bit (C_{t-1}, n bits, kept in
// L2) is tested before its delta is gathered, so unchanged neighbours cost no
// signature-sized read: worth it when the deltas are far larger than L2.
//
// PW: PROPAGATE-S passes as the words of one signature; m_active is counted
// per pass here (count_pass_words), in dense and sparse rounds alike.
template <int CW, int G, bool PW>
__global__ void __launch_bounds__(kBlock, CW <= 4 ? PG_PULL_MIN_BLOCKS : PG_PULL_MIN_BLOCKS_WIDE)
    k_pull(Params p) {
  Ctrl *ctrl = p.ctrl;
  if (*(volatile int32_t *)&ctrl->done) return;
  const int t = ctrl->t;
  const int mode = ctrl->mode;
  const int64_t gtid = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * kBlock;
  const RoundBufs rb = pull_begin(p, t, gtid, nthreads);
  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid >> 5;
  const int64_t nwarps = nthreads >> 5;
  // per-thread work counters: a thread sees at most tens of thousands of
  // arcs per launch, so 32 bits hold all but the seed-weighted work
  uint32_t my_mact = 0, my_scan = 0, my_gath = 0, my_items = 0, my_rows = 0;
  unsigned long long my_work = 0;
  __shared__ int32_t s_stage[kBlock / 32][kStageRows];  // staged frontier rows per warp
  int32_t *stage = s_stage[threadIdx.x >> 5];
  int scnt = 0;
  // dense rounds sweep every row; mixed rounds (a packed batch) sweep the rows
  // of the graphs that chose a full sweep and take the others' work list
  if ((mode == kModeDense && !p.dense_tma) || mode == kModeMixed)  // dense_tma: k_pull_tma
    pull_dense<CW, PW>(p, ctrl, rb.Dprev, rb.Cprev, rb.F, rb.Ccur, rb.Kcur, rb.Kwcur, lane, warp,
                       nwarps, my_mact, my_work, my_scan, my_gath, my_items, my_rows, stage,
                       scnt);
  if (mode == kModeSparse || mode == kModeMixed)
    pull_sparse<CW, G, PW>(p, ctrl, rb, lane, warp, nwarps, my_mact, my_work, my_scan, my_gath,
                           my_items, my_rows, stage, scnt);
  // push rounds for rows of up to 4 words of one graph (8-word rows and
  // packed batches push in k_push, launched after this kernel: the 8-word
  // kernel keeps its registers for the dense sweep)
  if constexpr (!PW && CW <= 4)
    if (mode == kModePush && !p.push_kernel)
      pull_push<CW>(p, ctrl, rb, t, lane, warp, nwarps, my_mact, my_work, my_scan, my_gath,
                    my_items, my_rows, stage, scnt);
  if (scnt) stage_flush(p, ctrl, rb.F, stage, scnt, lane);
  pull_end(p, ctrl, t, my_mact, my_work, my_scan, my_gath, my_items, my_rows);
}

using PullFn = void (*)(Params);
// Push rounds as a kernel of their own (k_push<CW, PW>, push.cu): 8-word
// rows, PROPAGATE-S passes as words and packed batches; it returns at once in
// rounds that are not pushed.
PullFn push_fn(int CW, bool pw);
// Dense rounds with TMA-gathered deltas (pull_tma.cu), for rows of CW = 4 or
// 8 words: the kernel, its dynamic shared memory, its launch, and the tensor
// map (a CUtensorMap, 128 bytes) over a delta buffer of `rows` rows.
const void *pull_tma_fn(int CW, bool pw);
size_t pull_tma_smem(int CW);
void launch_pull_tma(int CW, bool pw, const Params &p, const void *tm0, const void *tm1, int grid,
                     cudaStream_t st);
pg_status encode_delta_map(void *out, const uint64_t *D, int64_t rows, int Wp, int CW);
PullFn pull_fn_cw1(int G, bool pw);
PullFn pull_fn_cw2(int G, bool pw);
PullFn pull_fn_cw4(int G, bool pw);
PullFn pull_fn_cw8(int G, bool pw);
// Wide rows (more than 8 words): a warp per row piece, for Wp words per row.
PullFn pull_fn_wide(int Wp, bool pw = false);

}  // namespace pg
