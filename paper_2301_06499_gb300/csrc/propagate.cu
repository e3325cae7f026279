// PROPAGATE-P and PROPAGATE-S drivers: seed initialisation (Alg. 1's start,
// seed i's bit set on its own node; Alg. 2's per-seed plane set-up), the post
// kernel of every round (collision count, buffer sync, next work list,
// fixpoint test) and the host round loop.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "host.cuh"
#include "kernels.cuh"

namespace pg {

constexpr int32_t kStatusWindow = 100;  // device asks the host to move the counts window
constexpr int kSmemCountMax = 12288;    // per-seed counters kept in shared memory up to this s
constexpr int kWidePostWords = 16;      // rows of this many words take k_post's tiled part A
constexpr int kExpandArcs = 8;          // out-arcs per expansion piece (LE)
constexpr int kWidePiece = 256;         // in-arcs per piece of the wide-row pull

// ------------------------------------------------------------- k_zero
// Zeroes both signature buffers, the bitmaps, the pass's counts window and
// round statistics, and resets the control block.
__global__ void __launch_bounds__(kBlock) k_zero(Params p, int64_t count_words, int64_t rs_words) {
  const int64_t gtid = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * kBlock;
  const int64_t words = p.n * (int64_t)p.Wp;
  const int64_t pairs = words >> 1;
  ulonglong2 *x2 = reinterpret_cast<ulonglong2 *>(p.X);
  ulonglong2 *y2 = reinterpret_cast<ulonglong2 *>(p.Y);
  const ulonglong2 z = make_ulonglong2(0ULL, 0ULL);
  ulonglong2 *d0 = reinterpret_cast<ulonglong2 *>(p.D0);
  ulonglong2 *d1 = reinterpret_cast<ulonglong2 *>(p.D1);
  for (int64_t i = gtid; i < pairs; i += nth) {
    x2[i] = z;
    y2[i] = z;
    d0[i] = z;
    d1[i] = z;
  }
  if ((words & 1) && gtid == 0) {
    p.X[words - 1] = 0ULL;
    p.Y[words - 1] = 0ULL;
    p.D0[words - 1] = 0ULL;
    p.D1[words - 1] = 0ULL;
  }
  if (gtid < p.Wp) {  // the all-zero row past the last node
    p.D0[words + gtid] = 0ULL;
    p.D1[words + gtid] = 0ULL;
  }
  for (int64_t i = gtid; i < p.nbm; i += nth) {
    p.C0[i] = 0u;
    p.C1[i] = 0u;
    p.K0[i] = 0u;
    p.K1[i] = 0u;
    p.Sat[i] = 0u;
  }
  if (p.rowbits)
    for (int64_t i = gtid; i < p.n; i += nth) p.rowbits[i] = 0u;
  if (p.pass_words)
    for (int64_t i = gtid; i < p.nbm * p.Wp; i += nth) {
      p.Kw0[i] = 0u;
      p.Kw1[i] = 0u;
    }
  for (int64_t i = gtid; i < count_words; i += nth) p.counts[i] = 0u;
  unsigned long long *rsw = reinterpret_cast<unsigned long long *>(p.rs);
  for (int64_t i = gtid; i < rs_words; i += nth) rsw[i] = 0ULL;
  if (p.gmact)
    for (int64_t i = gtid; i < (int64_t)(p.row_cap + 2) * p.nseg; i += nth) p.gmact[i] = 0ULL;
  if (gtid == 0) {
    Ctrl *c = p.ctrl;
    c->t = 0;
    c->done = 0;
    c->status = 0;
    c->mode = kModeSparse;
    c->fpack = 0ULL;
    c->nA = 0ULL;
    c->nA_next = 0ULL;
    c->nE = 0ULL;
    c->blocks_done = 0u;
    c->last_round = 0;
    c->dense_rounds = 0;
    c->row_base = 0;
    c->iters = 0;
    c->ndense = 0;
    c->test = 1;
    c->bad_index = 0;
    c->nF_prev = 0ULL;
    c->nE_prev = 0ULL;
  }
}

// ------------------------------------------------------------- k_seed
// One block. Round 0 of the pass: seed i gets bit i (Sig(x_i)[i] = 1) as a
// change of round 0 (X = 0, Y = the bit), so the post kernel of round 0
// counts the pairs (x_i, x_i), records the seeds' deltas and expands them
// like any other frontier. A node may carry several seeds' bits (requests
// merged on one graph); it enters the frontier once.
__global__ void __launch_bounds__(1024) k_seed(Params p, const int32_t *seeds,
                                               const int32_t *seed_bit, int sp) {
  __shared__ unsigned long long tot;
  __shared__ unsigned int nf;
  if (threadIdx.x == 0) {
    tot = 0ULL;
    nf = 0u;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // whole warps iterate so that the warp-level appends see every lane
  for (int base = (threadIdx.x & ~31); base < sp; base += blockDim.x) {
    const int i = base + lane;
    unsigned long long od = 0;
    int32_t x = 0;
    bool first = false;
    if (i < sp) {
      x = seeds[i];
      if (p.perm) {  // the caller's id of a relabelled graph (of its copy k)
        const int64_t k = (int64_t)x / p.perm_n;
        x = (int32_t)(k * p.perm_n + __ldg(p.perm + ((int64_t)x - k * p.perm_n)));
      }
      const int bit = seed_bit ? seed_bit[i] : i;  // a batch: the seed's index in its graph
      atomicOr(reinterpret_cast<unsigned long long *>(p.Y + (size_t)x * p.Wp + (bit >> 6)),
               1ULL << (bit & 63));
      first = !set_bit(p.C0, x);
      if (first) {
        p.F0[atomicAdd(&nf, 1u)] = x;
        od = (unsigned long long)(p.out_ptr[x + 1] - p.out_ptr[x]);
        atomicAdd(&tot, od);
        if (p.gfsum && od) atomicAdd(p.gfsum + p.node_graph[x], od);  // round 0's parity
      }
    }
    const unsigned long long ne = first ? (od + p.LE - 1) / p.LE : 0ULL;
    warp_append_pieces(E_of(p, 0), &p.ctrl->nE, x, ne, lane);
  }
  __syncthreads();
  if (threadIdx.x == 0) p.ctrl->fpack = ((unsigned long long)nf << kFsumBits) | tot;
}

__device__ __forceinline__ bool row_full(const uint64_t *row, int Wp, int s) {
  bool full = true;
  for (int w = 0; w < Wp; ++w)
    full &= ((__ldg(reinterpret_cast<const unsigned long long *>(row) + w) | ~valid_mask(w, s)) ==
             ~0ULL);
  return full;
}

// 32 x 32 bit transpose across a warp: on entry lane r holds row r (bit c =
// M[r][c]); on exit lane c holds column c (bit r = M[r][c]). Five stages,
// each swapping the off-diagonal blocks of one bit level.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int j = 16 >> st;
    const uint32_t m = masks[st];
    const uint32_t y = __shfl_xor_sync(kFullMask, x, j);
    x = (lane & j) ? ((x & ~m) | ((y & ~m) >> j)) : ((x & m) | ((y & m) << j));
  }
  return x;
}

// ------------------------------------------------------------- k_post
// Round t, after the pull:
//  A. for v in F_t (a warp per 32 rows): d = X[v] ^ Y[v]; per seed i add bit
//     i of d over the 32 rows into the count of round t (Alg. 1:
//     Count += ||Sig_next(u) XOR Sig(u)||, kept per seed; a 32x32 bit
//     transpose puts each seed's bits of 32 rows in one lane for __popc);
//     X[v] = Y[v] (Alg. 1: Sig(u) = Sig_next(u)); mark v saturated when all
//     its s bits are set (skip rule, proof of Thm. 1).
//  B. choose the direction of round t+1 from the frontier's out-arc count;
//     if sparse, claim every unsaturated out-neighbour of F_t (out-arcs in
//     pieces of LE, flattened per warp like the pull) and list its in-arc
//     pieces, adding its in-degree to m_active[t+1].
//  C. last block: fixpoint test (Alg. 1: do ... while Count > 0), hand-over
//     to round t+1, and, inside a while-graph, the loop condition.
// Four resident blocks per SM (64 registers, no spills): like the pull, the
// kernel is latency-bound, and at the default 80 registers only three fit.
//
// WIDE (rows of 16 or more words, one graph): part A runs over tiles of 32
// frontier rows x 16 words, so that the grid spreads over the words of a row
// and not only over the rows; a row is saturated when its running count of
// set bits (rowbits) reaches s, which exactly one tile sees.
template <bool SMEM, bool WIDE>
__global__ void __launch_bounds__(kBlock, 4) k_post(Params p) {
  extern __shared__ uint32_t scnt[];
  Ctrl *ctrl = p.ctrl;
  if (*(volatile int32_t *)&ctrl->done) {
    if (p.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(p.cond, 0u);
    return;
  }
  const int t = ctrl->t;
  const int row = t - ctrl->row_base;  // row of round t in the counts window
  const unsigned long long fpack = ctrl->fpack;
  const int64_t nF = (int64_t)(fpack >> kFsumBits);
  const int64_t fsum = (int64_t)(fpack & kFsumMask);
  const int64_t nE = (int64_t)ctrl->nE;
  const int64_t nFprev = (int64_t)ctrl->nF_prev;
  const int32_t *F = (t & 1) ? p.F1 : p.F0;
  const int32_t *Fprev = (t & 1) ? p.F0 : p.F1;
  uint64_t *Dcur = (t & 1) ? p.D1 : p.D0;
  uint64_t *Dprev = (t & 1) ? p.D0 : p.D1;
  const uint32_t *Ccur = (t & 1) ? p.C1 : p.C0;
  uint32_t *Cnext = (t & 1) ? p.C0 : p.C1;
  uint32_t *Knext = (t & 1) ? p.K0 : p.K1;
  const int64_t gtid = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * kBlock;
  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid >> 5, nwarps = nth >> 5;
  const int Wp = p.Wp, s = p.s;
  uint32_t *crow = p.counts + (size_t)row * (size_t)p.ncols;

  uint32_t *cdst = SMEM ? scnt : crow;  // per-seed counters of this block / of the round
  if (SMEM) {
    for (int i = threadIdx.x; i < p.ncols; i += kBlock) scnt[i] = 0u;
    __syncthreads();
  }
  // A. count, record deltas, sync, saturation
  if constexpr (WIDE) {
    // tiles of 32 frontier rows x 16 words: each half-warp moves 16
    // consecutive words (128 bytes) of one row, so loads and stores are
    // coalesced; the deltas go through shared memory to a lane-per-row
    // layout for the per-seed bit transpose
    __shared__ uint64_t tile_s[kBlock / 32][32][17];
    uint64_t(*tl)[17] = tile_s[threadIdx.x >> 5];
    const int half = lane >> 4, wl = lane & 15;
    const int nblk = (Wp + 15) >> 4;
    const int64_t ntiles = ((nF + 31) >> 5) * (int64_t)nblk;
    for (int64_t tile = warp; tile < ntiles; tile += nwarps) {
      const int64_t grp = tile / nblk;
      const int w0 = (int)(tile - grp * nblk) * 16;
      const int64_t i = grp * 32 + lane;
      const int32_t vl = i < nF ? F[i] : -1;  // this lane's row in the transpose
      const int w = w0 + wl;
      const bool wok = w < Wp;
      for (int r0 = 0; r0 < 32; r0 += 8) {  // 4 rows per half-warp: 8 loads in flight
        int32_t v[4];
        uint64_t x[4], y[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          v[k] = __shfl_sync(kFullMask, vl, r0 + 2 * k + half);
          x[k] = y[k] = 0ULL;
          if (v[k] >= 0 && wok) {
            const size_t o = (size_t)v[k] * Wp + w;
            x[k] = p.X[o];
            y[k] = __ldg(reinterpret_cast<const unsigned long long *>(p.Y) + o);
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint64_t d = x[k] ^ y[k];
          if (d) {  // the delta buffer of this round is zero elsewhere
            const size_t o = (size_t)v[k] * Wp + w;
            p.X[o] = y[k];
            Dcur[o] = d;
          }
          tl[r0 + 2 * k + half][wl] = d;
        }
      }
      __syncwarp();
      uint32_t gained = 0;
      for (int k = 0; k < 16; ++k) {
        const uint64_t d = tl[lane][k];
        gained += (uint32_t)__popcll(d);
        if (__any_sync(kFullMask, d != 0ULL)) {
          const uint32_t n0 = __popc(transpose32((uint32_t)d, lane));
          const uint32_t n1 = __popc(transpose32((uint32_t)(d >> 32), lane));
          const int c0 = (w0 + k) * 64 + lane;
          if (n0) atomicAdd(&cdst[c0], n0);
          if (n1) atomicAdd(&cdst[c0 + 32], n1);
        }
      }
      __syncwarp();
      if (gained && atomicAdd(p.rowbits + vl, gained) + gained == (uint32_t)s) set_bit(p.Sat, vl);
    }
  } else {
    for (int64_t base = warp * 32; base < nF; base += nwarps * 32) {
      const int64_t i = base + lane;
      const bool valid = i < nF;
      const int32_t v = valid ? F[i] : 0;
      uint64_t *xr = p.X + (size_t)v * Wp;
      const uint64_t *yr = p.Y + (size_t)v * Wp;
      uint64_t *dr = Dcur + (size_t)v * Wp;
      // a batch of disjoint graphs: bit i of a node is its own graph's seed i
      int sv = s, c0v = 0, gid = -1;
      if (p.node_graph && valid) {
        gid = p.node_graph[v];
        sv = p.graph_s[gid];
        c0v = p.graph_col0[gid];
      }
      const int gid0 = __shfl_sync(kFullMask, gid, 0);
      const bool one_graph = !p.node_graph || __all_sync(kFullMask, !valid || gid == gid0);
      const int c0w = __shfl_sync(kFullMask, c0v, 0);
      if (!one_graph) {
        // rows of several graphs in this warp: count each graph's lanes apart
        // (the rows are not yet synced, so X ^ Y is still the delta)
        unsigned todo = __ballot_sync(kFullMask, valid);
        while (todo) {
          const int leader = __ffs(todo) - 1;
          const int gl = __shfl_sync(kFullMask, gid, leader);
          const int cg = __shfl_sync(kFullMask, c0v, leader);
          const bool mine = valid && gid == gl;
          todo &= ~__ballot_sync(kFullMask, mine);
          for (int w = 0; w < Wp; ++w) {
            const uint64_t d =
                mine ? (xr[w] ^ __ldg(reinterpret_cast<const unsigned long long *>(yr) + w)) : 0ULL;
            if (__any_sync(kFullMask, d != 0ULL)) {
              const uint32_t n0 = __popc(transpose32((uint32_t)d, lane));
              const uint32_t n1 = __popc(transpose32((uint32_t)(d >> 32), lane));
              const int c0 = cg + w * 64 + lane;
              if (n0) atomicAdd(&cdst[c0], n0);
              if (n1) atomicAdd(&cdst[c0 + 32], n1);
            }
          }
        }
      }
      bool full = valid;
      if ((Wp & 3) == 0) {  // 32-byte aligned rows: a row's 4 words per load
        for (int w = 0; w < Wp; w += 4) {
          uint64_t o[4] = {0ULL, 0ULL, 0ULL, 0ULL}, nw[4] = {0ULL, 0ULL, 0ULL, 0ULL};
          if (valid) {
            const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(xr + w);
            const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(xr + w + 2);
            o[0] = a.x;
            o[1] = a.y;
            o[2] = b.x;
            o[3] = b.y;
            ld_nc_256(nw, yr + w);
          }
          uint64_t d[4];
  #pragma unroll
          for (int k = 0; k < 4; ++k) d[k] = o[k] ^ nw[k];
          if ((d[0] | d[1] | d[2] | d[3]) != 0ULL) {  // the deltas were zero before
            store_words<4>(xr + w, nw);
            store_words<4>(dr + w, d);
          }
  #pragma unroll
          for (int k = 0; k < 4; ++k) {
            full = full && ((nw[k] | ~valid_mask(w + k, sv)) == ~0ULL);
            if (one_graph && __any_sync(kFullMask, d[k] != 0ULL)) {
              const uint32_t n0 = __popc(transpose32((uint32_t)d[k], lane));
              const uint32_t n1 = __popc(transpose32((uint32_t)(d[k] >> 32), lane));
              const int c0 = c0w + (w + k) * 64 + lane;
              if (n0) atomicAdd(&cdst[c0], n0);
              if (n1) atomicAdd(&cdst[c0 + 32], n1);
            }
          }
        }
      } else {
        for (int w = 0; w < Wp; ++w) {
          uint64_t o = 0, nw = 0;
          if (valid) {
            o = xr[w];
            nw = __ldg(reinterpret_cast<const unsigned long long *>(yr) + w);
          }
          const uint64_t d = o ^ nw;
          if (d) {
            xr[w] = nw;
            dr[w] = d;
          }
          full = full && ((nw | ~valid_mask(w, sv)) == ~0ULL);
          if (one_graph && __any_sync(kFullMask, d != 0ULL)) {
            const uint32_t n0 = __popc(transpose32((uint32_t)d, lane));
            const uint32_t n1 = __popc(transpose32((uint32_t)(d >> 32), lane));
            const int c0 = c0w + w * 64 + lane;
            if (n0) atomicAdd(&cdst[c0], n0);
            if (n1) atomicAdd(&cdst[c0 + 32], n1);
          }
        }
      }
      if (full) set_bit(p.Sat, v);
    }
  }
  // the deltas of round t-1 were read by the pull of round t: clear them
  if constexpr (WIDE) {  // a warp per row, 16 bytes a lane
    const ulonglong2 z = make_ulonglong2(0ULL, 0ULL);
    for (int64_t r = warp; r < nFprev; r += nwarps) {
      ulonglong2 *dr = reinterpret_cast<ulonglong2 *>(Dprev + (size_t)Fprev[r] * Wp);
      for (int k = lane; k < (Wp >> 1); k += 32) dr[k] = z;
    }
  } else {
    const ulonglong2 z = make_ulonglong2(0ULL, 0ULL);
    for (int64_t r = gtid; r < nFprev; r += nth) {  // a thread per row, no division
      uint64_t *dr = Dprev + (size_t)Fprev[r] * Wp;
      if ((Wp & 1) == 0)
        for (int w = 0; w < Wp; w += 2) *reinterpret_cast<ulonglong2 *>(dr + w) = z;
      else
        for (int w = 0; w < Wp; ++w) dr[w] = 0ULL;
    }
  }
  if (SMEM) {
    __syncthreads();
    for (int i = threadIdx.x; i < p.ncols; i += kBlock) {
      const uint32_t c = scnt[i];
      if (c) atomicAdd(&crow[i], c);
    }
  }
  for (int64_t i = gtid; i < p.nbm; i += nth) Cnext[i] = 0u;

  // B. next direction and sparse work list
  const bool next_dense =
      !p.gfsum && (p.direction == PG_DIR_DENSE ||
                   (p.direction == PG_DIR_AUTO &&
                    (double)fsum > (double)p.dense_threshold * (double)p.m));
  // a push round reads this frontier's out-arcs itself: nothing to claim
  // here (a packed batch that pushes: its sparse graphs push, none expands)
  const bool next_push = !next_dense && p.push && !p.gfsum;
  const bool expand =
      !next_dense && !next_push && !(p.gfsum && p.push) && nF > 0 && t + 1 <= p.max_rounds + 1;
  // a packed batch decides per graph: a graph whose frontier out-arcs exceed
  // its own threshold is swept whole in round t+1 and not expanded here
  const unsigned long long *gf_cur = p.gfsum ? p.gfsum + (size_t)(t & 1) * (size_t)p.nseg : nullptr;
  if (p.gfsum) {
    unsigned long long *gf_next = p.gfsum + (size_t)((t + 1) & 1) * (size_t)p.nseg;
    for (int64_t i = gtid; i < p.nseg; i += nth) gf_next[i] = 0ULL;
  }
  unsigned long long my_mact = 0, my_work = 0, my_rows = 0;
  if (expand) {
    // one thread per expansion piece of LE out-arcs, UNR arcs at a time
    constexpr int UNR = 4;
    for (int64_t base = warp * 32; base < nE; base += nwarps * 32) {
      const int64_t i = base + lane;
      int64_t ob = 0, oe = 0;
      if (i < nE) {
        const unsigned long long it = E_of(p, t)[i];
        const int32_t u = (int32_t)(it >> 32);
        const int64_t k = (int64_t)(it & 0xFFFFFFFFULL);
        const int gu = gf_cur ? __ldg(p.node_graph + u) : 0;
        if (!gf_cur || gf_cur[gu] <= __ldg(p.gthr + gu)) {
          const int64_t o1 = __ldg(p.out_ptr + u + 1);
          ob = __ldg(p.out_ptr + u) + k * p.LE;
          oe = min(o1, ob + (int64_t)p.LE);
        }
      }
      for (int h = 0; h < p.LE; h += UNR) {
        int32_t x[UNR];
#pragma unroll
        for (int q = 0; q < UNR; ++q) {
          const int64_t j = ob + h + q;
          x[q] = j < oe ? __ldg(p.out_col + j) : -1;
        }
        bool cand[UNR];
#pragma unroll
        for (int q = 0; q < UNR; ++q)
          cand[q] = x[q] >= 0 && !test_bit_live(p.Sat, x[q]) &&
                    !(test_bit(Ccur, x[q]) &&
                      row_full(p.Y + (size_t)x[q] * Wp, Wp,
                               p.node_graph ? p.graph_s[p.node_graph[x[q]]] : s));
        bool claim[UNR];
#pragma unroll
        for (int q = 0; q < UNR; ++q)  // a bit already seen set needs no atomic
          claim[q] = cand[q] && !test_bit_live(Knext, x[q]) && !set_bit(Knext, x[q]);
        uint32_t np[UNR];
#pragma unroll
        for (int q = 0; q < UNR; ++q) {
          np[q] = 0;
          if (claim[q]) {
            const int64_t indeg = __ldg(p.row_ptr + x[q] + 1) - __ldg(p.row_ptr + x[q]);
            if (!p.pass_words) {  // passes as words: the pull counts each pass
              my_mact += (unsigned long long)indeg;
              my_work += (unsigned long long)indeg * (unsigned long long)seeds_of(p, x[q]);
              ++my_rows;
              if (p.gmact)  // a packed batch: the claimed row's own graph, round t+1
                atomicAdd(p.gmact + (size_t)(row + 1) * (size_t)p.nseg + __ldg(p.node_graph + x[q]),
                          (unsigned long long)indeg);
            }
            np[q] = (uint32_t)((indeg + p.L - 1) / p.L);
          }
        }
        // the step's claims of all lanes: one reservation in the work list
        warp_append_items_n<UNR>(p.A, &ctrl->nA_next, p.row_ptr, x, p.L, np, lane);
      }
    }
  }
  RoundStats *rnext = p.rs + row + 1;
  {
    const unsigned long long vals[3] = {my_mact, my_work, my_rows};
    unsigned long long *const dsts[3] = {&rnext->m_active, &rnext->work, &rnext->rows};
    block_add<3>(vals, dsts);
  }

  // C. last block hands over
  __shared__ int am_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    am_last = atomicAdd(&ctrl->blocks_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (am_last && p.dlist) {
    // a packed batch: the graphs whose frontier chose a full sweep of round
    // t+1, in graph order, and the prefix of their chunk counts, so that the
    // next pull walks only their chunks (a finished graph costs nothing)
    __shared__ long long wsum[kBlock / 32][2];
    __shared__ long long carry[2];
    const unsigned long long *gf = p.gfsum + (size_t)(t & 1) * (size_t)p.nseg;
    const int wl = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry[0] = carry[1] = 0;
    __syncthreads();
    for (int g0 = 0; g0 < p.nseg; g0 += kBlock) {
      const int g = g0 + threadIdx.x;
      const bool d = g < p.nseg && gf[g] > __ldg(p.gthr + g);
      long long v[2] = {d ? 1 : 0, d ? (long long)(p.seg_chunk0[g + 1] - p.seg_chunk0[g]) : 0};
      long long ex[2];
      for (int k = 0; k < 2; ++k) {
        long long x = v[k];
        for (int off = 1; off < 32; off <<= 1) {
          const long long y = __shfl_up_sync(kFullMask, x, off);
          if (lane >= off) x += y;
        }
        ex[k] = x - v[k];
        if (lane == 31) wsum[wl][k] = x;
      }
      __syncthreads();
      for (int k = 0; k < 2; ++k) {
        long long before = carry[k];
        for (int w = 0; w < wl; ++w) before += wsum[w][k];
        ex[k] += before;
      }
      if (d) {
        p.dlist[ex[0]] = g;
        p.dpref[ex[0]] = ex[1];
      }
      __syncthreads();
      if (threadIdx.x == 0)
        for (int w = 0; w < kBlock / 32; ++w) {
          carry[0] += wsum[w][0];
          carry[1] += wsum[w][1];
        }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      p.dpref[carry[0]] = carry[1];
      ctrl->ndense = (int32_t)carry[0];
    }
    __syncthreads();
  }
  if (am_last && threadIdx.x == 0) {
    __threadfence();
    RoundStats *r = p.rs + row;
    r->changed = (unsigned long long)nF;
    r->fsum = (unsigned long long)fsum;
    ctrl->iters += 1;
    ctrl->nF_prev = (unsigned long long)nF;
    if (nF == 0) {
      ctrl->last_round = t - 1;
      ctrl->done = 1;
    } else if (t >= p.max_rounds + 1) {
      ctrl->last_round = t;
      ctrl->status = PG_ERANGE;
      ctrl->done = 1;
    } else if (ctrl->iters > p.iter_guard) {
      ctrl->last_round = t;
      ctrl->status = PG_EDEVICE;
      ctrl->done = 1;
    } else {
      ctrl->t = t + 1;
      ctrl->mode = p.gfsum      ? kModeMixed
                   : next_dense ? kModeDense
                   : next_push  ? kModePush
                                : kModeSparse;
      ctrl->test = (double)fsum < kTestDensity * (double)p.m ? 1 : 0;
      if (next_dense) ctrl->dense_rounds += 1;
      ctrl->nA = *(volatile unsigned long long *)&ctrl->nA_next;
      ctrl->nA_next = 0ULL;
      ctrl->fpack = 0ULL;
      ctrl->nE_prev = ctrl->nE;
      ctrl->nE = 0ULL;
      if (t + 1 - ctrl->row_base >= p.row_cap) {
        ctrl->status = kStatusWindow;
        ctrl->done = 1;
      }
    }
    ctrl->blocks_done = 0u;
    __threadfence();
    if (p.use_cond && ctrl->done) cudaGraphSetConditional(p.cond, 0u);
  }
}

// Moves the counts window after the host copied it out: the statistics slot
// of the next round (already holding its sparse m_active) becomes slot 0.
__global__ void k_window_shift(Params p, int64_t count_words, int32_t rs_slots) {
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  __shared__ RoundStats carry;
  if (threadIdx.x == 0 && blockIdx.x == 0) carry = p.rs[p.row_cap];
  for (int64_t i = gtid; i < count_words; i += nth) p.counts[i] = 0u;
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < rs_slots; i += blockDim.x) {
      if (i == 0)
        p.rs[0] = carry;
      else
        p.rs[i] = RoundStats{};
    }
  }
  if (p.gmact)  // per graph: the next round's slot to slot 0, the rest cleared
    for (int64_t k = gtid; k < p.nseg; k += nth) {
      const unsigned long long c = p.gmact[(size_t)p.row_cap * p.nseg + k];
      for (int32_t i = 1; i < rs_slots; ++i) p.gmact[(size_t)i * p.nseg + k] = 0ULL;
      p.gmact[k] = c;
    }
  if (gtid == 0) {
    p.ctrl->row_base += p.row_cap;
    p.ctrl->status = 0;
    p.ctrl->done = 0;
  }
}

// ---------------------------------------------------------------- host side
struct Plan {
  int CW = 1, G = 4, UNR = 8, L = 32, Wp = 1;
  bool wide = false;  // pull_wide: a warp per row piece
  PullFn pull = nullptr;
  int grid_pull = 1, grid_post = 1;
  size_t post_smem = 0;
  bool smem_counts = true;
  bool post_wide = false;  // k_post's tiled part A (rows of 16+ words, one graph)
  bool pw = false;         // PROPAGATE-S passes as words
  bool tma = false;        // dense rounds by k_pull_tma (TMA-gathered deltas)
  PullFn push = nullptr;   // k_push<CW>, launched after the pull (8-word rows, batches)
  int grid_push = 0;
  int grid_tma = 0;
  CUtensorMap tm0, tm1;    // over D0 and D1 (n + 1 rows)
};

static PullFn pick_pull(int CW, int G, bool pw = false) {
  switch (CW) {
    case 1: return pull_fn_cw1(G, pw);
    case 2: return pull_fn_cw2(G, pw);
    case 4: return pull_fn_cw4(G, pw);
    case 8: return pull_fn_cw8(G, pw);
  }
  return nullptr;
}

static int occupancy_grid(const void *fn, size_t smem, int64_t work_threads) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, smem);
  if (per_sm < 1) per_sm = 1;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  const int64_t need = (work_threads + kBlock - 1) / kBlock;
  return (int)std::max<int64_t>(1, std::min(cap, need));
}

// Group size: the smallest power of two whose piece (G * UNR arcs) covers the
// mean in-degree, so that a typical row is one piece.
static int auto_group(double mean_degree, int unr) {
  int G = 1;
  while (G < 32 && (double)(G * unr) < mean_degree) G <<= 1;
  return G;
}

static pg_status make_plan(const pg_graph *g, int sp, const pg_options &o, bool s_mode, Plan &pl) {
  const int W = s_mode ? 1 : (sp + 63) / 64;
  pl.CW = W <= 1 ? 1 : W <= 2 ? 2 : W <= 4 ? 4 : 8;
  if (o.words_per_thread != 0) {
    const int c = o.words_per_thread;
    if (c < 0 || c > 8 || (c & (c - 1))) return PG_EINVAL;
    pl.CW = std::min(pl.CW, c);
  }
  pl.Wp = (W + pl.CW - 1) / pl.CW * pl.CW;
  if (o.wide_rows < 0 || o.wide_rows > 2) return PG_EINVAL;
  if (W > 8 && o.wide_rows != 2) {
    // a warp per row piece, lanes over the row's words (pull_wide.cu)
    pl.CW = 8;
    pl.Wp = (W + 7) / 8 * 8;
    pl.UNR = 8;
    pl.G = 32;
    pl.L = kWidePiece;
    pl.pull = pull_fn_wide(pl.Wp);
    pl.smem_counts = sp <= kSmemCountMax;
    pl.post_smem = pl.smem_counts ? sizeof(uint32_t) * (size_t)sp : 0;
    pl.wide = true;
    return PG_OK;
  }
  pl.UNR = pl.CW <= 2 ? 8 : (pl.CW == 4 ? 4 : 2);
  int G = o.group_lanes > 0 ? o.group_lanes : auto_group(g->mean_degree, pl.UNR);
  if (G > 32 || (G & (G - 1))) return PG_EINVAL;
  pl.G = G;
  pl.L = G * pl.UNR;
  pl.pull = pick_pull(pl.CW, pl.G);
  if (!pl.pull) return PG_EINVAL;
  pl.smem_counts = sp <= kSmemCountMax;
  pl.post_smem = pl.smem_counts ? sizeof(uint32_t) * (size_t)sp : 0;
  return PG_OK;
}

static const void *post_fn(const Plan &pl) {
  if (pl.post_wide)
    return pl.smem_counts ? (const void *)&k_post<true, true> : (const void *)&k_post<false, true>;
  return pl.smem_counts ? (const void *)&k_post<true, false> : (const void *)&k_post<false, false>;
}

// Raises the dynamic shared memory limit of the shared-counter post kernels
// to the largest count window (once per device, before any launch, so that
// no thread changes it while another launches them).
static void post_smem_optin() {
  static std::mutex mu;
  static uint64_t done = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && (done >> dev) & 1ULL) return;
  const int mx = (int)(sizeof(uint32_t) * kSmemCountMax);
  cudaFuncSetAttribute((const void *)&k_post<true, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute((const void *)&k_post<true, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (dev < 64) done |= 1ULL << dev;
}

static void launch_post(const Plan &pl, const Params &p, cudaStream_t st) {
  const size_t smem = pl.smem_counts ? pl.post_smem : 0;
  if (pl.post_wide) {
    if (pl.smem_counts)
      k_post<true, true><<<pl.grid_post, kBlock, smem, st>>>(p);
    else
      k_post<false, true><<<pl.grid_post, kBlock, smem, st>>>(p);
  } else {
    if (pl.smem_counts)
      k_post<true, false><<<pl.grid_post, kBlock, smem, st>>>(p);
    else
      k_post<false, false><<<pl.grid_post, kBlock, smem, st>>>(p);
  }
}

// The pull of one round: k_pull_tma first when it sweeps the dense rounds
// (it returns at once in the others), then k_pull.
static void launch_pulls(const Plan &pl, const Params &p, cudaStream_t st) {
  if (pl.tma) launch_pull_tma(pl.CW, pl.pw, p, &pl.tm0, &pl.tm1, pl.grid_tma, st);
  pl.pull<<<pl.grid_pull, kBlock, 0, st>>>(p);
  if (pl.push) pl.push<<<pl.grid_push, kBlock, 0, st>>>(p);
}

// kernel launches of one round: the pulls and the post kernel
static int round_launches(const Plan &pl) { return 2 + (pl.tma ? 1 : 0) + (pl.push ? 1 : 0); }

static void launch_round(const Plan &pl, const Params &p, cudaStream_t st) {
  launch_pulls(pl, p, st);
  launch_post(pl, p, st);
}

// Raises the dynamic shared memory limit of the TMA pull kernels (once per
// device, before any launch).
static void tma_smem_optin() {
  static std::mutex mu;
  static uint64_t done = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && (done >> dev) & 1ULL) return;
  for (int cw : {4, 8})
    for (bool pw : {false, true})
      cudaFuncSetAttribute(pull_tma_fn(cw, pw), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)pull_tma_smem(cw));
  if (dev < 64) done |= 1ULL << dev;
}

struct PassOut {
  int32_t rounds = 0;
  int32_t status = 0;
  int32_t dense_rounds = 0;
  int32_t launches = 0;
  double ms_pull = 0, ms_post = 0, ms_init = 0;
  int32_t pull_launches = 0, post_launches = 0;
  bool tma = false;
};

struct Call {
  pg_graph *g;
  cudaStream_t st;
  pg_options o;
  int32_t s_total;
  int32_t max_rounds;
  uint32_t *counts_h;            // caller rows x s_total
  std::vector<RoundStats> rs_h;  // summed over passes, grown as rounds complete
  int32_t row_cap = 0;
  WindowSink sink = nullptr;
  void *sink_ctx = nullptr;
  std::vector<uint32_t> stage;
  const int32_t *perm = nullptr;  // relabelled graph: caller id -> internal id
  int64_t perm_n = 0;
  // a packed batch, on request: m_active of each graph by round ([round][graph])
  std::vector<unsigned long long> *gm_h = nullptr;
};

static pg_status copy_window(Call &cl, const Params &p, int col0, int32_t row_base, int32_t rows,
                             int32_t rs_rows) {
  rows = std::min(rows, cl.max_rounds + 1 - row_base);
  if (rows > 0 && cl.sink) {
    cl.stage.resize((size_t)rows * p.ncols);
    cudaError_t e = cudaMemcpyAsync(cl.stage.data(), p.counts,
                                    sizeof(uint32_t) * (size_t)rows * p.ncols,
                                    cudaMemcpyDeviceToHost, cl.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cl.st);
    if (e != cudaSuccess) return cuda_status(e);
    cl.sink(cl.sink_ctx, row_base, rows, cl.stage.data(), p.ncols);
  } else if (rows > 0) {
    cudaError_t e = cudaMemcpy2DAsync(cl.counts_h + (size_t)row_base * cl.s_total + col0,
                                      sizeof(uint32_t) * cl.s_total, p.counts,
                                      sizeof(uint32_t) * p.ncols, sizeof(uint32_t) * p.ncols, rows,
                                      cudaMemcpyDeviceToHost, cl.st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  rs_rows = std::min(rs_rows, cl.max_rounds + 2 - row_base);
  if (rs_rows > 0) {
    std::vector<RoundStats> tmp(rs_rows);
    cudaError_t e = cudaMemcpyAsync(tmp.data(), p.rs, sizeof(RoundStats) * rs_rows,
                                    cudaMemcpyDeviceToHost, cl.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cl.st);
    if (e != cudaSuccess) return cuda_status(e);
    if ((int64_t)cl.rs_h.size() < (int64_t)row_base + rs_rows)
      cl.rs_h.resize((size_t)row_base + rs_rows, RoundStats{});
    for (int i = 0; i < rs_rows; ++i) {
      RoundStats &d = cl.rs_h[(size_t)row_base + i];
      d.work += tmp[i].work;
      d.m_active += tmp[i].m_active;
      d.scanned += tmp[i].scanned;
      d.gathered += tmp[i].gathered;
      d.items += tmp[i].items;
      d.changed += tmp[i].changed;
      d.fsum += tmp[i].fsum;
      d.rows += tmp[i].rows;
    }
    if (p.gmact && cl.gm_h) {
      const size_t ns = (size_t)p.nseg;
      std::vector<unsigned long long> g((size_t)rs_rows * ns);
      e = cudaMemcpyAsync(g.data(), p.gmact, sizeof(unsigned long long) * g.size(),
                          cudaMemcpyDeviceToHost, cl.st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(cl.st);
      if (e != cudaSuccess) return cuda_status(e);
      std::vector<unsigned long long> &h = *cl.gm_h;
      if (h.size() < ((size_t)row_base + rs_rows) * ns) h.resize(((size_t)row_base + rs_rows) * ns, 0ULL);
      for (size_t i = 0; i < g.size(); ++i) h[(size_t)row_base * ns + i] += g[i];
    }
  }
  return cuda_status(cudaStreamSynchronize(cl.st));
}

// ------------------------------------------------------ captured round loop
// A device-driven while-loop graph whose body is one round (pull + post); the
// post kernel ends the loop at the fixpoint, on an error or when the counts
// window is full. Cached per graph handle while the launch parameters stay
// the same.
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  Params p{};
  PullFn pull = nullptr;
  int grid_pull = 0, grid_post = 0;
  size_t smem = 0;
  bool smem_counts = true;
  bool post_wide = false;
  bool tma = false;
  int grid_tma = 0;
  PullFn push = nullptr;
  int grid_push = 0;
  unsigned char tm[2][sizeof(CUtensorMap)] = {};
  cudaStream_t cap = nullptr;
};

static std::mutex g_cache_mu;
static std::vector<std::pair<pg_graph *, GraphCache>> g_caches;

static GraphCache &cache_for(pg_graph *g) {
  for (auto &pr : g_caches)
    if (pr.first == g) return pr.second;
  g_caches.push_back({g, GraphCache{}});
  return g_caches.back().second;
}

static pg_status ensure_while_graph(pg_graph *g, const Plan &pl, const Params &p,
                                    cudaGraphExec_t *out) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  GraphCache &c = cache_for(g);
  Params key = p;
  key.use_cond = 1;
  key.cond = c.p.cond;  // compare everything but the handle
  if (c.exec && c.pull == pl.pull && c.grid_pull == pl.grid_pull &&
      c.grid_post == pl.grid_post && c.smem == pl.post_smem && c.smem_counts == pl.smem_counts &&
      c.post_wide == pl.post_wide && c.tma == pl.tma && c.grid_tma == pl.grid_tma &&
      c.push == pl.push && c.grid_push == pl.grid_push &&
      (!pl.tma || (std::memcmp(c.tm[0], &pl.tm0, sizeof(CUtensorMap)) == 0 &&
                   std::memcmp(c.tm[1], &pl.tm1, sizeof(CUtensorMap)) == 0)) &&
      std::memcmp(&c.p, &key, sizeof(Params)) == 0) {
    *out = c.exec;
    return PG_OK;
  }
  if (c.exec) {
    cudaGraphExecDestroy(c.exec);
    c.exec = nullptr;
  }
  if (!c.cap && cudaStreamCreateWithFlags(&c.cap, cudaStreamNonBlocking) != cudaSuccess)
    return PG_ECUDA;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  if (e != cudaSuccess) return cuda_status(e);
  cudaGraphConditionalHandle h = 0;
  e = cudaGraphConditionalHandleCreate(&h, graph, 1u, cudaGraphCondAssignDefault);
  // cudaGraphNodeParams has no default constructor in C++ (a union of
  // structs); build it in zeroed raw storage, as the API requires.
  alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)];
  std::memset(np_raw, 0, sizeof(np_raw));
  cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(np_raw);
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  Params pc = p;
  pc.use_cond = 1;
  pc.cond = (unsigned long long)h;
  if (e == cudaSuccess) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c.cap, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      launch_round(pl, pc, c.cap);
      cudaGraph_t captured = nullptr;
      e = cudaStreamEndCapture(c.cap, &captured);
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c.exec = nullptr;
    return cuda_status(e);
  }
  c.p = pc;
  c.pull = pl.pull;
  c.grid_pull = pl.grid_pull;
  c.grid_post = pl.grid_post;
  c.smem = pl.post_smem;
  c.smem_counts = pl.smem_counts;
  c.post_wide = pl.post_wide;
  c.tma = pl.tma;
  c.grid_tma = pl.grid_tma;
  c.push = pl.push;
  c.grid_push = pl.grid_push;
  std::memcpy(c.tm[0], &pl.tm0, sizeof(CUtensorMap));
  std::memcpy(c.tm[1], &pl.tm1, sizeof(CUtensorMap));
  *out = c.exec;
  return PG_OK;
}

void drop_graph_cache(pg_graph *g) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  for (size_t i = 0; i < g_caches.size(); ++i)
    if (g_caches[i].first == g) {
      if (g_caches[i].second.exec) cudaGraphExecDestroy(g_caches[i].second.exec);
      if (g_caches[i].second.cap) cudaStreamDestroy(g_caches[i].second.cap);
      g_caches.erase(g_caches.begin() + i);
      return;
    }
}

// A batch of disjoint graphs packed into one graph (see pg_batch_run).
struct BatchSeg {
  const int32_t *node_graph;  // device, graph of each node
  const int32_t *graph_s;     // device, seeds of each graph
  const int32_t *graph_col0;  // device, first count column of each graph
  const int32_t *seed_bit;    // host, each seed's index within its graph
  int32_t ncols;              // count columns (sum of the graphs' seeds)
  int32_t s_bits;             // most seeds of one graph (bits per node)
  const int64_t *graph_m;     // host, arcs of each graph (per-graph round kinds)
};

// One pass: sp seeds of the call, columns [col0, col0+sp); or, with bs, all
// seeds of a packed batch.
// With pw, the sp seeds are ceil(sp/64) PROPAGATE-S passes of 64 planes run
// side by side as the words of one signature (m_active counted per pass).
static pg_status run_pass(Call &cl, const int32_t *seeds_h, int sp, int col0, bool eb,
                          int hint, PassOut &po, const BatchSeg *bs = nullptr, bool pw = false) {
  pg_graph *g = cl.g;
  Workspace &w = g->ext_ws ? *g->ext_ws : g->ws;
  cudaStream_t st = cl.st;
  Plan pl;
  const int s_bits = bs ? bs->s_bits : sp;
  const int ncols = bs ? bs->ncols : sp;
  pg_status rc = make_plan(g, s_bits, cl.o, eb, pl);
  if (rc) return rc;
  if (pw) {  // the instantiations that count m_active per pass
    pl.pull = pl.wide ? pull_fn_wide(pl.Wp, true) : pick_pull(pl.CW, pl.G, true);
    if (!pl.pull) return PG_EINVAL;
  }
  pl.pw = pw;
  if (bs) {  // a batch's columns: in shared memory when they fit
    pl.smem_counts = ncols <= kSmemCountMax;
    pl.post_smem = pl.smem_counts ? sizeof(uint32_t) * (size_t)ncols : 0;
  }
  // the list of every row's pieces is read only by the wide-row pull (its
  // dense rounds); the others take their dense rounds from the sliced-ELL
  // copy and size the sparse work list by a bound on the piece count
  if (pl.wide && (rc = ensure_pieces(g, pl.L, st))) return rc;
  const int64_t npieces = pl.wide ? g->pieces.count : g->n + g->m / pl.L + 1;
  if (cl.o.direction != PG_DIR_SPARSE && !pl.wide && (rc = ensure_sell(g, kSellPiece, st)))
    return rc;
  const int64_t n = g->n;
  const int64_t nbm = (n + 31) / 32;
  const int32_t row_cap = cl.row_cap;
  const int64_t e_cap = n + g->m / kExpandArcs + 1;
  const size_t sig_bytes = sizeof(uint64_t) * (size_t)n * pl.Wp;
  const size_t bm_bytes = sizeof(uint32_t) * (size_t)nbm;
  pl.post_wide = !bs && pl.Wp >= kWidePostWords;
  // the delta buffers keep one all-zero row past the last node (the row a
  // TMA gather of an empty slot reads)
  const size_t delta_bytes_alloc = sig_bytes + sizeof(uint64_t) * (size_t)pl.Wp;
  std::vector<std::pair<DevBuf *, size_t>> needs = {
      {&w.X, sig_bytes}, {&w.Y, sig_bytes}, {&w.D0, delta_bytes_alloc}, {&w.D1, delta_bytes_alloc},
      {&w.C0, bm_bytes}, {&w.C1, bm_bytes}, {&w.K0, bm_bytes}, {&w.K1, bm_bytes},
      {&w.Sat, bm_bytes},
      {&w.F0, sizeof(int32_t) * (size_t)n}, {&w.F1, sizeof(int32_t) * (size_t)n},
      {&w.E, sizeof(unsigned long long) * (size_t)e_cap},
      {&w.A, sizeof(ulonglong2) * (size_t)std::max<int64_t>(npieces, 1)},
      {&w.counts, sizeof(uint32_t) * (size_t)row_cap * (size_t)ncols},
      {&w.rs, sizeof(RoundStats) * (size_t)(row_cap + 2)},
      {&w.ctrl, sizeof(Ctrl)}, {&w.seeds, sizeof(int32_t) * (size_t)sp}};
  if (pl.post_wide) needs.push_back({&w.RB, sizeof(uint32_t) * (size_t)n});
  if (pw) {
    needs.push_back({&w.KW0, bm_bytes * (size_t)pl.Wp});
    needs.push_back({&w.KW1, bm_bytes * (size_t)pl.Wp});
  }
  if (bs) needs.push_back({&w.seed_bits, sizeof(int32_t) * (size_t)sp});
  // push rounds (rows of up to 8 words gathered whole): the frontier's
  // out-arc pieces by round parity. The default where they apply: measured
  // faster on the 4096^2 grid by 19%, on R-MAT 22 with s = 256 by 13%, on ER
  // 10^6 with s = 128 by 11%, on R-MAT 26 with s = 512 by 10% and on the
  // 512-graph mix (batched) by 3%
  const bool push_ok = !pl.wide && pl.CW == pl.Wp;
  const bool push = push_ok && cl.o.sparse_push != 1;
  if (push) needs.push_back({&w.E1, sizeof(unsigned long long) * (size_t)e_cap});
  if (bs && g->nseg > 0) {
    needs.push_back({&w.gfsum, 2 * sizeof(unsigned long long) * (size_t)g->nseg});
    needs.push_back({&w.gthr, sizeof(unsigned long long) * (size_t)g->nseg});
    needs.push_back({&w.dlist, sizeof(int32_t) * (size_t)g->nseg});
    needs.push_back({&w.dpref, sizeof(int64_t) * ((size_t)g->nseg + 1)});
  }
  // a packed batch whose caller asked for each graph's m_active: its window
  const bool gm_on = bs && g->nseg > 0 && bs->graph_m && !pw && cl.gm_h;
  if (gm_on)
    needs.push_back({&w.gm, sizeof(unsigned long long) * (size_t)(row_cap + 2) * (size_t)g->nseg});
  if ((rc = carve_workspace(w, needs))) return rc;
  if (!w.ctrl_h) {
    if (cudaMallocHost((void **)&w.ctrl_h, 2 * sizeof(Ctrl)) != cudaSuccess) {
      w.ctrl_h = nullptr;
      return PG_ENOMEM;
    }
    for (auto &e : w.ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return PG_ECUDA;
  }
  Params p{};
  p.n = n;
  p.m = g->m;
  p.row_ptr = g->row_ptr;
  p.col = g->col;
  p.out_ptr = g->out_ptr;
  p.out_col = g->out_col;
  p.X = (uint64_t *)w.X.p;
  p.Y = (uint64_t *)w.Y.p;
  p.D0 = (uint64_t *)w.D0.p;
  p.D1 = (uint64_t *)w.D1.p;
  p.Wp = pl.Wp;
  p.s = s_bits;
  p.C0 = (uint32_t *)w.C0.p;
  p.C1 = (uint32_t *)w.C1.p;
  p.K0 = (uint32_t *)w.K0.p;
  p.K1 = (uint32_t *)w.K1.p;
  p.Sat = (uint32_t *)w.Sat.p;
  p.rowbits = pl.post_wide ? (uint32_t *)w.RB.p : nullptr;
  p.pass_words = pw ? 1 : 0;
  p.Kw0 = pw ? (uint32_t *)w.KW0.p : nullptr;
  p.Kw1 = pw ? (uint32_t *)w.KW1.p : nullptr;
  p.nbm = nbm;
  p.F0 = (int32_t *)w.F0.p;
  p.F1 = (int32_t *)w.F1.p;
  p.E = (unsigned long long *)w.E.p;
  p.E1 = push ? (unsigned long long *)w.E1.p : nullptr;
  p.push = push ? 1 : 0;
  // k_pull pushes rows of up to 4 words of one graph, PROPAGATE-P or one
  // pass at a time, itself; the rest push in k_push
  const bool push_kernel = push && (bs != nullptr || pl.CW == 8 || pw);
  p.push_kernel = push_kernel ? 1 : 0;
  pl.push = push_kernel ? push_fn(pl.CW, pw) : nullptr;
  p.A = (ulonglong2 *)w.A.p;
  p.Pall = pl.wide ? (const ulonglong2 *)g->pieces.list.p : nullptr;
  p.nPall = pl.wide ? g->pieces.count : 0;
  p.sell_items = (const ulonglong2 *)g->sell.items.p;
  p.sell_col = (const int32_t *)g->sell.col.p;
  p.sell_off = (const int64_t *)g->sell.off.p;
  p.sell_len = (const int32_t *)g->sell.len.p;
  p.sell_chunks = cl.o.direction != PG_DIR_SPARSE && !pl.wide ? g->sell.nchunks : 0;
  p.L = pl.L;
  p.LE = kExpandArcs;
  p.counts = (uint32_t *)w.counts.p;
  p.ncols = ncols;
  p.node_graph = bs ? bs->node_graph : nullptr;
  p.graph_s = bs ? bs->graph_s : nullptr;
  p.graph_col0 = bs ? bs->graph_col0 : nullptr;
  // a packed batch: each graph picks its own kind of round (the sliced-ELL
  // chunks are per graph; finished graphs have no frontier and cost nothing)
  const bool seg = bs && g->nseg > 0 && bs->graph_m;
  p.gfsum = seg ? (unsigned long long *)w.gfsum.p : nullptr;
  p.gthr = seg ? (const unsigned long long *)w.gthr.p : nullptr;
  p.nseg = seg ? g->nseg : 0;
  p.sell_seg = seg && !pl.wide ? (const int32_t *)g->sell.seg.p : nullptr;
  // the dense sweep of a packed batch walks only the chunks of the graphs in
  // a full sweep (dlist, built by the post kernel)
  const bool dl = seg && !pl.wide && p.sell_chunks > 0 && g->sell.chunk0.p;
  p.seg_chunk0 = dl ? (const int64_t *)g->sell.chunk0.p : nullptr;
  p.dlist = dl ? (int32_t *)w.dlist.p : nullptr;
  p.dpref = dl ? (int64_t *)w.dpref.p : nullptr;
  p.gmact = gm_on ? (unsigned long long *)w.gm.p : nullptr;
  p.perm = cl.perm;
  p.perm_n = cl.perm_n;
  p.rs = (RoundStats *)w.rs.p;
  p.ctrl = (Ctrl *)w.ctrl.p;
  p.max_rounds = cl.max_rounds;
  p.row_cap = row_cap;
  p.direction = cl.o.direction;
  p.dense_threshold = cl.o.dense_threshold > 0 ? cl.o.dense_threshold : 0.05f;
  // gather deltas unconditionally while they stay mostly in L2; beyond that,
  // test the (L2-resident) changed bitmap first
  const int64_t delta_bytes = n * (int64_t)pl.Wp * 8;
  // 1: always test; 2: never; 3: per round; 0: per round once the deltas
  // outgrow L2 (a packed batch: always, its frontiers are per graph)
  const bool big = delta_bytes > (64LL << 20);
  p.test_changed = cl.o.test_changed == 1 || cl.o.test_changed == 3 ||
                   (cl.o.test_changed == 0 && big);
  p.test_adapt = !p.gfsum && (cl.o.test_changed == 3 || (cl.o.test_changed == 0 && big));
  p.use_cond = 0;
  p.cond = 0ULL;
  p.iter_guard = cl.max_rounds + 2;
  // TMA-gathered dense rounds: one graph (not a packed batch), rows of 4 or
  // 8 words gathered whole, a sliced-ELL copy to sweep
  const bool tma_ok = !bs && !pl.wide && pl.CW == pl.Wp && (pl.CW == 4 || pl.CW == 8) &&
                      p.sell_chunks > 0;
  // only on request: per-lane 256-bit loads measured faster on the
  // relabelled scale-26 R-MAT (99.5 vs 171.7 ms of pull per PROPAGATE-P call)
  pl.tma = tma_ok && cl.o.tma_gather == 2;
  if (pl.tma) {
    if ((rc = encode_delta_map(&pl.tm0, p.D0, n + 1, pl.Wp, pl.CW)) ||
        (rc = encode_delta_map(&pl.tm1, p.D1, n + 1, pl.Wp, pl.CW)))
      return rc;
    tma_smem_optin();
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pull_tma_fn(pl.CW, pw), kBlock,
                                                  pull_tma_smem(pl.CW));
    if (per_sm < 1) return PG_ECUDA;
    pl.grid_tma = sm_count() * per_sm;
  }
  p.dense_tma = pl.tma ? 1 : 0;

  const int64_t pull_threads = std::max<int64_t>({npieces * pl.G, nbm, p.sell_chunks * 32});
  pl.grid_pull = occupancy_grid((const void *)pl.pull, 0, pull_threads);
  if (pl.push) pl.grid_push = occupancy_grid((const void *)pl.push, 0, n + g->m / kExpandArcs + 1);
  // the wide part A has a warp per 32 rows x 16 words
  const int64_t post_threads =
      pl.post_wide ? (n + 31) / 32 * (int64_t)((pl.Wp + 15) / 16) * 32 : n;
  post_smem_optin();
  pl.grid_post = occupancy_grid(post_fn(pl), pl.post_smem, std::max<int64_t>(post_threads, nbm));

  const bool timing = cl.o.timing != 0;
  const bool graphs = cl.o.use_graphs != 0 && !timing;
  auto tev = [&](int idx) -> cudaEvent_t {
    while ((int)w.tev.size() <= idx) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      w.tev.push_back(e);
    }
    return w.tev[idx];
  };
  int ntev = 0;
  std::vector<std::pair<int, int>> pull_ev, post_ev;
  int init_ev0 = -1, init_ev1 = -1;

  // init: zero, seeds, post(0)
  if (timing) {
    init_ev0 = ntev++;
    cudaEventRecord(tev(init_ev0), st);
  }
  rc = cuda_status(cudaMemcpyAsync(w.seeds.p, seeds_h, sizeof(int32_t) * sp,
                                   cudaMemcpyHostToDevice, st));
  if (rc == PG_OK && p.gfsum) {
    std::vector<unsigned long long> thr((size_t)g->nseg);
    const double f = p.dense_threshold;
    for (int32_t k = 0; k < g->nseg; ++k)
      thr[k] = cl.o.direction == PG_DIR_DENSE    ? 0ULL
               : cl.o.direction == PG_DIR_SPARSE ? ~0ULL
                                                 : (unsigned long long)(f * (double)bs->graph_m[k]);
    rc = cuda_status(cudaMemsetAsync(p.gfsum, 0, 2 * sizeof(unsigned long long) * g->nseg, st));
    if (rc == PG_OK)
      rc = cuda_status(cudaMemcpyAsync(w.gthr.p, thr.data(), sizeof(unsigned long long) * g->nseg,
                                       cudaMemcpyHostToDevice, st));
    if (rc == PG_OK) rc = cuda_status(cudaStreamSynchronize(st));  // thr outlives the copy
  }
  if (rc == PG_OK && bs)
    rc = cuda_status(cudaMemcpyAsync(w.seed_bits.p, bs->seed_bit, sizeof(int32_t) * sp,
                                     cudaMemcpyHostToDevice, st));
  if (rc) return rc;
  const int64_t count_words = (int64_t)row_cap * ncols;
  const int64_t rs_words = (int64_t)(row_cap + 2) * (int64_t)(sizeof(RoundStats) / 8);
  const int64_t zero_work = std::max<int64_t>({n * pl.Wp / 2, nbm, count_words, rs_words, 1});
  k_zero<<<occupancy_grid((const void *)&k_zero, 0, zero_work), kBlock, 0, st>>>(p, count_words,
                                                                                rs_words);
  k_seed<<<1, 1024, 0, st>>>(p, (const int32_t *)w.seeds.p,
                             bs ? (const int32_t *)w.seed_bits.p : nullptr, sp);
  launch_post(pl, p, st);
  po.launches += 3;
  if (timing) {
    init_ev1 = ntev++;
    cudaEventRecord(tev(init_ev1), st);
  }
  if ((rc = cuda_status(cudaGetLastError()))) return rc;

  int32_t row_base = 0;
  Ctrl fin{};
  bool finished = false;
  if (graphs) {
    // Device-driven loop: one graph launch runs rounds until the fixpoint,
    // an error, or a full counts window.
    cudaGraphExec_t exec = nullptr;
    if ((rc = ensure_while_graph(g, pl, p, &exec))) return rc;
    int64_t launches_guard = (int64_t)cl.max_rounds / std::max<int32_t>(row_cap, 1) + 4;
    while (!finished) {
      if (launches_guard-- < 0) return PG_EDEVICE;
      if ((rc = cuda_status(cudaGraphLaunch(exec, st)))) return rc;
      cudaMemcpyAsync(&w.ctrl_h[0], p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
      if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
      const Ctrl c = w.ctrl_h[0];
      if (!c.done) return PG_EDEVICE;
      if (c.status == kStatusWindow) {
        if ((rc = copy_window(cl, p, col0, row_base, row_cap, row_cap))) return rc;
        k_window_shift<<<occupancy_grid((const void *)&k_window_shift, 0, count_words), kBlock,
                         0, st>>>(p, count_words, row_cap + 2);
        row_base += row_cap;
        if ((rc = cuda_status(cudaGetLastError()))) return rc;
        continue;
      }
      fin = c;
      finished = true;
    }
    // every round of the loop is its pull launches and one post launch;
    // iters counts the post launches of the pass, post(0) included
    po.launches = 3 + round_launches(pl) * (std::max(0, fin.iters) - 1);
  } else {
    // Host-driven loop: batches of K rounds; the host reads the control
    // block of the batch before last while the last one runs. A first batch
    // of `hint` rounds (the sweeps of the previous call on this graph) is
    // checked on its own, so a repeated call launches no idle rounds.
    int K = 2;
    if (hint > 0) {
      for (int k = 0; k < hint; ++k) {
        if (timing) {
          int a = ntev++, b = ntev++, c = ntev++;
          cudaEventRecord(tev(a), st);
          launch_pulls(pl, p, st);
          cudaEventRecord(tev(b), st);
          launch_post(pl, p, st);
          cudaEventRecord(tev(c), st);
          pull_ev.push_back({a, b});
          post_ev.push_back({b, c});
        } else {
          launch_round(pl, p, st);
        }
      }
      po.launches += round_launches(pl) * hint;
      if ((rc = cuda_status(cudaGetLastError()))) return rc;
      Ctrl cnow;
      if ((rc = cuda_status(cudaMemcpyAsync(&w.ctrl_h[0], p.ctrl, sizeof(Ctrl),
                                            cudaMemcpyDeviceToHost, st))) ||
          (rc = cuda_status(cudaStreamSynchronize(st))))
        return rc;
      cnow = w.ctrl_h[0];
      if (cnow.done && cnow.status != kStatusWindow) {
        fin = cnow;
        finished = true;
      }
      K = 4;
    }
    int slot = 0;
    int pending[2];
    int npending = 0;
    int64_t enqueued = 0;
    const int64_t guard = (int64_t)cl.max_rounds + 4 + 64;
    while (!finished) {
      for (int k = 0; k < K; ++k) {
        if (timing) {
          int a = ntev++, b = ntev++, c = ntev++;
          cudaEventRecord(tev(a), st);
          launch_pulls(pl, p, st);
          cudaEventRecord(tev(b), st);
          launch_post(pl, p, st);
          cudaEventRecord(tev(c), st);
          pull_ev.push_back({a, b});
          post_ev.push_back({b, c});
        } else {
          launch_round(pl, p, st);
        }
      }
      enqueued += K;
      po.launches += round_launches(pl) * K;
      if ((rc = cuda_status(cudaGetLastError()))) return rc;
      cudaMemcpyAsync(&w.ctrl_h[slot], p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
      cudaEventRecord(w.ev[slot], st);
      pending[npending++] = slot;
      slot ^= 1;
      K = std::min(K * 2, 16);
      if (npending == 2 || enqueued > guard) {
        const int s0 = pending[0];
        if ((rc = cuda_status(cudaEventSynchronize(w.ev[s0])))) return rc;
        pending[0] = pending[1];
        npending--;
        const Ctrl c = w.ctrl_h[s0];
        if (c.done) {
          if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
          npending = 0;
          Ctrl cnow;
          if ((rc = cuda_status(cudaMemcpy(&cnow, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost))))
            return rc;
          if (cnow.status == kStatusWindow) {
            if ((rc = copy_window(cl, p, col0, row_base, row_cap, row_cap))) return rc;
            k_window_shift<<<occupancy_grid((const void *)&k_window_shift, 0, count_words),
                             kBlock, 0, st>>>(p, count_words, row_cap + 2);
            po.launches += 1;
            row_base += row_cap;
            enqueued = 0;  // each shift is progress: the guard counts rounds since it
            if ((rc = cuda_status(cudaGetLastError()))) return rc;
            continue;
          }
          fin = cnow;
          finished = true;
        } else if (enqueued > guard) {
          return PG_EDEVICE;
        }
      }
    }
  }
  if (fin.status == PG_EDEVICE || fin.status == PG_ETIMEOUT) return (pg_status)fin.status;
  if (fin.bad_index) return PG_EDEVICE;  // a PG_DEBUG_BOUNDS build caught a bad gather
  const int32_t last = fin.status == PG_ERANGE ? cl.max_rounds : fin.last_round;
  const int32_t rows = last - row_base + 1;
  if ((rc = copy_window(cl, p, col0, row_base, rows, rows + 1))) return rc;
  po.rounds = fin.status == PG_ERANGE ? cl.max_rounds + 1 : fin.last_round;
  po.tma = pl.tma;
  po.status = fin.status;
  po.dense_rounds = fin.dense_rounds;
  if (timing) {
    float ms = 0;
    cudaEventElapsedTime(&ms, tev(init_ev0), tev(init_ev1));
    po.ms_init += ms;
    for (auto &pr : pull_ev) {
      cudaEventElapsedTime(&ms, tev(pr.first), tev(pr.second));
      po.ms_pull += ms;
    }
    for (auto &pr : post_ev) {
      cudaEventElapsedTime(&ms, tev(pr.first), tev(pr.second));
      po.ms_post += ms;
    }
    po.pull_launches += (int)pull_ev.size();
    po.post_launches += (int)post_ev.size();
  }
  return PG_OK;
}

// How many PROPAGATE-S passes run together (over replicas of the graph).
// Automatic: only while the copies together stay small (kReplicaArcs arcs):
// one pass of a larger graph already fills the GPU, and there the copies'
// per-graph bookkeeping costs more than the launches it saves (measured on
// a 65 M-arc R-MAT). Always as far as a quarter of the free device memory
// holds the copies and their workspace and node ids stay below 2^31.
constexpr int64_t kReplicaArcs = 1LL << 24;

static int passes_together(const pg_graph *g, int npasses, const pg_options &o) {
  if (npasses < 2 || o.passes_together == 1) return 1;
  int K = o.passes_together > 1
              ? std::min(o.passes_together, npasses)
              : (int)std::min<int64_t>(npasses, kReplicaArcs / std::max<int64_t>(g->m, 1));
  if (K < 2) return 1;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  const int64_t csr = (g->n + 1) * 8 + g->m * 4;
  // in/out CSR, sliced-ELL and piece lists, and a one-word workspace
  const int64_t per_copy = csr * (g->directed ? 2 : 1) + g->m * 5 + g->n * 64;
  while (K > 1 && ((int64_t)K * per_copy > (int64_t)(fr / 4) || (int64_t)K * g->n > kMaxNodes ||
                   (int64_t)K * g->m > kMaxArcs))
    --K;
  return K;
}

// PROPAGATE-S passes per propagation as words of one signature (see
// pg_options.pass_words): the requested number, else all of them, as far as
// a quarter of the free device memory holds the signatures (four buffers of
// n x words x 8 bytes).
static int pass_words_for(const pg_graph *g, int npasses, int planes, const pg_options &o) {
  if (planes != 64 || npasses < 2 || o.pass_words == 1 || o.passes_together > 1) return 1;
  int K = o.pass_words > 1 ? std::min(o.pass_words, npasses) : npasses;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  while (K > 1 && 4 * g->n * (int64_t)K * 8 > (int64_t)(fr / 4)) K /= 2;
  return K;
}

static pg_status check_seeds(const pg_graph *g, const int32_t *seeds, int32_t s) {
  if (!seeds || s < 1 || s > g->n) return PG_EINVAL;
  std::vector<int32_t> v(seeds, seeds + s);
  for (int32_t x : v)
    if (x < 0 || x >= g->n) return PG_EINVAL;
  std::sort(v.begin(), v.end());
  for (int32_t i = 1; i < s; ++i)
    if (v[i] == v[i - 1]) return PG_EINVAL;
  return PG_OK;
}

static pg_status propagate(pg_graph *g, const int32_t *seeds, int32_t s, pg_counts *out,
                           const pg_options *opt, void *stream, bool s_mode) {
  if (!g || !out || !out->counts || out->s != s || out->max_rounds < 0) return PG_EINVAL;
  std::lock_guard<std::mutex> lk(g->mu);
  pg_status rc = check_seeds(g, seeds, s);
  if (rc) return rc;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != g->device) return PG_EINVAL;
  Call cl;
  cl.g = g;
  cl.st = (cudaStream_t)stream;
  pg_default_options(&cl.o);
  if (opt) cl.o = *opt;
  if (cl.o.direction < 0 || cl.o.direction > 2) return PG_EINVAL;
  if (cl.o.pass_words < 0 || cl.o.test_changed < 0 || cl.o.test_changed > 3 ||
      cl.o.tma_gather < 0 || cl.o.tma_gather > 2 || cl.o.sparse_push < 0 ||
      cl.o.sparse_push > 2)
    return PG_EINVAL;
  cl.s_total = s;
  cl.max_rounds = out->max_rounds;
  cl.counts_h = out->counts;
  cl.perm = g->perm_ptr;
  cl.perm_n = g->n;
  const int planes =
      s_mode ? (cl.o.planes_per_pass > 0 ? std::min(cl.o.planes_per_pass, 64) : 64) : s;
  const int npasses = (s + planes - 1) / planes;
  // PROPAGATE-S: passes as signature words where they can be, else copies
  const int KW = s_mode ? pass_words_for(g, npasses, planes, cl.o) : 1;
  const int K = s_mode && KW <= 1 ? passes_together(g, npasses, cl.o) : 1;
  const int step = KW > 1 ? 64 * KW : planes;  // seeds per propagation
  const int widest = std::min(step, s);
  // counts window: up to max_rounds+1 rows, at most ~256 MB of counters
  int64_t cap_rows = std::max<int64_t>(64, (256LL << 20) / (4LL * widest));
  if (cl.o.window_rows > 0) cap_rows = cl.o.window_rows;
  cl.row_cap = (int32_t)std::min<int64_t>((int64_t)out->max_rounds + 1, cap_rows);
  if (cl.row_cap < 1) cl.row_cap = 1;
  pg_stats st{};
  int32_t T = 0, status = PG_OK;
  int passes = 0;
  int &hint = s_mode ? g->hint_s : g->hint_p;
  if (K > 1) {
    // PROPAGATE-S passes K at a time, as one propagation over K copies of the
    // graph: pass k's planes live in copy k (its seeds shifted by k*n), its
    // counts in columns k*planes.. of the group; copies never exchange bits
    if ((rc = make_replicas(g, K, cl.st))) return rc;
    pg_graph *r = g->rep;
    if ((rc = ensure(g->rep_graph_s, sizeof(int32_t) * K)) ||
        (rc = ensure(g->rep_graph_col0, sizeof(int32_t) * K)))
      return rc;
    for (int b0 = 0; b0 < s; b0 += K * planes) {
      const int ns = std::min(K * planes, s - b0);
      std::vector<int32_t> rs(ns), bit(ns), gs(K, 1), gc(K, 0);
      std::vector<int64_t> gm(K, g->m);
      for (int i = 0; i < ns; ++i) {
        const int k = i / planes;
        rs[i] = seeds[b0 + i] + (int32_t)((int64_t)k * g->n);
        bit[i] = i - k * planes;
        gs[k] = std::min(planes, ns - k * planes);
        gc[k] = k * planes;
      }
      if ((rc = cuda_status(cudaMemcpyAsync(g->rep_graph_s.p, gs.data(), sizeof(int32_t) * K,
                                            cudaMemcpyHostToDevice, cl.st))) ||
          (rc = cuda_status(cudaMemcpyAsync(g->rep_graph_col0.p, gc.data(), sizeof(int32_t) * K,
                                            cudaMemcpyHostToDevice, cl.st))))
        return rc;
      Call cr;
      cr.g = r;
      cr.st = cl.st;
      cr.o = cl.o;
      cr.s_total = s;
      cr.max_rounds = cl.max_rounds;
      cr.counts_h = cl.counts_h;
      cr.perm = cl.perm;
      cr.perm_n = cl.perm_n;
      int64_t rows = std::max<int64_t>(64, (256LL << 20) / (4LL * ns));
      if (cl.o.window_rows > 0) rows = cl.o.window_rows;
      cr.row_cap = (int32_t)std::max<int64_t>(1, std::min<int64_t>((int64_t)out->max_rounds + 1, rows));
      BatchSeg bs{(const int32_t *)g->rep_graph_of.p, (const int32_t *)g->rep_graph_s.p,
                  (const int32_t *)g->rep_graph_col0.p, bit.data(), ns, planes, gm.data()};
      PassOut po;
      rc = run_pass(cr, rs.data(), ns, b0, true, r->hint_s, po, &bs);
      if (rc == PG_OK && po.status == PG_OK) r->hint_s = std::min(po.rounds + 1, 64);
      if (rc) {
        cudaGetLastError();
        return rc;
      }
      passes += (ns + planes - 1) / planes;
      if (cl.rs_h.size() < cr.rs_h.size()) cl.rs_h.resize(cr.rs_h.size(), RoundStats{});
      for (size_t t = 0; t < cr.rs_h.size(); ++t) {
        RoundStats &d = cl.rs_h[t];
        const RoundStats &x = cr.rs_h[t];
        d.work += x.work;
        d.m_active += x.m_active;
        d.scanned += x.scanned;
        d.gathered += x.gathered;
        d.items += x.items;
        d.changed += x.changed;
        d.fsum += x.fsum;
        d.rows += x.rows;
      }
      // rows that only some groups reached: the others' columns are zero there
      if (po.rounds < T) {
        for (int32_t t = po.rounds + 1; t <= std::min(T, out->max_rounds); ++t)
          std::memset(out->counts + (size_t)t * s + b0, 0, sizeof(uint32_t) * ns);
      } else if (po.rounds > T && b0 > 0) {
        for (int32_t t = T + 1; t <= std::min(po.rounds, out->max_rounds); ++t)
          std::memset(out->counts + (size_t)t * s, 0, sizeof(uint32_t) * b0);
      }
      T = std::max(T, po.rounds);
      if (po.status == PG_ERANGE) status = PG_ERANGE;
      st.dense_rounds += po.dense_rounds;
      st.launches += po.launches;
      st.ms_pull += po.ms_pull;
      st.ms_post += po.ms_post;
      st.ms_init += po.ms_init;
      st.pull_launches += po.pull_launches;
      st.post_launches += po.post_launches;
    }
  }
  for (int b = 0; K <= 1 && b < s; b += step) {
    const int sp = std::min(step, s - b);
    PassOut po;
    rc = run_pass(cl, seeds + b, sp, b, s_mode && KW <= 1, hint, po, nullptr, KW > 1);
    if (rc == PG_OK && po.status == PG_OK) hint = std::min(po.rounds + 1, 64);
    if (rc) {
      cudaGetLastError();
      return rc;
    }
    passes += KW > 1 ? (sp + 63) / 64 : 1;
    // rows that only some passes reached: the others' columns are zero there
    if (po.rounds < T) {
      for (int32_t t = po.rounds + 1; t <= std::min(T, out->max_rounds); ++t)
        std::memset(out->counts + (size_t)t * s + b, 0, sizeof(uint32_t) * sp);
    } else if (po.rounds > T && b > 0) {
      for (int32_t t = T + 1; t <= std::min(po.rounds, out->max_rounds); ++t)
        std::memset(out->counts + (size_t)t * s, 0, sizeof(uint32_t) * b);
    }
    T = std::max(T, po.rounds);
    if (po.status == PG_ERANGE) status = PG_ERANGE;
    st.dense_rounds += po.dense_rounds;
    st.launches += po.launches;
    st.ms_pull += po.ms_pull;
    st.ms_post += po.ms_post;
    st.ms_init += po.ms_init;
    st.pull_launches += po.pull_launches;
    st.post_launches += po.post_launches;
    st.dense_tma |= po.tma ? 1 : 0;
  }
  out->rounds = T;
  const int32_t last_stats = std::min(T + 1, out->max_rounds + 1);
  if (cl.rs_h.size() < (size_t)last_stats + 1) cl.rs_h.resize((size_t)last_stats + 1, RoundStats{});
  if (out->m_active)
    for (int32_t t = 0; t <= last_stats; ++t) out->m_active[t] = cl.rs_h[t].m_active;
  for (int32_t t = 0; t <= last_stats; ++t) {
    const RoundStats &r = cl.rs_h[t];
    st.m_active_total += r.m_active;
    st.seed_edge_traversals += r.work;
    st.arcs_scanned += r.scanned;
    st.rows_gathered += r.gathered;
    st.items += r.items;
    st.changed_rows += r.changed;
    st.frontier_arcs += r.fsum;
    st.active_rows += r.rows;
  }
  st.sweeps = T + 1;
  st.passes = passes;
  Plan pl;
  make_plan(g, widest, cl.o, s_mode && KW <= 1, pl);
  st.words_per_row = pl.Wp;
  st.group_lanes = pl.G;
  st.pass_words = KW;
  st.words_per_gather = pl.wide ? 0 : pl.CW;
  st.test_changed = cl.o.test_changed == 1 || cl.o.test_changed == 3 ||
                    (cl.o.test_changed == 0 && g->n * (int64_t)pl.Wp * 8 > (64LL << 20));
  g->last = st;
  return status == PG_ERANGE ? PG_ERANGE : PG_OK;
}

// One PROPAGATE-P pass whose counts windows go to a sink: the seeds of a
// packed batch (bs set) or of several requests merged on one graph (seed i
// owns bit and column i; a node may carry several bits).
// mact (optional): m_active by round, rows 0..rounds+1, one column per graph
// of a packed batch (else one column).
static pg_status propagate_sink(pg_graph *g, const int32_t *seeds, int32_t nseeds,
                                const BatchSeg *bs, int32_t max_rounds, WindowSink sink,
                                void *sink_ctx, int32_t *rounds, const pg_options *opt,
                                void *stream, pg_stats *st_out,
                                std::vector<unsigned long long> *mact) {
  const int32_t ncols = bs ? bs->ncols : nseeds;
  if (!g || !seeds || nseeds < 1 || ncols < 1 || max_rounds < 0 || !sink || !rounds)
    return PG_EINVAL;
  for (int32_t i = 0; i < nseeds; ++i)
    if (seeds[i] < 0 || seeds[i] >= g->n) return PG_EINVAL;
  std::lock_guard<std::mutex> lk(g->mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != g->device) return PG_EINVAL;
  Call cl;
  cl.g = g;
  cl.st = (cudaStream_t)stream;
  pg_default_options(&cl.o);
  if (opt) cl.o = *opt;
  if (cl.o.direction < 0 || cl.o.direction > 2) return PG_EINVAL;
  if (cl.o.pass_words < 0) return PG_EINVAL;
  cl.s_total = ncols;
  cl.max_rounds = max_rounds;
  cl.counts_h = nullptr;
  cl.sink = sink;
  cl.sink_ctx = sink_ctx;
  cl.perm = g->perm_ptr;
  cl.perm_n = g->n;
  int64_t cap_rows = std::max<int64_t>(64, (256LL << 20) / (4LL * ncols));
  if (cl.o.window_rows > 0) cap_rows = cl.o.window_rows;
  cl.row_cap = (int32_t)std::max<int64_t>(1, std::min<int64_t>((int64_t)max_rounds + 1, cap_rows));
  // each graph's m_active of a packed batch comes from the kernels' window
  const bool per_graph = mact && bs && bs->graph_m && g->nseg > 0;
  std::vector<unsigned long long> gm;
  if (per_graph) cl.gm_h = &gm;
  PassOut po;
  pg_status rc = run_pass(cl, seeds, nseeds, 0, false, g->hint_p, po, bs);
  if (rc) {
    cudaGetLastError();
    return rc;
  }
  if (po.status == PG_OK) g->hint_p = std::min(po.rounds + 1, 64);
  *rounds = po.rounds;
  pg_stats st{};
  const int32_t last_stats = std::min(po.rounds + 1, max_rounds + 1);
  if (cl.rs_h.size() < (size_t)last_stats + 1) cl.rs_h.resize((size_t)last_stats + 1, RoundStats{});
  if (per_graph) {
    const size_t cols = (size_t)g->nseg;
    gm.resize(((size_t)last_stats + 1) * cols, 0ULL);
    mact->assign(gm.begin(), gm.begin() + ((size_t)last_stats + 1) * cols);
  } else if (mact) {
    mact->resize((size_t)last_stats + 1);
    for (int32_t t = 0; t <= last_stats; ++t) (*mact)[t] = cl.rs_h[t].m_active;
  }
  for (int32_t t = 0; t <= last_stats; ++t) {
    const RoundStats &r = cl.rs_h[t];
    st.m_active_total += r.m_active;
    st.seed_edge_traversals += r.work;
    st.arcs_scanned += r.scanned;
    st.rows_gathered += r.gathered;
    st.items += r.items;
    st.changed_rows += r.changed;
    st.frontier_arcs += r.fsum;
    st.active_rows += r.rows;
  }
  st.sweeps = po.rounds + 1;
  st.passes = 1;
  st.launches = po.launches;
  st.dense_rounds = po.dense_rounds;
  st.ms_pull = po.ms_pull;
  st.ms_post = po.ms_post;
  st.ms_init = po.ms_init;
  st.pull_launches = po.pull_launches;
  st.post_launches = po.post_launches;
  {
    Plan pl;
    if (make_plan(g, bs ? bs->s_bits : nseeds, cl.o, false, pl) == PG_OK) {
      st.words_per_row = pl.Wp;
      st.group_lanes = pl.G;
      st.pass_words = 1;
      st.words_per_gather = pl.wide ? 0 : pl.CW;
    }
  }
  st.test_changed = cl.o.test_changed == 1 || cl.o.test_changed == 3 ||
                    (cl.o.test_changed == 0 && g->n * (int64_t)st.words_per_row * 8 > (64LL << 20));
  g->last = st;
  if (st_out) *st_out = st;
  return po.status == PG_ERANGE ? PG_ERANGE : PG_OK;
}

pg_status propagate_batch_group(pg_graph *g, const int32_t *seeds, const int32_t *seed_bit,
                                int32_t nseeds, const int32_t *node_graph_d,
                                const int32_t *graph_s_d, const int32_t *graph_col0_d,
                                const int64_t *graph_m, int32_t ncols, int32_t s_bits,
                                int32_t max_rounds, WindowSink sink, void *sink_ctx,
                                int32_t *rounds, const pg_options *opt, void *stream,
                                pg_stats *st_out, std::vector<unsigned long long> *mact) {
  if (!seed_bit || !node_graph_d || !graph_s_d || !graph_col0_d || s_bits < 1) return PG_EINVAL;
  BatchSeg bs{node_graph_d, graph_s_d, graph_col0_d, seed_bit, ncols, s_bits, graph_m};
  return propagate_sink(g, seeds, nseeds, &bs, max_rounds, sink, sink_ctx, rounds, opt, stream,
                        st_out, mact);
}

int64_t workspace_bytes(const pg_graph *g, int32_t s, int32_t max_rounds, int32_t window_rows) {
  return workspace_bytes_nm(g->n, g->m, s, max_rounds, window_rows);
}

int64_t workspace_bytes_nm(int64_t n, int64_t m, int32_t s, int32_t max_rounds,
                           int32_t window_rows) {
  // the buffers run_pass ensures, sized for the widest plan of s seeds
  const int W = (s + 63) / 64;
  const int CW = W <= 1 ? 1 : W <= 2 ? 2 : W <= 4 ? 4 : 8;
  const int64_t Wp = (W + CW - 1) / CW * CW;
  const int64_t nbm = (n + 31) / 32;
  const int64_t pieces = n + m / 2 + 1;  // pieces hold at least 2 arcs
  const int64_t cap_rows =
      window_rows > 0 ? window_rows : std::max<int64_t>(64, (256LL << 20) / (4LL * s));
  const int64_t row_cap = std::max<int64_t>(1, std::min<int64_t>((int64_t)max_rounds + 1, cap_rows));
  // the frontier's out-arc pieces, twice for push rounds (rows of <= 8 words)
  const int64_t e_bufs = W <= 8 ? 2 : 1;
  return 4 * n * Wp * 8 + (5 + 2 * Wp) * nbm * 4 + 3 * n * 4 +
         e_bufs * (n + m / kExpandArcs + 1) * 8 + pieces * 16 + row_cap * s * 4 + (row_cap + 2) * (int64_t)sizeof(RoundStats) +
         (int64_t)s * 8 + 4096;
}

pg_status propagate_columns(pg_graph *g, const int32_t *seeds, int32_t nseeds, int32_t max_rounds,
                            WindowSink sink, void *sink_ctx, int32_t *rounds,
                            const pg_options *opt, void *stream, pg_stats *st_out,
                            std::vector<unsigned long long> *mact) {
  return propagate_sink(g, seeds, nseeds, nullptr, max_rounds, sink, sink_ctx, rounds, opt,
                        stream, st_out, mact);
}

}  // namespace pg

using namespace pg;

extern "C" {

void pg_default_options(pg_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->direction = PG_DIR_AUTO;
  o->dense_threshold = 0.05f;
  o->group_lanes = 0;
  o->test_changed = 0;
  o->planes_per_pass = 64;
  o->use_graphs = 1;
  o->timing = 0;
  o->window_rows = 0;
  o->words_per_thread = 0;
  o->wide_rows = 0;
  o->passes_together = 0;
  o->pass_words = 0;
  o->tma_gather = 0;
  o->sparse_push = 0;
}

pg_status pg_propagate_p(pg_graph *g, const int32_t *seeds, int32_t s, pg_counts *out,
                         const pg_options *opt, void *stream) {
  return propagate(g, seeds, s, out, opt, stream, false);
}

pg_status pg_propagate_s(pg_graph *g, const int32_t *seeds, int32_t s, pg_counts *out,
                         const pg_options *opt, void *stream) {
  return propagate(g, seeds, s, out, opt, stream, true);
}

pg_status pg_last_stats(const pg_graph *g, pg_stats *out) {
  if (!g || !out) return PG_EINVAL;
  *out = g->last;
  return PG_OK;
}

}  // extern "C"
