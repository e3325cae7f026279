// PROPAGATE-P and PROPAGATE-S drivers: seed initialisation (Alg. 1 lines
// setting Sig(x_i)[i] = 1; Alg. 2 per-seed plane set-up), the post kernel of
// every round (collision count, buffer sync, next work list, fixpoint test)
// and the host round loop.
#include <algorithm>
#include <cstring>
#include <vector>

#include "kernels.cuh"

namespace pg {

constexpr int32_t kStatusWindow = 100;  // device asks the host to move the counts window
constexpr int kSmemCountMax = 12288;    // per-seed counters kept in shared memory up to this s

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
  for (int64_t i = gtid; i < pairs; i += nth) {
    x2[i] = z;
    y2[i] = z;
  }
  if ((words & 1) && gtid == 0) {
    p.X[words - 1] = 0ULL;
    p.Y[words - 1] = 0ULL;
  }
  for (int64_t i = gtid; i < p.nbm; i += nth) {
    p.C0[i] = 0u;
    p.C1[i] = 0u;
    p.K0[i] = 0u;
    p.K1[i] = 0u;
    p.Sat[i] = 0u;
  }
  for (int64_t i = gtid; i < count_words; i += nth) p.counts[i] = 0u;
  unsigned long long *rsw = reinterpret_cast<unsigned long long *>(p.rs);
  for (int64_t i = gtid; i < rs_words; i += nth) rsw[i] = 0ULL;
  if (gtid == 0) {
    Ctrl *c = p.ctrl;
    c->t = 0;
    c->done = 0;
    c->status = 0;
    c->mode = kModeSparse;
    c->fpack = 0ULL;
    c->nA = 0ULL;
    c->nA_next = 0ULL;
    c->blocks_done = 0u;
    c->last_round = 0;
    c->dense_rounds = 0;
    c->row_base = 0;
  }
}

// ------------------------------------------------------------- k_seed
// One block. Seed i of the pass gets bit i (Sig(x_i)[i] = 1) in both buffers;
// round 0's frontier F_0 is the seed set, with its out-arc prefix; count row
// 0 is one pair (x_i, x_i) per seed.
__global__ void __launch_bounds__(1024) k_seed(Params p, const int32_t *seeds, int sp) {
  __shared__ unsigned long long wtot[32];
  __shared__ unsigned long long carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) carry = 0ULL;
  __syncthreads();
  for (int base = 0; base < sp; base += blockDim.x) {
    const int i = base + threadIdx.x;
    unsigned long long od = 0;
    int32_t x = 0;
    if (i < sp) {
      x = seeds[i];
      const uint64_t bit = 1ULL << (i & 63);
      p.X[(size_t)x * p.Wp + (i >> 6)] = bit;
      p.Y[(size_t)x * p.Wp + (i >> 6)] = bit;
      set_bit(p.C0, x);
      p.counts[i] = 1u;
      od = (unsigned long long)(p.out_ptr[x + 1] - p.out_ptr[x]);
    }
    unsigned long long incl = od;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFullMask, incl, off);
      if (lane >= off) incl += y;
    }
    if (lane == 31) wtot[w] = incl;
    __syncthreads();
    if (w == 0) {
      unsigned long long t = lane < nw ? wtot[lane] : 0ULL, ti = t;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFullMask, ti, off);
        if (lane >= off) ti += y;
      }
      if (lane < nw) wtot[lane] = ti - t;
    }
    __syncthreads();
    if (i < sp) {
      p.F[i] = x;
      p.Fpre[i] = (int64_t)(carry + wtot[w] + incl - od);
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += wtot[w] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) p.ctrl->fpack = ((unsigned long long)sp << kFsumBits) | carry;
}

__device__ __forceinline__ int64_t upper_bound_i64(const int64_t *a, int64_t lo, int64_t hi,
                                                   int64_t key) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) <= key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool row_full(const uint64_t *row, int Wp, int s) {
  bool full = true;
  for (int w = 0; w < Wp; ++w) full &= ((__ldg(reinterpret_cast<const unsigned long long *>(row) + w) | ~valid_mask(w, s)) == ~0ULL);
  return full;
}

// ------------------------------------------------------------- k_post
// Round t, after the pull:
//  A. for v in F_t: d = X[v] ^ Y[v]; per seed i add bit i of d into the
//     count of round t (Alg. 1: Count += ||Sig_next(u) XOR Sig(u)||, kept per
//     seed); X[v] = Y[v] (Alg. 1: Sig(u) = Sig_next(u)); mark v saturated when
//     all its s bits are set (skip rule, proof of Thm. 1).
//  B. choose the direction of round t+1 from the frontier's out-arc count;
//     if sparse, claim every unsaturated out-neighbour of F_t and list its
//     pieces (the rows round t+1 must revisit), adding its in-degree to
//     m_active[t+1].
//  C. last block: fixpoint test (Alg. 1: do ... while Count > 0) and the
//     hand-over to round t+1.
template <bool SMEM>
__global__ void __launch_bounds__(kBlock) k_post(Params p) {
  extern __shared__ uint32_t scnt[];
  Ctrl *ctrl = p.ctrl;
  if (*(volatile int32_t *)&ctrl->done) return;
  const int t = ctrl->t;
  const int row = t - ctrl->row_base;  // row of round t in the counts window
  const unsigned long long fpack = ctrl->fpack;
  const int64_t nF = (int64_t)(fpack >> kFsumBits);
  const int64_t fsum = (int64_t)(fpack & kFsumMask);
  const uint32_t *Ccur = (t & 1) ? p.C1 : p.C0;
  uint32_t *Cnext = (t & 1) ? p.C0 : p.C1;
  uint32_t *Knext = (t & 1) ? p.K0 : p.K1;
  const int64_t gtid = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * kBlock;
  const int lane = threadIdx.x & 31;
  const int64_t warp = gtid >> 5, nwarps = nth >> 5;
  const int Wp = p.Wp, s = p.s;
  uint32_t *crow = p.counts + (size_t)row * (size_t)s;

  if (SMEM) {
    for (int i = threadIdx.x; i < s; i += kBlock) scnt[i] = 0u;
    __syncthreads();
  }
  // A. count, sync, saturation
  for (int64_t i = gtid; i < nF; i += nth) {
    const int32_t v = p.F[i];
    uint64_t *xr = p.X + (size_t)v * Wp;
    const uint64_t *yr = p.Y + (size_t)v * Wp;
    bool full = true;
    for (int w = 0; w < Wp; ++w) {
      const uint64_t o = xr[w], nw = __ldg(reinterpret_cast<const unsigned long long *>(yr) + w);
      full &= ((nw | ~valid_mask(w, s)) == ~0ULL);
      uint64_t d = o ^ nw;
      if (d) {
        xr[w] = nw;
        do {
          const int bit = __ffsll((long long)d) - 1;
          if (SMEM)
            atomicAdd(&scnt[w * 64 + bit], 1u);
          else
            atomicAdd(&crow[w * 64 + bit], 1u);
          d &= d - 1ULL;
        } while (d);
      }
    }
    if (full) set_bit(p.Sat, v);
  }
  if (SMEM) {
    __syncthreads();
    for (int i = threadIdx.x; i < s; i += kBlock) {
      const uint32_t c = scnt[i];
      if (c) atomicAdd(&crow[i], c);
    }
  }
  for (int64_t i = gtid; i < p.nbm; i += nth) Cnext[i] = 0u;

  // B. next direction and sparse work list
  const bool next_dense =
      p.direction == PG_DIR_DENSE ||
      (p.direction == PG_DIR_AUTO && (double)fsum > (double)p.dense_threshold * (double)p.m);
  const bool expand = !next_dense && nF > 0 && t + 1 <= p.max_rounds + 1;
  unsigned long long my_mact = 0;
  if (expand) {
    constexpr int kEPL = 4;
    constexpr int64_t kChunk = 32 * kEPL;
    for (int64_t c0 = warp * kChunk; c0 < fsum; c0 += nwarps * kChunk) {
      const int64_t c1 = min(fsum, c0 + kChunk);
      int64_t lo = 0, hi = 0;
      if (lane == 0) {
        lo = upper_bound_i64(p.Fpre, 0, nF, c0) - 1;
        hi = upper_bound_i64(p.Fpre, lo, nF, c1 - 1);
      }
      lo = __shfl_sync(kFullMask, lo, 0);
      hi = __shfl_sync(kFullMask, hi, 0);
#pragma unroll 1
      for (int k = 0; k < kEPL; ++k) {
        const int64_t e = c0 + k * 32 + lane;
        bool claim = false;
        int32_t x = 0;
        unsigned long long np = 0;
        if (e < c1) {
          const int64_t i = upper_bound_i64(p.Fpre, lo, hi, e) - 1;
          const int32_t u = __ldg(p.F + i);
          x = __ldg(p.out_col + __ldg(p.out_ptr + u) + (e - __ldg(p.Fpre + i)));
          if (!test_bit_live(p.Sat, x)) {
            const bool sat_now = test_bit(Ccur, x) && row_full(p.Y + (size_t)x * Wp, Wp, s);
            if (!sat_now && !set_bit(Knext, x)) {
              const int64_t indeg = __ldg(p.row_ptr + x + 1) - __ldg(p.row_ptr + x);
              my_mact += (unsigned long long)indeg;
              np = (unsigned long long)((indeg + p.L - 1) / p.L);
              claim = true;
            }
          }
        }
        const unsigned mask = __ballot_sync(kFullMask, claim);
        if (mask) {
          unsigned long long incl = np;
#pragma unroll
          for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFullMask, incl, off);
            if (lane >= off) incl += y;
          }
          const unsigned long long total = __shfl_sync(kFullMask, incl, 31);
          unsigned long long basep = 0;
          if (lane == 0) basep = atomicAdd(&ctrl->nA_next, total);
          basep = __shfl_sync(kFullMask, basep, 0);
          if (claim) {
            const unsigned long long at = basep + incl - np;
            for (unsigned long long q = 0; q < np; ++q)
              p.A[at + q] = ((unsigned long long)(uint32_t)x << 32) | q;
          }
        }
      }
    }
  }
  RoundStats *rnext = p.rs + row + 1;
  block_add4(my_mact, 0ULL, 0ULL, 0ULL, &rnext->m_active, nullptr, nullptr, nullptr);

  // C. last block hands over
  __shared__ int am_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    am_last = atomicAdd(&ctrl->blocks_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (am_last && threadIdx.x == 0) {
    __threadfence();
    RoundStats *r = p.rs + row;
    r->changed = (unsigned long long)nF;
    r->fsum = (unsigned long long)fsum;
    if (nF == 0) {
      ctrl->last_round = t - 1;
      ctrl->done = 1;
    } else if (t >= p.max_rounds + 1) {
      ctrl->last_round = t;
      ctrl->status = PG_ERANGE;
      ctrl->done = 1;
    } else {
      ctrl->t = t + 1;
      ctrl->mode = next_dense ? kModeDense : kModeSparse;
      if (next_dense) ctrl->dense_rounds += 1;
      ctrl->nA = *(volatile unsigned long long *)&ctrl->nA_next;
      ctrl->nA_next = 0ULL;
      ctrl->fpack = 0ULL;
      if (t + 1 - ctrl->row_base >= p.row_cap) {
        ctrl->status = kStatusWindow;
        ctrl->done = 1;
      }
    }
    ctrl->blocks_done = 0u;
    __threadfence();
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
  if (gtid == 0) {
    p.ctrl->row_base += p.row_cap;
    p.ctrl->status = 0;
    p.ctrl->done = 0;
  }
}

// ---------------------------------------------------------------- host side
struct Plan {
  int CW = 1, G = 8, L = 32, Wp = 1;
  bool chg = true, eb = false;
  PullFn pull = nullptr;
  int grid_pull = 1, grid_post = 1;
  size_t post_smem = 0;
  bool smem_counts = true;
};

static PullFn pick_pull(int CW, int G, bool chg, bool eb) {
  switch (CW) {
    case 1: return pull_fn_cw1(G, chg, eb);
    case 2: return pull_fn_cw2(G, chg, eb);
    case 4: return pull_fn_cw4(G, chg, eb);
    case 8: return pull_fn_cw8(G, chg, eb);
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

static pg_status make_plan(const pg_graph *g, int sp, const pg_options &o, bool eb, Plan &pl) {
  const int W = eb ? 1 : (sp + 63) / 64;
  pl.CW = W <= 1 ? 1 : W <= 2 ? 2 : W <= 4 ? 4 : 8;
  pl.Wp = (W + pl.CW - 1) / pl.CW * pl.CW;
  int G = o.group_lanes;
  if (G <= 0) {
    const double d = g->mean_degree;
    G = d <= 6 ? 4 : d <= 12 ? 8 : d <= 40 ? 16 : 32;
  }
  if (G < 2) G = 2;
  if (G > 32 || (G & (G - 1))) return PG_EINVAL;
  pl.G = G;
  pl.L = o.piece_arcs > 0 ? o.piece_arcs : 4 * G;
  if (pl.L < 1) return PG_EINVAL;
  pl.chg = o.gather_changed_only != 0;
  pl.eb = eb;
  pl.pull = pick_pull(pl.CW, pl.G, pl.chg, pl.eb);
  if (!pl.pull) return PG_EINVAL;
  pl.smem_counts = sp <= kSmemCountMax;
  pl.post_smem = pl.smem_counts ? sizeof(uint32_t) * (size_t)sp : 0;
  return PG_OK;
}

static const void *post_fn(const Plan &pl) {
  return pl.smem_counts ? (const void *)&k_post<true> : (const void *)&k_post<false>;
}

static void launch_round(const Plan &pl, const Params &p, cudaStream_t st) {
  pl.pull<<<pl.grid_pull, kBlock, 0, st>>>(p);
  if (pl.smem_counts)
    k_post<true><<<pl.grid_post, kBlock, pl.post_smem, st>>>(p);
  else
    k_post<false><<<pl.grid_post, kBlock, 0, st>>>(p);
}

struct PassOut {
  int32_t rounds = 0;
  int32_t status = 0;
  int32_t dense_rounds = 0;
  int32_t launches = 0;
  double ms_pull = 0, ms_post = 0, ms_init = 0;
  int32_t pull_launches = 0, post_launches = 0;
};

struct Call {
  pg_graph *g;
  cudaStream_t st;
  pg_options o;
  int32_t s_total;
  int32_t max_rounds;
  uint32_t *counts_h;                 // caller rows x s_total
  std::vector<RoundStats> rs_h;       // summed over passes, rows 0..max_rounds+1
  int32_t row_cap = 0;
};

static pg_status copy_window(Call &cl, const Params &p, int col0, int32_t row_base, int32_t rows,
                             int32_t rs_rows) {
  // counts rows [row_base, row_base+rows) of this pass's columns
  rows = std::min(rows, cl.max_rounds + 1 - row_base);
  if (rows > 0) {
    cudaError_t e = cudaMemcpy2DAsync(cl.counts_h + (size_t)row_base * cl.s_total + col0,
                                      sizeof(uint32_t) * cl.s_total, p.counts,
                                      sizeof(uint32_t) * p.s, sizeof(uint32_t) * p.s, rows,
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
    for (int i = 0; i < rs_rows; ++i) {
      RoundStats &d = cl.rs_h[row_base + i];
      d.m_active += tmp[i].m_active;
      d.scanned += tmp[i].scanned;
      d.gathered += tmp[i].gathered;
      d.items += tmp[i].items;
      d.changed += tmp[i].changed;
      d.fsum += tmp[i].fsum;
    }
  }
  return cuda_status(cudaStreamSynchronize(cl.st));
}

static pg_status ensure_capture(pg_graph *g, const Plan &pl, const Params &p, int K,
                                cudaGraphExec_t *out);

// One pass: sp seeds of the call, columns [col0, col0+sp).
static pg_status run_pass(Call &cl, const int32_t *seeds_h, int sp, int col0, bool eb,
                          PassOut &po) {
  pg_graph *g = cl.g;
  Workspace &w = g->ws;
  cudaStream_t st = cl.st;
  Plan pl;
  pg_status rc = make_plan(g, sp, cl.o, eb, pl);
  if (rc) return rc;
  rc = ensure_pieces(g, pl.L, st);
  if (rc) return rc;
  const int64_t n = g->n;
  const int64_t nbm = (n + 31) / 32;
  const int32_t row_cap = cl.row_cap;
  size_t sig_bytes = sizeof(uint64_t) * (size_t)n * pl.Wp;
  if ((rc = ensure(w.X, sig_bytes)) || (rc = ensure(w.Y, sig_bytes))) return rc;
  for (DevBuf *b : {&w.C0, &w.C1, &w.K0, &w.K1, &w.Sat})
    if ((rc = ensure(*b, sizeof(uint32_t) * nbm))) return rc;
  if ((rc = ensure(w.F, sizeof(int32_t) * n)) || (rc = ensure(w.Fpre, sizeof(int64_t) * n)) ||
      (rc = ensure(w.A, sizeof(unsigned long long) * std::max<int64_t>(g->pieces.count, 1))) ||
      (rc = ensure(w.counts, sizeof(uint32_t) * (size_t)row_cap * sp)) ||
      (rc = ensure(w.rs, sizeof(RoundStats) * (size_t)(row_cap + 2))) ||
      (rc = ensure(w.ctrl, sizeof(Ctrl))) || (rc = ensure(w.seeds, sizeof(int32_t) * sp)))
    return rc;
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
  p.Wp = pl.Wp;
  p.s = sp;
  p.C0 = (uint32_t *)w.C0.p;
  p.C1 = (uint32_t *)w.C1.p;
  p.K0 = (uint32_t *)w.K0.p;
  p.K1 = (uint32_t *)w.K1.p;
  p.Sat = (uint32_t *)w.Sat.p;
  p.nbm = nbm;
  p.F = (int32_t *)w.F.p;
  p.Fpre = (int64_t *)w.Fpre.p;
  p.A = (unsigned long long *)w.A.p;
  p.Pall = (const unsigned long long *)g->pieces.list.p;
  p.nPall = g->pieces.count;
  p.L = pl.L;
  p.counts = (uint32_t *)w.counts.p;
  p.rs = (RoundStats *)w.rs.p;
  p.ctrl = (Ctrl *)w.ctrl.p;
  p.max_rounds = cl.max_rounds;
  p.row_cap = row_cap;
  p.direction = cl.o.direction;
  p.dense_threshold = cl.o.dense_threshold > 0 ? cl.o.dense_threshold : 0.05f;

  // grids
  const int64_t pull_threads = std::max<int64_t>(p.nPall * pl.G, nbm);
  pl.grid_pull = occupancy_grid((const void *)pl.pull, 0, pull_threads);
  pl.grid_post = occupancy_grid(post_fn(pl), pl.post_smem, std::max<int64_t>(n, nbm));
  if (pl.post_smem > 48 * 1024)
    cudaFuncSetAttribute(post_fn(pl), cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)pl.post_smem);

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
  if (rc) return rc;
  const int64_t count_words = (int64_t)row_cap * sp;
  const int64_t rs_words = (int64_t)(row_cap + 2) * (int64_t)(sizeof(RoundStats) / 8);
  const int64_t zero_work = std::max<int64_t>({n * pl.Wp / 2, nbm, count_words, rs_words, 1});
  k_zero<<<occupancy_grid((const void *)&k_zero, 0, zero_work), kBlock, 0, st>>>(p, count_words,
                                                                                rs_words);
  k_seed<<<1, 1024, 0, st>>>(p, (const int32_t *)w.seeds.p, sp);
  if (pl.smem_counts)
    k_post<true><<<pl.grid_post, kBlock, pl.post_smem, st>>>(p);
  else
    k_post<false><<<pl.grid_post, kBlock, 0, st>>>(p);
  po.launches += 3;
  if (timing) {
    init_ev1 = ntev++;
    cudaEventRecord(tev(init_ev1), st);
  }
  if ((rc = cuda_status(cudaGetLastError()))) return rc;

  // round loop: batches of K rounds, the host reads the control block of the
  // batch before last while the last one runs.
  constexpr int kGraphRounds = 16;
  int K = 2;
  int slot = 0;
  int pending[2];
  int npending = 0;
  int64_t enqueued = 0;
  int32_t row_base = 0;
  const int64_t guard = (int64_t)cl.max_rounds + 4 + 4 * kGraphRounds;
  Ctrl fin{};
  bool finished = false;
  cudaGraphExec_t gexec = nullptr;
  while (!finished) {
    if (graphs && K >= kGraphRounds) {
      if (!gexec && (rc = ensure_capture(g, pl, p, kGraphRounds, &gexec))) return rc;
      if ((rc = cuda_status(cudaGraphLaunch(gexec, st)))) return rc;
      enqueued += kGraphRounds;
      po.launches += 2 * kGraphRounds;
    } else {
      for (int k = 0; k < K; ++k) {
        if (timing) {
          int a = ntev++, b = ntev++, c = ntev++;
          cudaEventRecord(tev(a), st);
          pl.pull<<<pl.grid_pull, kBlock, 0, st>>>(p);
          cudaEventRecord(tev(b), st);
          if (pl.smem_counts)
            k_post<true><<<pl.grid_post, kBlock, pl.post_smem, st>>>(p);
          else
            k_post<false><<<pl.grid_post, kBlock, 0, st>>>(p);
          cudaEventRecord(tev(c), st);
          pull_ev.push_back({a, b});
          post_ev.push_back({b, c});
        } else {
          launch_round(pl, p, st);
        }
      }
      enqueued += K;
      po.launches += 2 * K;
      if ((rc = cuda_status(cudaGetLastError()))) return rc;
    }
    cudaMemcpyAsync(&w.ctrl_h[slot], p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    cudaEventRecord(w.ev[slot], st);
    pending[npending++] = slot;
    slot ^= 1;
    K = std::min(K * 2, kGraphRounds);
    if (npending == 2 || enqueued > guard) {
      const int s0 = pending[0];
      if ((rc = cuda_status(cudaEventSynchronize(w.ev[s0])))) return rc;
      pending[0] = pending[1];
      npending--;
      Ctrl c = w.ctrl_h[s0];
      if (c.done) {
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) return rc;
        npending = 0;
        Ctrl cnow;
        if ((rc = cuda_status(cudaMemcpy(&cnow, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost))))
          return rc;
        if (cnow.status == kStatusWindow) {
          if ((rc = copy_window(cl, p, col0, row_base, row_cap, row_cap))) return rc;
          k_window_shift<<<occupancy_grid((const void *)&k_window_shift, 0, count_words), kBlock,
                           0, st>>>(p, count_words, row_cap + 2);
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
  // final window: rows row_base .. last_round (+1 for the stats of the empty sweep)
  const int32_t last = fin.status == PG_ERANGE ? cl.max_rounds : fin.last_round;
  const int32_t rows = last - row_base + 1;
  if ((rc = copy_window(cl, p, col0, row_base, rows, rows + 1))) return rc;
  po.rounds = fin.status == PG_ERANGE ? cl.max_rounds + 1 : fin.last_round;
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

// Captures K rounds (pull + post each) into a CUDA graph on a private stream;
// cached on the graph handle while the launch parameters stay the same.
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  Params p{};
  PullFn pull = nullptr;
  int grid_pull = 0, grid_post = 0, K = 0;
  size_t smem = 0;
  bool smem_counts = true;
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

static pg_status ensure_capture(pg_graph *g, const Plan &pl, const Params &p, int K,
                                cudaGraphExec_t *out) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  GraphCache &c = cache_for(g);
  if (c.exec && c.pull == pl.pull && c.grid_pull == pl.grid_pull && c.grid_post == pl.grid_post &&
      c.K == K && c.smem == pl.post_smem && c.smem_counts == pl.smem_counts &&
      std::memcmp(&c.p, &p, sizeof(Params)) == 0) {
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
  cudaError_t e = cudaStreamBeginCapture(c.cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e);
  for (int k = 0; k < K; ++k) launch_round(pl, p, c.cap);
  e = cudaStreamEndCapture(c.cap, &graph);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaGraphInstantiate(&c.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    c.exec = nullptr;
    return cuda_status(e);
  }
  c.p = p;
  c.pull = pl.pull;
  c.grid_pull = pl.grid_pull;
  c.grid_post = pl.grid_post;
  c.K = K;
  c.smem = pl.post_smem;
  c.smem_counts = pl.smem_counts;
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
  cl.s_total = s;
  cl.max_rounds = out->max_rounds;
  cl.counts_h = out->counts;
  cl.rs_h.assign((size_t)out->max_rounds + 2, RoundStats{});
  const int planes = s_mode ? (cl.o.planes_per_pass > 0 ? std::min(cl.o.planes_per_pass, 64) : 64) : s;
  const int widest = std::min(planes, s);
  // counts window: up to max_rounds+1 rows, at most ~256 MB of counters
  int64_t cap_rows = std::max<int64_t>(64, (256LL << 20) / (4LL * widest));
  if (cl.o.window_rows > 0) cap_rows = cl.o.window_rows;
  cl.row_cap = (int32_t)std::min<int64_t>((int64_t)out->max_rounds + 1, cap_rows);
  if (cl.row_cap < 1) cl.row_cap = 1;
  std::memset(out->counts, 0, sizeof(uint32_t) * ((size_t)out->max_rounds + 1) * s);
  pg_stats st{};
  int32_t T = 0, status = PG_OK;
  int passes = 0;
  for (int b = 0; b < s; b += planes) {
    const int sp = std::min(planes, s - b);
    PassOut po;
    rc = run_pass(cl, seeds + b, sp, b, s_mode, po);
    if (rc) {
      cudaGetLastError();
      return rc;
    }
    ++passes;
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
  out->rounds = T;
  const int32_t last_stats = std::min(T + 1, out->max_rounds + 1);
  if (out->m_active)
    for (int32_t t = 0; t <= out->max_rounds + 1; ++t)
      out->m_active[t] = t <= last_stats ? cl.rs_h[t].m_active : 0ULL;
  for (int32_t t = 0; t <= last_stats; ++t) {
    const RoundStats &r = cl.rs_h[t];
    st.m_active_total += r.m_active;
    st.arcs_scanned += r.scanned;
    st.rows_gathered += r.gathered;
    st.items += r.items;
    st.changed_rows += r.changed;
    st.frontier_arcs += r.fsum;
  }
  st.sweeps = T + 1;
  st.passes = passes;
  Plan pl;
  make_plan(g, std::min(planes, s), cl.o, s_mode, pl);
  st.words_per_row = pl.Wp;
  st.group_lanes = pl.G;
  g->last = st;
  return status == PG_ERANGE ? PG_ERANGE : PG_OK;
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
  o->piece_arcs = 0;
  o->gather_changed_only = 1;
  o->planes_per_pass = 64;
  o->use_graphs = 1;
  o->timing = 0;
  o->window_rows = 0;
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
