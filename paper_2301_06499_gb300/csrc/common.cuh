// Internal declarations of the PROPAGATE library shared by its kernels (not
// part of the C ABI): launch constants, the control block, round statistics
// and the parameter block of the round kernels. Host-side structures are in
// host.cuh.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "propagate.h"

namespace pg {

constexpr int kBlock = 256;
constexpr unsigned kFullMask = 0xFFFFFFFFu;

// Packed frontier append: count of rows in the high bits, running sum of
// their out-degrees in the low kFsumBits bits (one 64-bit atomic keeps the
// two consistent, so every frontier row gets its out-arc prefix).
constexpr int kFsumBits = 37;
constexpr unsigned long long kFsumMask = (1ULL << kFsumBits) - 1ULL;
// Size limits that follow: a round's frontier has at most n rows, counted in
// the 64 - kFsumBits high bits, and its out-arc sum is at most m.
constexpr int64_t kMaxNodes = (1LL << (64 - kFsumBits)) - 1;  // 134,217,727
constexpr int64_t kMaxArcs = (1LL << kFsumBits) - 1;

// kModeMixed (packed batches): each graph of the union picks its own kind
// of round from its own frontier (see Params::gfsum).
// kModePush: a sparse round pushed from the frontier of round t-1 along its
// out-arcs (atomic OR of each changed row's delta into its out-neighbours).
enum : int32_t { kModeDense = 0, kModeSparse = 1, kModeMixed = 2, kModePush = 3 };

// Device-side control block of one propagation (one pass).
struct Ctrl {
  int32_t t;            // round being executed
  int32_t done;         // 1 once the fixpoint (or an error) is reached
  int32_t status;       // pg_status of the device side
  int32_t mode;         // kModeDense / kModeSparse / kModeMixed for round t
  unsigned long long fpack;  // frontier F_t: (count << kFsumBits) | out-arc sum
  unsigned long long nA;     // pieces in the sparse work list of round t
  unsigned long long nA_next;
  unsigned long long nE;     // expansion pieces of F_t (out-arcs in pieces of LE)
  uint32_t blocks_done;  // last-block detection in the post kernel
  int32_t last_round;    // T once done
  int32_t dense_rounds;
  int32_t row_base;      // round held in row 0 of the device counts window
  int32_t iters;         // post launches of this pass (termination guard)
  int32_t ndense;        // packed batch: graphs swept whole in round t (in dlist)
  int32_t test;          // round t tests changed bits before gathers (per-round mode)
  int32_t bad_index;     // PG_DEBUG_BOUNDS builds: a gather's index was out of range
  unsigned long long nF_prev;  // |F_{t-1}|
  unsigned long long nE_prev;  // out-arc pieces of F_{t-1} (read by a push round)
};

// Per-round work counters (device), indexed by round.
struct RoundStats {
  unsigned long long work;     // sum over active rows of s_graph(v) * indeg(v)
  unsigned long long m_active;
  unsigned long long scanned;
  unsigned long long gathered;
  unsigned long long items;
  unsigned long long changed;
  unsigned long long fsum;
  unsigned long long rows;     // active rows |A_t| (PROPAGATE-S passes as words: row x pass)
};

// Everything the round kernels need, passed by value.
// Per-round test of changed bits: a round tests them while the previous
// round's frontier out-arcs are below this fraction of all arcs (a random
// bitmap sector then costs less than gathering the zero deltas of the
// in-neighbours that did not change).
constexpr double kTestDensity = 0.5;

struct Params {
  int64_t n, m;
  const int64_t *row_ptr;  // in-CSR
  const int32_t *col;
  const int64_t *out_ptr;  // out-CSR (== in-CSR for symmetric graphs)
  const int32_t *out_col;
  uint64_t *X;  // signatures of round t-1 (read by the pull)
  uint64_t *Y;  // signatures of round t (written by the pull)
  uint64_t *D0, *D1;  // deltas: D_{t&1}[v] = bits v gained in round t (0 if unchanged)
  int32_t Wp;   // words per row (padded)
  int32_t s;    // seeds in this pass (valid bits)
  uint32_t *C0, *C1;   // changed-in-round bitmaps, alternating by round parity
  uint32_t *K0, *K1;   // claim / active bitmaps, alternating
  uint32_t *Sat;       // saturated (all s bits set)
  uint32_t *rowbits;   // wide rows: set bits of each row so far (else null)
  // PROPAGATE-S passes as the words of one signature: m_active per pass, with
  // one claim bit per (word, row) for rows cut into pieces, by round parity
  int32_t pass_words;
  uint32_t *Kw0, *Kw1;  // [Wp][nbm] each (null unless pass_words)
  int64_t nbm;         // 32-bit words per bitmap
  int32_t *F0, *F1;    // rows changed in round t, by round parity
  unsigned long long *E;  // out-arc pieces of F rows: (row << 32) | piece of LE arcs
  unsigned long long *E1; // with push rounds: the pieces of odd rounds (E: even), else null
  ulonglong2 *A;        // sparse work list: in-arc pieces of the claimed rows
  const ulonglong2 *Pall;  // every in-arc piece of every row (unused by dense rounds)
  const ulonglong2 *sell_items;  // dense rounds: sliced-ELL copy (see SellList)
  const int32_t *sell_col;
  const int64_t *sell_off;
  const int32_t *sell_len;
  int64_t sell_chunks;
  int64_t nPall;
  int32_t L;            // in-arcs per work piece
  int32_t LE;           // out-arcs per expansion piece
  uint32_t *counts;     // counts window [row_cap][ncols] of this pass
  int32_t ncols;        // count columns per round (s, or the batch's sum of s_g)
  const int32_t *node_graph;  // batch of disjoint graphs: graph of each node (else null)
  const int32_t *graph_s;     // batch: seeds of each graph
  const int32_t *graph_col0;  // batch: first count column of each graph
  const int32_t *sell_seg;    // batch: graph of each sliced-ELL chunk
  // batch: out-arc sum of each graph's frontier, [2][graphs] by round parity,
  // and the sum above which that graph's next round is a full sweep
  unsigned long long *gfsum;
  const unsigned long long *gthr;
  int32_t nseg;               // batch: graphs in the union
  // batch: first sliced-ELL chunk of each graph [nseg + 1]; the graphs swept
  // whole in the next round (dlist, ctrl->ndense of them) and the exclusive
  // prefix of their chunk counts (dpref), written by the post kernel
  const int64_t *seg_chunk0;
  int32_t *dlist;
  int64_t *dpref;
  // batch, on request: m_active of each graph by round, [row_cap + 2][nseg],
  // slot = round - row_base like rs (else null)
  unsigned long long *gmact;
  const int32_t *perm;  // relabelled graph: caller id -> internal id (else null)
  int64_t perm_n;       // nodes of the relabelled graph (replicas: a seed k*perm_n + x
                        // of copy k maps to k*perm_n + perm[x])
  RoundStats *rs;       // [row_cap + 2], slot = round - row_base
  Ctrl *ctrl;
  int32_t max_rounds;
  int32_t direction;
  float dense_threshold;
  int32_t row_cap;      // rows of the device counts window
  int32_t test_changed; // test C_{t-1} before gathering an in-neighbour's delta
  int32_t test_adapt;   // decide test_changed per round (ctrl->test, set by the post kernel)
  int32_t dense_tma;    // dense rounds are swept by k_pull_tma (launched before k_pull)
  int32_t push;         // sparse rounds push from the previous frontier (kModePush)
  int32_t push_kernel;  // ... in k_push, launched after the pull (else inside k_pull)
  int32_t use_cond;     // launched inside a conditional while-graph
  int32_t iter_guard;   // post launches after which a pass is abandoned
  unsigned long long cond;  // cudaGraphConditionalHandle of that graph
};

// Work item of the pull: one piece of a row's in-arcs. x = first arc, y =
// (row << 32) | (whole << 31) | arcs, `whole` marking a row of one piece.
__host__ __device__ __forceinline__ ulonglong2 make_item(int32_t v, int64_t first, int64_t len,
                                                         bool whole) {
  return make_ulonglong2((unsigned long long)first,
                         ((unsigned long long)(uint32_t)v << 32) | (whole ? 0x80000000ULL : 0ULL) |
                             (unsigned long long)len);
}

}  // namespace pg
