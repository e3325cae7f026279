// Internal declarations of the PROPAGATE library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <mutex>
#include <vector>

#include "propagate.h"

namespace pg {

constexpr int kBlock = 256;
constexpr unsigned kFullMask = 0xFFFFFFFFu;

// Packed frontier append: count of rows in the high bits, running sum of
// their out-degrees in the low kFsumBits bits (one 64-bit atomic keeps the
// two consistent, so every frontier row gets its out-arc prefix).
constexpr int kFsumBits = 37;
constexpr unsigned long long kFsumMask = (1ULL << kFsumBits) - 1ULL;

// kModeMixed (packed batches): each graph of the union picks its own kind
// of round from its own frontier (see Params::gfsum).
enum : int32_t { kModeDense = 0, kModeSparse = 1, kModeMixed = 2 };

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
  int32_t pad;
  unsigned long long nF_prev;  // |F_{t-1}|
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
};

// Everything the round kernels need, passed by value.
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
  RoundStats *rs;       // [row_cap + 2], slot = round - row_base
  Ctrl *ctrl;
  int32_t max_rounds;
  int32_t direction;
  float dense_threshold;
  int32_t row_cap;      // rows of the device counts window
  int32_t test_changed; // test C_{t-1} before gathering an in-neighbour's delta
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

// A device allocation owned by the library.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

struct Workspace {
  DevBuf X, Y, D0, D1, C0, C1, K0, K1, Sat, RB, KW0, KW1, F0, F1, E, A, counts, rs, ctrl, seeds,
      seed_bits, gfsum, gthr;
  Ctrl *ctrl_h = nullptr;  // pinned, 2 slots
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> tev;  // timing events
};

struct PieceList {
  int32_t L = 0;
  DevBuf list;
  int64_t count = 0;
};

// Sliced-ELL copy of the in-CSR for dense rounds: rows cut into pieces of at
// most Lmax arcs, pieces sorted by length (longest first), 32 per chunk; a
// chunk's column indices are stored column-major (arc k of lane l at
// off[c] + 32 k + l, -1 past a piece's end), so a warp reading step k of a
// chunk loads 128 contiguous bytes.
constexpr int32_t kSellPiece = 256;  // longest piece of the sliced-ELL copy

struct SellList {
  int32_t Lmax = 0;
  DevBuf items;  // ulonglong2 make_item per lane slot, nchunks * 32
  DevBuf col;    // int32
  DevBuf off;    // int64 per chunk
  DevBuf len;    // int32 per chunk (its longest piece)
  DevBuf seg;    // int32 per chunk: its graph, for a packed batch (else empty)
  int64_t nchunks = 0;
  int64_t slots = 0;  // total col entries
};

}  // namespace pg

struct pg_graph {
  int64_t n = 0, m = 0;
  int directed = 1;
  int device = 0;
  int64_t *row_ptr = nullptr;
  int32_t *col = nullptr;
  int64_t *out_ptr = nullptr;
  int32_t *out_col = nullptr;
  bool owns_in = true;
  bool owns_out = true;
  bool owns_sell = true;  // false in a view (make_view)
  // a packed batch: the graph of each node (device, borrowed) and how many
  const int32_t *seg_of = nullptr;
  int32_t nseg = 0;
  // PROPAGATE-S passes run together: rep_K copies of this graph side by side
  // (make_replicas), the copy of each node, and per-call pass tables
  pg_graph *rep = nullptr;
  int32_t rep_K = 0;
  pg::DevBuf rep_graph_of, rep_graph_s, rep_graph_col0;
  double mean_degree = 0.0;
  int64_t max_degree = 0;
  pg::PieceList pieces;
  pg::SellList sell;
  pg::Workspace ws;
  pg::Workspace *ext_ws = nullptr;  // a view running on its server slot's workspace
  pg_stats last{};
  int hint_p = 0, hint_s = 0;  // sweeps of the last pass, first batch of the next
  std::mutex mu;
};

namespace pg {

// Grow-only device buffer; contents are not preserved on growth.
pg_status ensure(DevBuf &b, size_t bytes);
void release(DevBuf &b);
// Frees every buffer, event and pinned block of a workspace.
void release_workspace(Workspace &w);
// Device bytes a workspace holds.
int64_t workspace_held(const Workspace &w);
pg_status cuda_status(cudaError_t e);
int sm_count();
// Dense piece list of g for piece length L (cached in g).
pg_status ensure_pieces(pg_graph *g, int32_t L, cudaStream_t st);
// Sliced-ELL copy of g's in-CSR for pieces of at most Lmax arcs (cached in g).
pg_status ensure_sell(pg_graph *g, int32_t Lmax, cudaStream_t st);
// Exclusive scan of int64 in place over n entries (device).
pg_status exclusive_scan_i64(int64_t *data, int64_t n, cudaStream_t st);
// Drops the CUDA graphs captured for g.
void drop_graph_cache(pg_graph *g);
// Receives each copied-out counts window of a batch run.
typedef void (*WindowSink)(void *ctx, int32_t row_base, int32_t rows, const uint32_t *data,
                           int32_t ncols);
// graph_m: host, arcs of each graph (each picks its own kind of round).
pg_status propagate_batch_group(pg_graph *g, const int32_t *seeds, const int32_t *seed_bit,
                                int32_t nseeds, const int32_t *node_graph_d,
                                const int32_t *graph_s_d, const int32_t *graph_col0_d,
                                const int64_t *graph_m, int32_t ncols, int32_t s_bits,
                                int32_t max_rounds, WindowSink sink, void *sink_ctx,
                                int32_t *rounds, const pg_options *opt, void *stream,
                                pg_stats *st_out);
// Seeds of several requests merged on one graph: seed i owns bit and count
// column i, and a node may carry several seeds; windows go to the sink.
pg_status propagate_columns(pg_graph *g, const int32_t *seeds, int32_t nseeds, int32_t max_rounds,
                            WindowSink sink, void *sink_ctx, int32_t *rounds,
                            const pg_options *opt, void *stream, pg_stats *st_out);
// A handle sharing master's device CSR, out-CSR and sliced-ELL copy (built
// first if missing) with its own workspace, piece list and CUDA graphs, so
// that several propagations on one graph can run at once on different
// streams. The master must outlive the view.
pg_status make_view(pg_graph *master, cudaStream_t st, pg_graph **out);
// One timed run of a tuning candidate: its time and a hash of its counts.
typedef std::function<pg_status(const pg_options &, double *ms, uint64_t *hash)> TuneRun;
// Coordinate descent over the schedule options (see tune.cu).
pg_status tune_options(const TuneRun &run, int32_t s_bits, int32_t max_trials, pg_options *inout,
                       pg_tune_report *rep, bool s_mode);
uint64_t fnv1a(uint64_t h, const void *data, size_t bytes);
// K copies of g side by side, cached in g (see pg_graph::rep); PG_EINVAL if
// they would not fit the index ranges.
pg_status make_replicas(pg_graph *g, int K, cudaStream_t st);
void drop_replicas(pg_graph *g);
// Device bytes a propagation of s seeds on g will hold in its workspace
// (window_rows as pg_options.window_rows).
int64_t workspace_bytes(const pg_graph *g, int32_t s, int32_t max_rounds, int32_t window_rows);

}  // namespace pg
