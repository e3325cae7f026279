// Host-side structures of the PROPAGATE library (not part of the C ABI):
// device buffers and workspaces, cached piece lists and sliced-ELL copies,
// the graph handle, and the internal entry points between translation units.
#pragma once

#include <functional>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace pg {

// A device allocation owned by the library.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  bool host = false;  // pinned host memory the device reads over C2C (ensure_host)
};

// The buffers of a propagation, carved out of one device allocation (arena)
// by carve_workspace; each buffer's p points into the arena.
struct Workspace {
  DevBuf arena;
  size_t used = 0;  // end of the laid-out parts in the arena
  DevBuf X, Y, D0, D1, C0, C1, K0, K1, Sat, RB, KW0, KW1, F0, F1, E, A, counts, rs, ctrl, seeds,
      seed_bits, gfsum, gthr, dlist, dpref, E1, gm;
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
  DevBuf chunk0; // int64 per graph + 1: a packed batch's first chunk of each graph
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
  // PG_HOST_CSR: the arc arrays (col, out_col and the sliced-ELL copy's
  // columns) live in pinned host memory and are read over C2C
  bool host_csr = false;
  bool col_host = false, out_col_host = false;
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
  // node relabelling (hubs first): original id -> internal id, owned here;
  // perm_ptr is that map (a view's is its master's), null when not relabelled
  pg::DevBuf perm;
  const int32_t *perm_ptr = nullptr;
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
// The same in pinned host memory, mapped into the device's address space.
pg_status ensure_host(DevBuf &b, size_t bytes);
void release(DevBuf &b);
// Frees every buffer, event and pinned block of a workspace.
void release_workspace(Workspace &w);
// Gives each listed buffer of w at least the listed bytes: one device
// allocation per workspace (with 1/32 of slack), carved 256-byte aligned.
// Buffers the layout lacks go into the slack when they fit; when a buffer
// must grow, or the slack is too small, the whole workspace is laid out
// again (contents are not kept); otherwise every buffer keeps its address.
pg_status carve_workspace(Workspace &w, const std::vector<std::pair<DevBuf *, size_t>> &needs);
// Device bytes a workspace holds.
int64_t workspace_held(const Workspace &w);
pg_status cuda_status(cudaError_t e);
int sm_count();
int64_t l2_bytes();  // of the current device
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
                                pg_stats *st_out, std::vector<unsigned long long> *mact = nullptr);
// Seeds of several requests merged on one graph: seed i owns bit and count
// column i, and a node may carry several seeds; windows go to the sink.
// mact (optional): m_active by round, rows 0..rounds+1 (a packed batch: one
// column per graph of the union, [round][graph]; else one column).
pg_status propagate_columns(pg_graph *g, const int32_t *seeds, int32_t nseeds, int32_t max_rounds,
                            WindowSink sink, void *sink_ctx, int32_t *rounds,
                            const pg_options *opt, void *stream, pg_stats *st_out,
                            std::vector<unsigned long long> *mact = nullptr);
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
// The same for a graph of n nodes and m arcs.
int64_t workspace_bytes_nm(int64_t n, int64_t m, int32_t s, int32_t max_rounds,
                           int32_t window_rows);

}  // namespace pg
