// Batched PROPAGATE-P over many graphs (pg_batch_*).
//
// Graphs of the same signature width are packed into one disjoint union — a
// CSR over in-edges with each graph's nodes and arcs shifted by its node
// offset — and that union runs through the same round kernels as a single
// graph: one pull and one post launch per round for every graph of the
// group, the round loop being one device-driven CUDA graph. No arc joins two
// graphs, so bit i of a node only ever means its own graph's seed i; the
// post kernel looks up each changed node's graph to add its new bits to that
// graph's count columns and to test saturation against that graph's seeds.
// A graph whose propagation ended simply has no frontier in later rounds.
//
// Large graphs run alone. A graph whose four signature arrays (X, Y and the
// two deltas) would fill half of L2 by themselves already gives a round
// enough rows to fill the GPU, and run alone it keeps part of its arrays in
// L2 from one round to the next; packed with others of its size, every
// round streams all of theirs. Four 982^2 grids with s = 512 took 992 ms
// packed and 818 ms one after another. Such a graph is a group of its own
// and goes through the single-graph path.
//
// The groups run concurrently, four at a time by default, each on a stream of
// its own driven by a host thread: a round of a sparse graph is a chain of
// short dependent launches that leaves most of the GPU idle, and other
// groups' rounds fill it (four 982^2 grids: 818 ms one after another, 583 ms
// on four streams). Groups start longest first (by the last run's time,
// else by size).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "host.cuh"

struct pg_batch {
  struct Item {
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col;
    std::vector<int32_t> seeds;
    int64_t n = 0, m = 0;
    int directed = 0;
    int32_t rounds = -1;
    std::vector<uint32_t> counts;  // (rounds+1) x s after a run
    std::vector<uint64_t> m_active;  // by round after a run (rows 0..rounds+1 at least)
    bool open = true;              // still receiving rows during a run
  };
  struct Group {
    std::vector<int32_t> members;
    pg_graph *g = nullptr;
    pg::DevBuf node_graph, graph_s, graph_col0;
    std::vector<int32_t> seeds, seed_bit, col0;
    std::vector<int64_t> graph_m;  // arcs of each member
    int32_t ncols = 0, s_bits = 0, max_rounds = 0;
    bool tuned = false;
    pg_options opt{};  // chosen by pg_batch_tune
    pg_stats last{};   // of the last run
    bool ran = false;
    bool solo = false;  // one large graph, through the single-graph path
    double last_ms = 0;  // host time of its last run
  };
  std::vector<Item> items;
  std::vector<Group> groups;
  std::vector<cudaStream_t> streams;  // the workers' streams
  int32_t nstreams = 4;               // groups run at once
  bool built = false;
  pg_batch_stats stats{};
  std::mutex mu;
};

namespace {

using namespace pg;


int width_class(int32_t s) {
  const int W = (s + 63) / 64;
  return W <= 1 ? 1 : W <= 2 ? 2 : W <= 4 ? 4 : ((W + 7) / 8) * 8;
}

// Whether a graph runs alone: at least 2^16 nodes, and its four signature
// arrays (n x words x 8 bytes each) fill at least half of L2.
bool runs_alone(const pg_batch::Item &it) {
  const int64_t words = width_class((int32_t)it.seeds.size());
  return it.n >= (1 << 16) && 4 * it.n * words * 8 >= l2_bytes() / 2;
}

pg_status build_solo(pg_batch *b, int32_t i, cudaStream_t st) {
  const auto &it = b->items[i];
  pg_batch::Group gr;
  gr.solo = true;
  gr.members.push_back(i);
  pg_status rc = pg_graph_from_csr(it.row_ptr.data(), it.col.data(), it.n, it.m, it.directed, 0,
                                   st, &gr.g);
  if (rc) return rc;
  const int32_t s = (int32_t)it.seeds.size();
  gr.seeds = it.seeds;
  gr.col0 = {0};
  gr.graph_m = {it.m};
  gr.ncols = s;
  gr.s_bits = s;
  gr.max_rounds = (int32_t)std::min<int64_t>(it.n - 1, 0x3FFFFFFF);
  b->groups.push_back(std::move(gr));
  return PG_OK;
}

// One propagation of group gr into sink (counts windows); mact (optional):
// m_active by round, one column per member ([round][member]).
pg_status run_group(pg_batch::Group &gr, WindowSink sink, void *ctx, int32_t *T,
                    const pg_options *o, void *stream, pg_stats *st,
                    std::vector<unsigned long long> *mact = nullptr) {
  if (gr.solo)
    return propagate_columns(gr.g, gr.seeds.data(), (int32_t)gr.seeds.size(), gr.max_rounds, sink,
                             ctx, T, o, stream, st, mact);
  return propagate_batch_group(gr.g, gr.seeds.data(), gr.seed_bit.data(), (int32_t)gr.seeds.size(),
                               (const int32_t *)gr.node_graph.p, (const int32_t *)gr.graph_s.p,
                               (const int32_t *)gr.graph_col0.p, gr.graph_m.data(), gr.ncols,
                               gr.s_bits, gr.max_rounds, sink, ctx, T, o, stream, st, mact);
}

void free_groups(pg_batch *b) {
  for (auto &gr : b->groups) {
    if (gr.g) pg_graph_free(gr.g);
    release(gr.node_graph);
    release(gr.graph_s);
    release(gr.graph_col0);
  }
  b->groups.clear();
  b->built = false;
}

pg_status build_groups(pg_batch *b, cudaStream_t st) {
  std::vector<int> classes;
  for (auto &it : b->items) {
    const int c = width_class((int32_t)it.seeds.size());
    if (std::find(classes.begin(), classes.end(), c) == classes.end()) classes.push_back(c);
  }
  std::sort(classes.begin(), classes.end());
  for (int c : classes) {
    std::vector<int32_t> packed, alone;
    for (int32_t i = 0; i < (int32_t)b->items.size(); ++i) {
      const auto &it = b->items[i];
      if (width_class((int32_t)it.seeds.size()) != c) continue;
      (runs_alone(it) ? alone : packed).push_back(i);
    }
    for (int32_t i : alone)
      if (pg_status rc = build_solo(b, i, st)) return rc;
    // one union per class, or several where the class's graphs together pass
    // the node or arc count one propagation can hold (kMaxNodes, kMaxArcs)
    for (size_t k0 = 0; k0 < packed.size();) {
      pg_batch::Group gr;
      int64_t n = 0, m = 0;
      int directed = 0;
      for (; k0 < packed.size(); ++k0) {
        const auto &it = b->items[packed[k0]];
        if (!gr.members.empty() && (n + it.n > kMaxNodes || m + it.m > kMaxArcs)) break;
        gr.members.push_back(packed[k0]);
        n += it.n;
        m += it.m;
        directed |= it.directed;
      }
      std::vector<int64_t> rp((size_t)n + 1);
      std::vector<int32_t> col((size_t)std::max<int64_t>(m, 1));
      std::vector<int32_t> node_graph((size_t)n), graph_s, graph_col0;
      int64_t v0 = 0, a0 = 0;
      int32_t ncols = 0, s_bits = 0, maxr = 0;
      for (size_t k = 0; k < gr.members.size(); ++k) {
        const auto &it = b->items[gr.members[k]];
        for (int64_t v = 0; v < it.n; ++v) {
          rp[(size_t)(v0 + v)] = a0 + it.row_ptr[(size_t)v];
          node_graph[(size_t)(v0 + v)] = (int32_t)k;
        }
        for (int64_t j = 0; j < it.m; ++j) col[(size_t)(a0 + j)] = (int32_t)(it.col[(size_t)j] + v0);
        const int32_t s = (int32_t)it.seeds.size();
        for (int32_t i = 0; i < s; ++i) {
          gr.seeds.push_back((int32_t)(it.seeds[(size_t)i] + v0));
          gr.seed_bit.push_back(i);
        }
        graph_s.push_back(s);
        graph_col0.push_back(ncols);
        gr.graph_m.push_back(it.m);
        ncols += s;
        s_bits = std::max(s_bits, s);
        maxr = std::max<int32_t>(maxr, (int32_t)std::min<int64_t>(it.n - 1, 0x3FFFFFFF));
        v0 += it.n;
        a0 += it.m;
      }
      rp[(size_t)n] = a0;
      // the union keeps its node order: each graph's nodes stay one block
      pg_status rc = pg_graph_from_csr(rp.data(), col.data(), n, m, directed, PG_KEEP_ORDER, st,
                                       &gr.g);
      if (rc) return rc;
      rc = ensure(gr.node_graph, sizeof(int32_t) * (size_t)n);
      if (!rc) {  // the packed graph knows its parts (sliced-ELL chunks per graph)
        gr.g->seg_of = (const int32_t *)gr.node_graph.p;
        gr.g->nseg = (int32_t)gr.members.size();
      }
      if (!rc) rc = ensure(gr.graph_s, sizeof(int32_t) * graph_s.size());
      if (!rc) rc = ensure(gr.graph_col0, sizeof(int32_t) * graph_col0.size());
      if (!rc) rc = cuda_status(cudaMemcpyAsync(gr.node_graph.p, node_graph.data(),
                                                sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, st));
      if (!rc) rc = cuda_status(cudaMemcpyAsync(gr.graph_s.p, graph_s.data(),
                                                sizeof(int32_t) * graph_s.size(), cudaMemcpyHostToDevice, st));
      if (!rc) rc = cuda_status(cudaMemcpyAsync(gr.graph_col0.p, graph_col0.data(),
                                                sizeof(int32_t) * graph_col0.size(),
                                                cudaMemcpyHostToDevice, st));
      if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
      gr.col0 = graph_col0;
      gr.ncols = ncols;
      gr.s_bits = s_bits;
      gr.max_rounds = maxr;
      b->groups.push_back(std::move(gr));
      if (rc) return rc;
    }
  }
  b->built = true;
  return PG_OK;
}

// Appends each graph's count columns, round by round, until the graph's first
// round without a new pair (its BFS layers are contiguous, so every later
// round is empty too).
struct SinkCtx {
  pg_batch *b;
  pg_batch::Group *gr;
};

void take_window(void *vctx, int32_t row_base, int32_t rows, const uint32_t *data, int32_t ncols) {
  SinkCtx *ctx = static_cast<SinkCtx *>(vctx);
  for (size_t k = 0; k < ctx->gr->members.size(); ++k) {
    auto &it = ctx->b->items[ctx->gr->members[k]];
    if (!it.open) continue;
    const int32_t s = (int32_t)it.seeds.size(), c0 = ctx->gr->col0[k];
    for (int32_t r = 0; r < rows && it.open; ++r) {
      const uint32_t *row = data + (size_t)r * ncols + c0;
      bool any = false;
      for (int32_t i = 0; i < s; ++i) any |= row[i] != 0u;
      if (!any && row_base + r > 0) {
        it.open = false;
        break;
      }
      it.counts.insert(it.counts.end(), row, row + s);
    }
  }
}

struct HashCtx {
  uint64_t h = 1469598103934665603ULL;
};

void hash_window(void *vctx, int32_t row_base, int32_t rows, const uint32_t *data, int32_t ncols) {
  HashCtx *c = static_cast<HashCtx *>(vctx);
  c->h = fnv1a(c->h, &row_base, sizeof(row_base));
  c->h = fnv1a(c->h, data, sizeof(uint32_t) * (size_t)rows * ncols);
}

}  // namespace

extern "C" {

pg_status pg_batch_create(pg_batch **out) {
  if (!out) return PG_EINVAL;
  *out = new pg_batch();
  return PG_OK;
}

void pg_batch_free(pg_batch *b) {
  if (!b) return;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    free_groups(b);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    b->streams.clear();
  }
  delete b;
}

pg_status pg_batch_add(pg_batch *b, const int64_t *row_ptr, const int32_t *col, int64_t n,
                       int64_t m, int directed, const int32_t *seeds, int32_t s,
                       int32_t *index) {
  if (!b || !row_ptr || (m > 0 && !col) || !seeds || n < 1 || m < 0 || s < 1 || s > n ||
      n > kMaxNodes || m > kMaxArcs || row_ptr[0] != 0 || row_ptr[n] != m)
    return PG_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  pg_batch::Item it;
  it.row_ptr.assign(row_ptr, row_ptr + n + 1);
  it.col.assign(col, col + m);
  it.seeds.assign(seeds, seeds + s);
  for (int32_t x : it.seeds)
    if (x < 0 || x >= n) return PG_EINVAL;
  std::vector<int32_t> sorted(it.seeds);
  std::sort(sorted.begin(), sorted.end());
  for (size_t i = 1; i < sorted.size(); ++i)
    if (sorted[i] == sorted[i - 1]) return PG_EINVAL;
  it.n = n;
  it.m = m;
  it.directed = directed ? 1 : 0;
  b->items.push_back(std::move(it));
  if (b->built) free_groups(b);  // regrouped on the next run
  if (index) *index = (int32_t)b->items.size() - 1;
  return PG_OK;
}

pg_status pg_batch_run(pg_batch *b, const pg_options *opt, void *stream) {
  if (!b) return PG_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  if (b->items.empty()) return PG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  pg_status rc = PG_OK;
  if (!b->built && (rc = build_groups(b, st))) {
    free_groups(b);
    return rc;
  }
  const int ng = (int)b->groups.size();
  const int nw = std::min<int>(b->nstreams, ng);
  while ((int)b->streams.size() < nw) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return PG_ECUDA;
    b->streams.push_back(s);
  }
  // the workers' streams start after the work already queued on `stream`
  cudaEvent_t ready = nullptr;
  if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) return PG_ECUDA;
  rc = cuda_status(cudaEventRecord(ready, st));
  for (int w = 0; w < nw && !rc; ++w) rc = cuda_status(cudaStreamWaitEvent(b->streams[w], ready, 0));
  cudaEventDestroy(ready);
  if (rc) return rc;
  for (auto &it : b->items) {
    it.counts.clear();
    it.m_active.clear();
    it.rounds = -1;
    it.open = true;
  }
  // longest first: by the last run's time, else by size
  std::vector<int> order(ng);
  std::iota(order.begin(), order.end(), 0);
  auto cost = [&](int k) {
    const auto &gr = b->groups[k];
    return gr.ran ? gr.last_ms : (double)(gr.g->n + gr.g->m) * (double)width_class(gr.s_bits);
  };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  int dev = 0;
  cudaGetDevice(&dev);
  std::atomic<int> next{0};
  std::atomic<int> failed{0};
  std::vector<pg_status> errs(nw, PG_OK);
  auto work = [&](int w) {
    cudaSetDevice(dev);
    for (int k; !failed.load() && (k = next.fetch_add(1)) < ng;) {
      auto &gr = b->groups[order[k]];
      SinkCtx ctx{b, &gr};
      int32_t T = 0;
      pg_stats st1{};
      const pg_options *o = opt ? opt : (gr.tuned ? &gr.opt : nullptr);
      const auto t0 = std::chrono::steady_clock::now();
      std::vector<unsigned long long> mact;
      const pg_status e = run_group(gr, &take_window, &ctx, &T, o, b->streams[w], &st1, &mact);
      if (e) {
        errs[w] = e;
        failed.store(1);
        return;
      }
      // each member's own m_active: its column of the group's
      const size_t cols = gr.members.size();
      const size_t rows = mact.size() / cols;
      for (size_t k = 0; k < cols; ++k) {
        auto &it = b->items[gr.members[k]];
        it.m_active.resize(rows);
        for (size_t t = 0; t < rows; ++t) it.m_active[t] = mact[t * cols + k];
      }
      gr.last_ms =
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      gr.last = st1;
      gr.ran = true;
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < nw; ++w) th.emplace_back(work, w);
  work(0);
  for (auto &t : th) t.join();
  for (pg_status e : errs)
    if (e && !rc) rc = e;
  if (rc) {
    for (auto &it : b->items) {
      it.counts.clear();
      it.m_active.clear();
      it.rounds = -1;
    }
    return rc;
  }
  pg_batch_stats bs{};
  bs.graphs = (int32_t)b->items.size();
  bs.groups = ng;
  for (auto &gr : b->groups) {
    bs.seed_edge_traversals += gr.last.seed_edge_traversals;
    bs.sweeps = std::max(bs.sweeps, gr.last.sweeps);
    bs.launches += gr.last.launches;
    for (int32_t k : gr.members) {
      auto &it = b->items[k];
      it.rounds = (int32_t)(it.counts.size() / it.seeds.size()) - 1;
    }
  }
  b->stats = bs;
  return PG_OK;
}

pg_status pg_batch_tune(pg_batch *b, int32_t max_trials, pg_tune_report *report, void *stream) {
  if (!b || max_trials < 1) return PG_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  if (b->items.empty()) return PG_EINVAL;
  pg_status rc = PG_OK;
  if (!b->built && (rc = build_groups(b, (cudaStream_t)stream))) {
    free_groups(b);
    return rc;
  }
  pg_tune_report sum{};
  for (auto &gr : b->groups) {
    TuneRun run = [&](const pg_options &o, double *ms, uint64_t *hash) -> pg_status {
      HashCtx hc;
      int32_t T = 0;
      const auto t0 = std::chrono::steady_clock::now();
      pg_status e = run_group(gr, &hash_window, &hc, &T, &o, stream, nullptr);
      const auto t1 = std::chrono::steady_clock::now();
      if (e) return e;
      *ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
      *hash = fnv1a(hc.h, &T, sizeof(T));
      return PG_OK;
    };
    pg_options o;
    pg_default_options(&o);
    pg_tune_report r{};
    if ((rc = tune_options(run, gr.s_bits, max_trials, &o, &r, false))) return rc;
    gr.opt = o;
    gr.tuned = true;
    sum.trials += r.trials;
    sum.improved += r.improved;
    sum.default_ms += r.default_ms;
    sum.best_ms += r.best_ms;
  }
  if (report) *report = sum;
  return PG_OK;
}

pg_status pg_batch_set_streams(pg_batch *b, int32_t streams) {
  if (!b || streams < 1 || streams > 16) return PG_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  b->nstreams = streams;
  return PG_OK;
}

pg_status pg_batch_group_stats(pg_batch *b, int32_t group, pg_stats *out) {
  if (!b || !out) return PG_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  if (group < 0 || group >= (int32_t)b->groups.size() || !b->groups[group].ran) return PG_EINVAL;
  *out = b->groups[group].last;
  return PG_OK;
}

pg_status pg_batch_get_options(pg_batch *b, int32_t group, pg_options *out, int32_t *graphs) {
  if (!b || !out) return PG_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  if (group < 0 || group >= (int32_t)b->groups.size()) return PG_EINVAL;
  const auto &gr = b->groups[group];
  if (gr.tuned)
    *out = gr.opt;
  else
    pg_default_options(out);
  if (graphs) *graphs = (int32_t)gr.members.size();
  return PG_OK;
}

pg_status pg_batch_result(pg_batch *b, int32_t index, pg_counts *out) {
  if (!b || !out || !out->counts) return PG_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  if (index < 0 || index >= (int32_t)b->items.size()) return PG_EINVAL;
  const auto &it = b->items[index];
  if (it.rounds < 0 || out->s != (int32_t)it.seeds.size()) return PG_EINVAL;
  const int32_t rows = std::min(it.rounds, out->max_rounds) + 1;
  std::memcpy(out->counts, it.counts.data(), sizeof(uint32_t) * (size_t)rows * out->s);
  out->rounds = it.rounds;
  if (out->m_active) {  // as pg_propagate_p: rounds 0..min(T + 1, max_rounds + 1)
    std::memset(out->m_active, 0, sizeof(uint64_t) * ((size_t)out->max_rounds + 2));
    const int32_t last = std::min(it.rounds + 1, out->max_rounds + 1);
    for (int32_t t = 0; t <= last && t < (int32_t)it.m_active.size(); ++t)
      out->m_active[t] = it.m_active[(size_t)t];
  }
  return it.rounds > out->max_rounds ? PG_ERANGE : PG_OK;
}

pg_status pg_batch_get_stats(pg_batch *b, pg_batch_stats *out) {
  if (!b || !out) return PG_EINVAL;
  std::lock_guard<std::mutex> lk(b->mu);
  *out = b->stats;
  return PG_OK;
}

}  // extern "C"
