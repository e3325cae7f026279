// Serving loop (pg_server_*): resident graphs, asynchronous metric requests,
// continuous batching.
//
// A request is (graph, seeds); its answer is the per-round, per-seed counts
// of PROPAGATE-P (Algorithm 1) on that graph, the same as pg_propagate_p
// alone. The server keeps every registered graph's CSR (and out-CSR and
// sliced-ELL copy) on the device. `slots` worker threads each own a CUDA
// stream and one grow-only workspace; a worker that is free takes the oldest
// queued request that fits the device-memory budget, merges into it the
// other queued requests on the same graph (seeds of different requests are
// independent bit columns, Sec. 4; a node may carry seeds of several
// requests), runs one propagation and splits the columns back per request.
// Requests submitted while others run are admitted as soon as a slot and the
// memory they need are free, and the propagations of different slots run
// concurrently on their streams.
//
// Memory: resident bytes (CSR, out-CSR, sliced-ELL, piece lists) plus, per
// slot, its workspace and the piece lists of the graphs it served, must stay
// within hbm_budget. A request whose footprint cannot fit even on an idle
// server is refused at submission (PG_ENOMEM). When admitting a request
// would exceed the budget, idle slots first drop what they hold; otherwise
// the request waits.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host.cuh"

namespace {

using namespace pg;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  int64_t id = 0;
  int32_t graph = 0;
  std::vector<int32_t> seeds;
  int32_t state = PG_REQ_QUEUED;
  int32_t status = PG_OK;
  int32_t rounds = -1;
  int32_t merged = 0;
  int64_t footprint = 0;
  int64_t submit_ns = 0, start_ns = 0, done_ns = 0;
  bool cancel = false;
  std::vector<uint32_t> counts;  // rows x s, filled by the worker
  bool open = true;              // still receiving rows during the run
};

struct Resident {
  pg_graph *g = nullptr;
  int64_t bytes = 0;
  int32_t active = 0;  // queued or running requests
  bool removing = false;
};

struct Slot {
  std::thread th;
  cudaStream_t stream = nullptr;
  Workspace ws;
  std::unordered_map<int32_t, pg_graph *> views;  // graph id -> view on ws
  bool busy = false;
  int64_t held = 0;  // workspace + views' piece lists, as charged
};

int64_t view_bytes(const pg_graph *v) { return (int64_t)v->pieces.list.bytes; }

// Counts window of a served propagation: rows kept on the device between
// copies to the host (more rounds move the window).
constexpr int32_t kServeWindowRows = 256;

}  // namespace

struct pg_server {
  pg_server_config cfg{};
  int device = 0;
  int64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv;       // workers: work or stop
  std::condition_variable done_cv;  // waiters: a request finished
  bool stop = false;
  std::map<int32_t, Resident> graphs;
  int32_t next_graph = 0;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  std::deque<int64_t> queue;
  int64_t next_req = 1;
  std::vector<std::unique_ptr<Slot>> slots;
  cudaStream_t ctl = nullptr;  // uploads
  pg_server_stats st{};
};

namespace {

int64_t resident_total(const pg_server *s) {
  int64_t b = 0;
  for (const auto &kv : s->graphs) b += kv.second.bytes;
  return b;
}

int64_t slots_total(const pg_server *s) {
  int64_t b = 0;
  for (const auto &sl : s->slots) b += sl->held;
  return b;
}

void recount(Slot &sl) {
  int64_t b = workspace_held(sl.ws);
  for (const auto &kv : sl.views) b += view_bytes(kv.second);
  sl.held = b;
}

// Drops what an idle slot holds (its views and its workspace).
void trim(Slot &sl) {
  for (auto &kv : sl.views) pg_graph_free(kv.second);
  sl.views.clear();
  release_workspace(sl.ws);
  sl.held = 0;
}

struct Job {
  std::vector<Request *> reqs;
  int32_t graph = -1;
  std::vector<int32_t> graphs;  // distinct graphs, first-taken first (several: a union)
  int64_t need = 0;             // slot bytes after the job
};

// Largest packed union a cross-graph propagation builds.
constexpr int64_t kUnionMaxNodes = 1LL << 22;
constexpr int64_t kUnionMaxArcs = 1LL << 27;

int width_class(int64_t s) {
  const int64_t W = (s + 63) / 64;
  return W <= 1 ? 1 : W <= 2 ? 2 : W <= 4 ? 4 : (int)((W + 7) / 8 * 8);
}

// Device bytes of the arrays of a union of n nodes and m arcs (directed:
// with its out-CSR): its CSR copies, node map and relabelling map, and its
// sliced-ELL copy and piece lists (the propagation's workspace is the slot's).
int64_t union_array_bytes(int64_t n, int64_t m, bool directed) {
  const int64_t csr = (n + 1) * 8 + m * 4;
  return csr * (directed ? 2 : 1) + n * 8 + (n + m / 2 + 1) * 16 * 2 + m * 4;
}

// Bytes the slot will hold after running s seeds on graph gid.
int64_t slot_need(const pg_server *srv, const Slot &sl, int32_t gid, int32_t s) {
  const pg_graph *g = srv->graphs.at(gid).g;
  const int32_t maxr = (int32_t)std::min<int64_t>(g->n - 1, 0x3FFFFFFF);
  int64_t ws = std::max(workspace_held(sl.ws),
                        workspace_bytes(g, s, maxr, srv->cfg.opt.window_rows));
  int64_t views = 0;
  for (const auto &kv : sl.views) views += view_bytes(kv.second);
  if (!sl.views.count(gid)) views += (g->n + g->m / 2 + 1) * 16;
  return ws + views;
}

// Under the lock: the oldest queued request that fits, with the other queued
// requests on its graph merged in. Returns false when none can start now.
bool pick(pg_server *srv, int k, Job &job) {
  Slot &me = *srv->slots[k];
  for (size_t qi = 0; qi < srv->queue.size(); ++qi) {
    Request *head = srv->reqs.at(srv->queue[qi]).get();
    std::vector<size_t> take{qi};
    int64_t s_total = (int64_t)head->seeds.size();
    // same graph first (as without unions), then, with cross_graph, queued
    // requests on other graphs whose seeds keep each graph within the
    // signature width the head's graph reached (those graphs run as one
    // union; a narrower graph only leaves words of its rows unused)
    for (size_t qj = qi + 1; qj < srv->queue.size(); ++qj) {
      if ((int32_t)take.size() >= srv->cfg.merge_max) break;
      Request *r = srv->reqs.at(srv->queue[qj]).get();
      if (r->graph != head->graph) continue;
      if (s_total + (int64_t)r->seeds.size() > srv->cfg.merge_max_seeds) continue;
      take.push_back(qj);
      s_total += (int64_t)r->seeds.size();
    }
    std::vector<std::pair<int32_t, int64_t>> per{{head->graph, s_total}};
    const pg_graph *hg = srv->graphs.at(head->graph).g;
    const int cls = width_class(s_total);
    int64_t un = hg->n, um = hg->m;
    bool udir = hg->directed != 0;
    int32_t umaxr = (int32_t)std::min<int64_t>(hg->n - 1, 0x3FFFFFFF);
    const bool cross = srv->cfg.cross_graph && cls <= 8 && hg->n <= kUnionMaxNodes / 2;
    for (size_t qj = qi + 1; cross && qj < srv->queue.size(); ++qj) {
      if ((int32_t)take.size() >= srv->cfg.merge_max) break;
      Request *r = srv->reqs.at(srv->queue[qj]).get();
      if (r->graph == head->graph) continue;
      const int64_t rs = (int64_t)r->seeds.size();
      if (s_total + rs > srv->cfg.merge_max_seeds) continue;
      auto it = std::find_if(per.begin(), per.end(),
                             [&](const std::pair<int32_t, int64_t> &x) { return x.first == r->graph; });
      if (it != per.end()) {
        if (width_class(it->second + rs) > cls) continue;
        it->second += rs;
      } else {
        if (width_class(rs) > cls) continue;
        const pg_graph *g = srv->graphs.at(r->graph).g;
        if (un + g->n > kUnionMaxNodes || um + g->m > kUnionMaxArcs) continue;
        per.push_back({r->graph, rs});
        un += g->n;
        um += g->m;
        udir = udir || g->directed;
        umaxr = std::max<int32_t>(umaxr, (int32_t)std::min<int64_t>(g->n - 1, 0x3FFFFFFF));
      }
      take.push_back(qj);
      s_total += rs;
    }
    int64_t smax = 0;
    for (auto &x : per) smax = std::max(smax, x.second);
    const bool uni = per.size() > 1;
    auto need_now = [&]() {
      if (!uni) return slot_need(srv, me, head->graph, (int32_t)s_total);
      int64_t views = 0;
      for (const auto &kv : me.views) views += view_bytes(kv.second);
      return std::max(workspace_held(me.ws),
                      workspace_bytes_nm(un, um, (int32_t)smax, umaxr,
                                         srv->cfg.opt.window_rows)) +
             views + union_array_bytes(un, um, udir);
    };
    int64_t need = need_now();
    const int64_t fixed = resident_total(srv);
    int64_t others = slots_total(srv) - me.held;
    auto fits = [&](int64_t nd) { return fixed + others + nd <= srv->budget; };
    if (!fits(need)) {
      // idle slots drop what they hold, largest first, until it fits
      std::vector<Slot *> idle;
      for (auto &sl : srv->slots)
        if (sl.get() != &me && !sl->busy && sl->held > 0) idle.push_back(sl.get());
      std::sort(idle.begin(), idle.end(), [](Slot *a, Slot *b) { return a->held > b->held; });
      for (Slot *sl : idle) {
        if (fits(need)) break;
        others -= sl->held;
        trim(*sl);
      }
    }
    if (!fits(need) && me.held > 0) {  // this slot's own cache may be in the way
      trim(me);
      need = need_now();
    }
    if (!fits(need)) continue;  // a younger, smaller request may fit
    std::sort(take.begin(), take.end());  // queue positions, erased from the back
    job.need = need;
    job.graph = head->graph;
    for (auto &x : per) job.graphs.push_back(x.first);
    for (size_t t : take) job.reqs.push_back(srv->reqs.at(srv->queue[t]).get());
    for (auto it = take.rbegin(); it != take.rend(); ++it)
      srv->queue.erase(srv->queue.begin() + (std::ptrdiff_t)*it);
    return true;
  }
  return false;
}

struct Split {
  std::vector<Request *> reqs;
  std::vector<int32_t> col0;
};

// Counts window sink: each request's columns, round by round, until its
// first round without a new pair (every later round is empty too).
void split_window(void *vctx, int32_t row_base, int32_t rows, const uint32_t *data,
                  int32_t ncols) {
  Split *sp = static_cast<Split *>(vctx);
  for (size_t k = 0; k < sp->reqs.size(); ++k) {
    Request *r = sp->reqs[k];
    if (!r->open) continue;
    const int32_t s = (int32_t)r->seeds.size(), c0 = sp->col0[k];
    for (int32_t i = 0; i < rows && r->open; ++i) {
      const uint32_t *row = data + (size_t)i * ncols + c0;
      bool any = false;
      for (int32_t j = 0; j < s; ++j) any |= row[j] != 0u;
      if (!any && row_base + i > 0) {
        r->open = false;
        break;
      }
      r->counts.insert(r->counts.end(), row, row + s);
    }
  }
}

// Union builder: graph k's rows at node offset v0 and arc offset a0.
__global__ void k_union_rows(const int64_t *rp, int64_t n, int64_t v0, int64_t a0, int64_t *rp_u,
                             int32_t *node_graph, int32_t k, const int32_t *perm,
                             int32_t *perm_u) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    rp_u[v0 + v] = rp[v] + a0;
    node_graph[v0 + v] = k;
    // a relabelled graph: the caller's id v0 + x maps to v0 + its internal id
    if (perm_u) perm_u[v0 + v] = (int32_t)(v0 + (perm ? perm[v] : v));
  }
}

__global__ void k_union_cols(const int32_t *col, int64_t m, int32_t v0, int64_t a0,
                             int32_t *col_u) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x)
    col_u[a0 + j] = col[j] + v0;
}

struct Union {
  pg_graph *g = nullptr;
  DevBuf node_graph, graph_s, graph_col0;
  std::vector<int64_t> v0, graph_m;
  int64_t last = 0;  // the last row pointer, the source of its copy
  ~Union() {
    if (g) pg_graph_free(g);
    release(node_graph);
    release(graph_s);
    release(graph_col0);
  }
};

// Packs the resident graphs `parts` into one disjoint union on the device (a
// packed batch, as build_groups does from host CSRs), with each part's seed
// count s[k] and first count column col0[k].
pg_status build_union(const std::vector<const pg_graph *> &parts, const std::vector<int32_t> &s,
                      const std::vector<int32_t> &col0, cudaStream_t st, Union &u) {
  const int K = (int)parts.size();
  int64_t n = 0, m = 0;
  bool directed = false, perm = false;
  int64_t maxdeg = 0;
  for (const pg_graph *g : parts) {
    u.v0.push_back(n);
    u.graph_m.push_back(g->m);
    n += g->n;
    m += g->m;
    directed = directed || g->directed;
    perm = perm || g->perm_ptr;
    maxdeg = std::max(maxdeg, g->max_degree);
  }
  pg_graph *ug = new pg_graph();
  u.g = ug;
  ug->n = n;
  ug->m = m;
  ug->directed = directed ? 1 : 0;
  cudaGetDevice(&ug->device);
  ug->max_degree = maxdeg;
  ug->mean_degree = (double)m / (double)std::max<int64_t>(n, 1);
  pg_status rc = cuda_status(cudaMalloc((void **)&ug->row_ptr, sizeof(int64_t) * (n + 1)));
  if (!rc) rc = cuda_status(cudaMalloc((void **)&ug->col, sizeof(int32_t) * std::max<int64_t>(m, 1)));
  if (!rc && directed) {
    rc = cuda_status(cudaMalloc((void **)&ug->out_ptr, sizeof(int64_t) * (n + 1)));
    if (!rc) rc = cuda_status(cudaMalloc((void **)&ug->out_col, sizeof(int32_t) * std::max<int64_t>(m, 1)));
  } else if (!rc) {
    ug->out_ptr = ug->row_ptr;
    ug->out_col = ug->col;
    ug->owns_out = false;
  }
  if (!rc) rc = ensure(u.node_graph, sizeof(int32_t) * (size_t)n);
  if (!rc && perm) rc = ensure(ug->perm, sizeof(int32_t) * (size_t)n);
  if (!rc) rc = ensure(u.graph_s, sizeof(int32_t) * (size_t)K);
  if (!rc) rc = ensure(u.graph_col0, sizeof(int32_t) * (size_t)K);
  int64_t a0 = 0;
  for (int k = 0; k < K && !rc; ++k) {
    const pg_graph *g = parts[k];
    const int blocks = (int)std::min<int64_t>(4096, (std::max(g->n, g->m) + kBlock - 1) / kBlock);
    k_union_rows<<<blocks, kBlock, 0, st>>>(g->row_ptr, g->n, u.v0[k], a0, ug->row_ptr,
                                            (int32_t *)u.node_graph.p, k, g->perm_ptr,
                                            perm ? (int32_t *)ug->perm.p : nullptr);
    k_union_cols<<<blocks, kBlock, 0, st>>>(g->col, g->m, (int32_t)u.v0[k], a0, ug->col);
    if (directed) {
      k_union_rows<<<blocks, kBlock, 0, st>>>(g->out_ptr, g->n, u.v0[k], a0, ug->out_ptr,
                                              (int32_t *)u.node_graph.p, k, nullptr, nullptr);
      k_union_cols<<<blocks, kBlock, 0, st>>>(g->out_col, g->m, (int32_t)u.v0[k], a0,
                                              ug->out_col);
    }
    rc = cuda_status(cudaGetLastError());
    a0 += g->m;
  }
  if (!rc) {  // the last row pointer, m (its source outlives the synchronisation below)
    u.last = m;
    rc = cuda_status(cudaMemcpyAsync(ug->row_ptr + n, &u.last, sizeof(int64_t),
                                     cudaMemcpyHostToDevice, st));
    if (!rc && directed)
      rc = cuda_status(cudaMemcpyAsync(ug->out_ptr + n, &u.last, sizeof(int64_t),
                                       cudaMemcpyHostToDevice, st));
    if (!rc)
      rc = cuda_status(cudaMemcpyAsync(u.graph_s.p, s.data(), sizeof(int32_t) * K,
                                       cudaMemcpyHostToDevice, st));
    if (!rc)
      rc = cuda_status(cudaMemcpyAsync(u.graph_col0.p, col0.data(), sizeof(int32_t) * K,
                                       cudaMemcpyHostToDevice, st));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
  }
  if (rc) return rc;
  ug->seg_of = (const int32_t *)u.node_graph.p;
  ug->nseg = K;
  if (perm) ug->perm_ptr = (const int32_t *)ug->perm.p;
  return PG_OK;
}

void worker(pg_server *srv, int k) {
  cudaSetDevice(srv->device);
  Slot &me = *srv->slots[k];
  for (;;) {
    Job job;
    pg_graph *master = nullptr;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      srv->cv.wait(lk, [&] { return srv->stop || (!srv->queue.empty() && pick(srv, k, job)); });
      if (job.reqs.empty()) return;  // stopping
      me.busy = true;
      me.held = job.need;  // charged up front; trued up after the run
      const int64_t t = now_ns();
      for (Request *r : job.reqs) {
        r->state = PG_REQ_RUNNING;
        r->start_ns = t;
        r->merged = (int32_t)job.reqs.size();
        r->footprint = job.need;
      }
      srv->st.running += (int32_t)job.reqs.size();
      srv->st.queued -= (int32_t)job.reqs.size();
      srv->st.inflight_bytes = slots_total(srv);
      srv->st.peak_bytes = std::max(srv->st.peak_bytes, resident_total(srv) + slots_total(srv));
      master = srv->graphs.at(job.graph).g;
    }
    // outside the lock: the propagation
    pg_status rc = PG_OK;
    Split sp;
    pg_stats pst{};
    int32_t T = 0;
    if (job.graphs.size() <= 1) {
      pg_graph *view = nullptr;
      auto it = me.views.find(job.graph);
      if (it != me.views.end()) {
        view = it->second;
      } else {
        rc = make_view(master, me.stream, &view);
        if (rc == PG_OK) {
          view->ext_ws = &me.ws;
          me.views[job.graph] = view;
        }
      }
      std::vector<int32_t> seeds;
      for (Request *r : job.reqs) {
        sp.reqs.push_back(r);
        sp.col0.push_back((int32_t)seeds.size());
        seeds.insert(seeds.end(), r->seeds.begin(), r->seeds.end());
        r->counts.clear();
        r->open = true;
      }
      if (rc == PG_OK) {
        const int32_t maxr = (int32_t)std::min<int64_t>(master->n - 1, 0x3FFFFFFF);
        rc = propagate_columns(view, seeds.data(), (int32_t)seeds.size(), maxr, &split_window,
                               &sp, &T, &srv->cfg.opt, me.stream, &pst);
      }
    } else {
      // several graphs: their requests' seeds as one packed union, each
      // graph's columns together (its requests in queue order)
      std::vector<const pg_graph *> parts;
      std::vector<int32_t> gs, gc0, seeds, bits;
      {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (int32_t gid : job.graphs) parts.push_back(srv->graphs.at(gid).g);
      }
      Union u;
      int32_t maxr = 0;
      for (size_t gk = 0; gk < job.graphs.size(); ++gk) {
        int32_t sk = 0;
        gc0.push_back((int32_t)seeds.size());
        maxr = std::max<int32_t>(maxr, (int32_t)std::min<int64_t>(parts[gk]->n - 1, 0x3FFFFFFF));
        for (Request *r : job.reqs) {
          if (r->graph != job.graphs[gk]) continue;
          sp.reqs.push_back(r);
          sp.col0.push_back((int32_t)seeds.size());
          for (int32_t x : r->seeds) {
            seeds.push_back(x);  // the caller's id; the union's offset is added below
            bits.push_back(sk++);
          }
          r->counts.clear();
          r->open = true;
        }
        gs.push_back(sk);
      }
      rc = build_union(parts, gs, gc0, me.stream, u);
      if (rc == PG_OK) {
        for (size_t gk = 0, i = 0; gk < job.graphs.size(); ++gk)
          for (int32_t b = 0; b < gs[gk]; ++b, ++i) seeds[i] += (int32_t)u.v0[gk];
        u.g->ext_ws = &me.ws;
        int32_t smax = 0;
        for (int32_t x : gs) smax = std::max(smax, x);
        rc = propagate_batch_group(u.g, seeds.data(), bits.data(), (int32_t)seeds.size(),
                                   (const int32_t *)u.node_graph.p,
                                   (const int32_t *)u.graph_s.p, (const int32_t *)u.graph_col0.p,
                                   u.graph_m.data(), (int32_t)seeds.size(), smax, maxr,
                                   &split_window, &sp, &T, &srv->cfg.opt, me.stream, &pst);
      }
      cudaStreamSynchronize(me.stream);  // the union's arrays are freed next
    }
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      me.busy = false;
      recount(me);
      const int64_t t = now_ns();
      for (Request *r : job.reqs) {
        r->done_ns = t;
        if (rc != PG_OK) {
          r->state = PG_REQ_FAILED;
          r->status = rc;
          r->counts.clear();
          srv->st.failed += 1;
        } else if (r->cancel) {
          r->state = PG_REQ_CANCELLED;
          r->status = PG_ECANCELLED;
          r->counts.clear();
          srv->st.cancelled += 1;
        } else {
          r->state = PG_REQ_DONE;
          r->rounds = (int32_t)(r->counts.size() / r->seeds.size()) - 1;
          srv->st.completed += 1;
        }
        srv->graphs.at(r->graph).active -= 1;
      }
      srv->st.running -= (int32_t)job.reqs.size();
      srv->st.propagations += 1;
      if (rc == PG_OK) {
        srv->st.seed_edge_traversals += pst.seed_edge_traversals;
        srv->st.gpu_launches += pst.launches;
      }
      srv->st.inflight_bytes = slots_total(srv);
    }
    srv->done_cv.notify_all();
    srv->cv.notify_all();  // memory may have freed up for a waiting request
  }
}

void fill_info(const Request &r, pg_request_info *info) {
  if (!info) return;
  info->state = r.state;
  info->status = r.status;
  info->rounds = r.rounds;
  info->s = (int32_t)r.seeds.size();
  info->graph = r.graph;
  info->merged = r.merged;
  info->footprint = r.footprint;
  info->submit_ns = r.submit_ns;
  info->start_ns = r.start_ns;
  info->done_ns = r.done_ns;
}

bool finished(const Request &r) {
  return r.state == PG_REQ_DONE || r.state == PG_REQ_FAILED || r.state == PG_REQ_CANCELLED;
}

}  // namespace

extern "C" {

void pg_server_default_config(pg_server_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->slots = 4;
  cfg->merge_max = 16;
  cfg->merge_max_seeds = 8192;
  cfg->cross_graph = 1;
  cfg->hbm_budget = 0;
  pg_default_options(&cfg->opt);
}

pg_status pg_server_create(const pg_server_config *cfg, pg_server **out) {
  if (!out) return PG_EINVAL;
  pg_server_config c;
  pg_server_default_config(&c);
  if (cfg) c = *cfg;
  if (c.slots < 1 || c.slots > 64 || c.merge_max < 1 || c.merge_max_seeds < 1 ||
      c.hbm_budget < 0 || c.opt.direction < 0 || c.opt.direction > 2)
    return PG_EINVAL;
  auto *srv = new pg_server();
  srv->cfg = c;
  srv->cfg.opt.timing = 0;
  if (srv->cfg.opt.window_rows <= 0) srv->cfg.opt.window_rows = kServeWindowRows;
  cudaGetDevice(&srv->device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    delete srv;
    return PG_ECUDA;
  }
  srv->budget = c.hbm_budget > 0 ? c.hbm_budget : (int64_t)(0.9 * (double)free_b);
  if (cudaStreamCreateWithFlags(&srv->ctl, cudaStreamNonBlocking) != cudaSuccess) {
    delete srv;
    return PG_ECUDA;
  }
  for (int k = 0; k < c.slots; ++k) {
    auto sl = std::make_unique<Slot>();
    if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto &x : srv->slots) cudaStreamDestroy(x->stream);
      cudaStreamDestroy(srv->ctl);
      delete srv;
      return PG_ECUDA;
    }
    srv->slots.push_back(std::move(sl));
  }
  for (int k = 0; k < c.slots; ++k) srv->slots[k]->th = std::thread(worker, srv, k);
  srv->st.budget_bytes = srv->budget;
  *out = srv;
  return PG_OK;
}

void pg_server_destroy(pg_server *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    for (int64_t id : srv->queue) {  // never started: cancelled
      Request &r = *srv->reqs.at(id);
      r.state = PG_REQ_CANCELLED;
      r.status = PG_ECANCELLED;
      r.done_ns = now_ns();
    }
    srv->queue.clear();
  }
  srv->cv.notify_all();
  srv->done_cv.notify_all();
  for (auto &sl : srv->slots)
    if (sl->th.joinable()) sl->th.join();  // running propagations finish first
  for (auto &sl : srv->slots) {
    trim(*sl);
    cudaStreamDestroy(sl->stream);
  }
  for (auto &kv : srv->graphs) pg_graph_free(kv.second.g);
  cudaStreamDestroy(srv->ctl);
  delete srv;
}

pg_status pg_server_add_graph(pg_server *srv, const int64_t *row_ptr, const int32_t *col,
                              int64_t n, int64_t m, int directed, int32_t *graph_id) {
  if (!srv || !graph_id) return PG_EINVAL;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != srv->device) return PG_EINVAL;
  pg_graph *g = nullptr;
  pg_status rc = pg_graph_from_csr(row_ptr, col, n, m, directed, 0, srv->ctl, &g);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g->mu);
    rc = ensure_sell(g, kSellPiece, srv->ctl);
    if (rc == PG_OK) rc = cuda_status(cudaStreamSynchronize(srv->ctl));
  }
  if (rc) {
    pg_graph_free(g);
    return rc;
  }
  int64_t bytes = (n + 1) * 8 + m * 4;
  if (g->out_ptr != g->row_ptr) bytes *= 2;
  bytes += (int64_t)(g->sell.items.bytes + g->sell.col.bytes + g->sell.off.bytes +
                     g->sell.len.bytes + g->pieces.list.bytes);
  std::lock_guard<std::mutex> lk(srv->mu);
  if (resident_total(srv) + bytes > srv->budget) {
    pg_graph_free(g);
    return PG_ENOMEM;
  }
  const int32_t id = srv->next_graph++;
  srv->graphs[id] = Resident{g, bytes, 0, false};
  srv->st.graphs += 1;
  srv->st.resident_bytes = resident_total(srv);
  *graph_id = id;
  return PG_OK;
}

pg_status pg_server_remove_graph(pg_server *srv, int32_t graph_id) {
  if (!srv) return PG_EINVAL;
  pg_graph *g = nullptr;
  {
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->graphs.find(graph_id);
    if (it == srv->graphs.end() || it->second.removing) return PG_EINVAL;
    if (it->second.active > 0) return PG_EINVAL;  // requests still queued or running
    // views on it are idle: drop them before the master
    for (auto &sl : srv->slots) {
      auto v = sl->views.find(graph_id);
      if (v != sl->views.end()) {
        pg_graph_free(v->second);
        sl->views.erase(v);
        recount(*sl);
      }
    }
    g = it->second.g;
    srv->graphs.erase(it);
    srv->st.graphs -= 1;
    srv->st.resident_bytes = resident_total(srv);
  }
  pg_graph_free(g);
  srv->cv.notify_all();
  return PG_OK;
}

pg_status pg_server_submit(pg_server *srv, int32_t graph_id, const int32_t *seeds, int32_t s,
                           int64_t *request_id) {
  if (!srv || !seeds || s < 1 || !request_id) return PG_EINVAL;
  auto r = std::make_unique<Request>();
  r->seeds.assign(seeds, seeds + s);
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->graphs.find(graph_id);
  if (it == srv->graphs.end() || it->second.removing) return PG_EINVAL;
  const pg_graph *g = it->second.g;
  if (s > g->n) return PG_EINVAL;
  {
    std::vector<int32_t> v(r->seeds);
    std::sort(v.begin(), v.end());
    if (v.front() < 0 || v.back() >= g->n) return PG_EINVAL;
    for (size_t i = 1; i < v.size(); ++i)
      if (v[i] == v[i - 1]) return PG_EINVAL;
  }
  // must fit an otherwise idle server
  const int32_t maxr = (int32_t)std::min<int64_t>(g->n - 1, 0x3FFFFFFF);
  const int64_t alone =
      workspace_bytes(g, s, maxr, srv->cfg.opt.window_rows) + (g->n + g->m / 2 + 1) * 16;
  if (resident_total(srv) + alone > srv->budget) return PG_ENOMEM;
  r->id = srv->next_req++;
  r->graph = graph_id;
  r->submit_ns = now_ns();
  *request_id = r->id;
  srv->queue.push_back(r->id);
  it->second.active += 1;
  srv->reqs[r->id] = std::move(r);
  srv->st.submitted += 1;
  srv->st.queued += 1;
  lk.unlock();
  srv->cv.notify_all();
  return PG_OK;
}

pg_status pg_server_poll(pg_server *srv, int64_t request_id, pg_request_info *info) {
  if (!srv || !info) return PG_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(request_id);
  if (it == srv->reqs.end()) return PG_EINVAL;
  fill_info(*it->second, info);
  return PG_OK;
}

pg_status pg_server_wait(pg_server *srv, int64_t request_id, int32_t timeout_ms,
                         pg_request_info *info) {
  if (!srv) return PG_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(request_id);
  if (it == srv->reqs.end()) return PG_EINVAL;
  Request *r = it->second.get();
  auto ready = [&] { return finished(*r); };
  if (timeout_ms < 0) {
    srv->done_cv.wait(lk, ready);
  } else if (!srv->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    fill_info(*r, info);
    return PG_ETIMEOUT;
  }
  fill_info(*r, info);
  return PG_OK;
}

pg_status pg_server_result(pg_server *srv, int64_t request_id, pg_counts *out,
                           pg_request_info *info) {
  if (!srv || !out || !out->counts) return PG_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(request_id);
  if (it == srv->reqs.end()) return PG_EINVAL;
  Request &r = *it->second;
  if (!finished(r)) return PG_EINVAL;
  fill_info(r, info);
  if (r.state != PG_REQ_DONE) {
    const pg_status st = (pg_status)r.status;
    srv->reqs.erase(it);
    return st;
  }
  if (out->s != (int32_t)r.seeds.size() || out->max_rounds < 0) return PG_EINVAL;
  const int32_t rows = std::min(r.rounds, out->max_rounds) + 1;
  std::memcpy(out->counts, r.counts.data(), sizeof(uint32_t) * (size_t)rows * out->s);
  out->rounds = r.rounds;
  if (out->m_active) std::memset(out->m_active, 0, sizeof(uint64_t) * ((size_t)out->max_rounds + 2));
  const pg_status st = r.rounds > out->max_rounds ? PG_ERANGE : PG_OK;
  if (st == PG_OK) srv->reqs.erase(it);
  return st;
}

pg_status pg_server_cancel(pg_server *srv, int64_t request_id) {
  if (!srv) return PG_EINVAL;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(request_id);
    if (it == srv->reqs.end()) return PG_EINVAL;
    Request &r = *it->second;
    if (r.state == PG_REQ_QUEUED) {
      auto q = std::find(srv->queue.begin(), srv->queue.end(), request_id);
      if (q != srv->queue.end()) srv->queue.erase(q);
      r.state = PG_REQ_CANCELLED;
      r.status = PG_ECANCELLED;
      r.done_ns = now_ns();
      srv->st.queued -= 1;
      srv->st.cancelled += 1;
      srv->graphs.at(r.graph).active -= 1;
    } else if (r.state == PG_REQ_RUNNING) {
      r.cancel = true;  // its propagation finishes; the result is dropped
    }
  }
  srv->done_cv.notify_all();
  return PG_OK;
}

pg_status pg_server_get_stats(pg_server *srv, pg_server_stats *out) {
  if (!srv || !out) return PG_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  *out = srv->st;
  out->inflight_bytes = slots_total(srv);
  out->resident_bytes = resident_total(srv);
  return PG_OK;
}

}  // extern "C"
