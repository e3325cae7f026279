/*
 * CPU oracle for PROPAGATE (Amati et al., "PROPAGATE: a seed propagation
 * framework to compute Distance-based metrics on Very Large Graphs").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * statement of what the propagation computes. Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the library's
 * product path never does. It shares no code, header or table with the CUDA
 * path.
 *
 * What it states:
 *   - Sec. 4 (paragraph on collisions) says that after r synchronous rounds
 *     the XOR-popcount of seed x's bit counts the nodes at distance exactly r
 *     from x. So the per-seed, per-round counts are the BFS distance
 *     histograms h_i[d] = |{v : d(x_i, v) = d}|, computed here with one FIFO
 *     queue BFS per seed along arcs u -> v (the rand-BFS visit of Sec. 5.1).
 *   - Floyd-Warshall all-pairs distances, the independent check of the BFS
 *     on tiny graphs.
 *   - The active-arc measure m_active(t) of the round-t sweep (the skip rule
 *     in the proof of Thm. 1: only nodes with a zero bit update, and only
 *     nodes with a neighbour that changed can change), restated from
 *     distances alone.
 *   - The metrics of Sec. 3 (Preliminaries) and of the last steps of
 *     Algorithm 1, in FP64 from exact 64-bit integer sums.
 *   - Algorithm 1 itself on the host, sweep by sweep over s-bit signatures:
 *     a second statement of the per-seed counts (checked against the BFS)
 *     and the paper's own method timed on the host cores.
 *
 * Graph input everywhere: a CSR over in-edges, row v lists every u with an
 * arc u -> v. Distances follow arcs forward from the seed.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_ERANGE (-3)

/* ------------------------------------------------------------ threading */
typedef struct {
  int64_t next; /* next item, taken under the lock */
  int64_t count;
  pthread_mutex_t lock;
  void (*fn)(void *ctx, int64_t item, int worker);
  void *ctx;
} or_pool;

typedef struct {
  or_pool *pool;
  int worker;
} or_worker_arg;

static void *or_worker(void *p) {
  or_worker_arg *a = (or_worker_arg *)p;
  or_pool *pool = a->pool;
  for (;;) {
    pthread_mutex_lock(&pool->lock);
    int64_t it = pool->next++;
    pthread_mutex_unlock(&pool->lock);
    if (it >= pool->count) break;
    pool->fn(pool->ctx, it, a->worker);
  }
  return NULL;
}

/* Runs fn(ctx, item, worker) for every item in [0, count) on `threads`
 * threads; items are independent. */
static int or_parallel(int64_t count, int threads, void (*fn)(void *, int64_t, int), void *ctx) {
  if (threads < 1) threads = 1;
  if (threads > count) threads = count > 0 ? (int)count : 1;
  or_pool pool;
  pool.next = 0;
  pool.count = count;
  pool.fn = fn;
  pool.ctx = ctx;
  pthread_mutex_init(&pool.lock, NULL);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
  or_worker_arg *args = (or_worker_arg *)malloc(sizeof(or_worker_arg) * (size_t)threads);
  if (!th || !args) {
    free(th);
    free(args);
    return OR_ENOMEM;
  }
  for (int t = 0; t < threads; ++t) {
    args[t].pool = &pool;
    args[t].worker = t;
    pthread_create(&th[t], NULL, or_worker, &args[t]);
  }
  for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&pool.lock);
  free(th);
  free(args);
  return OR_OK;
}

/* --------------------------------------------------------------- graph */
/* Out-edge lists (the transpose of the in-edge CSR), by counting. */
typedef struct {
  int64_t n;
  int64_t *ptr;
  int32_t *adj;
} or_out;

static int or_check_csr(int64_t n, const int64_t *row_ptr, const int32_t *col) {
  if (n < 1 || !row_ptr) return OR_EINVAL;
  if (row_ptr[0] != 0) return OR_EINVAL;
  for (int64_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return OR_EINVAL;
  int64_t m = row_ptr[n];
  if (m > 0 && !col) return OR_EINVAL;
  for (int64_t j = 0; j < m; ++j)
    if (col[j] < 0 || col[j] >= n) return OR_EINVAL;
  return OR_OK;
}

static int or_transpose(int64_t n, const int64_t *row_ptr, const int32_t *col, or_out *out) {
  int64_t m = row_ptr[n];
  out->n = n;
  out->ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  out->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  if (!out->ptr || !out->adj || !fill) {
    free(out->ptr);
    free(out->adj);
    free(fill);
    return OR_ENOMEM;
  }
  for (int64_t j = 0; j < m; ++j) out->ptr[col[j] + 1]++;
  for (int64_t u = 0; u < n; ++u) out->ptr[u + 1] += out->ptr[u];
  for (int64_t u = 0; u < n; ++u) fill[u] = out->ptr[u];
  for (int64_t v = 0; v < n; ++v)
    for (int64_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) out->adj[fill[col[j]]++] = (int32_t)v;
  free(fill);
  return OR_OK;
}

static void or_out_free(or_out *o) {
  free(o->ptr);
  free(o->adj);
}

/* One FIFO-queue BFS from `src` along out-edges. dist[v] = hops from src, or
 * -1 if v is not reachable. `queue` has room for n entries. */
static void or_bfs(const or_out *g, int32_t src, int32_t *dist, int32_t *queue) {
  for (int64_t v = 0; v < g->n; ++v) dist[v] = -1;
  int64_t head = 0, tail = 0;
  dist[src] = 0;
  queue[tail++] = src;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int64_t j = g->ptr[u]; j < g->ptr[u + 1]; ++j) {
      int32_t v = g->adj[j];
      if (dist[v] < 0) {
        dist[v] = dist[u] + 1;
        queue[tail++] = v;
      }
    }
  }
}

/* ------------------------------------------------ per-seed histograms */
typedef struct {
  const or_out *g;
  const int32_t *seeds;
  int64_t cap;
  int64_t *hist;   /* [s][cap] */
  int32_t *ecc;    /* [s] eccentricity of each seed */
  int32_t **dist;  /* per worker scratch */
  int32_t **queue; /* per worker scratch */
  int32_t *dmat;   /* optional [n][s] node-major distance matrix */
  int64_t s;
  int overflow;
} or_hist_ctx;

static void or_hist_item(void *p, int64_t i, int w) {
  or_hist_ctx *c = (or_hist_ctx *)p;
  int32_t *dist = c->dist[w];
  or_bfs(c->g, c->seeds[i], dist, c->queue[w]);
  int64_t *h = c->hist ? c->hist + i * c->cap : NULL;
  if (h)
    for (int64_t d = 0; d < c->cap; ++d) h[d] = 0;
  int32_t ecc = 0;
  for (int64_t v = 0; v < c->g->n; ++v) {
    int32_t d = dist[v];
    if (c->dmat) c->dmat[v * c->s + i] = d;
    if (d < 0) continue;
    if (d > ecc) ecc = d;
    if (h) {
      if (d < c->cap)
        h[d]++;
      else
        c->overflow = 1;
    }
  }
  if (c->ecc) c->ecc[i] = ecc;
}

/*
 * Per-seed distance histograms: hist[i*cap + d] = |{v : d(seeds[i], v) = d}|
 * for d < cap, and ecc[i] = max finite distance from seeds[i]. These are the
 * exact per-seed, per-round collision counts of PROPAGATE (Sec. 4, Alg. 1:
 * the round's count adds, over all nodes, the popcount of the XOR of the new
 * and the old signature; here restricted to bit i, seed i's).
 * dmat, if not NULL, receives the node-major distance matrix
 * dmat[v*s + i] = d(seeds[i], v) (-1 if unreachable).
 * Returns OR_ERANGE if some distance is >= cap (hist then holds the prefix).
 */
int or_seed_histograms(int64_t n, const int64_t *row_ptr, const int32_t *col,
                       const int32_t *seeds, int64_t s, int64_t cap, int64_t *hist,
                       int32_t *ecc, int32_t *dmat, int threads) {
  int rc = or_check_csr(n, row_ptr, col);
  if (rc) return rc;
  if (s < 0 || (s > 0 && !seeds) || cap < 1) return OR_EINVAL;
  for (int64_t i = 0; i < s; ++i)
    if (seeds[i] < 0 || seeds[i] >= n) return OR_EINVAL;
  if (threads < 1) threads = 1;
  or_out g;
  if ((rc = or_transpose(n, row_ptr, col, &g))) return rc;
  or_hist_ctx c;
  memset(&c, 0, sizeof(c));
  c.g = &g;
  c.seeds = seeds;
  c.cap = cap;
  c.hist = hist;
  c.ecc = ecc;
  c.dmat = dmat;
  c.s = s;
  c.dist = (int32_t **)calloc((size_t)threads, sizeof(int32_t *));
  c.queue = (int32_t **)calloc((size_t)threads, sizeof(int32_t *));
  rc = (c.dist && c.queue) ? OR_OK : OR_ENOMEM;
  for (int t = 0; t < threads && !rc; ++t) {
    c.dist[t] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    c.queue[t] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!c.dist[t] || !c.queue[t]) rc = OR_ENOMEM;
  }
  if (!rc) rc = or_parallel(s, threads, or_hist_item, &c);
  if (c.dist)
    for (int t = 0; t < threads; ++t) free(c.dist[t]);
  if (c.queue)
    for (int t = 0; t < threads; ++t) free(c.queue[t]);
  free(c.dist);
  free(c.queue);
  or_out_free(&g);
  if (!rc && c.overflow) rc = OR_ERANGE;
  return rc;
}

/* ---------------------------------------------------- Floyd-Warshall */
/*
 * All-pairs hop distances by Floyd-Warshall: dist[u*n + v] = d(u, v) along
 * arcs (u -> v present when u is in row v of the in-edge CSR), -1 if v is
 * not reachable from u, 0 on the diagonal. For tiny graphs only: O(n^3).
 */
int or_apsp_floyd_warshall(int64_t n, const int64_t *row_ptr, const int32_t *col,
                           int64_t *dist) {
  int rc = or_check_csr(n, row_ptr, col);
  if (rc) return rc;
  const int64_t INF = INT64_MAX / 4;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t v = 0; v < n; ++v) dist[u * n + v] = (u == v) ? 0 : INF;
  for (int64_t v = 0; v < n; ++v)
    for (int64_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
      int64_t u = col[j];
      if (u != v) dist[u * n + v] = 1;
    }
  for (int64_t k = 0; k < n; ++k)
    for (int64_t u = 0; u < n; ++u)
      for (int64_t v = 0; v < n; ++v)
        if (dist[u * n + k] + dist[k * n + v] < dist[u * n + v])
          dist[u * n + v] = dist[u * n + k] + dist[k * n + v];
  for (int64_t i = 0; i < n * n; ++i)
    if (dist[i] >= INF) dist[i] = -1;
  return OR_OK;
}

/* ------------------------------------------------- active-arc measure */
/*
 * m_active[t] for t in [0, rounds], from the node-major distance matrix
 * dmat[v*s + i] = d(x_i, v) (-1 unreachable) of the s seeds.
 *
 * In round t >= 1 of Algorithm 1, node v's signature can change only if some
 * in-neighbour u changed in round t-1, and, by the skip rule of the proof of
 * Thm. 1, only if v still has a zero bit. In terms of distances:
 *   u changed in round t-1   <=>  d(x_i, u) = t-1 for some seed i
 *   v has a zero bit before t <=> d(x_i, v) > t-1 or x_i never reaches v,
 *                                  for some seed i
 * A_t is the set of such v, and m_active[t] = sum over v in A_t of the
 * in-degree of v (the arcs a round-t pull sweep reads). m_active[0] = 0.
 */
typedef struct {
  int64_t n, s, rounds;
  const int64_t *row_ptr;
  const int32_t *col;
  const int32_t *dmat;
  uint64_t **acc;  /* per worker [rounds+1] */
  uint8_t **mark;  /* per worker [rounds+2] scratch */
  int64_t chunk;
} or_ma_ctx;

static void or_ma_item(void *p, int64_t item, int w) {
  or_ma_ctx *c = (or_ma_ctx *)p;
  int64_t v0 = item * c->chunk, v1 = v0 + c->chunk;
  if (v1 > c->n) v1 = c->n;
  uint8_t *mark = c->mark[w];
  uint64_t *acc = c->acc[w];
  for (int64_t v = v0; v < v1; ++v) {
    int64_t indeg = c->row_ptr[v + 1] - c->row_ptr[v];
    if (indeg == 0) continue;
    /* last round before which v still has a zero bit: v is unsaturated
     * before round t iff t <= sat_bound */
    int64_t maxd = 0;
    int unreached = 0;
    for (int64_t i = 0; i < c->s; ++i) {
      int32_t d = c->dmat[v * c->s + i];
      if (d < 0)
        unreached = 1;
      else if (d > maxd)
        maxd = d;
    }
    int64_t sat_bound = unreached ? c->rounds : maxd; /* unsaturated before t iff t <= maxd */
    if (sat_bound > c->rounds) sat_bound = c->rounds;
    for (int64_t t = 0; t <= c->rounds + 1; ++t) mark[t] = 0;
    for (int64_t j = c->row_ptr[v]; j < c->row_ptr[v + 1]; ++j) {
      int64_t u = c->col[j];
      for (int64_t i = 0; i < c->s; ++i) {
        int32_t d = c->dmat[u * c->s + i];
        if (d >= 0 && d + 1 <= sat_bound) mark[d + 1] = 1;
      }
    }
    for (int64_t t = 1; t <= sat_bound; ++t)
      if (mark[t]) acc[t] += (uint64_t)indeg;
  }
}

int or_m_active(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *dmat,
                int64_t s, int64_t rounds, uint64_t *m_active, int threads) {
  int rc = or_check_csr(n, row_ptr, col);
  if (rc) return rc;
  if (s < 1 || rounds < 0 || !dmat || !m_active) return OR_EINVAL;
  if (threads < 1) threads = 1;
  or_ma_ctx c;
  c.n = n;
  c.s = s;
  c.rounds = rounds;
  c.row_ptr = row_ptr;
  c.col = col;
  c.dmat = dmat;
  c.chunk = 4096;
  c.acc = (uint64_t **)calloc((size_t)threads, sizeof(uint64_t *));
  c.mark = (uint8_t **)calloc((size_t)threads, sizeof(uint8_t *));
  rc = (c.acc && c.mark) ? OR_OK : OR_ENOMEM;
  for (int t = 0; t < threads && !rc; ++t) {
    c.acc[t] = (uint64_t *)calloc((size_t)rounds + 1, sizeof(uint64_t));
    c.mark[t] = (uint8_t *)calloc((size_t)rounds + 2, 1);
    if (!c.acc[t] || !c.mark[t]) rc = OR_ENOMEM;
  }
  if (!rc) rc = or_parallel((n + c.chunk - 1) / c.chunk, threads, or_ma_item, &c);
  if (!rc) {
    for (int64_t t = 0; t <= rounds; ++t) {
      uint64_t sum = 0;
      for (int w = 0; w < threads; ++w) sum += c.acc[w][t];
      m_active[t] = sum;
    }
  }
  for (int t = 0; t < threads; ++t) {
    if (c.acc) free(c.acc[t]);
    if (c.mark) free(c.mark[t]);
  }
  free(c.acc);
  free(c.mark);
  return rc;
}

/* ------------------------------------------------------------ metrics */
typedef struct {
  int32_t diameter;               /* Delta_LB: last hop with a new pair */
  int32_t eff_diameter;           /* min k with R[k] >= tau * R[Delta_LB] */
  double eff_diameter_interp;     /* linear interpolation between k-1 and k */
  double avg_distance;            /* mean distance over reachable pairs u != v */
  double avg_distance_incl_self;  /* same sum divided by R[Delta_LB] */
  double connectivity_rate;       /* alpha */
  double reachable_pairs;         /* (n/s) * R[Delta_LB] */
  uint64_t R_last;                /* R[Delta_LB] over the s sampled seeds */
  uint64_t dist_sum;              /* sum over sampled pairs of r * (#pairs at r) */
} or_metrics_out;

/*
 * Metrics from per-seed histograms hist[i*cap + d] (d < cap) of s seeds on an
 * n-node graph, with threshold tau = tau_num / tau_den:
 *   R[r]          = sum_i sum_{d<=r} hist_i[d], the sampled neighbourhood
 *                   function; it counts the s pairs (x_i, x_i) (Sec. 3 defines
 *                   |N(r)| over V x V, so self-pairs belong to it).
 *   diameter      = T = the last r with a new pair, the Delta_LB of Alg. 1.
 *   eff_diameter  = min {k : R[k] >= tau * R[T]} (Sec. 3 and Alg. 1), compared
 *                   exactly as tau_den * R[k] >= tau_num * R[T].
 *   avg_distance  = sum_r r * (R[r] - R[r-1]) / (R[T] - s): the mean distance
 *                   over reachable pairs with u != v (the self-pairs add 0 to
 *                   the numerator and are left out of the denominator).
 *   avg_distance_incl_self = the same numerator over R[T], Alg. 1's division.
 *   connectivity_rate = (R[T] - s) / (s (n - 1)), the sampled alpha of Sec. 3.
 *   reachable_pairs   = (n / s) * R[T], Alg. 1's final scaling.
 */
int or_metrics(const int64_t *hist, int64_t s, int64_t cap, int64_t n, int64_t tau_num,
               int64_t tau_den, or_metrics_out *out) {
  if (!hist || !out || s < 1 || cap < 1 || n < 1 || tau_den < 1 || tau_num < 0 ||
      tau_num > tau_den)
    return OR_EINVAL;
  uint64_t *R = (uint64_t *)calloc((size_t)cap, sizeof(uint64_t));
  if (!R) return OR_ENOMEM;
  int64_t T = 0;
  uint64_t run = 0, dsum = 0;
  for (int64_t d = 0; d < cap; ++d) {
    uint64_t at = 0;
    for (int64_t i = 0; i < s; ++i) at += (uint64_t)hist[i * cap + d];
    run += at;
    R[d] = run;
    dsum += (uint64_t)d * at;
    if (at > 0) T = d;
  }
  int64_t k = 0;
  while ((unsigned __int128)tau_den * R[k] < (unsigned __int128)tau_num * R[T]) ++k;
  double tau = (double)tau_num / (double)tau_den;
  double interp = 0.0;
  if (k > 0) {
    double lo = (double)R[k - 1], hi = (double)R[k];
    interp = (double)(k - 1) + (tau * (double)R[T] - lo) / (hi - lo);
  }
  uint64_t others = R[T] - (uint64_t)s;
  out->diameter = (int32_t)T;
  out->eff_diameter = (int32_t)k;
  out->eff_diameter_interp = interp;
  out->avg_distance = others ? (double)dsum / (double)others : 0.0;
  out->avg_distance_incl_self = (double)dsum / (double)R[T];
  out->connectivity_rate = n > 1 ? (double)others / ((double)s * (double)(n - 1)) : 0.0;
  out->reachable_pairs = ((double)n / (double)s) * (double)R[T];
  out->R_last = R[T];
  out->dist_sum = dsum;
  free(R);
  return OR_OK;
}

/* ---------------------------------------------- Algorithm 1 on the host */
/*
 * PROPAGATE-P as Algorithm 1 states it. Every node has an s-bit signature
 * (W = ceil(s/64) words; seed i sets bit i of its own node). In each round
 * every node whose signature still has a zero bit (the skip rule of the
 * proof of Thm. 1) ORs the signatures of all its in-neighbours into its next
 * signature; all reads see the previous round's signatures (Sig, then
 * Sig = Sig_next). The bits a node gains in round t are the seeds at
 * distance exactly t (Sec. 4, paragraph on collisions), counted per seed.
 * The rounds stop when a round gains nothing; T is the last round that
 * gained a bit. Along the way each round's m_active is the in-degree sum of
 * the nodes the round revisits: those still missing a bit with an
 * in-neighbour that gained one in the previous round (a seed gains its own
 * bit in round 0), the skip rule of the proof of Thm. 1 taken literally.
 */
typedef struct {
  int64_t n;
  const int64_t *rp;
  const int32_t *col;
  int W;
  int64_t s;
  uint64_t last_mask; /* valid bits of word W-1 */
  const uint64_t *sig;
  uint64_t *nxt;
  const unsigned char *chg; /* node gained a bit in the previous round */
  unsigned char *chg_next;  /* ... in this round */
  uint32_t *cnt;            /* [workers][s] */
  uint64_t *mact;           /* [workers] */
  int64_t block;
} or_pp_ctx;

static void or_pp_item(void *p, int64_t item, int w) {
  or_pp_ctx *c = (or_pp_ctx *)p;
  const int W = c->W;
  uint32_t *cnt = c->cnt + (size_t)w * (size_t)c->s;
  int64_t v1 = (item + 1) * c->block;
  if (v1 > c->n) v1 = c->n;
  for (int64_t v = item * c->block; v < v1; ++v) {
    const uint64_t *sv = c->sig + (size_t)v * W;
    uint64_t *nv = c->nxt + (size_t)v * W;
    int full = 1;
    for (int k = 0; k < W; ++k) {
      nv[k] = sv[k];
      full = full && sv[k] == (k == W - 1 ? c->last_mask : ~0ULL);
    }
    c->chg_next[v] = 0;
    if (full) continue;
    int active = 0;
    for (int64_t j = c->rp[v]; j < c->rp[v + 1]; ++j) {
      const uint64_t *su = c->sig + (size_t)c->col[j] * W;
      for (int k = 0; k < W; ++k) nv[k] |= su[k];
      active = active || c->chg[c->col[j]];
    }
    if (active) c->mact[w] += (uint64_t)(c->rp[v + 1] - c->rp[v]);
    for (int k = 0; k < W; ++k) {
      uint64_t d = nv[k] ^ sv[k];
      if (d) c->chg_next[v] = 1;
      while (d) {
        cnt[k * 64 + __builtin_ctzll(d)] += 1;
        d &= d - 1;
      }
    }
  }
}

/*
 * counts: [cap+1][s] uint32, row t = per-seed nodes at distance exactly t
 * (row 0 = 1 for every seed); *rounds = T; m_active (may be NULL):
 * [cap+2] uint64, entries 0..T+1 written (entry T+1 is the final sweep that
 * gains nothing). OR_ERANGE when a round beyond cap still gains bits. Seeds
 * must be distinct and in range.
 */
int or_propagate_p(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *seeds,
                   int64_t s, int64_t cap, uint32_t *counts, int32_t *rounds, uint64_t *m_active,
                   int threads) {
  int rc = or_check_csr(n, row_ptr, col);
  if (rc) return rc;
  if (!seeds || s < 1 || s > n || cap < 0 || !counts || !rounds) return OR_EINVAL;
  if (threads < 1) threads = 1;
  const int W = (int)((s + 63) / 64);
  uint64_t *sig = (uint64_t *)calloc((size_t)n * W, sizeof(uint64_t));
  uint64_t *nxt = (uint64_t *)calloc((size_t)n * W, sizeof(uint64_t));
  uint32_t *cnt = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)threads * (size_t)s);
  uint64_t *mact = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)threads);
  unsigned char *chg = (unsigned char *)calloc((size_t)n, 1);
  unsigned char *chg_next = (unsigned char *)calloc((size_t)n, 1);
  int bad = !sig || !nxt || !cnt || !mact || !chg || !chg_next;
  if (bad) rc = OR_ENOMEM;
  for (int64_t i = 0; !bad && i < s; ++i) {
    const int32_t x = seeds[i];
    bad = x < 0 || x >= n || chg[x]; /* chg marks the seeds met so far */
    if (bad) rc = OR_EINVAL;
    if (!bad) {
      chg[x] = 1; /* a seed gains its own bit in round 0 */
      sig[(size_t)x * W + (size_t)(i / 64)] |= 1ULL << (i % 64);
      counts[i] = 1;
    }
  }
  if (bad) {
    free(sig);
    free(nxt);
    free(cnt);
    free(mact);
    free(chg);
    free(chg_next);
    return rc;
  }
  if (m_active) m_active[0] = 0;
  or_pp_ctx c;
  c.n = n;
  c.rp = row_ptr;
  c.col = col;
  c.W = W;
  c.s = s;
  c.last_mask = (s % 64) ? ((1ULL << (s % 64)) - 1ULL) : ~0ULL;
  c.cnt = cnt;
  c.mact = mact;
  c.block = 4096;
  const int64_t items = (n + c.block - 1) / c.block;
  int32_t T = 0;
  for (int64_t t = 1;; ++t) {
    memset(cnt, 0, sizeof(uint32_t) * (size_t)threads * (size_t)s);
    memset(mact, 0, sizeof(uint64_t) * (size_t)threads);
    c.sig = sig;
    c.nxt = nxt;
    c.chg = chg;
    c.chg_next = chg_next;
    rc = or_parallel(items, threads, or_pp_item, &c);
    if (rc) break;
    uint64_t total = 0, ma = 0;
    for (int64_t i = 0; i < s; ++i) {
      uint32_t a = 0;
      for (int k = 0; k < threads; ++k) a += cnt[(size_t)k * (size_t)s + (size_t)i];
      total += a;
      if (t <= cap) counts[(size_t)t * (size_t)s + (size_t)i] = a;
    }
    for (int k = 0; k < threads; ++k) ma += mact[k];
    if (m_active && t <= cap + 1) m_active[t] = ma;
    uint64_t *tmp = sig; /* Sig = Sig_next */
    sig = nxt;
    nxt = tmp;
    unsigned char *tc = chg;
    chg = chg_next;
    chg_next = tc;
    if (total == 0) break;
    if (t > cap) {
      rc = OR_ERANGE;
      break;
    }
    T = (int32_t)t;
  }
  free(sig);
  free(nxt);
  free(cnt);
  free(mact);
  free(chg);
  free(chg_next);
  if (rc) return rc;
  *rounds = T;
  return OR_OK;
}
