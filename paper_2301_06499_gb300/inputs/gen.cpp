// Seeded synthetic inputs: graphs (Erdos-Renyi, R-MAT, 2-D grid) as CSR over
// in-edges, and seed samples. This file holds no part of the propagation
// method; it produces the graphs and seed sets that both the CPU oracle and the
// CUDA path consume.
//
// Randomness: one counter-based generator. Value i of stream `stream` under
// key `seed` is SplitMix64's output function (Steele, Lea & Flood, "Fast
// splittable pseudorandom number generators", OOPSLA 2014) applied to
// key + (i + 1) * gamma, where key is itself SplitMix64 of the seed and the
// stream number. Every draw is addressable, so any thread can produce any
// edge and the result does not depend on the thread count.
//
// The paper's experiments use real graphs (Table 1); these generators are the
// synthetic stand-ins with the same structure classes: sparse uniform random
// (ER), skewed web/social (R-MAT) and long-diameter lattice (grid).

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <unordered_set>
#include <vector>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

inline uint64_t rng(uint64_t seed, uint64_t stream, uint64_t i) {
  const uint64_t key = mix64(mix64(seed + kGamma) + kGamma * (stream + 1));
  return mix64(key + kGamma * (i + 1));
}

// Uniform integer in [0, n) by the multiply-high map (bias < n / 2^64).
inline uint64_t below(uint64_t x, uint64_t n) {
  return (uint64_t)(((unsigned __int128)x * (unsigned __int128)n) >> 64);
}

constexpr uint64_t kNone = ~0ULL;

int pick_threads(int threads) {
  if (threads > 0) return threads;
  unsigned h = std::thread::hardware_concurrency();
  return h ? (int)h : 1;
}

template <class F>
void parallel_for(int64_t count, int threads, F &&f) {
  // f(begin, end, thread_index) over a static split of [0, count).
  threads = (int)std::max<int64_t>(1, std::min<int64_t>(threads, count));
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t) {
    int64_t b = count * t / threads, e = count * (t + 1) / threads;
    pool.emplace_back([=, &f] { f(b, e, t); });
  }
  for (auto &th : pool) th.join();
}

}  // namespace

extern "C" {

typedef struct pgi_csr {
  int64_t n;
  int64_t m;
  int64_t *row_ptr;  // n + 1
  int32_t *col;      // m
} pgi_csr;

uint64_t pgi_rand(uint64_t seed, uint64_t stream, uint64_t i) { return rng(seed, stream, i); }

void pgi_csr_free(pgi_csr *g) {
  if (!g) return;
  free(g->row_ptr);
  free(g->col);
  free(g);
}

// Builds the CSR over in-edges from packed arc keys (dst << 32 | src); keys
// equal to ~0 are skipped. Rows are sorted ascending and duplicates removed.
// Consumes (frees) `keys`. Returns NULL on allocation failure.
static pgi_csr *build_from_keys(int64_t n, uint64_t *keys, int64_t count, int threads) {
  threads = pick_threads(threads);
  const int64_t B = std::max<int64_t>(1, std::min<int64_t>(4096, n));
  auto bucket_of = [&](uint64_t k) -> int64_t {
    uint64_t dst = k >> 32;
    return (int64_t)((dst * (uint64_t)B) / (uint64_t)n);
  };
  const int T = (int)std::max<int64_t>(1, std::min<int64_t>(threads, count > 0 ? count : 1));
  std::vector<int64_t> cnt((size_t)T * B, 0);
  parallel_for(count, T, [&](int64_t b, int64_t e, int t) {
    int64_t *c = &cnt[(size_t)t * B];
    for (int64_t i = b; i < e; ++i)
      if (keys[i] != kNone) c[bucket_of(keys[i])]++;
  });
  // offsets: bucket-major, thread-minor
  std::vector<int64_t> off((size_t)T * B), bstart(B + 1);
  int64_t run = 0;
  for (int64_t k = 0; k < B; ++k) {
    bstart[k] = run;
    for (int t = 0; t < T; ++t) {
      off[(size_t)t * B + k] = run;
      run += cnt[(size_t)t * B + k];
    }
  }
  bstart[B] = run;
  const int64_t valid = run;
  uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(valid, 1));
  if (!tmp) { free(keys); return nullptr; }
  parallel_for(count, T, [&](int64_t b, int64_t e, int t) {
    int64_t *o = &off[(size_t)t * B];
    for (int64_t i = b; i < e; ++i)
      if (keys[i] != kNone) tmp[o[bucket_of(keys[i])]++] = keys[i];
  });
  free(keys);

  pgi_csr *g = (pgi_csr *)calloc(1, sizeof(pgi_csr));
  g->n = n;
  g->row_ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  if (!g->row_ptr) { free(tmp); free(g); return nullptr; }
  std::vector<int64_t> uniq(B, 0);
  std::atomic<int64_t> next(0);
  auto sort_bucket = [&](int) {
    for (;;) {
      int64_t k = next.fetch_add(1);
      if (k >= B) break;
      uint64_t *b = tmp + bstart[k], *e = tmp + bstart[k + 1];
      std::sort(b, e);
      uint64_t *u = std::unique(b, e);
      uniq[k] = u - b;
      for (uint64_t *p = b; p < u; ++p) g->row_ptr[(*p >> 32) + 1]++;
    }
  };
  {
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t) pool.emplace_back(sort_bucket, t);
    for (auto &th : pool) th.join();
  }
  for (int64_t v = 0; v < n; ++v) g->row_ptr[v + 1] += g->row_ptr[v];
  g->m = g->row_ptr[n];
  g->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)std::max<int64_t>(g->m, 1));
  if (!g->col) { free(tmp); pgi_csr_free(g); return nullptr; }
  next = 0;
  auto write_bucket = [&](int) {
    for (;;) {
      int64_t k = next.fetch_add(1);
      if (k >= B) break;
      const uint64_t *b = tmp + bstart[k];
      if (uniq[k] == 0) continue;
      int64_t pos = g->row_ptr[b[0] >> 32];
      for (int64_t i = 0; i < uniq[k]; ++i) g->col[pos + i] = (int32_t)(b[i] & 0xFFFFFFFFULL);
    }
  };
  {
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t) pool.emplace_back(write_bucket, t);
    for (auto &th : pool) th.join();
  }
  free(tmp);
  return g;
}

static inline uint64_t key(uint64_t src, uint64_t dst) { return (dst << 32) | src; }

// CSR over in-edges of the arc list src[i] -> dst[i]. Self-loops are kept
// when keep_self_loops is nonzero; duplicates are always removed.
pgi_csr *pgi_csr_from_arcs(int64_t n, int64_t count, const int32_t *src, const int32_t *dst,
                           int symmetrise, int keep_self_loops, int threads) {
  if (n <= 0 || n > 0x7FFFFFFFLL || count < 0) return nullptr;
  const int64_t total = symmetrise ? 2 * count : count;
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(total, 1));
  if (!keys) return nullptr;
  for (int64_t i = 0; i < count; ++i) {
    uint64_t u = (uint32_t)src[i], v = (uint32_t)dst[i];
    bool bad = (int64_t)u >= n || (int64_t)v >= n || (!keep_self_loops && u == v);
    keys[i] = bad ? kNone : key(u, v);
    if (symmetrise) keys[count + i] = bad ? kNone : key(v, u);
  }
  return build_from_keys(n, keys, total, threads);
}

// Undirected G(n, M) with M = round(n * avg_degree / 2) uniform pairs drawn
// with replacement; self-loops dropped, symmetrised, duplicates removed.
pgi_csr *pgi_er(int64_t n, double avg_degree, uint64_t seed, int threads) {
  if (n <= 0 || n > 0x7FFFFFFFLL || avg_degree < 0) return nullptr;
  const int64_t M = (int64_t)(n * avg_degree / 2.0 + 0.5);
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(2 * M, 1));
  if (!keys) return nullptr;
  parallel_for(M, pick_threads(threads), [&](int64_t b, int64_t e, int) {
    for (int64_t i = b; i < e; ++i) {
      uint64_t u = below(rng(seed, 0, 2 * (uint64_t)i), (uint64_t)n);
      uint64_t v = below(rng(seed, 0, 2 * (uint64_t)i + 1), (uint64_t)n);
      keys[i] = (u == v) ? kNone : key(u, v);
      keys[M + i] = (u == v) ? kNone : key(v, u);
    }
  });
  return build_from_keys(n, keys, 2 * M, threads);
}

// R-MAT (Chakrabarti, Zhan & Faloutsos 2004): 2^scale nodes, edge_factor *
// 2^scale edges, each placed by `scale` recursive quadrant choices with
// probabilities (a, b, c, 1-a-b-c), quantised to 16 bits per level. No noise,
// no vertex permutation. Self-loops dropped, duplicates removed. directed=1
// keeps arcs src->dst; directed=0 symmetrises.
pgi_csr *pgi_rmat(int scale, double edge_factor, double a, double b, double c, uint64_t seed,
                  int directed, int threads) {
  if (scale < 1 || scale > 30 || edge_factor < 0) return nullptr;
  const int64_t n = 1LL << scale;
  const int64_t M = (int64_t)(edge_factor * (double)n + 0.5);
  const uint32_t ta = (uint32_t)(a * 65536.0 + 0.5);
  const uint32_t tb = ta + (uint32_t)(b * 65536.0 + 0.5);
  const uint32_t tc = tb + (uint32_t)(c * 65536.0 + 0.5);
  const int64_t words_per_edge = (scale + 3) / 4;
  const int64_t total = directed ? M : 2 * M;
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(total, 1));
  if (!keys) return nullptr;
  parallel_for(M, pick_threads(threads), [&](int64_t bb, int64_t ee, int) {
    for (int64_t i = bb; i < ee; ++i) {
      uint64_t src = 0, dst = 0, r = 0;
      for (int l = 0; l < scale; ++l) {
        if ((l & 3) == 0) r = rng(seed, 1, (uint64_t)(i * words_per_edge + l / 4));
        uint32_t q = (uint32_t)(r & 0xFFFF);
        r >>= 16;
        uint64_t rb = (q >= tb) ? 1 : 0;                 // quadrants c, d: lower half
        uint64_t cb = (q >= ta && q < tb) || q >= tc;    // quadrants b, d: right half
        src = (src << 1) | rb;
        dst = (dst << 1) | cb;
      }
      bool loop = (src == dst);
      keys[i] = loop ? kNone : key(src, dst);
      if (!directed) keys[M + i] = loop ? kNone : key(dst, src);
    }
  });
  return build_from_keys(n, keys, total, threads);
}

// rows x cols 4-neighbour lattice; node (r, c) has id r * cols + c. Each of
// the lattice's undirected edges is deleted independently with probability
// p_delete. Symmetrised.
pgi_csr *pgi_grid(int64_t rows, int64_t cols, double p_delete, uint64_t seed, int threads) {
  if (rows <= 0 || cols <= 0 || rows * cols > 0x7FFFFFFFLL) return nullptr;
  const int64_t n = rows * cols;
  const int64_t H = rows * (cols - 1), V = (rows - 1) * cols, E = H + V;
  const double x = p_delete * 18446744073709551616.0;
  const uint64_t cut = x <= 0.0 ? 0 : (x >= 18446744073709551615.0 ? ~0ULL : (uint64_t)x);
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(2 * E, 1));
  if (!keys) return nullptr;
  parallel_for(E, pick_threads(threads), [&](int64_t b, int64_t e, int) {
    for (int64_t i = b; i < e; ++i) {
      uint64_t u, v;
      if (i < H) {
        int64_t r = i / (cols - 1), c = i % (cols - 1);
        u = r * cols + c;
        v = u + 1;
      } else {
        int64_t j = i - H, r = j / cols, c = j % cols;
        u = r * cols + c;
        v = u + cols;
      }
      bool del = rng(seed, 2, (uint64_t)i) < cut;
      keys[i] = del ? kNone : key(u, v);
      keys[E + i] = del ? kNone : key(v, u);
    }
  });
  return build_from_keys(n, keys, 2 * E, threads);
}

// s distinct nodes of [0, n), uniform without replacement (R. Floyd's
// sampling algorithm, Bentley & Floyd, CACM 1987). out[i] is the i-th node
// inserted. Returns 0 on success, -1 on bad arguments.
int pgi_seeds(int64_t n, int64_t s, uint64_t seed, int32_t *out) {
  if (n <= 0 || s < 0 || s > n || n > 0x7FFFFFFFLL) return -1;
  std::unordered_set<int64_t> taken;
  taken.reserve((size_t)s * 2);
  int64_t k = 0;
  for (int64_t j = n - s; j < n; ++j) {
    int64_t t = (int64_t)below(rng(seed, 3, (uint64_t)j), (uint64_t)(j + 1));
    int64_t pick = taken.count(t) ? j : t;
    taken.insert(pick);
    out[k++] = (int32_t)pick;
  }
  return 0;
}

}  // extern "C"
