// Seeded graph generators and the CSR builder, on the device.
//
// The synthetic graphs that stand in for the paper's datasets (Table 1:
// sparse uniform random, skewed web/social, long-diameter lattice) are drawn
// from one counter-based generator: value i of stream k under a seed is
// SplitMix64's output function (Steele, Lea and Flood, OOPSLA 2014) applied
// to key + (i + 1) * gamma, key itself SplitMix64 of the seed and stream.
// Every draw is addressable, so a thread per edge produces the same graph as
// any host implementation of the same definitions (the tests compare with
// the host generator byte for byte):
//   ER      G(n, M) with M = round(n d / 2) uniform pairs with replacement
//           (draws 2i and 2i+1 of stream 0), loops dropped, symmetrised;
//   R-MAT   2^scale nodes, round(ef 2^scale) edges, each by `scale`
//           quadrant choices with 16-bit thresholds (four levels per draw
//           of stream 1), loops dropped, symmetrised unless directed;
//   grid    rows x cols 4-neighbour lattice, edge i deleted when draw i of
//           stream 2 falls below p 2^64.
// Uniform integers in [0, n) take the high 64 bits of draw x n.
//
// CSR builder: every arc u -> v becomes the key (v << lg) | u (lg bits per
// id), a dropped arc all ones; a least-significant-digit radix sort over the
// key's 2 lg bits (8-bit digits, stable scatter per tile of 4096 keys) puts
// the arcs in (row, column) order with dropped ones last; unique keys are
// compacted by a scan, the columns read off them, and row v's start found by
// a binary search for the first key of row v. The arrays then become a
// pg_graph exactly as pg_graph_from_csr builds one (validation,
// relabelling, transpose).
#include <cstring>

#include "host.cuh"

namespace pg {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;
constexpr uint64_t kDrop = ~0ULL;
constexpr int kTile = 4096;  // keys per block tile of the radix sort
constexpr int kDigits = 256;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t i) {
  return mix64(key + kGamma * (i + 1));
}

uint64_t stream_key(uint64_t seed, uint64_t stream) {
  auto mix = [](uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  };
  return mix(mix(seed + kGamma) + kGamma * (stream + 1));
}

__device__ __forceinline__ uint64_t below(uint64_t x, uint64_t n) { return __umul64hi(x, n); }

__device__ __forceinline__ uint64_t arc_key(uint64_t src, uint64_t dst, int lg) {
  return (dst << lg) | src;
}

__global__ void k_gen_er(uint64_t key, int64_t n, int64_t M, int lg, uint64_t *keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t u = below(draw(key, 2 * (uint64_t)i), (uint64_t)n);
    const uint64_t v = below(draw(key, 2 * (uint64_t)i + 1), (uint64_t)n);
    keys[i] = u == v ? kDrop : arc_key(u, v, lg);
    keys[M + i] = u == v ? kDrop : arc_key(v, u, lg);
  }
}

__global__ void k_gen_rmat(uint64_t key, int scale, int64_t M, uint32_t ta, uint32_t tb,
                           uint32_t tc, int directed, int lg, uint64_t *keys) {
  const int64_t words = (scale + 3) / 4;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t src = 0, dst = 0, r = 0;
    for (int l = 0; l < scale; ++l) {
      if ((l & 3) == 0) r = draw(key, (uint64_t)(i * words + l / 4));
      const uint32_t q = (uint32_t)(r & 0xFFFF);
      r >>= 16;
      const uint64_t rb = q >= tb ? 1 : 0;                       // quadrants c, d: lower half
      const uint64_t cb = ((q >= ta && q < tb) || q >= tc) ? 1 : 0;  // b, d: right half
      src = (src << 1) | rb;
      dst = (dst << 1) | cb;
    }
    const bool loop = src == dst;
    keys[i] = loop ? kDrop : arc_key(src, dst, lg);
    if (!directed) keys[M + i] = loop ? kDrop : arc_key(dst, src, lg);
  }
}

__global__ void k_gen_grid(uint64_t key, int64_t rows, int64_t cols, uint64_t cut, int lg,
                           uint64_t *keys) {
  const int64_t H = rows * (cols - 1), E = H + (rows - 1) * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t u, v;
    if (i < H) {
      const int64_t r = i / (cols - 1), c = i % (cols - 1);
      u = (uint64_t)(r * cols + c);
      v = u + 1;
    } else {
      const int64_t j = i - H, r = j / cols, c = j % cols;
      u = (uint64_t)(r * cols + c);
      v = u + (uint64_t)cols;
    }
    const bool del = draw(key, (uint64_t)i) < cut;
    keys[i] = del ? kDrop : arc_key(u, v, lg);
    keys[E + i] = del ? kDrop : arc_key(v, u, lg);
  }
}

// Radix sort pass: digit counts per tile, digit-major (H[d * tiles + tile]).
__global__ void __launch_bounds__(kBlock) k_radix_hist(const uint64_t *keys, int64_t count,
                                                       int shift, int64_t tiles, int64_t *H) {
  __shared__ uint32_t h[kDigits];
  for (int d = threadIdx.x; d < kDigits; d += kBlock) h[d] = 0u;
  __syncthreads();
  const int64_t k0 = (int64_t)blockIdx.x * kTile;
  for (int i = threadIdx.x; i < kTile; i += kBlock) {
    const int64_t k = k0 + i;
    if (k < count) atomicAdd(&h[(keys[k] >> shift) & (kDigits - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kDigits; d += kBlock) H[(int64_t)d * tiles + blockIdx.x] = h[d];
}

// Stable scatter of one pass: a key goes to the scanned H[d * tiles + tile]
// plus the number of earlier keys of its tile with the same digit; the tile
// is walked in order, kBlock keys per step, warps counting their digit peers
// with match_any and adding the counts of the warps before them.
__global__ void __launch_bounds__(kBlock) k_radix_scatter(const uint64_t *in, uint64_t *out,
                                                          int64_t count, int shift,
                                                          int64_t tiles, const int64_t *H) {
  constexpr int kWarps = kBlock / 32;
  __shared__ int64_t base[kDigits];
  __shared__ uint16_t wcnt[kWarps][kDigits];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kDigits; d += kBlock) base[d] = H[(int64_t)d * tiles + blockIdx.x];
  const int64_t k0 = (int64_t)blockIdx.x * kTile;
  for (int i0 = 0; i0 < kTile; i0 += kBlock) {
    const int64_t k = k0 + i0 + threadIdx.x;
    const bool valid = k < count;
    const uint64_t key = valid ? in[k] : 0ULL;
    const int d = valid ? (int)((key >> shift) & (kDigits - 1)) : -1;
    const unsigned peers = __match_any_sync(kFullMask, d);
    const unsigned below = peers & ((1u << lane) - 1u);
    __syncthreads();
    for (int j = threadIdx.x; j < kWarps * kDigits; j += kBlock) (&wcnt[0][0])[j] = 0;
    __syncthreads();
    if (valid && below == 0u) wcnt[w][d] = (uint16_t)__popc(peers);
    __syncthreads();
    if (valid) {
      int64_t pos = base[d] + __popc(below);
      for (int j = 0; j < w; ++j) pos += wcnt[j][d];
      out[pos] = key;
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < kDigits; dd += kBlock) {
      int64_t add = 0;
      for (int j = 0; j < kWarps; ++j) add += wcnt[j][dd];
      base[dd] += add;
    }
  }
}

// 1 for the first of each run of equal keys (dropped arcs excluded).
__global__ void k_unique_flags(const uint64_t *keys, int64_t count, int64_t *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = keys[i] != kDrop && (i == 0 || keys[i - 1] != keys[i]) ? 1 : 0;
}

__global__ void k_unique_compact(const uint64_t *keys, int64_t count, const int64_t *pos,
                                 int lg, uint64_t *ukeys, int32_t *col) {
  const uint64_t mask = (1ULL << lg) - 1ULL;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    if (k != kDrop && (i == 0 || keys[i - 1] != k)) {
      ukeys[pos[i]] = k;
      col[pos[i]] = (int32_t)(k & mask);
    }
  }
}

// row_ptr[v] = the first unique key of row v or later (binary search).
__global__ void k_row_starts(const uint64_t *ukeys, int64_t m, int64_t n, int lg,
                             int64_t *row_ptr) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t want = (uint64_t)v << lg;
    int64_t lo = 0, hi = m;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (ukeys[mid] < want) lo = mid + 1; else hi = mid;
    }
    row_ptr[v] = lo;
  }
}

int grid_of(int64_t work) {
  const int64_t need = (work + kBlock - 1) / kBlock;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sm_count() * 8));
}

}  // namespace
}  // namespace pg

using namespace pg;

extern "C" pg_status pg_graph_generate(const pg_generator *gen, unsigned flags, void *stream,
                                       pg_graph **out) {
  if (!gen || !out || (flags & (PG_DEVICE_PTRS | PG_BORROW))) return PG_EINVAL;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t n = 0, total = 0;
  int directed = 0;
  if (gen->kind == PG_GEN_ER) {
    if (gen->n < 1 || gen->n > 0x7FFFFFFFLL || !(gen->avg_degree >= 0.0)) return PG_EINVAL;
    n = gen->n;
    total = 2 * (int64_t)((double)n * gen->avg_degree / 2.0 + 0.5);
  } else if (gen->kind == PG_GEN_RMAT) {
    if (gen->scale < 1 || gen->scale > 30 || !(gen->edge_factor >= 0.0) || gen->a < 0 ||
        gen->b < 0 || gen->c < 0 || gen->a + gen->b + gen->c > 1.0)
      return PG_EINVAL;
    n = 1LL << gen->scale;
    directed = gen->directed ? 1 : 0;
    const int64_t M = (int64_t)(gen->edge_factor * (double)n + 0.5);
    total = directed ? M : 2 * M;
  } else if (gen->kind == PG_GEN_GRID) {
    if (gen->rows < 1 || gen->cols < 1 || gen->rows * gen->cols > 0x7FFFFFFFLL ||
        !(gen->p_delete >= 0.0))
      return PG_EINVAL;
    n = gen->rows * gen->cols;
    total = 2 * (gen->rows * (gen->cols - 1) + (gen->rows - 1) * gen->cols);
  } else {
    return PG_EINVAL;
  }
  if (n > kMaxNodes || total > kMaxArcs) return PG_EINVAL;  // as pg_graph_from_csr
  int lg = 1;
  while ((1LL << lg) < n) ++lg;
  const int bits = 2 * lg;
  uint64_t *a = nullptr, *b = nullptr;
  int64_t *aux = nullptr, *row_ptr = nullptr;
  int32_t *col = nullptr;
  const int64_t tiles = (total + kTile - 1) / kTile;
  pg_status rc = cuda_status(cudaMallocAsync((void **)&a, sizeof(uint64_t) * std::max<int64_t>(total, 1), st));
  if (!rc) rc = cuda_status(cudaMallocAsync((void **)&b, sizeof(uint64_t) * std::max<int64_t>(total, 1), st));
  if (!rc)
    rc = cuda_status(cudaMallocAsync(
        (void **)&aux, sizeof(int64_t) * std::max<int64_t>(std::max<int64_t>(total + 1, tiles * kDigits), 1), st));
  // draw the arcs
  if (!rc && total > 0) {
    const int grid = grid_of(total / 2 + 1);
    if (gen->kind == PG_GEN_ER) {
      k_gen_er<<<grid, kBlock, 0, st>>>(stream_key(gen->seed, 0), n, total / 2, lg, a);
    } else if (gen->kind == PG_GEN_RMAT) {
      const uint32_t ta = (uint32_t)(gen->a * 65536.0 + 0.5);
      const uint32_t tb = ta + (uint32_t)(gen->b * 65536.0 + 0.5);
      const uint32_t tc = tb + (uint32_t)(gen->c * 65536.0 + 0.5);
      const int64_t M = directed ? total : total / 2;
      k_gen_rmat<<<grid, kBlock, 0, st>>>(stream_key(gen->seed, 1), gen->scale, M, ta, tb, tc,
                                          directed, lg, a);
    } else {
      const double x = gen->p_delete * 18446744073709551616.0;
      const uint64_t cut =
          x <= 0.0 ? 0 : (x >= 18446744073709551615.0 ? ~0ULL : (uint64_t)x);
      k_gen_grid<<<grid, kBlock, 0, st>>>(stream_key(gen->seed, 2), gen->rows, gen->cols, cut, lg,
                                          a);
    }
    rc = cuda_status(cudaGetLastError());
  }
  // sort the keys by their 2 lg bits, 8 at a time
  for (int shift = 0; !rc && total > 0 && shift < bits; shift += 8) {
    k_radix_hist<<<(unsigned)tiles, kBlock, 0, st>>>(a, total, shift, tiles, aux);
    rc = cuda_status(cudaGetLastError());
    if (!rc) rc = exclusive_scan_i64(aux, tiles * kDigits, st);
    if (!rc) {
      k_radix_scatter<<<(unsigned)tiles, kBlock, 0, st>>>(a, b, total, shift, tiles, aux);
      rc = cuda_status(cudaGetLastError());
    }
    std::swap(a, b);
  }
  // unique arcs: positions by a scan of first-of-run flags
  int64_t m = 0;
  if (!rc && total > 0) {
    k_unique_flags<<<grid_of(total), kBlock, 0, st>>>(a, total, aux);
    cudaMemsetAsync(aux + total, 0, sizeof(int64_t), st);
    rc = cuda_status(cudaGetLastError());
    if (!rc) rc = exclusive_scan_i64(aux, total + 1, st);
    if (!rc) rc = cuda_status(cudaMemcpyAsync(&m, aux + total, sizeof(int64_t),
                                              cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
  }
  if (!rc) rc = cuda_status(cudaMalloc((void **)&row_ptr, sizeof(int64_t) * (size_t)(n + 1)));
  if (!rc) rc = cuda_status(cudaMalloc((void **)&col, sizeof(int32_t) * (size_t)std::max<int64_t>(m, 1)));
  if (!rc && total > 0) {
    k_unique_compact<<<grid_of(total), kBlock, 0, st>>>(a, total, aux, lg, b, col);
    k_row_starts<<<grid_of(n + 1), kBlock, 0, st>>>(b, m, n, lg, row_ptr);
    rc = cuda_status(cudaGetLastError());
  } else if (!rc) {
    rc = cuda_status(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t) * (size_t)(n + 1), st));
  }
  if (a) cudaFreeAsync(a, st);
  if (b) cudaFreeAsync(b, st);
  if (aux) cudaFreeAsync(aux, st);
  if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
  // the graph: built on these arrays in place; they become the graph's own
  // unless relabelling or PG_HOST_CSR replaced them by new ones
  pg_graph *g = nullptr;
  if (!rc)
    rc = pg_graph_from_csr(row_ptr, col, n, m, directed,
                           (flags & ~(PG_HOST_CSR)) | PG_DEVICE_PTRS | PG_BORROW, stream, &g);
  if (rc) {
    if (row_ptr) cudaFree(row_ptr);
    if (col) cudaFree(col);
    return rc;
  }
  if (g->row_ptr == row_ptr) {  // the graph's in-CSR
    g->owns_in = true;
  } else if (g->out_ptr == row_ptr) {  // PG_REVERSE: its out-CSR
    g->owns_out = true;
  } else {  // relabelled: the graph holds its renumbered copy
    cudaFree(row_ptr);
    cudaFree(col);
  }
  *out = g;
  return PG_OK;
}

extern "C" pg_status pg_graph_copy_csr(const pg_graph *g, int64_t *row_ptr, int32_t *col,
                                       void *stream) {
  if (!g || !row_ptr || (g->m > 0 && !col)) return PG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  pg_status rc = cuda_status(cudaMemcpyAsync(row_ptr, g->row_ptr, sizeof(int64_t) * (size_t)(g->n + 1),
                                             cudaMemcpyDefault, st));
  if (!rc && g->m > 0)
    rc = cuda_status(cudaMemcpyAsync(col, g->col, sizeof(int32_t) * (size_t)g->m,
                                     cudaMemcpyDefault, st));
  if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
  return rc;
}
