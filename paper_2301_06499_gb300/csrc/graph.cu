// Graph construction: copy-in, on-device CSR validation, out-edge transpose,
// and the dense work list (every row cut into pieces of at most L arcs).
#include <algorithm>
#include <cstring>
#include <mutex>

#include <vector>

#include "host.cuh"

namespace pg {

pg_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return PG_OK;
  if (e == cudaErrorMemoryAllocation) return PG_ENOMEM;
  return PG_ECUDA;
}

// Sum over the warp (every lane gets it).
__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(kFullMask, x, off);
  return x;
}

pg_status ensure(DevBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes && !b.host) return PG_OK;
  if (b.p) {
    if (b.host)
      cudaFreeHost(b.p);
    else
      cudaFree(b.p);
  }
  b.p = nullptr;
  b.bytes = 0;
  b.host = false;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return cuda_status(e);
  }
  b.bytes = bytes;
  return PG_OK;
}

pg_status ensure_host(DevBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes && b.host) return PG_OK;
  release(b);
  cudaError_t e = cudaMallocHost(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return cuda_status(e);
  }
  b.bytes = bytes;
  b.host = true;
  return PG_OK;
}

void release(DevBuf &b) {
  if (b.p) {
    if (b.host)
      cudaFreeHost(b.p);
    else
      cudaFree(b.p);
  }
  b.p = nullptr;
  b.bytes = 0;
  b.host = false;
}

// Arc arrays of a graph: device memory, or pinned host memory (PG_HOST_CSR).
static cudaError_t alloc_arcs(void **p, size_t bytes, bool host) {
  return host ? cudaMallocHost(p, bytes) : cudaMalloc(p, bytes);
}

static void free_arcs(void *p, bool host) {
  if (!p) return;
  if (host)
    cudaFreeHost(p);
  else
    cudaFree(p);
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

int64_t l2_bytes() {
  int dev = 0, l2 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  return l2 > 0 ? l2 : (int64_t)128 << 20;
}

static int grid_for(int64_t work, int per_sm = 8) {
  int64_t cap = (int64_t)sm_count() * per_sm;
  int64_t need = (work + kBlock - 1) / kBlock;
  return (int)std::max<int64_t>(1, std::min(cap, need));
}

// ------------------------------------------------------------------ scan
constexpr int kScanPerThread = 8;
constexpr int kScanTile = kBlock * kScanPerThread;

__global__ void __launch_bounds__(kBlock) k_scan_tile(int64_t *data, int64_t n, int64_t *sums) {
  __shared__ int64_t warp_tot[kBlock / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPerThread;
  int64_t v[kScanPerThread];
  int64_t run = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    int64_t i = base + k;
    int64_t x = i < n ? data[i] : 0;
    v[k] = run;  // exclusive within the thread
    run += x;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t incl = run;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    int64_t y = __shfl_up_sync(kFullMask, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int64_t t = lane < kBlock / 32 ? warp_tot[lane] : 0;
    int64_t ti = t;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int64_t y = __shfl_up_sync(kFullMask, ti, off);
      if (lane >= off) ti += y;
    }
    if (lane < kBlock / 32) warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == kBlock / 32 - 1 && sums) sums[blockIdx.x] = ti;
  }
  __syncthreads();
  const int64_t off = warp_tot[w] + (incl - run);
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    int64_t i = base + k;
    if (i < n) data[i] = v[k] + off;
  }
}

__global__ void k_scan_add(int64_t *data, int64_t n, const int64_t *sums) {
  const int64_t tile = blockIdx.x;
  const int64_t add = sums[tile];
  const int64_t end = (tile + 1) * kScanTile < n ? (tile + 1) * kScanTile : n;
  for (int64_t i = tile * kScanTile + threadIdx.x; i < end; i += blockDim.x)
    data[i] += add;
}

pg_status exclusive_scan_i64(int64_t *data, int64_t n, cudaStream_t st) {
  if (n <= 0) return PG_OK;
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    k_scan_tile<<<1, kBlock, 0, st>>>(data, n, nullptr);
    return cuda_status(cudaGetLastError());
  }
  int64_t *sums = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&sums, sizeof(int64_t) * tiles, st);
  if (e != cudaSuccess) return cuda_status(e);
  k_scan_tile<<<(unsigned)tiles, kBlock, 0, st>>>(data, n, sums);
  pg_status rc = cuda_status(cudaGetLastError());
  if (rc == PG_OK) rc = exclusive_scan_i64(sums, tiles, st);
  if (rc == PG_OK) {
    k_scan_add<<<(unsigned)tiles, kBlock, 0, st>>>(data, n, sums);
    rc = cuda_status(cudaGetLastError());
  }
  cudaFreeAsync(sums, st);
  return rc;
}

// ------------------------------------------------------------ validation
// err bits: 1 row_ptr[0] != 0, 2 non-monotone / past m, 4 col out of range,
// 8 row not strictly increasing (set on the host), 16 row_ptr[n] != m.
// CSR validation in two flat passes (coalesced) and a count: the arcs pass
// counts descents (positions j > 0 with col[j-1] >= col[j]) into cnt[0]; the
// rows pass checks each row's bounds and counts the nonempty rows whose
// first arc is a descent into cnt[1]. The nonempty rows of a valid row_ptr
// start at distinct positions, so the two counts are equal exactly when
// every descent is the first arc of a row, i.e. when every row's columns
// strictly increase.
__global__ void k_validate_rows(const int64_t *rp, const int32_t *col, int64_t n, int64_t m,
                                unsigned long long *cnt, int *err) {
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  if (gtid == 0) {
    if (rp[0] != 0) atomicOr(err, 1);
    if (rp[n] != m) atomicOr(err, 16);
  }
  unsigned long long starts = 0;
  for (int64_t v = gtid; v < n; v += nth) {
    const int64_t b = rp[v], e = rp[v + 1];
    if (b > e || b < 0 || e > m)
      atomicOr(err, 2);
    else if (b < e && b > 0 && col[b - 1] >= col[b])
      ++starts;
  }
  const unsigned long long tot = warp_sum64(starts);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&cnt[1], tot);
}

__global__ void k_validate_arcs(const int32_t *col, int64_t n, int64_t m, unsigned long long *cnt,
                                int *err) {
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t nq = m / 4;  // whole quads, read as int4 (the array is 256-byte aligned)
  const int4 *q4 = reinterpret_cast<const int4 *>(col);
  unsigned long long desc = 0;
  bool out = false;
  for (int64_t q = gtid; q < nq; q += nth) {
    const int4 c = q4[q];
    const int32_t prev = q > 0 ? col[4 * q - 1] : INT32_MIN;
    out |= c.x < 0 || c.x >= n || c.y < 0 || c.y >= n || c.z < 0 || c.z >= n || c.w < 0 ||
           c.w >= n;
    desc += (q > 0 && prev >= c.x) + (c.x >= c.y) + (c.y >= c.z) + (c.z >= c.w);
  }
  if (gtid == 0)  // the last m % 4 arcs
    for (int64_t j = nq * 4; j < m; ++j) {
      const int32_t c = col[j];
      out |= c < 0 || c >= n;
      desc += j > 0 && col[j - 1] >= c;
    }
  if (out) atomicOr(err, 4);
  const unsigned long long tot = warp_sum64(desc);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&cnt[0], tot);
}

// --------------------------------------------------------------- transpose
__global__ void k_count_out(const int32_t *col, int64_t m, unsigned long long *cnt) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
       j += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[col[j]], 1ULL);
}

// Transpose scatter over row pieces of at most kScatterPiece arcs, a thread
// per piece. Rows are sorted, so at step k the lanes of a warp often hold the
// same source (a hub): lanes with equal sources take their slots with one
// fetch-and-add by the lowest of them, which keeps hub cursors uncontended.
constexpr int kScatterPiece = 32;

__global__ void __launch_bounds__(kBlock) k_scatter_out(const ulonglong2 *pieces, int64_t np,
                                                        const int32_t *col,
                                                        unsigned long long *cursor,
                                                        int32_t *out_col) {
  const int lane = threadIdx.x & 31;
  const int64_t nth = (int64_t)gridDim.x * kBlock;
  // whole warps iterate, so that the lane matching sees every lane
  for (int64_t base = ((int64_t)blockIdx.x * kBlock + threadIdx.x) & ~31LL; base < np;
       base += nth) {
    const int64_t i = base + lane;
    int64_t first = 0;
    int32_t v = 0;
    int len = 0;
    if (i < np) {
      const ulonglong2 it = pieces[i];
      first = (int64_t)it.x;
      v = (int32_t)(it.y >> 32);
      len = (int)(it.y & 0x7FFFFFFFULL);
    }
    int most = len;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) most = max(most, __shfl_xor_sync(kFullMask, most, off));
    for (int k = 0; k < most; ++k) {
      const int32_t u = k < len ? __ldg(col + first + k) : -1;
      const unsigned peers = __match_any_sync(kFullMask, u);
      const int leader = __ffs(peers) - 1;
      unsigned long long pos = 0;
      if (u >= 0 && lane == leader)
        pos = atomicAdd(&cursor[u], (unsigned long long)__popc(peers));
      pos = __shfl_sync(kFullMask, pos, leader);
      if (u >= 0) out_col[pos + __popc(peers & ((1u << lane) - 1u))] = v;
    }
  }
}

__global__ void k_max_degree(const int64_t *rp, int64_t n, unsigned long long *mx) {
  unsigned long long best = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    best = max(best, (unsigned long long)(rp[v + 1] - rp[v]));
  atomicMax(mx, best);
}

// ------------------------------------------------------------- work list
__global__ void k_piece_count(const int64_t *rp, int64_t n, int32_t L, int64_t *np) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = rp[v + 1] - rp[v];
    np[v] = (d + L - 1) / L;
  }
}

__global__ void k_piece_fill(const int64_t *rp, const int64_t *np_ex, int64_t n, int32_t L,
                             ulonglong2 *list) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = np_ex[v], e = np_ex[v + 1];
    const int64_t rb = rp[v], d = rp[v + 1] - rb;
    for (int64_t k = b; k < e; ++k) {
      const int64_t q = k - b;
      list[k] = make_item((int32_t)v, rb + q * L, min((int64_t)L, d - q * L), e - b == 1);
    }
  }
}

pg_status ensure_pieces(pg_graph *g, int32_t L, cudaStream_t st) {
  if (g->pieces.L == L && g->pieces.list.p) return PG_OK;
  int64_t *np = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&np, sizeof(int64_t) * (g->n + 1), st);
  if (e != cudaSuccess) return cuda_status(e);
  k_piece_count<<<grid_for(g->n), kBlock, 0, st>>>(g->row_ptr, g->n, L, np);
  cudaMemsetAsync(np + g->n, 0, sizeof(int64_t), st);
  pg_status rc = exclusive_scan_i64(np, g->n + 1, st);
  int64_t total = 0;
  if (rc == PG_OK)
    rc = cuda_status(cudaMemcpyAsync(&total, np + g->n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  if (rc == PG_OK) rc = cuda_status(cudaStreamSynchronize(st));
  if (rc == PG_OK) rc = ensure(g->pieces.list, sizeof(ulonglong2) * (size_t)std::max<int64_t>(total, 1));
  if (rc == PG_OK) {
    k_piece_fill<<<grid_for(g->n), kBlock, 0, st>>>(g->row_ptr, np, g->n, L,
                                                    (ulonglong2 *)g->pieces.list.p);
    rc = cuda_status(cudaGetLastError());
  }
  cudaFreeAsync(np, st);
  if (rc == PG_OK) rc = cuda_status(cudaStreamSynchronize(st));
  if (rc == PG_OK) {
    g->pieces.L = L;
    g->pieces.count = total;
  } else {
    g->pieces.L = 0;
  }
  return rc;
}

// ------------------------------------------------------------ sliced ELL
// Packed batch: bucket (graph, Lmax - len), so that each graph's pieces are
// contiguous (longest first) and can be padded to whole chunks.
__global__ void k_sell_hist_seg(const ulonglong2 *pieces, int64_t np, int32_t Lmax,
                                const int32_t *seg_of, unsigned long long *hist) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const ulonglong2 it = pieces[i];
    const int len = (int)(it.y & 0x7FFFFFFFULL);
    const int32_t v = (int32_t)(it.y >> 32);
    atomicAdd(&hist[(int64_t)seg_of[v] * (Lmax + 1) + (Lmax - len)], 1ULL);
  }
}

__global__ void k_sell_scatter_seg(const ulonglong2 *pieces, int64_t np, int32_t Lmax,
                                   const int32_t *seg_of, unsigned long long *cursor,
                                   ulonglong2 *sorted) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const ulonglong2 it = pieces[i];
    const int len = (int)(it.y & 0x7FFFFFFFULL);
    const int32_t v = (int32_t)(it.y >> 32);
    sorted[atomicAdd(&cursor[(int64_t)seg_of[v] * (Lmax + 1) + (Lmax - len)], 1ULL)] = it;
  }
}

// One graph: a counting sort of the pieces by length, longest first, with
// block-local counters. Block b takes a contiguous range of the (row-ordered)
// piece list; k_sell_bhist counts its pieces per length into bh[len' * B + b]
// (len' = Lmax - len), whose exclusive scan is where block b's pieces of each
// length start; k_sell_bscatter places them there, the lanes of a warp with
// equal lengths taking consecutive slots with one shared-memory atomic. (One
// global atomic per piece on a handful of bucket counters serialised at the
// L2: 62 ms for the ~10^8 pieces of a scale-26 R-MAT.)
__global__ void __launch_bounds__(kBlock) k_sell_bhist(const ulonglong2 *pieces, int64_t np,
                                                       int32_t Lmax, int64_t per_block,
                                                       int64_t *bh) {
  __shared__ uint32_t h[kSellPiece + 1];
  for (int k = threadIdx.x; k <= Lmax; k += kBlock) h[k] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t lo = (int64_t)blockIdx.x * per_block, hi = min(np, lo + per_block);
  for (int64_t base = lo; base < hi; base += kBlock) {  // block-uniform trip count
    const int64_t i = base + threadIdx.x;
    const int key = i < hi ? Lmax - (int)(pieces[i].y & 0x7FFFFFFFULL) : -1;
    const unsigned peers = __match_any_sync(kFullMask, key);
    if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&h[key], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int k = threadIdx.x; k <= Lmax; k += kBlock) bh[(int64_t)k * gridDim.x + blockIdx.x] = h[k];
}

__global__ void __launch_bounds__(kBlock) k_sell_bscatter(const ulonglong2 *pieces, int64_t np,
                                                          int32_t Lmax, int64_t per_block,
                                                          const int64_t *bh,
                                                          ulonglong2 *sorted) {
  __shared__ int64_t start[kSellPiece + 1];
  __shared__ uint32_t used[kSellPiece + 1];
  for (int k = threadIdx.x; k <= Lmax; k += kBlock) {
    start[k] = bh[(int64_t)k * gridDim.x + blockIdx.x];
    used[k] = 0u;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t lo = (int64_t)blockIdx.x * per_block, hi = min(np, lo + per_block);
  for (int64_t base = lo; base < hi; base += kBlock) {
    const int64_t i = base + threadIdx.x;
    ulonglong2 it = make_ulonglong2(0ULL, 0ULL);
    int key = -1;
    if (i < hi) {
      it = pieces[i];
      key = Lmax - (int)(it.y & 0x7FFFFFFFULL);
    }
    const unsigned peers = __match_any_sync(kFullMask, key);
    const int leader = __ffs(peers) - 1;
    uint32_t at = 0;
    if (key >= 0 && lane == leader) at = atomicAdd(&used[key], (uint32_t)__popc(peers));
    at = __shfl_sync(kFullMask, at, leader);
    if (key >= 0) sorted[start[key] + at + __popc(peers & ((1u << lane) - 1u))] = it;
  }
}

// chunk c: longest piece is lane 0's (sorted); slots = 32 x that length
__global__ void k_sell_chunks(const ulonglong2 *sorted, int64_t np, int64_t nchunks,
                              int32_t *clen, int64_t *coff) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nchunks;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int len = (int)(sorted[c * 32].y & 0x7FFFFFFFULL);
    clen[c] = len;
    coff[c] = 32LL * len;
  }
  (void)np;
}

__global__ void k_sell_fill(const ulonglong2 *sorted, int64_t nchunks, const int32_t *clen,
                            const int64_t *coff, const int32_t *col, int32_t *scol) {
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t w = gtid; w < nchunks * 32; w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = w >> 5;
    const int lane = (int)(w & 31);
    const ulonglong2 it = sorted[w];
    const int len = (int)(it.y & 0x7FFFFFFFULL);
    const int64_t first = (int64_t)it.x;
    const int cl = clen[c];
    int32_t *dst = scol + coff[c] + lane;
    for (int k = 0; k < cl; ++k) dst[32LL * k] = k < len ? col[first + k] : -1;
  }
}

pg_status ensure_sell(pg_graph *g, int32_t Lmax, cudaStream_t st) {
  SellList &sl = g->sell;
  if (sl.Lmax == Lmax && sl.items.p) return PG_OK;
  if (Lmax < 1 || Lmax > kSellPiece) return PG_EINVAL;  // the sort's shared counters
  // pieces of at most Lmax arcs, in row order (the cached piece list is reused
  // as scratch and rebuilt on its next use)
  PieceList saved;
  std::swap(saved, g->pieces);
  pg_status rc = ensure_pieces(g, Lmax, st);
  PieceList tmp;
  std::swap(tmp, g->pieces);
  std::swap(saved, g->pieces);
  if (rc) {
    release(tmp.list);
    return rc;
  }
  const int64_t np = tmp.count;
  int64_t nchunks = (np + 31) / 32;
  unsigned long long *hist = nullptr;
  int64_t *coff_tmp = nullptr;
  if (g->seg_of && g->nseg > 0) {
    // a packed batch: each graph's pieces sorted by length and padded to
    // whole chunks, so that a chunk belongs to one graph
    const int64_t nb = (int64_t)g->nseg * (Lmax + 1);
    std::vector<unsigned long long> h((size_t)nb);
    rc = cuda_status(cudaMallocAsync((void **)&hist, sizeof(unsigned long long) * nb, st));
    if (rc == PG_OK) {
      cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * nb, st);
      k_sell_hist_seg<<<grid_for(np), kBlock, 0, st>>>((const ulonglong2 *)tmp.list.p, np, Lmax,
                                                       g->seg_of, hist);
      rc = cuda_status(cudaGetLastError());
    }
    if (rc == PG_OK)
      rc = cuda_status(cudaMemcpyAsync(h.data(), hist, sizeof(unsigned long long) * nb,
                                       cudaMemcpyDeviceToHost, st));
    if (rc == PG_OK) rc = cuda_status(cudaStreamSynchronize(st));
    std::vector<int32_t> chunk_seg;
    std::vector<int64_t> chunk0((size_t)g->nseg + 1, 0);
    unsigned long long base = 0;
    for (int32_t k = 0; rc == PG_OK && k < g->nseg; ++k) {
      chunk0[(size_t)k] = (int64_t)(base / 32);
      unsigned long long run = base;
      for (int32_t b = 0; b <= Lmax; ++b) {
        const unsigned long long c = h[(size_t)k * (Lmax + 1) + b];
        h[(size_t)k * (Lmax + 1) + b] = run;
        run += c;
      }
      const unsigned long long padded = (run - base + 31) / 32 * 32;
      chunk_seg.insert(chunk_seg.end(), (size_t)(padded / 32), k);
      base += padded;
    }
    nchunks = (int64_t)(base / 32);
    chunk0[(size_t)g->nseg] = nchunks;
    if (rc == PG_OK) rc = ensure(sl.chunk0, sizeof(int64_t) * chunk0.size());
    if (rc == PG_OK)
      rc = cuda_status(cudaMemcpyAsync(sl.chunk0.p, chunk0.data(), sizeof(int64_t) * chunk0.size(),
                                       cudaMemcpyHostToDevice, st));
    if (rc == PG_OK) rc = ensure(sl.items, sizeof(ulonglong2) * (size_t)std::max<int64_t>(nchunks * 32, 1));
    if (rc == PG_OK) rc = ensure(sl.off, sizeof(int64_t) * (size_t)(nchunks + 1));
    if (rc == PG_OK) rc = ensure(sl.len, sizeof(int32_t) * (size_t)std::max<int64_t>(nchunks, 1));
    if (rc == PG_OK) rc = ensure(sl.seg, sizeof(int32_t) * (size_t)std::max<int64_t>(nchunks, 1));
    if (rc == PG_OK && nchunks > 0)
      rc = cuda_status(cudaMemcpyAsync(sl.seg.p, chunk_seg.data(), sizeof(int32_t) * nchunks,
                                       cudaMemcpyHostToDevice, st));
    if (rc == PG_OK)
      rc = cuda_status(cudaMemcpyAsync(hist, h.data(), sizeof(unsigned long long) * nb,
                                       cudaMemcpyHostToDevice, st));
    if (rc == PG_OK) {
      cudaMemsetAsync(sl.items.p, 0, sizeof(ulonglong2) * (size_t)std::max<int64_t>(nchunks * 32, 1), st);
      k_sell_scatter_seg<<<grid_for(np), kBlock, 0, st>>>((const ulonglong2 *)tmp.list.p, np, Lmax,
                                                          g->seg_of, hist,
                                                          (ulonglong2 *)sl.items.p);
      k_sell_chunks<<<grid_for(nchunks), kBlock, 0, st>>>((const ulonglong2 *)sl.items.p, np,
                                                          nchunks, (int32_t *)sl.len.p,
                                                          (int64_t *)sl.off.p);
      cudaMemsetAsync((int64_t *)sl.off.p + nchunks, 0, sizeof(int64_t), st);
      rc = cuda_status(cudaGetLastError());
    }
    if (rc == PG_OK) rc = cuda_status(cudaStreamSynchronize(st));  // h outlives the copy
  } else {
    release(sl.seg);
    release(sl.chunk0);
    // blocks of the counting sort: contiguous ranges of >= 4096 pieces
    const int64_t nblk = std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * 8,
                                                                (np + 4095) / 4096));
    const int64_t per_block = (np + nblk - 1) / nblk;
    const int64_t nbh = (int64_t)(Lmax + 1) * nblk + 1;
    rc = cuda_status(cudaMallocAsync((void **)&hist, sizeof(int64_t) * nbh, st));
    if (rc == PG_OK) rc = ensure(sl.items, sizeof(ulonglong2) * (size_t)std::max<int64_t>(nchunks * 32, 1));
    if (rc == PG_OK) rc = ensure(sl.off, sizeof(int64_t) * (size_t)(nchunks + 1));
    if (rc == PG_OK) rc = ensure(sl.len, sizeof(int32_t) * (size_t)std::max<int64_t>(nchunks, 1));
    if (rc == PG_OK) {
      cudaMemsetAsync(hist, 0, sizeof(int64_t) * nbh, st);
      // padding slots: zero-length items of row 0 (never active)
      cudaMemsetAsync(sl.items.p, 0, sizeof(ulonglong2) * (size_t)std::max<int64_t>(nchunks * 32, 1), st);
      k_sell_bhist<<<(unsigned)nblk, kBlock, 0, st>>>((const ulonglong2 *)tmp.list.p, np, Lmax,
                                                      per_block, (int64_t *)hist);
      rc = exclusive_scan_i64((int64_t *)hist, nbh, st);
    }
    if (rc == PG_OK) {
      k_sell_bscatter<<<(unsigned)nblk, kBlock, 0, st>>>((const ulonglong2 *)tmp.list.p, np, Lmax,
                                                         per_block, (const int64_t *)hist,
                                                         (ulonglong2 *)sl.items.p);
      k_sell_chunks<<<grid_for(nchunks), kBlock, 0, st>>>((const ulonglong2 *)sl.items.p, np,
                                                          nchunks, (int32_t *)sl.len.p,
                                                          (int64_t *)sl.off.p);
      cudaMemsetAsync((int64_t *)sl.off.p + nchunks, 0, sizeof(int64_t), st);
      rc = cuda_status(cudaGetLastError());
    }
  }
  if (rc == PG_OK) rc = exclusive_scan_i64((int64_t *)sl.off.p, nchunks + 1, st);
  int64_t slots = 0;
  if (rc == PG_OK)
    rc = cuda_status(cudaMemcpyAsync(&slots, (int64_t *)sl.off.p + nchunks, sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st));
  if (rc == PG_OK) rc = cuda_status(cudaStreamSynchronize(st));
  if (rc == PG_OK) {
    const size_t cb = sizeof(int32_t) * (size_t)std::max<int64_t>(slots, 1);
    rc = g->host_csr ? ensure_host(sl.col, cb) : ensure(sl.col, cb);
  }
  if (rc == PG_OK) {
    k_sell_fill<<<grid_for(nchunks * 32), kBlock, 0, st>>>(
        (const ulonglong2 *)sl.items.p, nchunks, (const int32_t *)sl.len.p,
        (const int64_t *)sl.off.p, g->col, (int32_t *)sl.col.p);
    rc = cuda_status(cudaGetLastError());
  }
  if (hist) cudaFreeAsync(hist, st);
  (void)coff_tmp;
  if (rc == PG_OK) rc = cuda_status(cudaStreamSynchronize(st));
  release(tmp.list);
  if (rc == PG_OK) {
    sl.Lmax = Lmax;
    sl.nchunks = nchunks;
    sl.slots = slots;
  } else {
    sl.Lmax = 0;
  }
  return rc;
}

// The workspace's buffers in arena order.
static std::vector<DevBuf *> workspace_parts(Workspace &w) {
  return {&w.X,  &w.Y,  &w.D0,     &w.D1, &w.C0,   &w.C1,   &w.K0,    &w.K1,
          &w.Sat, &w.RB, &w.KW0,   &w.KW1, &w.F0,  &w.F1,   &w.E,     &w.A,
          &w.counts, &w.rs, &w.ctrl, &w.seeds, &w.seed_bits, &w.gfsum, &w.gthr,
          &w.dlist, &w.dpref, &w.E1, &w.gm};
}

pg_status carve_workspace(Workspace &w, const std::vector<std::pair<DevBuf *, size_t>> &needs) {
  constexpr size_t kAlign = 256;
  bool fits = w.arena.p != nullptr;
  for (const auto &nd : needs)
    if (!nd.first->p || nd.first->bytes < std::max<size_t>(nd.second, 16)) fits = false;
  if (fits) return PG_OK;
  std::vector<DevBuf *> parts = workspace_parts(w);
  if (w.arena.p) {
    // only parts the layout does not have yet: placed after it, in the
    // arena's slack, when they fit (the other parts keep their place)
    size_t off = w.used;
    bool extra_ok = true;
    std::vector<std::pair<DevBuf *, size_t>> add;
    for (const auto &nd : needs) {
      const size_t want = std::max<size_t>(nd.second, 16);
      if (nd.first->p && nd.first->bytes >= want) continue;
      if (nd.first->p) extra_ok = false;  // a part that has to grow
      add.push_back({nd.first, want});
      off += (want + kAlign - 1) / kAlign * kAlign;
    }
    if (extra_ok && off <= w.arena.bytes) {
      char *base = (char *)w.arena.p;
      for (auto &a : add) {
        a.first->p = base + w.used;
        a.first->bytes = a.second;
        w.used += (a.second + kAlign - 1) / kAlign * kAlign;
      }
      return PG_OK;
    }
  }
  std::vector<size_t> cap(parts.size());
  for (size_t i = 0; i < parts.size(); ++i) cap[i] = parts[i]->p ? parts[i]->bytes : 0;
  for (const auto &nd : needs) {
    const size_t want = std::max<size_t>(nd.second, 16);
    size_t i = 0;
    while (i < parts.size() && parts[i] != nd.first) ++i;
    if (i == parts.size()) return PG_EINVAL;  // not a buffer of this workspace
    cap[i] = std::max(cap[i], want);
  }
  size_t total = 0;
  for (size_t c : cap) total += (c + kAlign - 1) / kAlign * kAlign;
  for (DevBuf *b : parts) {  // the old layout is void from here on
    b->p = nullptr;
    b->bytes = 0;
  }
  w.used = 0;
  // 1/32 of slack, so that parts a later call adds (PROPAGATE-S's per-pass
  // claim bits after a PROPAGATE-P call) need no new arena
  pg_status rc = ensure(w.arena, total + total / 32);
  if (rc) return rc;
  char *base = (char *)w.arena.p;
  size_t off = 0;
  for (size_t i = 0; i < parts.size(); ++i) {
    if (!cap[i]) continue;
    parts[i]->p = base + off;
    parts[i]->bytes = cap[i];
    off += (cap[i] + kAlign - 1) / kAlign * kAlign;
  }
  w.used = off;
  return PG_OK;
}

void release_workspace(Workspace &w) {
  release(w.arena);
  w.used = 0;
  for (DevBuf *b : workspace_parts(w)) {  // they pointed into the arena
    b->p = nullptr;
    b->bytes = 0;
  }
  if (w.ctrl_h) cudaFreeHost(w.ctrl_h);
  w.ctrl_h = nullptr;
  for (auto &e : w.ev)
    if (e) cudaEventDestroy(e);
  w.ev[0] = w.ev[1] = nullptr;
  for (auto &e : w.tev)
    if (e) cudaEventDestroy(e);
  w.tev.clear();
}

int64_t workspace_held(const Workspace &w) { return (int64_t)w.arena.bytes; }

// K copies of a CSR side by side: copy k's rows are k*n.., its arcs k*m..,
// its column indices shifted by k*n.
__global__ void k_replicate(const int64_t *rp, const int32_t *col, int64_t n, int64_t m, int K,
                            int64_t *rp_out, int32_t *col_out) {
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = gtid; i < (int64_t)K * n; i += nth) {
    const int64_t k = i / n;
    rp_out[i] = k * m + rp[i - k * n];
  }
  if (gtid == 0) rp_out[(int64_t)K * n] = (int64_t)K * m;
  for (int64_t j = gtid; j < (int64_t)K * m; j += nth) {
    const int64_t k = j / m;
    col_out[j] = (int32_t)(col[j - k * m] + k * n);
  }
}

__global__ void k_fill_graph_of(int32_t *node_graph, int64_t n, int K) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)K * n;
       i += (int64_t)gridDim.x * blockDim.x)
    node_graph[i] = (int32_t)(i / n);
}

// ------------------------------------------------------------ relabelling
// A permutation of the node ids that puts high in-degree nodes first, in
// buckets of 16 per octave of degree (exact below 32), each bucket in the
// original id order (a stable counting sort). The counts are per seed, so
// they do not depend on node ids: the library maps each seed through the
// permutation and returns the same counts, m_active and metrics. What
// changes is where the rows sit in memory: the most gathered rows (a
// neighbour's delta is read once per arc to it) share cache lines and stay
// in L2, and a dense sweep's rows, already grouped by length, become
// consecutive ids, so their own signatures are read and written together.
constexpr int kRelabelOct = 37;                          // degrees below 2^37
constexpr int kRelabelBuckets = kRelabelOct * 16 + 1;    // + degree 0
constexpr int kRelabelTile = 8192;                       // nodes per block

__device__ __forceinline__ int degree_bucket(int64_t d) {
  if (d <= 0) return kRelabelBuckets - 1;  // isolated nodes last
  const int lg = 63 - __clzll((unsigned long long)d);
  const int sub = lg >= 4 ? (int)((d >> (lg - 4)) & 15) : (int)((d << (4 - lg)) & 15);
  return (kRelabelBuckets - 2) - (lg * 16 + sub);  // higher degree, smaller bucket
}

// Bucket sizes per tile of kRelabelTile nodes, bucket-major: H[b * tiles + tile].
__global__ void __launch_bounds__(kBlock) k_relabel_hist(const int64_t *rp, int64_t n,
                                                         int64_t tiles, int64_t *H) {
  __shared__ uint32_t h[kRelabelBuckets];
  for (int b = threadIdx.x; b < kRelabelBuckets; b += kBlock) h[b] = 0u;
  __syncthreads();
  const int64_t v0 = (int64_t)blockIdx.x * kRelabelTile;
  for (int i = threadIdx.x; i < kRelabelTile; i += kBlock) {
    const int64_t v = v0 + i;
    if (v < n) atomicAdd(&h[degree_bucket(rp[v + 1] - rp[v])], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kRelabelBuckets; b += kBlock)
    H[(int64_t)b * tiles + blockIdx.x] = h[b];
}

// Stable scatter: node v goes to H[b * tiles + tile] (scanned) plus the number
// of earlier nodes of its tile in the same bucket. The tile is walked in id
// order, kBlock nodes per step; within a step, warps count their bucket
// peers (match_any) and add the counts of the warps before them.
__global__ void __launch_bounds__(kBlock) k_relabel_scatter(const int64_t *rp, int64_t n,
                                                            int64_t tiles, const int64_t *H,
                                                            int32_t *new_of, int32_t *old_of) {
  constexpr int kWarps = kBlock / 32;
  __shared__ int64_t base[kRelabelBuckets];
  __shared__ uint16_t wcnt[kWarps][kRelabelBuckets];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int b = threadIdx.x; b < kRelabelBuckets; b += kBlock)
    base[b] = H[(int64_t)b * tiles + blockIdx.x];
  const int64_t v0 = (int64_t)blockIdx.x * kRelabelTile;
  for (int i0 = 0; i0 < kRelabelTile; i0 += kBlock) {
    const int64_t v = v0 + i0 + threadIdx.x;
    const bool valid = v < n;
    const int b = valid ? degree_bucket(rp[v + 1] - rp[v]) : -1;
    const unsigned peers = __match_any_sync(kFullMask, b);
    const unsigned below = peers & ((1u << lane) - 1u);
    __syncthreads();  // the previous step's counts are read and added
    for (int k = threadIdx.x; k < kWarps * kRelabelBuckets; k += kBlock)
      (&wcnt[0][0])[k] = 0;
    __syncthreads();
    if (valid && below == 0u) wcnt[w][b] = (uint16_t)__popc(peers);
    __syncthreads();
    if (valid) {
      int64_t pos = base[b] + __popc(below);
      for (int k = 0; k < w; ++k) pos += wcnt[k][b];
      new_of[v] = (int32_t)pos;
      old_of[pos] = (int32_t)v;
    }
    __syncthreads();
    for (int bb = threadIdx.x; bb < kRelabelBuckets; bb += kBlock) {
      int64_t add = 0;
      for (int k = 0; k < kWarps; ++k) add += wcnt[k][bb];
      base[bb] += add;
    }
  }
}

// In-degree of each new row (the exclusive scan of this gives the row pointers).
__global__ void k_relabel_degrees(const int64_t *rp, const int32_t *old_of, int64_t n,
                                  int64_t *nrp) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = old_of[r];
    nrp[r] = rp[v + 1] - rp[v];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) nrp[n] = 0;
}

// New rows four at a time per warp (new ids in order, so the longest rows
// come first): four rows of at most 64 arcs take 8 lanes each, otherwise the
// whole warp takes the four rows one after another. Each row's arcs keep
// their original order, each source renamed. (A warp per row left most lanes
// idle on the short rows that make up most of a power-law graph.)
__global__ void __launch_bounds__(kBlock) k_relabel_arcs(const int64_t *rp, const int32_t *col,
                                                         const int32_t *new_of,
                                                         const int32_t *old_of, int64_t n,
                                                         const int64_t *nrp, int32_t *ncol) {
  const int lane = threadIdx.x & 31;
  const int q = lane >> 3, l = lane & 7;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 4; r0 < n;
       r0 += nw * 4) {
    const int64_t r = r0 + q;
    int64_t o = 0, d = 0;
    if (r < n) {
      o = nrp[r];
      d = nrp[r + 1] - o;
    }
    if (__all_sync(kFullMask, d <= 64)) {
      if (d > 0) {
        const int64_t b = rp[old_of[r]];
        int64_t k = l;
        for (; k + 24 < d; k += 32) {  // four independent renames in flight
          const int32_t a0 = col[b + k], a1 = col[b + k + 8], a2 = col[b + k + 16],
                        a3 = col[b + k + 24];
          const int32_t c0 = new_of[a0], c1 = new_of[a1], c2 = new_of[a2], c3 = new_of[a3];
          ncol[o + k] = c0;
          ncol[o + k + 8] = c1;
          ncol[o + k + 16] = c2;
          ncol[o + k + 24] = c3;
        }
        for (; k < d; k += 8) ncol[o + k] = new_of[col[b + k]];
      }
      continue;
    }
    for (int qq = 0; qq < 4; ++qq) {
      const int64_t oo = __shfl_sync(kFullMask, o, qq * 8);
      const int64_t dd = __shfl_sync(kFullMask, d, qq * 8);
      if (dd == 0) continue;  // warp-uniform (also rows past n)
      const int64_t b = rp[old_of[r0 + qq]];
      int64_t k = lane;
      for (; k + 96 < dd; k += 128) {  // four independent renames in flight
        const int32_t a0 = col[b + k], a1 = col[b + k + 32], a2 = col[b + k + 64],
                      a3 = col[b + k + 96];
        const int32_t c0 = new_of[a0], c1 = new_of[a1], c2 = new_of[a2], c3 = new_of[a3];
        ncol[oo + k] = c0;
        ncol[oo + k + 32] = c1;
        ncol[oo + k + 64] = c2;
        ncol[oo + k + 96] = c3;
      }
      for (; k < dd; k += 32) ncol[oo + k] = new_of[col[b + k]];
    }
  }
}

// Relabels g's in-CSR in place (new arrays, owned by g) and keeps the map
// from original to new ids in g->perm.
static pg_status relabel_by_degree(pg_graph *g, cudaStream_t st) {
  const int64_t n = g->n, m = g->m;
  const int64_t tiles = (n + kRelabelTile - 1) / kRelabelTile;
  int64_t *H = nullptr, *nrp = nullptr;
  int32_t *old_of = nullptr, *ncol = nullptr;
  pg_status rc = ensure(g->perm, sizeof(int32_t) * (size_t)n);
  if (!rc) rc = cuda_status(cudaMallocAsync((void **)&H, sizeof(int64_t) * (size_t)(tiles * kRelabelBuckets), st));
  if (!rc) rc = cuda_status(cudaMallocAsync((void **)&old_of, sizeof(int32_t) * (size_t)n, st));
  if (!rc) rc = cuda_status(cudaMalloc((void **)&nrp, sizeof(int64_t) * (size_t)(n + 1)));
  if (!rc)
    rc = cuda_status(alloc_arcs((void **)&ncol, sizeof(int32_t) * (size_t)std::max<int64_t>(m, 1),
                                g->host_csr));
  if (!rc) {
    k_relabel_hist<<<(unsigned)tiles, kBlock, 0, st>>>(g->row_ptr, n, tiles, H);
    rc = cuda_status(cudaGetLastError());
  }
  if (!rc) rc = exclusive_scan_i64(H, tiles * kRelabelBuckets, st);
  if (!rc) {
    k_relabel_scatter<<<(unsigned)tiles, kBlock, 0, st>>>(g->row_ptr, n, tiles, H,
                                                          (int32_t *)g->perm.p, old_of);
    k_relabel_degrees<<<grid_for(n), kBlock, 0, st>>>(g->row_ptr, old_of, n, nrp);
    rc = cuda_status(cudaGetLastError());
  }
  if (!rc) rc = exclusive_scan_i64(nrp, n + 1, st);
  if (!rc && m > 0) {
    k_relabel_arcs<<<grid_for(n * 8), kBlock, 0, st>>>(g->row_ptr, g->col, (const int32_t *)g->perm.p,
                                                       old_of, n, nrp, ncol);
    rc = cuda_status(cudaGetLastError());
  }
  if (H) cudaFreeAsync(H, st);
  if (old_of) cudaFreeAsync(old_of, st);
  if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
  if (rc) {
    if (nrp) cudaFree(nrp);
    free_arcs(ncol, g->host_csr);
    release(g->perm);
    return rc;
  }
  if (g->owns_in) {
    cudaFree(g->row_ptr);
    free_arcs(g->col, g->col_host);
  }
  g->row_ptr = nrp;
  g->col = ncol;
  g->col_host = g->host_csr;
  g->owns_in = true;
  return PG_OK;
}

pg_status make_replicas(pg_graph *g, int K, cudaStream_t st) {
  if (g->rep && g->rep_K == K) return PG_OK;
  drop_replicas(g);
  const int64_t n = g->n, m = g->m, Kn = (int64_t)K * n, Km = (int64_t)K * m;
  if (K < 2 || Kn > kMaxNodes || Km > kMaxArcs) return PG_EINVAL;
  pg_graph *r = new pg_graph();
  r->n = Kn;
  r->m = Km;
  r->directed = g->directed;
  r->device = g->device;
  r->mean_degree = g->mean_degree;
  r->max_degree = g->max_degree;
  pg_status rc = cuda_status(cudaMalloc((void **)&r->row_ptr, sizeof(int64_t) * (Kn + 1)));
  if (!rc) rc = cuda_status(cudaMalloc((void **)&r->col, sizeof(int32_t) * std::max<int64_t>(Km, 1)));
  if (!rc) {
    k_replicate<<<grid_for(std::max(Kn, Km)), kBlock, 0, st>>>(g->row_ptr, g->col, n, m, K,
                                                               r->row_ptr, r->col);
    rc = cuda_status(cudaGetLastError());
  }
  if (!rc && g->out_ptr == g->row_ptr) {
    r->out_ptr = r->row_ptr;
    r->out_col = r->col;
    r->owns_out = false;
  } else if (!rc) {
    rc = cuda_status(cudaMalloc((void **)&r->out_ptr, sizeof(int64_t) * (Kn + 1)));
    if (!rc)
      rc = cuda_status(cudaMalloc((void **)&r->out_col, sizeof(int32_t) * std::max<int64_t>(Km, 1)));
    if (!rc) {
      k_replicate<<<grid_for(std::max(Kn, Km)), kBlock, 0, st>>>(g->out_ptr, g->out_col, n, m, K,
                                                                 r->out_ptr, r->out_col);
      rc = cuda_status(cudaGetLastError());
    }
  }
  if (!rc) rc = ensure(g->rep_graph_of, sizeof(int32_t) * (size_t)Kn);
  if (!rc) {
    k_fill_graph_of<<<grid_for(Kn), kBlock, 0, st>>>((int32_t *)g->rep_graph_of.p, n, K);
    rc = cuda_status(cudaGetLastError());
  }
  if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
  if (rc) {
    pg_graph_free(r);
    release(g->rep_graph_of);
    return rc;
  }
  r->seg_of = (const int32_t *)g->rep_graph_of.p;
  r->nseg = K;
  g->rep = r;
  g->rep_K = K;
  return PG_OK;
}

void drop_replicas(pg_graph *g) {
  if (g->rep) pg_graph_free(g->rep);
  g->rep = nullptr;
  g->rep_K = 0;
  for (DevBuf *b : {&g->rep_graph_of, &g->rep_graph_s, &g->rep_graph_col0}) release(*b);
}

pg_status make_view(pg_graph *master, cudaStream_t st, pg_graph **out) {
  if (!master || !out) return PG_EINVAL;
  pg_graph *v = new pg_graph();
  {
    std::lock_guard<std::mutex> lk(master->mu);
    pg_status rc = ensure_sell(master, kSellPiece, st);
    if (rc == PG_OK) rc = cuda_status(cudaStreamSynchronize(st));
    if (rc) {
      delete v;
      return rc;
    }
    v->n = master->n;
    v->m = master->m;
    v->directed = master->directed;
    v->device = master->device;
    v->row_ptr = master->row_ptr;
    v->col = master->col;
    v->out_ptr = master->out_ptr;
    v->out_col = master->out_col;
    v->mean_degree = master->mean_degree;
    v->max_degree = master->max_degree;
    v->sell = master->sell;
    v->perm_ptr = (const int32_t *)master->perm.p;
  }
  v->owns_in = v->owns_out = v->owns_sell = false;
  *out = v;
  return PG_OK;
}

}  // namespace pg

using namespace pg;

extern "C" {

const char *pg_version(void) { return "propagate-gb300 1.0 (sm_103a)"; }

const char *pg_strerror(pg_status st) {
  switch (st) {
    case PG_OK: return "ok";
    case PG_EINVAL: return "invalid argument";
    case PG_ENOMEM: return "out of memory";
    case PG_ECUDA: return "CUDA runtime error";
    case PG_ETIMEOUT: return "device-side wait timed out";
    case PG_EDEVICE: return "inconsistent device state";
    case PG_ECANCELLED: return "cancelled";
    case PG_ERANGE: return "more rounds than max_rounds";
    case PG_ETOOBIG: return "problem larger than the fixed scratch of the allocation-free entry point";
  }
  return "unknown status";
}

static void free_graph_arrays(pg_graph *g) {
  if (g->owns_in) {
    if (g->row_ptr) cudaFree(g->row_ptr);
    free_arcs(g->col, g->col_host);
  }
  if (g->owns_out && g->out_ptr != g->row_ptr) {
    if (g->out_ptr) cudaFree(g->out_ptr);
    free_arcs(g->out_col, g->out_col_host);
  }
  g->row_ptr = g->out_ptr = nullptr;
  g->col = g->out_col = nullptr;
}

void pg_graph_free(pg_graph *g) {
  if (!g) return;
  drop_graph_cache(g);
  {
    std::lock_guard<std::mutex> lk(g->mu);
    free_graph_arrays(g);
    release(g->pieces.list);
    if (g->owns_sell)
      for (DevBuf *b : {&g->sell.items, &g->sell.col, &g->sell.off, &g->sell.len, &g->sell.seg,
                        &g->sell.chunk0})
        release(*b);
    drop_replicas(g);
    release_workspace(g->ws);
    release(g->perm);
  }
  delete g;
}

pg_status pg_graph_info(const pg_graph *g, int64_t *n, int64_t *m) {
  if (!g) return PG_EINVAL;
  if (n) *n = g->n;
  if (m) *m = g->m;
  return PG_OK;
}

pg_status pg_query_rounds_bound(const pg_graph *g, int32_t *max_rounds) {
  if (!g || !max_rounds) return PG_EINVAL;
  *max_rounds = (int32_t)std::min<int64_t>(g->n - 1, 0x7FFFFFF0LL);
  return PG_OK;
}

pg_status pg_graph_from_csr(const int64_t *row_ptr, const int32_t *col, int64_t n, int64_t m,
                            int directed, unsigned flags, void *stream, pg_graph **out) {
  if (!out) return PG_EINVAL;
  *out = nullptr;
  if (n < 1 || n > kMaxNodes || m < 0 || m > kMaxArcs || !row_ptr || (m > 0 && !col))
    return PG_EINVAL;
  if ((flags & PG_BORROW) && !(flags & PG_DEVICE_PTRS)) return PG_EINVAL;
  if ((flags & PG_HOST_CSR) && (flags & PG_BORROW)) return PG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  pg_graph *g = new pg_graph();
  g->n = n;
  g->m = m;
  g->directed = directed ? 1 : 0;
  g->host_csr = (flags & PG_HOST_CSR) != 0;
  cudaGetDevice(&g->device);
  pg_status rc = PG_OK;
  const bool dev = flags & PG_DEVICE_PTRS;
  if (flags & PG_BORROW) {
    g->row_ptr = const_cast<int64_t *>(row_ptr);
    g->col = const_cast<int32_t *>(col);
    g->owns_in = false;
  } else {
    rc = cuda_status(cudaMalloc((void **)&g->row_ptr, sizeof(int64_t) * (n + 1)));
    if (rc == PG_OK)
      rc = cuda_status(alloc_arcs((void **)&g->col, sizeof(int32_t) * std::max<int64_t>(m, 1),
                                  g->host_csr));
    g->col_host = g->host_csr;
    cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (g->host_csr) kind = cudaMemcpyDefault;
    if (rc == PG_OK)
      rc = cuda_status(cudaMemcpyAsync(g->row_ptr, row_ptr, sizeof(int64_t) * (n + 1),
                                       g->host_csr ? cudaMemcpyDefault : kind, st));
    if (rc == PG_OK && m > 0)
      rc = cuda_status(cudaMemcpyAsync(g->col, col, sizeof(int32_t) * m, kind, st));
  }
  // one small block: [0] error bits, [1] max degree, [2..3] the two counts
  unsigned long long *vb = nullptr;
  if (rc == PG_OK) rc = cuda_status(cudaMallocAsync((void **)&vb, 4 * sizeof(unsigned long long), st));
  if (rc == PG_OK) {
    cudaMemsetAsync(vb, 0, 4 * sizeof(unsigned long long), st);
    int *err = reinterpret_cast<int *>(vb);
    k_validate_rows<<<grid_for(n), kBlock, 0, st>>>(g->row_ptr, g->col, n, m, vb + 2, err);
    k_validate_arcs<<<grid_for((m + 3) / 4), kBlock, 0, st>>>(g->col, n, m, vb + 2, err);
    k_max_degree<<<grid_for(n), kBlock, 0, st>>>(g->row_ptr, n, vb + 1);
    rc = cuda_status(cudaGetLastError());
  }
  unsigned long long vb_h[4] = {0, 0, 0, 0};
  if (rc == PG_OK) rc = cuda_status(cudaMemcpyAsync(vb_h, vb, sizeof(vb_h), cudaMemcpyDeviceToHost, st));
  if (rc == PG_OK) rc = cuda_status(cudaStreamSynchronize(st));
  if (vb) cudaFreeAsync(vb, st);
  int err_h = (int)(vb_h[0] & 0xFFFFFFFFULL);
  if (!(err_h & 2) && vb_h[2] != vb_h[3]) err_h |= 8;  // a descent inside a row
  const unsigned long long mx_h = vb_h[1];
  if (rc == PG_OK && err_h) rc = PG_EINVAL;
  g->max_degree = (int64_t)mx_h;
  g->mean_degree = (double)m / (double)n;
  // relabel (hubs first) when asked, or by default when the in-degrees are
  // skewed (a power-law graph) and the graph is large enough for locality
  // to matter; a lattice or a uniform random graph keeps its order
  const bool relabel = !(flags & PG_KEEP_ORDER) &&
                       ((flags & PG_RELABEL) ||
                        (n >= (1LL << 16) && (double)g->max_degree >= 16.0 * g->mean_degree));
  if (rc == PG_OK && relabel && m > 0) {
    rc = relabel_by_degree(g, st);
    if (rc == PG_OK) g->perm_ptr = (const int32_t *)g->perm.p;
  }
  if (rc == PG_OK) {
    if (!directed) {
      g->out_ptr = g->row_ptr;
      g->out_col = g->col;
      g->owns_out = false;
    } else {
      rc = cuda_status(cudaMalloc((void **)&g->out_ptr, sizeof(int64_t) * (n + 1)));
      if (rc == PG_OK)
        rc = cuda_status(alloc_arcs((void **)&g->out_col,
                                    sizeof(int32_t) * std::max<int64_t>(m, 1), g->host_csr));
      g->out_col_host = g->host_csr;
      unsigned long long *cursor = nullptr;
      if (rc == PG_OK) rc = cuda_status(cudaMallocAsync((void **)&cursor, sizeof(unsigned long long) * n, st));
      if (rc == PG_OK) {
        cudaMemsetAsync(g->out_ptr, 0, sizeof(int64_t) * (n + 1), st);
        k_count_out<<<grid_for(m), kBlock, 0, st>>>(g->col, m, (unsigned long long *)g->out_ptr);
        rc = cuda_status(cudaGetLastError());
      }
      if (rc == PG_OK) rc = exclusive_scan_i64(g->out_ptr, n + 1, st);
      if (rc == PG_OK) {
        cudaMemcpyAsync(cursor, g->out_ptr, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, st);
        // row pieces of at most kScatterPiece arcs (scratch; the graph's
        // cached piece list is built later for the pull's own piece length)
        rc = ensure_pieces(g, kScatterPiece, st);
        if (rc == PG_OK) {
          k_scatter_out<<<grid_for(g->pieces.count), kBlock, 0, st>>>(
              (const ulonglong2 *)g->pieces.list.p, g->pieces.count, g->col, cursor, g->out_col);
          rc = cuda_status(cudaGetLastError());
        }
      }
      if (cursor) cudaFreeAsync(cursor, st);
      if (rc == PG_OK) rc = cuda_status(cudaStreamSynchronize(st));
      release(g->pieces.list);  // scratch of the scatter, not a cached list
      g->pieces.L = 0;
      g->pieces.count = 0;
    }
  }
  if (rc == PG_OK && (flags & PG_REVERSE) && directed) {
    // pull over the transpose: rows become out-lists, the out-side in-lists
    std::swap(g->row_ptr, g->out_ptr);
    std::swap(g->col, g->out_col);
    std::swap(g->owns_in, g->owns_out);
    std::swap(g->col_host, g->out_col_host);
    release(g->pieces.list);  // built over the other side for the transpose
    g->pieces.L = 0;
    unsigned long long *mx2 = nullptr;
    rc = cuda_status(cudaMallocAsync((void **)&mx2, sizeof(unsigned long long), st));
    unsigned long long mxo = 0;
    if (rc == PG_OK) {
      cudaMemsetAsync(mx2, 0, sizeof(unsigned long long), st);
      k_max_degree<<<grid_for(n), kBlock, 0, st>>>(g->row_ptr, n, mx2);
      rc = cuda_status(cudaMemcpyAsync(&mxo, mx2, sizeof(mxo), cudaMemcpyDeviceToHost, st));
      cudaFreeAsync(mx2, st);
      if (rc == PG_OK) rc = cuda_status(cudaStreamSynchronize(st));
    }
    g->max_degree = (int64_t)mxo;
  }
  if (rc != PG_OK) {
    cudaGetLastError();
    free_graph_arrays(g);
    release(g->pieces.list);
    release(g->perm);
    delete g;
    return rc;
  }
  *out = g;
  return PG_OK;
}

pg_status pg_graph_is_relabelled(const pg_graph *g, int32_t *relabelled) {
  if (!g || !relabelled) return PG_EINVAL;
  *relabelled = g->perm_ptr != nullptr;
  return PG_OK;
}

}  // extern "C"
