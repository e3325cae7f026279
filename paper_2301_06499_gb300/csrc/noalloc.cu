// Allocation-free PROPAGATE-P for callers that must not allocate device
// memory once they are running: for instance a serving process that reserves
// all of its device memory at start-up and whose allocator would be thrown off
// by a stray cudaMalloc, or a latency-critical loop that cannot afford the
// device-wide synchronisation an allocation may cause. pg_propagate_p keeps a
// workspace per graph and grows it with cudaMalloc; this entry point instead
// works in one fixed file-scope device array, so the caller only supplies
// the graph, the seeds and the output buffer.
//
// The array is a static __device__ object: every GPU that loads the library
// holds PG_NOALLOC_SCRATCH_BYTES of it until the process exits. Host code may
// not pass the symbol itself to a kernel (on the host it names a stand-in,
// not device memory), so the device address is looked up once per device with
// cudaGetSymbolAddress and cached.
//
// Every call uses the same array and leaves its contents behind; each call
// clears what it needs before use. Calls whose work overlaps on the GPU (on
// different streams, or from different host threads) race on the array; the
// host side serialises calls made through this entry point, but only stream
// order protects the device work, so callers on several streams must order
// them themselves.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "host.cuh"

namespace pg {
namespace {

constexpr size_t kScratchWords = (size_t)PG_NOALLOC_SCRATCH_BYTES / 8;
constexpr int kMaxDevices = 64;
constexpr int kHeaderWords = 8;  // [0] error bits, [1] changed flag
constexpr int kMaxSeeds = PG_NOALLOC_MAX_SEEDS;
constexpr int kSeedWords = kMaxSeeds / 2;

__device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

std::mutex g_noalloc_mu;
unsigned long long *g_noalloc_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ uint64_t na_valid(int w, int s) {
  const int lo = w * 64;
  if (lo + 64 <= s) return ~0ULL;
  if (lo >= s) return 0ULL;
  return (1ULL << (s - lo)) - 1ULL;
}

// err bits: 1 row_ptr[0] != 0, 2 non-monotone / past m, 4 col out of range,
// 16 row_ptr[n] != m. Rows and arcs are checked by separate grid-stride
// loops, so a long row does not serialise on one thread.
__global__ void k_na_validate(const int64_t *rp, const int32_t *col, int64_t n, int64_t m,
                              unsigned long long *hdr) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  if (tid == 0) {
    if (rp[0] != 0) atomicOr(&hdr[0], 1ULL);
    if (rp[n] != m) atomicOr(&hdr[0], 16ULL);
  }
  bool bad_row = false, bad_col = false;
  for (int64_t v = tid; v < n; v += nth) {
    const int64_t b = rp[v], e = rp[v + 1];
    bad_row |= b > e || b < 0 || e > m;
  }
  for (int64_t j = tid; j < m; j += nth) bad_col |= col[j] < 0 || col[j] >= n;
  if (bad_row) atomicOr(&hdr[0], 2ULL);
  if (bad_col) atomicOr(&hdr[0], 4ULL);
}

// Clears the signatures, deltas and the caller's counts; round 0 puts seed
// i's bit into Y (a change of round 0, counted by the first post).
__global__ void k_na_init(unsigned long long *sc, int64_t n, int Wp, int s, uint32_t *counts,
                          int64_t count_words) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  unsigned long long *sig = sc + kHeaderWords + kSeedWords;
  for (int64_t i = tid; i < 4 * n * Wp; i += nth) sig[i] = 0ULL;
  for (int64_t i = tid; i < count_words; i += nth) counts[i] = 0u;
  if (tid == 0) sc[1] = 0ULL;
  (void)s;
}

__global__ void k_na_seed(unsigned long long *sc, int64_t n, int Wp, int s) {
  const int32_t *seeds = reinterpret_cast<const int32_t *>(sc + kHeaderWords);
  unsigned long long *Y = sc + kHeaderWords + kSeedWords + (size_t)n * Wp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s; i += gridDim.x * blockDim.x)
    Y[(size_t)seeds[i] * Wp + (i >> 6)] = 1ULL << (i & 63);
}

// Round t >= 1, one thread per node: OR the deltas of round t-1 over the
// in-neighbours; write Y where the signature grows.
__global__ void k_na_pull(unsigned long long *sc, const int64_t *rp, const int32_t *col, int64_t n,
                          int Wp, int t) {
  unsigned long long *base = sc + kHeaderWords + kSeedWords;
  const unsigned long long *X = base;
  unsigned long long *Y = base + (size_t)n * Wp;
  const unsigned long long *D = base + (size_t)(2 + ((t - 1) & 1)) * n * Wp;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    for (int w = 0; w < Wp; ++w) {
      unsigned long long acc = 0;
      for (int64_t j = rp[v]; j < rp[v + 1]; ++j) acc |= D[(size_t)col[j] * Wp + w];
      const unsigned long long o = X[(size_t)v * Wp + w];
      if ((o | acc) != o) Y[(size_t)v * Wp + w] = o | acc;
    }
  }
}

// Round t, one thread per node: d = X ^ Y is the round's new bits; count them
// per seed into row t, keep them as the deltas of round t, and set X = Y.
// Per-seed counts gather in shared memory (s <= PG_NOALLOC_MAX_SEEDS) and go
// to the caller's row with one global add per seed and block.
__global__ void k_na_post(unsigned long long *sc, int64_t n, int Wp, int s, int t,
                          uint32_t *counts, int count_row) {
  __shared__ uint32_t cnt[kMaxSeeds];
  for (int i = threadIdx.x; i < s; i += blockDim.x) cnt[i] = 0u;
  __syncthreads();
  unsigned long long *base = sc + kHeaderWords + kSeedWords;
  unsigned long long *X = base;
  const unsigned long long *Y = base + (size_t)n * Wp;
  unsigned long long *D = base + (size_t)(2 + (t & 1)) * n * Wp;
  bool any = false;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    for (int w = 0; w < Wp; ++w) {
      const size_t k = (size_t)v * Wp + w;
      unsigned long long d = (X[k] ^ Y[k]) & na_valid(w, s);
      D[k] = d;
      if (!d) continue;
      any = true;
      X[k] = Y[k];
      while (d) {
        const int bit = __ffsll((long long)d) - 1;
        atomicAdd(&cnt[w * 64 + bit], 1u);
        d &= d - 1ULL;
      }
    }
  }
  __syncthreads();
  if (count_row >= 0)
    for (int i = threadIdx.x; i < s; i += blockDim.x)
      if (cnt[i]) atomicAdd(&counts[(size_t)count_row * s + i], cnt[i]);
  if (any) atomicOr(&sc[1], 1ULL);
}

__global__ void k_na_clear_flag(unsigned long long *sc) { sc[1] = 0ULL; }

pg_status scratch_for_current_device(unsigned long long **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PG_ECUDA;
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return PG_ECUDA;
    }
    g_noalloc_ptr[dev] = static_cast<unsigned long long *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return PG_OK;
}

}  // namespace
}  // namespace pg

using namespace pg;

extern "C" pg_status pg_propagate_p_noalloc(const int64_t *row_ptr, const int32_t *col, int64_t n,
                                            int64_t m, const int32_t *seeds, int32_t s,
                                            uint32_t *counts, int32_t max_rounds,
                                            int32_t *rounds, void *stream) {
  if (!row_ptr || (m > 0 && !col) || !seeds || !counts || !rounds || n < 1 || m < 0 ||
      n >= 0x7FFFFFFFLL || s < 1 || s > n || max_rounds < 0)
    return PG_EINVAL;
  const int W = (s + 63) / 64;
  if (s > kMaxSeeds ||
      (size_t)kHeaderWords + kSeedWords + 4 * (size_t)n * (size_t)W > kScratchWords)
    return PG_ETOOBIG;
  for (int32_t i = 0; i < s; ++i) {
    if (seeds[i] < 0 || seeds[i] >= n) return PG_EINVAL;
    for (int32_t j = 0; j < i; ++j)
      if (seeds[j] == seeds[i]) return PG_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  unsigned long long *sc = nullptr;
  pg_status rc = scratch_for_current_device(&sc);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4LL * sms));
  unsigned long long hdr[2] = {0ULL, 0ULL};
  // header and seeds: the call's only host-to-device traffic
  cudaError_t e = cudaMemcpyAsync(sc, hdr, sizeof(hdr), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sc + kHeaderWords, seeds, sizeof(int32_t) * s, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e);
  k_na_validate<<<blocks, 256, 0, st>>>(row_ptr, col, n, m, sc);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
  e = cudaMemcpyAsync(hdr, sc, sizeof(hdr), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  if (hdr[0]) return PG_EINVAL;
  const int64_t count_words = ((int64_t)max_rounds + 1) * s;
  k_na_init<<<blocks, 256, 0, st>>>(sc, n, W, s, counts, count_words);
  k_na_seed<<<1, 256, 0, st>>>(sc, n, W, s);
  k_na_post<<<blocks, 256, 0, st>>>(sc, n, W, s, 0, counts, 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
  int32_t T = 0;
  for (int32_t t = 1;; ++t) {
    k_na_clear_flag<<<1, 1, 0, st>>>(sc);
    k_na_pull<<<blocks, 256, 0, st>>>(sc, row_ptr, col, n, W, t);
    k_na_post<<<blocks, 256, 0, st>>>(sc, n, W, s, t, counts, t <= max_rounds ? t : -1);
    // a failed launch must not read back as "no change" (a silent PG_OK)
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);
    e = cudaMemcpyAsync(hdr + 1, sc + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    if (!hdr[1]) {
      T = t - 1;
      break;
    }
    if (t > max_rounds) {
      *rounds = max_rounds + 1;
      return PG_ERANGE;
    }
  }
  *rounds = T;
  return PG_OK;
}
