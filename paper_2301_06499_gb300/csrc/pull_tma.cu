// Dense rounds of the pull with the gathered deltas moved by the tensor
// memory accelerator (TMA) instead of per-lane loads.
//
// Same round as pull_dense in kernels.cuh (Alg. 1's inner OR over the deltas
// of round t-1, sliced-ELL chunks of 32 row pieces, lane l owning piece l):
// only the delta rows travel differently. At step k of a chunk the warp holds
// the column indices of arc k of its 32 pieces; the valid ones (in range,
// row not saturated, and, when tested, in-neighbour changed in round t-1)
// are packed into slots, and every fourth lane issues one
// cp.async.bulk.tensor ... tile::gather4 that copies four whole delta rows
// (a 2-D tensor map over D, one row of CW words per node) from L2/HBM into
// shared memory, completing on the step's mbarrier. Each warp keeps a ring
// of kStages such steps in flight, so up to kStages x 32 delta rows per warp
// are outstanding without holding a register each, and the gathers bypass
// the load/store unit's per-request tag lookups (the pull's measured bound).
// A lane then ORs its slot's row from shared memory into its accumulator.
// Sparse rounds and packed batches are left to k_pull, which this kernel
// runs before in each round (it returns at once outside dense rounds).
//
// Rows past a piece's end and skipped in-neighbours are not copied; a
// gather4 whose last slots are empty reads row n, an all-zero row kept past
// the last node of both delta buffers. Every wait on an mbarrier is bounded:
// if a step's copies do not complete, the kernel records PG_ETIMEOUT in the
// control block, ends the round loop, waits (again bounded) for its copies
// still in flight and returns.
#include <cuda.h>

#include "kernels.cuh"

namespace pg {

#ifndef PG_TMA_STAGES
#define PG_TMA_STAGES 6
#endif

namespace {

constexpr int kStages = PG_TMA_STAGES;
constexpr uint32_t kSpinLimit = 1u << 22;  // try_wait polls before a step is abandoned

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Four rows r0..r3 of the 2-D tensor map (x = 0, the row's first word) into
// shared memory at dst, one after another.
__device__ __forceinline__ void gather4(uint32_t dst, const CUtensorMap *tm, int32_t r0,
                                        int32_t r1, int32_t r2, int32_t r3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(tm), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
      : "memory");
}

// Orders this thread's generic-proxy accesses to shared memory before later
// async-proxy (TMA) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Waits, all lanes, until the phase `parity` of bar completed; false after
// kSpinLimit polls without it.
__device__ __forceinline__ bool wait_step(uint32_t bar, uint32_t parity) {
  for (uint32_t spins = 0;; ++spins) {
    const bool ok = mbar_try_wait(bar, parity);
    if (__all_sync(kFullMask, ok)) return true;
    if (spins >= kSpinLimit) return false;
  }
}

}  // namespace

// Shared memory of one block: per warp kStages stages of 32 rows of CW words,
// their mbarriers, their valid-lane masks and a 32-entry slot table.
template <int CW>
constexpr size_t tma_smem_bytes() {
  return (size_t)(kBlock / 32) * ((size_t)kStages * 32 * CW * 8 + (size_t)kStages * 8 +
                                  (size_t)kStages * 4 + 32 * 4) +
         128;
}

template <int CW, bool PW>
__global__ void __launch_bounds__(kBlock, 1)
    k_pull_tma(Params p, const __grid_constant__ CUtensorMap tm0,
               const __grid_constant__ CUtensorMap tm1) {
  constexpr int ROWB = CW * 8;
  constexpr int STAGEB = 32 * ROWB;
  constexpr int NW = kBlock / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Ctrl *ctrl = p.ctrl;
  if (*(volatile int32_t *)&ctrl->done) return;
  if (ctrl->mode != kModeDense) return;  // sparse rounds: k_pull's work list
  const int t = ctrl->t;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned char *smem =
      reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  unsigned char *stages = smem + (size_t)wib * kStages * STAGEB;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)NW * kStages * STAGEB) +
                   (size_t)wib * kStages;
  uint32_t *vmask = reinterpret_cast<uint32_t *>(smem + (size_t)NW * kStages * (STAGEB + 8)) +
                    (size_t)wib * kStages;
  int32_t *slots = reinterpret_cast<int32_t *>(smem + (size_t)NW * kStages * (STAGEB + 12)) +
                   (size_t)wib * 32;
  if (lane < kStages) mbar_init(smem_addr(bars + lane), 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();

  const uint64_t *Dprev = (t & 1) ? p.D0 : p.D1;
  const CUtensorMap *tm = (t & 1) ? &tm0 : &tm1;
  const uint32_t *Cprev = (t & 1) ? p.C0 : p.C1;
  int32_t *F = (t & 1) ? p.F1 : p.F0;
  uint32_t *Ccur = (t & 1) ? p.C1 : p.C0;
  uint32_t *Kcur = (t & 1) ? p.K1 : p.K0;
  uint32_t *Kwcur = (t & 1) ? p.Kw1 : p.Kw0;
  (void)Dprev;
  const bool tc = test_changed_now(p, ctrl);
  const int64_t gw = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kBlock) >> 5;
  const int64_t nch = p.sell_chunks;
  const int32_t zrow = (int32_t)p.n;  // the all-zero row past the last node
  uint32_t my_mact = 0, my_scan = 0, my_gath = 0, my_items = 0, my_rows = 0;
  unsigned long long my_work = 0;

  // producer: the step (chunk pc, arc pk) whose delta rows are issued next
  int64_t pc = gw;
  int pk = 0, p_steps = 1, p_len = 0;
  int64_t p_off = 0;
  bool p_act = false;
  auto p_chunk = [&]() {
    if (pc < nch) {
      const ulonglong2 it = p.sell_items[pc * 32 + lane];
      const int clen = __ldg(p.sell_len + pc);
      p_steps = clen > 0 ? clen : 1;
      p_off = __ldg(p.sell_off + pc);
      p_len = (int)(it.y & 0x7FFFFFFFULL);
      p_act = p_len > 0 && !test_bit(p.Sat, (int32_t)(it.y >> 32));
    }
  };
  p_chunk();
  uint32_t issued = 0, consumed = 0;
  auto issue = [&]() {
    if (pc >= nch) return;
    const int st = (int)(issued % kStages);
    const uint32_t bar = smem_addr(bars + st);
    int32_t u = (p_act && pk < p_len) ? __ldg(p.sell_col + p_off + 32LL * pk + lane) : -1;
    if (u >= 0 && !gather_ok(p, u, CW - 1)) u = -1;
    if (u >= 0 && tc && !test_bit(Cprev, u)) u = -1;
    const unsigned vm = __ballot_sync(kFullMask, u >= 0);
    const int nv = __popc(vm);
    const int ng = (nv + 3) >> 2;
    __syncwarp();  // the previous step's slot reads are done
    if (u >= 0) slots[__popc(vm & ((1u << lane) - 1u))] = u;
    if (lane == 0) {
      vmask[st] = vm;
      if (ng)
        mbar_arrive_expect_tx(bar, (uint32_t)(ng * 4 * ROWB));
      else
        mbar_arrive(bar);
    }
    __syncwarp();
    if (lane < ng) {
      int32_t r[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) r[q] = 4 * lane + q < nv ? slots[4 * lane + q] : zrow;
      gather4(smem_addr(stages + (size_t)st * STAGEB + (size_t)lane * 4 * ROWB), tm, r[0], r[1],
              r[2], r[3], bar);
    }
    ++issued;
    if (++pk >= p_steps) {
      pc += nw;
      pk = 0;
      p_chunk();
    }
  };

  // consumer: the chunk being accumulated
  int64_t cc = gw;
  int ck = 0, c_steps = 1, c_len = 0;
  int32_t c_v = 0;
  bool c_whole = true, c_act = false;
  uint64_t acc[CW];
  auto c_chunk = [&]() {
#pragma unroll
    for (int k = 0; k < CW; ++k) acc[k] = 0ULL;
    if (cc < nch) {
      const ulonglong2 it = p.sell_items[cc * 32 + lane];
      const int clen = __ldg(p.sell_len + cc);
      c_steps = clen > 0 ? clen : 1;
      c_v = (int32_t)(it.y >> 32);
      c_whole = (it.y & 0x80000000ULL) != 0ULL;
      c_len = (int)(it.y & 0x7FFFFFFFULL);
      c_act = c_len > 0 && !test_bit(p.Sat, c_v);
    }
  };
  // the end of a chunk: as pull_dense (compare with X, write Y or OR into
  // it for split rows, activity, frontier append)
  auto c_finish = [&]() {
    const int32_t v = c_v;
    const bool whole = c_whole;
    bool act = c_act;
    uint64_t own[CW];
#pragma unroll
    for (int k = 0; k < CW; ++k) own[k] = 0ULL;
    if (act && whole) load_words<CW>(own, p.X + (size_t)v * (size_t)p.Wp);
    bool any_delta = false;
#pragma unroll
    for (int k = 0; k < CW; ++k) any_delta |= acc[k] != 0ULL;
    uint32_t pw_words = 0, pw_seeds = 0;
    if constexpr (PW)
      if (act) count_pass_words<CW>(p, v, 0, whole, own, acc, Kwcur, pw_words, pw_seeds);
    const bool row_changed = act && finish_piece<CW>(p, v, 0, whole, own, acc);
    if (act) {
      ++my_items;
      my_scan += (uint32_t)c_len;
    }
    act = act && any_delta;
    if (PW && act) {
      if (pw_words) {
        const uint32_t deg =
            whole ? (uint32_t)c_len : (uint32_t)(__ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v));
        my_mact += deg * pw_words;
        my_work += (unsigned long long)deg * (unsigned long long)pw_seeds;
        my_rows += pw_words;
      }
    } else if (act) {
      uint32_t deg = 0;
      if (whole) {
        deg = (uint32_t)c_len;
        ++my_rows;
      } else if (!set_bit(Kcur, v)) {
        deg = (uint32_t)(__ldg(p.row_ptr + v + 1) - __ldg(p.row_ptr + v));
        ++my_rows;
      }
      my_mact += deg;
      my_work += (unsigned long long)deg * (unsigned long long)p.s;
    }
    bool app = false;
    if (act && row_changed) {
      if (whole) {
        atomicOr(Ccur + (v >> 5), 1u << (v & 31));
        app = true;
      } else {
        app = !set_bit(Ccur, v);
      }
    }
    frontier_append(p, ctrl, F, v, app, lane);
  };

  for (int k = 0; k < kStages; ++k) issue();
  c_chunk();
  bool timed_out = false;
  while (consumed < issued) {
    const int st = (int)(consumed % kStages);
    if (!wait_step(smem_addr(bars + st), (consumed / kStages) & 1u)) {
      timed_out = true;
      break;
    }
    const unsigned vm = vmask[st];
    if ((vm >> lane) & 1u) {
      const int slot = __popc(vm & ((1u << lane) - 1u));
      const ulonglong2 *row =
          reinterpret_cast<const ulonglong2 *>(stages + (size_t)st * STAGEB + (size_t)slot * ROWB);
#pragma unroll
      for (int q = 0; q < CW / 2; ++q) {
        const ulonglong2 x = row[q];
        acc[2 * q] |= x.x;
        acc[2 * q + 1] |= x.y;
      }
      ++my_gath;
    }
    __syncwarp();
    fence_proxy_async_smem();  // this stage's reads before the TMA refills it
    ++consumed;
    if (++ck >= c_steps) {
      c_finish();
      cc += nw;
      ck = 0;
      c_chunk();
    }
    issue();
  }
  if (timed_out) {
    if (lane == 0) {
      ctrl->status = PG_ETIMEOUT;
      __threadfence();
      *(volatile int32_t *)&ctrl->done = 1;
    }
    // the copies still in flight land in this block's shared memory: wait
    // for them (bounded) before the block may exit
    for (; consumed < issued; ++consumed)
      if (!wait_step(smem_addr(bars + consumed % kStages), (consumed / kStages) & 1u)) break;
  }
  pull_end(p, ctrl, t, my_mact, my_work, my_scan, my_gath, my_items, my_rows);
}

template <int CW, bool PW>
static void launch_one(const Params &p, const CUtensorMap &t0, const CUtensorMap &t1, int grid,
                       cudaStream_t st) {
  k_pull_tma<CW, PW><<<grid, kBlock, tma_smem_bytes<CW>(), st>>>(p, t0, t1);
}

size_t pull_tma_smem(int CW) { return CW == 8 ? tma_smem_bytes<8>() : tma_smem_bytes<4>(); }

const void *pull_tma_fn(int CW, bool pw) {
  if (CW == 8) return pw ? (const void *)&k_pull_tma<8, true> : (const void *)&k_pull_tma<8, false>;
  if (CW == 4) return pw ? (const void *)&k_pull_tma<4, true> : (const void *)&k_pull_tma<4, false>;
  return nullptr;
}

void launch_pull_tma(int CW, bool pw, const Params &p, const void *tm0, const void *tm1, int grid,
                     cudaStream_t st) {
  const CUtensorMap &a = *static_cast<const CUtensorMap *>(tm0);
  const CUtensorMap &b = *static_cast<const CUtensorMap *>(tm1);
  if (CW == 8) {
    if (pw)
      launch_one<8, true>(p, a, b, grid, st);
    else
      launch_one<8, false>(p, a, b, grid, st);
  } else {
    if (pw)
      launch_one<4, true>(p, a, b, grid, st);
    else
      launch_one<4, false>(p, a, b, grid, st);
  }
}

// A 2-D tensor map over a delta buffer: n + 1 rows (row n all zero) of Wp
// 64-bit words, boxes of one row of CW words (the tile::gather4 layout).
pg_status encode_delta_map(void *out, const uint64_t *D, int64_t rows, int Wp, int CW) {
  using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  if (!fn) {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f) {
      cudaGetLastError();
      return PG_ECUDA;
    }
    fn = reinterpret_cast<EncodeFn>(f);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)Wp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Wp * 8};
  const cuuint32_t box[2] = {(cuuint32_t)CW, 1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(static_cast<CUtensorMap *>(out), CU_TENSOR_MAP_DATA_TYPE_UINT64, 2,
                        const_cast<uint64_t *>(D), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? PG_OK : PG_EINVAL;
}

}  // namespace pg
