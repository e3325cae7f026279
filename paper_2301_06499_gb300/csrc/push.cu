// Push rounds in a kernel of their own: rows of 8 words, PROPAGATE-S passes
// run as words (m_active counted per pass), and packed batches (whose sparse
// graphs push while the graphs in a full sweep are swept by k_pull in the
// same round). The round is pull_push in kernels.cuh: every row
// that changed in round t-1 ORs its delta into its unsaturated out-neighbours
// with atomics, claiming them for m_active on the way. Launched after k_pull
// in every round of a propagation that pushes; it returns at once in the
// rounds that do not.
#include "kernels.cuh"

namespace pg {

template <int CW, bool PW>
__global__ void __launch_bounds__(kBlock, 4) k_push(Params p) {
  Ctrl *ctrl = p.ctrl;
  if (*(volatile int32_t *)&ctrl->done) return;
  const int mode = ctrl->mode;
  if (!(mode == kModePush || (mode == kModeMixed && p.push))) return;
  const int t = ctrl->t;
  RoundBufs rb;  // the buffers of round t (k_pull cleared the next claims)
  rb.Dprev = (t & 1) ? p.D0 : p.D1;
  rb.Cprev = (t & 1) ? p.C0 : p.C1;
  rb.F = (t & 1) ? p.F1 : p.F0;
  rb.Ccur = (t & 1) ? p.C1 : p.C0;
  rb.Kcur = (t & 1) ? p.K1 : p.K0;
  rb.Kwcur = (t & 1) ? p.Kw1 : p.Kw0;
  const int64_t gtid = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int lane = threadIdx.x & 31;
  uint32_t my_mact = 0, my_scan = 0, my_gath = 0, my_items = 0, my_rows = 0;
  unsigned long long my_work = 0;
  __shared__ int32_t s_stage[kBlock / 32][kStageRows];  // staged frontier rows per warp
  int32_t *stage = s_stage[threadIdx.x >> 5];
  int scnt = 0;
  pull_push<CW, PW>(p, ctrl, rb, t, lane, gtid >> 5, ((int64_t)gridDim.x * kBlock) >> 5,
                    my_mact, my_work, my_scan, my_gath, my_items, my_rows, stage, scnt);
  if (scnt) stage_flush(p, ctrl, rb.F, stage, scnt, lane);
  pull_end(p, ctrl, t, my_mact, my_work, my_scan, my_gath, my_items, my_rows);
}

PullFn push_fn(int CW, bool pw) {
  switch (CW) {
    case 1: return pw ? &k_push<1, true> : &k_push<1, false>;
    case 2: return pw ? &k_push<2, true> : &k_push<2, false>;
    case 4: return pw ? &k_push<4, true> : &k_push<4, false>;
    case 8: return pw ? &k_push<8, true> : &k_push<8, false>;
  }
  return nullptr;
}

}  // namespace pg
