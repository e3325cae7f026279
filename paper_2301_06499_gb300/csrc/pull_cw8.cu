// Pull kernels with 8 signature word(s) per lane load sequence.
#include "kernels.cuh"

namespace pg {

PullFn pull_fn_cw8(int G, bool chg, bool eb) {
  if (eb) return nullptr;
  switch (G) {
    case 2: return chg ? &k_pull<8, 2, true, false> : &k_pull<8, 2, false, false>;
    case 4: return chg ? &k_pull<8, 4, true, false> : &k_pull<8, 4, false, false>;
    case 8: return chg ? &k_pull<8, 8, true, false> : &k_pull<8, 8, false, false>;
    case 16: return chg ? &k_pull<8, 16, true, false> : &k_pull<8, 16, false, false>;
    case 32: return chg ? &k_pull<8, 32, true, false> : &k_pull<8, 32, false, false>;
  }
  return nullptr;
}

}  // namespace pg
