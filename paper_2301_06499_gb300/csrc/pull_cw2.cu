// Pull kernels with 2 signature word(s) per lane load sequence.
#include "kernels.cuh"

namespace pg {

PullFn pull_fn_cw2(int G, bool chg, bool eb) {
  if (eb) return nullptr;
  switch (G) {
    case 2: return chg ? &k_pull<2, 2, true, false> : &k_pull<2, 2, false, false>;
    case 4: return chg ? &k_pull<2, 4, true, false> : &k_pull<2, 4, false, false>;
    case 8: return chg ? &k_pull<2, 8, true, false> : &k_pull<2, 8, false, false>;
    case 16: return chg ? &k_pull<2, 16, true, false> : &k_pull<2, 16, false, false>;
    case 32: return chg ? &k_pull<2, 32, true, false> : &k_pull<2, 32, false, false>;
  }
  return nullptr;
}

}  // namespace pg
