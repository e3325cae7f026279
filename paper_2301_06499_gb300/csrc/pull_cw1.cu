// Pull kernels with 1 signature word(s) per lane load sequence.
#include "kernels.cuh"

namespace pg {

PullFn pull_fn_cw1(int G, bool chg, bool eb) {
  if (eb) {
    switch (G) {
      case 2: return chg ? &k_pull<1, 2, true, true> : &k_pull<1, 2, false, true>;
      case 4: return chg ? &k_pull<1, 4, true, true> : &k_pull<1, 4, false, true>;
      case 8: return chg ? &k_pull<1, 8, true, true> : &k_pull<1, 8, false, true>;
      case 16: return chg ? &k_pull<1, 16, true, true> : &k_pull<1, 16, false, true>;
      case 32: return chg ? &k_pull<1, 32, true, true> : &k_pull<1, 32, false, true>;
    }
    return nullptr;
  }
  switch (G) {
    case 2: return chg ? &k_pull<1, 2, true, false> : &k_pull<1, 2, false, false>;
    case 4: return chg ? &k_pull<1, 4, true, false> : &k_pull<1, 4, false, false>;
    case 8: return chg ? &k_pull<1, 8, true, false> : &k_pull<1, 8, false, false>;
    case 16: return chg ? &k_pull<1, 16, true, false> : &k_pull<1, 16, false, false>;
    case 32: return chg ? &k_pull<1, 32, true, false> : &k_pull<1, 32, false, false>;
  }
  return nullptr;
}

}  // namespace pg
