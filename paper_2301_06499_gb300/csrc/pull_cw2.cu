// Pull kernels with 2 signature word(s) per gather.
#include "kernels.cuh"

namespace pg {

PullFn pull_fn_cw2(int G) {
  switch (G) {
    case 1: return &k_pull<2, 1>;
    case 2: return &k_pull<2, 2>;
    case 4: return &k_pull<2, 4>;
    case 8: return &k_pull<2, 8>;
    case 16: return &k_pull<2, 16>;
    case 32: return &k_pull<2, 32>;
  }
  return nullptr;
}

}  // namespace pg
