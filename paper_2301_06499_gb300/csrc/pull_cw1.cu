// Pull kernels with 1 signature word(s) per gather.
#include "kernels.cuh"

namespace pg {

PullFn pull_fn_cw1(int G) {
  switch (G) {
    case 1: return &k_pull<1, 1>;
    case 2: return &k_pull<1, 2>;
    case 4: return &k_pull<1, 4>;
    case 8: return &k_pull<1, 8>;
    case 16: return &k_pull<1, 16>;
    case 32: return &k_pull<1, 32>;
  }
  return nullptr;
}

}  // namespace pg
