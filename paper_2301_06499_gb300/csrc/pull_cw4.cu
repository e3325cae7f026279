// Pull kernels with 4 signature word(s) per gather.
#include "kernels.cuh"

namespace pg {

PullFn pull_fn_cw4(int G) {
  switch (G) {
    case 1: return &k_pull<4, 1>;
    case 2: return &k_pull<4, 2>;
    case 4: return &k_pull<4, 4>;
    case 8: return &k_pull<4, 8>;
    case 16: return &k_pull<4, 16>;
    case 32: return &k_pull<4, 32>;
  }
  return nullptr;
}

}  // namespace pg
