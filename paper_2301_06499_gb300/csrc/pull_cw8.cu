// Pull kernels with 8 signature word(s) per gather.
#include "kernels.cuh"

namespace pg {

PullFn pull_fn_cw8(int G) {
  switch (G) {
    case 1: return &k_pull<8, 1>;
    case 2: return &k_pull<8, 2>;
    case 4: return &k_pull<8, 4>;
    case 8: return &k_pull<8, 8>;
    case 16: return &k_pull<8, 16>;
    case 32: return &k_pull<8, 32>;
  }
  return nullptr;
}

}  // namespace pg
