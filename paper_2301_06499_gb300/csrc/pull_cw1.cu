// Pull kernels with 1 signature word(s) per gather.
#include "kernels.cuh"

namespace pg {

template <bool PW>
static PullFn pick(int G) {
  switch (G) {
    case 1: return &k_pull<1, 1, PW>;
    case 2: return &k_pull<1, 2, PW>;
    case 4: return &k_pull<1, 4, PW>;
    case 8: return &k_pull<1, 8, PW>;
    case 16: return &k_pull<1, 16, PW>;
    case 32: return &k_pull<1, 32, PW>;
  }
  return nullptr;
}

PullFn pull_fn_cw1(int G, bool pw) { return pw ? pick<true>(G) : pick<false>(G); }

}  // namespace pg
