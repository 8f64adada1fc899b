// Parameter-homotopy (term table) tracking kernels, FP64, n = 1..24.
// lanes = 0 selects the default group width; the mixed kernels also come
// with one path per warp (lanes = 32) for the autotuner.
#include "term_param.cuh"

namespace hc {

KernelRef term_ref_64(int n, int lanes) {
  switch (n) {
    case 1: return term_ref<false, 1>();
    case 2: return term_ref<false, 2>();
    case 3: return term_ref<false, 3>();
    case 4: return term_ref<false, 4>();
    case 5: return term_ref<false, 5>();
    case 6: return term_ref<false, 6>();
    case 7: return term_ref<false, 7>();
    case 8: return term_ref<false, 8>();
    case 9: return term_ref<false, 9>();
    case 10: return term_ref<false, 10>();
    case 11: return term_ref<false, 11>();
    case 12: return term_ref<false, 12>();
    case 13: return term_ref<false, 13>();
    case 14: return term_ref<false, 14>();
    case 15: return term_ref<false, 15>();
    case 16: return term_ref<false, 16>();
    case 17: return term_ref<false, 17>();
    case 18: return term_ref<false, 18>();
    case 19: return term_ref<false, 19>();
    case 20: return term_ref<false, 20>();
    case 21: return term_ref<false, 21>();
    case 22: return term_ref<false, 22>();
    case 23: return term_ref<false, 23>();
    case 24: return term_ref<false, 24>();
    default: return KernelRef{nullptr, 0};
  }
}

}  // namespace hc
