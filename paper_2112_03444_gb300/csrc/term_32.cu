// Parameter-homotopy (term table) tracking kernels, mixed FP32/FP64, n = 1..24.
// lanes = 0 selects the default group width; the mixed kernels also come
// with one path per warp (lanes = 32) for the autotuner.
#include "term_param.cuh"

namespace hc {

KernelRef term_ref_32(int n, int lanes) {
  if (lanes == 32) {
    switch (n) {
      case 1: return term_ref<true, 1, 32>();
      case 2: return term_ref<true, 2, 32>();
      case 3: return term_ref<true, 3, 32>();
      case 4: return term_ref<true, 4, 32>();
      case 5: return term_ref<true, 5, 32>();
      case 6: return term_ref<true, 6, 32>();
      case 7: return term_ref<true, 7, 32>();
      case 8: return term_ref<true, 8, 32>();
      case 9: return term_ref<true, 9, 32>();
      case 10: return term_ref<true, 10, 32>();
      case 11: return term_ref<true, 11, 32>();
      case 12: return term_ref<true, 12, 32>();
      case 13: return term_ref<true, 13, 32>();
      case 14: return term_ref<true, 14, 32>();
      case 15: return term_ref<true, 15, 32>();
      case 16: return term_ref<true, 16, 32>();
      default: break;
    }
  }
  switch (n) {
    case 1: return term_ref<true, 1>();
    case 2: return term_ref<true, 2>();
    case 3: return term_ref<true, 3>();
    case 4: return term_ref<true, 4>();
    case 5: return term_ref<true, 5>();
    case 6: return term_ref<true, 6>();
    case 7: return term_ref<true, 7>();
    case 8: return term_ref<true, 8>();
    case 9: return term_ref<true, 9>();
    case 10: return term_ref<true, 10>();
    case 11: return term_ref<true, 11>();
    case 12: return term_ref<true, 12>();
    case 13: return term_ref<true, 13>();
    case 14: return term_ref<true, 14>();
    case 15: return term_ref<true, 15>();
    case 16: return term_ref<true, 16>();
    case 17: return term_ref<true, 17>();
    case 18: return term_ref<true, 18>();
    case 19: return term_ref<true, 19>();
    case 20: return term_ref<true, 20>();
    case 21: return term_ref<true, 21>();
    case 22: return term_ref<true, 22>();
    case 23: return term_ref<true, 23>();
    case 24: return term_ref<true, 24>();
    default: return KernelRef{nullptr, 0};
  }
}

}  // namespace hc
