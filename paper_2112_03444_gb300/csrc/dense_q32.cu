// Dense total-degree tracking kernels: degree 2, mixed FP32/FP64, n = 1..12.
// lanes = 0 selects the default group width; lanes = 32 one path per warp with
// every row's contraction split over the warp (autotuner candidate).
#include "dense_kernel.cuh"

namespace hc {

KernelRef dense_ref_d2_32(int n, int lanes) {
  if (lanes == 32) {
    switch (n) {
      case 1: return dense_ref<2, true, 1, 32>();
      case 2: return dense_ref<2, true, 2, 32>();
      case 3: return dense_ref<2, true, 3, 32>();
      case 4: return dense_ref<2, true, 4, 32>();
      case 5: return dense_ref<2, true, 5, 32>();
      case 6: return dense_ref<2, true, 6, 32>();
      case 7: return dense_ref<2, true, 7, 32>();
      case 8: return dense_ref<2, true, 8, 32>();
      case 9: return dense_ref<2, true, 9, 32>();
      case 10: return dense_ref<2, true, 10, 32>();
      case 11: return dense_ref<2, true, 11, 32>();
      case 12: return dense_ref<2, true, 12, 32>();
      default: break;
    }
  }
  switch (n) {
    case 1: return dense_ref<2, true, 1>();
    case 2: return dense_ref<2, true, 2>();
    case 3: return dense_ref<2, true, 3>();
    case 4: return dense_ref<2, true, 4>();
    case 5: return dense_ref<2, true, 5>();
    case 6: return dense_ref<2, true, 6>();
    case 7: return dense_ref<2, true, 7>();
    case 8: return dense_ref<2, true, 8>();
    case 9: return dense_ref<2, true, 9>();
    case 10: return dense_ref<2, true, 10>();
    case 11: return dense_ref<2, true, 11>();
    case 12: return dense_ref<2, true, 12>();
    default: return KernelRef{nullptr, 0};
  }
}

}  // namespace hc
