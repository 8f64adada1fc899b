// Dense total-degree tracking kernels: degree 2, double-float arithmetic
// (HC_PREC_DF), n = 1..12, one path per warp with every row's contraction
// split over the warp (the last re-tracking tier of the mixed pipeline, and
// precision HC_PREC_DF).
#include "dense_kernel.cuh"

namespace hc {

KernelRef dense_ref_d2_df(int n) {
  switch (n) {
    case 1: return dense_ref<2, HC_PREC_DF, 1, 32>();
    case 2: return dense_ref<2, HC_PREC_DF, 2, 32>();
    case 3: return dense_ref<2, HC_PREC_DF, 3, 32>();
    case 4: return dense_ref<2, HC_PREC_DF, 4, 32>();
    case 5: return dense_ref<2, HC_PREC_DF, 5, 32>();
    case 6: return dense_ref<2, HC_PREC_DF, 6, 32>();
    case 7: return dense_ref<2, HC_PREC_DF, 7, 32>();
    case 8: return dense_ref<2, HC_PREC_DF, 8, 32>();
    case 9: return dense_ref<2, HC_PREC_DF, 9, 32>();
    case 10: return dense_ref<2, HC_PREC_DF, 10, 32>();
    case 11: return dense_ref<2, HC_PREC_DF, 11, 32>();
    case 12: return dense_ref<2, HC_PREC_DF, 12, 32>();
    default: return KernelRef{nullptr, 0};
  }
}

}  // namespace hc
