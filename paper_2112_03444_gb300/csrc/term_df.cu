// Parameter-homotopy (term table) tracking kernels in double-float
// arithmetic (HC_PREC_DF), n = 1..24, default group width (the last
// re-tracking tier of the mixed pipeline, and precision HC_PREC_DF).
#include "term_param.cuh"

namespace hc {

KernelRef term_ref_df(int n) {
  switch (n) {
    case 1: return term_ref<HC_PREC_DF, 1>();
    case 2: return term_ref<HC_PREC_DF, 2>();
    case 3: return term_ref<HC_PREC_DF, 3>();
    case 4: return term_ref<HC_PREC_DF, 4>();
    case 5: return term_ref<HC_PREC_DF, 5>();
    case 6: return term_ref<HC_PREC_DF, 6>();
    case 7: return term_ref<HC_PREC_DF, 7>();
    case 8: return term_ref<HC_PREC_DF, 8>();
    case 9: return term_ref<HC_PREC_DF, 9>();
    case 10: return term_ref<HC_PREC_DF, 10>();
    case 11: return term_ref<HC_PREC_DF, 11>();
    case 12: return term_ref<HC_PREC_DF, 12>();
    case 13: return term_ref<HC_PREC_DF, 13>();
    case 14: return term_ref<HC_PREC_DF, 14>();
    case 15: return term_ref<HC_PREC_DF, 15>();
    case 16: return term_ref<HC_PREC_DF, 16>();
    case 17: return term_ref<HC_PREC_DF, 17>();
    case 18: return term_ref<HC_PREC_DF, 18>();
    case 19: return term_ref<HC_PREC_DF, 19>();
    case 20: return term_ref<HC_PREC_DF, 20>();
    case 21: return term_ref<HC_PREC_DF, 21>();
    case 22: return term_ref<HC_PREC_DF, 22>();
    case 23: return term_ref<HC_PREC_DF, 23>();
    case 24: return term_ref<HC_PREC_DF, 24>();
    default: return KernelRef{nullptr, 0};
  }
}

}  // namespace hc
