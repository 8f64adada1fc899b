// Evaluation kernels of hc_evaluate for parameter and coefficient-
// interpolation homotopies (term tables), n = 1..24, in FP32, FP64 and
// double-float arithmetic, with the default group width of the tracking
// kernels.
#include <type_traits>

#include "evaluate.cuh"
#include "term_param.cuh"

namespace hc {

template <int N, int PREC, int L>
__global__ void __launch_bounds__(kBlock) term_eval(const __grid_constant__ TermEvalArgs ea) {
  constexpr bool MIXED = PREC == HC_PREC_MIXED;
  using R = typename std::conditional<
      MIXED, float, typename std::conditional<PREC == HC_PREC_DF, df, double>::type>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const Group g = make_group<L>();
  const GroupMem sm = make_group_mem<L>(smem, ea.a.extra, term_acc_bytes<N, MIXED, L>(), 0,
                                        PREC == HC_PREC_DF ? 1 : 0);
  TermProblem<N, L, MIXED> prob{&ea.a, g, sm};
  eval_points<N, L, R>(prob, ea.e, g, sm);
}

template <int PREC, int N>
KernelRef term_eval_ref() {
  constexpr int L = (N <= 4) ? 4 : (N <= 8) ? 8 : (N <= 16) ? 16 : 32;
  return KernelRef{reinterpret_cast<const void*>(&term_eval<N, PREC, L>), L, 0,
                   term_acc_bytes<N, PREC == HC_PREC_MIXED, L>(), 0,
                   PREC == HC_PREC_DF ? 1 : 0};
}

template <int PREC, int N>
KernelRef pick_term_eval(int n) {
  if constexpr (N == 0)
    return KernelRef{nullptr, 0};
  else
    return n == N ? term_eval_ref<PREC, N>() : pick_term_eval<PREC, N - 1>(n);
}

KernelRef term_eval_kernel(int n, int prec) {
  if (prec == HC_PREC_MIXED) return pick_term_eval<HC_PREC_MIXED, 24>(n);
  if (prec == HC_PREC_DF) return pick_term_eval<HC_PREC_DF, 24>(n);
  return pick_term_eval<HC_PREC_FP64, 24>(n);
}

}  // namespace hc
