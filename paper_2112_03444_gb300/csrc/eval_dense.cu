// Evaluation kernels of hc_evaluate for dense total-degree systems: degree 2
// with n = 1..12 and degree 3 with n = 1..8, in FP32, FP64 and double-float
// arithmetic, with the group widths of the tracking kernels.
#include <type_traits>

#include "dense_kernel.cuh"
#include "evaluate.cuh"

namespace hc {

template <int N, int DEG, int PREC, int L>
__global__ void __launch_bounds__(kBlock) dense_eval(const DenseEvalArgs ea) {
  using R = typename std::conditional<
      PREC == HC_PREC_MIXED, float,
      typename std::conditional<PREC == HC_PREC_DF, df, double>::type>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const Group g = make_group<L>();
  const GroupMem sm =
      make_group_mem<L>(smem, DenseShape<N, DEG>::EXTRA, 0, 0, PREC == HC_PREC_DF ? 1 : 0);
  DenseProblem<N, DEG, L> prob{&ea.a, sm, g.mask};
  eval_points<N, L, R>(prob, ea.e, g, sm);
}

template <int DEG, int PREC, int N>
KernelRef dense_eval_ref() {
  constexpr int L = PREC == HC_PREC_DF ? 32 : ((N <= 4) ? 4 : (N <= 8) ? 8 : 16);
  return KernelRef{reinterpret_cast<const void*>(&dense_eval<N, DEG, PREC, L>), L,
                   DenseShape<N, DEG>::EXTRA, 0, 0, PREC == HC_PREC_DF ? 1 : 0};
}

template <int DEG, int PREC, int N>
KernelRef pick_dense_eval(int n) {
  if constexpr (N == 0)
    return KernelRef{nullptr, 0};
  else
    return n == N ? dense_eval_ref<DEG, PREC, N>() : pick_dense_eval<DEG, PREC, N - 1>(n);
}

template <int PREC>
KernelRef dense_eval_prec(int deg, int n) {
  if (deg == 2) return pick_dense_eval<2, PREC, 12>(n);
  if (deg == 3) return pick_dense_eval<3, PREC, 8>(n);
  return KernelRef{nullptr, 0};
}

KernelRef dense_eval_kernel(int deg, int n, int prec) {
  if (prec == HC_PREC_MIXED) return dense_eval_prec<HC_PREC_MIXED>(deg, n);
  if (prec == HC_PREC_DF) return dense_eval_prec<HC_PREC_DF>(deg, n);
  return dense_eval_prec<HC_PREC_FP64>(deg, n);
}

}  // namespace hc
