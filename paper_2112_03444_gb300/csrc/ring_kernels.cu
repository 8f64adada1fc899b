// The resident-launch variants of the mixed-precision tracking kernels
// (hc_stream): default group width, dense degree 2 (n = 1..12) and 3
// (n = 1..8), term tables (n = 1..24).  The batch kernels carry none of the
// ring code (it cost 2-5 % of their time when compiled in).
#include "dense_kernel.cuh"
#include "term_param.cuh"

namespace hc {

template <int DEG, int N>
KernelRef pick_dense_ring(int n) {
  if constexpr (N == 0)
    return KernelRef{nullptr, 0};
  else
    return n == N ? dense_ref<DEG, HC_PREC_MIXED, N, 0, true>() : pick_dense_ring<DEG, N - 1>(n);
}

template <int N>
KernelRef pick_term_ring(int n) {
  if constexpr (N == 0)
    return KernelRef{nullptr, 0};
  else
    return n == N ? term_ref<HC_PREC_MIXED, N, 0, true>() : pick_term_ring<N - 1>(n);
}

KernelRef ring_kernel(bool terms, int deg, int n) {
  if (terms) return pick_term_ring<24>(n);
  if (deg == 2) return pick_dense_ring<2, 12>(n);
  if (deg == 3) return pick_dense_ring<3, 8>(n);
  return KernelRef{nullptr, 0};
}

}  // namespace hc
