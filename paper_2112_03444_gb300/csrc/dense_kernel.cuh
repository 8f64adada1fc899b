// The persistent dense total-degree tracking kernel (instantiated per n,
// degree and precision in dense_*.cu).
#pragma once

#include "dense_td.cuh"
#include "kernels.cuh"
#include "tracker.cuh"

namespace hc {

template <int N, int DEG, int L>
struct DenseProblem {
  const DenseArgs* a;
  GroupMem sm;
  unsigned gmask;
  __device__ __forceinline__ DenseTD<N, DEG, L> hom(int64_t inst) const {
    DenseTD<N, DEG, L> h;
    h.gmask = gmask;
    h.D32 = a->D32 ? a->D32 + inst * a->Dstride : nullptr;
    h.D64 = a->D64 ? a->D64 + inst * a->Dstride : nullptr;
    h.E = a->E + inst * a->Estride;
    h.Edf = a->Edf ? a->Edf + inst * a->Estride : nullptr;
    h.gammadf = a->gammadf;
    h.gamma = a->gamma;
    h.gamma32 = a->gamma32;
    h.Vf = sm.vf;
    h.Vd = sm.vd;
    return h;
  }
};

template <int N, int DEG, bool MIXED, int L>
__global__ void __launch_bounds__(kBlock, 4) dense_td_kernel(const DenseArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Group g = make_group<L>();
  const GroupMem sm =
      make_group_mem<L>(smem, DenseShape<N, DEG>::EXTRA, 0, endgame_smem_bytes(L, MIXED));
  DenseProblem<N, DEG, L> prob{&a, sm, g.mask};
  run_tracker<N, L, MIXED>(prob, a.c, g, sm);
}

// lanes = 0: the default lanes_for(N); otherwise that group width.
template <int DEG, bool MIXED, int N, int LANES = 0>
KernelRef dense_ref() {
  constexpr int L = LANES ? LANES : ((N <= 4) ? 4 : (N <= 8) ? 8 : (N <= 16) ? 16 : 32);
  return KernelRef{reinterpret_cast<const void*>(&dense_td_kernel<N, DEG, MIXED, L>), L,
                   DenseShape<N, DEG>::EXTRA, 0, endgame_smem_bytes(L, MIXED)};
}

}  // namespace hc
