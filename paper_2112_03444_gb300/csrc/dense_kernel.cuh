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
    h.Ddf = a->Ddf ? a->Ddf + inst * a->Dstride : nullptr;
    h.E = a->E + inst * a->Estride;
    h.Edf = a->Edf ? a->Edf + inst * a->Estride : nullptr;
    h.gammadf = a->gammadf;
    h.gamma = a->gamma;
    h.gamma32 = a->gamma32;
    h.Vf = sm.vf;
    h.Vd = sm.vd;
    h.Vx = sm.vx;
    return h;
  }
};

// Resident blocks per SM the FP32 and FP64 kernels are compiled for (128
// registers a thread); 3 and 5 (168 and 96 registers) measured no faster on
// the cubic n = 8 and quadratic n = 12 classes.
constexpr int kTrackMinBlocks = 4;

// PREC: HC_PREC_MIXED (FP32 tracking, FP64 state where needed),
// HC_PREC_FP64, or HC_PREC_DF (FP64 state, double-float evaluation and
// solve).  The double-float kernels hold every complex number in four
// registers and run one path per warp: they get the registers of one block
// per SM rather than of four.
template <int N, int DEG, int PREC, int L, bool RING = false>
__global__ void __launch_bounds__(kBlock, PREC == HC_PREC_DF ? 1 : kTrackMinBlocks)
    dense_td_kernel(const DenseArgs a) {
  constexpr bool MIXED = PREC == HC_PREC_MIXED;
  constexpr bool XDF = PREC == HC_PREC_DF;
  using RE = typename std::conditional<XDF, df, double>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const Group g = make_group<L>();
  const GroupMem sm = make_group_mem<L>(smem, DenseShape<N, DEG>::EXTRA, 0,
                                        endgame_smem_bytes(L, MIXED), XDF ? 1 : 0);
  DenseProblem<N, DEG, L> prob{&a, sm, g.mask};
  run_tracker<N, L, MIXED, DenseProblem<N, DEG, L>, RE, RING>(prob, a.c, g, sm);
}

// lanes = 0: the default lanes_for(N); otherwise that group width.  RING:
// the resident-launch variant (hc_stream).
template <int DEG, int PREC, int N, int LANES = 0, bool RING = false>
KernelRef dense_ref() {
  constexpr int L = LANES ? LANES : ((N <= 4) ? 4 : (N <= 8) ? 8 : (N <= 16) ? 16 : 32);
  return KernelRef{reinterpret_cast<const void*>(&dense_td_kernel<N, DEG, PREC, L, RING>), L,
                   DenseShape<N, DEG>::EXTRA, 0, endgame_smem_bytes(L, PREC == HC_PREC_MIXED),
                   PREC == HC_PREC_DF ? 1 : 0};
}

}  // namespace hc
