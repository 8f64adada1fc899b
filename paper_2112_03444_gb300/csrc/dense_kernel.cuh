// The persistent dense total-degree tracking kernel (instantiated per n,
// degree and precision in dense_*.cu).
#pragma once

#include "dense_td.cuh"
#include "kernels.cuh"
#include "tracker.cuh"

namespace hc {

template <int N, int DEG, bool MIXED>
__global__ void __launch_bounds__(kBlock) dense_td_kernel(const DenseArgs a) {
  constexpr int L = (N <= 4) ? 4 : (N <= 8) ? 8 : (N <= 16) ? 16 : 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const Group g = make_group<L>();
  const int grp = threadIdx.x / L;
  cx<double>* vb = reinterpret_cast<cx<double>*>(smem) + grp * 2 * L;
  void* sb = vb + L;
  const LaunchCommon& c = a.c;
  const int64_t total = c.count_dev ? (int64_t)(*c.count_dev) : c.n_items;
  const int leader = g.wl & ~(L - 1);
#pragma unroll 1
  for (;;) {
    __syncwarp(g.mask);
    unsigned long long it = 0;
    if (g.gl == 0) it = atomicAdd(c.queue, 1ull);
    it = __shfl_sync(g.mask, it, leader);
    if ((int64_t)it >= total) break;
    const int64_t item = c.items ? c.items[it] : (int64_t)it;
    const int64_t inst = item / c.paths;
    const int64_t path = item - inst * c.paths;
    DenseTD<N, DEG, L> hom;
    hom.D32 = a.D32 ? a.D32 + inst * a.Dstride : nullptr;
    hom.D64 = a.D64 ? a.D64 + inst * a.Dstride : nullptr;
    hom.E = a.E + inst * a.Estride;
    hom.gamma = a.gamma;
    PathOut o;
    track_path<N, L, MIXED>(hom, c.s, g, vb, sb, path, o);
    if (g.gl < N)
      reinterpret_cast<double2*>(c.x_out)[item * N + g.gl] = make_double2(o.x.re, o.x.im);
    if (g.gl == 0) {
      c.status_out[item] = (uint8_t)o.status;
      c.steps_out[item * 3 + 0] = o.nacc;
      c.steps_out[item * 3 + 1] = o.nrej;
      c.steps_out[item * 3 + 2] = o.nnewt;
      if (c.be_out) c.be_out[item] = (double)o.be;
      if (MIXED && c.esc_list && (o.status & 0x7f) != ST_FINITE) {
        const unsigned long long pos = atomicAdd(c.esc_count, 1ull);
        c.esc_list[pos] = item;
      }
    }
  }
}

template <int DEG, bool MIXED, int N>
KernelRef dense_ref() {
  return KernelRef{reinterpret_cast<const void*>(&dense_td_kernel<N, DEG, MIXED>), lanes_for(N)};
}

}  // namespace hc
