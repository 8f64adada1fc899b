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
  static_assert(sizeof(GroupSmem<L>) == kGroupSmemBytesPerLane * L, "group smem layout");
  extern __shared__ __align__(16) unsigned char smem[];
  const Group g = make_group<L>();
  GroupSmem<L>* sm = reinterpret_cast<GroupSmem<L>*>(smem) + threadIdx.x / L;
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
    double t0 = 0.0;
    const double2* x0 = nullptr;
    if (!MIXED && c.t_io) {
      t0 = c.t_io[item];
      if (t0 > 0.0) x0 = reinterpret_cast<const double2*>(c.x_out) + item * N;
    }
    PathOut o;
    track_path<N, L, MIXED>(hom, c.s, g, sm, path, t0, x0, o);
    __syncwarp(g.mask);  // every lane has read its resume state before it is overwritten
    const int base = o.status & 0x7f;
    if (g.gl < N) {
      reinterpret_cast<double2*>(c.x_out)[item * N + g.gl] = make_double2(o.x.re, o.x.im);
      if (MIXED && c.x32_out)
        c.x32_out[item * N + g.gl] = base == ST_FINITE
                                         ? make_float2((float)o.x.re, (float)o.x.im)
                                         : make_float2(__int_as_float(0x7fc00000), 0.f);
    }
    if (g.gl == 0) {
      c.status_out[item] = (uint8_t)o.status;
      if (c.be_out) c.be_out[item] = (double)o.be;
      if (MIXED) {
        c.steps_out[item * 3 + 0] = o.nacc;
        c.steps_out[item * 3 + 1] = o.nrej;
        c.steps_out[item * 3 + 2] = o.nnewt;
        if (c.esc_list && base != ST_FINITE) {
          // resume point for the FP64 tier: the last accepted point for a
          // step-size or budget failure, t = 1 (refine + exact condition)
          // for a suspect-condition endpoint, a fresh start otherwise
          if (c.t_io)
            c.t_io[item] = (base == ST_FAIL_STEP || base == ST_FAIL_MAXSTEPS) ? o.t
                           : (base == ST_SINGULAR)                            ? 1.0
                                                                             : 0.0;
          const unsigned long long pos = atomicAdd(c.esc_count, 1ull);
          c.esc_list[pos] = item;
        } else if (c.t_io) {
          c.t_io[item] = 0.0;
        }
      } else {
        c.steps_out[item * 3 + 0] += o.nacc;
        c.steps_out[item * 3 + 1] += o.nrej;
        c.steps_out[item * 3 + 2] += o.nnewt;
        if (c.esc_steps) {
          atomicAdd(c.esc_steps + 0, (unsigned long long)o.nacc);
          atomicAdd(c.esc_steps + 1, (unsigned long long)o.nrej);
          atomicAdd(c.esc_steps + 2, (unsigned long long)o.nnewt);
        }
      }
    }
  }
}

template <int DEG, bool MIXED, int N>
KernelRef dense_ref() {
  return KernelRef{reinterpret_cast<const void*>(&dense_td_kernel<N, DEG, MIXED>), lanes_for(N)};
}

}  // namespace hc
