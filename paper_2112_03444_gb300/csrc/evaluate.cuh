// Evaluation of the homotopy at given points with the tracker's own
// evaluators (hc_evaluate): for point k, lane group k writes the point into
// the group's shared copies exactly as the tracker does before an
// evaluation, calls eval<R> once and stores row i of dH/dx, H_i and dH_i/dt.
// The paper (Sec. 6) evaluates dH/dx, dH/dt and H together in one pass; this
// is that pass, exposed so that it can be checked point by point.
#pragma once

#include "kernels.cuh"
#include "tracker.cuh"

namespace hc {

template <int N, int L, class R, class PROB>
__device__ __forceinline__ void eval_points(const PROB& prob, const EvalPoints& e,
                                            const Group& g, const GroupMem& sm) {
  using HOM = decltype(prob.hom(0));
  const int64_t gpb = blockDim.x / L;
  const int64_t stride = (int64_t)gridDim.x * gpb;
  const bool act = g.gl < N;
  for (int64_t k = blockIdx.x * gpb + threadIdx.x / L; k < e.n_points; k += stride) {
    HOM hom = prob.hom(e.inst[k]);
    hom.init(g);
    const double2 xv = act ? e.x[k * N + g.gl] : make_double2(0.0, 0.0);
    const cx<double> xk = mk<double>(xv.x, xv.y);
    if (act) {
      sm.vd[g.gl] = xk;
      sm.vf[g.gl] = cvt<float>(xk);
    }
    __syncwarp(g.mask);
    cx<R> x[N];  // the evaluators read the point from shared memory
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = czero<R>();
    cx<R> row[N + 1], H, Ht;
    const double t = e.t[k];
    hom.template eval<R>(x, g.gl, (R)t, (R)(1.0 - t), row, H, Ht);
    if (act) {
      double2* hx = e.Hx + (k * N + g.gl) * N;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const cx<double> v = cvt<double>(row[j]);
        hx[j] = make_double2(v.re, v.im);
      }
      const cx<double> h = cvt<double>(H), ht = cvt<double>(Ht);
      e.H[k * N + g.gl] = make_double2(h.re, h.im);
      e.Ht[k * N + g.gl] = make_double2(ht.re, ht.im);
    }
    __syncwarp(g.mask);
  }
}

}  // namespace hc
