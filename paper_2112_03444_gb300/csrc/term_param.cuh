// Parameter homotopy H(x, t) = F(x; p(t)), p(t) = (1-t) p0 + t p1, evaluated
// from homogenised term tuples (paper Sec. 6).
//
// Every entry of row i -- dH_i/dx_j (j < N), dH_i/dt and H_i -- is a sum of
// K_e tuples (s, m_1, ..., m_D): s * V[m_1] * ... * V[m_D], where V is the
// per-path vector
//   V = [ x_0 .. x_{N-1} | pad to L | 1 | p(t)_0 .. p(t)_{P-1} | dp_0 .. dp_{P-1} | p0 ]
// (dp = p1 - p0 = dp/dt; p0 is kept so that FP32 evaluations form p(t) =
// p0 + t dp without FP64 arithmetic).  As in the paper, every entry is padded to the same
// number of tuples K_e for all rows, and here also to the same number of
// factors D_e (padding factors point at the constant 1), so that the lanes of
// a path -- one row each -- run the same loop.  The library derives the
// tuples symbolically from the term list: x-derivatives by the power rule,
// the t-derivative by the product rule over the parameter factors.
//
// V lives in the lane group's shared memory behind the point written by the
// tracker: FP32 copy for the FP32 tier, FP64 copy for FP64 evaluations.
#pragma once

#include "kernels.cuh"
#include "tracker.cuh"

namespace hc {

// The tuple tables and the V index positions (1 at LS, p(t) at LS + 1, dp at
// LS + 1 + P) use the encoding's lane stride LS = a->ls, independent of the
// kernel's group width L.
template <int N, int L>
struct TermEval {
  const TermArgs* a;
  int64_t inst;
  Group g;
  cx<float>* Vf;
  cx<double>* Vd;

  // constant part of V for this path: the 1, dp and (FP32) p0
  __device__ __forceinline__ void init(const Group&) const {
    const int P = a->P, LS = a->ls;
    const double2* p1 = a->p1 + inst * P;
    if (g.gl == 0) {
      Vf[LS] = mk<float>(1.f, 0.f);
      Vd[LS] = mk<double>(1.0, 0.0);
    }
    for (int l = g.gl; l < P; l += L) {
      const cx<double> d = mk<double>(p1[l].x - a->p0[l].x, p1[l].y - a->p0[l].y);
      Vd[LS + 1 + P + l] = d;
      Vf[LS + 1 + P + l] = cvt<float>(d);
      Vf[LS + 1 + 2 * P + l] = mk<float>((float)a->p0[l].x, (float)a->p0[l].y);
    }
  }

  __device__ __forceinline__ cx<double> start(int64_t path, int i) const {
    const double2 v = a->start[path * N + i];
    return mk<double>(v.x, v.y);
  }

  template <class R>
  __device__ __forceinline__ cx<R>* vptr() const {
    if constexpr (std::is_same<R, float>::value)
      return Vf;
    else
      return Vd;
  }

  // p(t) into V (each lane a share), then wait for the group.  FP64:
  // (1-t) p0 + t p1 from the inputs; FP32: p0 + t dp from the FP32 copies.
  template <class R>
  __device__ __forceinline__ void put_params(R t) const {
    const int P = a->P, LS = a->ls;
    if constexpr (std::is_same<R, float>::value) {
      for (int l = g.gl; l < P; l += L)
        Vf[LS + 1 + l] = cfma(mk<float>(t, 0.f), Vf[LS + 1 + P + l], Vf[LS + 1 + 2 * P + l]);
    } else {
      const double2* p1 = a->p1 + inst * P;
      for (int l = g.gl; l < P; l += L) {
        const double2 q0 = a->p0[l], q1 = p1[l];
        Vd[LS + 1 + l] = mk<double>((1.0 - t) * q0.x + t * q1.x, (1.0 - t) * q0.y + t * q1.y);
      }
    }
    __syncwarp(g.mask);
  }

  template <class R>
  __device__ __forceinline__ cx<R> entry(int e, int i, const cx<R>* V) const {
    const int K = a->kcnt[e], D = a->kdeg[e], base = a->koff[e];
    cx<R> acc = czero<R>();
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      const int64_t r = (int64_t)(base + k) * a->ls + i;
      const TermRec rc = a->rec[r];
      cx<R> prod = V[rc.idx[0]];
#pragma unroll 1
      for (int f = 1; f < D; ++f) prod = prod * V[rc.idx[f]];
      cx<R> s;
      if constexpr (std::is_same<R, float>::value)
        s = mk<float>(rc.s.x, rc.s.y);
      else
        s = mk<double>(a->s64[r].x, a->s64[r].y);
      acc = cfma(s, prod, acc);
    }
    return acc;
  }

  template <class R>
  __device__ __forceinline__ void eval(const cx<R> (&)[N], int i, R t, R, cx<R> (&row)[N + 1],
                                       cx<R>& H, cx<R>& Ht) const {
    put_params<R>(t);
    const cx<R>* V = vptr<R>();
    const int ii = i < N ? i : 0;
#pragma unroll
    for (int j = 0; j < N; ++j) row[j] = entry<R>(j, ii, V);
    Ht = entry<R>(N, ii, V);
    H = entry<R>(N + 1, ii, V);
  }

  template <bool SCALE>
  __device__ __forceinline__ void residual64(const cx<double>*, int i, double t, double,
                                             cx<double>& H, double& sc) const {
    put_params<double>(t);
    const int e = N + 1, K = a->kcnt[e], D = a->kdeg[e], base = a->koff[e];
    const int ii = i < N ? i : 0;
    cx<double> acc = czero<double>();
    float s_abs = 0.f;
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      const int64_t r = (int64_t)(base + k) * a->ls + ii;
      const TermRec rc = a->rec[r];
      cx<double> prod = Vd[rc.idx[0]];
#pragma unroll 1
      for (int f = 1; f < D; ++f) prod = prod * Vd[rc.idx[f]];
      const cx<double> s = mk<double>(a->s64[r].x, a->s64[r].y);
      acc = cfma(s, prod, acc);
      if (SCALE) s_abs += cabs2(cvt<float>(s)) * cabs2(cvt<float>(prod));
    }
    H = acc;
    sc = SCALE ? (double)s_abs : 0.0;
  }
};

template <int N, int L>
struct TermProblem {
  const TermArgs* a;
  Group g;
  GroupMem sm;
  __device__ __forceinline__ TermEval<N, L> hom(int64_t inst) const {
    return TermEval<N, L>{a, inst, g, sm.vf, sm.vd};
  }
};

template <int N, bool MIXED, int L>
__global__ void __launch_bounds__(kBlock) term_param_kernel(const __grid_constant__ TermArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Group g = make_group<L>();
  const GroupMem sm = make_group_mem<L>(smem, a.extra);
  TermProblem<N, L> prob{&a, g, sm};
  run_tracker<N, L, MIXED>(prob, a.c, g, sm);
}

template <bool MIXED, int N, int LANES = 0>
KernelRef term_ref() {
  constexpr int L = LANES ? LANES : ((N <= 4) ? 4 : (N <= 8) ? 8 : (N <= 16) ? 16 : 32);
  return KernelRef{reinterpret_cast<const void*>(&term_param_kernel<N, MIXED, L>), L};
}

}  // namespace hc
