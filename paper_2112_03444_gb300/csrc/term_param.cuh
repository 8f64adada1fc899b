// Parameter homotopy H(x, t) = F(x; p(t)), p(t) = (1-t) p0 + t p1, evaluated
// from the terms of the equations (paper Sec. 6).
//
// Every term of equation i is a coefficient times a product of factors
// taken from the per-path vector
//   V = [ x_0 .. x_{N-1} | pad to L | 1 | p(t)_0 .. p(t)_{P-1} | dp_0 .. dp_{P-1} | p0 ]
// (dp = p1 - p0 = dp/dt; p0 is kept so that FP32 evaluations form p(t) =
// p0 + t dp without FP64 arithmetic); a power x_j^a is a repeated factor.
// Lane i evaluates row i: for each term it forms the prefix products of the
// factors, then walks them backwards with the suffix product, so that one
// pass yields the term itself (its contribution to H_i) and its derivative
// with respect to every factor (product rule; a repeated factor contributes
// once per occurrence, which is the power rule).  A derivative with respect
// to x_j adds to dH_i/dx_j, one with respect to a parameter adds, times
// dp, to dH_i/dt.  Those targets differ from term to term, so each lane
// accumulates its row in its own slice of shared memory and reads the row
// back at the end.  The paper's homogenised tuples enumerate every entry of
// the Jacobian row as separate factor products; this form shares the
// products between all entries of a term.
//
// The term tables are padded per row to the same number of term slots and,
// at each slot, to the same number of factors (padding factor: the 1), so
// that the lanes of a path -- one row each -- and the paths of a warp run
// the same loop.
#pragma once

#include "kernels.cuh"
#include "tracker.cuh"

namespace hc {

// The term tables and the V index positions (1 at LS, p(t) at LS + 1, dp at
// LS + 1 + P, p0 at LS + 1 + 2P) use the encoding's lane stride LS = a->ls,
// independent of the kernel's group width L.
//
// The high-precision copy of V (Vd, 16 bytes per entry) holds complex FP64
// in the all-FP64 kernels and double-floats (dfloat.cuh) in the
// mixed-precision ones (DF), whose residuals run in double-float arithmetic.
// Sum of a lane's value and its partner's (lane xor o), the lower lane's
// value first on both lanes so that the two copies agree bit for bit.
template <class R>
__device__ __forceinline__ R pair_sum(R v, int o, bool upper) {
  R w;
  if constexpr (std::is_same<R, df>::value)
    w = shfl_xor_df(v, o);
  else
    w = __shfl_xor_sync(0xffffffffu, v, o);
  return upper ? w + v : v + w;
}
template <class R>
__device__ __forceinline__ cx<R> pair_sum(cx<R> v, int o, bool upper) {
  return {pair_sum<R>(v.re, o, upper), pair_sum<R>(v.im, o, upper)};
}
__device__ __forceinline__ cdf pair_sum(cdf v, int o, bool upper) {
  const cdf w{__shfl_xor_sync(0xffffffffu, v.hr, o), __shfl_xor_sync(0xffffffffu, v.hi_, o),
              __shfl_xor_sync(0xffffffffu, v.lr, o), __shfl_xor_sync(0xffffffffu, v.li, o)};
  return upper ? cdf_add(w, v) : cdf_add(v, w);
}

template <int N, int L, bool DF>
struct TermEval {
  // One path per warp (L = 32, N <= 16; the autotuner's lanes = 32
  // candidate): every row on two lanes, each taking every other term slot,
  // so that the warp's lanes all work.  Otherwise one row per lane.
  static constexpr int PARTS = (L == 32 && N <= 16) ? 2 : 1;
  static constexpr int ROWL = L / PARTS;
  // residuals are computed by each group alone (no cooperative form)
  static constexpr bool kCoop = false;
  const TermArgs* a;
  int64_t inst;
  Group g;
  cx<float>* Vf;
  cx<double>* Vd;
  unsigned char* acc;  // [N + 2][L] accumulators of cx<R>, this lane at column g.gl
  cx<df>* Vx;          // double-float kernels: V as double-floats; nullptr otherwise

  // constant part of V for this path: the 1, dp and p0 (FP32 copies, and
  // for DF double-float copies of dp and p0 in Vd)
  __device__ __forceinline__ void init(const Group&) const {
    const int P = a->P, LS = a->ls;
    const double2* p1 = a->p1 + inst * P;
    cdf* Vdf = reinterpret_cast<cdf*>(Vd);
    if (g.gl == 0) {
      Vf[LS] = mk<float>(1.f, 0.f);
      if constexpr (DF)
        Vdf[LS] = cdf{1.f, 0.f, 0.f, 0.f};
      else
        Vd[LS] = mk<double>(1.0, 0.0);
    }
    if (Vx && g.gl == 0) Vx[LS] = mk<df>(df(1), df(0));
    for (int l = g.gl; l < P; l += L) {
      const cx<double> d = mk<double>(p1[l].x - a->p0[l].x, p1[l].y - a->p0[l].y);
      if (Vx) {
        Vx[LS + 1 + P + l] = to_cxdf(d);
        Vx[LS + 1 + 2 * P + l] = to_cxdf(mk<double>(a->p0[l].x, a->p0[l].y));
      }
      if constexpr (DF) {
        Vdf[LS + 1 + P + l] = to_cdf(d);
        Vdf[LS + 1 + 2 * P + l] = to_cdf(mk<double>(a->p0[l].x, a->p0[l].y));
      } else {
        Vd[LS + 1 + P + l] = d;
      }
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
    else if constexpr (std::is_same<R, df>::value)
      return Vx;
    else
      return Vd;
  }

  // p(t) into V (each lane a share), then wait for the group.  FP64:
  // (1-t) p0 + t p1 from the inputs; FP32: p0 + t dp from the FP32 copies;
  // double-float: p0 + t dp from the double-float copies, and the point
  // (which the tracker keeps in FP64 in Vd) split into double-floats.
  template <class R>
  __device__ __forceinline__ void put_params(R t) const {
    const int P = a->P, LS = a->ls;
    if constexpr (std::is_same<R, float>::value) {
      for (int l = g.gl; l < P; l += L)
        Vf[LS + 1 + l] = cfma(mk<float>(t, 0.f), Vf[LS + 1 + P + l], Vf[LS + 1 + 2 * P + l]);
    } else if constexpr (std::is_same<R, df>::value) {
      if (g.gl < N) Vx[g.gl] = to_cxdf(Vd[g.gl]);
      for (int l = g.gl; l < P; l += L) Vx[LS + 1 + l] = Vx[LS + 1 + 2 * P + l] + t * Vx[LS + 1 + P + l];
    } else {
      const double2* p1 = a->p1 + inst * P;
      // DF: the 1 of V is held as a double-float between FP64 residuals
      if (DF && g.gl == 0) Vd[LS] = mk<double>(1.0, 0.0);
      for (int l = g.gl; l < P; l += L) {
        const double2 q0 = a->p0[l], q1 = p1[l];
        Vd[LS + 1 + l] = mk<double>((1.0 - t) * q0.x + t * q1.x, (1.0 - t) * q0.y + t * q1.y);
      }
    }
    __syncwarp(g.mask);
  }

  // One term of D factors: add its value to h and its derivatives to the
  // lane's accumulators (the coefficient rides in the suffix product).
  // Returns the product of the factors (without the coefficient).
  template <int D, class R>
  __device__ __forceinline__ cx<R> term(const TermRec& rc, cx<R> s, const cx<R>* V, cx<R>* A,
                                        cx<R>& h) const {
    cx<R> pre[D];
    cx<R> run = mk<R>(R(1), R(0));
#pragma unroll
    for (int f = 0; f < D; ++f) {
      pre[f] = run;
      run = run * V[rc.idx[f]];
    }
    h = cfma(s, run, h);
    cx<R> suf = s;
#pragma unroll
    for (int f = D - 1; f >= 0; --f) {
      const int tg = rc.tgt[f];
      const cx<R> v = V[rc.idx[f]];
      const cx<R> dv = pre[f] * suf;
      if (tg < N) {
        A[tg * L] = A[tg * L] + dv;
      } else if (tg == N) {  // a parameter factor: d/dt through dp
        A[N * L] = cfma(dv, V[rc.idx[f] + a->P], A[N * L]);
      }
      if (f > 0) suf = suf * v;
    }
    return run;
  }

  // Coefficient interpolation (a->coef_mode): the coefficient of record r
  // at time t, c0 + t dc, and its t-derivative dc, for this instance.
  template <class R>
  __device__ __forceinline__ void coef_at(int64_t r, R t, cx<R>& s, cx<R>& dcr) const {
    const int64_t rd = inst * (int64_t)a->TT * a->ls + r;
    if constexpr (std::is_same<R, float>::value) {
      const float2 c = a->c0f[r], d = a->dcf[rd];
      dcr = mk<float>(d.x, d.y);
      s = cfma(mk<float>(t, 0.f), dcr, mk<float>(c.x, c.y));
    } else if constexpr (std::is_same<R, df>::value) {
      dcr = to_cxdf(a->dcdf[rd]);
      s = to_cxdf(a->c0df[r]) + t * dcr;
    } else {
      const double2 c = a->c0[r], d = a->dc[rd];
      dcr = mk<double>(d.x, d.y);
      s = cfma(mk<double>(t, 0.0), dcr, mk<double>(c.x, c.y));
    }
  }

  template <class R>
  __device__ __forceinline__ void eval(const cx<R> (&)[N], int i, R t, R, cx<R> (&row)[N + 1],
                                       cx<R>& H, cx<R>& Ht) const {
    put_params<R>(t);
    const cx<R>* V = vptr<R>();
    const int rr = i & (ROWL - 1), part = i / ROWL;  // row, and share of the term slots
    const int ii = rr < N ? rr : 0;
    cx<R>* A = reinterpret_cast<cx<R>*>(acc) + g.gl;
#pragma unroll
    for (int e = 0; e <= N; ++e) A[e * L] = czero<R>();
    cx<R> h = czero<R>();
#pragma unroll 1
    for (int k = part; k < a->TT; k += PARTS) {
      const int64_t r = (int64_t)k * a->ls + ii;
      const TermRec rc = a->rec[r];
      cx<R> s, dcr = czero<R>();
      if (a->coef_mode)
        coef_at<R>(r, t, s, dcr);
      else if constexpr (std::is_same<R, float>::value)
        s = mk<float>(rc.s.x, rc.s.y);
      else if constexpr (std::is_same<R, df>::value)
        s = to_cxdf(a->sdf[r]);
      else
        s = mk<double>(a->s64[r].x, a->s64[r].y);
      cx<R> run = czero<R>();
      switch (rc.d) {  // the same at a slot for every row and path: no divergence
        case 1: run = term<1, R>(rc, s, V, A, h); break;
        case 2: run = term<2, R>(rc, s, V, A, h); break;
        case 3: run = term<3, R>(rc, s, V, A, h); break;
        case 4: run = term<4, R>(rc, s, V, A, h); break;
        case 5: run = term<5, R>(rc, s, V, A, h); break;
        case 6: run = term<6, R>(rc, s, V, A, h); break;
        case 7: run = term<7, R>(rc, s, V, A, h); break;
        case 8: run = term<8, R>(rc, s, V, A, h); break;
        default: break;
      }
      // coefficient interpolation: d/dt of (c0 + t dc) x^a is dc x^a
      if (a->coef_mode) A[N * L] = cfma(dcr, run, A[N * L]);
    }
    if constexpr (PARTS > 1) {  // add the two halves, part 0's first
      __syncwarp(g.mask);
      const cx<R>* A0 = reinterpret_cast<const cx<R>*>(acc) + rr;
#pragma unroll
      for (int j = 0; j < N; ++j) row[j] = A0[j * L] + A0[j * L + ROWL];
      Ht = A0[N * L] + A0[N * L + ROWL];
      H = pair_sum(h, ROWL, part == 1);
    } else {
#pragma unroll
      for (int j = 0; j < N; ++j) row[j] = A[j * L];
      Ht = A[N * L];
      H = h;
    }
  }

  template <bool SCALE, int EP = 1>
  __device__ __forceinline__ void residual64(const cx<double>*, int i, double t, double,
                                             cx<double>& H, double& sc) const {
    put_params<double>(t);
    const int rr = i & (ROWL - 1), part = i / ROWL;
    const int ii = rr < N ? rr : 0;
    cx<double> h = czero<double>();
    float s_abs = 0.f;
#pragma unroll 1
    for (int k = part; k < a->TT; k += PARTS) {
      const int64_t r = (int64_t)k * a->ls + ii;
      const TermRec rc = a->rec[r];
      cx<double> prod = Vd[rc.idx[0]];
#pragma unroll 1
      for (int f = 1; f < rc.d; ++f) prod = prod * Vd[rc.idx[f]];
      cx<double> s, dcr;
      if (a->coef_mode)
        coef_at<double>(r, t, s, dcr);
      else
        s = mk<double>(a->s64[r].x, a->s64[r].y);
      h = cfma(s, prod, h);
      if (SCALE) s_abs += cabs2(cvt<float>(s)) * cabs2(cvt<float>(prod));
    }
    if constexpr (PARTS > 1) {
      h = pair_sum(h, ROWL, part == 1);
      if (SCALE) s_abs = pair_sum(s_abs, ROWL, part == 1);
    }
    H = h;
    sc = SCALE ? (double)s_abs : 0.0;
  }
  // The residual in double-float arithmetic (DF): p(t) = p0 + t dp formed
  // in double-floats from the per-path copies, then every term's product of
  // factors and coefficient (table sdf) as in residual64.  H is returned
  // rounded to FP32 (its error is a small multiple of 2^-48 times the
  // backward-error scale sc).
  template <bool SCALE, int EP = 1>
  __device__ __forceinline__ void residual_df(const cdf*, int i, double t, cx<float>& H,
                                              float& sc) const {
    const int P = a->P, LS = a->ls;
    cdf* V = reinterpret_cast<cdf*>(Vd);
    const df tdf = to_df(t);
    if (g.gl == 0) V[LS] = cdf{1.f, 0.f, 0.f, 0.f};
    for (int l = g.gl; l < P; l += L)
      V[LS + 1 + l] = cdf_add(V[LS + 1 + 2 * P + l], cdf_scale(tdf, V[LS + 1 + P + l]));
    __syncwarp(g.mask);
    const int rr = i & (ROWL - 1), part = i / ROWL;
    const int ii = rr < N ? rr : 0;
    cdf h = cdf_zero();
    float s_abs = 0.f;
#pragma unroll 1
    for (int k = part; k < a->TT; k += PARTS) {
      const int64_t r = (int64_t)k * a->ls + ii;
      const TermRec rc = a->rec[r];
      cdf prod = V[rc.idx[0]];
#pragma unroll 1
      for (int f = 1; f < rc.d; ++f) prod = cdf_mul(prod, V[rc.idx[f]]);
      const cdf s = a->coef_mode
                        ? cdf_add(a->c0df[r],
                                  cdf_scale(tdf, a->dcdf[inst * (int64_t)a->TT * a->ls + r]))
                        : a->sdf[r];
      h = cdf_fma(s, prod, h);
      if (SCALE) s_abs += cdf_abs_hi(s) * cdf_abs_hi(prod);
    }
    if constexpr (PARTS > 1) {
      h = pair_sum(h, ROWL, part == 1);
      if (SCALE) s_abs = pair_sum(s_abs, ROWL, part == 1);
    }
    H = cdf_to_cf(h);
    sc = SCALE ? s_abs : 0.f;
  }
};

template <int N, int L, bool DF>
struct TermProblem {
  const TermArgs* a;
  Group g;
  GroupMem sm;
  __device__ __forceinline__ TermEval<N, L, DF> hom(int64_t inst) const {
    return TermEval<N, L, DF>{a, inst, g, sm.vf, sm.vd, sm.acc, sm.vx};
  }
};

// accumulator bytes of a group: N + 1 entries (row and dH/dt) of L lanes
template <int N, bool MIXED, int L>
__host__ __device__ constexpr int term_acc_bytes() {
  return (N + 1) * L * (MIXED ? 8 : 16);
}

// PREC: HC_PREC_MIXED, HC_PREC_FP64 or HC_PREC_DF (as the dense kernels)
template <int N, int PREC, int L, bool RING = false>
__global__ void __launch_bounds__(kBlock) term_param_kernel(const __grid_constant__ TermArgs a) {
  constexpr bool MIXED = PREC == HC_PREC_MIXED;
  constexpr bool XDF = PREC == HC_PREC_DF;
  using RE = typename std::conditional<XDF, df, double>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  const Group g = make_group<L>();
  const GroupMem sm = make_group_mem<L>(smem, a.extra, term_acc_bytes<N, MIXED, L>(),
                                        endgame_smem_bytes(L, MIXED), XDF ? 1 : 0);
  TermProblem<N, L, MIXED> prob{&a, g, sm};
  run_tracker<N, L, MIXED, TermProblem<N, L, MIXED>, RE, RING>(prob, a.c, g, sm);
}

template <int PREC, int N, int LANES = 0, bool RING = false>
KernelRef term_ref() {
  constexpr bool MIXED = PREC == HC_PREC_MIXED;
  constexpr int L = LANES ? LANES : ((N <= 4) ? 4 : (N <= 8) ? 8 : (N <= 16) ? 16 : 32);
  return KernelRef{reinterpret_cast<const void*>(&term_param_kernel<N, PREC, L, RING>), L, 0,
                   term_acc_bytes<N, MIXED, L>(), endgame_smem_bytes(L, MIXED),
                   PREC == HC_PREC_DF ? 1 : 0};
}

}  // namespace hc
