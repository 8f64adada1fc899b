// Total-degree homotopy for dense systems of degree 2 or 3 (every monomial of
// degree <= d present in every equation):
//   H(x,t) = (1-t) gamma G(x) + t F(x),  G_i = x_i^d - 1        (paper Eq. 1)
// with the random unit gamma.  Start point k: x_i = exp(2 pi i k_i / d),
// k_i the i-th base-d digit of k (variable 1 least significant).
//
// Evaluation (paper Sec. 6: one Jacobian row per lane, coefficients shared
// by the paths of a system).  For a dense system the homogenised term tuples
// of Sec. 6 have a fixed pattern, so they are not stored: row i of dF/dx is
//   dF_i/dx_j = sum_m D[j][m][i] mu_m(x),   mu = monomials of degree <= d-1,
// with D the coefficient of mu_m in dF_i/dx_j (exponent multiplicity folded
// in), and F_i follows from the same partial sums by Euler's identity on each
// homogeneous part:  F_i = c_i0 + sum_j x_j (a0_j + a1_j / 2 + a2_j / 3),
// where a_e is the part of dF_i/dx_j built from degree-e monomials.
//
// High-precision residuals use the monomial coefficients in nested Horner order
//   F_i = c0 + sum_j x_j (b_j + sum_{k<=j} x_k (q_jk + sum_{l<=k} r_jkl x_l)),
// one complex FMA per monomial: in FP64 (all-FP64 kernels, table E) or in
// double-float arithmetic (mixed-precision kernels, table Edf: the same
// coefficients split into FP32 pairs, see dfloat.cuh).
//
// Data layout (per instance, lane stride L so that the L lanes of a path read
// consecutive addresses):
//   D: [(N+1) slices][MPP/2 monomial pairs][L][2]: lane i reads the two
//      coefficients of a pair with one 16-byte load (FP32); the constant,
//      linear and quadratic monomials each start a new pair (dense_slot in
//      kernels.cuh); slice N pair 0 holds the constant c_i0.
//   E: [M][L] complex double, nested Horner order; Edf the same entries as
//      double-floats (16 bytes each: hi re, hi im, lo re, lo im).
//   Ddf: D as complex double-floats (cx<df>: re hi, re lo, im hi, im lo), the
//      table of the double-float kernels, which evaluate with R = df.
#pragma once

#include <type_traits>

#include "dfloat.cuh"
#include "hc_device.cuh"
#include "kernels.cuh"

namespace hc {

template <int N, int DEG>
struct DenseShape {
  static_assert(DEG == 2 || DEG == 3, "dense evaluator: degree 2 or 3");
  static constexpr int MP = (DEG == 2) ? (N + 1) : (1 + N + N * (N + 1) / 2);
  static constexpr int M = (DEG == 2) ? ((N + 1) * (N + 2) / 2) : ((N + 1) * (N + 2) * (N + 3) / 6);
  // graded-lex index of x_k x_l (k <= l) among the monomials of degree <= 2
  static constexpr __host__ __device__ int idx2(int k, int l) {
    return 1 + N + k * N - k * (k - 1) / 2 + (l - k);
  }
  // quadratic monomials x_k x_l (k <= l), formed per evaluation in the
  // group's shared memory behind the lane slots of the point (cubic systems
  // only; padded to an even count like the table)
  static constexpr int NQ = N * (N + 1) / 2;
  static constexpr int N2 = N + (N & 1);                    // linear monomials, padded
  static constexpr int NQ2 = (DEG == 3) ? NQ + (NQ & 1) : 0;  // quadratic ones, padded
  static constexpr int MPP = dense_mpp(N, DEG);             // padded monomials per slice
  static constexpr int EXTRA = NQ2;
};

template <int N, int DEG, int L_GROUP>
struct DenseTD {
  using S = DenseShape<N, DEG>;
  // Lane stride of the encoded coefficients: fixed by the encoding (the
  // default group width for N), independent of the kernel's group width.
  static constexpr int L = (N <= 4) ? 4 : (N <= 8) ? 8 : (N <= 16) ? 16 : 32;
  const cx<float>* D32;
  const cx<double>* D64;
  const cx<df>* Ddf;
  const cx<double>* E;
  const cdf* Edf;
  cx<double> gamma;
  cx<float> gamma32;
  cdf gammadf;
  cx<float>* Vf;   // the group's shared copies of the evaluation point (+ monomials)
  cx<double>* Vd;
  cx<df>* Vx;      // double-float kernels: the point as double-floats (+ monomials)
  unsigned gmask;  // lanes of the group

  template <class R>
  __device__ __forceinline__ const cx<R>* dptr() const;
  template <class R>
  __device__ __forceinline__ cx<R>* vptr() const {
    if constexpr (std::is_same<R, float>::value)
      return Vf;
    else if constexpr (std::is_same<R, df>::value)
      return Vx;
    else
      return Vd;
  }

  // Groups wider than the encoding stride (one path per warp) split every
  // row's contraction over PARTS lanes -- lane i works on row i mod L, part
  // i / L -- and add the partial sums with shuffles: a path then keeps the
  // whole warp busy, which is what bounds the FP64 re-tracking of a handful
  // of hard paths (an FP64 warp instruction costs the same pipe time with 8
  // or 32 active lanes).
  static constexpr int PARTS = (L_GROUP > L) ? L_GROUP / L : 1;
  static constexpr int ROWL = (PARTS > 1) ? L : L_GROUP;  // lanes per row replica
  static_assert(PARTS == 1 || L_GROUP == 32, "split rows need the whole warp");

  template <class R>
  __device__ __forceinline__ static cx<R> part_sum(cx<R> v) {
    if constexpr (PARTS > 1) {
#pragma unroll
      for (int o = L; o < L * PARTS; o <<= 1) {
        if constexpr (std::is_same<R, df>::value) {
          v.re = v.re + shfl_xor_df(v.re, o);
          v.im = v.im + shfl_xor_df(v.im, o);
        } else {
          v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
          v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
        }
      }
    }
    return v;
  }
  // m-th outer index of a part: zigzag over blocks of PARTS indices, so that
  // triangular inner loops give every part the same work (identity for
  // PARTS = 1)
  template <int P = PARTS>
  __device__ __forceinline__ static int zigzag(int m, int part) {
    return (m & 1) ? ((m + 1) * P - 1 - part) : (m * P + part);
  }

  // Residuals of the mixed kernels whose groups are narrower than a warp
  // (several paths per warp).  A residual there is needed by one group at a
  // time (its path is in the FP64-state phase or at its endpoint while the
  // other paths of the warp track in FP32), and a group computing it alone
  // keeps the rest of the warp idle for the whole Horner evaluation.  So the
  // tracker has every lane of the warp compute a share of it: the outer
  // index j is split over WP = 32 / L parts (zigzag, as for split rows), the
  // parts are added by a butterfly over the warp, and the group then holds
  // the rows' residuals (the *_coop functions below).  Where a group must
  // compute a residual alone (the resident-launch kernels, whose groups wait
  // for work independently), it forms the same WP partial sums one after the
  // other and adds them in the butterfly's order (the *_seq functions), so
  // that both forms give the same bits.
  static constexpr bool kCoop = (PARTS == 1 && L_GROUP < 32);
  static constexpr int WP = 32 / L;

  // Two consecutive complex numbers (16-byte aligned): one 16-byte load in
  // FP32, two in FP64.
  template <class R>
  __device__ __forceinline__ static void ld2(const cx<R>* p, cx<R>& c0, cx<R>& c1) {
    if constexpr (std::is_same<R, float>::value) {
      const float4 f = *reinterpret_cast<const float4*>(p);
      c0 = mk<float>(f.x, f.y);
      c1 = mk<float>(f.z, f.w);
    } else {
      c0 = p[0];
      c1 = p[1];
    }
  }

  // The contraction indices run in loops that are not unrolled (pairs of
  // point entries and quadratic monomials are read from the group's shared
  // memory); the rows j stay unrolled so that the accumulators live in
  // registers.  The point is read from shared memory too (x is not needed in
  // registers).
  template <class R>
  __device__ __forceinline__ void eval(const cx<R> (&)[N], int i, R t, R omt, cx<R> (&row)[N + 1],
                                       cx<R>& H, cx<R>& Ht) const {
    const int r = i & (L - 1);                   // this lane's row
    const int rr = r < N ? r : 0;
    const int part = (PARTS > 1) ? i / L : 0;    // and its share of the contraction
    const cx<R>* D = dptr<R>();
    // the pair q of slice j, this lane's row
    auto pair = [&](int j, int q) { return D + ((int64_t)(j * (S::MPP / 2) + q) * L + rr) * 2; };
    cx<R>* V = vptr<R>();
    cx<R>* Q = V + L_GROUP;
    if constexpr (std::is_same<R, df>::value) {
      // the tracker keeps the point in FP64 (Vd): split it once per evaluation
      if (i < N) V[i] = to_cxdf(Vd[i]);
      __syncwarp(gmask);
    }
    if constexpr (DEG == 3) {
      // x_k x_l for k <= l in graded order: row k of the triangle, lane i
      // forming x_k x_(k+i) (no index search, no divergence)
#pragma unroll 1
      for (int k = 0; k < N; ++k)
        if (i < N - k) Q[S::idx2(k, k + i) - 1 - N] = V[k] * V[k + i];
      __syncwarp(gmask);
    }
    cx<R> a1[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a1[j] = czero<R>();
#pragma unroll 1
    for (int q = part; q < S::N2 / 2; q += PARTS) {
      cx<R> x0, x1;
      ld2(V + 2 * q, x0, x1);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        cx<R> c0, c1;
        ld2(pair(j, 1 + q), c0, c1);
        a1[j] = cfma(c1, x1, cfma(c0, x0, a1[j]));
      }
    }
    cx<R> F = pair(N, 0)[0];
    if constexpr (DEG == 2) {
      if constexpr (PARTS > 1) {
#pragma unroll
        for (int j = 0; j < N; ++j) a1[j] = part_sum(a1[j]);
      }
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const cx<R> a0 = pair(j, 0)[0];
        row[j] = a0 + a1[j];
        F = cfma(V[j], a0 + R(0.5) * a1[j], F);
      }
    } else {
      cx<R> a2[N];
#pragma unroll
      for (int j = 0; j < N; ++j) a2[j] = czero<R>();
#pragma unroll 1
      for (int q = part; q < S::NQ2 / 2; q += PARTS) {
        cx<R> m0, m1;
        ld2(Q + 2 * q, m0, m1);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          cx<R> c0, c1;
          ld2(pair(j, 1 + S::N2 / 2 + q), c0, c1);
          a2[j] = cfma(c1, m1, cfma(c0, m0, a2[j]));
        }
      }
      if constexpr (PARTS > 1) {
        // partial rows and the partial Euler sum, then one reduction each
        cx<R> fp = czero<R>();
#pragma unroll
        for (int j = 0; j < N; ++j) {
          fp = cfma(V[j], R(0.5) * a1[j] + R(1.0 / 3.0) * a2[j], fp);
          a1[j] = part_sum(a1[j] + a2[j]);
        }
        F = F + part_sum(fp);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const cx<R> a0 = pair(j, 0)[0];
          row[j] = a0 + a1[j];
          F = cfma(V[j], a0, F);
        }
      } else {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const cx<R> a0 = pair(j, 0)[0];
          row[j] = a0 + a1[j] + a2[j];
          F = cfma(V[j], a0 + R(0.5) * a1[j] + R(1.0 / 3.0) * a2[j], F);
        }
      }
    }
    const cx<R> xi = V[rr];
    // G_i = xi^d - 1, dG_i/dx_i = d xi^(d-1)
    const cx<R> xi2 = xi * xi;
    const cx<R> G = (DEG == 2 ? xi2 : xi2 * xi) - mk<R>(R(1), R(0));
    const cx<R> Gd = R(DEG) * (DEG == 2 ? xi : xi2);
    cx<R> gm;
    if constexpr (std::is_same<R, float>::value)
      gm = gamma32;
    else if constexpr (std::is_same<R, df>::value)
      gm = to_cxdf(gammadf);
    else
      gm = gamma;
    const cx<R> gG = gm * G;
    H = t * F + omt * gG;
    Ht = F - gG;
    const cx<R> gd = omt * (gm * Gd);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      row[j] = t * row[j];
      if (j == r) row[j] = row[j] + gd;
    }
  }

  // FP64 residual of row i at (x, t); x is read from the group's shared copy
  // (xs[k], k < N) so that no FP64 vector occupies registers.  With SCALE the
  // backward-error denominator sum |c| |x^a| (FP32 accuracy is enough for a
  // ratio test) is returned in sc.  Runtime loops: this code runs a few
  // times per path and must not crowd the tracking loop out of the
  // instruction cache.  Split over PARTS lanes like eval (outer index j).
  // EP > 1 (groups narrower than a warp): the WP-part order of the
  // cooperative form, computed by the group alone.
  template <bool SCALE_T, int EP = 1>
  __device__ __forceinline__ void residual64(const cx<double>* xs, int i, double t, double omt,
                                             cx<double>& H, double& sc) const {
    if constexpr (EP > 1) {
      static_assert(EP == WP && kCoop, "sequential parts: groups narrower than a warp");
      residual64_seq(xs, i, t, omt, SCALE_T, H, sc);
    } else {
      residual64_impl(xs, i, t, omt, SCALE_T, H, sc);
    }
  }

  // partial sums of row r over the outer indices j of part `part` of a
  // P-way split: F (the constant term in part 0) and the scale's share S
  template <int P>
  __device__ __noinline__ void residual64_part(const cx<double>* xs, int r, int part, bool scale,
                                               cx<double>& Fo, float& So) const {
    const cx<double>* e = E + (r < N ? r : 0);
    cx<double> F = part == 0 ? e[0] : czero<double>();
    float Ssum = (scale && part == 0) ? cabs2(cvt<float>(e[0])) : 0.f;
#pragma unroll 1
    for (int mm = 0;; ++mm) {
      const int j = zigzag<P>(mm, part);
      if (j >= N) break;
      // first Horner coefficient of block j: 1 + sum over earlier blocks
      // (block j' holds 1 + sum_{k <= j'} (DEG == 2 ? 1 : k + 2) entries)
      int m = 1;
#pragma unroll 1
      for (int jj = 0; jj < j; ++jj)
        m += 1 + (DEG == 2 ? jj + 1 : (jj + 1) * jj / 2 + 2 * (jj + 1));
      cx<double> in = e[m * L];
      float ins = scale ? cabs2(cvt<float>(e[m * L])) : 0.f;
      ++m;
#pragma unroll 1
      for (int k = 0; k <= j; ++k) {
        const cx<double> xk = xs[k];
        if constexpr (DEG == 2) {
          in = cfma(e[m * L], xk, in);
          if (scale) ins += cabs2(cvt<float>(e[m * L])) * cabs2(cvt<float>(xk));
          ++m;
        } else {
          cx<double> in2 = e[m * L];
          float in2s = scale ? cabs2(cvt<float>(e[m * L])) : 0.f;
          ++m;
#pragma unroll 1
          for (int l = 0; l <= k; ++l) {
            const cx<double> xl = xs[l];
            in2 = cfma(e[m * L], xl, in2);
            if (scale) in2s += cabs2(cvt<float>(e[m * L])) * cabs2(cvt<float>(xl));
            ++m;
          }
          in = cfma(xk, in2, in);
          if (scale) ins += cabs2(cvt<float>(xk)) * in2s;
        }
      }
      const cx<double> xj = xs[j];
      F = cfma(xj, in, F);
      if (scale) Ssum += cabs2(cvt<float>(xj)) * ins;
    }
    Fo = F;
    So = Ssum;
  }

  // H = t F + (1 - t) gamma G_r and the scale, from the summed parts
  __device__ __noinline__ void residual64_finish(const cx<double>* xs, int r, double t, double omt,
                                                 bool scale, cx<double> F, float Ssum,
                                                 cx<double>& H, double& sc) const {
    const cx<double> xi = xs[r < N ? r : 0];
    const cx<double> xi2 = xi * xi;
    const cx<double> G = (DEG == 2 ? xi2 : xi2 * xi) - mk<double>(1.0, 0.0);
    H = t * F + omt * (gamma * G);
    if (scale) {
      const float axi = cabs2(cvt<float>(xi));
      sc = t * (double)Ssum + omt * (double)(1.0f + (DEG == 2 ? axi * axi : axi * axi * axi));
    } else {
      sc = 0.0;
    }
  }

  __device__ __forceinline__ void residual64_impl(const cx<double>* xs, int i, double t, double omt,
                                                  bool scale, cx<double>& H, double& sc) const {
    const int r = i & (L - 1);
    const int part = (PARTS > 1) ? i / L : 0;
    cx<double> F;
    float Ssum;
    residual64_part<PARTS>(xs, r, part, scale, F, Ssum);
    if constexpr (PARTS > 1) {
      F = part_sum(F);
      if (scale) {
#pragma unroll
        for (int o = L; o < L * PARTS; o <<= 1) Ssum += __shfl_xor_sync(0xffffffffu, Ssum, o);
      }
    }
    residual64_finish(xs, r, t, omt, scale, F, Ssum, H, sc);
  }

  // the WP parts one after the other, added in the butterfly's order
  __device__ __forceinline__ void residual64_seq(const cx<double>* xs, int i, double t, double omt,
                                                 bool scale, cx<double>& H, double& sc) const {
    const int r = i & (L - 1);
    cx<double> F[WP];
    float S[WP];
#pragma unroll
    for (int p = 0; p < WP; ++p) residual64_part<WP>(xs, r, p, scale, F[p], S[p]);
#pragma unroll
    for (int w = 1; w < WP; w <<= 1) {
#pragma unroll
      for (int p = 0; p < WP; p += 2 * w) {
        F[p] = F[p] + F[p + w];
        S[p] = S[p] + S[p + w];
      }
    }
    residual64_finish(xs, r, t, omt, scale, F[0], S[0], H, sc);
  }

  // Cooperative form: called by every lane of the warp (wl = lane index)
  // for the group whose point xs is; lane wl computes part wl / L of row
  // wl mod L, and after the butterfly every lane holds its row's residual.
  __device__ __forceinline__ void residual64_coop(const cx<double>* xs, int wl, double t,
                                                  bool scale, cx<double>& H, double& sc) const {
    static_assert(kCoop, "cooperative residuals: groups narrower than a warp");
    const int r = wl & (L - 1);
    cx<double> F;
    float S;
    residual64_part<WP>(xs, r, wl / L, scale, F, S);
#pragma unroll
    for (int o = L; o < 32; o <<= 1) {
      cx<double> w;
      w.re = __shfl_xor_sync(0xffffffffu, F.re, o);
      w.im = __shfl_xor_sync(0xffffffffu, F.im, o);
      F = F + w;
      S = S + __shfl_xor_sync(0xffffffffu, S, o);
    }
    residual64_finish(xs, r, t, 1.0 - t, scale, F, S, H, sc);
  }

  // The residual of row i in double-float arithmetic (mixed-precision
  // kernels): the nested Horner order of residual64 over Edf, the point read
  // as double-floats from the group's shared copy.  H is returned rounded to
  // FP32: its error is a small multiple of 2^-48 times the size of the terms
  // (the backward-error scale sc, formed as in residual64), far below the
  // tolerances the FP64 residual serves, and only the FP32 solve consumes it.
  template <bool SCALE_T, int EP = 1>
  __device__ __forceinline__ void residual_df(const cdf* xs, int i, double t, cx<float>& H,
                                              float& sc) const {
    if constexpr (EP > 1) {
      static_assert(EP == WP && kCoop, "sequential parts: groups narrower than a warp");
      residual_df_seq(xs, i, t, SCALE_T, H, sc);
    } else {
      residual_df_impl(xs, i, t, SCALE_T, H, sc);
    }
  }

  __device__ static cdf part_sum_cdf(cdf v) {
    if constexpr (PARTS > 1) {
#pragma unroll
      for (int o = L; o < L * PARTS; o <<= 1) v = cdf_add(v, shfl_xor_cdf(v, o));
    }
    return v;
  }
  __device__ __forceinline__ static cdf shfl_xor_cdf(cdf v, int o) {
    cdf w;
    w.hr = __shfl_xor_sync(0xffffffffu, v.hr, o);
    w.hi_ = __shfl_xor_sync(0xffffffffu, v.hi_, o);
    w.lr = __shfl_xor_sync(0xffffffffu, v.lr, o);
    w.li = __shfl_xor_sync(0xffffffffu, v.li, o);
    return w;
  }

  // partial sums of row r over part `part` of a P-way split (as residual64_part)
  template <int P>
  __device__ __noinline__ void residual_df_part(const cdf* xs, int r, int part, bool scale,
                                                cdf& Fo, float& So) const {
    const cdf* e = Edf + (r < N ? r : 0);
    cdf F = part == 0 ? e[0] : cdf_zero();
    float Ssum = (scale && part == 0) ? cdf_abs_hi(e[0]) : 0.f;
#pragma unroll 1
    for (int mm = 0;; ++mm) {
      const int j = zigzag<P>(mm, part);
      if (j >= N) break;
      int m = 1;
#pragma unroll 1
      for (int jj = 0; jj < j; ++jj)
        m += 1 + (DEG == 2 ? jj + 1 : (jj + 1) * jj / 2 + 2 * (jj + 1));
      cdf in = e[m * L];
      float ins = scale ? cdf_abs_hi(e[m * L]) : 0.f;
      ++m;
#pragma unroll 1
      for (int k = 0; k <= j; ++k) {
        const cdf xk = xs[k];
        if constexpr (DEG == 2) {
          in = cdf_fma(e[m * L], xk, in);
          if (scale) ins += cdf_abs_hi(e[m * L]) * cdf_abs_hi(xk);
          ++m;
        } else {
          cdf in2 = e[m * L];
          float in2s = scale ? cdf_abs_hi(e[m * L]) : 0.f;
          ++m;
#pragma unroll 1
          for (int l = 0; l <= k; ++l) {
            const cdf xl = xs[l];
            in2 = cdf_fma(e[m * L], xl, in2);
            if (scale) in2s += cdf_abs_hi(e[m * L]) * cdf_abs_hi(xl);
            ++m;
          }
          in = cdf_fma(xk, in2, in);
          if (scale) ins += cdf_abs_hi(xk) * in2s;
        }
      }
      const cdf xj = xs[j];
      F = cdf_fma(xj, in, F);
      if (scale) Ssum += cdf_abs_hi(xj) * ins;
    }
    Fo = F;
    So = Ssum;
  }

  // H = t F + (1 - t) gamma G_r rounded to FP32, and the scale
  __device__ __noinline__ void residual_df_finish(const cdf* xs, int r, double t, bool scale,
                                                  cdf F, float Ssum, cx<float>& H,
                                                  float& sc) const {
    const cdf xi = xs[r < N ? r : 0];
    const cdf xi2 = cdf_mul(xi, xi);
    const cdf one{1.f, 0.f, 0.f, 0.f};
    const cdf G = cdf_sub(DEG == 2 ? xi2 : cdf_mul(xi2, xi), one);
    const cdf Hd = cdf_add(cdf_scale(to_df(t), F), cdf_scale(to_df(1.0 - t), cdf_mul(gammadf, G)));
    H = cdf_to_cf(Hd);
    if (scale) {
      const float axi = cdf_abs_hi(xi);
      sc = (float)t * Ssum + (float)(1.0 - t) * (1.0f + (DEG == 2 ? axi * axi : axi * axi * axi));
    } else {
      sc = 0.f;
    }
  }

  __device__ __forceinline__ void residual_df_impl(const cdf* xs, int i, double t, bool scale,
                                                   cx<float>& H, float& sc) const {
    const int r = i & (L - 1);
    const int part = (PARTS > 1) ? i / L : 0;
    cdf F;
    float Ssum;
    residual_df_part<PARTS>(xs, r, part, scale, F, Ssum);
    if constexpr (PARTS > 1) {
      F = part_sum_cdf(F);
      if (scale) {
#pragma unroll
        for (int o = L; o < L * PARTS; o <<= 1) Ssum += __shfl_xor_sync(0xffffffffu, Ssum, o);
      }
    }
    residual_df_finish(xs, r, t, scale, F, Ssum, H, sc);
  }

  // the WP parts one after the other, added in the butterfly's order
  __device__ __forceinline__ void residual_df_seq(const cdf* xs, int i, double t, bool scale,
                                                  cx<float>& H, float& sc) const {
    const int r = i & (L - 1);
    cdf F[WP];
    float S[WP];
#pragma unroll
    for (int p = 0; p < WP; ++p) residual_df_part<WP>(xs, r, p, scale, F[p], S[p]);
#pragma unroll
    for (int w = 1; w < WP; w <<= 1) {
#pragma unroll
      for (int p = 0; p < WP; p += 2 * w) {
        F[p] = cdf_add(F[p], F[p + w]);
        S[p] = S[p] + S[p + w];
      }
    }
    residual_df_finish(xs, r, t, scale, F[0], S[0], H, sc);
  }

  // Cooperative form (as residual64_coop)
  __device__ __forceinline__ void residual_df_coop(const cdf* xs, int wl, double t, bool scale,
                                                   cx<float>& H, float& sc) const {
    static_assert(kCoop, "cooperative residuals: groups narrower than a warp");
    const int r = wl & (L - 1);
    cdf F;
    float S;
    residual_df_part<WP>(xs, r, wl / L, scale, F, S);
#pragma unroll
    for (int o = L; o < 32; o <<= 1) {
      F = cdf_add(F, shfl_xor_cdf(F, o));
      S = S + __shfl_xor_sync(0xffffffffu, S, o);
    }
    residual_df_finish(xs, r, t, scale, F, S, H, sc);
  }

  // per path: the pad entries behind the point (odd N) and behind the
  // quadratic monomials (odd count) are read by the pair loads as zeros
  __device__ __forceinline__ void init(const Group& g) const {
    if (g.gl == 0) {
      if constexpr (N & 1) {
        Vf[N] = czero<float>();
        Vd[N] = czero<double>();
        if (Vx) Vx[N] = czero<df>();
      }
      if constexpr (DEG == 3 && (S::NQ & 1)) {
        Vf[L_GROUP + S::NQ] = czero<float>();
        Vd[L_GROUP + S::NQ] = czero<double>();
        if (Vx) Vx[L_GROUP + S::NQ] = czero<df>();
      }
    }
  }

  __device__ __forceinline__ cx<double> start(int64_t path, int i) const {
    int64_t k = path;
#pragma unroll 1
    for (int v = 0; v < i; ++v) k /= DEG;
    const int ki = (int)(k % DEG);
    double s, c;
    sincospi(2.0 * (double)ki / (double)DEG, &s, &c);
    return mk<double>(c, s);
  }
};

template <int N, int DEG, int LG>
template <class R>
__device__ __forceinline__ const cx<R>* DenseTD<N, DEG, LG>::dptr() const {
  if constexpr (std::is_same<R, float>::value)
    return D32;
  else if constexpr (std::is_same<R, df>::value)
    return Ddf;
  else
    return D64;
}

}  // namespace hc
