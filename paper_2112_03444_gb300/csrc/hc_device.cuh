// Device building blocks of the tracker: complex arithmetic, lane-group
// primitives and the register-resident dense solve (Sec. 6 of the paper).
//
// Layout: one path is owned by a group of L lanes of a warp (L = 4, 8, 16 or
// 32); lane i of the group holds row i of the augmented matrix [A | b] in
// registers.  Pivot search is one warp-reduction instruction over the group,
// and the pivot row reaches the other lanes through shuffles.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hc {

// Aligned to its size so that one complex number moves in one 64-bit (FP32)
// or 128-bit (FP64) load or store.
template <class R>
struct __align__(2 * sizeof(R)) cx {
  R re, im;
};

template <class R>
__device__ __forceinline__ cx<R> mk(R re, R im) { return cx<R>{re, im}; }
template <class R>
__device__ __forceinline__ cx<R> czero() { return cx<R>{R(0), R(0)}; }

template <class R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R>
__device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
template <class R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
template <class R>
__device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return {s * a.re, s * a.im}; }

// acc + a*b (four FMAs)
template <class R>
__device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> acc) {
  return {fma(a.re, b.re, fma(-a.im, b.im, acc.re)), fma(a.re, b.im, fma(a.im, b.re, acc.im))};
}
// acc - a*b
template <class R>
__device__ __forceinline__ cx<R> cfms(cx<R> a, cx<R> b, cx<R> acc) {
  return {fma(-a.re, b.re, fma(a.im, b.im, acc.re)), fma(-a.re, b.im, fma(-a.im, b.re, acc.im))};
}

// Reciprocals: FP32 with the hardware approximation (relative error about
// one ulp, ample for the FP32 solve); FP64 correctly rounded.
__device__ __forceinline__ float rcp(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ double rcp(double v) { return __drcp_rn(v); }

// 1/z.  FP64: with scaling by max(|re|, |im|) so that |z|^2 cannot overflow
// for |z| up to the format's range.  FP32: conj(z) / |z|^2 directly -- the
// FP32 tracker's Jacobian entries stay far inside 1e-19 < |z| < 1e19 (a
// pivot outside that range makes the reciprocal non-finite and the step is
// rejected, as for a singular matrix).
template <class R>
__device__ __forceinline__ cx<R> crecip(cx<R> z) {
  if constexpr (sizeof(R) == 4) {
    const R d = rcp(fma(z.re, z.re, z.im * z.im));
    return {z.re * d, -z.im * d};
  } else {
    const R s = fmax(fabs(z.re), fabs(z.im));
    const R inv_s = rcp(s);
    const R zr = z.re * inv_s, zi = z.im * inv_s;
    const R d = rcp(s * fma(zr, zr, zi * zi));
    return {zr * d, -zi * d};
  }
}

template <class R>
__device__ __forceinline__ R cnorm2(cx<R> z) { return fma(z.re, z.re, z.im * z.im); }

// sqrt of a non-negative float for threshold tests (approximate, 0 -> 0)
__device__ __forceinline__ float sqrt_approx(float v) { return v > 0.f ? v * rsqrtf(v) : 0.f; }

template <class R>
__device__ __forceinline__ R cabs1(cx<R> z) { return fabs(z.re) + fabs(z.im); }
template <class R>
__device__ __forceinline__ R cabs2(cx<R> z) { return sqrt(fma(z.re, z.re, z.im * z.im)); }

template <class D, class S>
__device__ __forceinline__ cx<D> cvt(cx<S> z) { return {(D)z.re, (D)z.im}; }

template <class R>
__device__ __forceinline__ bool cfinite(cx<R> z) { return isfinite(z.re) && isfinite(z.im); }

// ---------------------------------------------------------------- lane groups
struct Group {
  int gl;          // lane index inside the group (row index)
  int wl;          // lane index inside the warp
  unsigned mask;   // lanes of this group
};

template <int L>
__device__ __forceinline__ Group make_group() {
  Group g;
  g.wl = threadIdx.x & 31;
  g.gl = g.wl & (L - 1);
  g.mask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g.wl & ~(L - 1)));
  return g;
}

template <class R>
__device__ __forceinline__ cx<R> shfl(unsigned mask, cx<R> v, int src) {
  return {__shfl_sync(mask, v.re, src), __shfl_sync(mask, v.im, src)};
}

// max over the group of a non-negative float (NaN compares above everything)
__device__ __forceinline__ float gmaxf(const Group& g, float v) {
  unsigned b = __reduce_max_sync(g.mask, __float_as_uint(fmaxf(v, 0.0f)) | (isnan(v) ? 0x7fc00000u : 0u));
  return __uint_as_float(b);
}
__device__ __forceinline__ bool gany(const Group& g, bool v) {
  return __reduce_or_sync(g.mask, v ? 1u : 0u) != 0u;
}
// sum over the group (butterfly)
template <int L, class R>
__device__ __forceinline__ R gsum(const Group& g, R v) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(g.mask, v, o);
  return v;
}

// ---------------------------------------------------------------- dense solve
//
// Gauss-Jordan elimination with partial pivoting on the augmented matrix
// [A | B] (N rows, N + NR columns), row i in lane i.  The paper (Sec. 6)
// factors [A b] by LU, which carries the L-solve inside the factorisation,
// and finishes with a back substitution on the cached U.  With one row per
// lane the back substitution would be N serial broadcast steps; eliminating
// above the pivot as well (Gauss-Jordan) costs no extra latency because those
// rows sit in otherwise idle lanes, and it removes the back substitution.
//
// Pivot: the largest |Re| + |Im| among rows not yet used, lowest lane on
// ties, found with one __reduce_max_sync on a key whose high bits are the
// magnitude's float bits and whose low 5 bits encode the lane.
//
// The pivot row reaches the other lanes through shared memory: the pivot
// lane stores its remaining columns (FP32: two complex numbers per 16-byte
// store; the pivot column's slot carries 1/pivot), the group synchronises,
// and every lane reads them back with 16-byte broadcast loads (FP64 and
// double-float: one complex entry per 16-byte word).  Two buffers
// alternate, so one __syncwarp per pivot step orders writes after the
// previous step's reads.  pv: 2 * ((N + NR + 1) & ~1) entries, 16-byte
// aligned, private to the group.
//
// On return lane i with i < N holds in col the column it pivoted on and in
// sol[r] the solution component x[col] of right-hand side r.  Returns false
// if a pivot was zero or non-finite (the caller rejects the step).
template <int N, int NR, class R>
__device__ __forceinline__ bool gj_solve(const Group& g, cx<R> (&a)[N + NR], cx<R> (&sol)[NR],
                                         int& col, cx<R>* pv) {
  constexpr int W = N + NR;
  constexpr int S = (W + 1) & ~1;  // entries per buffer (even: FP32 pairs stay 16-byte aligned)
  bool used = g.gl >= N;
  cx<R> dinv = mk<R>(R(1), R(0));  // 1 / pivot of this lane's row
  col = -1;
  // smallest and largest pivot magnitude (float bits, lane bits cleared):
  // every pivot was nonzero and finite iff lo != 0 and hi < +inf
  unsigned lo = 0xffffffffu, hi = 0u;
  // Pivot search of column k: every lane forms 1 / a[k] of its own row while
  // the reduction picks the pivot (the reciprocal stays off the critical
  // path).  The search of column k + 1 starts as soon as column k + 1 is
  // updated, so that its reduction overlaps the rest of step k's update.
  auto search = [&](int k, cx<R>& inv, unsigned& kmax) {
    inv = crecip(a[k]);
    const float m = (float)cabs1(a[k]);
    const unsigned key = used ? 0u : ((__float_as_uint(m) & ~31u) | (unsigned)(31 - g.wl));
    kmax = __reduce_max_sync(g.mask, key);
  };
  cx<R> inv;
  unsigned kmax;
  search(0, inv, kmax);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    lo = min(lo, kmax);
    hi = max(hi, kmax);
    const int p = 31 - (int)(kmax & 31u);
    const bool me = (g.wl == p);
    cx<R>* buf = pv + (k & 1) * S;
    const int j0 = k & ~1;  // first stored column (k, or k - 1 whose slot is ignored)
    if (me) {
      if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int j = j0; j < W; j += 2) {
          const cx<R> v0 = (j == k) ? inv : a[j];
          const cx<R> v1 = (j + 1 == k) ? inv : (j + 1 < W ? a[j + 1 < W ? j + 1 : 0] : czero<R>());
          reinterpret_cast<float4*>(buf)[j >> 1] = make_float4(v0.re, v0.im, v1.re, v1.im);
        }
      } else {  // FP64 or double-float: one 16-byte store per entry
#pragma unroll
        for (int j = k; j < W; ++j) buf[j] = (j == k) ? inv : a[j];
      }
      used = true;
      dinv = inv;
      col = k;
    }
    __syncwarp(g.mask);
    cx<R> row_p[W];  // the pivot row, columns k .. W-1 (slot k: 1/pivot)
    if constexpr (sizeof(R) == 4) {
#pragma unroll
      for (int j = j0; j < W; j += 2) {
        const float4 q = reinterpret_cast<const float4*>(buf)[j >> 1];
        row_p[j] = mk<R>(q.x, q.y);
        if (j + 1 < W) row_p[j + 1 < W ? j + 1 : 0] = mk<R>(q.z, q.w);
      }
    } else {
#pragma unroll
      for (int j = k; j < W; ++j) row_p[j] = buf[j];
    }
    const cx<R> l = me ? czero<R>() : a[k] * row_p[k];
    a[k + 1] = cfms(l, row_p[k + 1], a[k + 1]);
    if (k + 1 < N) search(k + 1 < N ? k + 1 : 0, inv, kmax);
#pragma unroll
    for (int j = k + 2; j < W; ++j) a[j] = cfms(l, row_p[j], a[j]);
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) sol[r] = a[N + r] * dinv;
  return (lo & ~31u) != 0u && (hi & ~31u) < 0x7f800000u;
}

// The same elimination for groups whose rows are replicated over PARTS
// lanes (one path per warp with the evaluation split over the warp, L0 =
// lanes per replica): lane gl holds row r = gl mod L0 and owns the columns j
// with j mod PARTS = gl / L0, the only ones it updates.  At step k the owners
// of column k search the pivot; every owner publishes its row's entry of
// column k (the multiplier's numerator) and the pivot row's lanes publish
// their columns, all through shared memory; then each lane updates its own
// columns.  The FP64 re-tracking tiers run this form: their cost is the
// FP64 instructions per lane.  pv: 2 * ((N + 2) & ~1) entries, then L0
// reciprocals and L0 ints; mkbuf: 2 * L0 entries.  NR = 1.  On return the
// owner of column N in each pivoted row holds col and sol; col = -1 elsewhere.
template <int N, class R, int L0, int PARTS>
__device__ __forceinline__ bool gj_solve_parts(const Group& g, cx<R> (&a)[N + 1], cx<R> (&sol)[1],
                                               int& col, cx<R>* pv, cx<R>* mkbuf) {
  constexpr int W = N + 1;
  constexpr int S = (W + 1) & ~1;
  const int r = g.gl & (L0 - 1);
  const int part = g.gl / L0;
  cx<R>* dv = pv + 2 * S;                     // 1 / pivot of each row
  int* pc = reinterpret_cast<int*>(dv + L0);  // pivot column of each row
  bool used = r >= N;
  unsigned lo = 0xffffffffu, hi = 0u;
  col = -1;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const bool own = (part == k % PARTS);
    const cx<R> inv = crecip(a[k]);
    const float m = (float)cabs1(a[k]);
    const unsigned key =
        (used || !own) ? 0u : ((__float_as_uint(m) & ~31u) | (unsigned)(31 - g.wl));
    const unsigned kmax = __reduce_max_sync(g.mask, key);
    lo = min(lo, kmax);
    hi = max(hi, kmax);
    const int p = 31 - (int)(kmax & 31u);
    const int rp = p & (L0 - 1);
    cx<R>* buf = pv + (k & 1) * S;
    cx<R>* mk = mkbuf + (k & 1) * L0;
    if (own) mk[r] = a[k];
    if (r == rp) {
#pragma unroll
      for (int j = k; j < W; ++j)
        if (j % PARTS == part) buf[j] = (j == k) ? inv : a[j];
      used = true;
    }
    if (g.wl == p) {
      dv[r] = inv;
      pc[r] = k;
    }
    __syncwarp(g.mask);
    const cx<R> l = (r == rp) ? czero<R>() : mk[r] * buf[k];
#pragma unroll
    for (int j = k + 1; j < W; ++j)
      if (j % PARTS == part) a[j] = cfms(l, buf[j], a[j]);
  }
  __syncwarp(g.mask);
  if (part == N % PARTS && r < N) {
    col = pc[r];
    sol[0] = a[N] * dv[r];
  }
  return (lo & ~31u) != 0u && (hi & ~31u) < 0x7f800000u;
}

// ---------------------------------------------------------------- settings
struct DevSettings {
  double dt_min, dt_max, dt_init, newton_tol, newton_tol_fp32, max_first_corr;
  double refine_tol, r_inf, finite_tol, real_tol, singular_cond, t_endgame;
  double dt_min_fp32, max_first_corr_fp32;
  double eg_s0, eg_ratio, eg_tol;
  int max_newton, max_steps, grow_after, refine_iters, max_steps_fp32, max_newton_ir;
  int endgame, eg_cmax, eg_samples;
};

enum : int {
  ST_FINITE = 1, ST_DIVERGED = 2, ST_FAIL_STEP = 3, ST_FAIL_MAXSTEPS = 4,
  ST_FAIL_NAN = 5, ST_SINGULAR = 6, ST_FAIL_REFINE = 7, ST_REAL = 0x80
};

// Largest FP32 condition estimate that still certifies cond_1 < 1e12 with
// room to spare: an FP32 inverse is accurate to about n * cond * 6e-8, so an
// estimate of 2e6 bounds the true value within a small factor, six orders
// below the singular threshold; above it the endpoint is re-checked in FP64.
constexpr double kFp32CondTrust = 2.0e6;

}  // namespace hc
