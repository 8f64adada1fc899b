// Double-float arithmetic for the high-precision residuals of the mixed
// precision tracker.
//
// A double-float is the unevaluated sum hi + lo of two FP32 numbers
// (|lo| <= ulp(hi) / 2 after normalisation): about 48 significant bits with
// FP32's exponent range.  Its sums and products are built from error-free
// transformations:
//   TwoSum      (Knuth, TAOCP vol. 2, Sec. 4.2.2): s + e = a + b exactly,
//   TwoProd     with a fused multiply-add:          p + e = a * b exactly,
// in the arrangement of the double-word algorithms analysed by Joldes,
// Muller and Popescu, "Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic" (ACM TOMS 44(2), 2017).  Everything runs
// on the FP32 pipe: GB300 issues FP64 FMAs at about 1/74 of its FP32 rate,
// so a double-float complex multiply-add (about 60 FP32 instructions) costs a
// fifth of the pipe time of the 4 native FP64 FMAs it replaces.
//
// What the tracker needs from it is a residual H(x, t) whose error is small
// against the size of the terms it sums (the backward-error scale): the
// accumulations below bound the absolute error of c + a b by a small
// multiple of u^2 (|c| + |a| |b|), u = 2^-24, which is what a cancelling sum
// needs; the relative error of a result that cancels is not bounded, and is
// not needed.
//
// The intrinsics __fadd_rn, __fsub_rn, __fmul_rn and __fmaf_rn are never
// contracted or reassociated by the compiler, which the transformations rely on.
#pragma once

#include "hc_device.cuh"

namespace hc {

// Besides the explicit functions below, df is an arithmetic type (the
// operators and overloads at the end of this file), so that the evaluators
// and the dense solve -- templates on their real type R -- run in
// double-floats with R = df: the kernels of the double-float precision
// (HC_PREC_DF) and of the last re-tracking tier of the mixed pipeline.
struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit df(int v) : hi((float)v), lo(0.f) {}
  // nearest double-float to v (hi carries the leading 24 bits)
  __host__ __device__ explicit df(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator float() const { return hi + lo; }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (six operations, no precondition)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// p + e = a * b exactly (barring underflow)
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// nearest double-float to a double (hi carries the leading 24 bits)
__device__ __forceinline__ df to_df(double v) {
  const float h = __double2float_rn(v);
  return df{h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ float df_to_float(df a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

// c + x1 y1 + x2 y2.  The two leading products are exact (TwoProd); their
// errors and the cross terms hi * lo go into the low part (the dropped
// lo * lo terms are below u^2 |x y|); the high parts are added by TwoSum and
// the result renormalised by a final TwoSum.
__device__ __forceinline__ df df_dot2(df c, df x1, df y1, df x2, df y2) {
  float p1, e1, p2, e2;
  two_prod(x1.hi, y1.hi, p1, e1);
  two_prod(x2.hi, y2.hi, p2, e2);
  float l = __fmaf_rn(x1.hi, y1.lo, __fmaf_rn(x1.lo, y1.hi, e1));
  l = __fadd_rn(l, __fmaf_rn(x2.hi, y2.lo, __fmaf_rn(x2.lo, y2.hi, e2)));
  float s, es, s2, es2;
  two_sum(c.hi, p1, s, es);
  two_sum(s, p2, s2, es2);
  const float lo = __fadd_rn(__fadd_rn(c.lo, l), __fadd_rn(es, es2));
  df r;
  two_sum(s2, lo, r.hi, r.lo);
  return r;
}

// a + b
__device__ __forceinline__ df df_add(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  const float lo = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  df r;
  two_sum(s, lo, r.hi, r.lo);
  return r;
}

// Complex double-float: one 16-byte word (hi.re, hi.im, lo.re, lo.im) in
// shared or global memory.
struct __align__(16) cdf {
  float hr, hi_, lr, li;  // hi part (re, im), lo part (re, im)
  __device__ __forceinline__ df re() const { return df{hr, lr}; }
  __device__ __forceinline__ df im() const { return df{hi_, li}; }
};

__device__ __forceinline__ cdf mk_cdf(df re, df im) { return cdf{re.hi, im.hi, re.lo, im.lo}; }
__device__ __forceinline__ cdf to_cdf(cx<double> z) { return mk_cdf(to_df(z.re), to_df(z.im)); }
__device__ __forceinline__ cdf cdf_zero() { return cdf{0.f, 0.f, 0.f, 0.f}; }
__device__ __forceinline__ cx<float> cdf_to_cf(cdf z) {
  return cx<float>{df_to_float(z.re()), df_to_float(z.im())};
}
__device__ __forceinline__ cx<double> cdf_to_cd(cdf z) {
  return cx<double>{df_to_double(z.re()), df_to_double(z.im())};
}

// acc + a b
__device__ __forceinline__ cdf cdf_fma(cdf a, cdf b, cdf acc) {
  return mk_cdf(df_dot2(acc.re(), a.re(), b.re(), df_neg(a.im()), b.im()),
                df_dot2(acc.im(), a.re(), b.im(), a.im(), b.re()));
}
// a b
__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) { return cdf_fma(a, b, cdf_zero()); }
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) {
  return mk_cdf(df_add(a.re(), b.re()), df_add(a.im(), b.im()));
}
__device__ __forceinline__ cdf cdf_sub(cdf a, cdf b) {
  return mk_cdf(df_add(a.re(), df_neg(b.re())), df_add(a.im(), df_neg(b.im())));
}
// a real double-float times a complex one
__device__ __forceinline__ cdf cdf_scale(df s, cdf a) {
  const df z{0.f, 0.f};
  return mk_cdf(df_dot2(z, s, a.re(), z, z), df_dot2(z, s, a.im(), z, z));
}

// host-side split of a complex double (tables and launch arguments)
inline cdf split_cdf_host(double re, double im) {
  const float hr = (float)re, hi = (float)im;
  return cdf{hr, hi, (float)(re - (double)hr), (float)(im - (double)hi)};
}

// |z| from the high parts (scales and tests need FP32 accuracy only)
__device__ __forceinline__ float cdf_abs_hi(cdf z) { return sqrtf(fmaf(z.hr, z.hr, z.hi_ * z.hi_)); }

// ---------------------------------------------------------------- df as R
// Real operations.  Sums: df_add (TwoSum of the high parts, the low parts
// added, renormalised).  Products: x y with the exact TwoProd of the high
// parts plus the cross terms.  Both are accurate to a small multiple of
// u^2 = 2^-48 relative to the operands' magnitudes.
__device__ __forceinline__ df operator+(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ df operator-(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df operator-(df a, df b) { return df_add(a, df{-b.hi, -b.lo}); }
__device__ __forceinline__ df operator*(df a, df b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  df r;
  two_sum(p, e, r.hi, r.lo);
  return r;
}

// x1 y1 + x2 y2 (df_dot2 without the addend)
__device__ __forceinline__ df df_sdot2(df x1, df y1, df x2, df y2) {
  float p1, e1, p2, e2;
  two_prod(x1.hi, y1.hi, p1, e1);
  two_prod(x2.hi, y2.hi, p2, e2);
  float l = __fmaf_rn(x1.hi, y1.lo, __fmaf_rn(x1.lo, y1.hi, e1));
  l = __fadd_rn(l, __fmaf_rn(x2.hi, y2.lo, __fmaf_rn(x2.lo, y2.hi, e2)));
  float s, es;
  two_sum(p1, p2, s, es);
  df r;
  two_sum(s, __fadd_rn(l, es), r.hi, r.lo);
  return r;
}

// 1 / d: one Newton step r = r0 + r0 (1 - d r0) from the FP32 reciprocal
// r0 of the high part; the residual 1 - d r0 is formed with df_dot2, which
// keeps it exact to u^2 while it cancels (accuracy about u^2 relative).
__device__ __forceinline__ df df_recip(df d) {
  const float r0 = __frcp_rn(d.hi);
  const df one{1.f, 0.f}, z{0.f, 0.f};
  const df e = df_dot2(one, df{-d.hi, -d.lo}, df{r0, 0.f}, z, z);
  return df_add(df{r0, 0.f}, df{r0, 0.f} * e);
}

// Complex operations on cx<df> (overloads of the templates in
// hc_device.cuh; a complex product is two two-term dot products).
__device__ __forceinline__ cx<df> operator*(cx<df> a, cx<df> b) {
  return {df_sdot2(a.re, b.re, -a.im, b.im), df_sdot2(a.re, b.im, a.im, b.re)};
}
__device__ __forceinline__ cx<df> cfma(cx<df> a, cx<df> b, cx<df> acc) {
  return {df_dot2(acc.re, a.re, b.re, -a.im, b.im), df_dot2(acc.im, a.re, b.im, a.im, b.re)};
}
__device__ __forceinline__ cx<df> cfms(cx<df> a, cx<df> b, cx<df> acc) {
  return {df_dot2(acc.re, -a.re, b.re, a.im, b.im), df_dot2(acc.im, -a.re, b.im, -a.im, b.re)};
}
// 1/z = conj(z) / |z|^2 (|z| must stay inside FP32's range, as for the
// FP32 solve: a pivot outside it gives a non-finite reciprocal and the step
// is rejected)
__device__ __forceinline__ cx<df> crecip(cx<df> z) {
  const df inv = df_recip(df_sdot2(z.re, z.re, z.im, z.im));
  return {z.re * inv, -(z.im * inv)};
}
// magnitudes for pivot choice and tests: FP32 accuracy from the high parts
__device__ __forceinline__ float cabs1(cx<df> z) { return fabsf(z.re.hi) + fabsf(z.im.hi); }
__device__ __forceinline__ float cnorm2(cx<df> z) {
  return fmaf(z.re.hi, z.re.hi, z.im.hi * z.im.hi);
}
__device__ __forceinline__ float cabs2(cx<df> z) { return sqrtf(cnorm2(z)); }
// complex double <-> complex double-float
__device__ __forceinline__ cx<df> to_cxdf(cx<double> z) { return {df(z.re), df(z.im)}; }
__device__ __forceinline__ cx<df> to_cxdf(cdf z) { return {z.re(), z.im()}; }
// butterfly sum over the lanes xor o (o = L .. L * PARTS / 2) of a warp
__device__ __forceinline__ df shfl_xor_df(df v, int o) {
  return df{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

}  // namespace hc
