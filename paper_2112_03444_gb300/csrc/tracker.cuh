// Per-path predictor-corrector tracker executed by one lane group.
//
// Method (paper Sec. 3): from a start solution at t = 0, repeat
//   predictor: classical RK4 on dx/dt = -(dH/dx)^-1 dH/dt   (Eqs. 2-4; the
//              paper names a 4th-order Runge-Kutta; the tableau is classical)
//   corrector: Newton x <- x - (dH/dx)^-1 H at t + dt          (Eqs. 5-6)
// until t = 1, then refine the endpoint with Newton on F = H(., 1) and
// classify it.  Step control (the paper is silent) is the library's rule:
// accept iff Newton converges within max_newton iterations and its first
// correction is small; double dt after grow_after accepts; halve on reject.
//
// Precision.  MIXED = false: everything in complex FP64.  MIXED = true: the
// four RK4 stages and the Newton iterations evaluate and solve in complex
// FP32; the path state x and t stay FP64; for t > t_endgame the corrector's
// residual H is evaluated in FP64 (iterative refinement with the FP32
// solve), and the final refinement and the backward error use FP64
// residuals.  GB300 issues FP64 at a small fraction of the FP32 rate, so
// FP64 is spent only where it buys accuracy.
//
// Evaluator interface (HOM):
//   template <class R> eval(x[N], i, t, 1-t, row[N+1], H, Ht)
//       row[j] = dH_i/dx_j (j < N), H = H_i, Ht = dH_i/dt, all at (x, t)
//   residual64<SCALE>(x[N], i, t, 1-t, H, scale)   H_i in FP64, and with
//       SCALE the backward-error denominator sum |c| |x^a| of row i
//   start(path, i)                                 start component x_i(0)
#pragma once

#include <type_traits>

#include "hc_device.cuh"

namespace hc {

struct PathOut {
  cx<double> x;  // this lane's component of the endpoint
  int status, nacc, nrej, nnewt;
  float be;
};

template <int N, class R>
__device__ __forceinline__ void load_vec(const cx<double>* buf, cx<R> (&x)[N]) {
#pragma unroll
  for (int k = 0; k < N; ++k) x[k] = cvt<R>(buf[k]);
}

// 1-norm condition number of dH/dx(x, 1) from an explicit inverse in chunks
// of NR columns (Gauss-Jordan on [A | e_c ... e_{c+NR-1}]).
template <int N, int L, class R, class HOM>
__device__ __forceinline__ float cond1(const HOM& hom, const Group& g, const cx<R> (&x)[N]) {
  constexpr int NR = N < 4 ? N : 4;
  cx<R> a[N + NR];
  cx<R> row[N + 1];
  cx<R> H, Ht;
  hom.template eval<R>(x, g.gl, R(1), R(0), row, H, Ht);
  const bool act = g.gl < N;
  float anorm = 0.f;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const float cs = gsum<L, float>(g, act ? (float)cabs2(row[j]) : 0.f);
    anorm = fmaxf(anorm, cs);
  }
  float inorm = 0.f;
#pragma unroll 1
  for (int c0 = 0; c0 < N; c0 += NR) {
    hom.template eval<R>(x, g.gl, R(1), R(0), row, H, Ht);
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = row[j];
#pragma unroll
    for (int r = 0; r < NR; ++r)
      a[N + r] = mk<R>((act && g.gl == c0 + r) ? R(1) : R(0), R(0));
    cx<R> sol[NR];
    int col;
    const bool ok = gj_solve<N, NR, R>(g, a, sol, col);
    if (!ok) return INFINITY;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const float v = (col >= 0 && c0 + r < N) ? (float)cabs2(sol[r]) : 0.f;
      inorm = fmaxf(inorm, gsum<L, float>(g, v));
    }
  }
  return anorm * inorm;
}

template <int N, int L, bool MIXED, class HOM>
__device__ __forceinline__ void track_path(const HOM& hom, const DevSettings& s, const Group& g,
                                           cx<double>* vb, void* sb_raw, int64_t path,
                                           PathOut& o) {
  using R = typename std::conditional<MIXED, float, double>::type;
  cx<R>* sb = reinterpret_cast<cx<R>*>(sb_raw);
  const bool act = g.gl < N;
  cx<double> xi = act ? hom.start(path, g.gl) : czero<double>();
  double t = 0.0, dt = s.dt_init;
  int consec = 0, nacc = 0, nrej = 0, nnewt = 0, status = 0;
  const float tolc = MIXED ? (float)s.newton_tol_fp32 : (float)s.newton_tol;
  cx<R> row[N + 1];
  cx<R> x[N];
  cx<R> sol[1];
  int col;

  // Share one component per lane through the group's vector buffer and load
  // the whole vector into registers (every lane evaluates its row at x).
  auto publish = [&](const cx<double>& v) {
    if (act) vb[g.gl] = v;
    __syncwarp(g.mask);
    load_vec<N, R>(vb, x);
  };
  // Scatter the solve's components (lane with pivot column c holds x[c]) and
  // return this lane's own component.
  auto exchange = [&](const cx<R>& v, int c) -> cx<R> {
    if (c >= 0) sb[c] = v;
    __syncwarp(g.mask);
    return act ? sb[g.gl] : czero<R>();
  };

#pragma unroll 1
  while (t < 1.0) {
    if (nacc + nrej >= s.max_steps) {
      status = ST_FAIL_MAXSTEPS;
      break;
    }
    const bool last = dt >= 1.0 - t;
    const double h = last ? 1.0 - t : dt;
    const double t1 = last ? 1.0 : t + h;
    bool ok = true;

    // ---- predictor: classical RK4 (stages at t, t+h/2, t+h/2, t+h)
    cx<double> ksum = czero<double>();
    cx<R> kprev = czero<R>();
#pragma unroll 1
    for (int st = 0; st < 4; ++st) {
      const double c = (st == 0) ? 0.0 : (st == 3 ? 1.0 : 0.5);
      const double ts = t + c * h;
      publish(xi + (c * h) * cvt<double>(kprev));
      cx<R> H, Ht;
      hom.template eval<R>(x, g.gl, (R)ts, (R)(1.0 - ts), row, H, Ht);
      row[N] = -Ht;
      ok = gj_solve<N, 1, R>(g, row, sol, col) && ok;
      kprev = exchange(sol[0], col);
      ksum = ksum + ((st == 0 || st == 3) ? 1.0 : 2.0) * cvt<double>(kprev);
    }
    cx<double> xp = xi + (h / 6.0) * ksum;

    // ---- corrector: Newton at t1
    bool conv = false;
    float xn = 0.f;
    const bool endgame = MIXED && (t1 > s.t_endgame);
    if (ok) {
#pragma unroll 1
      for (int it = 0; it < s.max_newton; ++it) {
        publish(xp);
        cx<R> H, Ht;
        hom.template eval<R>(x, g.gl, (R)t1, (R)(1.0 - t1), row, H, Ht);
        if (endgame) {
          cx<double> xd[N];
          load_vec<N, double>(vb, xd);
          cx<double> H64;
          double sc;
          hom.template residual64<false>(xd, g.gl, t1, 1.0 - t1, H64, sc);
          row[N] = cvt<R>(-H64);
        } else {
          row[N] = -H;
        }
        const bool sok = gj_solve<N, 1, R>(g, row, sol, col);
        const cx<R> d = exchange(sol[0], col);
        xp = xp + cvt<double>(d);
        ++nnewt;
        const float dn = gmaxf(g, act ? (float)cabs2(d) : 0.f);
        xn = gmaxf(g, act ? (float)cabs2(xp) : 0.f);
        if (!sok || !(dn <= 3.0e38f) || !(xn <= 3.0e38f)) break;
        if (it == 0 && dn > (float)s.max_first_corr * (1.f + xn)) break;
        if (dn <= tolc * (1.f + xn)) {
          conv = true;
          break;
        }
      }
    }

    // ---- step control
    if (conv) {
      xi = xp;
      t = t1;
      ++nacc;
      if (++consec >= s.grow_after) {
        dt = fmin(2.0 * dt, s.dt_max);
        consec = 0;
      }
      if ((double)xn > s.r_inf) {
        status = ST_DIVERGED;
        break;
      }
    } else {
      ++nrej;
      consec = 0;
      dt *= 0.5;
      if (dt < s.dt_min) {
        status = ST_FAIL_STEP;
        break;
      }
    }
  }

  float be = 0.f;
  if (status == 0) {
    // ---- endpoint refinement: Newton on F with FP64 residuals
#pragma unroll 1
    for (int it = 0; it < s.refine_iters; ++it) {
      publish(xi);
      cx<double> xd[N];
      load_vec<N, double>(vb, xd);
      cx<R> H, Ht;
      hom.template eval<R>(x, g.gl, R(1), R(0), row, H, Ht);
      cx<double> H64;
      double sc;
      hom.template residual64<false>(xd, g.gl, 1.0, 0.0, H64, sc);
      row[N] = cvt<R>(-H64);
      const bool sok = gj_solve<N, 1, R>(g, row, sol, col);
      const cx<R> d = exchange(sol[0], col);
      const cx<double> xnew = xi + cvt<double>(d);
      const float dn = gmaxf(g, act ? (float)cabs2(d) : 0.f);
      const float xnn = gmaxf(g, act ? (float)cabs2(xnew) : 0.f);
      if (!sok || !(dn <= 3.0e38f) || !(xnn <= 3.0e38f)) break;
      xi = xnew;
      if (dn <= (float)s.refine_tol * (1.f + xnn)) break;
    }

    // ---- classification (same order and thresholds as the settings define)
    publish(xi);
    cx<double> xd[N];
    load_vec<N, double>(vb, xd);
    const bool fin = !gany(g, act && !cfinite(xi));
    const float xnf = gmaxf(g, act ? (float)cabs2(xi) : 0.f);
    if (!fin) {
      status = ST_FAIL_NAN;
    } else if ((double)xnf > s.r_inf) {
      status = ST_DIVERGED;
    } else {
      cx<double> H64;
      double sc;
      hom.template residual64<true>(xd, g.gl, 1.0, 0.0, H64, sc);
      const double r = cabs2(H64);
      const double bei = act ? (sc > 0.0 ? r / sc : r) : 0.0;
      be = gmaxf(g, (float)bei);
      if (!((double)be <= s.finite_tol)) {
        status = ST_FAIL_REFINE;
      } else {
        const float cnd = cond1<N, L, R>(hom, g, x);
        const double lim = MIXED ? fmin(s.singular_cond, kFp32CondTrust) : s.singular_cond;
        if (!((double)cnd <= lim)) {
          status = ST_SINGULAR;
        } else {
          const float im = gmaxf(g, act ? (float)fabs(xi.im) : 0.f);
          status = ST_FINITE;
          if ((double)im <= s.real_tol * fmax(1.0, (double)xnf)) status |= ST_REAL;
        }
      }
    }
  } else if (gany(g, act && !cfinite(xi))) {
    status = ST_FAIL_NAN;
  }
  o.x = xi;
  o.status = status;
  o.nacc = nacc;
  o.nrej = nrej;
  o.nnewt = nnewt;
  o.be = be;
}

}  // namespace hc
