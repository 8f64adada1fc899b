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
// Code shape.  Every phase of the method needs the same work item: evaluate
// row i of [dH/dx | rhs] at some point and time, solve, and scatter the
// solution.  The tracker is therefore one loop around ONE copy of the
// (fully unrolled) evaluation and solve, driven by a small per-path state
// machine: RK stage 1..4, Newton iteration, endpoint refinement, condition
// columns.  Inlining a copy per phase multiplied the kernel's code size and
// made instruction fetch the dominant stall once the lane groups of an SM
// drifted into different phases.
//
// Precision tiers.
//   MIXED = false: every operation in complex FP64 (the plain form).
//   MIXED = true : for t < t_endgame the state, the RK4 stages and the Newton
//     iterations are complex FP32 and no FP64 instruction executes; for
//     t > t_endgame the state is FP64 and the corrector's residual H is
//     evaluated in FP64 while the Jacobian and the solve stay FP32 (mixed
//     precision iterative refinement); the final refinement and the backward
//     error use FP64 residuals the same way.  GB300 issues FP64 FMAs at about
//     1/74 of its FP32 rate (measured), so FP64 is kept to a few residuals per
//     path.  A path the FP32 tier cannot resolve (step below dt_min_fp32,
//     step budget, suspect condition) is reported failed and re-tracked by
//     the FP64 tier.
//
// Evaluator interface (HOM):
//   template <class R> eval(x[N], i, t, 1-t, row[N+1], H, Ht)
//       row[j] = dH_i/dx_j (j < N), H = H_i, Ht = dH_i/dt, all at (x, t)
//   residual64<SCALE>(xs, i, t, 1-t, H, scale)   H_i in FP64 at the point
//       xs[0..N) (shared memory), and with SCALE the backward-error
//       denominator sum |c| |x^a| of row i
//   start(path, i)                                 start component x_i(0)
#pragma once

#include <type_traits>

#include "hc_device.cuh"

namespace hc {

struct PathOut {
  cx<double> x;  // this lane's component of the endpoint
  double t;      // where tracking stopped (1 unless the path failed on the way)
  int status, nacc, nrej, nnewt;
  float be;
};

template <int N, class S, class R>
__device__ __forceinline__ void load_vec(const cx<S>* buf, cx<R> (&x)[N]) {
#pragma unroll
  for (int k = 0; k < N; ++k) x[k] = cvt<R>(buf[k]);
}

enum : int { M_RK = 0, M_NEWTON = 1, M_REFINE = 2, M_COND = 3, M_DONE = 4 };

// Shared memory of one lane group: vf = FP32 copy of the evaluation point,
// vd = FP64 copy (phases with FP64 state), sb = solution scatter buffer.
template <int L>
struct GroupSmem {
  cx<double> vd[L];
  cx<double> sb[L];  // holds L values of cx<R>
  cx<float> vf[L];
};


template <int N, int L, bool MIXED, class HOM>
__device__ __forceinline__ void track_path(const HOM& hom, const DevSettings& s, const Group& g,
                                           GroupSmem<L>* sm, int64_t path, double t0,
                                           const double2* x0, PathOut& o) {
  using R = typename std::conditional<MIXED, float, double>::type;
  cx<R>* sb = reinterpret_cast<cx<R>*>(sm->sb);
  const bool act = g.gl < N;
  o.be = 0.f;

  // ---- path state (identical control state in all lanes of the group); a
  // path handed over by the FP32 tier resumes from its last accepted point.
  cx<double> xd = czero<double>();  // FP64 state
  if (act) {
    if (x0) {
      const double2 v = x0[g.gl];
      xd = mk<double>(v.x, v.y);
    } else {
      xd = hom.start(path, g.gl);
    }
  }
  cx<float> xf = cvt<float>(xd);  // FP32 state
  bool hi = !MIXED;  // state lives in xd (FP64) rather than xf
  double t = x0 ? t0 : 0.0, dt = s.dt_init, h = 0.0, t1 = 0.0;
  int consec = 0, nacc = 0, nrej = 0, nnewt = 0, status = 0;
  const double tA = MIXED ? fmin(s.t_endgame, 1.0) : 1.0;  // end of the FP32 phase
  const float tol = MIXED ? (float)s.newton_tol_fp32 : (float)s.newton_tol;
  const float corr1 = MIXED ? (float)s.max_first_corr_fp32 : (float)s.max_first_corr;
  const double dtmin = MIXED ? s.dt_min_fp32 : s.dt_min;
  const int maxsteps = MIXED ? s.max_steps_fp32 : s.max_steps;

  int mode = M_RK, stage = 0, it = 0;
  cx<R> kprev = czero<R>(), ksum = czero<R>();
  cx<float> xpf = xf;       // corrector iterate (FP32 phase)
  cx<double> xpd = xd;      // corrector iterate (FP64 state)
  bool step_ok = true;
  float cond_inorm = 0.f, cond_anorm = 0.f;

  cx<R> row[N + 1];
  cx<R> x[N];
  cx<R> sol[1];
  int col;

  // Begins a step from (t, state): picks h, t1 for the current phase.
  auto begin_step = [&]() {
    const double t_stop = hi ? 1.0 : tA;
    const bool last = dt >= t_stop - t;
    h = last ? t_stop - t : dt;
    t1 = last ? t_stop : t + h;
    stage = 0;
    ksum = czero<R>();
    kprev = czero<R>();
    step_ok = true;
    mode = M_RK;
  };
  auto enter_refine = [&]() {
    if (!hi) xd = cvt<double>(xf);
    hi = true;
    mode = M_REFINE;
    it = 0;
  };
  auto reject = [&]() {
    ++nrej;
    consec = 0;
    dt *= 0.5;
    if (dt < dtmin) {
      status = ST_FAIL_STEP;
      mode = M_DONE;
    } else {
      begin_step();
    }
  };
  begin_step();

#pragma unroll 1
  for (;;) {
    if (mode == M_DONE) break;
    if (mode == M_RK && stage == 0 && nacc + nrej >= maxsteps) {
      status = ST_FAIL_MAXSTEPS;
      break;
    }
    // ---- 1. evaluation point and time
    double te;
    bool need64 = false;
    if (mode == M_RK) {
      const double c = (stage == 0) ? 0.0 : (stage == 3 ? 1.0 : 0.5);
      te = (stage == 3) ? t1 : t + c * h;
      if (hi) {
        const cx<double> p = xd + (c * h) * cvt<double>(kprev);
        if (act) sm->vd[g.gl] = p;
        if (act) sm->vf[g.gl] = cvt<float>(p);
      } else {
        const cx<float> p = xf + ((float)c * (float)h) * cvt<float>(kprev);
        if (act) sm->vf[g.gl] = p;
      }
    } else if (mode == M_NEWTON) {
      te = t1;
      need64 = MIXED && hi;
      if (hi) {
        if (act) sm->vd[g.gl] = xpd;
        if (act) sm->vf[g.gl] = cvt<float>(xpd);
      } else {
        if (act) sm->vf[g.gl] = xpf;
      }
    } else {  // M_REFINE, M_COND: at the endpoint, t = 1
      te = 1.0;
      need64 = (mode == M_REFINE);
      if (act) sm->vd[g.gl] = xd;
      if (act) sm->vf[g.gl] = cvt<float>(xd);
    }
    __syncwarp(g.mask);
    if constexpr (MIXED) {
      load_vec<N, float, float>(sm->vf, x);
    } else {
      load_vec<N, double, double>(sm->vd, x);
    }

    // ---- 2. row i of [dH/dx | rhs] and the solve
    {
      cx<R> H, Ht;
      const R ter = (R)te;
      const R omt = hi ? (R)(1.0 - te) : R(1) - ter;
      hom.template eval<R>(x, g.gl, ter, omt, row, H, Ht);
      if (mode == M_RK) {
        row[N] = -Ht;
      } else if (mode == M_COND) {
        if (stage == 0) {  // first column pass: 1-norm of the matrix
          float an = 0.f;
#pragma unroll
          for (int j = 0; j < N; ++j)
            an = fmaxf(an, gsum<L, float>(g, act ? cabs2(cvt<float>(row[j])) : 0.f));
          cond_anorm = an;
        }
        row[N] = mk<R>((act && g.gl == stage) ? R(1) : R(0), R(0));
      } else if (need64) {
        cx<double> H64;
        double sc;
        hom.template residual64<false>(sm->vd, g.gl, te, 1.0 - te, H64, sc);
        row[N] = cvt<R>(-H64);
      } else {
        row[N] = -H;
      }
    }
    const bool sok = gj_solve<N, 1, R>(g, row, sol, col);
    if (col >= 0) sb[col] = sol[0];
    __syncwarp(g.mask);
    const cx<R> d = act ? sb[g.gl] : czero<R>();

    // ---- 3. state machine
    if (mode == M_RK) {
      step_ok = step_ok && sok;
      kprev = d;
      ksum = ksum + ((stage == 0 || stage == 3) ? R(1) : R(2)) * d;
      if (++stage == 4) {
        if (!step_ok) {
          reject();
          continue;
        }
        if (hi)
          xpd = xd + (h / 6.0) * cvt<double>(ksum);
        else
          xpf = xf + ((float)h / 6.0f) * cvt<float>(ksum);
        mode = M_NEWTON;
        it = 0;
      }
    } else if (mode == M_NEWTON) {
      float xn2;
      if (hi) {
        xpd = xpd + cvt<double>(d);
        xn2 = gmaxf(g, act ? cnorm2(cvt<float>(xpd)) : 0.f);
      } else {
        xpf = xpf + cvt<float>(d);
        xn2 = gmaxf(g, act ? cnorm2(xpf) : 0.f);
      }
      ++nnewt;
      const float xn = sqrt_approx(xn2);
      const float dn = sqrt_approx(gmaxf(g, act ? (float)cnorm2(d) : 0.f));
      const bool bad = !sok || !(dn <= 3.0e38f) || !(xn <= 3.0e38f) ||
                       (it == 0 && dn > corr1 * (1.f + xn));
      if (!bad && dn <= tol * (1.f + xn)) {
        // accept
        if (hi) xd = xpd; else xf = xpf;
        t = t1;
        ++nacc;
        if (++consec >= s.grow_after) {
          dt = fmin(2.0 * dt, s.dt_max);
          consec = 0;
        }
        if ((double)xn > s.r_inf) {
          status = ST_DIVERGED;
          mode = M_DONE;
        } else if (t >= 1.0) {
          enter_refine();
        } else {
          if (!hi && t >= tA) {  // enter the FP64-state phase
            xd = cvt<double>(xf);
            hi = true;
          }
          begin_step();
        }
      } else if (bad || ++it >= s.max_newton) {
        reject();
      }
    } else if (mode == M_REFINE) {
      const cx<double> xnew = xd + cvt<double>(d);
      const float dn = sqrt_approx(gmaxf(g, act ? (float)cnorm2(d) : 0.f));
      const float xnn = sqrt_approx(gmaxf(g, act ? cnorm2(cvt<float>(xnew)) : 0.f));
      const bool bad = !sok || !(dn <= 3.0e38f) || !(xnn <= 3.0e38f);
      if (!bad) xd = xnew;
      if (bad || dn <= (float)s.refine_tol * (1.f + xnn) || ++it >= s.refine_iters) {
        // classify: finiteness, divergence, backward error (FP64 residual)
        const bool fin = !gany(g, act && !cfinite(xd));
        const float xnf = gmaxf(g, act ? cabs2(cvt<float>(xd)) : 0.f);
        if (!fin) {
          status = ST_FAIL_NAN;
          mode = M_DONE;
        } else if ((double)xnf > s.r_inf) {
          status = ST_DIVERGED;
          mode = M_DONE;
        } else {
          __syncwarp(g.mask);
          if (act) sm->vd[g.gl] = xd;
          __syncwarp(g.mask);
          cx<double> H64;
          double sc;
          hom.template residual64<true>(sm->vd, g.gl, 1.0, 0.0, H64, sc);
          const double r = (double)cabs2(cvt<float>(H64));
          const double bei = act ? (sc > 0.0 ? r / sc : r) : 0.0;
          o.be = gmaxf(g, (float)bei);
          if (!((double)o.be <= s.finite_tol)) {
            status = ST_FAIL_REFINE;
            mode = M_DONE;
          } else {
            mode = M_COND;  // condition number: one solve per column of the inverse
            stage = 0;
            cond_inorm = 0.f;
          }
        }
      }
    } else {  // M_COND
      if (!sok) cond_inorm = INFINITY;
      cond_inorm = fmaxf(cond_inorm, gsum<L, float>(g, (act && col >= 0) ? cabs2(cvt<float>(d)) : 0.f));
      if (++stage >= N) {
        const double cnd = (double)cond_anorm * (double)cond_inorm;
        const double lim = MIXED ? fmin(s.singular_cond, kFp32CondTrust) : s.singular_cond;
        if (!(cnd <= lim)) {
          status = ST_SINGULAR;
        } else {
          const float xnf = gmaxf(g, act ? cabs2(cvt<float>(xd)) : 0.f);
          const float im = gmaxf(g, act ? fabsf((float)xd.im) : 0.f);
          status = ST_FINITE;
          if ((double)im <= s.real_tol * fmax(1.0, (double)xnf)) status |= ST_REAL;
        }
        mode = M_DONE;
      }
    }
  }

  if (!hi) xd = cvt<double>(xf);
  if ((status & 0x7f) != ST_FINITE && status != ST_FAIL_NAN && gany(g, act && !cfinite(xd)))
    status = ST_FAIL_NAN;
  o.x = xd;
  o.t = t;
  o.status = status;
  o.nacc = nacc;
  o.nrej = nrej;
  o.nnewt = nnewt;
}

}  // namespace hc
