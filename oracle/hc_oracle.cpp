// Plain, slow, FP64 CPU oracle for homotopy-continuation path tracking.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
// leg of the benchmark may load this library.  It shares no code, header,
// table or helper with the CUDA path; the two meet only in the term-list
// input format and the numeric status codes documented below.
//
// What it computes (paper: "GPU-Based Homotopy Continuation for Minimal
// Problems in Computer Vision", Chien et al., arXiv 2112.03444):
//   * Sec. 3, Eq. 1: the homotopy H(x,t) = (1-t) G(x) + t F(x), here with the
//     usual random unit constant gamma in front of G (the paper has none), or
//     the parameter homotopy H(x,t) = F(x; p(t)), p(t) = (1-t) p0 + t p1
//     (Sec. 6 interpolates the system's coefficients between start and target;
//     this oracle interpolates the parameters they depend on, which is the same
//     thing when coefficients are linear in the parameters; kind 2 interpolates
//     the coefficients themselves, c_k(t) = (1-t) c_k(p0) + t c_k(p1)).
//   * Sec. 3, Eqs. 2-4: dx/dt = -(dH/dx)^-1 dH/dt; the predictor is the
//     4th-order Runge-Kutta the paper names (classical tableau).
//   * Sec. 3, Eqs. 5-6: Newton correction at t + dt.
//   * Sec. 6: each linear system A x = b is solved by LU with partial pivoting
//     on the augmented matrix [A b] followed by back substitution with U.
//   * Step control, endgame refinement and classification: the paper is silent;
//     a step is accepted iff Newton converges within max_newton iterations and
//     its first correction is at most max_first_corr * (1 + |x|_inf);
//     the rules below are this project's reading and are shared with the GPU
//     through the settings values, not through code.
//
// Evaluation is by direct expansion of each monomial x^alpha and its
// gradient alpha_j x^(alpha - e_j); it does not use the homogenised term
// tuples of Sec. 6 (that encoding belongs to the CUDA path).
//
// Status codes (numbers are the interface):
//   1 finite, 2 diverged, 3 step underflow, 4 too many steps, 5 non-finite,
//   6 singular endpoint, 7 refinement failed; bit 0x80 = real (finite only).
//
// Parity pins for every function are in tests/test_oracle_pins.py.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

using cd = std::complex<double>;

enum : int { KIND_TOTAL_DEGREE = 0, KIND_PARAMETER = 1, KIND_COEFFICIENT = 2 };
enum : int {
  ST_FINITE = 1, ST_DIVERGED = 2, ST_FAIL_STEP = 3, ST_FAIL_MAXSTEPS = 4,
  ST_FAIL_NAN = 5, ST_SINGULAR = 6, ST_FAIL_REFINE = 7, ST_REAL_BIT = 0x80
};

struct Settings {
  double dt_min, dt_max, dt_init, newton_tol;
  int max_newton, max_steps, grow_after;
  double refine_tol;
  int refine_iters;
  double r_inf, finite_tol, real_tol, singular_cond;
  double max_first_corr;
  // power-series endgame (off when endgame == 0)
  int endgame;
  double eg_s0, eg_ratio, eg_tol;
  int eg_cmax, eg_samples;
};

Settings settings_from(const double* s) {
  Settings o;
  o.dt_min = s[0]; o.dt_max = s[1]; o.dt_init = s[2]; o.newton_tol = s[3];
  o.max_newton = (int)s[4]; o.max_steps = (int)s[5]; o.grow_after = (int)s[6];
  o.refine_tol = s[7]; o.refine_iters = (int)s[8];
  o.r_inf = s[9]; o.finite_tol = s[10]; o.real_tol = s[11]; o.singular_cond = s[12];
  o.max_first_corr = s[13];
  o.endgame = (int)s[14]; o.eg_s0 = s[15]; o.eg_ratio = s[16]; o.eg_tol = s[17];
  o.eg_cmax = (int)s[18]; o.eg_samples = (int)s[19];
  return o;
}

struct Problem {
  int n = 0, T = 0, kind = 0, P = 0, maxpf = 0;
  std::vector<int> eq;
  std::vector<cd> coef;
  std::vector<int> exps;      // T*n
  std::vector<int> pfac;      // T*maxpf, -1 = none
  std::vector<int> deg;       // total degree of each equation
  cd gamma{1.0, 0.0};
  std::vector<cd> p0, p1;
};

cd ipow(cd z, int e) {
  cd r(1.0, 0.0);
  for (int k = 0; k < e; ++k) r *= z;
  return r;
}

// Coefficient of term k at parameter point p, and its t-derivative along
// dp = p1 - p0 (product rule over the parameter factors).
void term_coefficient(const Problem& pr, int k, const cd* p, const cd* dp,
                      cd* c, cd* dc) {
  cd val = pr.coef[k];
  cd der(0.0, 0.0);
  for (int f = 0; f < pr.maxpf; ++f) {
    int l = pr.pfac[(size_t)k * pr.maxpf + f];
    if (l < 0) continue;
    // d(val * p_l) = der * p_l + val * dp_l
    der = der * p[l] + val * dp[l];
    val = val * p[l];
  }
  *c = val;
  *dc = der;
}

// H (n), Hx (n*n row-major, Hx[i*n+j] = dH_i/dx_j), Ht (n) at (x, t).
void evaluate(const Problem& pr, const cd* x, double t, cd* H, cd* Hx, cd* Ht) {
  const int n = pr.n;
  for (int i = 0; i < n; ++i) { H[i] = 0; Ht[i] = 0; }
  for (int i = 0; i < n * n; ++i) Hx[i] = 0;

  std::vector<cd> p(pr.P), dp(pr.P), zero(pr.P, 0.0);
  for (int l = 0; l < pr.P; ++l) {
    if (pr.kind == KIND_PARAMETER) {
      p[l] = (1.0 - t) * pr.p0[l] + t * pr.p1[l];
      dp[l] = pr.p1[l] - pr.p0[l];
    } else {
      p[l] = pr.p1.empty() ? cd(0.0) : pr.p1[l];
      dp[l] = 0.0;
    }
  }

  // F (or F(.; p(t))) and its x-gradient.
  std::vector<cd> F(n, 0.0), Fx((size_t)n * n, 0.0), Ft(n, 0.0);
  for (int k = 0; k < pr.T; ++k) {
    const int i = pr.eq[k];
    const int* a = &pr.exps[(size_t)k * n];
    cd c, dc;
    if (pr.kind == KIND_COEFFICIENT) {
      // Sec. 6: the coefficients themselves are interpolated between the
      // start system (parameters p0) and the target system (p1)
      cd c0, c1, unused;
      term_coefficient(pr, k, pr.p0.data(), zero.data(), &c0, &unused);
      term_coefficient(pr, k, pr.p1.data(), zero.data(), &c1, &unused);
      c = (1.0 - t) * c0 + t * c1;
      dc = c1 - c0;
    } else {
      term_coefficient(pr, k, p.data(), dp.data(), &c, &dc);
    }
    cd mono(1.0, 0.0);
    for (int j = 0; j < n; ++j) mono *= ipow(x[j], a[j]);
    F[i] += c * mono;
    Ft[i] += dc * mono;
    for (int j = 0; j < n; ++j) {
      if (a[j] == 0) continue;
      cd g((double)a[j], 0.0);
      for (int l = 0; l < n; ++l) g *= ipow(x[l], l == j ? a[l] - 1 : a[l]);
      Fx[(size_t)i * n + j] += c * g;
    }
  }

  if (pr.kind == KIND_PARAMETER || pr.kind == KIND_COEFFICIENT) {
    for (int i = 0; i < n; ++i) { H[i] = F[i]; Ht[i] = Ft[i]; }
    for (int i = 0; i < n * n; ++i) Hx[i] = Fx[i];
    return;
  }
  // Total degree: G_i = x_i^{d_i} - 1;  H = (1-t) gamma G + t F.
  for (int i = 0; i < n; ++i) {
    const int d = pr.deg[i];
    cd G = ipow(x[i], d) - 1.0;
    cd Gxi = (double)d * ipow(x[i], d - 1);
    H[i] = (1.0 - t) * pr.gamma * G + t * F[i];
    Ht[i] = F[i] - pr.gamma * G;
    for (int j = 0; j < n; ++j) Hx[(size_t)i * n + j] = t * Fx[(size_t)i * n + j];
    Hx[(size_t)i * n + i] += (1.0 - t) * pr.gamma * Gxi;
  }
}

double pivot_mag(cd z) { return std::fabs(z.real()) + std::fabs(z.imag()); }

// Sec. 6: LU with partial pivoting applied to the augmented matrix [A b]
// (the L-solve rides along in the elimination), then back substitution with
// the cached U.  A is n*n row-major and is overwritten; returns false if a
// pivot is exactly zero or anything is non-finite.
bool lu_solve_augmented(int n, cd* A, cd* b, cd* x) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = pivot_mag(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double m = pivot_mag(A[(size_t)i * n + k]);
      if (m > best) { best = m; p = i; }
    }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
      std::swap(b[k], b[p]);
    }
    const cd piv = A[(size_t)k * n + k];
    for (int i = k + 1; i < n; ++i) {
      const cd l = A[(size_t)i * n + k] / piv;
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
      b[i] -= l * b[k];
      A[(size_t)i * n + k] = 0.0;
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    cd s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[(size_t)k * n + j] * x[j];
    x[k] = s / A[(size_t)k * n + k];
    if (!std::isfinite(x[k].real()) || !std::isfinite(x[k].imag())) return false;
  }
  return true;
}

double norm_inf(int n, const cd* v) {
  double m = 0.0;
  for (int i = 0; i < n; ++i) m = std::max(m, std::abs(v[i]));
  return m;
}

bool all_finite(int n, const cd* v) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i].real()) || !std::isfinite(v[i].imag())) return false;
  return true;
}

// Eqs. 3-4: dx/dt = -(Hx)^-1 Ht at (x, t).
bool davidenko(const Problem& pr, const cd* x, double t, cd* dxdt) {
  const int n = pr.n;
  std::vector<cd> H(n), Hx((size_t)n * n), Ht(n), rhs(n);
  evaluate(pr, x, t, H.data(), Hx.data(), Ht.data());
  for (int i = 0; i < n; ++i) rhs[i] = -Ht[i];
  return lu_solve_augmented(n, Hx.data(), rhs.data(), dxdt);
}

// Classical RK4 on the Davidenko ODE (Sec. 3, the higher-order predictor).
bool rk4(const Problem& pr, const cd* x, double t, double h, cd* xout) {
  const int n = pr.n;
  std::vector<cd> k1(n), k2(n), k3(n), k4(n), y(n);
  if (!davidenko(pr, x, t, k1.data())) return false;
  for (int i = 0; i < n; ++i) y[i] = x[i] + (h / 2.0) * k1[i];
  if (!davidenko(pr, y.data(), t + h / 2.0, k2.data())) return false;
  for (int i = 0; i < n; ++i) y[i] = x[i] + (h / 2.0) * k2[i];
  if (!davidenko(pr, y.data(), t + h / 2.0, k3.data())) return false;
  for (int i = 0; i < n; ++i) y[i] = x[i] + h * k3[i];
  if (!davidenko(pr, y.data(), t + h, k4.data())) return false;
  for (int i = 0; i < n; ++i)
    xout[i] = x[i] + (h / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  return all_finite(n, xout);
}

// Eqs. 5-6: one Newton correction x <- x - Hx^-1 H at time t.  Returns the
// infinity norm of the update in *dnorm.
bool newton_step(const Problem& pr, cd* x, double t, double* dnorm) {
  const int n = pr.n;
  std::vector<cd> H(n), Hx((size_t)n * n), Ht(n), rhs(n), d(n);
  evaluate(pr, x, t, H.data(), Hx.data(), Ht.data());
  for (int i = 0; i < n; ++i) rhs[i] = -H[i];
  if (!lu_solve_augmented(n, Hx.data(), rhs.data(), d.data())) return false;
  for (int i = 0; i < n; ++i) x[i] += d[i];
  *dnorm = norm_inf(n, d.data());
  return all_finite(n, x);
}

// Backward error max_i |F_i(x)| / sum_k |c_k| |x^alpha_k| at t = 1.
double backward_error(const Problem& pr, const cd* x) {
  const int n = pr.n;
  std::vector<cd> F(n, 0.0);
  std::vector<double> S(n, 0.0);
  std::vector<cd> p(pr.P), dp(pr.P, 0.0);
  for (int l = 0; l < pr.P; ++l) p[l] = pr.p1.empty() ? cd(0.0) : pr.p1[l];
  for (int k = 0; k < pr.T; ++k) {
    const int i = pr.eq[k];
    const int* a = &pr.exps[(size_t)k * n];
    cd c, dc;
    term_coefficient(pr, k, p.data(), dp.data(), &c, &dc);
    cd mono(1.0, 0.0);
    for (int j = 0; j < n; ++j) mono *= ipow(x[j], a[j]);
    F[i] += c * mono;
    S[i] += std::abs(c) * std::abs(mono);
  }
  double be = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = std::abs(F[i]);
    be = std::max(be, S[i] > 0.0 ? r / S[i] : r);
  }
  return be;
}

double norm1(int n, const cd* A) {
  double m = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += std::abs(A[(size_t)i * n + j]);
    m = std::max(m, s);
  }
  return m;
}

// 1-norm condition number of Fx(x) at t = 1 (explicit inverse by LU solves).
double cond1_at_end(const Problem& pr, const cd* x) {
  const int n = pr.n;
  std::vector<cd> H(n), Hx((size_t)n * n), Ht(n);
  evaluate(pr, x, 1.0, H.data(), Hx.data(), Ht.data());
  const double an = norm1(n, Hx.data());
  std::vector<cd> inv((size_t)n * n), A((size_t)n * n), e(n), col(n);
  for (int j = 0; j < n; ++j) {
    A = Hx;
    for (int i = 0; i < n; ++i) e[i] = (i == j) ? 1.0 : 0.0;
    if (!lu_solve_augmented(n, A.data(), e.data(), col.data())) return INFINITY;
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + j] = col[i];
  }
  return an * norm1(n, inv.data());
}

// ---------------------------------------------------------------- endgame
// Power-series endgame (Morgan, Sommese & Wampler, "A power series method for
// computing singular solutions to nonlinear analytic systems", Numer. Math.
// 63, 1992; the paper itself is silent on endgames).  With s = 1 - t, a path
// ending at a root of multiplicity m has a fractional power series
// x(s) = sum_k a_k s^(k/c), c the cycle (winding) number; it is analytic in
// w = s^(1/c).  Samples at geometric s_k = s0 h^k give c from the ratio of
// successive differences (|x_k - x_(k+1)| ~ s_k^(1/c)), and the value at
// w = 0 of the cubic Hermite interpolant of two samples (values and
// dx/dw = dx/ds c w^(c-1)) predicts the endpoint.
struct Endgame {
  int n = 0, samples = 0, c = 1, next = 0;
  double s_next = 0.0, dn_prev = 0.0;
  bool have_pred = false;
  std::vector<cd> xa, da, pred;  // previous sample, its dx/ds, the last prediction
};

// value at w = 0 of the cubic Hermite interpolant through (wb, xb, Db) and
// (wa, xa, Da), wb < wa
cd hermite_at_zero(double wb, cd xb, cd Db, double wa, cd xa, cd Da) {
  const double dl = wa - wb, tau = -wb / dl;
  const double t2 = tau * tau, t3 = t2 * tau;
  const double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + tau;
  const double h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
  return h00 * xb + h10 * dl * Db + h01 * xa + h11 * dl * Da;
}

// A sample at s (the path point x and dx/ds there).  A prediction is made
// only while the samples converge: the difference to the previous sample
// shrinks, and the predicted endpoint lies within the tail such a series
// leaves, 4 |x_k - x_(k-1)| / (1 - h^(1/c)), of the sample (paths to
// infinity, whose differences grow, get none).  Returns true once two
// successive predictions with the same cycle number c > 1 agree within
// eg_tol (1 + |x|): eg.pred then holds the endpoint and eg.c the cycle number.
// (A path with c = 1 ends at a nonsingular root that ordinary tracking
// reaches; a Newton refinement started from a misjudged c = 1 prediction
// next to a multiple root could land anywhere.)
bool endgame_sample(Endgame& eg, const Settings& s, double sk, const cd* x, const cd* dxds) {
  const int n = eg.n;
  bool done = false;
  if (eg.samples >= 1) {
    double dn = 0.0;
    for (int i = 0; i < n; ++i) dn = std::max(dn, std::abs(x[i] - eg.xa[i]));
    bool predicted = false;
    if (eg.samples >= 2 && dn > 0.0 && eg.dn_prev > 0.0 && dn < eg.dn_prev) {
      const double r = std::log(s.eg_ratio) / std::log(dn / eg.dn_prev);
      const int c = std::min(std::max((int)std::lround(r), 1), s.eg_cmax);
      const double sa = sk / s.eg_ratio;  // the previous sample's s
      const double wb = std::pow(sk, 1.0 / c), wa = std::pow(sa, 1.0 / c);
      std::vector<cd> P(n);
      double pn = 0.0, dp = 0.0, dx = 0.0;
      for (int i = 0; i < n; ++i) {
        const cd Db = dxds[i] * ((double)c * std::pow(wb, c - 1));
        const cd Da = eg.da[i] * ((double)c * std::pow(wa, c - 1));
        P[i] = hermite_at_zero(wb, x[i], Db, wa, eg.xa[i], Da);
        pn = std::max(pn, std::abs(P[i]));
        dx = std::max(dx, std::abs(P[i] - x[i]));
        if (eg.have_pred) dp = std::max(dp, std::abs(P[i] - eg.pred[i]));
      }
      const double tail = 4.0 * dn / (1.0 - std::pow(s.eg_ratio, 1.0 / c));
      if (dx <= tail) {
        done = c > 1 && eg.have_pred && c == eg.c && dp <= s.eg_tol * (1.0 + pn);
        eg.pred = P;
        eg.c = c;
        predicted = true;
      }
    }
    eg.have_pred = predicted;
    eg.dn_prev = dn;
  }
  eg.xa.assign(x, x + n);
  eg.da.assign(dxds, dxds + n);
  ++eg.samples;
  return done;
}

struct PathResult {
  std::vector<cd> x;
  int status = 0;
  int accepted = 0, rejected = 0, newton = 0;
  double be = 0.0, cond = 0.0, t = 0.0;
};

// One path from t = 0 to t = 1, then refinement and classification.
PathResult track_one(const Problem& pr, const Settings& s, const cd* x0) {
  const int n = pr.n;
  PathResult r;
  r.x.assign(x0, x0 + n);
  std::vector<cd> xp(n);
  double t = 0.0, dt = s.dt_init;
  int consec = 0;
  bool failed = false;

  // endgame: sample times 1 - s_k, s_k = s0 h^k (k < eg_samples), formed by
  // repeated multiplication; the step control lands on each of them
  Endgame eg;
  eg.n = n;
  eg.s_next = s.eg_s0;
  bool eg_done = false;
  while (s.endgame && eg.next < s.eg_samples && 1.0 - eg.s_next <= t) {
    eg.s_next *= s.eg_ratio;
    ++eg.next;
  }
  auto eg_active = [&]() { return s.endgame && eg.next < s.eg_samples; };

  while (t < 1.0) {
    if (r.accepted + r.rejected >= s.max_steps) { r.status = ST_FAIL_MAXSTEPS; failed = true; break; }
    const double target = eg_active() ? 1.0 - eg.s_next : 1.0;
    const bool last = dt >= target - t;
    const double h = last ? target - t : dt;
    const double t1 = last ? target : t + h;
    const bool landing = last && eg_active();
    bool conv = false;
    if (rk4(pr, r.x.data(), t, h, xp.data())) {
      for (int it = 0; it < s.max_newton; ++it) {
        double dn;
        if (!newton_step(pr, xp.data(), t1, &dn)) break;
        ++r.newton;
        const double scale = 1.0 + norm_inf(n, xp.data());
        // A first correction this large means the predictor left the
        // corrector's basin (a likely path jump): reject the step.
        if (it == 0 && dn > s.max_first_corr * scale) break;
        if (dn <= s.newton_tol * scale) { conv = true; break; }
      }
    }
    if (conv) {
      r.x = xp;
      t = t1;
      ++r.accepted;
      if (++consec >= s.grow_after) { dt = std::min(2.0 * dt, s.dt_max); consec = 0; }
      if (norm_inf(n, r.x.data()) > s.r_inf) { r.status = ST_DIVERGED; failed = true; break; }
      if (landing) {
        // a sample: dx/ds = -dx/dt from the Davidenko equation at (x, t)
        std::vector<cd> dxdt(n), dxds(n);
        const double sk = eg.s_next;
        eg.s_next *= s.eg_ratio;
        ++eg.next;
        if (davidenko(pr, r.x.data(), t, dxdt.data())) {
          for (int i = 0; i < n; ++i) dxds[i] = -dxdt[i];
          if (endgame_sample(eg, s, sk, r.x.data(), dxds.data())) { eg_done = true; break; }
        }
      }
    } else {
      ++r.rejected;
      consec = 0;
      dt *= 0.5;
      if (dt < s.dt_min) {
        // inside the endgame the last prediction stands in for the endpoint
        if (s.endgame && eg.have_pred && eg.c > 1) { eg_done = true; break; }
        r.status = ST_FAIL_STEP; failed = true; break;
      }
    }
  }
  if (eg_done) {
    r.x = eg.pred;
    t = 1.0;
    if (eg.c > 1) {
      // a root of multiplicity > 1: the prediction is the endpoint (a Newton
      // step there divides rounding noise by rounding noise), singular by its
      // cycle number; the backward error alone decides
      r.t = t;
      if (!all_finite(n, r.x.data())) { r.status = ST_FAIL_NAN; return r; }
      if (norm_inf(n, r.x.data()) > s.r_inf) { r.status = ST_DIVERGED; return r; }
      r.be = backward_error(pr, r.x.data());
      r.status = (r.be <= s.finite_tol) ? ST_SINGULAR : ST_FAIL_REFINE;
      return r;
    }
  }
  r.t = t;
  if (failed) {
    if (!all_finite(n, r.x.data())) r.status = ST_FAIL_NAN;
    return r;
  }
  // Endgame: Newton on F = H(., 1) to a tight relative fixed point.
  for (int it = 0; it < s.refine_iters; ++it) {
    std::vector<cd> keep = r.x;
    double dn;
    if (!newton_step(pr, r.x.data(), 1.0, &dn)) { r.x = keep; break; }
    if (dn <= s.refine_tol * (1.0 + norm_inf(n, r.x.data()))) break;
  }
  if (!all_finite(n, r.x.data())) { r.status = ST_FAIL_NAN; return r; }
  const double xn = norm_inf(n, r.x.data());
  if (xn > s.r_inf) { r.status = ST_DIVERGED; return r; }
  r.be = backward_error(pr, r.x.data());
  if (!(r.be <= s.finite_tol)) { r.status = ST_FAIL_REFINE; return r; }
  r.cond = cond1_at_end(pr, r.x.data());
  if (!(r.cond <= s.singular_cond)) { r.status = ST_SINGULAR; return r; }
  r.status = ST_FINITE;
  double im = 0.0;
  for (int i = 0; i < n; ++i) im = std::max(im, std::fabs(r.x[i].imag()));
  if (im <= s.real_tol * std::max(1.0, xn)) r.status |= ST_REAL_BIT;
  return r;
}

// Start point k of the total-degree start system x_i^{d_i} = 1: the digits of
// k in mixed radix (d_1, d_2, ...), variable 1 least significant, give
// x_i = exp(2 pi i k_i / d_i).
void start_point(const Problem& pr, int64_t k, cd* x) {
  for (int i = 0; i < pr.n; ++i) {
    const int d = pr.deg[i];
    const int64_t ki = k % d;
    k /= d;
    x[i] = std::polar(1.0, 2.0 * M_PI * (double)ki / (double)d);
  }
}

}  // namespace

extern "C" {

int oracle_abi_version() { return 1; }

void* oracle_problem_new(int n, int T, const int* term_eq, const double* term_coef,
                         const uint8_t* term_exp, int maxpf, const int* term_param,
                         int P, int kind, double gamma_re, double gamma_im,
                         const double* p0, const double* p1) {
  Problem* pr = new Problem;
  pr->n = n; pr->T = T; pr->kind = kind; pr->P = P; pr->maxpf = maxpf;
  pr->eq.assign(term_eq, term_eq + T);
  pr->coef.resize(T);
  for (int k = 0; k < T; ++k) pr->coef[k] = cd(term_coef[2 * k], term_coef[2 * k + 1]);
  pr->exps.resize((size_t)T * n);
  for (size_t k = 0; k < (size_t)T * n; ++k) pr->exps[k] = term_exp[k];
  pr->pfac.assign(term_param, term_param + (size_t)T * maxpf);
  pr->gamma = cd(gamma_re, gamma_im);
  pr->deg.assign(n, 0);
  for (int k = 0; k < T; ++k) {
    int d = 0;
    for (int j = 0; j < n; ++j) d += pr->exps[(size_t)k * n + j];
    pr->deg[pr->eq[k]] = std::max(pr->deg[pr->eq[k]], d);
  }
  if (P > 0) {
    pr->p0.resize(P); pr->p1.resize(P);
    for (int l = 0; l < P; ++l) {
      pr->p0[l] = p0 ? cd(p0[2 * l], p0[2 * l + 1]) : cd(0.0);
      pr->p1[l] = p1 ? cd(p1[2 * l], p1[2 * l + 1]) : cd(0.0);
    }
  }
  return pr;
}

void oracle_problem_free(void* h) { delete static_cast<Problem*>(h); }

int64_t oracle_total_degree_paths(void* h) {
  const Problem& pr = *static_cast<Problem*>(h);
  int64_t c = 1;
  for (int d : pr.deg) c *= d;
  return c;
}

void oracle_start_point(void* h, int64_t k, double* x) {
  const Problem& pr = *static_cast<Problem*>(h);
  std::vector<cd> v(pr.n);
  start_point(pr, k, v.data());
  for (int i = 0; i < pr.n; ++i) { x[2 * i] = v[i].real(); x[2 * i + 1] = v[i].imag(); }
}

void oracle_eval(void* h, const double* x, double t, double* H, double* Hx, double* Ht) {
  const Problem& pr = *static_cast<Problem*>(h);
  const int n = pr.n;
  std::vector<cd> xv(n), Hv(n), Hxv((size_t)n * n), Htv(n);
  for (int i = 0; i < n; ++i) xv[i] = cd(x[2 * i], x[2 * i + 1]);
  evaluate(pr, xv.data(), t, Hv.data(), Hxv.data(), Htv.data());
  for (int i = 0; i < n; ++i) {
    H[2 * i] = Hv[i].real(); H[2 * i + 1] = Hv[i].imag();
    Ht[2 * i] = Htv[i].real(); Ht[2 * i + 1] = Htv[i].imag();
  }
  for (size_t i = 0; i < (size_t)n * n; ++i) { Hx[2 * i] = Hxv[i].real(); Hx[2 * i + 1] = Hxv[i].imag(); }
}

// Dense complex solve A x = b (A row-major n*n), Sec. 6 augmented LU.
int oracle_solve(int n, const double* A, const double* b, double* x) {
  std::vector<cd> Av((size_t)n * n), bv(n), xv(n);
  for (size_t i = 0; i < (size_t)n * n; ++i) Av[i] = cd(A[2 * i], A[2 * i + 1]);
  for (int i = 0; i < n; ++i) bv[i] = cd(b[2 * i], b[2 * i + 1]);
  bool ok = lu_solve_augmented(n, Av.data(), bv.data(), xv.data());
  for (int i = 0; i < n; ++i) { x[2 * i] = xv[i].real(); x[2 * i + 1] = xv[i].imag(); }
  return ok ? 0 : 1;
}

int oracle_rk4_step(void* h, const double* x, double t, double dt, double* xout) {
  const Problem& pr = *static_cast<Problem*>(h);
  const int n = pr.n;
  std::vector<cd> xv(n), yv(n);
  for (int i = 0; i < n; ++i) xv[i] = cd(x[2 * i], x[2 * i + 1]);
  bool ok = rk4(pr, xv.data(), t, dt, yv.data());
  for (int i = 0; i < n; ++i) { xout[2 * i] = yv[i].real(); xout[2 * i + 1] = yv[i].imag(); }
  return ok ? 0 : 1;
}

int oracle_newton_step(void* h, double* x, double t, double* dnorm) {
  const Problem& pr = *static_cast<Problem*>(h);
  const int n = pr.n;
  std::vector<cd> xv(n);
  for (int i = 0; i < n; ++i) xv[i] = cd(x[2 * i], x[2 * i + 1]);
  bool ok = newton_step(pr, xv.data(), t, dnorm);
  for (int i = 0; i < n; ++i) { x[2 * i] = xv[i].real(); x[2 * i + 1] = xv[i].imag(); }
  return ok ? 0 : 1;
}

// Track n_paths paths.  start: [n_paths, n] complex (interleaved) or NULL for
// the total-degree start points selected by path_ids (NULL = 0..n_paths-1).
// Outputs: x [n_paths, n] complex, status u8, counts int32 [n_paths, 3]
// (accepted, rejected, Newton iterations), be/cond/t double.
void oracle_track(void* h, int64_t n_paths, const double* start, const int64_t* path_ids,
                  const double* settings, int n_threads, double* out_x, uint8_t* out_status,
                  int32_t* out_counts, double* out_be, double* out_cond, double* out_t) {
  const Problem& pr = *static_cast<Problem*>(h);
  const Settings s = settings_from(settings);
  const int n = pr.n;
  std::atomic<int64_t> next(0);
  auto worker = [&]() {
    std::vector<cd> x0(n);
    for (;;) {
      const int64_t k = next.fetch_add(1);
      if (k >= n_paths) break;
      if (start) {
        for (int i = 0; i < n; ++i)
          x0[i] = cd(start[(k * n + i) * 2], start[(k * n + i) * 2 + 1]);
      } else {
        start_point(pr, path_ids ? path_ids[k] : k, x0.data());
      }
      PathResult r = track_one(pr, s, x0.data());
      for (int i = 0; i < n; ++i) {
        out_x[(k * n + i) * 2] = r.x[i].real();
        out_x[(k * n + i) * 2 + 1] = r.x[i].imag();
      }
      out_status[k] = (uint8_t)r.status;
      if (out_counts) {
        out_counts[k * 3] = r.accepted; out_counts[k * 3 + 1] = r.rejected;
        out_counts[k * 3 + 2] = r.newton;
      }
      if (out_be) out_be[k] = r.be;
      if (out_cond) out_cond[k] = r.cond;
      if (out_t) out_t[k] = r.t;
    }
  };
  if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (n_threads == 1) { worker(); return; }
  std::vector<std::thread> pool;
  for (int i = 0; i < n_threads; ++i) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
}

// Backward error max_i |F_i(x)| / sum_k |c_k| |x^alpha_k| and the 1-norm
// condition number of dF/dx, both at t = 1 and a given point x (the two
// classification quantities of track_one, exposed for their pins).
double oracle_backward_error(void* h, const double* x) {
  const Problem& pr = *static_cast<Problem*>(h);
  std::vector<cd> xv(pr.n);
  for (int i = 0; i < pr.n; ++i) xv[i] = cd(x[2 * i], x[2 * i + 1]);
  return backward_error(pr, xv.data());
}

double oracle_cond1(void* h, const double* x) {
  const Problem& pr = *static_cast<Problem*>(h);
  std::vector<cd> xv(pr.n);
  for (int i = 0; i < pr.n; ++i) xv[i] = cd(x[2 * i], x[2 * i + 1]);
  return cond1_at_end(pr, xv.data());
}

int oracle_hardware_threads() { return (int)std::max(1u, std::thread::hardware_concurrency()); }

}  // extern "C"
