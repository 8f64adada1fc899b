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
// solution.  A lane group therefore runs ONE loop around ONE copy of the
// (fully unrolled) evaluation and solve, driven by a small state machine:
// fetch the next path (retire/refill of the persistent launch), RK stage
// 1..4, Newton iteration, endpoint refinement, condition columns, write the
// result.  Inlining a copy per phase multiplied the code size and made
// instruction fetch the dominant stall; keeping path fetch and output inside
// the same loop keeps the lane groups that share a warp executing the heavy
// body together even when their paths start and end at different times.
//
// Precision tiers.
//   MIXED = false, RE = double: every operation in complex FP64 (the plain form).
//   MIXED = false, RE = df: the same state, time, step control, corrector
//     and refinement residuals and classification in FP64, but the RK4
//     stages, the Jacobians and the solves -- nearly all of the arithmetic --
//     in complex double-float arithmetic (FP32 pairs, about 48 bits, see
//     dfloat.cuh) on the FP32 pipe.  After a path's first rejected step the
//     corrector takes its residual in FP64: iterative refinement with a
//     48-bit solve, which reaches what an FP64 corrector reaches (a path of
//     condition 1e10 would otherwise sit at a double-float noise floor of
//     1e-5), and the FP64 residual costs a fraction of an FP64 evaluation
//     with its Jacobian.
//   MIXED = true : for t < t_endgame the state, the RK4 stages and the Newton
//     iterations are complex FP32 and no FP64 instruction executes; for
//     t > t_endgame the state is FP64 and the corrector's residual H is
//     evaluated in double-float arithmetic -- in FP64 once a step of the
//     path has been rejected there -- while the Jacobian and the solve stay
//     FP32 (mixed precision iterative refinement, converged to the FP64
//     tolerance within max_newton_ir iterations: each contracts only
//     linearly, by about cond * 6e-8, so one exact Newton step is worth
//     about two); the final refinement and the backward error use
//     double-float residuals the same way (their error, about 2^-48 times
//     the backward-error scale, lies three orders below the refinement
//     target 1e-13 and five below the finite-root bound 1e-10).
//     A path whose FP32 steps fall below dt_min_fp32 (the corrector stalls
//     at the FP32 noise floor near an ill-conditioned stretch) or exhaust
//     max_steps_fp32 switches to that high-precision-residual mode at once.
//     GB300 issues FP64 FMAs at about 1/74 of its FP32 rate (measured), so
//     the residuals run on the FP32 pipe where their precision suffices.
//     Paths that still fail, paths whose endpoints collide (a path jump) and
//     endpoints whose FP32 condition estimate is suspect are re-tracked by
//     an FP64-state kernel (RE = df by default, settings.retrack_precision).
//
// Evaluator interface (HOM):
//   template <class R> eval(x[N], i, t, 1-t, row[N+1], H, Ht)
//       row[j] = dH_i/dx_j (j < N), H = H_i, Ht = dH_i/dt, all at (x, t)
//   residual64<SCALE>(xs, i, t, 1-t, H, scale)   H_i in FP64 at the point
//       xs[0..N) (shared memory), and with SCALE the backward-error
//       denominator sum |c| |x^a| of row i (FP64-state kernels)
//   residual_df<SCALE>(xs, i, t, H, scale)         the same in double-float
//       arithmetic, xs as double-floats, H rounded to FP32 (mixed kernels)
//   start(path, i)                                 start component x_i(0)
//   init(g)                                        per-path set-up (once per path)
// Evaluators read the point from the group's shared copy written by the
// tracker before every evaluation (vf for FP32, vd for FP64; the
// double-float evaluations split vd into their own copy vx) or from x[].
#pragma once

#include <type_traits>

#include "hc_device.cuh"
#include "kernels.cuh"

namespace hc {

template <int N, class S, class R>
__device__ __forceinline__ void load_vec(const cx<S>* buf, cx<R> (&x)[N]) {
#pragma unroll
  for (int k = 0; k < N; ++k) x[k] = cvt<R>(buf[k]);
}

// M_IDLE: a group without work waiting for the other groups of its warp
// (kernels with cooperative residuals, which keep the warp together)
enum : int { M_RK = 0, M_NEWTON = 1, M_REFINE = 2, M_COND = 3, M_DONE = 4, M_FETCH = 5, M_IDLE = 6 };

// Shared memory of one lane group: pv = two pivot-row buffers of the solve,
// acc = evaluator accumulators (term evaluator only), vd = high-precision
// copy of the evaluation point (complex FP64 in the all-FP64 kernels,
// double-floats in the mixed ones, 16 bytes per entry either way; written
// where a high-precision residual follows), sb = solution scatter buffer,
// vf = FP32 copy of the point.  vf and vd hold L + extra entries: the point
// occupies [0, N) and an evaluator may keep its own per-path values behind
// index L.  Size: group_smem_bytes (kernels.cuh).
struct GroupMem {
  unsigned char* pv;   // 32 (L + 2) bytes, 16-byte aligned
  unsigned char* acc;  // acc_bytes, 16-byte aligned
  cx<double>* vd;
  cx<double>* sb;  // holds L values of cx<R>
  cx<float>* vf;
  cx<double>* eg;  // FP64-state kernels: endgame samples [3][L] (previous sample,
                   // its dx/ds, the last prediction), 16-byte aligned
  cx<df>* vx;      // double-float kernels: the evaluator's double-float copy of
                   // vd (L + extra entries), 16-byte aligned; nullptr otherwise
  int stride;      // bytes from one group's memory to the next group's
};

template <int L>
__device__ __forceinline__ GroupMem make_group_mem(unsigned char* smem, int extra,
                                                   int acc_bytes = 0, int eg_bytes = 0,
                                                   int vx = 0) {
  const int stride = group_smem_bytes(L, extra, acc_bytes, eg_bytes, vx);
  unsigned char* b = smem + (threadIdx.x / L) * stride;
  GroupMem m;
  m.stride = stride;
  m.pv = b;
  b += 32 * (L + 2);
  m.acc = b;
  b += acc_bytes;
  m.eg = reinterpret_cast<cx<double>*>(b);
  b += eg_bytes;
  m.vx = vx ? reinterpret_cast<cx<df>*>(b) : nullptr;
  b += vx ? (L + extra) * 16 : 0;
  m.vd = reinterpret_cast<cx<double>*>(b);
  m.sb = reinterpret_cast<cx<double>*>(b + (L + extra) * 16);
  m.vf = reinterpret_cast<cx<float>*>(b + (L + extra) * 16 + L * 16);
  return m;
}

// Accesses to the resident launch's control words: the published tail and
// the stop word in device memory (written by copies on the host's staging
// stream), the completion flags in mapped host memory.
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int ld_relaxed_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// max over the group of a double (butterfly over the group's L lanes)
template <int L>
__device__ __forceinline__ double gmaxd(const Group& g, double v) {
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(g.mask, v, o));
  return v;
}

// Value at w = 0 of the cubic Hermite interpolant through (wb, xb, Db) and
// (wa, xa, Da), wb < wa (the power-series endgame's prediction).
__device__ __forceinline__ cx<double> hermite_at_zero(double wb, cx<double> xb, cx<double> Db,
                                                      double wa, cx<double> xa, cx<double> Da) {
  const double dl = wa - wb, tau = -wb / dl;
  const double t2 = tau * tau, t3 = t2 * tau;
  const double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + tau;
  const double h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
  return h00 * xb + (h10 * dl) * Db + h01 * xa + (h11 * dl) * Da;
}

// Persistent loop of one lane group over the work items of a launch.
// PROB::hom(inst) binds the evaluator to an instance.  RE: the arithmetic of
// the evaluation and the solve in the FP64-state kernels (MIXED = false):
// double, or df for the double-float kernels, whose state, step control,
// refinement residual and classification stay in FP64 exactly as in the
// FP64 kernels.  RING: the resident launch of a stream (hc_stream), whose
// items come from the host-filled ring (LaunchCommon ring_*); compiled only
// into the kernels the streams use.
template <int N, int L, bool MIXED, class PROB, class RE = double, bool RING = false>
__device__ __forceinline__ void run_tracker(const PROB& prob, const LaunchCommon& c,
                                            const Group& g, const GroupMem& sm) {
  using R = typename std::conditional<MIXED, float, RE>::type;
  using HOM = decltype(prob.hom(0));
  // double-float kernels: their Newton corrector takes its residual in FP64
  // once a step of the path has been rejected (before that, from the
  // double-float evaluation), as the mixed kernels' FP64-state phase does,
  // and always with the endgame, whose samples need FP64 accuracy
  constexpr bool XDF = std::is_same<R, df>::value;
  // Cooperative residuals (mixed kernels with several paths per warp, see
  // the dense evaluator): every high-precision residual the warp's groups
  // need in an iteration is computed by the whole warp at one point of the
  // loop (COOP).  The whole warp stays in the loop until all of its groups
  // are out of work (M_IDLE), and that point holds the loop's only
  // warp-wide synchronisation, so every lane meets every other lane there.
  // The resident-launch kernels (whose groups wait for tickets on their own)
  // compute the same partial sums in the same order group by group (EP).
  constexpr bool COOP_EVAL = MIXED && HOM::kCoop;
  constexpr bool COOP = COOP_EVAL && !RING;
  constexpr int EP = COOP_EVAL ? 32 / L : 1;
  const DevSettings& s = c.s;
  cx<R>* sb = reinterpret_cast<cx<R>*>(sm.sb);
  const bool act = g.gl < N;
  const int leader = g.wl & ~(L - 1);
  const int64_t total = c.count_dev ? (int64_t)(*c.count_dev) : c.n_items;

  const double tA = MIXED ? fmin(s.t_endgame, 1.0) : 1.0;  // end of the FP32 phase
  // FP32-state steps use the FP32 tier's tolerances; FP64-state steps (plain
  // FP64, or FP32 solves refined by FP64 residuals) use the FP64 ones.
  const float tol32 = (float)s.newton_tol_fp32, tol64 = (float)s.newton_tol;
  const float corr32 = (float)s.max_first_corr_fp32, corr64 = (float)s.max_first_corr;
  // Step control of the FP32 phase runs on FP32 copies of t, dt and the
  // limits: the FP64 pipe issues at a small fraction of the FP32 rate, so a
  // handful of FP64 bookkeeping instructions per evaluation would cost as
  // much issue time as the evaluation itself.  t is exact to FP32 rounding
  // there, far below the FP32 corrector's tolerance.
  const float tAf = (float)tA, dt_maxf = (float)s.dt_max, dt_min32f = (float)s.dt_min_fp32;
  const float rinf_f = (float)fmin(s.r_inf, 3.0e38);

  // ---- per-path state (identical control state in all lanes of the group)
  HOM hom = prob.hom(0);
  int64_t item = 0;
  int64_t inst_cur = 0;    // the instance of the group's path
  bool be_bad = false;     // COOP: the endpoint failed the backward-error test
  unsigned long long ticket = 0;  // resident launches: the claimed ticket
  (void)ticket;
  cx<double> xd = czero<double>();  // FP64 state
  cx<float> xf = czero<float>();    // FP32 state
  bool hi = !MIXED;                 // the state lives in xd rather than xf
  // t, dt, h, t1: FP64-state phase; tf, dtf, hf, t1f: FP32 phase
  double t = 0.0, dt = 0.0, h = 0.0, t1 = 0.0;
  float tf = 0.f, dtf = 0.f, hf = 0.f, t1f = 0.f;
  int consec = 0, nacc = 0, nrej = 0, nnewt = 0, status = 0;
  int mode = M_FETCH, stage = 0, it = 0;
  cx<R> kprev = czero<R>(), ksum = czero<R>();
  cx<float> xpf = czero<float>();   // corrector iterate (FP32 state)
  cx<double> xpd = czero<double>(); // corrector iterate (FP64 state)
  bool step_ok = true;
  bool first_fetch = true;
  // mixed kernels: the FP64-state corrector's residual runs in double-float
  // arithmetic until the path's first rejected FP64-state step, then in FP64
  bool res64 = false;
  float cond_inorm = 0.f, cond_anorm = 0.f, be = 0.f;
  // Power-series endgame (all-FP64 kernels, settings.endgame): the index and
  // s = 1 - t of the next sample, the s of the sample awaiting its dx/ds, the
  // samples taken, the cycle number of the last prediction, the previous
  // sample difference; landing: the current step ends on a sample; pending:
  // the point is a sample whose derivative the next RK stage 1 gives; have:
  // a prediction stands; sing: the endpoint came from a prediction with c > 1.
  int eg_next = 0, eg_count = 0, eg_c = 1;
  double eg_s = 0.0, eg_s_sample = 0.0, eg_dnprev = 0.0;
  bool eg_landing = false, eg_pending = false, eg_have = false, eg_sing = false;
  const bool eg_on = !MIXED && s.endgame != 0;
  auto eg_active = [&]() { return eg_on && eg_next < s.eg_samples; };

  cx<R> row[N + 1];
  cx<R> x[N];
  cx<R> sol[1];
  int col;

  // hi is constant true in the plain FP64 kernel; say so to the compiler
  auto HI = [&]() { return !MIXED || hi; };
  // this lane's entry of the high-precision point copy, as double-floats
  // (as_df) or complex FP64
  auto put_hi = [&](const cx<double>& v, bool as_df) {
    if (MIXED && as_df)
      reinterpret_cast<cdf*>(sm.vd)[g.gl] = to_cdf(v);
    else
      sm.vd[g.gl] = v;
  };
  auto begin_step = [&]() {
    if (HI()) {
      // with the endgame the step ends at the next sample time at the latest
      const bool ega = eg_active();
      const double target = ega ? 1.0 - eg_s : 1.0;
      const bool last = dt >= target - t;
      h = last ? target - t : dt;
      t1 = last ? target : t + h;
      eg_landing = last && ega;
    } else {
      // a step ending within FP32 rounding of the phase end takes the rest
      const bool last = 1.0001f * dtf >= tAf - tf;
      hf = last ? tAf - tf : dtf;
      t1f = last ? tAf : tf + hf;
    }
    stage = 0;
    ksum = czero<R>();
    kprev = czero<R>();
    step_ok = true;
    mode = M_RK;
  };
  // FP32 phase -> FP64-state phase at the current accepted point
  auto promote = [&](double dt_new) {
    xd = cvt<double>(xf);
    t = (double)tf;
    dt = dt_new;
    hi = true;
  };
  auto enter_refine = [&]() {
    if (!HI()) xd = cvt<double>(xf);
    hi = true;
    mode = M_REFINE;
    it = 0;
  };
  // the endgame's prediction (cycle number > 1) as the endpoint: no Newton
  // step (at a multiple root it divides rounding noise by rounding noise),
  // the backward error alone decides
  auto eg_finish = [&]() {
    xd = (g.gl < N) ? sm.eg[2 * L + g.gl] : czero<double>();
    t = 1.0;
    enter_refine();
    eg_sing = true;
  };
  // A sample at s = eg_s_sample: the point xd and dx/ds = -dxdt.  A
  // prediction is made only while the samples converge (the difference to
  // the previous sample shrinks, and the prediction lies within the tail
  // 4 |x_k - x_(k-1)| / (1 - h^(1/c)) of the sample); true once two successive
  // predictions with the same cycle number c > 1 agree within eg_tol (1 + |x|)
  // (paths with c = 1 end at nonsingular roots that ordinary tracking
  // reaches; a refinement from a misjudged c = 1 prediction next to a
  // multiple root could land anywhere).
  auto eg_sample = [&](cx<double> dxdt) -> bool {
    cx<double>* xa = sm.eg;
    cx<double>* da = sm.eg + L;
    cx<double>* pr = sm.eg + 2 * L;
    const cx<double> xk = act ? xd : czero<double>();
    const cx<double> dk = act ? -dxdt : czero<double>();
    bool done = false;
    if (eg_count >= 1) {
      const double dn = gmaxd<L>(g, act ? cabs2(xk - xa[g.gl]) : 0.0);
      bool predicted = false;
      if (eg_count >= 2 && dn > 0.0 && eg_dnprev > 0.0 && dn < eg_dnprev) {
        const double r = log(s.eg_ratio) / log(dn / eg_dnprev);
        const int cc = min(max((int)lround(r), 1), s.eg_cmax);
        const double sk = eg_s_sample, sa = sk / s.eg_ratio;
        const double wb = pow(sk, 1.0 / cc), wa = pow(sa, 1.0 / cc);
        const double fb = (double)cc * pow(wb, cc - 1), fa = (double)cc * pow(wa, cc - 1);
        const cx<double> P =
            act ? hermite_at_zero(wb, xk, fb * dk, wa, xa[g.gl], fa * da[g.gl]) : czero<double>();
        const double pn = gmaxd<L>(g, act ? cabs2(P) : 0.0);
        const double dx = gmaxd<L>(g, act ? cabs2(P - xk) : 0.0);
        const double dp = gmaxd<L>(g, (act && eg_have) ? cabs2(P - pr[g.gl]) : 0.0);
        const double tail = 4.0 * dn / (1.0 - pow(s.eg_ratio, 1.0 / cc));
        if (dx <= tail) {
          done = cc > 1 && eg_have && cc == eg_c && dp <= s.eg_tol * (1.0 + pn);
          if (act) pr[g.gl] = P;
          eg_c = cc;
          predicted = true;
        }
      }
      eg_have = predicted;
      eg_dnprev = dn;
    }
    if (act) {
      xa[g.gl] = xk;
      da[g.gl] = dk;
    }
    ++eg_count;
    __syncwarp(g.mask);
    return done;
  };
  auto reject = [&]() {
    ++nrej;
    consec = 0;
    if (HI()) {
      res64 = true;
      dt *= 0.5;
      if (dt < s.dt_min) {
        if (eg_on && eg_have && eg_c > 1) {  // inside the endgame the last prediction stands in
          eg_finish();
        } else {
          status = ST_FAIL_STEP;
          mode = M_DONE;
        }
      } else {
        begin_step();
      }
    } else {
      dtf *= 0.5f;
      if (dtf < dt_min32f) {
        // FP32 cannot resolve this stretch of the path (its corrector stalls
        // at the FP32 noise floor): continue from the last accepted point
        // with the FP64 state and FP64 residuals instead of failing the path.
        promote(s.dt_min_fp32);
      }
      begin_step();
    }
  };

#pragma unroll 1
  for (;;) {
    // ---- 0. retire the finished path and refill the group with the next one
    if (mode == M_DONE) {
      if (!hi) xd = cvt<double>(xf);
      if ((status & 0x7f) != ST_FINITE && status != ST_FAIL_NAN && gany(g, act && !cfinite(xd)))
        status = ST_FAIL_NAN;
      const int base = status & 0x7f;
      if (act) {
        reinterpret_cast<double2*>(c.x_out)[item * N + g.gl] = make_double2(xd.re, xd.im);
        // endpoint copy for duplicate detection: finite endpoints and those
        // whose FP32 condition estimate is suspect (a path that jumped onto
        // another path's root must not escape the check by that route)
        if (MIXED && c.x32_out)
          c.x32_out[item * N + g.gl] = (base == ST_FINITE || base == ST_SINGULAR)
                                           ? make_float2((float)xd.re, (float)xd.im)
                                           : make_float2(__int_as_float(0x7fc00000), 0.f);
      }
      if (g.gl == 0) {
        c.status_out[item] = (uint8_t)status;
        if (c.be_out) c.be_out[item] = (double)be;
        if (c.step_budget) atomicAdd(c.step_total, (unsigned long long)(nacc + nrej));
        if (MIXED) {
          c.steps_out[item * 3 + 0] = nacc;
          c.steps_out[item * 3 + 1] = nrej;
          c.steps_out[item * 3 + 2] = nnewt;
          if (c.esc_list && base != ST_FINITE) {
            // Step-size and budget failures (of the FP64-residual mode) and
            // suspect-condition endpoints go to the all-FP64 kernel, resuming
            // from the last accepted point (t = 1: refinement and exact
            // condition only).  Other failures of the FP32 tier (divergence,
            // non-finite state, failed refinement) are first re-tracked from
            // t = 0 with FP64 residuals, like colliding paths.
            const bool to64 = base == ST_FAIL_STEP || base == ST_FAIL_MAXSTEPS ||
                              base == ST_SINGULAR || c.start_hi || !c.dup_list;
            if (c.t_io)
              c.t_io[item] = (base == ST_FAIL_STEP || base == ST_FAIL_MAXSTEPS) ? (hi ? t : (double)tf)
                             : (base == ST_SINGULAR)                            ? 1.0
                                                                               : 0.0;
            // resident launches: per-slot lists of slot-relative items
            const int64_t slot = RING ? item / c.paths : 0;
            const int64_t rec = RING ? item - slot * c.paths : item;
            if (to64) {
              const unsigned long long pos = atomicAdd(c.esc_count + slot, 1ull);
              c.esc_list[slot * c.paths + pos] = rec;
            } else {
              const unsigned long long pos = atomicAdd(c.dup_count + slot, 1ull);
              c.dup_list[slot * c.paths + pos] = rec;
            }
          } else if (c.t_io) {
            c.t_io[item] = 0.0;
          }
        } else {
          c.steps_out[item * 3 + 0] += nacc;
          c.steps_out[item * 3 + 1] += nrej;
          c.steps_out[item * 3 + 2] += nnewt;
          if (c.esc_steps) {
            atomicAdd(c.esc_steps + 0, (unsigned long long)nacc);
            atomicAdd(c.esc_steps + 1, (unsigned long long)nrej);
            atomicAdd(c.esc_steps + 2, (unsigned long long)nnewt);
          }
        }
      }
      if constexpr (RING) {
        // the slot's last path tells the host (mapped memory) that the
        // slot's tracking launch work is complete
        __threadfence();
        __syncwarp(g.mask);
        if (g.gl == 0) {
          const int64_t slot = item / c.paths;
          const unsigned prev = atomicAdd(c.ring_done + slot, 1u);
          if ((int64_t)prev + 1 == c.paths) {
            atomicExch(c.ring_done + slot, 0u);
            __threadfence_system();
            st_release_sys(c.ring_flag + slot, ticket / c.ring_items + 1);
          }
        }
      }
      mode = M_FETCH;
    }
    if (RING && mode == M_FETCH) {
      // resident launch: claim the next published ticket, or sleep and poll
      // (bounded: the stop word or ring_idle_ns without work end the launch)
      unsigned long long q = 0;
      unsigned got = 0;
      if (g.gl == 0) {
        const unsigned long long t_wait = global_ns();
        unsigned sleep_ns = 500;
        for (;;) {
          if (ld_relaxed_gpu(c.ring_stop)) break;
          const unsigned long long pub = ld_acquire_gpu(c.ring_tail);
          const unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(c.queue);
          if (cur < pub) {
            if (atomicCAS(c.queue, cur, cur + 1) == cur) {
              q = cur;
              got = 1;
              break;
            }
            continue;
          }
          if (global_ns() - t_wait > c.ring_idle_ns) break;
          __nanosleep(sleep_ns);  // back off while there is no work
          sleep_ns = min(2u * sleep_ns, 32000u);
        }
      }
      if (!__shfl_sync(g.mask, got, leader)) break;
      ticket = __shfl_sync(g.mask, q, leader);
      (void)ld_acquire_gpu(c.ring_tail);  // every lane: the slot's inputs are visible
      item = (int64_t)(ticket % c.ring_items);
    }
    if (mode == M_FETCH) {
      bool stop = false;  // no further path for this group
      if (c.step_budget && !c.items) {
        // the budget stops new paths of the launch; started ones finish
        unsigned long long spent = 0;
        if (g.gl == 0) spent = *reinterpret_cast<volatile unsigned long long*>(c.step_total);
        stop = __shfl_sync(g.mask, spent, leader) >= c.step_budget;
      }
      unsigned long long q = 0;
      if (stop || RING) {
        // nothing to claim, or the item was claimed above
      } else if (c.spread && first_fetch) {
        // ticket = slot * blocks + block: consecutive items on different blocks
        // (and so, for the first blocks of the grid, on different SMs)
        q = (unsigned long long)(threadIdx.x / L) * gridDim.x + blockIdx.x;
        first_fetch = false;
      } else {
        if (g.gl == 0) q = atomicAdd(c.queue, 1ull);
        q = __shfl_sync(g.mask, q, leader);
        if (c.spread) q += (unsigned long long)gridDim.x * (blockDim.x / L);
      }
      if (!RING && !stop) stop = (int64_t)q >= total;
      if (stop) {
        if constexpr (COOP)
          mode = M_IDLE;
        else
          break;
      } else {
        if (!RING) item = c.items ? c.items[q] : (int64_t)q;
        const int64_t inst = item / c.paths;
        inst_cur = inst;
        const int64_t k_in = item - inst * c.paths;
        const int64_t path = c.path_ids ? c.path_ids[item] : c.path_map ? c.path_map[k_in] : k_in;
        hom = prob.hom(inst);
        hom.init(g);  // per-path constants of the evaluator (shared memory)
        // a path handed over by the FP32 tier resumes from its last accepted point
        const double t0 = (!MIXED && c.t_io) ? c.t_io[item] : 0.0;
        __syncwarp(g.mask);
        xd = czero<double>();
        if (act) {
          if (t0 > 0.0) {
            const double2 v = reinterpret_cast<const double2*>(c.x_out)[item * N + g.gl];
            xd = mk<double>(v.x, v.y);
          } else {
            xd = hom.start(path, g.gl);
          }
        }
        xf = cvt<float>(xd);
        hi = !MIXED || c.start_hi;
        t = t0 > 0.0 ? t0 : 0.0;
        dt = s.dt_init;
        tf = (float)t;
        dtf = (float)s.dt_init;
        consec = nacc = nrej = nnewt = status = 0;
        res64 = false;
        be = 0.f;
        // endgame: the first sample time after the start point
        eg_count = 0;
        eg_c = 1;
        eg_dnprev = 0.0;
        eg_landing = eg_pending = eg_have = eg_sing = false;
        eg_next = 0;
        eg_s = s.eg_s0;
        if (eg_on)
          while (eg_next < s.eg_samples && 1.0 - eg_s <= t) {
            eg_s *= s.eg_ratio;
            ++eg_next;
          }
        if (t >= 1.0)
          enter_refine();
        else
          begin_step();
      }
    }
    if (mode == M_RK && stage == 0) {
      if (nacc + nrej >= s.max_steps) {
        status = ST_FAIL_MAXSTEPS;
        mode = M_DONE;
        continue;
      }
      if (!HI() && nacc + nrej >= s.max_steps_fp32) {  // FP32 step budget spent
        promote((double)dtf);
        begin_step();
      }
    }

    // ---- 1. evaluation point and time (FP32 arithmetic in the FP32 phase)
    double te = 1.0;      // FP64-state phases
    R ter = R(1), omt = R(0);  // the time the evaluator sees, and 1 - t
    bool need64 = false;
    // COOP: the residual this group needs at te (0 none, 1 double-float,
    // 2 FP64, 3 double-float with the backward-error scale)
    int res_code = 0;
    if (mode == M_RK) {
      if (HI()) {
        const double cst = (stage == 0) ? 0.0 : (stage == 3 ? 1.0 : 0.5);
        te = (stage == 3) ? t1 : t + cst * h;
        ter = (R)te;
        omt = (R)(1.0 - te);
        const cx<double> p = xd + (cst * h) * cvt<double>(kprev);
        if (!MIXED && act) sm.vd[g.gl] = p;  // the FP32 evaluation reads vf only
        if (act) sm.vf[g.gl] = cvt<float>(p);
      } else {
        const float cst = (stage == 0) ? 0.f : (stage == 3 ? 1.f : 0.5f);
        const float tt = (stage == 3) ? t1f : tf + cst * hf;
        ter = (R)tt;
        omt = (R)(1.f - tt);
        const cx<float> p = xf + (cst * hf) * cvt<float>(kprev);
        if (act) sm.vf[g.gl] = p;
      }
    } else if (mode == M_NEWTON) {
      if (HI()) {
        te = t1;
        ter = (R)t1;
        omt = (R)(1.0 - t1);
        need64 = MIXED || (XDF && (res64 || eg_on));
        if (MIXED) res_code = res64 ? 2 : 1;
        if (act) put_hi(xpd, !res64);
        if (act) sm.vf[g.gl] = cvt<float>(xpd);
      } else {
        ter = (R)t1f;
        omt = (R)(1.f - t1f);
        if (act) sm.vf[g.gl] = xpf;
      }
    } else {  // M_REFINE, M_COND (M_IDLE: nothing to evaluate): at the endpoint, t = 1
      need64 = (mode == M_REFINE);
      // COOP: the backward error of a refined endpoint comes with the first
      // condition pass (the same point)
      const bool be_now = COOP && mode == M_COND && stage == 0;
      if (act && (need64 || be_now || !MIXED)) put_hi(xd, MIXED);
      if (MIXED) res_code = need64 ? 1 : be_now ? 3 : 0;
      if (act) sm.vf[g.gl] = cvt<float>(xd);
    }
    __syncwarp(g.mask);
    if constexpr (MIXED) {
      load_vec<N, float, float>(sm.vf, x);
    } else {
      load_vec<N, double, R>(sm.vd, x);
    }

    if constexpr (COOP) {
      // The loop's one warp-wide meeting point: leave together once every
      // group is idle, else compute the groups' residuals one group at a
      // time with all lanes of the warp.  A lane of the group served keeps
      // its row's residual (FP32-rounded) and scale in its own entry of the
      // group's scatter buffer, which is free until the solve.
      const unsigned live = __ballot_sync(0xffffffffu, g.gl == 0 && mode != M_IDLE);
      if (live == 0u) break;
      const unsigned want = __ballot_sync(0xffffffffu, g.gl == 0 && res_code != 0);
      if (want != 0u) {
        __syncwarp(0xffffffffu);  // the groups' point copies, before other groups read them
        unsigned rem = want;
        while (rem != 0u) {
          const int src = __ffs(rem) - 1;  // leader lane of the group served
          rem &= rem - 1u;
          const int code = __shfl_sync(0xffffffffu, res_code, src);
          const double tG = __shfl_sync(0xffffffffu, te, src);
          const long long iG = __shfl_sync(0xffffffffu, (long long)inst_cur, src);
          const HOM hG = prob.hom((int64_t)iG);
          const unsigned char* vdG =
              reinterpret_cast<const unsigned char*>(sm.vd) + (src / L - g.wl / L) * sm.stride;
          cx<float> hf;
          float scf = 0.f;
          if (code == 2) {
            cx<double> h64;
            double sc64;
            hG.residual64_coop(reinterpret_cast<const cx<double>*>(vdG), g.wl, tG, false, h64,
                               sc64);
            hf = cvt<float>(h64);
          } else {
            hG.residual_df_coop(reinterpret_cast<const cdf*>(vdG), g.wl, tG, code == 3, hf, scf);
          }
          if ((g.wl / L) == (src / L))
            reinterpret_cast<float4*>(sm.sb)[g.gl] = make_float4(hf.re, hf.im, scf, 0.f);
        }
        __syncwarp(0xffffffffu);  // every read of the point copies done
      }
      if (res_code == 3) {  // backward error of the refined endpoint
        const float4 v = reinterpret_cast<const float4*>(sm.sb)[g.gl];
        const double r = (double)cabs2(mk<float>(v.x, v.y)), sc = (double)v.z;
        const double bei = act ? (sc > 0.0 ? r / sc : r) : 0.0;
        be = gmaxf(g, (float)bei);
        be_bad = !((double)be <= s.finite_tol);
      }
    }

    // ---- 2. row i of [dH/dx | rhs] and the solve
    {
      cx<R> H, Ht;
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
        // unit vector e_stage (on every replica of row stage)
        const int grow = g.gl & (HOM::ROWL - 1);
        row[N] = mk<R>((grow < N && grow == stage) ? R(1) : R(0), R(0));
      } else if (need64) {
        if constexpr (COOP) {
          const float4 v = reinterpret_cast<const float4*>(sm.sb)[g.gl];
          row[N] = mk<R>(-v.x, -v.y);
        } else if (MIXED && (mode == M_REFINE || !res64)) {
          cx<float> Hf;
          float sc;
          hom.template residual_df<false, EP>(reinterpret_cast<const cdf*>(sm.vd), g.gl, te, Hf,
                                              sc);
          row[N] = cvt<R>(-Hf);
        } else {
          cx<double> H64;
          double sc;
          hom.template residual64<false, EP>(sm.vd, g.gl, te, 1.0 - te, H64, sc);
          row[N] = cvt<R>(-H64);
        }
      } else {
        row[N] = -H;
      }
    }
    bool sok;
    if constexpr (HOM::PARTS > 1)
      sok = gj_solve_parts<N, R, HOM::ROWL, HOM::PARTS>(g, row, sol, col,
                                                       reinterpret_cast<cx<R>*>(sm.pv),
                                                       reinterpret_cast<cx<R>*>(sm.sb));
    else
      sok = gj_solve<N, 1, R>(g, row, sol, col, reinterpret_cast<cx<R>*>(sm.pv));
    if (col >= 0) sb[col] = sol[0];
    __syncwarp(g.mask);
    const cx<R> d = act ? sb[g.gl] : czero<R>();

    // ---- 3. state machine
    if (mode == M_RK) {
      if constexpr (!MIXED) {
        // stage 1 at a sample point gives its dx/dt
        if (stage == 0 && eg_pending) {
          eg_pending = false;
          if (sok && eg_sample(cvt<double>(d))) {
            eg_finish();
            continue;
          }
        }
      }
      step_ok = step_ok && sok;
      kprev = d;
      ksum = ksum + ((stage == 0 || stage == 3) ? R(1) : R(2)) * d;
      if (++stage == 4) {
        if (!step_ok) {
          reject();
        } else {
          if (HI())
            xpd = xd + (h / 6.0) * cvt<double>(ksum);
          else
            xpf = xf + (hf / 6.0f) * cvt<float>(ksum);
          mode = M_NEWTON;
          it = 0;
        }
      }
    } else if (mode == M_NEWTON) {
      float xn2;
      if (HI()) {
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
                       (it == 0 && dn > (HI() ? corr64 : corr32) * (1.f + xn));
      if (!bad && dn <= (HI() ? tol64 : tol32) * (1.f + xn)) {
        // accept the step
        bool at_end;
        ++nacc;
        const bool grow = ++consec >= s.grow_after;
        if (grow) consec = 0;
        if (HI()) {
          xd = xpd;
          t = t1;
          if (grow) dt = fmin(2.0 * dt, s.dt_max);
          at_end = t >= 1.0;
        } else {
          xf = xpf;
          tf = t1f;
          if (grow) dtf = fminf(2.f * dtf, dt_maxf);
          at_end = tf >= 1.f;
        }
        if (xn > rinf_f) {
          status = ST_DIVERGED;
          mode = M_DONE;
        } else if (at_end) {
          enter_refine();
        } else {
          if (!HI() && tf >= tAf) promote((double)dtf);  // enter the FP64-state phase
          if (eg_on && eg_landing) {  // the step ended on a sample time
            eg_pending = true;
            eg_s_sample = eg_s;
            eg_s *= s.eg_ratio;
            ++eg_next;
          }
          begin_step();
        }
      } else if (bad || ++it >= ((MIXED && HI()) ? s.max_newton_ir : s.max_newton)) {
        reject();
      }
    } else if (mode == M_REFINE) {
      const cx<double> xnew = xd + cvt<double>(d);
      const float dn = sqrt_approx(gmaxf(g, act ? (float)cnorm2(d) : 0.f));
      const float xnn = sqrt_approx(gmaxf(g, act ? cnorm2(cvt<float>(xnew)) : 0.f));
      const bool bad = !sok || !(dn <= 3.0e38f) || !(xnn <= 3.0e38f);
      if (!bad && !eg_sing) xd = xnew;
      if (bad || eg_sing || dn <= (float)s.refine_tol * (1.f + xnn) || ++it >= s.refine_iters) {
        // classify: finiteness, divergence, backward error (FP64 residual)
        const bool fin = !gany(g, act && !cfinite(xd));
        const float xnf = gmaxf(g, act ? cabs2(cvt<float>(xd)) : 0.f);
        if (!fin) {
          status = ST_FAIL_NAN;
          mode = M_DONE;
        } else if (xnf > rinf_f) {
          status = ST_DIVERGED;
          mode = M_DONE;
        } else if constexpr (COOP) {
          mode = M_COND;  // the backward error comes with the first condition pass
          stage = 0;
          cond_inorm = 0.f;
        } else {
          __syncwarp(g.mask);
          if (act) put_hi(xd, MIXED);
          __syncwarp(g.mask);
          double r, sc;
          if constexpr (MIXED) {  // double-float residual: its error is ~2^-48 sc
            cx<float> Hf;
            float scf;
            hom.template residual_df<true, EP>(reinterpret_cast<const cdf*>(sm.vd), g.gl, 1.0,
                                               Hf, scf);
            r = (double)cabs2(Hf);
            sc = (double)scf;
          } else {
            cx<double> H64;
            hom.template residual64<true>(sm.vd, g.gl, 1.0, 0.0, H64, sc);
            r = (double)cabs2(cvt<float>(H64));
          }
          const double bei = act ? (sc > 0.0 ? r / sc : r) : 0.0;
          be = gmaxf(g, (float)bei);
          if (!((double)be <= s.finite_tol)) {
            status = ST_FAIL_REFINE;
            mode = M_DONE;
          } else if (eg_sing) {  // cycle number > 1: a singular root
            status = ST_SINGULAR;
            mode = M_DONE;
          } else {
            mode = M_COND;  // condition number: one solve per column of the inverse
            stage = 0;
            cond_inorm = 0.f;
          }
        }
      }
    } else if (mode == M_COND && COOP && stage == 0 && be_bad) {
      status = ST_FAIL_REFINE;  // the refined endpoint failed the backward-error test
      mode = M_DONE;
    } else if (mode == M_COND) {
      if (!sok) cond_inorm = INFINITY;
      cond_inorm =
          fmaxf(cond_inorm, gsum<L, float>(g, (act && col >= 0) ? cabs2(cvt<float>(d)) : 0.f));
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
}

}  // namespace hc
