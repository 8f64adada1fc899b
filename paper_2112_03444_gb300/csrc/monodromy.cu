// Monodromy solving on the GPU: all isolated solutions of a parameterised
// family F(x; p) at a generic parameter point p0, from one seed solution.
//
// The paper (Sec. 7) obtains the start systems of its vision problems from
// the monodromy module of Macaulay2 at a generic complex point.  Here the
// same method runs with this library's tracker: starting from the known
// solutions S at p0, every solution is carried around triangle loops
// p0 -> pa -> pb -> p0 through random complex parameter points (parameter
// homotopies, each leg one hc_track_batch); the endpoints that are not yet
// in S are new solutions of F(x; p0).  Each round runs several independent
// loops (the first leg of all of them in one batch, one instance per loop),
// and the search stops after stall_loops consecutive loops without a new
// solution.  With sign symmetries in the family, every new solution's sign
// images are added as well, and the legs track one start per orbit.
//
// The host work between legs -- drawing the loop points, collecting
// endpoints and matching them against S -- is O(|S| log |S|) per round;
// every path is tracked on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "hc.h"
#include "kernels.cuh"

namespace {

// splitmix64 (Steele, Lea and Flood, OOPSLA 2014): the loop points' generator
struct SplitMix {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  // a standard complex normal number (Box-Muller), re and im ~ N(0, 1)
  void cnormal(double* z) {
    const double r = std::sqrt(-2.0 * std::log(uniform())), th = 6.283185307179586 * uniform();
    z[0] = r * std::cos(th);
    z[1] = r * std::sin(th);
  }
};

// A set of points of C^n with lookup to a relative tolerance.
struct PointSet {
  int n;
  double tol;
  std::vector<double> pts;                        // [count][n][2]
  std::vector<std::pair<double, int64_t>> index;  // sorted by key
  double key(const double* x) const {
    double v = 0.0;
    for (int j = 0; j < n; ++j) v += (1.0 + 0.37 * j) * (x[2 * j] + 0.61 * x[2 * j + 1]);
    return v;
  }
  double wsum() const {
    double w = 0.0;
    for (int j = 0; j < n; ++j) w += 1.61 * (1.0 + 0.37 * j);
    return w;
  }
  int64_t size() const { return (int64_t)(pts.size() / (2 * n)); }
  bool contains(const double* y) const {
    double ymax = 1.0;
    for (int j = 0; j < 2 * n; ++j) ymax = std::max(ymax, std::fabs(y[j]));
    const double t = tol * ymax, ky = key(y), kt = 2.0 * t * wsum();
    auto it = std::lower_bound(index.begin(), index.end(), std::make_pair(ky - kt, (int64_t)-1));
    for (; it != index.end() && it->first <= ky + kt; ++it) {
      const double* x = pts.data() + 2 * n * it->second;
      bool same = true;
      for (int j = 0; j < 2 * n && same; ++j) same = std::fabs(x[j] - y[j]) <= t;
      if (same) return true;
    }
    return false;
  }
  void add(const double* y) {
    const int64_t id = size();
    pts.insert(pts.end(), y, y + 2 * n);
    const auto e = std::make_pair(key(y), id);
    index.insert(std::upper_bound(index.begin(), index.end(), e), e);
  }
};

// Tracks `starts` (count x n complex) of the family from p_from to each of
// the n_targets parameter vectors; returns per target the finite endpoints.
hc_status track_leg(const hc_problem_desc& fam, const double* p_from, const std::vector<double>& starts,
                    const double* targets, int n_targets, bool use_sym,
                    std::vector<std::vector<double>>& out, int64_t& tracked) {
  const int n = fam.n;
  const int64_t S = (int64_t)(starts.size() / (2 * n));
  out.assign(n_targets, {});
  if (S == 0) return HC_OK;
  hc_problem_desc d = fam;
  d.p0 = p_from;
  d.start = starts.data();
  d.n_start = S;
  if (!use_sym) d.n_sym = 0;
  hc_problem* pr = nullptr;
  hc_status rc = hc_create_problem(&d, &pr);
  if (rc != HC_OK) return rc;
  std::vector<double> x((size_t)n_targets * S * n * 2);
  std::vector<uint8_t> st((size_t)n_targets * S);
  hc_batch_desc b;
  std::memset(&b, 0, sizeof(b));
  b.n_instances = n_targets;
  b.p1 = targets;
  b.x_out = x.data();
  b.status_out = st.data();
  hc_batch* bt = nullptr;
  rc = hc_track_batch(pr, &b, &bt);
  if (rc == HC_OK) {
    rc = hc_poll(bt, -1, nullptr);
    hc_destroy(bt);
  }
  hc_destroy(pr);
  if (rc != HC_OK) return rc;
  tracked += (int64_t)n_targets * S;
  for (int k = 0; k < n_targets; ++k)
    for (int64_t s = 0; s < S; ++s)
      if ((st[(size_t)k * S + s] & 0x7f) == HC_PATH_FINITE) {
        const double* xp = x.data() + ((size_t)k * S + s) * n * 2;
        out[k].insert(out[k].end(), xp, xp + 2 * n);
      }
  return HC_OK;
}

}  // namespace

extern "C" hc_status hc_monodromy_solve(const hc_monodromy_desc* d, int64_t* n_solutions,
                                        hc_monodromy_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!d || !d->family || !d->x0 || !d->p0 || !d->out || !n_solutions ||
      (d->family->kind != HC_PARAMETER && d->family->kind != HC_COEFFICIENT) ||
      d->family->n < 1 || d->family->n_params < 1 ||
      d->stall_loops < 1 || d->max_loops < 1 || d->loops_per_round < 1 ||
      d->max_solutions < 1 || d->reserved != 0) {
    hc::set_last_error("hc_monodromy_solve: invalid descriptor");
    return HC_ERR_INVALID;
  }
  const hc_problem_desc& fam = *d->family;
  const int n = fam.n, P = fam.n_params, K = d->loops_per_round;
  if (fam.n_sym < 0 || fam.n_sym > 4) {
    hc::set_last_error("hc_monodromy_solve: n_sym must be 0..4");
    return HC_ERR_INVALID;
  }
  std::vector<uint32_t> group(1u << fam.n_sym, 0u);
  for (size_t e = 0; e < group.size(); ++e)
    for (int k = 0; k < fam.n_sym; ++k)
      if (e >> k & 1) group[e] ^= fam.sym_mask[k];
  PointSet S{n, 1e-6, {}, {}};
  auto add_with_images = [&](const double* y) -> int {
    int added = 0;
    std::vector<double> img(2 * n);
    for (uint32_t m : group) {
      for (int j = 0; j < n; ++j) {
        const double sg = (m >> j & 1u) ? -1.0 : 1.0;
        img[2 * j] = sg * y[2 * j];
        img[2 * j + 1] = sg * y[2 * j + 1];
      }
      if (!S.contains(img.data())) {
        S.add(img.data());
        ++added;
      }
    }
    return added;
  };
  add_with_images(d->x0);
  SplitMix rng{d->seed ^ 0x6D6F6E6F64726F6Dull};
  int64_t tracked = 0;
  int loops = 0, stall = 0, rounds = 0;
  std::vector<double> pa((size_t)K * P * 2), pb((size_t)K * P * 2);
  std::vector<std::vector<double>> X1, X2, X3;
  while (stall < d->stall_loops && loops < d->max_loops) {
    for (size_t i = 0; i < pa.size(); i += 2) rng.cnormal(&pa[i]);
    for (size_t i = 0; i < pb.size(); i += 2) rng.cnormal(&pb[i]);
    hc_status rc;
    // leg 1 of every loop in one batch: p0 -> pa[k]
    if ((rc = track_leg(fam, d->p0, S.pts, pa.data(), K, true, X1, tracked)) != HC_OK) return rc;
    int new_this_round = 0;
    for (int k = 0; k < K; ++k) {
      // leg 2: pa[k] -> pb[k], leg 3: pb[k] -> p0
      if ((rc = track_leg(fam, &pa[(size_t)k * P * 2], X1[k], &pb[(size_t)k * P * 2], 1, true, X2,
                          tracked)) != HC_OK)
        return rc;
      if ((rc = track_leg(fam, &pb[(size_t)k * P * 2], X2[0], d->p0, 1, true, X3, tracked)) !=
          HC_OK)
        return rc;
      int added = 0;
      for (size_t i = 0; i < X3[0].size(); i += 2 * n) added += add_with_images(&X3[0][i]);
      new_this_round += added;
      ++loops;
      stall = added ? 0 : stall + 1;
    }
    ++rounds;
    if (S.size() > d->max_solutions) break;
    (void)new_this_round;
  }
  *n_solutions = S.size();
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->loops = loops;
    info->rounds = rounds;
    info->paths_tracked = tracked;
    info->seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (S.size() > d->max_solutions) {
    hc::set_last_error("hc_monodromy_solve: more solutions than max_solutions");
    return HC_ERR_INVALID;
  }
  std::memcpy(d->out, S.pts.data(), sizeof(double) * S.pts.size());
  return HC_OK;
}
