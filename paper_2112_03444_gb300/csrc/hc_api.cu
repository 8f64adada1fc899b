// Host runtime behind the C-ABI of include/hc.h: problem validation and
// encoding, device staging, persistent tracking launches, FP64 escalation of
// failed mixed-precision paths, result summary and the asynchronous poll.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "hc.h"
#include "kernels.cuh"

namespace hc {
KernelRef dense_ref_d2_64(int n, int lanes);
KernelRef dense_ref_d2_32(int n, int lanes);
KernelRef dense_ref_d3_64(int n, int lanes);
KernelRef dense_ref_d3_32(int n, int lanes);

KernelRef dense_ref_d2_df(int n);
KernelRef dense_ref_d3_df(int n);

KernelRef term_ref_64(int n, int lanes);
KernelRef term_ref_32(int n, int lanes);
KernelRef term_ref_df(int n);

// The double-float kernels come in one width each: one path per warp for
// dense systems, the default width for term tables.
KernelRef term_kernel(int n, int prec, int lanes) {
  if (prec == HC_PREC_DF) return term_ref_df(n);
  return prec == HC_PREC_MIXED ? term_ref_32(n, lanes) : term_ref_64(n, lanes);
}

KernelRef dense_kernel(int deg, int n, int prec, int lanes) {
  const bool mixed = prec == HC_PREC_MIXED;
  if (prec == HC_PREC_DF) {
    if (deg == 2) return dense_ref_d2_df(n);
    if (deg == 3) return dense_ref_d3_df(n);
    return KernelRef{nullptr, 0};
  }
  if (deg == 2) return mixed ? dense_ref_d2_32(n, lanes) : dense_ref_d2_64(n, lanes);
  if (deg == 3) return mixed ? dense_ref_d3_32(n, lanes) : dense_ref_d3_64(n, lanes);
  return KernelRef{nullptr, 0};
}
}  // namespace hc

using hc::cx;

namespace {

constexpr uint32_t kProblemMagic = 0x48435042u;  // "HCPB"
constexpr uint32_t kBatchMagic = 0x48434254u;    // "HCBT"

thread_local std::string g_err;

void set_err(const std::string& s) { g_err = s; }

#define HC_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_err(std::string(#call) + ": " + cudaGetErrorString(e_));                 \
      return e_ == cudaErrorMemoryAllocation ? HC_ERR_OOM : HC_ERR_CUDA;           \
    }                                                                              \
  } while (0)

// ------------------------------------------------------------------ kernels
__global__ void stage_dense_kernel(int64_t n_inst, int T, const double2* __restrict__ coef,
                                   int64_t coef_stride, const int* __restrict__ emap, int ndc,
                                   const int* __restrict__ dterm, const int* __restrict__ dslot,
                                   const float* __restrict__ dmult, double2* E, hc::cdf* Edf,
                                   int64_t Es, float2* D32, double2* D64, float4* Ddf,
                                   int64_t Ds) {
  const int64_t per = (int64_t)T + ndc;
  const int64_t total = n_inst * per;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < total;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t inst = w / per;
    int64_t r = w - inst * per;
    const double2* c = coef + inst * coef_stride;
    if (r < T) {
      E[inst * Es + emap[r]] = c[r];
      if (Edf) Edf[inst * Es + emap[r]] = hc::to_cdf(cx<double>{c[r].x, c[r].y});
    } else {
      r -= T;
      const double2 v = c[dterm[r]];
      const double m = (double)dmult[r];
      const double2 dv = make_double2(m * v.x, m * v.y);
      if (D64) D64[inst * Ds + dslot[r]] = dv;
      if (D32) D32[inst * Ds + dslot[r]] = make_float2((float)dv.x, (float)dv.y);
      if (Ddf) {  // cx<df> layout: re hi, re lo, im hi, im lo
        const hc::df re(dv.x), im(dv.y);
        Ddf[inst * Ds + dslot[r]] = make_float4(re.hi, re.lo, im.hi, im.lo);
      }
    }
  }
}

// Duplicate endpoints within an instance (path jumping): an item whose FP32
// endpoint copy lies within tol (relative, inf-norm) of another item's gets
// resume time 0 and is appended to out_list -- unless its status is
// singular: the tracking kernel has already queued such an endpoint for the
// all-FP64 tier, which then re-tracks it from t = 0 instead of only checking
// it at t = 1.  list == nullptr checks every item; otherwise only the
// *list_count items of list (endpoints that were re-tracked), against every
// item of their instance.  One thread per item scans the other items of its
// instance; x32 holds NaN for paths that did not end finite, which then
// never match.  With sign symmetries (n_group > 1) the items are orbit
// representatives and an endpoint is compared with every sign image of the
// others (group[e]: the unknowns element e negates).
__global__ void dedupe_kernel(int64_t items, int64_t paths, int n, const float2* __restrict__ x32,
                              const uint8_t* __restrict__ status, float tol,
                              const int64_t* __restrict__ list,
                              const unsigned long long* list_count, int64_t* out_list,
                              unsigned long long* out_count, double* t_io, int n_group,
                              const uint32_t* __restrict__ group) {
  const int64_t total = list ? (int64_t)*list_count : items;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = list ? list[idx] : idx;
    const float2* xa = x32 + a * n;
    const float2 v0 = xa[0];
    if (isnan(v0.x)) continue;
    float sc = 1.f;
    for (int k = 0; k < n; ++k) sc = fmaxf(sc, fmaxf(fabsf(xa[k].x), fabsf(xa[k].y)));
    const float thr = tol * sc;
    const int64_t b0 = (a / paths) * paths;
    bool dup = false;
    for (int64_t b = b0; b < b0 + paths && !dup; ++b) {
      if (b == a) continue;
      const float2* xb = x32 + b * n;
      for (int e = 0; e < n_group && !dup; ++e) {  // b's endpoint and its sign images
        const uint32_t m = group ? group[e] : 0u;
        const float s0 = (m & 1u) ? -1.f : 1.f;
        const float2 w = xb[0];
        if (!(fabsf(s0 * w.x - v0.x) <= thr) || !(fabsf(s0 * w.y - v0.y) <= thr)) continue;
        bool same = true;
        for (int k = 1; k < n && same; ++k) {
          const float sk = (m >> k & 1u) ? -1.f : 1.f;
          const float2 p = xa[k], q = xb[k];
          same = (fabsf(p.x - sk * q.x) <= thr) && (fabsf(p.y - sk * q.y) <= thr);
        }
        dup = same;
      }
    }
    if (dup) {
      t_io[a] = 0.0;
      if ((status[a] & 0x7f) != HC_PATH_SINGULAR) {
        const unsigned long long pos = atomicAdd(out_count, 1ull);
        out_list[pos] = a;
      }
    }
  }
}

// The same check for the *list_count listed items only, one warp per item
// (the lanes split the scan of its instance): a few re-tracked endpoints
// against every endpoint of their instance.
__global__ void dedupe_list_kernel(int64_t paths, int n, const float2* __restrict__ x32,
                                   const uint8_t* __restrict__ status, float tol,
                                   const int64_t* __restrict__ list,
                                   const unsigned long long* list_count, int64_t* out_list,
                                   unsigned long long* out_count, double* t_io, int n_group,
                                   const uint32_t* __restrict__ group) {
  const int lane = threadIdx.x & 31;
  const int64_t total = (int64_t)*list_count;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
  for (int64_t w = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32; w < total;
       w += warps) {
    const int64_t a = list[w];
    const float2* xa = x32 + a * n;
    if (isnan(xa[0].x)) continue;  // uniform over the warp
    float sc = 1.f;
    for (int k = 0; k < n; ++k) sc = fmaxf(sc, fmaxf(fabsf(xa[k].x), fabsf(xa[k].y)));
    const float thr = tol * sc;
    const int64_t b0 = (a / paths) * paths;
    bool dup = false;
    for (int64_t b = b0 + lane; b < b0 + paths && !dup; b += 32) {
      if (b == a) continue;
      const float2* xb = x32 + b * n;
      for (int e = 0; e < n_group && !dup; ++e) {
        const uint32_t m = group ? group[e] : 0u;
        bool same = true;
        for (int k = 0; k < n && same; ++k) {
          const float sk = (m >> k & 1u) ? -1.f : 1.f;
          const float2 p = xa[k], q = xb[k];
          same = (fabsf(p.x - sk * q.x) <= thr) && (fabsf(p.y - sk * q.y) <= thr);
        }
        dup = same;
      }
    }
    if (__any_sync(0xffffffffu, dup) && lane == 0) {
      t_io[a] = 0.0;
      if ((status[a] & 0x7f) != HC_PATH_SINGULAR) {
        const unsigned long long pos = atomicAdd(out_count, 1ull);
        out_list[pos] = a;
      }
    }
  }
}

// Batch summary: [0] finite [1] real [2] diverged [3] singular [4] failed
// [5] accepted steps [6] rejected steps [7] Newton iterations; untracked
// paths (HC_PATH_NONE) are counted in *untracked as well as in [4]
// Step counters are summed over the step_items tracked items (with sign
// symmetries the orbit representatives: the work done), statuses over the
// items of the output.
__global__ void summarize_kernel(int64_t items, const uint8_t* __restrict__ st,
                                 int64_t step_items, const int32_t* __restrict__ steps,
                                 unsigned long long* out, unsigned long long* untracked) {
  unsigned long long c[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t lim = items > step_items ? items : step_items;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < lim;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < items) {
      const int s = st[i];
      const int b = s & 0x7f;
      c[0] += (b == hc::ST_FINITE);
      c[1] += (b == hc::ST_FINITE) && (s & hc::ST_REAL);
      c[2] += (b == hc::ST_DIVERGED);
      c[3] += (b == hc::ST_SINGULAR);
      c[4] += (b != hc::ST_FINITE && b != hc::ST_DIVERGED && b != hc::ST_SINGULAR);
      c[8] += (s == 0);
    }
    if (i < step_items) {
      c[5] += (unsigned)steps[i * 3 + 0];
      c[6] += (unsigned)steps[i * 3 + 1];
      c[7] += (unsigned)steps[i * 3 + 2];
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    unsigned long long v = c[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(k < 8 ? out + k : untracked, v);
  }
}

// Coefficient interpolation (HC_COEFFICIENT): per instance and (slot, row)
// of the term tables, dc = c(p1) - c(p0), c(p) the slot's coefficient times
// its parameter factors at p (cpar, -1: none), in FP64, FP32 and
// double-float.  One thread per entry.
__global__ void stage_coef_kernel(int64_t n_inst, int64_t slots, int mp,
                                  const int32_t* __restrict__ cpar,
                                  const double2* __restrict__ s64, const double2* __restrict__ c0,
                                  const double2* __restrict__ p1, int P, double2* dc, float2* dcf,
                                  hc::cdf* dcdf) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n_inst * slots;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t inst = w / slots, k = w - inst * slots;
    double re = s64[k].x, im = s64[k].y;
    for (int f = 0; f < mp; ++f) {
      const int l = cpar[k * mp + f];
      if (l < 0) continue;
      const double2 v = p1[inst * P + l];
      const double nr = re * v.x - im * v.y, ni = re * v.y + im * v.x;
      re = nr;
      im = ni;
    }
    const double2 d = make_double2(re - c0[k].x, im - c0[k].y);
    dc[w] = d;
    dcf[w] = make_float2((float)d.x, (float)d.y);
    dcdf[w] = hc::to_cdf(cx<double>{d.x, d.y});
  }
}

// Outputs of a batch tracked on orbit representatives (sign symmetries):
// start j of instance i takes its representative's results, the unknowns of
// group[sign[j]] negated.  One thread per output item.
__global__ void expand_orbits_kernel(int64_t items, int64_t paths, int64_t n_rep, int n,
                                     const int32_t* __restrict__ rep_pos,
                                     const uint8_t* __restrict__ sign,
                                     const uint32_t* __restrict__ group,
                                     const double2* __restrict__ cx, const uint8_t* __restrict__ cst,
                                     const int32_t* __restrict__ csteps,
                                     const double* __restrict__ cbe, double2* x, uint8_t* st,
                                     int32_t* steps, double* be) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < items;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t inst = w / paths, j = w - inst * paths;
    const int64_t r = inst * n_rep + rep_pos[j];
    const uint32_t m = group[sign[j]];
    for (int k = 0; k < n; ++k) {
      const double2 v = cx[r * n + k];
      x[w * n + k] = (m >> k & 1u) ? make_double2(-v.x, -v.y) : v;
    }
    st[w] = cst[r];
    if (steps)
      for (int k = 0; k < 3; ++k) steps[w * 3 + k] = csteps[r * 3 + k];
    if (be) be[w] = cbe[r];
  }
}

// ------------------------------------------------------------------ helpers
int binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return (int)r;
}

// Graded-lex index of an exponent vector among the monomials of degree <= dmax
// in n variables (degree 0 first; inside a degree, the sorted variable tuple
// in lexicographic order).
int graded_index(int n, const std::vector<int>& vars /* sorted ascending */) {
  const int deg = (int)vars.size();
  int idx = 0;
  for (int e = 0; e < deg; ++e) idx += binom(n + e - 1, e);  // monomials of lower degree
  // rank of the multiset among combinations_with_replacement(range(n), deg)
  int prev = 0;
  for (int p = 0; p < deg; ++p) {
    for (int v = prev; v < vars[p]; ++v) idx += binom((n - v) + (deg - p - 1) - 1, deg - p - 1);
    prev = vars[p];
  }
  return idx;
}

struct DeviceBuf {
  void* p = nullptr;
};

}  // namespace

// ------------------------------------------------------------------ problem
struct hc_problem {
  uint32_t magic = kProblemMagic;
  int n = 0, T = 0, kind = 0, maxpf = 0, P = 0, device = 0;
  hc_settings s{};
  double gamma[2] = {1.0, 0.0};
  std::vector<int> eq;
  std::vector<double> coef;  // [T][2]
  std::vector<uint8_t> exps;
  std::vector<int> par;
  std::vector<double> p0, start;
  int64_t n_start = 0;
  int64_t paths = 0;
  // dense total-degree encoding
  bool dense = false;
  int deg = 0, MP = 0, M = 0, L = 0;
  int64_t Dstride = 0, Estride = 0;
  int* d_emap = nullptr;
  int ndc = 0;
  int* d_dterm = nullptr;
  int* d_dslot = nullptr;
  float* d_dmult = nullptr;
  double* d_coef = nullptr;  // default coefficients [T][2]
  // parameter homotopy (term tables, see encode_terms)
  bool terms = false;
  int TT = 0;  // term slots per row
  int extra = 0;
  hc::TermRec* d_rec = nullptr;
  double2* d_s64 = nullptr;
  hc::cdf* d_sdf = nullptr;  // the coefficients as double-floats
  // coefficient interpolation: per (slot, row) the term's parameter factors
  // [TT][L][maxpf] (-1: none), and c(p0) in FP64 / FP32 / double-float
  bool coef_mode = false;
  int32_t* d_cpar = nullptr;
  double2* d_c0 = nullptr;
  float2* d_c0f = nullptr;
  hc::cdf* d_c0df = nullptr;
  // sign symmetries (parameter homotopies): group element masks, one tracked
  // start per orbit (reps), and per start its representative's position in
  // reps and the group element mapping the representative onto it
  int n_group = 1;
  std::vector<uint32_t> group;
  int64_t n_rep = 0;
  uint32_t* d_group = nullptr;
  int64_t* d_reps = nullptr;
  int32_t* d_rep_pos = nullptr;
  uint8_t* d_sign = nullptr;
  double2* d_p0 = nullptr;
  double2* d_start = nullptr;
};

struct hc_batch {
  uint32_t magic = kBatchMagic;
  hc_problem* p = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t evk0 = nullptr, evk1 = nullptr, evk2 = nullptr;  // around the tracking launches
  int64_t n_inst = 0, items = 0;
  bool done = false;
  std::vector<void*> dev;  // device allocations (stream-ordered)
  unsigned long long* d_ctl = nullptr;
  unsigned long long* h_ctl = nullptr;  // pinned: [0..7] summary, [8] escalated
  // host outputs needing a copy at poll time (pageable destinations)
  struct HostCopy {
    void* dst;
    void* pinned;
    size_t bytes;
  };
  std::vector<HostCopy> copies;
  std::vector<void*> pinned;
  bool owns_ctl = false;            // h_ctl from the pinned pool (else a plan's)
  bool owns_kernel_events = false;  // evk* created for this batch (else a plan's)
  int64_t step_budget = 0;
  std::shared_ptr<void> admission;  // in-flight record under a memory cap
};

namespace {

// Pinned host slots for the per-batch control words (cudaMallocHost per
// batch would cost far more than a small batch's tracking).
struct PinnedPool {
  std::mutex mu;
  std::vector<void*> free_slots;
};
PinnedPool& pinned_pool() {
  static PinnedPool pool;
  return pool;
}
// control words of a batch: [0] queue [1] FP64 queue [2] FP64 list count
// [3..5] FP64 steps [6] re-track queue [7] re-track list count [8..15]
// summary [16] untracked paths [17] steps counted against the budget
constexpr int kCtlWords = 24;
constexpr size_t kCtlBytes = sizeof(unsigned long long) * kCtlWords;
void* pinned_slot_get() {
  PinnedPool& pp = pinned_pool();
  std::lock_guard<std::mutex> lk(pp.mu);
  if (pp.free_slots.empty()) {
    void* chunk = nullptr;
    if (cudaMallocHost(&chunk, kCtlBytes * 256) != cudaSuccess) return nullptr;
    for (int i = 0; i < 256; ++i) pp.free_slots.push_back(static_cast<char*>(chunk) + i * kCtlBytes);
  }
  void* q = pp.free_slots.back();
  pp.free_slots.pop_back();
  return q;
}
void pinned_slot_put(void* q) {
  PinnedPool& pp = pinned_pool();
  std::lock_guard<std::mutex> lk(pp.mu);
  pp.free_slots.push_back(q);
}

// High-priority streams for the re-tracking branch of hc_track_batch, handed
// out round-robin: when block slots free up they go to these small launches
// before the pending blocks of other, normal-priority persistent launches,
// and there are enough of them that concurrent batches (several classes,
// the server's slots) rarely queue one batch's re-tracking behind another's.
// Creation is attempted once per device; a slot whose creation failed is
// skipped (nullptr only if every creation failed: the caller then runs the
// re-tracking on its own stream).
cudaStream_t retrack_stream(int device) {
  constexpr int kPerDevice = 16, kMaxDev = 64;
  static std::mutex mu;
  static cudaStream_t streams[kMaxDev][kPerDevice] = {};
  static bool tried[kMaxDev] = {};
  static int next[kMaxDev] = {};
  if (device < 0 || device >= kMaxDev) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!tried[device]) {
    tried[device] = true;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    for (int i = 0; i < kPerDevice; ++i)
      if (cudaStreamCreateWithPriority(&streams[device][i], cudaStreamNonBlocking, hi) !=
          cudaSuccess) {
        streams[device][i] = nullptr;
        cudaGetLastError();
      }
  }
  for (int k = 0; k < kPerDevice; ++k) {
    cudaStream_t s = streams[device][next[device]];
    next[device] = (next[device] + 1) % kPerDevice;
    if (s) return s;
  }
  return nullptr;
}

// Admission under a device-memory cap (hc_set_memory_cap): the batches in
// flight on a device and their device bytes.  Each record owns an event
// recorded after its batch's last copy, so completion can be observed (and
// waited for) without touching the batch, which its owner may destroy.
struct AdmitRecord {
  cudaEvent_t done = nullptr;
  int64_t bytes = 0;
  ~AdmitRecord() {
    if (done) cudaEventDestroy(done);
  }
};
struct AdmitState {
  std::mutex mu;
  int64_t cap = 0, inflight = 0;
  std::vector<std::shared_ptr<AdmitRecord>> recs;  // admission order
};
constexpr int kAdmitDevices = 64;
AdmitState& admit_state(int dev) {
  static AdmitState st[kAdmitDevices];
  return st[dev < 0 || dev >= kAdmitDevices ? 0 : dev];
}
// drop records whose batches have finished (caller holds the lock)
void admit_reap(AdmitState& a) {
  for (size_t i = 0; i < a.recs.size();) {
    if (cudaEventQuery(a.recs[i]->done) == cudaSuccess) {
      a.inflight -= a.recs[i]->bytes;
      a.recs.erase(a.recs.begin() + (long)i);
    } else {
      cudaGetLastError();  // not ready is not an error of the caller's
      ++i;
    }
  }
}
void admit_release(int dev, const std::shared_ptr<void>& rec) {
  if (!rec) return;
  AdmitState& a = admit_state(dev);
  std::lock_guard<std::mutex> lk(a.mu);
  for (size_t i = 0; i < a.recs.size(); ++i)
    if (a.recs[i].get() == rec.get()) {
      a.inflight -= a.recs[i]->bytes;
      a.recs.erase(a.recs.begin() + (long)i);
      break;
    }
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool is_pinned_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

hc::DevSettings dev_settings(const hc_settings& s) {
  hc::DevSettings d;
  d.dt_min = s.dt_min;
  d.dt_max = s.dt_max;
  d.dt_init = s.dt_init;
  d.newton_tol = s.newton_tol;
  d.newton_tol_fp32 = s.newton_tol_fp32;
  d.max_first_corr = s.max_first_corr;
  d.refine_tol = s.refine_tol;
  d.r_inf = s.r_inf;
  d.finite_tol = s.finite_tol;
  d.real_tol = s.real_tol;
  d.singular_cond = s.singular_cond;
  d.t_endgame = s.t_endgame;
  d.dt_min_fp32 = s.dt_min_fp32;
  d.max_first_corr_fp32 = s.max_first_corr_fp32;
  d.max_steps_fp32 = s.max_steps_fp32;
  d.max_newton_ir = s.max_newton_ir;
  d.max_newton = s.max_newton;
  d.max_steps = s.max_steps;
  d.grow_after = s.grow_after;
  d.refine_iters = s.refine_iters;
  d.endgame = s.endgame;
  d.eg_cmax = s.eg_cmax;
  d.eg_samples = s.eg_samples;
  d.eg_s0 = s.eg_s0;
  d.eg_ratio = s.eg_ratio;
  d.eg_tol = s.eg_tol;
  return d;
}

hc_status validate_settings(const hc_settings& s) {
  if (!(s.dt_min > 0) || !(s.dt_max >= s.dt_min) || !(s.dt_init >= s.dt_min) ||
      !(s.dt_init <= s.dt_max) || s.max_newton < 1 || s.max_newton > 16 || s.max_steps < 1 ||
      s.grow_after < 1 || s.refine_iters < 0 || s.refine_iters > 64 || !(s.newton_tol > 0) ||
      !(s.newton_tol_fp32 > 0) || !(s.max_first_corr > 0) || !(s.r_inf > 0) ||
      !(s.dt_min_fp32 >= s.dt_min) || !(s.max_first_corr_fp32 > 0) || s.max_steps_fp32 < 1 ||
      (s.precision != HC_PREC_FP64 && s.precision != HC_PREC_MIXED &&
       s.precision != HC_PREC_DF) ||
      (s.retrack_precision != HC_PREC_FP64 && s.retrack_precision != HC_PREC_DF) ||
      (s.lanes != 0 && s.lanes != 32) || s.max_newton_ir < 1 || s.max_newton_ir > 32 ||
      (s.block_threads != 0 && s.block_threads != 32 && s.block_threads != 64 &&
       s.block_threads != 128) ||
      (s.endgame != 0 && s.endgame != 1) ||
      (s.endgame && (!(s.eg_s0 > 0 && s.eg_s0 < 1) || !(s.eg_ratio > 0 && s.eg_ratio < 1) ||
                     !(s.eg_tol > 0) || s.eg_cmax < 1 || s.eg_cmax > 16 || s.eg_samples < 1 ||
                     s.eg_samples > 60))) {
    set_err("invalid settings");
    return HC_ERR_INVALID;
  }
  return HC_OK;
}

// Dense degree-d detection and encoding maps.
bool encode_dense(hc_problem* p, std::vector<int>& emap, std::vector<int>& dterm,
                  std::vector<int>& dslot, std::vector<float>& dmult) {
  const int n = p->n;
  if (p->kind != HC_TOTAL_DEGREE || p->maxpf != 0) return false;
  // degrees
  std::vector<int> deg(n, 0);
  for (int k = 0; k < p->T; ++k) {
    int d = 0;
    for (int j = 0; j < n; ++j) d += p->exps[(size_t)k * n + j];
    deg[p->eq[k]] = std::max(deg[p->eq[k]], d);
  }
  const int d = deg[0];
  for (int i = 0; i < n; ++i)
    if (deg[i] != d) return false;
  if (d != 2 && d != 3) return false;
  if ((d == 2 && n > 12) || (d == 3 && n > 8)) return false;
  const int M = binom(n + d, d);
  if (p->T != n * M) return false;
  const int L = hc::lanes_for(n);
  const int MP = binom(n + d - 1, d - 1);
  // nested Horner order of F_i's monomials
  std::map<std::vector<int>, int> nested;  // sorted var tuple (ascending) -> index
  {
    int m = 0;
    nested[{}] = m++;
    for (int j = 0; j < n; ++j) {
      nested[{j}] = m++;
      for (int k = 0; k <= j; ++k) {
        nested[{k, j}] = m++;
        if (d == 3)
          for (int l = 0; l <= k; ++l) nested[{l, k, j}] = m++;
      }
    }
    if (m != M) return false;
  }
  std::vector<int> seen((size_t)n * M, 0);
  emap.assign(p->T, 0);
  dterm.clear();
  dslot.clear();
  dmult.clear();
  for (int k = 0; k < p->T; ++k) {
    const int i = p->eq[k];
    std::vector<int> vars;
    for (int j = 0; j < n; ++j)
      for (int e = 0; e < p->exps[(size_t)k * n + j]; ++e) vars.push_back(j);
    auto it = nested.find(vars);
    if (it == nested.end()) return false;
    if (seen[(size_t)i * M + it->second]++) return false;  // duplicate monomial
    emap[k] = it->second * L + i;
    if (vars.empty()) {
      dterm.push_back(k);
      dslot.push_back((int)hc::dense_slot(n, d, L, n, 0, i));
      dmult.push_back(1.0f);
      continue;
    }
    for (int j = 0; j < n; ++j) {
      const int a = p->exps[(size_t)k * n + j];
      if (a == 0) continue;
      std::vector<int> rest;
      bool dropped = false;
      for (int v : vars) {
        if (v == j && !dropped) {
          dropped = true;
          continue;
        }
        rest.push_back(v);
      }
      const int mp = graded_index(n, rest);
      dterm.push_back(k);
      dslot.push_back((int)hc::dense_slot(n, d, L, j, mp, i));
      dmult.push_back((float)a);
    }
  }
  p->dense = true;
  p->deg = d;
  p->M = M;
  p->MP = MP;
  p->L = L;
  p->Dstride = (int64_t)(n + 1) * hc::dense_mpp(n, d) * L;
  p->Estride = (int64_t)M * L;
  int64_t paths = 1;
  for (int i = 0; i < n; ++i) paths *= d;
  p->paths = paths;
  return true;
}


// Sign symmetries of a parameter homotopy (hc_problem_desc.sym_mask): every
// term must have even degree in the unknowns of every mask; the start set
// must be closed under the masks.  Fills the group, the orbit
// representatives and per start its representative's position and sign
// element.  Returns an error message, or nullptr.
const char* build_orbits(hc_problem* p, int n_sym, const uint32_t* masks,
                         std::vector<int64_t>& reps, std::vector<int32_t>& rep_pos,
                         std::vector<uint8_t>& sign) {
  const int n = p->n;
  if (n_sym < 0 || n_sym > 4) return "n_sym must be 0..4";
  for (int k = 0; k < n_sym; ++k) {
    if (masks[k] == 0 || (n < 32 && (masks[k] >> n) != 0)) return "sym_mask: empty or beyond n";
    for (int t = 0; t < p->T; ++t) {
      int deg = 0;
      for (int j = 0; j < n; ++j)
        if (masks[k] >> j & 1u) deg += p->exps[(size_t)t * n + j];
      if (deg & 1) return "sym_mask: a term has odd degree in the masked unknowns";
    }
  }
  const int G = 1 << n_sym;
  p->group.assign(G, 0u);
  for (int e = 0; e < G; ++e)
    for (int k = 0; k < n_sym; ++k)
      if (e >> k & 1) p->group[e] ^= masks[k];
  // lookup of a point in the start set: starts sorted by a linear key
  const int64_t S = p->n_start;
  const double* st = p->start.data();
  auto key = [&](const double* x) {
    double v = 0.0;
    for (int j = 0; j < n; ++j) v += (1.0 + 0.37 * j) * (x[2 * j] + 0.61 * x[2 * j + 1]);
    return v;
  };
  double wsum = 0.0;
  for (int j = 0; j < n; ++j) wsum += 1.61 * (1.0 + 0.37 * j);
  std::vector<std::pair<double, int64_t>> order((size_t)S);
  for (int64_t s = 0; s < S; ++s) order[(size_t)s] = {key(st + 2 * n * s), s};
  std::sort(order.begin(), order.end());
  std::vector<double> img(2 * n);
  auto find = [&](const double* y) -> int64_t {
    double ymax = 1.0;
    for (int j = 0; j < 2 * n; ++j) ymax = std::max(ymax, std::fabs(y[j]));
    const double tol = 1e-9 * ymax;
    const double ky = key(y), kt = 2.0 * tol * wsum;
    auto it = std::lower_bound(order.begin(), order.end(), std::make_pair(ky - kt, (int64_t)-1));
    for (; it != order.end() && it->first <= ky + kt; ++it) {
      const double* x = st + 2 * n * it->second;
      bool same = true;
      for (int j = 0; j < 2 * n && same; ++j) same = std::fabs(x[j] - y[j]) <= tol;
      if (same) return it->second;
    }
    return -1;
  };
  std::vector<int64_t> rep_of((size_t)S);
  sign.assign((size_t)S, 0);
  for (int64_t s = 0; s < S; ++s) {
    int64_t best = s;
    int be = 0;
    for (int e = 1; e < G; ++e) {
      for (int j = 0; j < n; ++j) {
        const double sg = (p->group[e] >> j & 1u) ? -1.0 : 1.0;
        img[2 * j] = sg * st[2 * n * s + 2 * j];
        img[2 * j + 1] = sg * st[2 * n * s + 2 * j + 1];
      }
      const int64_t i = find(img.data());
      if (i < 0) return "the start set is not closed under the sign symmetries";
      if (i < best) {
        best = i;
        be = e;
      }
    }
    rep_of[(size_t)s] = best;  // s = group[be] applied to start best
    sign[(size_t)s] = (uint8_t)be;
  }
  reps.clear();
  std::vector<int32_t> pos((size_t)S, -1);
  for (int64_t s = 0; s < S; ++s)
    if (rep_of[(size_t)s] == s) {
      pos[(size_t)s] = (int32_t)reps.size();
      reps.push_back(s);
    }
  rep_pos.assign((size_t)S, 0);
  for (int64_t s = 0; s < S; ++s) rep_pos[(size_t)s] = pos[(size_t)rep_of[(size_t)s]];
  p->n_group = G;
  p->n_rep = (int64_t)reps.size();
  return nullptr;
}

// Term tables of a parameter homotopy (paper Sec. 6 evaluates the terms of
// the equations per row): for every row i its terms, each a coefficient and
// up to 8 factor positions in V = [x | pad to L | 1 | p(t) | dp | p0] (a
// power x_j^a as a repeated factor), with the entry every factor's
// derivative feeds (x_j -> j, a parameter -> n, i.e. dH/dt through dp).  Rows
// are padded to the same number of term slots, and every slot to the largest
// factor count of its terms over the rows (padding factor: the 1).
// With coefficient interpolation (HC_COEFFICIENT) the parameter factors are
// left out of the records and listed per (slot, row) in cpar instead.
bool encode_terms(hc_problem* p, std::vector<hc::TermRec>& rec, std::vector<double2>& s64,
                  std::vector<int32_t>& cpar) {
  const int n = p->n, P = p->P, L = hc::lanes_for(n);
  const int one = L, pbase = L + 1, dbase = L + 1 + P;
  if (p->kind == HC_TOTAL_DEGREE || n + 2 > hc::kMaxTermEntries || dbase + P > 255) return false;
  const bool cmode = p->kind == HC_COEFFICIENT;
  // per row: its terms as (coefficient, factors, targets, parameter list)
  struct Term {
    double re, im;
    std::vector<int> f, tg, par;
  };
  std::vector<std::vector<Term>> rows(n);
  for (int k = 0; k < p->T; ++k) {
    Term t;
    t.re = p->coef[2 * k];
    t.im = p->coef[2 * k + 1];
    for (int j = 0; j < n; ++j)
      for (int a = 0; a < p->exps[(size_t)k * n + j]; ++a) {
        t.f.push_back(j);
        t.tg.push_back(j);
      }
    for (int f = 0; f < p->maxpf; ++f) {
      const int l = p->par[(size_t)k * p->maxpf + f];
      if (l >= 0 && cmode) {
        t.par.push_back(l);
      } else if (l >= 0) {
        t.f.push_back(pbase + l);
        t.tg.push_back(n);
      }
    }
    if (t.f.empty()) {  // a constant term: the factor 1, no derivative
      t.f.push_back(one);
      t.tg.push_back(255);
    }
    if ((int)t.f.size() > hc::kMaxTermFactors) return false;
    rows[p->eq[k]].push_back(std::move(t));
  }
  // slots: every row's terms by decreasing factor count, rows padded to the
  // longest; at each slot the factor count is the largest over the rows
  int TT = 0;
  for (auto& r : rows) {
    std::stable_sort(r.begin(), r.end(),
                     [](const Term& x, const Term& y) { return x.f.size() > y.f.size(); });
    TT = std::max(TT, (int)r.size());
  }
  rec.assign((size_t)TT * L, hc::TermRec{});
  s64.assign((size_t)TT * L, make_double2(0.0, 0.0));
  const int mp = std::max(p->maxpf, 1);
  cpar.assign(cmode ? (size_t)TT * L * mp : 0, -1);
  for (int k = 0; k < TT; ++k) {
    int d = 1;
    for (int i = 0; i < n; ++i)
      if (k < (int)rows[i].size()) d = std::max(d, (int)rows[i][k].f.size());
    for (int i = 0; i < L; ++i) {
      hc::TermRec& r = rec[(size_t)k * L + i];
      for (int f = 0; f < hc::kMaxTermFactors; ++f) {
        r.idx[f] = (uint8_t)one;
        r.tgt[f] = 255;
      }
      r.d = (uint8_t)d;
      if (i >= n || k >= (int)rows[i].size()) continue;  // zero coefficient
      const Term& t = rows[i][k];
      r.s = make_float2((float)t.re, (float)t.im);
      for (size_t f = 0; f < t.f.size(); ++f) {
        r.idx[f] = (uint8_t)t.f[f];
        r.tgt[f] = (uint8_t)t.tg[f];
      }
      s64[(size_t)k * L + i] = make_double2(t.re, t.im);
      for (size_t f = 0; cmode && f < t.par.size(); ++f)
        cpar[((size_t)k * L + i) * mp + f] = t.par[f];
    }
  }
  p->TT = TT;
  p->terms = true;
  p->coef_mode = cmode;
  p->L = L;
  p->extra = 1 + 3 * P;
  p->paths = p->n_start;
  return true;
}

template <class T>
hc_status upload(const std::vector<T>& v, T** out) {
  *out = nullptr;
  if (v.empty()) return HC_OK;
  HC_CUDA(cudaMalloc((void**)out, v.size() * sizeof(T)));
  HC_CUDA(cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HC_OK;
}

void free_problem(hc_problem* p) {
  if (!p) return;
  cudaFree(p->d_emap);
  cudaFree(p->d_dterm);
  cudaFree(p->d_dslot);
  cudaFree(p->d_dmult);
  cudaFree(p->d_coef);
  cudaFree(p->d_rec);
  cudaFree(p->d_s64);
  cudaFree(p->d_sdf);
  cudaFree(p->d_cpar);
  cudaFree(p->d_c0);
  cudaFree(p->d_c0f);
  cudaFree(p->d_c0df);
  cudaFree(p->d_group);
  cudaFree(p->d_reps);
  cudaFree(p->d_rep_pos);
  cudaFree(p->d_sign);
  cudaFree(p->d_p0);
  cudaFree(p->d_start);
  p->magic = 0;
  delete p;
}

struct Occ {
  int blocks = 0;
  int sms = 0;
};

Occ occupancy(const void* fn, size_t smem, int threads) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, size_t, int>, Occ> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_tuple(fn, smem, threads);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  Occ o;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.blocks, fn, threads, smem);
  if (o.blocks < 1) o.blocks = 1;
  cache[key] = o;
  return o;
}

// Largest dynamic shared memory a block may opt in to on the current device.
size_t max_block_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return (size_t)v;
}

// Persistent launch: grid = resident blocks per SM x SMs, or fewer when the
// items (at most max_items) need fewer groups.
hc_status launch_generic(const hc::KernelRef& k, void* args, size_t smem, int64_t max_items,
                         cudaStream_t st, int threads = hc::kBlock) {
  if (smem > 48 * 1024)
    HC_CUDA(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const Occ o = occupancy(k.fn, smem, threads);
  const int64_t groups_per_block = threads / k.lanes;
  int64_t want = (max_items + groups_per_block - 1) / groups_per_block;
  int64_t grid = std::min<int64_t>((int64_t)o.blocks * o.sms, std::max<int64_t>(want, 1));
  void* argv[] = {args};
  HC_CUDA(cudaLaunchKernel(k.fn, dim3((unsigned)grid), dim3(threads), argv, smem, st));
  return HC_OK;
}

hc_status launch_tracker(const hc::KernelRef& k, const hc::DenseArgs& a, int64_t max_items,
                         cudaStream_t st, int threads = hc::kBlock) {
  const size_t smem =
      (size_t)hc::block_smem_bytes(k.lanes, k.extra, 0, threads, k.eg_bytes, k.vx);
  return launch_generic(k, (void*)&a, smem, max_items, st, threads);
}

}  // namespace

// ------------------------------------------------------------------ C-ABI
namespace hc {
KernelRef retrack_kernel(int deg, int n, int prec) {
  const KernelRef k = dense_kernel(deg, n, prec, 32);
  return k.fn ? k : dense_kernel(deg, n, prec, 0);
}
}  // namespace hc
using hc::retrack_kernel;

namespace {
// The tuning cache: a JSON object {"<key>": {"precision": p, "lanes": l,
// "block_threads": b, "max_first_corr_fp32": c}, ...}, one entry per line
// as written by write_tune_cache.  The reader accepts what the writer
// writes (and an absent or empty file); anything else is refused.
bool read_tune_cache(const char* path, std::map<std::string, std::string>& out) {
  FILE* f = std::fopen(path, "r");
  if (!f) return true;  // no cache yet
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  std::fclose(f);
  size_t pos = text.find('{');
  if (pos == std::string::npos) return text.find_first_not_of(" \t\r\n") == std::string::npos;
  for (;;) {
    const size_t k0 = text.find('"', pos + 1);
    if (k0 == std::string::npos) break;
    const size_t k1 = text.find('"', k0 + 1);
    const size_t o0 = text.find('{', k1);
    const size_t o1 = text.find('}', o0);
    if (k1 == std::string::npos || o0 == std::string::npos || o1 == std::string::npos) return false;
    out[text.substr(k0 + 1, k1 - k0 - 1)] = text.substr(o0, o1 - o0 + 1);
    pos = o1;
  }
  return true;
}

bool write_tune_cache(const char* path, const std::map<std::string, std::string>& entries) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return false;
  std::fprintf(f, "{\n");
  size_t i = 0;
  for (const auto& e : entries)
    std::fprintf(f, "  \"%s\": %s%s\n", e.first.c_str(), e.second.c_str(),
                 ++i < entries.size() ? "," : "");
  std::fprintf(f, "}\n");
  const bool ok = std::fclose(f) == 0;
  return ok && std::rename(tmp.c_str(), path) == 0;
}

bool parse_tune_entry(const std::string& obj, hc_settings& s) {
  auto num = [&](const char* name, double& v) {
    const size_t at = obj.find(std::string("\"") + name + "\"");
    if (at == std::string::npos) return false;
    const size_t colon = obj.find(':', at);
    if (colon == std::string::npos) return false;
    char* end = nullptr;
    v = std::strtod(obj.c_str() + colon + 1, &end);
    return end != obj.c_str() + colon + 1;
  };
  double prec, lanes, block, corr;
  if (!num("precision", prec) || !num("lanes", lanes) || !num("block_threads", block) ||
      !num("max_first_corr_fp32", corr))
    return false;
  s.precision = (int32_t)prec;
  s.lanes = (int32_t)lanes;
  s.block_threads = (int32_t)block;
  s.max_first_corr_fp32 = corr;
  return true;
}
}  // namespace

namespace hc {
// Device bytes one instance of a batch needs with P paths per instance
// (inputs, encoded tables, outputs, scratch): the admission measure.
int64_t instance_device_bytes(const hc_problem* p, int64_t P) {
  const int64_t n = p->n;
  int64_t b = 16 * (int64_t)(p->kind != HC_TOTAL_DEGREE ? p->P : p->T);  // inputs
  if (p->coef_mode) b += 40 * (int64_t)p->TT * p->L;                      // dc tables
  if (!p->terms) b += 32 * p->Estride + 24 * p->Dstride;              // E, Edf, D64, D32
  b += P * (16 * n + 1 + 12 + 8);                                     // x, status, steps, be
  b += P * (8 + 8 + 8 + 8 * n + 8);                                   // lists, t_io, x32, ids
  return b;
}
}  // namespace hc

extern "C" {

const char* hc_status_string(int32_t s) {
  switch (s) {
    case HC_OK: return "ok";
    case HC_PENDING: return "pending";
    case HC_ERR_INVALID: return "invalid argument";
    case HC_ERR_OOM: return "out of memory";
    case HC_ERR_CUDA: return "CUDA error";
    case HC_ERR_TIMEOUT: return "device step budget exhausted";
    case HC_ERR_NUMERIC: return "non-finite input";
    case HC_ERR_BUSY: return "admission refused";
    case HC_ERR_UNSUPPORTED: return "unsupported problem shape";
    default: return "unknown status";
  }
}

const char* hc_last_error(void) { return g_err.c_str(); }

hc_settings hc_default_settings(void) {
  hc_settings s;
  std::memset(&s, 0, sizeof(s));
  s.dt_min = 1e-6;
  s.dt_max = 0.05;
  s.dt_init = 0.01;
  s.newton_tol = 1e-8;
  s.newton_tol_fp32 = 1e-4;
  s.max_first_corr = 0.1;
  s.refine_tol = 1e-13;
  s.r_inf = 1e8;
  s.finite_tol = 1e-10;
  s.real_tol = 1e-8;
  s.singular_cond = 1e12;
  s.t_endgame = 0.95;
  s.dt_min_fp32 = 1e-4;
  s.max_first_corr_fp32 = 0.01;
  s.max_steps_fp32 = 2000;
  s.max_newton = 3;
  s.max_steps = 100000;
  s.grow_after = 3;
  s.refine_iters = 8;
  s.precision = HC_PREC_MIXED;
  s.escalate = 1;
  s.lanes = 0;
  s.max_newton_ir = 6;
  s.block_threads = 0;
  s.endgame = 0;
  s.eg_cmax = 8;
  s.eg_samples = 40;
  s.retrack_precision = HC_PREC_DF;
  s.eg_s0 = 0.1;
  s.eg_ratio = 0.5;
  s.eg_tol = 1e-8;
  return s;
}

hc_status hc_create_problem(const hc_problem_desc* d, hc_problem** out) {
  g_err.clear();
  if (!d || !out) {
    set_err("null descriptor or output");
    return HC_ERR_INVALID;
  }
  const int n = d->n, T = d->n_terms;
  if (n < 1 || n > 32 || T < 1 || !d->term_eq || !d->term_coef || !d->term_exp ||
      d->max_pfac < 0 || d->max_pfac > 8 || (d->max_pfac > 0 && !d->term_param) ||
      (d->kind != HC_TOTAL_DEGREE && d->kind != HC_PARAMETER && d->kind != HC_COEFFICIENT) ||
      d->n_params < 0) {
    set_err("invalid problem descriptor");
    return HC_ERR_INVALID;
  }
  hc_status vs = validate_settings(d->settings);
  if (vs != HC_OK) return vs;
  std::vector<int> eqcount(n, 0);
  for (int k = 0; k < T; ++k) {
    if (d->term_eq[k] < 0 || d->term_eq[k] >= n) {
      set_err("term_eq out of range");
      return HC_ERR_INVALID;
    }
    ++eqcount[d->term_eq[k]];
    int tot = 0;
    for (int j = 0; j < n; ++j) tot += d->term_exp[(size_t)k * n + j];
    if (tot > 15) {
      set_err("term degree above 15");
      return HC_ERR_INVALID;
    }
    for (int f = 0; f < d->max_pfac; ++f) {
      const int l = d->term_param[(size_t)k * d->max_pfac + f];
      if (l < -1 || l >= d->n_params) {
        set_err("term_param out of range");
        return HC_ERR_INVALID;
      }
    }
    if (!std::isfinite(d->term_coef[2 * k]) || !std::isfinite(d->term_coef[2 * k + 1])) {
      set_err("non-finite coefficient");
      return HC_ERR_NUMERIC;
    }
  }
  for (int i = 0; i < n; ++i)
    if (eqcount[i] == 0) {
      set_err("an equation has no terms");
      return HC_ERR_INVALID;
    }
  if (d->n_sym != 0 && d->kind == HC_TOTAL_DEGREE) {
    set_err("sign symmetries need a parameter homotopy");
    return HC_ERR_INVALID;
  }
  if (d->kind == HC_TOTAL_DEGREE &&
      !(std::fabs(std::hypot(d->gamma[0], d->gamma[1]) - 1.0) < 1e-6)) {
    set_err("gamma must have unit modulus");
    return HC_ERR_INVALID;
  }
  if (d->kind != HC_TOTAL_DEGREE && (d->n_params < 1 || !d->p0 || d->n_start < 1 || !d->start)) {
    set_err("parameter homotopy needs p0 and start solutions");
    return HC_ERR_INVALID;
  }

  hc_problem* p = new hc_problem;
  p->n = n;
  p->T = T;
  p->kind = d->kind;
  p->maxpf = d->max_pfac;
  p->P = d->n_params;
  p->s = d->settings;
  p->gamma[0] = d->gamma[0];
  p->gamma[1] = d->gamma[1];
  p->eq.assign(d->term_eq, d->term_eq + T);
  p->coef.assign(d->term_coef, d->term_coef + 2 * (size_t)T);
  p->exps.assign(d->term_exp, d->term_exp + (size_t)T * n);
  if (p->maxpf) p->par.assign(d->term_param, d->term_param + (size_t)T * p->maxpf);
  cudaGetDevice(&p->device);

  if (d->kind != HC_TOTAL_DEGREE) {
    p->n_start = d->n_start;
    for (int64_t k = 0; k < (int64_t)d->n_params * 2; ++k)
      if (!std::isfinite(d->p0[k])) {
        delete p;
        set_err("non-finite p0");
        return HC_ERR_NUMERIC;
      }
    p->start.assign(d->start, d->start + 2 * (size_t)d->n_start * n);
    std::vector<int64_t> reps;
    std::vector<int32_t> rep_pos;
    std::vector<uint8_t> sign;
    if (d->n_sym != 0) {
      const char* why = build_orbits(p, d->n_sym, d->sym_mask, reps, rep_pos, sign);
      if (why) {
        delete p;
        set_err(why);
        return HC_ERR_INVALID;
      }
    }
    std::vector<hc::TermRec> rec;
    std::vector<double2> s64;
    std::vector<int32_t> cpar;
    if (!encode_terms(p, rec, s64, cpar)) {
      delete p;
      set_err("parameter homotopy: n <= 32, at most 8 factors per term, L + 1 + 2 n_params <= 255");
      return HC_ERR_UNSUPPORTED;
    }
    if (!hc::term_kernel(n, HC_PREC_MIXED, 0).fn) {
      delete p;
      set_err("this build has parameter-homotopy kernels for n <= 24");
      return HC_ERR_UNSUPPORTED;
    }
    // double-float split of every coefficient: hi the nearest float, lo the
    // nearest float to the remainder
    std::vector<hc::cdf> sdf(s64.size());
    for (size_t k = 0; k < s64.size(); ++k) sdf[k] = hc::split_cdf_host(s64[k].x, s64[k].y);
    // coefficient interpolation: c(p0) of every (slot, row), the term
    // coefficient times its parameter factors at p0
    std::vector<double2> c0;
    std::vector<float2> c0f;
    std::vector<hc::cdf> c0df;
    if (p->coef_mode) {
      const int mp = std::max(p->maxpf, 1);
      c0.resize(s64.size());
      c0f.resize(s64.size());
      c0df.resize(s64.size());
      for (size_t k = 0; k < s64.size(); ++k) {
        double re = s64[k].x, im = s64[k].y;
        for (int f = 0; f < mp; ++f) {
          const int l = cpar[k * mp + f];
          if (l < 0) continue;
          const double pr = d->p0[2 * l], pi = d->p0[2 * l + 1];
          const double nr = re * pr - im * pi, ni = re * pi + im * pr;
          re = nr;
          im = ni;
        }
        c0[k] = make_double2(re, im);
        c0f[k] = make_float2((float)re, (float)im);
        c0df[k] = hc::split_cdf_host(re, im);
      }
    }
    std::vector<double2> p0v(d->n_params), sv((size_t)d->n_start * n);
    for (int l = 0; l < d->n_params; ++l) p0v[l] = make_double2(d->p0[2 * l], d->p0[2 * l + 1]);
    for (size_t k = 0; k < sv.size(); ++k) sv[k] = make_double2(d->start[2 * k], d->start[2 * k + 1]);
    hc_status st;
    if ((st = upload(rec, &p->d_rec)) != HC_OK || (st = upload(s64, &p->d_s64)) != HC_OK ||
        (st = upload(sdf, &p->d_sdf)) != HC_OK || (st = upload(cpar, &p->d_cpar)) != HC_OK ||
        (st = upload(c0, &p->d_c0)) != HC_OK || (st = upload(c0f, &p->d_c0f)) != HC_OK ||
        (st = upload(c0df, &p->d_c0df)) != HC_OK ||
        (st = upload(p0v, &p->d_p0)) != HC_OK || (st = upload(sv, &p->d_start)) != HC_OK ||
        (st = upload(p->group, &p->d_group)) != HC_OK || (st = upload(reps, &p->d_reps)) != HC_OK ||
        (st = upload(rep_pos, &p->d_rep_pos)) != HC_OK || (st = upload(sign, &p->d_sign)) != HC_OK) {
      free_problem(p);
      return st;
    }
    *out = p;
    return HC_OK;
  }
  std::vector<int> emap, dterm, dslot;
  std::vector<float> dmult;
  if (!encode_dense(p, emap, dterm, dslot, dmult)) {
    delete p;
    set_err("this build tracks total-degree homotopies of dense systems of degree 2 (n <= 12) "
            "or 3 (n <= 8)");
    return HC_ERR_UNSUPPORTED;
  }
  p->ndc = (int)dterm.size();
  hc_status st;
  if ((st = upload(emap, &p->d_emap)) != HC_OK || (st = upload(dterm, &p->d_dterm)) != HC_OK ||
      (st = upload(dslot, &p->d_dslot)) != HC_OK || (st = upload(dmult, &p->d_dmult)) != HC_OK ||
      (st = upload(p->coef, &p->d_coef)) != HC_OK) {
    free_problem(p);
    return st;
  }
  *out = p;
  return HC_OK;
}

int64_t hc_problem_paths(const hc_problem* p) {
  if (!p || p->magic != kProblemMagic) return -1;
  return p->paths;
}

hc_status hc_problem_query(const hc_problem* p, hc_problem_info* out) {
  if (!p || p->magic != kProblemMagic || !out) {
    set_err("invalid problem");
    return HC_ERR_INVALID;
  }
  out->n = p->n;
  out->kind = p->kind;
  out->inputs_per_instance = p->kind != HC_TOTAL_DEGREE ? p->P : p->T;
  out->lanes = p->terms ? hc::term_kernel(p->n, HC_PREC_MIXED, 0).lanes : p->L;
  out->paths = p->paths;
  out->device_bytes_per_instance = hc::instance_device_bytes(p, p->paths);
  return HC_OK;
}

}  // extern "C"

namespace {

// Device buffers of one batch.
struct Bufs {
  int64_t paths = 0;                 // paths per instance of this batch (subset size)
  const int64_t* path_ids = nullptr; // device [instances][paths] start indices, or null
  int64_t step_budget = 0;           // 0: none
  const double* d_coef = nullptr;  // dense: per-instance coefficients (or the problem's)
  int64_t coef_stride = 0;
  const double2* d_p1 = nullptr;   // parameter families: target parameters
  void *E = nullptr, *Edf = nullptr, *D64 = nullptr, *D32 = nullptr, *Ddf = nullptr;
  double* d_x = nullptr;
  uint8_t* d_status = nullptr;
  int32_t* d_steps = nullptr;
  double* d_be = nullptr;
  unsigned long long* d_ctl = nullptr;  // kCtlWords control words (see kCtlBytes)
  unsigned long long* h_ctl = nullptr;  // pinned copy of d_ctl
  int64_t* esc_list = nullptr;
  int64_t* dup_list = nullptr;
  double* t_io = nullptr;
  float2* x32 = nullptr;
  // sign symmetries: results of the tracked orbit representatives, expanded
  // into d_x .. d_be at the end
  double* cx = nullptr;
  uint8_t* cst = nullptr;
  int32_t* csteps = nullptr;
  double* cbe = nullptr;
  // coefficient interpolation: per-instance coefficient changes
  double2* dc = nullptr;
  float2* dcf = nullptr;
  hc::cdf* dcdf = nullptr;
};

// The batch tracks orbit representatives (sign symmetries, no start subset).
bool sym_active(const hc_problem* p, const Bufs& B) { return p->n_group > 1 && !B.path_ids; }
// Paths per instance the kernels track.
int64_t tracked_paths(const hc_problem* p, const Bufs& B) {
  return sym_active(p, B) ? p->n_rep : B.paths;
}

// Scratch of a batch (encoded coefficients, control words, re-tracking lists);
// alloc(bytes, &ptr) returns an hc_status.
template <class A>
hc_status alloc_scratch(hc_problem* p, int64_t n_inst, Bufs& B, A&& alloc) {
  const bool mixed = p->s.precision == HC_PREC_MIXED;
  const bool escalate = mixed && p->s.escalate;
  const int64_t items = n_inst * tracked_paths(p, B);
  void* q;
  hc_status rc;
  if (p->coef_mode) {
    const size_t e = (size_t)n_inst * p->TT * p->L;
    if ((rc = alloc(sizeof(double2) * e, &q)) != HC_OK) return rc;
    B.dc = (double2*)q;
    if ((rc = alloc(sizeof(float2) * e, &q)) != HC_OK) return rc;
    B.dcf = (float2*)q;
    if ((rc = alloc(sizeof(hc::cdf) * e, &q)) != HC_OK) return rc;
    B.dcdf = (hc::cdf*)q;
  }
  if (sym_active(p, B)) {
    if ((rc = alloc(sizeof(double) * 2 * p->n * items, &q)) != HC_OK) return rc;
    B.cx = (double*)q;
    if ((rc = alloc((size_t)items, &q)) != HC_OK) return rc;
    B.cst = (uint8_t*)q;
    if ((rc = alloc(sizeof(int32_t) * 3 * items, &q)) != HC_OK) return rc;
    B.csteps = (int32_t*)q;
    if ((rc = alloc(sizeof(double) * items, &q)) != HC_OK) return rc;
    B.cbe = (double*)q;
  }
  if (!p->terms) {
    const int prec = p->s.precision, last = hc::last_tier_precision(p->s);
    if ((rc = alloc(sizeof(cx<double>) * p->Estride * n_inst, &B.E)) != HC_OK) return rc;
    if (prec == HC_PREC_FP64 || (escalate && last == HC_PREC_FP64))
      if ((rc = alloc(sizeof(cx<double>) * p->Dstride * n_inst, &B.D64)) != HC_OK) return rc;
    if (prec == HC_PREC_DF || (escalate && last == HC_PREC_DF))
      if ((rc = alloc(sizeof(cx<hc::df>) * p->Dstride * n_inst, &B.Ddf)) != HC_OK) return rc;
    if (mixed) {
      if ((rc = alloc(sizeof(cx<float>) * p->Dstride * n_inst, &B.D32)) != HC_OK) return rc;
      if ((rc = alloc(sizeof(hc::cdf) * p->Estride * n_inst, &B.Edf)) != HC_OK) return rc;
    }
  }
  if ((rc = alloc(kCtlBytes, &q)) != HC_OK) return rc;
  B.d_ctl = (unsigned long long*)q;
  if (escalate) {
    if ((rc = alloc(sizeof(int64_t) * items, &q)) != HC_OK) return rc;
    B.esc_list = (int64_t*)q;
    if ((rc = alloc(sizeof(int64_t) * items, &q)) != HC_OK) return rc;
    B.dup_list = (int64_t*)q;
    if ((rc = alloc(sizeof(double) * items, &q)) != HC_OK) return rc;
    B.t_io = (double*)q;
    if ((rc = alloc(sizeof(float2) * p->n * items, &q)) != HC_OK) return rc;
    B.x32 = (float2*)q;
  }
  return HC_OK;
}

// Threads per block of the main tracking launch (settings.block_threads).
int main_threads(const hc_settings& s) { return s.block_threads ? s.block_threads : hc::kBlock; }

// Events of one enqueue: ek0..ek2 time the tracking launch and the
// re-tracking tiers; fork and join order the re-tracking stream after the
// tracking launch and the summary after the re-tracking.  Under stream
// capture the timing events become event-record nodes of the graph
// (external), the fork/join events only graph edges.
struct EnqEvents {
  cudaEvent_t ek0, ek1, ek2, fork, join;
  bool capture;
};

// Enqueues one batch on st: clearing, staging, the tracking launch, the
// re-tracking tiers (on the stream hs, event-ordered), the summary and the
// copy of the control words to B.h_ctl.  Allocates nothing and never waits
// on the host, so it can be captured into a CUDA graph.
hc_status enqueue_compute(hc_problem* p, int64_t n_inst, const Bufs& B, cudaStream_t st,
                          cudaStream_t hs, const EnqEvents& ev) {
  auto mark = [&](cudaEvent_t e, cudaStream_t s) {
    return ev.capture ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                      : cudaEventRecord(e, s);
  };
  const bool mixed = p->s.precision == HC_PREC_MIXED;
  const bool escalate = mixed && p->s.escalate;
  const bool sym = sym_active(p, B);
  const int64_t paths = tracked_paths(p, B);  // tracked paths per instance
  const int64_t items = n_inst * paths;       // tracked items
  const int64_t out_items = n_inst * B.paths;
  double* tx = sym ? B.cx : B.d_x;             // the tracking launches' outputs
  uint8_t* tst = sym ? B.cst : B.d_status;
  int32_t* tsteps = sym ? B.csteps : B.d_steps;
  double* tbe = sym ? B.cbe : B.d_be;
  const int n_group = sym ? p->n_group : 1;
  const uint32_t* group = sym ? p->d_group : nullptr;
  const int n = p->n;
  if (!p->terms) {
    HC_CUDA(cudaMemsetAsync(B.E, 0, sizeof(cx<double>) * p->Estride * n_inst, st));
    if (B.Edf) HC_CUDA(cudaMemsetAsync(B.Edf, 0, sizeof(hc::cdf) * p->Estride * n_inst, st));
    if (B.D64) HC_CUDA(cudaMemsetAsync(B.D64, 0, sizeof(cx<double>) * p->Dstride * n_inst, st));
    if (B.Ddf) HC_CUDA(cudaMemsetAsync(B.Ddf, 0, sizeof(cx<hc::df>) * p->Dstride * n_inst, st));
    if (B.D32) HC_CUDA(cudaMemsetAsync(B.D32, 0, sizeof(cx<float>) * p->Dstride * n_inst, st));
    const int64_t work = n_inst * (p->T + p->ndc);
    const int grid = (int)std::min<int64_t>((work + 255) / 256, 4096);
    stage_dense_kernel<<<grid, 256, 0, st>>>(n_inst, p->T, (const double2*)B.d_coef, B.coef_stride,
                                            p->d_emap, p->ndc, p->d_dterm, p->d_dslot,
                                            p->d_dmult, (double2*)B.E, (hc::cdf*)B.Edf, p->Estride,
                                            (float2*)B.D32,
                                            (double2*)B.D64, (float4*)B.Ddf, p->Dstride);
    HC_CUDA(cudaGetLastError());
  }
  HC_CUDA(cudaMemsetAsync(B.d_ctl, 0, kCtlBytes, st));
  HC_CUDA(cudaMemsetAsync(tsteps, 0, sizeof(int32_t) * 3 * items, st));
  if (B.step_budget > 0) {
    // paths the budget leaves unstarted keep HC_PATH_NONE and a NaN
    // endpoint copy (the duplicate check skips them)
    HC_CUDA(cudaMemsetAsync(tst, 0, (size_t)items, st));
    if (B.x32) HC_CUDA(cudaMemsetAsync(B.x32, 0xff, sizeof(float2) * n * items, st));
  }

  hc::LaunchCommon cm;
  std::memset(&cm, 0, sizeof(cm));
  cm.s = dev_settings(p->s);
  cm.n_items = items;
  cm.queue = B.d_ctl + 0;
  cm.paths = paths;
  cm.path_ids = B.path_ids;
  cm.path_map = sym ? p->d_reps : nullptr;
  cm.step_total = B.d_ctl + 17;
  cm.step_budget = (unsigned long long)B.step_budget;
  cm.x_out = tx;
  cm.status_out = tst;
  cm.steps_out = tsteps;
  cm.be_out = tbe;
  cm.esc_list = B.esc_list;
  cm.esc_count = B.d_ctl + 2;
  cm.t_io = B.t_io;
  cm.x32_out = B.x32;
  cm.dup_list = B.dup_list;
  cm.dup_count = B.d_ctl + 7;
  // Re-tracking tiers.  Colliding endpoints (path jumps, found by the
  // duplicate check) and FP32-tier failures other than step-size ones
  // (divergence, non-finite state, failed refinement: dup_list, ctl[7]) run
  // again from t = 0 in the mixed kernel with the FP64 state, FP64 residuals
  // and FP64 tolerances.  Whatever still fails or collides after that tier,
  // step-size failures and suspect-condition endpoints (esc_list, ctl[2])
  // run in the all-FP64 kernel: from t = 0, from the last accepted point, or
  // only the refinement and condition at t = 1.
  hc::LaunchCommon cd = cm;
  cd.count_dev = B.d_ctl + 7;
  cd.items = B.dup_list;
  cd.queue = B.d_ctl + 6;
  cd.start_hi = 1;
  cd.spread = 1;
  cd.dup_list = nullptr;
  cd.dup_count = nullptr;
  hc::LaunchCommon ce = cm;
  ce.count_dev = B.d_ctl + 2;
  ce.items = B.esc_list;
  ce.queue = B.d_ctl + 1;
  ce.esc_list = nullptr;
  ce.x32_out = nullptr;
  ce.esc_steps = B.d_ctl + 3;
  ce.spread = 1;
  ce.dup_list = nullptr;
  ce.dup_count = nullptr;
  // the count of re-tracked items is only known on the device: the grid
  // covers up to every item (capped at full occupancy by the launcher)
  const int64_t esc_groups = items;
  if (!hs) hs = st;
  auto dedupe = [&]() -> hc_status {
    HC_CUDA(cudaStreamWaitEvent(hs, ev.capture ? ev.fork : ev.ek1, 0));
    const int grid = (int)std::min<int64_t>((items + 255) / 256, 65535);
    dedupe_kernel<<<std::max(grid, 1), 256, 0, hs>>>(items, paths, n, B.x32, tst, 1e-6f,
                                                    nullptr, nullptr, B.dup_list, B.d_ctl + 7,
                                                    B.t_io, n_group, group);
    HC_CUDA(cudaGetLastError());
    return HC_OK;
  };
  // after the FP64-residual re-track: a re-tracked endpoint that collides
  // goes to the all-FP64 tier, from t = 0
  auto dedupe_again = [&]() -> hc_status {
    const int grid = (int)std::min<int64_t>((items + 7) / 8, 1024);  // 8 warps per block
    dedupe_list_kernel<<<std::max(grid, 1), 256, 0, hs>>>(paths, n, B.x32, tst, 1e-6f,
                                                         B.dup_list, B.d_ctl + 7, B.esc_list,
                                                         B.d_ctl + 2, B.t_io, n_group, group);
    HC_CUDA(cudaGetLastError());
    return HC_OK;
  };
  hc_status rc;
  if (p->terms) {
    hc::TermArgs ta;
    std::memset(&ta, 0, sizeof(ta));
    ta.c = cm;
    ta.rec = p->d_rec;
    ta.s64 = p->d_s64;
    ta.sdf = p->d_sdf;
    ta.TT = p->TT;
    ta.P = p->P;
    ta.ls = p->L;
    ta.extra = p->extra;
    ta.p0 = p->d_p0;
    ta.p1 = B.d_p1;
    ta.start = p->d_start;
    if (p->coef_mode) {
      const int64_t slots = (int64_t)p->TT * p->L;
      const int gs = (int)std::min<int64_t>((n_inst * slots + 255) / 256, 4096);
      stage_coef_kernel<<<std::max(gs, 1), 256, 0, st>>>(n_inst, slots, std::max(p->maxpf, 1),
                                                         p->d_cpar, p->d_s64, p->d_c0, B.d_p1,
                                                         p->P, B.dc, B.dcf, B.dcdf);
      HC_CUDA(cudaGetLastError());
      ta.coef_mode = 1;
      ta.c0 = p->d_c0;
      ta.c0f = p->d_c0f;
      ta.c0df = p->d_c0df;
      ta.dc = B.dc;
      ta.dcf = B.dcf;
      ta.dcdf = B.dcdf;
    }
    const hc::KernelRef k = hc::term_kernel(n, p->s.precision, mixed ? p->s.lanes : 0);
    auto smem_of = [&](const hc::KernelRef& kr, int threads = hc::kBlock) {
      return (size_t)hc::block_smem_bytes(kr.lanes, p->extra, kr.acc_bytes, threads, kr.eg_bytes,
                                          kr.vx);
    };
    // fewer paths per block where a block's groups would not fit in shared
    // memory (many parameters: V holds 1 + 3 P entries per group)
    const size_t smem_cap = max_block_smem();
    auto fit = [&](const hc::KernelRef& kr, int threads) {
      while (threads > 32 && threads > kr.lanes && smem_of(kr, threads) > smem_cap) threads /= 2;
      return threads;
    };
    HC_CUDA(mark(ev.ek0, st));
    const int bth = fit(k, std::max(main_threads(p->s), k.lanes));
    if ((rc = launch_generic(k, &ta, smem_of(k, bth), items, st, bth)) != HC_OK) return rc;
    HC_CUDA(mark(ev.ek1, st));
    if (escalate) {
      if (ev.capture) HC_CUDA(cudaEventRecord(ev.fork, st));
      if ((rc = dedupe()) != HC_OK) return rc;
      hc::TermArgs td = ta;
      td.c = cd;
      const int th = fit(k, hc::retrack_threads(k.lanes));
      if ((rc = launch_generic(k, &td, smem_of(k, th), esc_groups, hs, th)) != HC_OK) return rc;
      if ((rc = dedupe_again()) != HC_OK) return rc;
      hc::TermArgs te = ta;
      te.c = ce;
      const hc::KernelRef k64 = hc::term_kernel(n, hc::last_tier_precision(p->s), 0);
      const int th64 = fit(k64, hc::retrack_threads(k64.lanes));
      if ((rc = launch_generic(k64, &te, smem_of(k64, th64), esc_groups, hs, th64)) != HC_OK)
        return rc;
      HC_CUDA(mark(ev.ek2, hs));
      if (ev.capture) HC_CUDA(cudaEventRecord(ev.join, hs));
      HC_CUDA(cudaStreamWaitEvent(st, ev.capture ? ev.join : ev.ek2, 0));
    } else {
      HC_CUDA(mark(ev.ek2, st));
    }
  } else {
    hc::DenseArgs a;
    std::memset(&a, 0, sizeof(a));
    a.c = cm;
    a.D32 = (const cx<float>*)B.D32;
    a.D64 = (const cx<double>*)B.D64;
    a.Ddf = (const cx<hc::df>*)B.Ddf;
    a.E = (const cx<double>*)B.E;
    a.Edf = (const hc::cdf*)B.Edf;
    a.Dstride = p->Dstride;
    a.Estride = p->Estride;
    a.gamma = cx<double>{p->gamma[0], p->gamma[1]};
    a.gamma32 = cx<float>{(float)p->gamma[0], (float)p->gamma[1]};
    a.gammadf = hc::split_cdf_host(p->gamma[0], p->gamma[1]);
    const hc::KernelRef k = hc::dense_kernel(p->deg, n, p->s.precision, mixed ? p->s.lanes : 0);
    if (!k.fn) {
      set_err("no kernel for this problem shape");
      return HC_ERR_UNSUPPORTED;
    }
    HC_CUDA(mark(ev.ek0, st));
    if ((rc = launch_tracker(k, a, items, st, std::max(main_threads(p->s), k.lanes))) != HC_OK)
      return rc;
    HC_CUDA(mark(ev.ek1, st));
    if (escalate) {
      if (ev.capture) HC_CUDA(cudaEventRecord(ev.fork, st));
      if ((rc = dedupe()) != HC_OK) return rc;
      // the re-tracking tiers see a few paths each: one path per warp with
      // the rows split over the warp where that variant exists
      hc::DenseArgs dd = a;
      dd.c = cd;
      const hc::KernelRef kr = retrack_kernel(p->deg, n, HC_PREC_MIXED);
      if ((rc = launch_tracker(kr, dd, esc_groups, hs, hc::retrack_threads(kr.lanes))) != HC_OK)
        return rc;
      if ((rc = dedupe_again()) != HC_OK) return rc;
      hc::DenseArgs e = a;
      e.c = ce;
      const hc::KernelRef k64 = retrack_kernel(p->deg, n, hc::last_tier_precision(p->s));
      if ((rc = launch_tracker(k64, e, esc_groups, hs, hc::retrack_threads(k64.lanes))) != HC_OK)
        return rc;
      HC_CUDA(mark(ev.ek2, hs));
      if (ev.capture) HC_CUDA(cudaEventRecord(ev.join, hs));
      HC_CUDA(cudaStreamWaitEvent(st, ev.capture ? ev.join : ev.ek2, 0));
    } else {
      HC_CUDA(mark(ev.ek2, st));
    }
  }
  if (sym) {
    const int eg = (int)std::min<int64_t>((out_items + 255) / 256, 4096);
    expand_orbits_kernel<<<std::max(eg, 1), 256, 0, st>>>(
        out_items, B.paths, paths, n, p->d_rep_pos, p->d_sign, p->d_group, (const double2*)tx, tst,
        tsteps, tbe, (double2*)B.d_x, B.d_status, B.d_steps, B.d_be);
    HC_CUDA(cudaGetLastError());
  }
  const int grid = (int)std::min<int64_t>((std::max(items, out_items) + 255) / 256, 1024);
  summarize_kernel<<<std::max(grid, 1), 256, 0, st>>>(out_items, B.d_status, items, tsteps,
                                                     B.d_ctl + 8, B.d_ctl + 16);
  HC_CUDA(cudaGetLastError());
  if (B.h_ctl)
    HC_CUDA(cudaMemcpyAsync(B.h_ctl, B.d_ctl, kCtlBytes, cudaMemcpyDeviceToHost, st));
  return HC_OK;
}

hc_status validate_batch(hc_problem* p, const hc_batch_desc* b) {
  if (!p || p->magic != kProblemMagic || !b || b->n_instances < 1 || !b->x_out ||
      !b->status_out || b->step_budget < 0 || b->n_subset < 0 || b->reserved != 0 ||
      (b->n_subset > 0 && !b->path_ids)) {
    set_err("invalid batch descriptor");
    return HC_ERR_INVALID;
  }
  if (b->n_subset > 0) {
    const int64_t cnt = (int64_t)b->n_instances * b->n_subset;
    for (int64_t k = 0; k < cnt; ++k)
      if (b->path_ids[k] < 0 || b->path_ids[k] >= p->paths) {
        set_err("path_ids: a start index is out of range");
        return HC_ERR_INVALID;
      }
  }
  if (p->kind != HC_TOTAL_DEGREE && !b->p1) {
    set_err("parameter homotopy batch needs p1");
    return HC_ERR_INVALID;
  }
  return HC_OK;
}

void release_batch(hc_batch* bt) {
  admit_release(bt->p ? bt->p->device : 0, bt->admission);
  bt->admission.reset();
  for (void* q : bt->dev) cudaFree(q);
  for (void* q : bt->pinned) cudaFreeHost(q);
  if (bt->h_ctl && bt->owns_ctl) pinned_slot_put(bt->h_ctl);
  for (cudaEvent_t e : {bt->ev0, bt->ev1})
    if (e) cudaEventDestroy(e);
  if (bt->owns_kernel_events)
    for (cudaEvent_t e : {bt->evk0, bt->evk1, bt->evk2})
      if (e) cudaEventDestroy(e);
  bt->magic = 0;
  delete bt;
}

// Output side of a batch: device destinations for the kernels (the user's
// device buffers, or fresh ones copied back to the user's host buffers).
hc_status setup_outputs(hc_batch* bt, const hc_batch_desc* b, int n, int64_t items, bool devptrs,
                        Bufs& B, std::vector<void*>& d2h,
                        const std::function<hc_status(size_t, void**)>& dalloc) {
  B.d_x = b->x_out;
  B.d_status = b->status_out;
  B.d_steps = b->steps_out;
  B.d_be = b->be_out;
  auto out_buffer = [&](void* user, size_t bytes, void** dptr) -> hc_status {
    hc_status s = dalloc(bytes, dptr);
    if (s != HC_OK) return s;
    if (user) {
      if (is_pinned_host(user)) {
        bt->copies.push_back({user, nullptr, bytes});
      } else {
        void* pin;
        if (cudaMallocHost(&pin, bytes) != cudaSuccess) {
          set_err("cudaMallocHost failed");
          return HC_ERR_OOM;
        }
        bt->pinned.push_back(pin);
        bt->copies.push_back({user, pin, bytes});
      }
      d2h.push_back(*dptr);
    }
    return HC_OK;
  };
  hc_status rc;
  void* q;
  if (!devptrs) {
    if ((rc = out_buffer(b->x_out, sizeof(double) * 2 * n * items, &q)) != HC_OK) return rc;
    B.d_x = (double*)q;
    if ((rc = out_buffer(b->status_out, items, &q)) != HC_OK) return rc;
    B.d_status = (uint8_t*)q;
    if ((rc = out_buffer(b->steps_out, sizeof(int32_t) * 3 * items, &q)) != HC_OK) return rc;
    B.d_steps = (int32_t*)q;
    B.d_be = nullptr;
    if (b->be_out) {
      if ((rc = out_buffer(b->be_out, sizeof(double) * items, &q)) != HC_OK) return rc;
      B.d_be = (double*)q;
    }
  } else if (!B.d_steps) {
    if ((rc = dalloc(sizeof(int32_t) * 3 * items, &q)) != HC_OK) return rc;
    B.d_steps = (int32_t*)q;
  }
  return HC_OK;
}

}  // namespace

extern "C" {

hc_status hc_track_batch(hc_problem* p, const hc_batch_desc* b, hc_batch** out) {
  g_err.clear();
  cudaGetLastError();  // launch errors checked below are this call's own
  hc_status rc = validate_batch(p, b);
  if (rc != HC_OK || !out) return rc != HC_OK ? rc : HC_ERR_INVALID;
  int cur = 0;
  HC_CUDA(cudaGetDevice(&cur));
  if (cur != p->device) HC_CUDA(cudaSetDevice(p->device));
  const bool devptrs = (b->flags & HC_DEVICE_PTRS) != 0;

  const int64_t paths_eff = b->n_subset > 0 ? (int64_t)b->n_subset : p->paths;
  // ---- admission under the device-memory cap
  std::shared_ptr<AdmitRecord> adm;
  {
    AdmitState& a = admit_state(p->device);
    std::unique_lock<std::mutex> lk(a.mu);
    if (a.cap > 0) {
      const int64_t need = hc::instance_device_bytes(p, paths_eff) * b->n_instances;
      admit_reap(a);
      while (a.inflight + need > a.cap && !a.recs.empty()) {
        if (!(b->flags & HC_BLOCKING_ADMIT)) {
          set_err("admission refused: the batches in flight and this one exceed the memory cap");
          if (cur != p->device) cudaSetDevice(cur);
          return HC_ERR_BUSY;
        }
        std::shared_ptr<AdmitRecord> oldest = a.recs.front();
        lk.unlock();
        cudaEventSynchronize(oldest->done);
        lk.lock();
        admit_reap(a);
      }
      adm = std::make_shared<AdmitRecord>();
      adm->bytes = need;
      if (cudaEventCreateWithFlags(&adm->done, cudaEventDisableTiming) != cudaSuccess) {
        set_err("cudaEventCreate failed");
        if (cur != p->device) cudaSetDevice(cur);
        return HC_ERR_CUDA;
      }
      a.inflight += need;
      a.recs.push_back(adm);
    }
  }

  hc_batch* bt = new hc_batch;
  bt->p = p;
  bt->stream = (cudaStream_t)b->stream;
  bt->n_inst = b->n_instances;
  bt->items = bt->n_inst * paths_eff;
  bt->step_budget = b->step_budget;
  bt->admission = adm;
  const int64_t items = bt->items;
  cudaStream_t st = bt->stream;
  auto fail = [&](hc_status s) {
    cudaStreamSynchronize(st);
    release_batch(bt);
    if (cur != p->device) cudaSetDevice(cur);
    return s;
  };
  std::function<hc_status(size_t, void**)> dalloc = [&](size_t bytes, void** q) -> hc_status {
    cudaError_t e = cudaMallocAsync(q, std::max<size_t>(bytes, 16), st);
    if (e != cudaSuccess) {
      set_err(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? HC_ERR_OOM : HC_ERR_CUDA;
    }
    bt->dev.push_back(*q);
    return HC_OK;
  };
#define HC_TRY(x)                     \
  do {                                \
    hc_status s_ = (x);               \
    if (s_ != HC_OK) return fail(s_); \
  } while (0)
#define HC_TRYCUDA(call)                                           \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      set_err(std::string(#call) + ": " + cudaGetErrorString(e_)); \
      return fail(HC_ERR_CUDA);                                    \
    }                                                              \
  } while (0)
  for (cudaEvent_t* e : {&bt->ev0, &bt->ev1, &bt->evk0, &bt->evk1, &bt->evk2})
    HC_TRYCUDA(cudaEventCreate(e));
  bt->owns_kernel_events = true;
  HC_TRYCUDA(cudaEventRecord(bt->ev0, st));

  Bufs B;
  B.paths = paths_eff;
  B.step_budget = b->step_budget;
  if (b->n_subset > 0) {
    void* q;
    const size_t bytes = sizeof(int64_t) * (size_t)bt->items;
    HC_TRY(dalloc(bytes, &q));
    // the caller may free path_ids on return: copy through a pinned buffer
    // the batch owns, so the upload stays asynchronous
    void* pin = nullptr;
    if (cudaMallocHost(&pin, bytes) != cudaSuccess) {
      set_err("cudaMallocHost failed");
      return fail(HC_ERR_OOM);
    }
    bt->pinned.push_back(pin);
    std::memcpy(pin, b->path_ids, bytes);
    HC_TRYCUDA(cudaMemcpyAsync(q, pin, bytes, cudaMemcpyHostToDevice, st));
    B.path_ids = (const int64_t*)q;
  }
  // ---- inputs on the device
  if (p->terms) {
    if (devptrs || is_device_ptr(b->p1)) {
      B.d_p1 = (const double2*)b->p1;
    } else {
      void* q;
      HC_TRY(dalloc(sizeof(double2) * p->P * bt->n_inst, &q));
      HC_TRYCUDA(cudaMemcpyAsync(q, b->p1, sizeof(double2) * p->P * bt->n_inst,
                                 cudaMemcpyHostToDevice, st));
      B.d_p1 = (const double2*)q;
    }
  } else {
    B.d_coef = p->d_coef;
    if (b->coef) {
      B.coef_stride = (int64_t)p->T;
      if (devptrs || is_device_ptr(b->coef)) {
        B.d_coef = b->coef;
      } else {
        void* q;
        HC_TRY(dalloc(sizeof(double) * 2 * p->T * bt->n_inst, &q));
        HC_TRYCUDA(cudaMemcpyAsync(q, b->coef, sizeof(double) * 2 * p->T * bt->n_inst,
                                   cudaMemcpyHostToDevice, st));
        B.d_coef = (const double*)q;
      }
    }
  }
  // ---- outputs and scratch
  std::vector<void*> d2h;
  HC_TRY(setup_outputs(bt, b, p->n, items, devptrs, B, d2h, dalloc));
  HC_TRY(alloc_scratch(p, bt->n_inst, B, [&](size_t bytes, void** q) { return dalloc(bytes, q); }));
  void* pin = pinned_slot_get();
  if (!pin) {
    set_err("cudaMallocHost failed");
    return fail(HC_ERR_OOM);
  }
  bt->h_ctl = (unsigned long long*)pin;
  bt->owns_ctl = true;
  std::memset(pin, 0, kCtlBytes);
  B.h_ctl = bt->h_ctl;
  bt->d_ctl = B.d_ctl;
  // ---- the computation
  const EnqEvents ev{bt->evk0, bt->evk1, bt->evk2, nullptr, nullptr, false};
  HC_TRY(enqueue_compute(p, bt->n_inst, B, st, retrack_stream(p->device), ev));
  for (size_t i = 0; i < bt->copies.size(); ++i) {
    void* dst = bt->copies[i].pinned ? bt->copies[i].pinned : bt->copies[i].dst;
    HC_TRYCUDA(cudaMemcpyAsync(dst, d2h[i], bt->copies[i].bytes, cudaMemcpyDeviceToHost, st));
  }
  HC_TRYCUDA(cudaEventRecord(bt->ev1, st));
  if (adm) HC_TRYCUDA(cudaEventRecord(adm->done, st));
  if (cur != p->device) cudaSetDevice(cur);
  *out = bt;
  return HC_OK;
#undef HC_TRY
#undef HC_TRYCUDA
}

}  // extern "C"

// ------------------------------------------------------------------ plans (CUDA graphs)
struct hc_plan {
  uint32_t magic = 0x48435050u;  // "HCPP"
  hc_problem* p = nullptr;
  int64_t n_inst = 0, items = 0;
  Bufs B;
  void* d_in = nullptr;  // inputs of the instances (coef or p1)
  size_t in_bytes = 0;
  std::vector<void*> dev;
  cudaEvent_t ek0 = nullptr, ek1 = nullptr, ek2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;  // graph edges of the re-tracking branch
  cudaEvent_t done = nullptr;  // recorded after each run's last copy
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {
void free_plan(hc_plan* pl) {
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->done) cudaEventSynchronize(pl->done);
  for (void* q : pl->dev) cudaFree(q);
  for (cudaEvent_t e : {pl->ek0, pl->ek1, pl->ek2, pl->fork, pl->join, pl->done})
    if (e) cudaEventDestroy(e);
  pl->magic = 0;
  delete pl;
}
}  // namespace

namespace hc {
bool destroy_plan_if(void* handle, uint32_t magic) {
  if (magic != 0x48435050u) return false;
  free_plan(static_cast<hc_plan*>(handle));
  return true;
}
}  // namespace hc

extern "C" {

hc_status hc_plan_create(hc_problem* p, int32_t n_instances, hc_plan** out) {
  g_err.clear();
  cudaGetLastError();  // launch errors checked below are this call's own
  if (!p || p->magic != kProblemMagic || n_instances < 1 || !out) {
    set_err("invalid plan arguments");
    return HC_ERR_INVALID;
  }
  int cur = 0;
  HC_CUDA(cudaGetDevice(&cur));
  if (cur != p->device) HC_CUDA(cudaSetDevice(p->device));
  hc_plan* pl = new hc_plan;
  pl->p = p;
  pl->n_inst = n_instances;
  pl->items = pl->n_inst * p->paths;
  pl->B.paths = p->paths;
  auto fail = [&](hc_status s) {
    free_plan(pl);
    if (cur != p->device) cudaSetDevice(cur);
    return s;
  };
  auto dalloc = [&](size_t bytes, void** q) -> hc_status {
    cudaError_t e = cudaMalloc(q, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
      set_err(std::string("cudaMalloc: ") + cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? HC_ERR_OOM : HC_ERR_CUDA;
    }
    pl->dev.push_back(*q);
    return HC_OK;
  };
  hc_status rc;
  const int64_t items = pl->items;
  const int n = p->n;
  pl->in_bytes = sizeof(double2) * (p->terms ? p->P : p->T) * pl->n_inst;
  if ((rc = dalloc(pl->in_bytes, &pl->d_in)) != HC_OK) return fail(rc);
  if (p->terms) {
    pl->B.d_p1 = (const double2*)pl->d_in;
  } else {
    pl->B.d_coef = (const double*)pl->d_in;
    pl->B.coef_stride = p->T;
  }
  void* q;
  if ((rc = dalloc(sizeof(double) * 2 * n * items, &q)) != HC_OK) return fail(rc);
  pl->B.d_x = (double*)q;
  if ((rc = dalloc(items, &q)) != HC_OK) return fail(rc);
  pl->B.d_status = (uint8_t*)q;
  if ((rc = dalloc(sizeof(int32_t) * 3 * items, &q)) != HC_OK) return fail(rc);
  pl->B.d_steps = (int32_t*)q;
  if ((rc = dalloc(sizeof(double) * items, &q)) != HC_OK) return fail(rc);
  pl->B.d_be = (double*)q;
  if ((rc = alloc_scratch(p, pl->n_inst, pl->B, dalloc)) != HC_OK) return fail(rc);
  for (cudaEvent_t* e : {&pl->ek0, &pl->ek1, &pl->ek2, &pl->fork, &pl->join, &pl->done})
    if (cudaEventCreate(e) != cudaSuccess) {
      set_err("cudaEventCreate failed");
      return fail(HC_ERR_CUDA);
    }
  // Capture on private streams (a shared stream could pick up another
  // thread's work while it is being captured); the re-tracking branch keeps
  // the high priority it has outside graphs.
  cudaStream_t cap = nullptr, cap_hi = nullptr;
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithPriority(&cap_hi, cudaStreamNonBlocking, hi) != cudaSuccess) {
    if (cap) cudaStreamDestroy(cap);
    set_err("cudaStreamCreate failed");
    return fail(HC_ERR_CUDA);
  }
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const EnqEvents ev{pl->ek0, pl->ek1, pl->ek2, pl->fork, pl->join, true};
    rc = enqueue_compute(p, pl->n_inst, pl->B, cap, cap_hi, ev);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    pl->graph = g;
    if (rc == HC_OK && e == cudaSuccess)
      e = cudaGraphInstantiateWithFlags(&pl->exec, pl->graph,
                                        cudaGraphInstantiateFlagUseNodePriority);
  }
  cudaStreamDestroy(cap_hi);
  cudaStreamDestroy(cap);
  if (rc != HC_OK) return fail(rc);
  if (e != cudaSuccess) {
    set_err(std::string("graph capture: ") + cudaGetErrorString(e));
    return fail(HC_ERR_CUDA);
  }
  if (cur != p->device) cudaSetDevice(cur);
  *out = pl;
  return HC_OK;
}

hc_status hc_plan_run(hc_plan* pl, const hc_batch_desc* b, hc_batch** out) {
  g_err.clear();
  cudaGetLastError();  // launch errors checked below are this call's own
  if (!pl || pl->magic != 0x48435050u || !out) {
    set_err("invalid plan");
    return HC_ERR_INVALID;
  }
  hc_problem* p = pl->p;
  hc_status rc = validate_batch(p, b);
  if (rc != HC_OK) return rc;
  if (b->n_instances != pl->n_inst) {
    set_err("batch size differs from the plan's");
    return HC_ERR_INVALID;
  }
  if (b->n_subset != 0 || b->step_budget != 0) {
    set_err("plans take no start subset and no step budget");
    return HC_ERR_INVALID;
  }
  int cur = 0;
  HC_CUDA(cudaGetDevice(&cur));
  if (cur != p->device) HC_CUDA(cudaSetDevice(p->device));
  const bool devptrs = (b->flags & HC_DEVICE_PTRS) != 0;
  hc_batch* bt = new hc_batch;
  bt->p = p;
  bt->stream = (cudaStream_t)b->stream;
  bt->n_inst = pl->n_inst;
  bt->items = pl->items;
  bt->evk0 = pl->ek0;
  bt->evk1 = pl->ek1;
  bt->evk2 = pl->ek2;
  bt->owns_kernel_events = false;
  cudaStream_t st = bt->stream;
  auto fail = [&](hc_status s) {
    cudaStreamSynchronize(st);
    release_batch(bt);
    if (cur != p->device) cudaSetDevice(cur);
    return s;
  };
#define HC_TRYCUDA(call)                                           \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) {                                       \
      set_err(std::string(#call) + ": " + cudaGetErrorString(e_)); \
      return fail(HC_ERR_CUDA);                                    \
    }                                                              \
  } while (0)
  HC_TRYCUDA(cudaEventCreate(&bt->ev0));
  HC_TRYCUDA(cudaEventCreate(&bt->ev1));
  void* pin = pinned_slot_get();
  if (!pin) {
    set_err("cudaMallocHost failed");
    return fail(HC_ERR_OOM);
  }
  bt->h_ctl = (unsigned long long*)pin;
  bt->owns_ctl = true;
  std::memset(pin, 0, kCtlBytes);
  // runs of one plan share its device buffers: each starts after the
  // previous one's last copy, whatever stream it was enqueued on
  HC_TRYCUDA(cudaStreamWaitEvent(st, pl->done, 0));
  HC_TRYCUDA(cudaEventRecord(bt->ev0, st));
  const void* src = p->terms ? (const void*)b->p1 : (const void*)b->coef;
  if (src) {
    HC_TRYCUDA(cudaMemcpyAsync(pl->d_in, src, pl->in_bytes, cudaMemcpyDefault, st));
  } else if (!p->terms) {  // every instance uses the problem's coefficients
    for (int64_t i = 0; i < pl->n_inst; ++i)
      HC_TRYCUDA(cudaMemcpyAsync(static_cast<char*>(pl->d_in) + i * 16 * p->T, p->d_coef,
                                 16 * (size_t)p->T, cudaMemcpyDeviceToDevice, st));
  }
  HC_TRYCUDA(cudaGraphLaunch(pl->exec, st));
  HC_TRYCUDA(cudaMemcpyAsync(bt->h_ctl, pl->B.d_ctl, kCtlBytes, cudaMemcpyDeviceToHost, st));
  const int64_t items = pl->items;
  const size_t xb = sizeof(double) * 2 * p->n * items;
  struct Out {
    void* user;
    const void* dev;
    size_t bytes;
  };
  const Out outs[4] = {{b->x_out, pl->B.d_x, xb},
                       {b->status_out, pl->B.d_status, (size_t)items},
                       {b->steps_out, pl->B.d_steps, sizeof(int32_t) * 3 * items},
                       {b->be_out, pl->B.d_be, sizeof(double) * items}};
  for (const Out& o : outs) {
    if (!o.user) continue;
    if (devptrs || is_pinned_host(o.user) || is_device_ptr(o.user)) {
      HC_TRYCUDA(cudaMemcpyAsync(o.user, o.dev, o.bytes, cudaMemcpyDefault, st));
    } else {
      void* pin;
      if (cudaMallocHost(&pin, o.bytes) != cudaSuccess) {
        set_err("cudaMallocHost failed");
        return fail(HC_ERR_OOM);
      }
      bt->pinned.push_back(pin);
      bt->copies.push_back({o.user, pin, o.bytes});
      HC_TRYCUDA(cudaMemcpyAsync(pin, o.dev, o.bytes, cudaMemcpyDeviceToHost, st));
    }
  }
  HC_TRYCUDA(cudaEventRecord(bt->ev1, st));
  HC_TRYCUDA(cudaEventRecord(pl->done, st));
#undef HC_TRYCUDA
  if (cur != p->device) cudaSetDevice(cur);
  *out = bt;
  return HC_OK;
}

hc_status hc_poll(hc_batch* b, int64_t timeout_us, hc_batch_result* r) {
  g_err.clear();
  if (!b || b->magic != kBatchMagic) {
    set_err("invalid batch");
    return HC_ERR_INVALID;
  }
  if (!b->done) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      cudaError_t e = cudaEventQuery(b->ev1);
      if (e == cudaSuccess) break;
      if (e != cudaErrorNotReady) {
        set_err(std::string("cudaEventQuery: ") + cudaGetErrorString(e));
        return HC_ERR_CUDA;
      }
      if (timeout_us == 0) return HC_PENDING;
      const auto el = std::chrono::duration_cast<std::chrono::microseconds>(
                          std::chrono::steady_clock::now() - t0)
                          .count();
      if (timeout_us > 0 && el >= timeout_us) return HC_PENDING;
      std::this_thread::sleep_for(std::chrono::microseconds(el < 200 ? 2 : 50));
    }
    for (auto& c : b->copies)
      if (c.pinned) std::memcpy(c.dst, c.pinned, c.bytes);
    b->done = true;
    admit_release(b->p->device, b->admission);
    b->admission.reset();
  }
  if (r) {
    std::memset(r, 0, sizeof(*r));
    r->paths = b->items;
    const unsigned long long* s = b->h_ctl + 8;
    r->finite = (int64_t)s[0];
    r->real = (int64_t)s[1];
    r->diverged = (int64_t)s[2];
    r->singular = (int64_t)s[3];
    r->failed = (int64_t)s[4];
    r->steps_accepted = (int64_t)s[5];
    r->steps_rejected = (int64_t)s[6];
    r->newton_iters = (int64_t)s[7];
    r->escalated = (int64_t)b->h_ctl[2] + (int64_t)b->h_ctl[7];
    r->esc_accepted = (int64_t)b->h_ctl[3];
    r->esc_rejected = (int64_t)b->h_ctl[4];
    r->esc_newton = (int64_t)b->h_ctl[5];
    auto elapsed = [](cudaEvent_t a, cudaEvent_t z) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, a, z) == cudaSuccess) return (double)ms;
      cudaGetLastError();  // not recorded: report 0 and leave no error behind
      return 0.0;
    };
    r->device_ms = elapsed(b->ev0, b->ev1);
    r->track_ms = elapsed(b->evk0, b->evk1);
    r->escalate_ms = elapsed(b->evk1, b->evk2);
    r->untracked = (int64_t)b->h_ctl[16];
    r->steps_total = (int64_t)b->h_ctl[17];
  }
  if (b->step_budget > 0 && b->h_ctl[16] > 0) {
    set_err("the batch's step budget ran out before every path started");
    return HC_ERR_TIMEOUT;
  }
  return HC_OK;
}

hc_status hc_set_memory_cap(int64_t max_device_bytes) {
  g_err.clear();
  if (max_device_bytes < 0) {
    set_err("negative memory cap");
    return HC_ERR_INVALID;
  }
  int dev = 0;
  HC_CUDA(cudaGetDevice(&dev));
  AdmitState& a = admit_state(dev);
  std::lock_guard<std::mutex> lk(a.mu);
  a.cap = max_device_bytes;
  return HC_OK;
}

hc_status hc_autotune(hc_problem* p, const hc_batch_desc* sample, hc_tune_report* report) {
  if (!p || p->magic != kProblemMagic || !sample) {
    set_err("invalid autotune arguments");
    return HC_ERR_INVALID;
  }
  const hc_settings base = p->s;
  std::vector<hc_settings> cand;
  hc_settings c = base;
  c.precision = HC_PREC_FP64;
  cand.push_back(c);  // the recovery reference
  for (int lanes : {0, 32}) {
    const bool has = p->terms ? hc::term_kernel(p->n, HC_PREC_MIXED, lanes).lanes == (lanes ? lanes : hc::term_kernel(p->n, HC_PREC_MIXED, 0).lanes)
                              : hc::dense_kernel(p->deg, p->n, HC_PREC_MIXED, lanes).lanes == (lanes ? lanes : p->L);
    if (lanes && (!has || p->n > 16)) continue;
    for (int block : {128, 64})
      for (double corr : {0.01, 0.1}) {
        c = base;
        c.precision = HC_PREC_MIXED;
        c.escalate = 1;
        c.lanes = lanes;
        c.block_threads = block;
        c.max_first_corr_fp32 = corr;
        cand.push_back(c);
      }
  }
  if (cand.size() > 16) cand.resize(16);
  std::vector<double> ms(cand.size(), 0.0);
  std::vector<int64_t> fin(cand.size(), -1);
  for (size_t i = 0; i < cand.size(); ++i) {
    p->s = cand[i];
    for (int rep = 0; rep < 2; ++rep) {
      hc_batch* b = nullptr;
      hc_status rc = hc_track_batch(p, sample, &b);
      if (rc != HC_OK) {
        p->s = base;
        return rc;
      }
      hc_batch_result r;
      rc = hc_poll(b, -1, &r);
      hc_destroy(b);
      if (rc != HC_OK) {
        p->s = base;
        return rc;
      }
      ms[i] = r.device_ms;
      fin[i] = r.finite;
    }
  }
  size_t best = 0;
  for (size_t i = 1; i < cand.size(); ++i)
    if (fin[i] >= fin[0] && ms[i] < ms[best]) best = i;
  p->s = cand[best];
  if (report) {
    std::memset(report, 0, sizeof(*report));
    report->n_candidates = (int32_t)cand.size();
    report->best = (int32_t)best;
    for (size_t i = 0; i < cand.size(); ++i) {
      report->ms[i] = ms[i];
      report->finite[i] = fin[i];
      report->tried[i] = cand[i];
    }
  }
  return HC_OK;
}

hc_status hc_autotune_cached(hc_problem* p, const hc_batch_desc* sample, const char* cache_path,
                             hc_tune_report* report) {
  if (!p || p->magic != kProblemMagic || !sample || !cache_path) {
    set_err("invalid autotune arguments");
    return HC_ERR_INVALID;
  }
  int deg = 0;
  for (int k = 0; k < p->T; ++k) {
    int d = 0;
    for (int j = 0; j < p->n; ++j) d += p->exps[(size_t)k * p->n + j];
    deg = std::max(deg, d);
  }
  char key[160];
  std::snprintf(key, sizeof(key), "kind=%d n=%d deg=%d terms=%d params=%d sym=%d prec=%d", p->kind,
                p->n, deg, p->T, p->P, p->n_group, p->s.precision);
  std::map<std::string, std::string> entries;  // key -> its JSON object text
  if (!read_tune_cache(cache_path, entries)) {
    set_err("hc_autotune_cached: the cache file is not a tuning cache");
    return HC_ERR_INVALID;
  }
  auto it = entries.find(key);
  if (it != entries.end()) {
    hc_settings s = p->s;
    if (!parse_tune_entry(it->second, s) || validate_settings(s) != HC_OK) {
      set_err("hc_autotune_cached: malformed cache entry");
      return HC_ERR_INVALID;
    }
    p->s = s;
    if (report) {
      std::memset(report, 0, sizeof(*report));
      report->cached = 1;
      report->tried[0] = s;
    }
    return HC_OK;
  }
  hc_tune_report local;
  hc_tune_report* rep = report ? report : &local;
  hc_status rc = hc_autotune(p, sample, rep);
  if (rc != HC_OK) return rc;
  char obj[200];
  std::snprintf(obj, sizeof(obj),
                "{\"precision\": %d, \"lanes\": %d, \"block_threads\": %d, "
                "\"max_first_corr_fp32\": %.17g}",
                p->s.precision, p->s.lanes, p->s.block_threads, p->s.max_first_corr_fp32);
  entries[key] = obj;
  if (!write_tune_cache(cache_path, entries)) {
    set_err("hc_autotune_cached: cannot write the cache file");
    return HC_ERR_INVALID;
  }
  return HC_OK;
}

void hc_destroy(void* handle) {
  if (!handle) return;
  const uint32_t magic = *static_cast<uint32_t*>(handle);
  if (hc::destroy_server_if(handle, magic)) return;
  if (magic == kProblemMagic) {
    free_problem(static_cast<hc_problem*>(handle));
  } else if (magic == kBatchMagic) {
    hc_batch* b = static_cast<hc_batch*>(handle);
    if (!b->done) cudaEventSynchronize(b->ev1);
    for (void* q : b->dev) cudaFreeAsync(q, b->stream);
    b->dev.clear();
    cudaStreamSynchronize(b->stream);
    release_batch(b);
  } else {
    hc::destroy_plan_if(handle, magic);
  }
}

}  // extern "C"

// ------------------------------------------------------------------ helpers shared with noalloc.cu
namespace hc {

void set_last_error(const char* msg) { set_err(msg); }

cudaError_t launch_dedupe(int64_t items, int64_t paths, int n, const float2* x32,
                          const uint8_t* status, float tol, const int64_t* list,
                          const unsigned long long* list_count, int64_t* out_list,
                          unsigned long long* out_count, double* t_io, cudaStream_t st) {
  if (list) {
    const int grid = (int)std::min<int64_t>((items + 7) / 8, 1024);
    dedupe_list_kernel<<<std::max(grid, 1), 256, 0, st>>>(paths, n, x32, status, tol, list,
                                                         list_count, out_list, out_count, t_io,
                                                         1, nullptr);
  } else {
    const int grid = (int)std::min<int64_t>((items + 255) / 256, 65535);
    dedupe_kernel<<<std::max(grid, 1), 256, 0, st>>>(items, paths, n, x32, status, tol, nullptr,
                                                    nullptr, out_list, out_count, t_io, 1,
                                                    nullptr);
  }
  return cudaGetLastError();
}

}  // namespace hc

namespace hc {
DevSettings to_dev_settings(const hc_settings& s) { return dev_settings(s); }
hc_status check_settings(const hc_settings& s) { return validate_settings(s); }
}  // namespace hc

// ------------------------------------------------------------------ hc_evaluate
extern "C" hc_status hc_evaluate(const hc_problem* p, int32_t precision, int32_t n_instances,
                                 const double* inputs, int64_t n_points, const int64_t* instance,
                                 const double* x, const double* t, double* H, double* Hx,
                                 double* Ht) {
  if (!p || p->magic != kProblemMagic || n_instances < 1 || n_points < 0 ||
      (n_points > 0 && (!instance || !x || !t || !H || !Hx || !Ht)) ||
      (precision != HC_PREC_FP64 && precision != HC_PREC_MIXED && precision != HC_PREC_DF) ||
      (p->kind != HC_TOTAL_DEGREE && !inputs)) {
    set_err("hc_evaluate: invalid arguments");
    return HC_ERR_INVALID;
  }
  for (int64_t k = 0; k < n_points; ++k)
    if (instance[k] < 0 || instance[k] >= n_instances) {
      set_err("hc_evaluate: an instance index is out of range");
      return HC_ERR_INVALID;
    }
  if (n_points == 0) return HC_OK;
  const hc::KernelRef k = p->terms ? hc::term_eval_kernel(p->n, precision)
                                   : hc::dense_eval_kernel(p->deg, p->n, precision);
  if (!k.fn) {
    set_err("hc_evaluate: no evaluation kernel for this problem shape");
    return HC_ERR_UNSUPPORTED;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != p->device) HC_CUDA(cudaSetDevice(p->device));
  const int n = p->n;
  std::vector<void*> mem;
  cudaStream_t st = nullptr;
  hc_status rc = HC_OK;
  auto dalloc = [&](size_t bytes, void** q) -> hc_status {
    *q = nullptr;
    if (cudaMalloc(q, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      set_err("hc_evaluate: cudaMalloc failed");
      return HC_ERR_OOM;
    }
    mem.push_back(*q);
    return HC_OK;
  };
  auto up = [&](const void* src, size_t bytes, void** q) -> hc_status {
    hc_status r = dalloc(bytes, q);
    if (r != HC_OK) return r;
    if (cudaMemcpyAsync(*q, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      set_err("hc_evaluate: upload failed");
      return HC_ERR_CUDA;
    }
    return HC_OK;
  };
  auto body = [&]() -> hc_status {
    HC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    hc::EvalPoints e;
    void *dinst, *dx, *dt, *dH, *dHx, *dHt;
    hc_status r;
    if ((r = up(instance, sizeof(int64_t) * n_points, &dinst)) != HC_OK ||
        (r = up(x, sizeof(double2) * n * n_points, &dx)) != HC_OK ||
        (r = up(t, sizeof(double) * n_points, &dt)) != HC_OK ||
        (r = dalloc(sizeof(double2) * n * n_points, &dH)) != HC_OK ||
        (r = dalloc(sizeof(double2) * n * n * n_points, &dHx)) != HC_OK ||
        (r = dalloc(sizeof(double2) * n * n_points, &dHt)) != HC_OK)
      return r;
    e.n_points = n_points;
    e.inst = (const int64_t*)dinst;
    e.x = (const double2*)dx;
    e.t = (const double*)dt;
    e.H = (double2*)dH;
    e.Hx = (double2*)dHx;
    e.Ht = (double2*)dHt;
    const int threads = hc::kBlock;
    size_t smem = 0;
    void* argp = nullptr;
    hc::DenseEvalArgs da;
    hc::TermEvalArgs ta;
    std::memset(&da, 0, sizeof(da));
    std::memset(&ta, 0, sizeof(ta));
    if (p->terms) {
      void* dp1;
      if ((r = up(inputs, sizeof(double2) * p->P * n_instances, &dp1)) != HC_OK) return r;
      hc::TermArgs& a = ta.a;
      a.rec = p->d_rec;
      a.s64 = p->d_s64;
      a.sdf = p->d_sdf;
      a.TT = p->TT;
      a.P = p->P;
      a.ls = p->L;
      a.extra = p->extra;
      a.p0 = p->d_p0;
      a.p1 = (const double2*)dp1;
      a.start = p->d_start;
      if (p->coef_mode) {
        const int64_t slots = (int64_t)p->TT * p->L, cnt = slots * n_instances;
        void *dc, *dcf, *dcdf;
        if ((r = dalloc(sizeof(double2) * cnt, &dc)) != HC_OK ||
            (r = dalloc(sizeof(float2) * cnt, &dcf)) != HC_OK ||
            (r = dalloc(sizeof(hc::cdf) * cnt, &dcdf)) != HC_OK)
          return r;
        const int gs = (int)std::min<int64_t>((cnt + 255) / 256, 4096);
        stage_coef_kernel<<<std::max(gs, 1), 256, 0, st>>>(
            n_instances, slots, std::max(p->maxpf, 1), p->d_cpar, p->d_s64, p->d_c0,
            (const double2*)dp1, p->P, (double2*)dc, (float2*)dcf, (hc::cdf*)dcdf);
        HC_CUDA(cudaGetLastError());
        a.coef_mode = 1;
        a.c0 = p->d_c0;
        a.c0f = p->d_c0f;
        a.c0df = p->d_c0df;
        a.dc = (const double2*)dc;
        a.dcf = (const float2*)dcf;
        a.dcdf = (const hc::cdf*)dcdf;
      }
      ta.e = e;
      smem = (size_t)hc::block_smem_bytes(k.lanes, p->extra, k.acc_bytes, threads, 0, k.vx);
      argp = &ta;
    } else {
      const void* coef = p->d_coef;
      int64_t stride = 0;
      if (inputs) {
        void* dcoef;
        if ((r = up(inputs, sizeof(double2) * p->T * n_instances, &dcoef)) != HC_OK) return r;
        coef = dcoef;
        stride = p->T;
      }
      void *E, *D32 = nullptr, *D64 = nullptr, *Ddf = nullptr;
      const size_t es = (size_t)p->Estride * n_instances, ds = (size_t)p->Dstride * n_instances;
      if ((r = dalloc(sizeof(double2) * es, &E)) != HC_OK) return r;
      if (precision == HC_PREC_MIXED && (r = dalloc(sizeof(float2) * ds, &D32)) != HC_OK) return r;
      if (precision == HC_PREC_FP64 && (r = dalloc(sizeof(double2) * ds, &D64)) != HC_OK) return r;
      if (precision == HC_PREC_DF && (r = dalloc(sizeof(float4) * ds, &Ddf)) != HC_OK) return r;
      HC_CUDA(cudaMemsetAsync(E, 0, sizeof(double2) * es, st));
      if (D32) HC_CUDA(cudaMemsetAsync(D32, 0, sizeof(float2) * ds, st));
      if (D64) HC_CUDA(cudaMemsetAsync(D64, 0, sizeof(double2) * ds, st));
      if (Ddf) HC_CUDA(cudaMemsetAsync(Ddf, 0, sizeof(float4) * ds, st));
      const int64_t work = (int64_t)n_instances * (p->T + p->ndc);
      const int grid = (int)std::min<int64_t>((work + 255) / 256, 4096);
      stage_dense_kernel<<<std::max(grid, 1), 256, 0, st>>>(
          n_instances, p->T, (const double2*)coef, stride, p->d_emap, p->ndc, p->d_dterm,
          p->d_dslot, p->d_dmult, (double2*)E, nullptr, p->Estride, (float2*)D32,
          (double2*)D64, (float4*)Ddf, p->Dstride);
      HC_CUDA(cudaGetLastError());
      hc::DenseArgs& a = da.a;
      a.D32 = (const cx<float>*)D32;
      a.D64 = (const cx<double>*)D64;
      a.Ddf = (const cx<hc::df>*)Ddf;
      a.E = (const cx<double>*)E;
      a.Dstride = p->Dstride;
      a.Estride = p->Estride;
      a.gamma = cx<double>{p->gamma[0], p->gamma[1]};
      a.gamma32 = cx<float>{(float)p->gamma[0], (float)p->gamma[1]};
      a.gammadf = hc::split_cdf_host(p->gamma[0], p->gamma[1]);
      da.e = e;
      smem = (size_t)hc::block_smem_bytes(k.lanes, k.extra, 0, threads, 0, k.vx);
      argp = &da;
    }
    if (smem > 48 * 1024)
      HC_CUDA(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t groups = (n_points + threads / k.lanes - 1) / (threads / k.lanes);
    const int grid = (int)std::min<int64_t>(groups, 65535);
    void* argv[] = {argp};
    HC_CUDA(cudaLaunchKernel(k.fn, dim3((unsigned)grid), dim3(threads), argv, smem, st));
    HC_CUDA(cudaMemcpyAsync(H, dH, sizeof(double2) * n * n_points, cudaMemcpyDeviceToHost, st));
    HC_CUDA(cudaMemcpyAsync(Hx, dHx, sizeof(double2) * n * n * n_points, cudaMemcpyDeviceToHost,
                            st));
    HC_CUDA(cudaMemcpyAsync(Ht, dHt, sizeof(double2) * n * n_points, cudaMemcpyDeviceToHost, st));
    HC_CUDA(cudaStreamSynchronize(st));
    return HC_OK;
  };
  rc = body();
  if (st) cudaStreamSynchronize(st);
  for (void* q : mem) cudaFree(q);
  if (st) cudaStreamDestroy(st);
  if (cur != p->device) cudaSetDevice(cur);
  return rc;
}

// ------------------------------------------------------------------ hc_stream
// Continuous admission into a running launch: a ring of instance slots in
// device memory, a resident tracking launch that takes the next path of the
// next published slot whenever one of its lane groups frees up, and per slot
// the re-tracking tiers of enqueue_compute (duplicate check, high-precision
// residual re-track, last tier) once the slot's paths are done.
struct hc_stream {
  uint32_t magic = 0x48435354u;  // "HCST"
  hc_problem* p = nullptr;
  int S = 0;                     // slots
  int64_t paths = 0;
  int64_t idle_ns = 0;
  int64_t next_ticket = 0;
  bool launched = false;
  int grid = 0, threads = 0;
  size_t smem = 0;
  hc::KernelRef kt{}, kr{}, kl{};  // tracking, re-tracking, last tier
  cudaStream_t ks = nullptr, cs = nullptr;  // resident launch, copies and staging
  std::vector<cudaStream_t> es;             // re-tracking streams, slot k on es[k % size]
  cudaEvent_t kdone = nullptr;
  std::vector<cudaEvent_t> edone;
  std::vector<int> state;        // 0 free, 1 tracking, 2 escalating
  std::vector<int64_t> ticket;   // ticket held by each slot
  // pinned host words: completion flags (mapped, written by the device) and
  // the sources of the tail and stop copies
  unsigned long long* h_flag = nullptr;
  unsigned long long* h_tailv = nullptr;  // [S] tail value published with each slot
  unsigned int* h_stopv = nullptr;
  unsigned long long* d_flag = nullptr;   // device view of h_flag
  unsigned long long* d_tail = nullptr;   // device memory
  unsigned int* d_stop = nullptr;         // device memory
  // device ring
  std::vector<void*> mem;
  unsigned long long* d_queue = nullptr;
  unsigned int* d_done = nullptr;
  unsigned long long* d_esc = nullptr;  // [S] per-slot counters
  unsigned long long* d_dup = nullptr;  // [S]
  unsigned long long* d_sctl = nullptr; // [S][8] per-slot queues and step sums
  double2* d_in = nullptr;              // [S][T] coefficients or [S][P] parameters
  double2 *E = nullptr, *D64 = nullptr;
  hc::cdf* Edf = nullptr;
  float2* D32 = nullptr;
  float4* Ddf = nullptr;
  double2* dc = nullptr;
  float2* dcf = nullptr;
  hc::cdf* dcdf = nullptr;
  double2* x = nullptr;
  uint8_t* st = nullptr;
  int32_t* steps = nullptr;
  double* be = nullptr;
  int64_t* esc_list = nullptr;
  int64_t* dup_list = nullptr;
  double* t_io = nullptr;
  float2* x32 = nullptr;
};

namespace {
constexpr uint32_t kStreamMagic = 0x48435354u;

void free_stream(hc_stream* s) {
  if (s->ks) cudaStreamSynchronize(s->ks);
  for (cudaStream_t e : s->es)
    if (e) cudaStreamSynchronize(e);
  if (s->cs) cudaStreamSynchronize(s->cs);
  for (void* q : s->mem) cudaFree(q);
  for (cudaEvent_t e : s->edone)
    if (e) cudaEventDestroy(e);
  if (s->kdone) cudaEventDestroy(s->kdone);
  if (s->ks) cudaStreamDestroy(s->ks);
  if (s->cs) cudaStreamDestroy(s->cs);
  for (cudaStream_t e : s->es)
    if (e) cudaStreamDestroy(e);
  if (s->h_flag) cudaFreeHost(s->h_flag);
  delete s;
}

// the launch descriptor common to the resident launch and a slot's tiers
hc::LaunchCommon stream_common(const hc_stream* s) {
  hc::LaunchCommon c;
  std::memset(&c, 0, sizeof(c));
  c.s = dev_settings(s->p->s);
  c.paths = s->paths;
  return c;
}
}  // namespace

extern "C" hc_status hc_stream_create(hc_problem* p, int32_t slots, int64_t idle_us,
                                      hc_stream** out) {
  if (!p || p->magic != kProblemMagic || !out || slots < 1 || slots > 4096 || idle_us < 1 ||
      idle_us > 10000000) {
    set_err("hc_stream_create: invalid arguments (slots 1..4096, idle_us 1..1e7)");
    return HC_ERR_INVALID;
  }
  *out = nullptr;
  const int prec = p->s.precision;
  const bool mixed = prec == HC_PREC_MIXED;
  const int n = p->n;
  if (!mixed) {
    set_err("hc_stream_create: streams track in mixed precision (settings.precision)");
    return HC_ERR_UNSUPPORTED;
  }
  hc_stream* s = new hc_stream();
  s->p = p;
  s->S = slots;
  s->paths = p->paths;
  s->idle_ns = idle_us * 1000;
  s->state.assign(slots, 0);
  s->ticket.assign(slots, -1);
  s->edone.assign(slots, nullptr);
  s->kt = hc::ring_kernel(p->terms, p->deg, n);
  if (p->terms) {
    s->kr = hc::term_kernel(n, HC_PREC_MIXED, 0);
    s->kl = hc::term_kernel(n, hc::last_tier_precision(p->s), 0);
  } else {
    s->kr = retrack_kernel(p->deg, n, HC_PREC_MIXED);
    s->kl = retrack_kernel(p->deg, n, hc::last_tier_precision(p->s));
  }
  if (!s->kt.fn || !s->kr.fn || !s->kl.fn) {
    delete s;
    set_err("hc_stream_create: no kernel for this problem shape");
    return HC_ERR_UNSUPPORTED;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != p->device && cudaSetDevice(p->device) != cudaSuccess) {
    delete s;
    set_err("hc_stream_create: cudaSetDevice failed");
    return HC_ERR_CUDA;
  }
  auto fail = [&](hc_status rc, const char* what) {
    set_err(std::string("hc_stream_create: ") + what);
    free_stream(s);
    if (cur != p->device) cudaSetDevice(cur);
    return rc;
  };
  auto dalloc = [&](size_t bytes, auto** q) -> bool {
    void* v = nullptr;
    if (cudaMalloc(&v, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
    s->mem.push_back(v);
    *q = reinterpret_cast<std::remove_pointer_t<decltype(q)>>(v);
    return cudaMemset(v, 0, std::max<size_t>(bytes, 16)) == cudaSuccess;
  };
  if (cudaStreamCreateWithFlags(&s->ks, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->kdone, cudaEventDisableTiming) != cudaSuccess)
    return fail(HC_ERR_CUDA, "stream or event creation failed");
  // the slots' re-tracking tiers overlap on several streams (one stream
  // would queue every slot's latency-bound tail behind the previous one)
  s->es.assign(std::min(slots, 32), nullptr);
  for (auto& e : s->es)
    if (cudaStreamCreateWithFlags(&e, cudaStreamNonBlocking) != cudaSuccess)
      return fail(HC_ERR_CUDA, "stream creation failed");
  for (int k = 0; k < slots; ++k)
    if (cudaEventCreateWithFlags(&s->edone[k], cudaEventDisableTiming) != cudaSuccess)
      return fail(HC_ERR_CUDA, "event creation failed");
  // pinned host words: one completion flag per slot (mapped), the tail value
  // of each slot's publication and the stop word (copy sources)
  void* h = nullptr;
  const size_t hbytes = 16 * (size_t)slots + 16;
  if (cudaHostAlloc(&h, hbytes, cudaHostAllocMapped) != cudaSuccess)
    return fail(HC_ERR_OOM, "cudaHostAlloc failed");
  std::memset(h, 0, hbytes);
  s->h_flag = static_cast<unsigned long long*>(h);
  s->h_tailv = s->h_flag + slots;
  s->h_stopv = reinterpret_cast<unsigned int*>(s->h_tailv + slots);
  void* dh = nullptr;
  if (cudaHostGetDevicePointer(&dh, h, 0) != cudaSuccess)
    return fail(HC_ERR_CUDA, "cudaHostGetDevicePointer failed");
  s->d_flag = static_cast<unsigned long long*>(dh);
  const int64_t ring = (int64_t)slots * s->paths;
  const size_t in_per = p->terms ? (size_t)p->P : (size_t)p->T;
  bool ok = dalloc(8, &s->d_queue) && dalloc(8, &s->d_tail) && dalloc(8, &s->d_stop) &&
            dalloc(4 * (size_t)slots, &s->d_done) &&
            dalloc(8 * (size_t)slots, &s->d_esc) && dalloc(8 * (size_t)slots, &s->d_dup) &&
            dalloc(64 * (size_t)slots, &s->d_sctl) &&
            dalloc(sizeof(double2) * in_per * slots, &s->d_in) &&
            dalloc(sizeof(double2) * n * ring, &s->x) && dalloc((size_t)ring, &s->st) &&
            dalloc(sizeof(int32_t) * 3 * ring, &s->steps) && dalloc(sizeof(double) * ring, &s->be) &&
            dalloc(sizeof(int64_t) * ring, &s->esc_list) &&
            dalloc(sizeof(int64_t) * ring, &s->dup_list) && dalloc(sizeof(double) * ring, &s->t_io) &&
            dalloc(sizeof(float2) * n * ring, &s->x32);
  if (ok && !p->terms) {
    const int last = hc::last_tier_precision(p->s);
    const size_t es = (size_t)p->Estride * slots, ds = (size_t)p->Dstride * slots;
    ok = dalloc(sizeof(double2) * es, &s->E) &&
         (!mixed || (dalloc(sizeof(hc::cdf) * es, &s->Edf) && dalloc(sizeof(float2) * ds, &s->D32))) &&
         ((prec != HC_PREC_FP64 && !(mixed && last == HC_PREC_FP64)) ||
          dalloc(sizeof(double2) * ds, &s->D64)) &&
         ((prec != HC_PREC_DF && !(mixed && last == HC_PREC_DF)) ||
          dalloc(sizeof(float4) * ds, &s->Ddf));
  }
  if (ok && p->terms && p->coef_mode) {
    const size_t e = (size_t)p->TT * p->L * slots;
    ok = dalloc(sizeof(double2) * e, &s->dc) && dalloc(sizeof(float2) * e, &s->dcf) &&
         dalloc(sizeof(hc::cdf) * e, &s->dcdf);
  }
  if (!ok) return fail(HC_ERR_OOM, "device allocation failed");
  // the resident launch leaves a quarter of the SMs' block slots to the
  // staging and re-tracking launches that run beside it
  s->threads = std::max(main_threads(p->s), s->kt.lanes);
  s->smem = p->terms ? (size_t)hc::block_smem_bytes(s->kt.lanes, p->extra, s->kt.acc_bytes,
                                                     s->threads, s->kt.eg_bytes, s->kt.vx)
                     : (size_t)hc::block_smem_bytes(s->kt.lanes, s->kt.extra, 0, s->threads,
                                                    s->kt.eg_bytes, s->kt.vx);
  if (s->smem > 48 * 1024 &&
      cudaFuncSetAttribute(s->kt.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)s->smem) != cudaSuccess)
    return fail(HC_ERR_CUDA, "shared memory attribute");
  const Occ o = occupancy(s->kt.fn, s->smem, s->threads);
  s->grid = std::max(o.sms, (o.blocks * o.sms * 3) / 4);
  if (cur != p->device) cudaSetDevice(cur);
  *out = s;
  return HC_OK;
}

namespace {
// Tracking arguments for slot `slot` viewed as a one-instance batch (slot <
// 0: the whole ring, for the resident launch).
hc::DenseArgs stream_dense_args(const hc_stream* s, int64_t slot) {
  const hc_problem* p = s->p;
  const int64_t o = slot < 0 ? 0 : slot;
  hc::DenseArgs a;
  std::memset(&a, 0, sizeof(a));
  a.c = stream_common(s);
  a.D32 = s->D32 ? (const cx<float>*)(s->D32 + o * p->Dstride) : nullptr;
  a.D64 = s->D64 ? (const cx<double>*)(s->D64 + o * p->Dstride) : nullptr;
  a.Ddf = s->Ddf ? (const cx<hc::df>*)(s->Ddf + o * p->Dstride) : nullptr;
  a.E = (const cx<double>*)(s->E + o * p->Estride);
  a.Edf = s->Edf ? s->Edf + o * p->Estride : nullptr;
  a.Dstride = p->Dstride;
  a.Estride = p->Estride;
  a.gamma = cx<double>{p->gamma[0], p->gamma[1]};
  a.gamma32 = cx<float>{(float)p->gamma[0], (float)p->gamma[1]};
  a.gammadf = hc::split_cdf_host(p->gamma[0], p->gamma[1]);
  return a;
}

hc::TermArgs stream_term_args(const hc_stream* s, int64_t slot) {
  const hc_problem* p = s->p;
  const int64_t o = slot < 0 ? 0 : slot;
  hc::TermArgs a;
  std::memset(&a, 0, sizeof(a));
  a.c = stream_common(s);
  a.rec = p->d_rec;
  a.s64 = p->d_s64;
  a.sdf = p->d_sdf;
  a.TT = p->TT;
  a.P = p->P;
  a.ls = p->L;
  a.extra = p->extra;
  a.p0 = p->d_p0;
  a.p1 = s->d_in + o * p->P;
  a.start = p->d_start;
  if (p->coef_mode) {
    const int64_t e = (int64_t)p->TT * p->L * o;
    a.coef_mode = 1;
    a.c0 = p->d_c0;
    a.c0f = p->d_c0f;
    a.c0df = p->d_c0df;
    a.dc = s->dc + e;
    a.dcf = s->dcf + e;
    a.dcdf = s->dcdf + e;
  }
  return a;
}

// outputs and re-tracking state of one slot (or the ring, slot < 0)
void stream_outputs(const hc_stream* s, int64_t slot, hc::LaunchCommon& c) {
  const int64_t o = (slot < 0 ? 0 : slot) * s->paths;
  const int n = s->p->n;
  const bool esc = s->p->s.precision == HC_PREC_MIXED && s->p->s.escalate;
  c.x_out = reinterpret_cast<double*>(s->x + o * n);
  c.status_out = s->st + o;
  c.steps_out = s->steps + o * 3;
  c.be_out = s->be + o;
  if (esc) {
    c.esc_list = s->esc_list + o;
    c.dup_list = s->dup_list + o;
    c.t_io = s->t_io + o;
    c.x32_out = s->x32 + o * n;
    c.esc_count = s->d_esc + (slot < 0 ? 0 : slot);
    c.dup_count = s->d_dup + (slot < 0 ? 0 : slot);
  }
}

bool stream_running(hc_stream* s) {
  return s->launched && cudaEventQuery(s->kdone) == cudaErrorNotReady;
}

// (Re)launch the resident tracking launch if it is not running and a
// published slot still has paths to claim.
hc_status stream_kick(hc_stream* s) {
  bool pending = false;
  for (int k = 0; k < s->S; ++k)
    if (s->state[k] == 1 &&
        __atomic_load_n(&s->h_flag[k], __ATOMIC_ACQUIRE) != (unsigned long long)(s->ticket[k] / s->S + 1))
      pending = true;
  if (!pending || stream_running(s)) return HC_OK;
  hc::LaunchCommon c = stream_common(s);
  stream_outputs(s, -1, c);
  c.queue = s->d_queue;
  c.ring_items = (unsigned long long)s->S * s->paths;
  c.ring_tail = s->d_tail;
  c.ring_stop = s->d_stop;
  c.ring_idle_ns = (unsigned long long)s->idle_ns;
  c.ring_done = s->d_done;
  c.ring_flag = s->d_flag;
  void* argp;
  hc::DenseArgs da;
  hc::TermArgs ta;
  if (s->p->terms) {
    ta = stream_term_args(s, -1);
    ta.c = c;
    argp = &ta;
  } else {
    da = stream_dense_args(s, -1);
    da.c = c;
    argp = &da;
  }
  void* argv[] = {argp};
  HC_CUDA(cudaLaunchKernel(s->kt.fn, dim3((unsigned)s->grid), dim3(s->threads), argv, s->smem,
                           s->ks));
  HC_CUDA(cudaEventRecord(s->kdone, s->ks));
  s->launched = true;
  return HC_OK;
}
}  // namespace

namespace {
// The re-tracking tiers of one slot whose tracking is complete (as
// enqueue_compute runs them for a batch), then the slot's completion event.
hc_status stream_escalate(hc_stream* s, int64_t slot) {
  const hc_problem* p = s->p;
  const bool esc = p->s.precision == HC_PREC_MIXED && p->s.escalate;
  cudaStream_t es = s->es[slot % (int64_t)s->es.size()];
  if (esc) {
    const int n = p->n;
    const int64_t P = s->paths, o = slot * P;
    unsigned long long* ctl = s->d_sctl + slot * 8;
    HC_CUDA(hc::launch_dedupe(P, P, n, s->x32 + o * n, s->st + o, 1e-6f, nullptr, nullptr,
                              s->dup_list + o, s->d_dup + slot, s->t_io + o, es));
    hc::LaunchCommon cd = stream_common(s);
    stream_outputs(s, slot, cd);
    cd.count_dev = s->d_dup + slot;
    cd.items = s->dup_list + o;
    cd.queue = ctl + 0;
    cd.start_hi = 1;
    cd.spread = 1;
    cd.dup_list = nullptr;
    cd.dup_count = nullptr;
    hc::LaunchCommon ce = stream_common(s);
    stream_outputs(s, slot, ce);
    ce.count_dev = s->d_esc + slot;
    ce.items = s->esc_list + o;
    ce.queue = ctl + 1;
    ce.esc_list = nullptr;
    ce.x32_out = nullptr;
    ce.esc_steps = ctl + 2;
    ce.spread = 1;
    ce.dup_list = nullptr;
    ce.dup_count = nullptr;
    // one warp per block: the blocks must fit beside the resident launch's
    // (the double-float kernels hold up to 255 registers a thread)
    auto run = [&](const hc::KernelRef& k, const hc::LaunchCommon& c) -> hc_status {
      const int th = 32;
      if (p->terms) {
        hc::TermArgs a = stream_term_args(s, slot);
        a.c = c;
        const size_t sm = (size_t)hc::block_smem_bytes(k.lanes, p->extra, k.acc_bytes, th,
                                                       k.eg_bytes, k.vx);
        return launch_generic(k, &a, sm, P, es, th);
      }
      hc::DenseArgs a = stream_dense_args(s, slot);
      a.c = c;
      return launch_tracker(k, a, P, es, th);
    };
    hc_status rc;
    if ((rc = run(s->kr, cd)) != HC_OK) return rc;
    HC_CUDA(hc::launch_dedupe(P, P, n, s->x32 + o * n, s->st + o, 1e-6f, s->dup_list + o,
                              s->d_dup + slot, s->esc_list + o, s->d_esc + slot, s->t_io + o,
                              es));
    if ((rc = run(s->kl, ce)) != HC_OK) return rc;
  }
  HC_CUDA(cudaEventRecord(s->edone[slot], es));
  return HC_OK;
}
}  // namespace

namespace {
// Starts the re-tracking tiers of every slot whose tracking is complete and
// (re)launches the resident launch if published paths wait for it.
hc_status stream_progress(hc_stream* s) {
  for (int k = 0; k < s->S; ++k)
    if (s->state[k] == 1 && __atomic_load_n(&s->h_flag[k], __ATOMIC_ACQUIRE) ==
                                (unsigned long long)(s->ticket[k] / s->S + 1)) {
      const hc_status rc = stream_escalate(s, k);
      if (rc != HC_OK) return rc;
      s->state[k] = 2;
    }
  return stream_kick(s);
}
}  // namespace

extern "C" hc_status hc_stream_submit(hc_stream* s, const double* inputs, int64_t* ticket) {
  if (!s || s->magic != kStreamMagic || !ticket || (s->p->kind != HC_TOTAL_DEGREE && !inputs)) {
    set_err("hc_stream_submit: invalid arguments");
    return HC_ERR_INVALID;
  }
  const hc_problem* p = s->p;
  const int64_t k = s->next_ticket;
  const int slot = (int)(k % s->S);
  if (s->state[slot] != 0) {
    const hc_status rc = stream_progress(s);
    if (rc != HC_OK) return rc;
    set_err("hc_stream_submit: every slot holds a request that has not been collected");
    return HC_ERR_BUSY;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != p->device) HC_CUDA(cudaSetDevice(p->device));
  auto body = [&]() -> hc_status {
    const size_t in_per = p->terms ? (size_t)p->P : (size_t)p->T;
    double2* in = s->d_in + (size_t)slot * in_per;
    if (inputs)
      HC_CUDA(cudaMemcpyAsync(in, inputs, sizeof(double2) * in_per, cudaMemcpyHostToDevice, s->cs));
    else
      HC_CUDA(cudaMemcpyAsync(in, p->d_coef, sizeof(double2) * in_per, cudaMemcpyDeviceToDevice,
                              s->cs));
    HC_CUDA(cudaMemsetAsync(s->d_esc + slot, 0, 8, s->cs));
    HC_CUDA(cudaMemsetAsync(s->d_dup + slot, 0, 8, s->cs));
    HC_CUDA(cudaMemsetAsync(s->d_sctl + (size_t)slot * 8, 0, 64, s->cs));
    HC_CUDA(cudaMemsetAsync(s->steps + (size_t)slot * s->paths * 3, 0,
                            sizeof(int32_t) * 3 * s->paths, s->cs));
    if (!p->terms) {
      const size_t Es = p->Estride, Ds = p->Dstride;
      HC_CUDA(cudaMemsetAsync(s->E + slot * Es, 0, sizeof(double2) * Es, s->cs));
      if (s->Edf) HC_CUDA(cudaMemsetAsync(s->Edf + slot * Es, 0, sizeof(hc::cdf) * Es, s->cs));
      if (s->D32) HC_CUDA(cudaMemsetAsync(s->D32 + slot * Ds, 0, sizeof(float2) * Ds, s->cs));
      if (s->D64) HC_CUDA(cudaMemsetAsync(s->D64 + slot * Ds, 0, sizeof(double2) * Ds, s->cs));
      if (s->Ddf) HC_CUDA(cudaMemsetAsync(s->Ddf + slot * Ds, 0, sizeof(float4) * Ds, s->cs));
      const int grid = (int)std::min<int64_t>((p->T + p->ndc + 255) / 256, 4096);
      stage_dense_kernel<<<std::max(grid, 1), 256, 0, s->cs>>>(
          1, p->T, in, 0, p->d_emap, p->ndc, p->d_dterm, p->d_dslot, p->d_dmult,
          s->E + slot * Es, s->Edf ? s->Edf + slot * Es : nullptr, Es,
          s->D32 ? s->D32 + slot * Ds : nullptr, s->D64 ? s->D64 + slot * Ds : nullptr,
          s->Ddf ? s->Ddf + slot * Ds : nullptr, Ds);
      HC_CUDA(cudaGetLastError());
    } else if (p->coef_mode) {
      const int64_t slots = (int64_t)p->TT * p->L;
      const int gs = (int)std::min<int64_t>((slots + 255) / 256, 4096);
      stage_coef_kernel<<<std::max(gs, 1), 256, 0, s->cs>>>(
          1, slots, std::max(p->maxpf, 1), p->d_cpar, p->d_s64, p->d_c0, in, p->P,
          s->dc + slot * slots, s->dcf + slot * slots, s->dcdf + slot * slots);
      HC_CUDA(cudaGetLastError());
    }
    // publish the slot's tickets behind its inputs on the same stream (the
    // resident launch reads the tail with acquire semantics)
    s->h_tailv[slot] = (unsigned long long)(k + 1) * s->paths;
    HC_CUDA(cudaMemcpyAsync(s->d_tail, s->h_tailv + slot, 8, cudaMemcpyHostToDevice, s->cs));
    s->ticket[slot] = k;
    s->state[slot] = 1;
    ++s->next_ticket;
    *ticket = k;
    return stream_progress(s);
  };
  const hc_status rc = body();
  if (cur != p->device) cudaSetDevice(cur);
  return rc;
}

extern "C" hc_status hc_stream_poll(hc_stream* s, int64_t ticket, int64_t timeout_us,
                                    double* x_out, uint8_t* status_out, int32_t* steps_out,
                                    double* be_out) {
  if (!s || s->magic != kStreamMagic || ticket < 0 || !x_out || !status_out) {
    set_err("hc_stream_poll: invalid arguments");
    return HC_ERR_INVALID;
  }
  const int slot = (int)(ticket % s->S);
  if (s->ticket[slot] != ticket || s->state[slot] == 0) {
    set_err("hc_stream_poll: unknown or already collected ticket");
    return HC_ERR_INVALID;
  }
  const hc_problem* p = s->p;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != p->device) HC_CUDA(cudaSetDevice(p->device));
  const auto t0 = std::chrono::steady_clock::now();
  auto body = [&]() -> hc_status {
    for (;;) {
      {  // every waiting slot's next stage, not only this ticket's
        const hc_status rc = stream_progress(s);
        if (rc != HC_OK) return rc;
      }
      if (s->state[slot] == 2) {
        const cudaError_t q = cudaEventQuery(s->edone[slot]);
        if (q == cudaSuccess) {
          const int64_t P = s->paths, o = (int64_t)slot * P;
          const int n = p->n;
          HC_CUDA(cudaMemcpyAsync(x_out, s->x + o * n, sizeof(double2) * n * P,
                                  cudaMemcpyDeviceToHost, s->cs));
          HC_CUDA(cudaMemcpyAsync(status_out, s->st + o, (size_t)P, cudaMemcpyDeviceToHost, s->cs));
          if (steps_out)
            HC_CUDA(cudaMemcpyAsync(steps_out, s->steps + o * 3, sizeof(int32_t) * 3 * P,
                                    cudaMemcpyDeviceToHost, s->cs));
          if (be_out)
            HC_CUDA(cudaMemcpyAsync(be_out, s->be + o, sizeof(double) * P, cudaMemcpyDeviceToHost,
                                    s->cs));
          HC_CUDA(cudaStreamSynchronize(s->cs));
          s->state[slot] = 0;
          return HC_OK;
        }
        if (q != cudaErrorNotReady) HC_CUDA(q);
      }
      const double us =
          std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
      if (timeout_us >= 0 && us >= (double)timeout_us) return HC_ERR_TIMEOUT;
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  };
  const hc_status rc = body();
  if (cur != p->device) cudaSetDevice(cur);
  return rc;
}

extern "C" hc_status hc_stream_destroy(hc_stream* s) {
  if (!s) return HC_OK;
  if (s->magic != kStreamMagic) {
    set_err("hc_stream_destroy: not a stream");
    return HC_ERR_INVALID;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != s->p->device) cudaSetDevice(s->p->device);
  // the resident launch's groups leave at their next fetch
  *s->h_stopv = 1u;
  cudaMemcpyAsync(s->d_stop, s->h_stopv, 4, cudaMemcpyHostToDevice, s->cs);
  cudaStreamSynchronize(s->cs);
  s->magic = 0;
  const int dev = s->p->device;
  free_stream(s);
  if (cur != dev) cudaSetDevice(cur);
  return HC_OK;
}
