// Tracking entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the time they track: code
// running inside a memory pool or arena that owns the whole device, real-time
// loops that must not enter the CUDA allocator (cudaMalloc can synchronize the
// device and take unbounded time), or hosts whose allocator is reserved for
// another framework.  For them hc_track_dense_noalloc runs the same dense
// total-degree tracking kernels as hc_track_batch, but every buffer the
// kernels need besides the caller's inputs and outputs (control words, the
// encoded coefficients, the FP64 re-tracking list, resume times, the
// endpoint copy for duplicate detection) lives in one file-scope device
// array of kNoAllocScratchBytes.  Every GPU that loads this library holds
// that array until the process exits.
//
// The array's host-side name is not a device address.  The first call on a
// device (with that device current) looks its address up with
// cudaGetSymbolAddress and caches it per device; make that first call before
// any stream capture.  All calls share the array and it keeps the last
// call's contents: each call clears what must start at zero, and calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on it and must be serialized by the caller.
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "dense_td.cuh"
#include "hc.h"
#include "kernels.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

hc_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    hc::set_last_error("hc_track_dense_noalloc: no usable current device");
    return HC_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      hc::set_last_error("hc_track_dense_noalloc: cudaGetSymbolAddress of the scratch array failed");
      return HC_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HC_OK;
}

__device__ int binom_d(int n, int k) {
  if (k < 0 || k > n) return 0;
  int r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// Monomial m of the graded order (degree 0 first; inside a degree the sorted
// variable tuple in lexicographic order) -> ascending variable tuple.
__device__ int unrank_graded(int n, int m, int* vars) {
  int g = 0, base = 0;
  for (;;) {
    const int cnt = binom_d(n + g - 1, g);
    if (m < base + cnt) break;
    base += cnt;
    ++g;
  }
  int r = m - base, prev = 0;
  for (int p = 0; p < g; ++p) {
    for (int v = prev;; ++v) {
      const int cnt = binom_d((n - v) + (g - p - 1) - 1, g - p - 1);
      if (r < cnt) {
        vars[p] = v;
        prev = v;
        break;
      }
      r -= cnt;
    }
  }
  return g;
}

__device__ int rank_graded(int n, const int* vars, int g) {
  int idx = 0;
  for (int e = 0; e < g; ++e) idx += binom_d(n + e - 1, e);
  int prev = 0;
  for (int p = 0; p < g; ++p) {
    for (int v = prev; v < vars[p]; ++v) idx += binom_d((n - v) + (g - p - 1) - 1, g - p - 1);
    prev = vars[p];
  }
  return idx;
}

// Position of an ascending tuple in the nested Horner order used by E.
__device__ int nested_index(int n, int d, const int* vars, int g) {
  if (g == 0) return 0;
  int m = 1;
  for (int j = 0; j < n; ++j) {
    if (g == 1 && vars[0] == j) return m;
    ++m;
    for (int k = 0; k <= j; ++k) {
      if (g == 2 && vars[0] == k && vars[1] == j) return m;
      ++m;
      if (d == 3)
        for (int l = 0; l <= k; ++l) {
          if (g == 3 && vars[0] == l && vars[1] == k && vars[2] == j) return m;
          ++m;
        }
    }
  }
  return -1;
}

// Encodes coefficients given in the canonical dense order
// coef[inst][i][m] (equation i, monomial m of the graded order) into E, D64
// and D32 (and Ddf, the double-float table, if given), computing the index
// maps on the fly.
__device__ __forceinline__ void put_d(double2* D64, float2* D32, float4* Ddf, int64_t slot,
                                      double2 v) {
  D64[slot] = v;
  D32[slot] = make_float2((float)v.x, (float)v.y);
  if (Ddf) {  // cx<df> layout: re hi, re lo, im hi, im lo
    const hc::df re(v.x), im(v.y);
    Ddf[slot] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

__global__ void stage_canonical_kernel(int64_t n_inst, int n, int d, int M, int MP, int L,
                                       const double2* __restrict__ coef, double2* E,
                                       hc::cdf* Edf, int64_t Es, double2* D64, float2* D32,
                                       float4* Ddf, int64_t Ds) {
  const int64_t total = n_inst * n * M;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < total;
       w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t inst = w / ((int64_t)n * M);
    const int r = (int)(w - inst * (int64_t)n * M);
    const int i = r / M, m = r - i * M;
    const double2 c = coef[w];
    int vars[4];
    const int g = unrank_graded(n, m, vars);
    const int64_t eslot = inst * Es + (int64_t)nested_index(n, d, vars, g) * L + i;
    E[eslot] = c;
    Edf[eslot] = hc::to_cdf(hc::cx<double>{c.x, c.y});
    if (g == 0) {
      put_d(D64, D32, Ddf, inst * Ds + hc::dense_slot(n, d, L, n, 0, i), c);
      continue;
    }
    for (int p = 0; p < g; ++p) {
      if (p > 0 && vars[p] == vars[p - 1]) continue;  // one slot per distinct variable
      const int j = vars[p];
      int a = 0, rest[4], nr = 0;
      bool dropped = false;
      for (int q = 0; q < g; ++q) {
        if (vars[q] == j) ++a;
        if (vars[q] == j && !dropped) {
          dropped = true;
          continue;
        }
        rest[nr++] = vars[q];
      }
      const int mp = rank_graded(n, rest, nr);
      put_d(D64, D32, Ddf, inst * Ds + hc::dense_slot(n, d, L, j, mp, i),
            make_double2(a * c.x, a * c.y));
    }
  }
}

int binom_h(int n, int k) {
  if (k < 0 || k > n) return 0;
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return (int)r;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" hc_status hc_track_dense_noalloc(int32_t n, int32_t degree, const double* gamma,
                                            const hc_settings* settings, int32_t n_instances,
                                            const double* coef, double* x_out,
                                            uint8_t* status_out, int32_t* steps_out,
                                            double* be_out, void* stream) {
  if (!gamma || !settings || !coef || !x_out || !status_out || !steps_out || n_instances < 1 ||
      !((degree == 2 && n >= 1 && n <= 12) || (degree == 3 && n >= 1 && n <= 8))) {
    hc::set_last_error("hc_track_dense_noalloc: invalid arguments (degree 2 with n <= 12 or "
                       "degree 3 with n <= 8; coef, x_out, status_out, steps_out required)");
    return HC_ERR_INVALID;
  }
  const hc_status vs = hc::check_settings(*settings);
  if (vs != HC_OK) return vs;
  const bool mixed = settings->precision == HC_PREC_MIXED;
  const bool escalate = mixed && settings->escalate;
  const bool use_df = settings->precision == HC_PREC_DF ||
                      (escalate && hc::last_tier_precision(*settings) == HC_PREC_DF);
  const int L = hc::lanes_for(n);
  const int M = binom_h(n + degree, degree);
  const int MP = binom_h(n + degree - 1, degree - 1);
  int64_t paths = 1;
  for (int i = 0; i < n; ++i) paths *= degree;
  const int64_t items = (int64_t)n_instances * paths;
  const int64_t Es = (int64_t)M * L, Ds = (int64_t)(n + 1) * hc::dense_mpp(n, degree) * L;

  // scratch layout
  const size_t ctl_b = align256(sizeof(unsigned long long) * 16);
  const size_t e_b = align256(sizeof(double2) * Es * n_instances);
  const size_t edf_b = align256(sizeof(hc::cdf) * Es * n_instances);
  const size_t d64_b = align256(sizeof(double2) * Ds * n_instances);
  const size_t d32_b = align256(sizeof(float2) * Ds * n_instances);
  const size_t ddf_b = use_df ? align256(sizeof(float4) * Ds * n_instances) : 0;
  const size_t esc_b = escalate ? align256(sizeof(int64_t) * items) : 0;
  const size_t dup_b = esc_b;
  const size_t tio_b = escalate ? align256(sizeof(double) * items) : 0;
  const size_t x32_b = escalate ? align256(sizeof(float2) * n * items) : 0;
  const size_t need =
      ctl_b + e_b + edf_b + d64_b + d32_b + ddf_b + esc_b + dup_b + tio_b + x32_b;
  if (need > kNoAllocScratchBytes) {
    char msg[200];
    std::snprintf(msg, sizeof(msg),
                  "hc_track_dense_noalloc: batch needs %zu bytes of scratch, the fixed array "
                  "holds %zu; track fewer instances per call",
                  need, kNoAllocScratchBytes);
    hc::set_last_error(msg);
    return HC_ERR_INVALID;
  }
  void* base = nullptr;
  hc_status rc = scratch_address(&base);
  if (rc != HC_OK) return rc;
  unsigned char* p = static_cast<unsigned char*>(base);
  unsigned long long* ctl = reinterpret_cast<unsigned long long*>(p);
  p += ctl_b;
  double2* E = reinterpret_cast<double2*>(p);
  p += e_b;
  hc::cdf* Edf = reinterpret_cast<hc::cdf*>(p);
  p += edf_b;
  double2* D64 = reinterpret_cast<double2*>(p);
  p += d64_b;
  float2* D32 = reinterpret_cast<float2*>(p);
  p += d32_b;
  float4* Ddf = use_df ? reinterpret_cast<float4*>(p) : nullptr;
  p += ddf_b;
  int64_t* esc = escalate ? reinterpret_cast<int64_t*>(p) : nullptr;
  p += esc_b;
  int64_t* dup = escalate ? reinterpret_cast<int64_t*>(p) : nullptr;
  p += dup_b;
  double* t_io = escalate ? reinterpret_cast<double*>(p) : nullptr;
  p += tio_b;
  float2* x32 = escalate ? reinterpret_cast<float2*>(p) : nullptr;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
#define NA_CUDA(call)                                                                   \
  do {                                                                                  \
    if ((call) != cudaSuccess) {                                                        \
      hc::set_last_error("hc_track_dense_noalloc: " #call " failed");                   \
      return HC_ERR_CUDA;                                                               \
    }                                                                                   \
  } while (0)
  // the array keeps the previous call's contents: clear what starts at zero
  NA_CUDA(cudaMemsetAsync(ctl, 0, ctl_b + e_b + edf_b + d64_b + d32_b + ddf_b, st));
  NA_CUDA(cudaMemsetAsync(steps_out, 0, sizeof(int32_t) * 3 * items, st));
  {
    const int64_t work = (int64_t)n_instances * n * M;
    const int grid = (int)((work + 255) / 256 < 4096 ? (work + 255) / 256 : 4096);
    stage_canonical_kernel<<<grid, 256, 0, st>>>(n_instances, n, degree, M, MP, L,
                                                 reinterpret_cast<const double2*>(coef), E, Edf,
                                                 Es, D64, D32, Ddf, Ds);
    NA_CUDA(cudaGetLastError());
  }

  hc::DenseArgs a;
  std::memset(&a, 0, sizeof(a));
  a.c.s = hc::to_dev_settings(*settings);
  a.c.n_items = items;
  a.c.queue = ctl + 0;
  a.c.paths = paths;
  a.c.x_out = x_out;
  a.c.status_out = status_out;
  a.c.steps_out = steps_out;
  a.c.be_out = be_out;
  a.c.esc_list = esc;
  a.c.esc_count = ctl + 2;
  a.c.t_io = t_io;
  a.c.x32_out = x32;
  a.c.dup_list = escalate ? dup : nullptr;
  a.c.dup_count = ctl + 7;
  a.D32 = reinterpret_cast<const hc::cx<float>*>(D32);
  a.D64 = reinterpret_cast<const hc::cx<double>*>(D64);
  a.Ddf = reinterpret_cast<const hc::cx<hc::df>*>(Ddf);
  a.E = reinterpret_cast<const hc::cx<double>*>(E);
  a.Edf = Edf;
  a.Dstride = Ds;
  a.Estride = Es;
  a.gamma = hc::cx<double>{gamma[0], gamma[1]};
  a.gamma32 = hc::cx<float>{(float)gamma[0], (float)gamma[1]};
  a.gammadf = hc::split_cdf_host(gamma[0], gamma[1]);

  int dev = 0, sms = 0;
  NA_CUDA(cudaGetDevice(&dev));
  NA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  auto launch = [&](const hc::KernelRef& k, const hc::DenseArgs& args, int64_t max_items,
                    int threads = hc::kBlock) {
    const size_t smem =
        (size_t)hc::block_smem_bytes(k.lanes, k.extra, 0, threads, k.eg_bytes, k.vx);
    int blocks = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k.fn, threads, smem) !=
        cudaSuccess)
      return cudaErrorUnknown;
    if (blocks < 1) blocks = 1;
    const int64_t gpb = threads / k.lanes;
    int64_t grid = (int64_t)blocks * sms;
    const int64_t want = (max_items + gpb - 1) / gpb;
    if (want < grid) grid = want < 1 ? 1 : want;
    void* argv[] = {(void*)&args};
    return cudaLaunchKernel(k.fn, dim3((unsigned)grid), dim3(threads), argv, smem, st);
  };
  // the autotuner's group width where that variant exists (as hc_track_batch)
  hc::KernelRef k =
      hc::dense_kernel(degree, n, settings->precision, mixed ? settings->lanes : 0);
  if (!k.fn) k = hc::dense_kernel(degree, n, settings->precision, 0);
  if (!k.fn) {
    hc::set_last_error("hc_track_dense_noalloc: no kernel for this shape");
    return HC_ERR_UNSUPPORTED;
  }
  NA_CUDA(launch(k, a, items));
  if (escalate) {
    NA_CUDA(hc::launch_dedupe(items, paths, n, x32, status_out, 1e-6f, nullptr, nullptr, dup,
                              ctl + 7, t_io, st));
    hc::DenseArgs dd = a;
    dd.c.count_dev = ctl + 7;
    dd.c.items = dup;
    dd.c.queue = ctl + 6;
    dd.c.start_hi = 1;
    dd.c.spread = 1;
    dd.c.dup_list = nullptr;
    dd.c.dup_count = nullptr;
    const hc::KernelRef kr = hc::retrack_kernel(degree, n, HC_PREC_MIXED);
    NA_CUDA(launch(kr, dd, items, hc::retrack_threads(kr.lanes)));
    NA_CUDA(hc::launch_dedupe(items, paths, n, x32, status_out, 1e-6f, dup, ctl + 7, esc, ctl + 2,
                              t_io, st));
    hc::DenseArgs e = a;
    e.c.count_dev = ctl + 2;
    e.c.items = esc;
    e.c.queue = ctl + 1;
    e.c.esc_list = nullptr;
    e.c.x32_out = nullptr;
    e.c.esc_steps = ctl + 3;
    e.c.spread = 1;
    e.c.dup_list = nullptr;
    e.c.dup_count = nullptr;
    const hc::KernelRef k64 = hc::retrack_kernel(degree, n, hc::last_tier_precision(*settings));
    NA_CUDA(launch(k64, e, items, hc::retrack_threads(k64.lanes)));
  }
#undef NA_CUDA
  return HC_OK;
}
