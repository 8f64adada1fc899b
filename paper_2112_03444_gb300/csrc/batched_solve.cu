// Standalone batched dense complex solve A x = b: the fused linear solver of
// paper Sec. 6 (LU with partial pivoting on the augmented matrix [A b] and
// the triangular solve in one kernel, data kept in registers), measured on
// its own in the paper's Fig. 3 (1000 matrices of 4x4 to 20x20 against
// cuBLAS and MAGMA).  It is the same register-resident elimination the
// tracker runs per path (gj_solve in hc_device.cuh): one lane group per
// system, row i of [A | b] in lane i, Gauss-Jordan with partial pivoting, so
// the back substitution is folded into the elimination.
//
// Data path: a block's systems are contiguous in A (row-major, system after
// system), so the block stages them through shared memory with consecutive
// threads reading consecutive complex numbers (coalesced), then each lane
// takes its row from shared memory; solutions go out the same way.
#include <cstdint>

#include <cuda_runtime.h>

#include "hc.h"
#include "hc_device.cuh"
#include "kernels.cuh"

namespace {

using hc::cx;

constexpr int kThreads = 128;

template <int N>
constexpr int solve_lanes() {
  return N <= 4 ? 4 : N <= 8 ? 8 : N <= 16 ? 16 : 32;
}

// Shared memory of one block: the staged augmented matrices [G][N][N + 1],
// then per group the two pivot-row buffers and the solution scatter buffer.
template <int N, class R>
constexpr size_t solve_smem_bytes() {
  constexpr int L = solve_lanes<N>(), G = kThreads / L;
  constexpr int S = (N + 2) & ~1;  // entries per pivot buffer (gj_solve, NR = 1)
  return sizeof(cx<R>) * ((size_t)G * N * (N + 1) + (size_t)G * 2 * S + (size_t)G * L);
}

template <int N, class R>
__global__ void __launch_bounds__(kThreads) batched_solve_kernel(int64_t batch,
                                                                 const cx<R>* __restrict__ A,
                                                                 const cx<R>* __restrict__ b,
                                                                 cx<R>* __restrict__ x,
                                                                 int32_t* __restrict__ info) {
  constexpr int L = solve_lanes<N>(), G = kThreads / L, W = N + 1;
  constexpr int S = (N + 2) & ~1;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<R>* stage = reinterpret_cast<cx<R>*>(smem);
  cx<R>* pvbuf = stage + (size_t)G * N * W;
  cx<R>* sbuf = pvbuf + (size_t)G * 2 * S;
  const hc::Group g = hc::make_group<L>();
  const int grp = threadIdx.x / L;
  cx<R>* pv = pvbuf + grp * 2 * S;
  cx<R>* sb = sbuf + grp * L;
  for (int64_t base = (int64_t)blockIdx.x * G; base < batch; base += (int64_t)gridDim.x * G) {
    const int cnt = (int)((batch - base) < G ? (batch - base) : G);
    // coalesced staging of the block's matrices and right-hand sides
    const cx<R>* Ab = A + base * N * N;
    for (int idx = threadIdx.x; idx < cnt * N * N; idx += kThreads) {
      const int sys = idx / (N * N), r = idx % (N * N);
      stage[(sys * N + r / N) * W + r % N] = Ab[idx];
    }
    const cx<R>* bb = b + base * N;
    for (int idx = threadIdx.x; idx < cnt * N; idx += kThreads)
      stage[(idx / N * N + idx % N) * W + N] = bb[idx];
    __syncthreads();
    cx<R> a[W];
    const bool live = grp < cnt;
#pragma unroll
    for (int j = 0; j < W; ++j)
      a[j] = (live && g.gl < N) ? stage[(grp * N + g.gl) * W + j] : hc::czero<R>();
    __syncthreads();  // the stage is free for the next round once every row is in registers
    if (live) {
      cx<R> sol[1];
      int col;
      const bool ok = hc::gj_solve<N, 1, R>(g, a, sol, col, pv);
      if (col >= 0) sb[col] = sol[0];
      __syncwarp(g.mask);
      if (g.gl < N) x[(base + grp) * N + g.gl] = sb[g.gl];
      if (g.gl == 0 && info) info[base + grp] = ok ? 0 : 1;
      __syncwarp(g.mask);
    }
  }
}

struct SolveRef {
  const void* fn;
  size_t smem;
  int per_block;
};

template <int N, class R>
SolveRef solve_ref() {
  return SolveRef{reinterpret_cast<const void*>(&batched_solve_kernel<N, R>),
                  solve_smem_bytes<N, R>(), kThreads / solve_lanes<N>()};
}

template <class R, int N = 1>
SolveRef solve_dispatch(int n) {
  if constexpr (N > 32) {
    return SolveRef{nullptr, 0, 0};
  } else {
    if (n == N) return solve_ref<N, R>();
    return solve_dispatch<R, N + 1>(n);
  }
}

}  // namespace

extern "C" hc_status hc_batched_solve(int32_t n, int64_t batch, int32_t fp32, const void* A,
                                      const void* b, void* x, int32_t* info, void* stream) {
  if (n < 1 || n > 32 || batch < 0 || (batch > 0 && (!A || !b || !x)) || (fp32 != 0 && fp32 != 1)) {
    hc::set_last_error("hc_batched_solve: n must be 1..32, batch >= 0, A, b, x non-null");
    return HC_ERR_INVALID;
  }
  if (batch == 0) return HC_OK;
  const SolveRef k = fp32 ? solve_dispatch<float>(n) : solve_dispatch<double>(n);
  if (!k.fn) {
    hc::set_last_error("hc_batched_solve: no kernel for this size");
    return HC_ERR_UNSUPPORTED;
  }
  cudaGetLastError();
  if (k.smem > 48 * 1024 &&
      cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) !=
          cudaSuccess) {
    hc::set_last_error("hc_batched_solve: shared-memory attribute refused");
    return HC_ERR_CUDA;
  }
  int dev = 0, sms = 0, per_sm = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, kThreads, k.smem) !=
          cudaSuccess) {
    hc::set_last_error("hc_batched_solve: device query failed");
    return HC_ERR_CUDA;
  }
  // one wave of resident blocks at most; each block strides over the batch
  const int64_t want = (batch + k.per_block - 1) / k.per_block;
  const int64_t cap = (int64_t)(per_sm < 1 ? 1 : per_sm) * sms;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  void* args[] = {&batch, &A, &b, &x, &info};
  if (cudaLaunchKernel(k.fn, dim3(grid), dim3(kThreads), args, k.smem,
                       static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    hc::set_last_error("hc_batched_solve: launch failed");
    return HC_ERR_CUDA;
  }
  return HC_OK;
}
