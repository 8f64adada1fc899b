// Kernel entry points and their host-visible launch descriptors.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dfloat.cuh"
#include "hc.h"
#include "hc_device.cuh"

namespace hc {

constexpr int kBlock = 128;  // threads per block of the tracking kernels

// Shared memory of one lane group of L lanes (layout in tracker.cuh):
// pivot-row buffers 32 (L + 2), evaluator accumulators acc bytes, FP64
// point (L + extra) 16, solution scatter L 16, FP32 point (L + extra) 8.
// The stride between groups is 16 bytes past a multiple of 128: the groups
// of a warp reading their own broadcast word (a point entry, a monomial,
// the pivot row) then hit different banks.
// The FP64-state kernels (precision FP64 and double-float) add eg bytes for
// the endgame's samples (three complex doubles per lane: the previous
// sample, its dx/ds, the last prediction); the double-float kernels (vx)
// also a double-float copy of the point, (L + extra) 16.
__host__ __device__ constexpr int group_smem_bytes(int L, int extra, int acc = 0, int eg = 0,
                                                   int vx = 0) {
  return ((32 * (L + 2) + acc + (L + extra) * 16 + L * 16 + (L + extra) * 8 + eg +
           (vx ? (L + extra) * 16 : 0) + 127) &
          ~127) +
         16;
}
__host__ __device__ constexpr int endgame_smem_bytes(int L, bool mixed) { return mixed ? 0 : 48 * L; }
// Dynamic shared memory of one tracking block of `threads` threads
__host__ __device__ constexpr int block_smem_bytes(int L, int extra, int acc = 0,
                                                   int threads = kBlock, int eg = 0, int vx = 0) {
  return (threads / L) * group_smem_bytes(L, extra, acc, eg, vx);
}
// Threads per block of a launch: one warp for one-path-per-warp launches of
// the re-tracking tiers (a hard path then holds only its own warp's
// registers, not three idle warps' beside the other classes' launches),
// kBlock otherwise.
inline int retrack_threads(int lanes) { return lanes == 32 ? 32 : kBlock; }

// Dense coefficient tables D (see dense_td.cuh): per slice j (the partial
// derivative dF_i/dx_j; slice n holds the constant term), the monomials of
// degree < d are stored in pairs per lane, so that one 16-byte load brings
// two FP32 coefficients.  The constant, the linear and the quadratic
// monomials each start a new pair (each range padded to an even count).
__host__ __device__ constexpr int dense_mpp(int n, int d) {  // padded monomials per slice
  return 2 + (n + (n & 1)) + ((d == 3) ? (n * (n + 1) / 2 + ((n * (n + 1) / 2) & 1)) : 0);
}
// padded position of the monomial with graded index mp (0 constant, 1..n
// linear, then the quadratic ones)
__host__ __device__ constexpr int dense_mslot(int n, int mp) {
  return mp == 0 ? 0 : (mp <= n ? 1 + mp : 2 + (n + (n & 1)) + (mp - 1 - n));
}
// entry of (slice j, monomial mp, row i) in an instance's table of lane stride L
__host__ __device__ constexpr int64_t dense_slot(int n, int d, int L, int j, int mp, int i) {
  return ((int64_t)(j * (dense_mpp(n, d) / 2) + (dense_mslot(n, mp) >> 1)) * L + i) * 2 +
         (dense_mslot(n, mp) & 1);
}

// Work distribution of a tracking launch: work item = output slot
// item = instance * paths + k, k < paths; its start path is k, or
// path_ids[item] when the batch tracks a subset of the starts.  A lane group
// takes the next item with one atomicAdd on *queue (retire/refill: a group
// that finishes a path pulls the next one), until the items are exhausted
// or, with a step budget, the finished paths' steps reach it.
struct LaunchCommon {
  DevSettings s;
  int64_t n_items;                      // used when count_dev == nullptr
  const unsigned long long* count_dev;  // number of items, read on the device
  const int64_t* items;                 // optional explicit item list
  unsigned long long* queue;            // next item counter (zeroed before launch)
  int64_t paths;                        // items (output slots) per instance
  const int64_t* path_ids;              // optional start index of every item
  const int64_t* path_map;              // optional start index of item k of each instance
  unsigned long long* step_total;       // steps of the finished paths (atomic)
  unsigned long long step_budget;       // 0: none; else no item is started once
                                        // *step_total reaches it (implicit lists only)
  double* x_out;                        // [items][n] complex
  uint8_t* status_out;                  // [items]
  int32_t* steps_out;                   // [items][3]
  double* be_out;                       // [items] (optional)
  int64_t* esc_list;                    // mixed precision: items to re-track in FP64
  unsigned long long* esc_count;
  // Hand-over between the FP32 and FP64 tiers:
  double* t_io;                 // per item: t to resume from in FP64 (0 = restart at t = 0)
  float2* x32_out;              // per item endpoint copy for duplicate detection (NaN if not finite)
  unsigned long long* esc_steps;  // FP64 tier: accepted, rejected, Newton totals (atomic)
  int64_t* dup_list;            // mixed kernel: failures to re-track with FP64 residuals
  unsigned long long* dup_count;
  int start_hi;                 // mixed kernel: track every path with the FP64 state, FP64
                                // residuals and FP64 tolerances from t = 0 (re-tracking of
                                // colliding and failed paths)
  int spread;                   // first round of items round-robin over the blocks (one
                                // per block before any second), then the queue: a short
                                // list of FP64-heavy paths lands on as many SMs as it can
  // Resident launches (hc_stream): items come from a ring of instance slots
  // that the host fills while the launch runs.  Ticket q (claimed from
  // *queue only while q < *ring_tail, which the host's staging stream writes
  // after the slot's inputs) is item q mod ring_items, slot
  // (q mod ring_items) / paths.  A group that finds no ticket sleeps (backing
  // off) and polls, and leaves the launch once *ring_stop is set or
  // ring_idle_ns pass without a ticket.  The last path of a slot to finish
  // stores the ticket's generation (q / ring_items + 1) into ring_flag[slot]
  // (mapped host memory).  Re-tracking lists are kept per slot,
  // slot-relative: esc_list / dup_list + slot * paths, counters
  // esc_count / dup_count + slot.
  unsigned long long ring_items;         // 0: not resident
  const unsigned long long* ring_tail;   // device memory
  const unsigned int* ring_stop;         // device memory
  unsigned long long ring_idle_ns;
  unsigned int* ring_done;               // [slots] paths finished (device)
  unsigned long long* ring_flag;         // [slots] mapped host memory
};

struct DenseArgs {
  LaunchCommon c;
  const cx<float>* D32;
  const cx<double>* D64;
  const cx<df>* Ddf;         // D as double-floats (double-float kernels)
  const cx<double>* E;
  const cdf* Edf;            // E as double-floats (mixed-precision kernels' residuals)
  int64_t Dstride, Estride;  // complex elements per instance
  cx<double> gamma;
  cx<float> gamma32;         // FP32 copy (FP32 evaluations convert nothing)
  cdf gammadf;               // double-float copy
};

// One term of an equation (paper Sec. 6: a coefficient times a product of
// factors taken from the per-path vector V, see term_param.cuh).  d is the
// number of factors evaluated for this term slot: the same for every row at
// a slot (rows with fewer factors are padded with the constant 1), so the
// lanes of a warp run the same loop.  tgt[f] names the entry of row i that
// the derivative with respect to factor f contributes to: x_j -> j, a
// parameter -> N (dH/dt, multiplied by dp), 255 -> none (the padding 1).
constexpr int kMaxTermFactors = 8;
struct TermRec {
  float2 s;                        // coefficient (FP32 copy)
  uint8_t idx[kMaxTermFactors];    // factor positions in V
  uint8_t tgt[kMaxTermFactors];
  uint8_t d;
  uint8_t pad[7];
};
static_assert(sizeof(TermRec) == 32, "term record layout");
constexpr int kMaxTermEntries = 34;  // N + 2 entries per row, N <= 32

struct TermArgs {
  LaunchCommon c;
  const TermRec* rec;    // [TT][ls]: term slot k of row i at k * ls + i
  const double2* s64;    // FP64 coefficients, same layout
  const cdf* sdf;        // the same as double-floats (mixed-precision residuals)
  int TT;                // term slots per row (rows padded with zero terms)
  int P;                 // number of parameters
  int ls;                // lane stride of the tables (and V's offset of the 1)
  int extra;             // shared-memory entries behind the point: 1 + 3P
  const double2* p0;     // [P]
  const double2* p1;     // [instances][P]
  const double2* start;  // [paths][n]
  // coefficient interpolation (HC_COEFFICIENT): the records carry no
  // parameter factors; the coefficient of slot k, row i at time t is
  // c0 + t dc, c0 = c(p0) shared, dc = c(p1) - c(p0) per instance, each in
  // FP64, FP32 and double-float, layout [TT][ls] (dc: [instances][TT][ls])
  int coef_mode;
  const double2* c0;
  const float2* c0f;
  const cdf* c0df;
  const double2* dc;
  const float2* dcf;
  const cdf* dcdf;
};

// Points at which hc_evaluate evaluates the homotopy (device buffers):
// point k belongs to instance inst[k], lies at x[k] (n complex) and t[k];
// outputs dH/dx row-major [k][i][j], H [k][i] and dH/dt [k][i].
struct EvalPoints {
  int64_t n_points;
  const int64_t* inst;
  const double2* x;
  const double* t;
  double2* Hx;
  double2* H;
  double2* Ht;
};
struct DenseEvalArgs {
  DenseArgs a;
  EvalPoints e;
};
struct TermEvalArgs {
  TermArgs a;
  EvalPoints e;
};

struct KernelRef {
  const void* fn;   // __global__ function
  int lanes;        // lanes per path (L)
  int extra;        // per-group shared entries behind the point the kernel itself needs
  int acc_bytes;    // bytes of one evaluator accumulator (per lane and row entry), 0: none
  int eg_bytes;     // per-group endgame sample bytes (FP64-state kernels), 0: none
  int vx;           // 1: double-float kernel (a double-float copy of the point)
};

// Lanes per path chosen for n unknowns (one row per lane, groups are powers
// of two so that a warp holds 32 / L paths).
inline int lanes_for(int n) { return n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : 32; }

// prec: HC_PREC_FP64, HC_PREC_MIXED or HC_PREC_DF.  lanes = 0: default
// group width; 32: one path per warp (mixed kernels, n <= 16)
KernelRef dense_kernel(int deg, int n, int prec, int lanes);  // fn == nullptr if absent
KernelRef term_kernel(int n, int prec, int lanes);            // fn == nullptr if absent
// Kernel of the re-tracking tiers (few paths): one path per warp with split
// rows where available, else the default width.
KernelRef retrack_kernel(int deg, int n, int prec);
// Precision of the mixed pipeline's last re-tracking tier: retrack_precision,
// except with the endgame, which keeps FP64: its cycle-number estimate and
// Hermite extrapolation use dx/ds at the samples, and near a multiple root
// the double-float solve loses five bits of it to the Jacobian's condition.
inline int last_tier_precision(const hc_settings& s) {
  return s.endgame ? HC_PREC_FP64 : s.retrack_precision;
}

// Resident-launch (hc_stream) variant of the mixed tracking kernel for a
// problem: term tables or dense of degree deg; fn == nullptr if absent.
KernelRef ring_kernel(bool terms, int deg, int n);

// Evaluation kernels of hc_evaluate (prec: HC_PREC_FP64, HC_PREC_MIXED =
// FP32 evaluation, HC_PREC_DF); fn == nullptr if absent.
KernelRef dense_eval_kernel(int deg, int n, int prec);
KernelRef term_eval_kernel(int n, int prec);

// Defined in server.cu: frees a server if magic is the server's magic.
bool destroy_server_if(void* handle, uint32_t magic);

// Host helpers defined in hc_api.cu.
void set_last_error(const char* msg);
DevSettings to_dev_settings(const hc_settings& s);
hc_status check_settings(const hc_settings& s);
cudaError_t launch_dedupe(int64_t items, int64_t paths, int n, const float2* x32,
                          const uint8_t* status, float tol, const int64_t* list,
                          const unsigned long long* list_count, int64_t* out_list,
                          unsigned long long* out_count, double* t_io, cudaStream_t st);

}  // namespace hc
