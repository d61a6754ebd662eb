// Device-side declarations shared by the factorization and the sweep (library-internal).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "internal.h"

#define CUDA_TRY(x)                                                            \
  do {                                                                         \
    cudaError_t e_ = (x);                                                      \
    if (e_ != cudaSuccess) {                                                   \
      err = std::string(#x) + ": " + cudaGetErrorString(e_);                   \
      return PEERS_ECUDA;                                                      \
    }                                                                          \
  } while (0)

namespace peers {

// Makes `device` current for the guard's lifetime and then restores the calling thread's
// previous device, so that no library call leaves its caller on another device.
class DeviceGuard {
 public:
  explicit DeviceGuard(int device) {
    status_ = cudaGetDevice(&prev_);
    if (status_ == cudaSuccess && prev_ != device) {
      status_ = cudaSetDevice(device);
      switched_ = status_ == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (switched_) cudaSetDevice(prev_);
  }
  DeviceGuard(const DeviceGuard &) = delete;
  DeviceGuard &operator=(const DeviceGuard &) = delete;
  cudaError_t status() const { return status_; }

 private:
  int prev_ = 0;
  bool switched_ = false;
  cudaError_t status_ = cudaSuccess;
};

// Declares a DeviceGuard for `dev` in the enclosing scope and returns PEERS_ECUDA (with `err`
// set) if the device cannot be made current.
#define DEVICE_SCOPE(dev)                 \
  ::peers::DeviceGuard device_guard_(dev); \
  CUDA_TRY(device_guard_.status())

constexpr int kErrNotSpd = 1;
constexpr int kErrBounds = 2;

// Bounds checks of the PEERS_BOUNDS=1 build (libpeers_bounds.so): PEERS_IN(i, n, status) is
// true when 0 <= i < n; otherwise it records kErrBounds and the source line in `status` (the
// first failure wins) and is false, and the caller skips the access.  In the regular build
// it is the constant true and costs nothing.
#if defined(PEERS_BOUNDS) && PEERS_BOUNDS
#define PEERS_IN(i, n, status) ::peers::in_bounds((i), (n), (status), __LINE__)
#else
#define PEERS_IN(i, n, status) true
#endif

// Records the first error code and where it happened; later errors are dropped.
__device__ inline void flag_error(int *status, int code, int where) {
  if (atomicCAS(status, 0, code) == 0) atomicExch(status + 1, where);
}

__device__ inline bool in_bounds(int64_t i, int64_t n, int *status, int line) {
  if (i >= 0 && i < n) return true;
  if (status) flag_error(status, kErrBounds, line);
  return false;
}

// Dynamic shared memory of the running launch, in doubles.
__device__ inline int64_t dynamic_smem_doubles() {
  uint32_t bytes;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(bytes));
  return bytes / 8;
}

// Device pointers used by the factorization kernels.
struct FactorArgs {
  double *panel, *U, *tinv, *d, *dinv;
  const int32_t *first, *nb, *rmap;
  const int64_t *panel_off, *tinv_off, *u_off, *rows_off;
  int *status;
  int64_t panel_total;   // extent of `panel` (bounds-checked build)
};

struct FactorDevice {
  FactorArgs args;
  const int64_t *a_dest;
  const double *a_val;
  const int32_t *fac_sn;     // blocked supernodes by level (Symbolic::fac_sn)
  const int32_t *fuse_sn;    // supernodes factored whole by one CTA (Symbolic::fuse_sn)
  const int32_t *child_ptr, *child_list;
  const int32_t *ea_pairs;
  const int64_t *trail_prefix;
};

// Device pointers used by the sweep kernel.
struct SweepArgs {
  const double *panel, *tinv, *dinv;
  const int32_t *first, *nb, *rmap;
  const int64_t *panel_off, *tinv_off, *rows_off;
  const int32_t *qa, *qb;
  const int64_t *qorig;
  const SweepDesc *ldesc;   // two-branch walk steps (kind-1 items)
  double *carry;   // carry_slots x nbmax: the B-part of each query's front, slot-major
  double *racc;    // carry_slots: running sum_k y_k^2 / d_k of each query
  double *R;       // nq results in the caller's query order
  const int64_t *two_user;   // two-branch combine: user index, slot a, slot b per query
  const int32_t *two_a, *two_b;
  int64_t nbmax;
  int64_t wave_base;
  // fronts of supernodes that do not fit shared memory (items with spill == 1): CTA b of the
  // spilled launch keeps its tile's fronts at spill + b * spill_stride; spill_counter holds
  // one work counter per level (zeroed before each wave)
  double *spill;
  int64_t spill_stride;
  int *spill_counter;
  // extents for the bounds-checked build: error flag (2 ints), carry slots, results, the
  // two-branch step list
  int *status;
  int64_t carry_slots, nq, nldesc;
};

// CUDA streams over which a call spreads the lanes' independent subtrees (see kLanes), and
// the events that order them against the context's stream.
struct Lanes {
  cudaStream_t stream[kLanes];
  cudaStream_t top, top1;     // the device's highest stream priority: the part above the
                              // lanes, on the critical path, gets SMs first (top1 carries
                              // work that overlaps the top stream's, e.g. its phase 1)
  cudaEvent_t done[kLanes];   // recorded on a lane's stream when its work is issued
  cudaEvent_t start;          // recorded on the context's stream where the lanes may begin
  cudaEvent_t top_done;       // recorded on the top stream when the top part is issued
  // factorization, per lane and for the part above the lanes (index kLanes): a split group's
  // chain stream (diagonal blocks, panel rows, next columns; highest priority) and
  // update-matrix stream, and the events that order them with the group's own stream
  cudaStream_t chain[kLanes + 1], upd[kLanes + 1];
  cudaEvent_t ev_start[kLanes + 1], ev_panel[kLanes + 1], ev_rest[kLanes + 1];
  cudaEvent_t ev_chain[kLanes + 1], ev_upd[kLanes + 1];
};

// Runs the whole factorization on `stream` (and the lanes' subtrees on `lanes`' streams when
// it is non-null); adds the number of kernels launched to *launches.
int run_factor(const Symbolic &S, const FactorDevice &D, cudaStream_t stream, const Lanes *lanes,
               int64_t *launches, std::string &err);

// Launches the sweep of one wave, level by level.  If `events` is non-null it must hold
// 2 * nlevels events; launch l is bracketed by events[2l], events[2l+1].
int run_sweep_wave(const Symbolic &S, const SweepWave &W, const SweepItem *d_items,
                   const SweepArgs &args, cudaStream_t stream, cudaEvent_t *events,
                   int64_t *launches, std::string &err);

// Finishes the two-branch queries [k0, k1) of a wave: R[user] = r of slot a (+ r of slot b
// when the two branches end in different etree roots).
int run_two_branch_combine(const SweepArgs &args, const int64_t *two_user, const int32_t *two_a,
                           const int32_t *two_b, int64_t k0, int64_t k1, cudaStream_t stream,
                           int64_t *launches, std::string &err);

// One k_sweep launch over an arbitrary item list (the autotuner's timing runs).
int run_items(const SweepItem *d_items, int64_t n, const SweepArgs &args, int64_t smem,
              cudaStream_t stream, std::string &err);

// One launch of the multi-graph (persistent) sweep kernel: nitems items, each with its
// argument block table[item.g]; CTAs pull items through *counter (zero before the launch).
int run_multi_step(const SweepItem *items, int64_t nitems, const SweepArgs *table, int *counter,
                   int64_t smem, int64_t grid, cudaStream_t stream, std::string &err);
// Grid of a persistent multi-graph launch (CTAs that fit the GPU at once, at most nitems);
// also raises the kernel's dynamic shared-memory limit to smem.  Call outside stream capture.
int multi_step_grid(int64_t smem, int64_t nitems, int64_t *grid, std::string &err);
// Raises `kernel`'s dynamic shared-memory limit on the current device to at least `bytes`;
// `configured` holds the limit set so far per device (64 entries).  Thread-safe (sweep.cu).
int raise_smem_limit(const void *kernel, int *configured, int64_t bytes, std::string &err);

// The sweep with its scratch in the library's static device array (sweep_static.cu); no
// device memory is allocated or freed.  R is a device array of S.nq doubles.
int query_noalloc(cudaStream_t stream, int device, const Symbolic &S, const SweepArgs &base,
                  const SweepItem *items, const int64_t *wave_item_off,
                  const int64_t *two_user, const int32_t *two_a, const int32_t *two_b,
                  double *R, int64_t *launches, std::string &err);

// Checks that a caller's device result pointer is device (or managed) memory reachable from
// `device` before any kernel writes through it; PEERS_EINVAL otherwise (capi.cu).
int check_device_result(int device, const void *p, std::string &err);

// FP64 throughput probes (TFLOP/s) on the current device: out[0] DFMA (CUDA cores),
// out[1] mma.sync m8n8k4 f64 (the FP64 tensor path).
int fp64_peak(cudaStream_t stream, double out[3], std::string &err);
// Every f64 mma.sync shape (TFLOP/s): out[0] m8n8k4, out[1] m16n8k4, out[2] m16n8k8,
// out[3] m16n8k16.
int fp64_mma_shapes(cudaStream_t stream, double out[4], std::string &err);

}  // namespace peers
