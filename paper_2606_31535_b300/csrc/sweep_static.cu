// peers_query_noalloc: the sweep with its scratch in a fixed, library-owned device array.
//
// Some callers cannot let a library call cudaMalloc or cudaFree.  Examples are a host
// framework that owns every byte of device memory through its own pool, and a latency-bound
// loop that cannot afford the device-wide synchronisation an allocation or a free may cause.
// For them this entry point runs the same sweep kernels as peers_query, but the query fronts
// carried between levels and the running sums live in `g_noalloc_scratch` below, a file-scope
// device array of kNoAllocScratchDoubles doubles.  Every GPU that loads the library holds
// this array until the process exits.  The caller still passes its inputs (the plan and the
// resident factor) and its output (a device array for R).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "device.cuh"
#include "internal.h"
#include "peers.h"

namespace peers {

// 16 MiB of scratch per device: the carried fronts (carry_slots x nbmax doubles) followed by
// the per-slot running sums (carry_slots doubles).
constexpr int64_t kNoAllocScratchDoubles = int64_t(2) << 20;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).  The name
// g_noalloc_scratch in host code is only a host-side stand-in for the symbol, so it must never
// be handed to a kernel; the real address is looked up once per device and cached.
int scratch_on_device(int device, double **out, std::string &err) {
  if (device < 0 || device >= kMaxDevices) {
    err = "device index out of range for the no-allocation scratch table";
    return PEERS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_setup_lock);
  if (!g_scratch_ptr[device]) {
    void *p = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_ptr[device] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[device];
  return PEERS_OK;
}

}  // namespace

int query_noalloc(cudaStream_t stream, int device, const Symbolic &S, const SweepArgs &base,
                  const SweepItem *items, const int64_t *wave_item_off,
                  const int64_t *two_user, const int32_t *two_a, const int32_t *two_b,
                  double *R, int64_t *launches, std::string &err) {
  if (S.spill_stride > 0) {
    err = "the plan keeps supernode fronts in global memory (fronts larger than shared "
          "memory), which needs scratch beyond the static buffer: use peers_query";
    return PEERS_EINVAL;
  }
  const int64_t need = S.carry_slots * (int64_t(S.nbmax) + 1);
  if (need > kNoAllocScratchDoubles) {
    // The analysis counts 8 (nbmax + 1) bytes per query slot against the carry budget, so a
    // budget of at most the static buffer's size always yields a plan that fits.
    err = "the plan needs " + std::to_string(need) + " doubles of sweep scratch (" +
          std::to_string(S.carry_slots) + " query slots x (" + std::to_string(S.nbmax) +
          " + 1)) but the static buffer holds " + std::to_string(kNoAllocScratchDoubles) +
          "; analyse with peers_options.carry_budget <= " +
          std::to_string(kNoAllocScratchDoubles * 8) + " bytes, or use peers_query";
    return PEERS_EINVAL;
  }
  DEVICE_SCOPE(device);
  if (S.nq > 0) {
    const int rc0 = check_device_result(device, R, err);
    if (rc0 != PEERS_OK) return rc0;
  }
  double *scratch = nullptr;
  int rc = scratch_on_device(device, &scratch, err);
  if (rc != PEERS_OK) return rc;
  SweepArgs a = base;
  a.carry = scratch;
  a.racc = scratch + S.carry_slots * int64_t(S.nbmax);
  a.R = R;
  // Every carry slot and running sum is written by a query's first step before any later
  // step reads it, so nothing in the scratch has to start at zero.  R does: queries with
  // u == v are never walked.
  if (S.nq > 0) CUDA_TRY(cudaMemsetAsync(R, 0, sizeof(double) * S.nq, stream));
  for (size_t w = 0; w < S.waves.size() && S.nsorted + S.nq_two > 0; ++w) {
    const SweepWave &W = S.waves[w];
    rc = run_sweep_wave(S, W, items + wave_item_off[w], a, stream, nullptr, launches, err);
    if (rc != PEERS_OK) return rc;
    if (W.two_end > W.two_begin) {
      SweepArgs c = a;
      c.wave_base = W.q_begin;
      rc = run_two_branch_combine(c, two_user, two_a, two_b, W.two_begin, W.two_end, stream,
                                  launches, err);
      if (rc != PEERS_OK) return rc;
    }
  }
  CUDA_TRY(cudaStreamSynchronize(stream));
  CUDA_TRY(cudaGetLastError());
  return PEERS_OK;
}

}  // namespace peers
