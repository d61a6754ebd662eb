// Batched sweep of many independent graphs: one persistent launch per etree level for all
// of them, captured once in a CUDA graph and replayed.
//
// Each graph keeps its own plan and factor (peers_analyze / peers_factor).  The batch
// aligns the graphs' step sequences (wave by wave, level by level, plus the two-branch
// combine of a wave) at their last step, and merges the t-th step from the end of every
// graph into one list of work items, each tagged with its graph's argument block.  A launch covers one merged step, so a batch
// of G graphs of height H needs max_g H_g launches instead of sum_g H_g.  Results are
// identical to the single-graph sweep bit for bit: an item's arithmetic depends only on its
// own supernode and queries.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "device.cuh"
#include "handles.h"
#include "internal.h"
#include "peers.h"

struct peers_batch {
  int device = 0;
  int32_t count = 0;
  std::vector<const peers_symbolic *> syms;
  std::vector<const peers_numeric *> nums;
  std::vector<int64_t> r_off;          // offset of graph i's results in d_R
  int64_t r_total = 0;
  std::vector<int64_t> step_ptr;       // items of step t: [step_ptr[t], step_ptr[t+1])
  std::vector<int64_t> step_smem;
  std::vector<int64_t> step_grid;
  std::vector<void *> allocs;
  double *d_R = nullptr, *d_scratch = nullptr;
  peers::SweepArgs *d_table = nullptr;
  SweepItem *d_items = nullptr;
  int *d_counters = nullptr;
  int64_t nitems = 0, scratch_doubles = 0;
  bool use_graph = false;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t captured_on = nullptr;
};

namespace {

int balloc(peers_batch *b, void **p, size_t bytes, std::string &err) {
  *p = nullptr;
  if (bytes == 0) return PEERS_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    err = "cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PEERS_ENOMEM : PEERS_ECUDA;
  }
  b->allocs.push_back(*p);
  return PEERS_OK;
}

// Rough FMA count of an item, used only to order a step's items largest first.
int64_t item_cost(const Symbolic &S, const SweepItem &it) {
  if (it.kind == 2) return it.nq;
  const int64_t nc = peers::sn_nc(S, it.s), N = nc + S.nb[it.s], cols = nc - it.j0;
  return int64_t(it.nq) * cols * (N - it.j0 - cols / 2);
}

int build(peers_ctx *ctx, peers_batch *b, std::string &err) {
  DEVICE_SCOPE(ctx->device);
  b->device = ctx->device;
  // results and scratch: one carry region per graph (its waves run one after another)
  std::vector<int64_t> carry_off(b->count), racc_off(b->count);
  b->r_off.assign(b->count + 1, 0);
  int64_t sc = 0;
  for (int32_t i = 0; i < b->count; ++i) {
    const Symbolic &S = b->syms[i]->S;
    b->r_off[i + 1] = b->r_off[i] + S.nq;
    carry_off[i] = sc;
    sc += S.carry_slots * int64_t(S.nbmax);
    racc_off[i] = sc;
    sc += S.carry_slots;
  }
  b->r_total = b->r_off[b->count];
  b->scratch_doubles = sc;
  int rc = balloc(b, reinterpret_cast<void **>(&b->d_R), sizeof(double) * std::max<int64_t>(1, b->r_total), err);
  if (rc) return rc;
  rc = balloc(b, reinterpret_cast<void **>(&b->d_scratch), sizeof(double) * std::max<int64_t>(1, sc), err);
  if (rc) return rc;
  // one argument block per (graph, wave); each graph's step sequence
  std::vector<peers::SweepArgs> table;
  struct Step { int32_t g; int64_t i0, i1; int64_t k0, k1; const SweepItem *items; };
  std::vector<std::vector<Step>> seq(b->count);
  for (int32_t i = 0; i < b->count; ++i) {
    const Symbolic &S = b->syms[i]->S;
    const peers_numeric *num = b->nums[i];
    if (S.nsorted + S.nq_two == 0) continue;
    for (size_t w = 0; w < S.waves.size(); ++w) {
      const peers::SweepWave &W = S.waves[w];
      peers::SweepArgs a = sweep_args_of(num, S);
      a.carry = b->d_scratch + carry_off[i];
      a.racc = b->d_scratch + racc_off[i];
      a.R = b->d_R + b->r_off[i];
      a.wave_base = W.q_begin;
      const int32_t g = static_cast<int32_t>(table.size());
      table.push_back(a);
      for (int32_t l = 0; l < S.nlevels; ++l)
        if (W.level_ptr[l + 1] > W.level_ptr[l])
          seq[i].push_back({g, W.level_ptr[l], W.level_ptr[l + 1], 0, 0, W.items.data()});
      if (W.two_end > W.two_begin)
        seq[i].push_back({g, 0, 0, W.two_begin, W.two_end, nullptr});
    }
  }
  size_t T = 0;
  for (auto &q : seq) T = std::max(T, q.size());
  std::vector<SweepItem> all;
  std::vector<std::pair<int64_t, SweepItem>> step;
  b->step_ptr.assign(1, 0);
  b->step_smem.clear();
  for (size_t t = 0; t < T; ++t) {
    step.clear();
    int64_t smem = 0;
    for (int32_t i = 0; i < b->count; ++i) {
      // graphs are aligned at the top: every graph's last step (its roots) runs in the last
      // launch, so the heavy top levels of all graphs share launches instead of the deepest
      // graphs' top levels running nearly alone at the end
      const size_t lead = T - seq[i].size();
      if (t < lead) continue;
      const Step &st = seq[i][t - lead];
      const Symbolic &S = b->syms[i]->S;
      if (st.items) {
        for (int64_t k = st.i0; k < st.i1; ++k) {
          SweepItem it = st.items[k];
          it.g = st.g;
          step.push_back({item_cost(S, it), it});
          smem = std::max(smem, peers::sweep_smem_bytes(peers::sn_nc(S, it.s) + S.nb[it.s], it.nq));
        }
      } else {
        for (int64_t k = st.k0; k < st.k1; k += 4096) {
          SweepItem it{};
          it.kind = 2;
          it.q0 = static_cast<int32_t>(k);
          it.nq = static_cast<int32_t>(std::min<int64_t>(4096, st.k1 - k));
          it.g = st.g;
          step.push_back({item_cost(S, it), it});
        }
      }
    }
    std::stable_sort(step.begin(), step.end(),
                     [](const auto &x, const auto &y) { return x.first > y.first; });
    for (auto &x : step) all.push_back(x.second);
    b->step_ptr.push_back(static_cast<int64_t>(all.size()));
    b->step_smem.push_back(std::max<int64_t>(smem, 1024));
    int64_t grid = 0;
    rc = peers::multi_step_grid(b->step_smem.back(), static_cast<int64_t>(step.size()), &grid, err);
    if (rc) return rc;
    b->step_grid.push_back(grid);
  }
  b->nitems = static_cast<int64_t>(all.size());
  rc = balloc(b, reinterpret_cast<void **>(&b->d_items), sizeof(SweepItem) * std::max<size_t>(1, all.size()), err);
  if (rc) return rc;
  rc = balloc(b, reinterpret_cast<void **>(&b->d_table), sizeof(peers::SweepArgs) * std::max<size_t>(1, table.size()), err);
  if (rc) return rc;
  rc = balloc(b, reinterpret_cast<void **>(&b->d_counters), sizeof(int) * std::max<size_t>(1, T), err);
  if (rc) return rc;
  if (!all.empty())
    CUDA_TRY(cudaMemcpyAsync(b->d_items, all.data(), sizeof(SweepItem) * all.size(),
                             cudaMemcpyHostToDevice, ctx->stream));
  if (!table.empty())
    CUDA_TRY(cudaMemcpyAsync(b->d_table, table.data(), sizeof(peers::SweepArgs) * table.size(),
                             cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return PEERS_OK;
}

// The whole batched sweep as stream work (captured into a CUDA graph on first use).
int enqueue(peers_batch *b, cudaStream_t st, std::string &err) {
  const int64_t T = static_cast<int64_t>(b->step_smem.size());
  if (T > 0) CUDA_TRY(cudaMemsetAsync(b->d_counters, 0, sizeof(int) * T, st));
  if (b->r_total > 0) CUDA_TRY(cudaMemsetAsync(b->d_R, 0, sizeof(double) * b->r_total, st));
  for (int64_t t = 0; t < T; ++t) {
    const int64_t i0 = b->step_ptr[t], n = b->step_ptr[t + 1] - i0;
    if (n == 0) continue;
    int rc = peers::run_multi_step(b->d_items + i0, n, b->d_table, b->d_counters + t,
                                   b->step_smem[t], b->step_grid[t], st, err);
    if (rc != PEERS_OK) return rc;
  }
  return PEERS_OK;
}

int query(peers_ctx *ctx, peers_batch *b, double *const *R, int flags, std::string &err) {
  DEVICE_SCOPE(ctx->device);
  cudaStream_t st = ctx->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ctx->timing) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  if (b->use_graph) {
    if (!b->exec || b->captured_on != st) {
      if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
      }
      // warm the launch configuration (attributes, occupancy) outside the capture
      int rc = enqueue(b, st, err);
      if (rc != PEERS_OK) return rc;
      CUDA_TRY(cudaStreamSynchronize(st));
      cudaGraph_t graph = nullptr;
      CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      rc = enqueue(b, st, err);
      cudaError_t ec = cudaStreamEndCapture(st, &graph);
      if (rc != PEERS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (ec != cudaSuccess) {
        err = std::string("stream capture: ") + cudaGetErrorString(ec);
        return PEERS_ECUDA;
      }
      ec = cudaGraphInstantiate(&b->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ec != cudaSuccess) {
        err = std::string("graph instantiate: ") + cudaGetErrorString(ec);
        b->exec = nullptr;
        return PEERS_ECUDA;
      }
      b->captured_on = st;
    }
    CUDA_TRY(cudaGraphLaunch(b->exec, st));
  } else {
    int rc = enqueue(b, st, err);
    if (rc != PEERS_OK) return rc;
  }
  if (ctx->timing) {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ctx->stats.sweep_s = ms * 1e-3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  int64_t launches = 0;
  for (size_t t = 0; t + 1 < b->step_ptr.size(); ++t) launches += b->step_ptr[t + 1] > b->step_ptr[t];
  ctx->stats.sweep_launches = launches;
  ctx->stats.h2d_bytes = 0;
  ctx->stats.d2h_bytes = 0;
  if (R) {
    const cudaMemcpyKind kind = (flags & PEERS_OUT_DEVICE) ? cudaMemcpyDeviceToDevice
                                                           : cudaMemcpyDeviceToHost;
    for (int32_t i = 0; i < b->count; ++i) {
      const int64_t n = b->r_off[i + 1] - b->r_off[i];
      if (n > 0 && R[i]) {
        CUDA_TRY(cudaMemcpyAsync(R[i], b->d_R + b->r_off[i], sizeof(double) * n, kind, st));
        if (!(flags & PEERS_OUT_DEVICE)) ctx->stats.d2h_bytes += int64_t(sizeof(double)) * n;
      }
    }
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  CUDA_TRY(cudaGetLastError());
  return PEERS_OK;
}

}  // namespace

extern "C" {

int peers_batch_create(peers_ctx *ctx, int32_t count, const peers_symbolic *const *syms,
                       const peers_numeric *const *nums, int flags, peers_batch **out) {
  if (!out) return peers_fail(PEERS_EINVAL, "null output pointer");
  *out = nullptr;
  if (!ctx || count < 0 || (count > 0 && (!syms || !nums)))
    return peers_fail(PEERS_EINVAL, "null context or handle arrays");
  auto *b = new (std::nothrow) peers_batch;
  if (!b) return peers_fail(PEERS_ENOMEM, "host allocation");
  b->count = count;
  for (int32_t i = 0; i < count; ++i) {
    if (!syms[i] || !nums[i] || nums[i]->sym != syms[i] || nums[i]->device != ctx->device) {
      delete b;
      return peers_fail(PEERS_EINVAL, "batch entry " + std::to_string(i) +
                                          ": missing handle, foreign factor or other device");
    }
    if (syms[i]->S.spill_stride > 0) {
      delete b;
      return peers_fail(PEERS_EINVAL, "batch entry " + std::to_string(i) +
                                          " keeps fronts larger than shared memory in global "
                                          "memory; sweep it with peers_query");
    }
    b->syms.push_back(syms[i]);
    b->nums.push_back(nums[i]);
  }
  b->use_graph = (flags & PEERS_BATCH_CUDA_GRAPH) != 0;
  std::string err;
  int rc = build(ctx, b, err);
  if (rc != PEERS_OK) {
    peers_batch_free(b);
    return peers_fail(rc, err);
  }
  *out = b;
  return PEERS_OK;
}

int peers_batch_query(peers_ctx *ctx, peers_batch *b, double *const *R, int flags) {
  if (!ctx || !b) return peers_fail(PEERS_EINVAL, "null argument");
  if (b->device != ctx->device) return peers_fail(PEERS_EINVAL, "batch on another device");
  std::string err;
  int rc = query(ctx, b, R, flags, err);
  return rc == PEERS_OK ? rc : peers_fail(rc, err);
}

int peers_batch_info(const peers_batch *b, int64_t out[4]) {
  if (!b || !out) return peers_fail(PEERS_EINVAL, "null argument");
  int64_t launches = 0;
  for (size_t t = 0; t + 1 < b->step_ptr.size(); ++t) launches += b->step_ptr[t + 1] > b->step_ptr[t];
  out[0] = static_cast<int64_t>(b->step_smem.size());
  out[1] = b->nitems;
  out[2] = launches;
  out[3] = 8 * (b->r_total + b->scratch_doubles) +
           int64_t(sizeof(SweepItem)) * b->nitems;
  return PEERS_OK;
}

void peers_batch_free(peers_batch *b) {
  if (!b) return;
  {
    peers::DeviceGuard guard(b->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (void *p : b->allocs) cudaFree(p);
  }
  delete b;
}

int peers_query_batch(peers_ctx *ctx, int32_t count, const peers_symbolic *const *syms,
                      const peers_numeric *const *nums, double *const *R, int flags) {
  peers_batch *b = nullptr;
  int rc = peers_batch_create(ctx, count, syms, nums, 0, &b);
  if (rc != PEERS_OK) return rc;
  rc = peers_batch_query(ctx, b, R, flags);
  peers_batch_free(b);
  return rc;
}

}  // extern "C"
