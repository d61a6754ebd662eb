// Serving loop: requests (graph + queries) arrive at any time; each is analysed and factored
// by a worker thread, admitted by device-memory footprint, and then swept together with every
// other admitted request by continuous batching: one persistent launch per step carries work
// of every active request, requests join at the next step after their factor is ready and
// leave after their last level.  A request's arithmetic is exactly that of peers_query, so its
// result is the same alone and in the mix, bit for bit.
//
// Time slicing.  The items of one etree level of one request are independent of each other
// (eq. 16-18 per query; a query's next level needs only its own previous level), so a level
// may be spread over several steps.  Each step gives every active request a share of about
// kStepQuantum / (active requests) multiply-adds of its current level (whole levels when they
// are smaller, at least one item), so a step lasts about one quantum whatever the requests'
// sizes: a small request is never held for the length of a large request's root level, and
// a large one keeps the GPU busy between the small ones' levels.
//
// Device memory.  Every request's factor and sweep scratch come from one memory pool of the
// server, allocated on the worker's stream and returned on the server's stream
// (cudaMallocFromPoolAsync / cudaFreeAsync), so neither admitting nor retiring a request
// synchronises the device under the running steps.  Results are copied to pinned staging
// buffers, one per step in flight, so the copy does not block the step thread either.
//
// Threads: `workers` analysis/factor threads (each with its own CUDA stream, so factoring
// overlaps the sweep on the device) and one device thread that runs the steps.  The device
// thread prepares step t+1 while step t runs and retires the requests finished by step t
// once its completion event fires.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "device.cuh"
#include "handles.h"
#include "internal.h"
#include "peers.h"

namespace {

using Clock = std::chrono::steady_clock;

// Multiply-adds of one step (about 4 ms of the sweep kernel on a B300 at its FP64 rate).
constexpr int64_t kStepQuantum = int64_t(2500) * 1000 * 1000;

struct ReqStep {
  int32_t wave;           // argument block of the request: slot base + wave
  int64_t i0, i1;         // items of the wave's level (when combine == false)
  int64_t k0, k1;         // two-branch queries to combine (when combine == true)
  bool combine;
};

struct Request {
  int64_t ticket = 0;
  // inputs (copied at submit)
  int64_t n = 0;
  std::vector<int64_t> indptr;
  std::vector<int32_t> indices;
  std::vector<double> w;
  int32_t ground = 0;
  bool all_edges = true;
  std::vector<int32_t> qu, qv;
  std::vector<double> coords;
  int dim = 0;
  // state
  int status = PEERS_OK;
  std::string err;
  bool done = false;
  peers_symbolic *sym = nullptr;
  peers_numeric *num = nullptr;
  int64_t footprint = 0;
  double *d_scratch = nullptr, *d_R = nullptr;
  std::vector<ReqStep> steps;
  size_t pos = 0;          // current entry of `steps`
  int64_t next = 0;        // items of steps[pos] already issued
  int64_t issue_end = 0;   // items of steps[pos] issued once the step being prepared runs
  int64_t steps_in = 0;    // sweep steps that carried work of this request
  int32_t slot = -1;
  int64_t staged = -1;     // offset of the results in the pinned staging buffer
  std::vector<double> R;
  Clock::time_point t_submit, t_done;
};

}  // namespace

struct peers_server {
  int device = 0;
  peers_options opt{};
  int64_t budget = 0;
  int32_t max_active = 0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  bool hold = false;                                // factored requests wait to join
  int64_t next_ticket = 1;
  std::map<int64_t, std::shared_ptr<Request>> reqs;
  std::deque<std::shared_ptr<Request>> pending;    // waiting for a worker
  std::deque<std::shared_ptr<Request>> factored;   // ready to join the sweep
  int64_t used_bytes = 0, peak_bytes = 0;
  int32_t admitted = 0;                             // factored + active
  std::vector<std::thread> workers;
  std::thread device_thread;
  // device memory of the requests (stream-ordered)
  cudaMemPool_t pool = nullptr;
  // device thread state
  cudaStream_t stream = nullptr;
  peers::SweepArgs *d_table = nullptr;
  peers::SweepArgs *h_table = nullptr;              // pinned mirror of d_table
  std::vector<char> slot_used;
  SweepItem *d_items[2] = {nullptr, nullptr};
  SweepItem *h_items[2] = {nullptr, nullptr};
  int64_t items_cap[2] = {0, 0};
  double *h_stage[2] = {nullptr, nullptr};          // pinned result staging per step in flight
  int64_t stage_cap[2] = {0, 0};
  int *d_counter = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // statistics
  std::vector<double> latencies;
  int64_t completed = 0, failed = 0, queries = 0, steps = 0, launches = 0;
  int64_t max_step_requests = 0, request_steps = 0;
  Clock::time_point t_first, t_last;
  bool any_submit = false;
  std::string fatal;
};

namespace {

constexpr int32_t kTableSlots = 16384;

// Returns a request's device memory to the server's pool, ordered after the work already
// issued on `stream`.
void release_device(Request &r, cudaStream_t stream) {
  if (r.d_scratch) cudaFreeAsync(r.d_scratch, stream);
  if (r.d_R) cudaFreeAsync(r.d_R, stream);
  r.d_scratch = r.d_R = nullptr;
  if (r.num) {
    r.num->pool_stream = stream;
    peers_free_numeric(r.num);
  }
  r.num = nullptr;
}

// Worker: analyse, wait for room under the memory budget, factor, allocate the sweep's
// per-request scratch, hand the request to the device thread.
void worker_main(peers_server *sv) {
  cudaSetDevice(sv->device);
  // the workers already analyse requests side by side: each analysis keeps to its thread, so
  // that they leave the host cores to each other and to the device thread
  peers::set_host_thread_cap(1);
  peers_ctx *ctx = nullptr;
  if (peers_create(&ctx, sv->device, nullptr) != PEERS_OK) return;
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv.wait(lk, [&] { return sv->stop || !sv->pending.empty(); });
      if (sv->pending.empty()) break;
      r = sv->pending.front();
      sv->pending.pop_front();
    }
    int rc = peers_analyze(nullptr, r->n, r->indptr.data(), r->indices.data(), r->w.data(),
                           r->ground, r->all_edges ? -1 : static_cast<int64_t>(r->qu.size()),
                           r->all_edges ? nullptr : r->qu.data(),
                           r->all_edges ? nullptr : r->qv.data(),
                           r->coords.empty() ? nullptr : r->coords.data(), r->dim, &sv->opt,
                           &r->sym);
    bool reserved = false;
    if (rc == PEERS_OK && r->sym->S.spill_stride > 0) {
      rc = PEERS_EINVAL;
      r->err = "the request has supernode fronts larger than shared memory, which the server's "
               "batched sweep does not take: use peers_query";
    }
    if (rc == PEERS_OK) {
      const Symbolic &S = r->sym->S;
      r->footprint = peers_footprint_bytes(r->sym);
      // admission by footprint: wait until the request fits next to the admitted ones
      std::unique_lock<std::mutex> lk(sv->mu);
      if (r->footprint > sv->budget) {
        rc = PEERS_ENOMEM;
        r->err = "request needs " + std::to_string(r->footprint) +
                 " device bytes, more than the server's budget";
      } else {
        sv->cv.wait(lk, [&] {
          return sv->stop || (sv->used_bytes + r->footprint <= sv->budget &&
                              sv->admitted < sv->max_active);
        });
        if (sv->stop) {
          rc = PEERS_EINVAL;
          r->err = "server stopped";
        } else {
          sv->used_bytes += r->footprint;
          sv->peak_bytes = std::max(sv->peak_bytes, sv->used_bytes);
          sv->admitted++;
          reserved = true;
        }
      }
      lk.unlock();
      if (rc == PEERS_OK) {
        std::string err;
        rc = factor_from_pool(ctx, r->sym, nullptr, sv->pool, &r->num, err);
        if (rc != PEERS_OK) r->err = err;
      }
      if (rc == PEERS_OK) {
        const int64_t sc = S.carry_slots * (int64_t(S.nbmax) + 1);
        void *a = nullptr, *b = nullptr;
        if (cudaMallocFromPoolAsync(&a, sizeof(double) * std::max<int64_t>(1, sc), sv->pool,
                                    ctx->stream) != cudaSuccess ||
            cudaMallocFromPoolAsync(&b, sizeof(double) * std::max<int64_t>(1, S.nq), sv->pool,
                                    ctx->stream) != cudaSuccess) {
          cudaGetLastError();
          rc = PEERS_ENOMEM;
          r->err = "device allocation of the request's sweep scratch";
        }
        r->d_scratch = static_cast<double *>(a);
        r->d_R = static_cast<double *>(b);
        if (rc == PEERS_OK && S.nq > 0 &&
            cudaMemsetAsync(r->d_R, 0, sizeof(double) * S.nq, ctx->stream) != cudaSuccess) {
          rc = PEERS_ECUDA;
          r->err = "clearing the request's results";
        }
        // the factor, the scratch and the cleared R are ready for the server's stream
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && rc == PEERS_OK) {
          rc = PEERS_ECUDA;
          r->err = "factorization stream failed";
        }
      }
      if (rc == PEERS_OK) {
        for (size_t wv = 0; wv < S.waves.size() && S.nsorted + S.nq_two > 0; ++wv) {
          const peers::SweepWave &W = S.waves[wv];
          for (int32_t l = 0; l < S.nlevels; ++l)
            if (W.level_ptr[l + 1] > W.level_ptr[l])
              r->steps.push_back({static_cast<int32_t>(wv), W.level_ptr[l], W.level_ptr[l + 1],
                                  0, 0, false});
          if (W.two_end > W.two_begin)
            r->steps.push_back({static_cast<int32_t>(wv), 0, 0, W.two_begin, W.two_end, true});
        }
      }
      if (rc != PEERS_OK && reserved) {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->used_bytes -= r->footprint;
        sv->admitted--;
      }
    } else if (r->err.empty()) {
      r->err = peers_last_error();
    }
    if (rc != PEERS_OK) {
      release_device(*r, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (rc != PEERS_OK) {
      r->status = rc;
      r->done = true;
      r->t_done = Clock::now();
      sv->failed++;
    } else {
      sv->factored.push_back(r);
    }
    sv->cv.notify_all();
  }
  peers_destroy(ctx);
}

// Grows a pinned/device buffer pair of the step thread to hold at least n entries.  Only
// called for buffer b while no step that reads it is in flight.
int ensure_items(peers_server *sv, int b, int64_t n) {
  if (n <= sv->items_cap[b]) return PEERS_OK;
  const int64_t cap = std::max<int64_t>(n, 2 * sv->items_cap[b]);
  if (sv->d_items[b]) cudaFreeAsync(sv->d_items[b], sv->stream);
  if (sv->h_items[b]) cudaFreeHost(sv->h_items[b]);
  sv->d_items[b] = nullptr;
  sv->h_items[b] = nullptr;
  sv->items_cap[b] = 0;
  void *d = nullptr;
  if (cudaMallocFromPoolAsync(&d, sizeof(SweepItem) * cap, sv->pool, sv->stream) != cudaSuccess ||
      cudaMallocHost(&sv->h_items[b], sizeof(SweepItem) * cap) != cudaSuccess) {
    cudaGetLastError();
    if (d) cudaFreeAsync(d, sv->stream);
    return PEERS_ENOMEM;
  }
  sv->d_items[b] = static_cast<SweepItem *>(d);
  sv->items_cap[b] = cap;
  return PEERS_OK;
}

int ensure_stage(peers_server *sv, int b, int64_t n) {
  if (n <= sv->stage_cap[b]) return PEERS_OK;
  const int64_t cap = std::max<int64_t>(n, 2 * sv->stage_cap[b]);
  if (sv->h_stage[b]) cudaFreeHost(sv->h_stage[b]);
  sv->h_stage[b] = nullptr;
  sv->stage_cap[b] = 0;
  if (cudaMallocHost(&sv->h_stage[b], sizeof(double) * cap) != cudaSuccess) {
    cudaGetLastError();
    return PEERS_ENOMEM;
  }
  sv->stage_cap[b] = cap;
  return PEERS_OK;
}

int64_t step_cost(const Symbolic &S, const SweepItem &it) {
  if (it.kind == 2) return it.nq;
  const int64_t nc = peers::sn_nc(S, it.s), N = nc + S.nb[it.s], cols = nc - it.j0;
  return std::max<int64_t>(1, int64_t(it.nq) * cols * (N - it.j0 - cols / 2));
}

// Fills buffer b with the next step: a share of the current level of every active request
// (see the time slicing note at the top).  Sets each request's issue_end; returns the item
// count, the launch's shared memory and the number of requests in the step.
int64_t prepare_step(peers_server *sv, int b, std::vector<std::shared_ptr<Request>> &active,
                     int64_t *smem_out, int64_t *nreq_out, std::string &err) {
  std::vector<std::pair<int64_t, SweepItem>> step;
  int64_t smem = 1024, nreq = 0;
  int64_t sweeping = 0;
  for (auto &r : active)
    if (r->pos < r->steps.size() && !r->steps[r->pos].combine) ++sweeping;
  const int64_t share = std::max<int64_t>(1, kStepQuantum / std::max<int64_t>(1, sweeping));
  for (auto &r : active) {
    r->issue_end = r->next;
    if (r->pos >= r->steps.size()) continue;
    const ReqStep &st = r->steps[r->pos];
    const Symbolic &S = r->sym->S;
    const int32_t g = r->slot + st.wave;
    ++nreq;
    if (!st.combine) {
      const SweepItem *src = S.waves[st.wave].items.data();
      int64_t k = st.i0 + r->next, spent = 0;
      while (k < st.i1 && (spent < share || k == st.i0 + r->next)) {
        SweepItem it = src[k];
        it.g = g;
        const int64_t c = step_cost(S, it);
        spent += c;
        step.push_back({c, it});
        smem = std::max(smem, peers::sweep_smem_bytes(peers::sn_nc(S, it.s) + S.nb[it.s], it.nq));
        ++k;
      }
      r->issue_end = k - st.i0;
    } else {
      for (int64_t k = st.k0; k < st.k1; k += 4096) {
        SweepItem it{};
        it.kind = 2;
        it.q0 = static_cast<int32_t>(k);
        it.nq = static_cast<int32_t>(std::min<int64_t>(4096, st.k1 - k));
        it.g = g;
        step.push_back({it.nq, it});
      }
      r->issue_end = 0;
    }
  }
  std::stable_sort(step.begin(), step.end(),
                   [](const auto &x, const auto &y) { return x.first > y.first; });
  const int64_t n = static_cast<int64_t>(step.size());
  *nreq_out = nreq;
  if (n == 0) return 0;
  if (ensure_items(sv, b, n) != PEERS_OK) {
    err = "allocation of the step's work list";
    return -1;
  }
  for (int64_t i = 0; i < n; ++i) sv->h_items[b][i] = step[i].second;
  *smem_out = smem;
  return n;
}

// Records the completion of the requests of finishing[b] (their step has finished).
void retire(peers_server *sv, std::vector<std::shared_ptr<Request>> &fin, int b, cudaError_t e) {
  std::lock_guard<std::mutex> lk(sv->mu);
  if (e != cudaSuccess) sv->fatal = cudaGetErrorString(e);
  for (auto &r : fin) {
    r->t_done = Clock::now();
    const int64_t nq = r->sym->S.nq;
    if (e == cudaSuccess && nq > 0 && r->staged >= 0)
      std::memcpy(r->R.data(), sv->h_stage[b] + r->staged, sizeof(double) * nq);
    for (int32_t k = 0; k < static_cast<int32_t>(r->sym->S.waves.size()); ++k)
      sv->slot_used[r->slot + k] = 0;
    release_device(*r, sv->stream);
    sv->used_bytes -= r->footprint;
    sv->admitted--;
    r->done = true;
    if (e != cudaSuccess) {
      r->status = PEERS_ECUDA;
      r->err = std::string("sweep step failed: ") + cudaGetErrorString(e);
      sv->failed++;
    } else {
      sv->completed++;
      sv->queries += nq;
      sv->request_steps += r->steps_in;
      sv->latencies.push_back(std::chrono::duration<double>(r->t_done - r->t_submit).count());
      sv->t_last = r->t_done;
    }
  }
  fin.clear();
  sv->cv.notify_all();
}

void device_main(peers_server *sv) {
  cudaSetDevice(sv->device);
  std::vector<std::shared_ptr<Request>> active;
  std::vector<std::shared_ptr<Request>> finishing[2];
  bool in_flight[2] = {false, false};
  int cur = 0;
  std::string err;
  auto fail_all = [&](const std::string &msg) {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->fatal = msg;
    for (auto &r : active) {
      r->status = PEERS_ECUDA;
      r->err = msg;
      r->done = true;
      r->t_done = Clock::now();
      sv->failed++;
    }
    active.clear();
    sv->cv.notify_all();
  };
  for (;;) {
    // 1. admit factored requests (they join at the next prepared step)
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      if (active.empty() && !in_flight[0] && !in_flight[1]) {
        sv->cv.wait(lk, [&] { return sv->stop || (!sv->factored.empty() && !sv->hold); });
        if (sv->factored.empty() && sv->stop && sv->pending.empty() && sv->admitted == 0) break;
        if (sv->factored.empty() && sv->stop) {
          // stop requested while workers still hold requests: keep waiting for them
          sv->cv.wait_for(lk, std::chrono::milliseconds(5));
          if (sv->factored.empty()) {
            if (sv->pending.empty() && sv->admitted == 0) break;
            continue;
          }
        }
      }
      while (!sv->factored.empty() && !sv->hold) {
        auto r = sv->factored.front();
        const int32_t need = static_cast<int32_t>(r->sym->S.waves.size());
        int32_t base = -1;
        for (int32_t s0 = 0; s0 + need <= kTableSlots && base < 0; ++s0) {
          bool ok = true;
          for (int32_t k = 0; k < need && ok; ++k) ok = !sv->slot_used[s0 + k];
          if (ok) base = s0;
        }
        if (base < 0) break;   // table full: wait for retirements
        sv->factored.pop_front();
        for (int32_t k = 0; k < need; ++k) sv->slot_used[base + k] = 1;
        r->slot = base;
        const Symbolic &S = r->sym->S;
        for (int32_t k = 0; k < need; ++k) {
          peers::SweepArgs a = sweep_args_of(r->num, S);
          a.carry = r->d_scratch;
          a.racc = r->d_scratch + S.carry_slots * int64_t(S.nbmax);
          a.R = r->d_R;
          a.wave_base = S.waves[k].q_begin;
          sv->h_table[base + k] = a;   // slots of retired requests only: no copy reads them
        }
        if (need > 0)
          cudaMemcpyAsync(sv->d_table + base, sv->h_table + base, sizeof(peers::SweepArgs) * need,
                          cudaMemcpyHostToDevice, sv->stream);
        r->R.resize(static_cast<size_t>(S.nq));
        if (r->steps.empty()) {   // nothing to walk (no queries or only u == v)
          finishing[cur].push_back(r);
        } else {
          active.push_back(r);
        }
      }
    }
    // 2. prepare and launch step `cur`
    int64_t smem = 0, nreq = 0;
    const int64_t n = prepare_step(sv, cur, active, &smem, &nreq, err);
    if (n < 0) {
      fail_all(err);
      continue;
    }
    if (n > 0) {
      int64_t grid = 0;
      bool ok = cudaMemcpyAsync(sv->d_items[cur], sv->h_items[cur], sizeof(SweepItem) * n,
                                cudaMemcpyHostToDevice, sv->stream) == cudaSuccess &&
                cudaMemsetAsync(sv->d_counter + cur, 0, sizeof(int), sv->stream) == cudaSuccess &&
                peers::multi_step_grid(smem, n, &grid, err) == PEERS_OK &&
                peers::run_multi_step(sv->d_items[cur], n, sv->d_table, sv->d_counter + cur,
                                      smem, grid, sv->stream, err) == PEERS_OK;
      if (!ok) {
        fail_all("sweep step launch failed: " + err);
        continue;
      }
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->steps++;
      sv->launches++;
      sv->max_step_requests = std::max(sv->max_step_requests, nreq);
    }
    // advance every request past what this step issued; the finished ones retire when the
    // step completes
    std::vector<std::shared_ptr<Request>> still;
    for (auto &r : active) {
      if (r->pos < r->steps.size()) {
        r->steps_in++;
        const ReqStep &st = r->steps[r->pos];
        if (st.combine || r->issue_end >= st.i1 - st.i0) {
          r->pos++;
          r->next = 0;
        } else {
          r->next = r->issue_end;
        }
      }
      if (r->pos >= r->steps.size()) finishing[cur].push_back(r);
      else still.push_back(r);
    }
    active.swap(still);
    {
      int64_t total = 0;
      for (auto &r : finishing[cur]) total += r->sym->S.nq;
      if (ensure_stage(sv, cur, total) != PEERS_OK) {
        fail_all("pinned allocation of the result staging buffer");
        continue;
      }
      int64_t off = 0;
      for (auto &r : finishing[cur]) {
        const int64_t nq = r->sym->S.nq;
        r->staged = off;
        if (nq > 0)
          cudaMemcpyAsync(sv->h_stage[cur] + off, r->d_R, sizeof(double) * nq,
                          cudaMemcpyDeviceToHost, sv->stream);
        off += nq;
      }
    }
    cudaEventRecord(sv->ev[cur], sv->stream);
    in_flight[cur] = true;
    // 3. retire the previous step's finished requests once it has completed
    const int prev = cur ^ 1;
    if (in_flight[prev]) {
      const cudaError_t e = cudaEventSynchronize(sv->ev[prev]);
      in_flight[prev] = false;
      retire(sv, finishing[prev], prev, e);
      if (e != cudaSuccess) {
        fail_all(std::string("sweep step failed: ") + cudaGetErrorString(e));
        continue;
      }
    }
    cur ^= 1;
    if (active.empty() && in_flight[cur ^ 1]) {
      // nothing new to launch: drain the last step before sleeping
      const int last = cur ^ 1;
      const cudaError_t e = cudaEventSynchronize(sv->ev[last]);
      in_flight[last] = false;
      retire(sv, finishing[last], last, e);
    }
  }
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double idx = p * (v.size() - 1);
  const size_t lo = static_cast<size_t>(idx);
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (v[hi] - v[lo]) * (idx - lo);
}

}  // namespace

extern "C" {

int peers_server_create(int device, int64_t mem_budget_bytes, int32_t max_active,
                        int32_t workers, const peers_options *opt, peers_server **out) {
  if (!out) return peers_fail(PEERS_EINVAL, "null output pointer");
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return peers_fail(PEERS_EINVAL, "no such CUDA device");
  }
  auto *sv = new (std::nothrow) peers_server;
  if (!sv) return peers_fail(PEERS_ENOMEM, "host allocation");
  sv->device = device;
  if (opt) sv->opt = *opt;
  sv->budget = mem_budget_bytes > 0 ? mem_budget_bytes : (int64_t(64) << 30);
  sv->max_active = max_active > 0 ? max_active : 64;
  if (workers <= 0) workers = 4;
  peers::DeviceGuard guard(device);
  sv->slot_used.assign(kTableSlots, 0);
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  // keep freed memory in the pool (no release to the driver at synchronisation points)
  uint64_t keep = UINT64_MAX;
  void *tbl = nullptr, *ctr = nullptr;
  if (guard.status() != cudaSuccess ||
      cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMemPoolCreate(&sv->pool, &props) != cudaSuccess ||
      cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
      cudaMalloc(&tbl, sizeof(peers::SweepArgs) * kTableSlots) != cudaSuccess ||
      cudaMallocHost(&sv->h_table, sizeof(peers::SweepArgs) * kTableSlots) != cudaSuccess ||
      cudaMalloc(&ctr, sizeof(int) * 2) != cudaSuccess ||
      cudaEventCreateWithFlags(&sv->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&sv->ev[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    sv->d_table = static_cast<peers::SweepArgs *>(tbl);
    sv->d_counter = static_cast<int *>(ctr);
    peers_server_destroy(sv);
    return peers_fail(PEERS_ECUDA, "server device setup failed");
  }
  sv->d_table = static_cast<peers::SweepArgs *>(tbl);
  sv->d_counter = static_cast<int *>(ctr);
  for (int32_t i = 0; i < workers; ++i) sv->workers.emplace_back(worker_main, sv);
  sv->device_thread = std::thread(device_main, sv);
  *out = sv;
  return PEERS_OK;
}

int peers_server_submit(peers_server *sv, int64_t n, const int64_t *indptr,
                        const int32_t *indices, const double *w, int32_t ground, int64_t nq,
                        const int32_t *qu, const int32_t *qv, const double *coords, int dim,
                        int64_t *ticket) {
  if (!sv || !ticket || !indptr || !indices || !w || n < 2)
    return peers_fail(PEERS_EINVAL, "null argument or graph with fewer than two nodes");
  auto r = std::make_shared<Request>();
  r->n = n;
  r->indptr.assign(indptr, indptr + n + 1);
  const int64_t nnz = indptr[n];
  if (nnz < 0) return peers_fail(PEERS_EINVAL, "bad indptr");
  r->indices.assign(indices, indices + nnz);
  r->w.assign(w, w + nnz);
  r->ground = ground;
  r->all_edges = nq < 0 || !qu || !qv;
  if (!r->all_edges) {
    r->qu.assign(qu, qu + nq);
    r->qv.assign(qv, qv + nq);
  }
  if (coords && dim > 0) {
    r->coords.assign(coords, coords + n * dim);
    r->dim = dim;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) return peers_fail(PEERS_EINVAL, "server is stopping");
  r->ticket = sv->next_ticket++;
  r->t_submit = Clock::now();
  if (!sv->any_submit) {
    sv->any_submit = true;
    sv->t_first = r->t_submit;
  }
  sv->reqs[r->ticket] = r;
  sv->pending.push_back(r);
  *ticket = r->ticket;
  sv->cv.notify_all();
  return PEERS_OK;
}

int peers_server_poll(peers_server *sv, int64_t ticket) {
  if (!sv) return peers_fail(PEERS_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return peers_fail(PEERS_EINVAL, "unknown ticket");
  if (!it->second->done) return 0;
  return it->second->status == PEERS_OK ? 1 : it->second->status;
}

int peers_server_wait(peers_server *sv, int64_t ticket, double *R, int64_t cap,
                      double *latency_s) {
  if (!sv) return peers_fail(PEERS_EINVAL, "null server");
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return peers_fail(PEERS_EINVAL, "unknown ticket");
    r = it->second;
    sv->cv.wait(lk, [&] { return r->done; });
    sv->reqs.erase(it);
  }
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  if (r->status != PEERS_OK) return peers_fail(r->status, r->err);
  if (R) {
    const int64_t n = std::min<int64_t>(cap, static_cast<int64_t>(r->R.size()));
    std::copy(r->R.begin(), r->R.begin() + n, R);
  }
  if (r->sym) peers_free_symbolic(r->sym);
  r->sym = nullptr;
  return PEERS_OK;
}

int peers_server_get_stats(peers_server *sv, peers_server_stats *out) {
  if (!sv || !out) return peers_fail(PEERS_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = sv->next_ticket - 1;
  out->completed = sv->completed;
  out->failed = sv->failed;
  out->queries = sv->queries;
  out->steps = sv->steps;
  out->launches = sv->launches;
  out->peak_bytes = sv->peak_bytes;
  out->p50_s = percentile(sv->latencies, 0.50);
  out->p99_s = percentile(sv->latencies, 0.99);
  double sum = 0;
  for (double x : sv->latencies) sum += x;
  out->mean_s = sv->latencies.empty() ? 0.0 : sum / sv->latencies.size();
  out->wall_s = sv->any_submit && sv->completed
                    ? std::chrono::duration<double>(sv->t_last - sv->t_first).count()
                    : 0.0;
  out->qps = out->wall_s > 0 ? sv->queries / out->wall_s : 0.0;
  out->max_step_requests = sv->max_step_requests;
  out->request_steps = sv->request_steps;
  out->ready = static_cast<int64_t>(sv->factored.size());
  return PEERS_OK;
}

int peers_server_hold(peers_server *sv, int hold) {
  if (!sv) return peers_fail(PEERS_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->hold = hold != 0;
  sv->cv.notify_all();
  return PEERS_OK;
}

void peers_server_destroy(peers_server *sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->hold = false;
  }
  sv->cv.notify_all();
  for (auto &t : sv->workers)
    if (t.joinable()) t.join();
  sv->cv.notify_all();
  if (sv->device_thread.joinable()) sv->device_thread.join();
  peers::DeviceGuard guard(sv->device);
  for (auto &kv : sv->reqs) {
    if (sv->stream) release_device(*kv.second, sv->stream);
    if (kv.second->sym) peers_free_symbolic(kv.second->sym);
  }
  for (int b = 0; b < 2; ++b) {
    if (sv->d_items[b]) cudaFreeAsync(sv->d_items[b], sv->stream);
    if (sv->h_items[b]) cudaFreeHost(sv->h_items[b]);
    if (sv->h_stage[b]) cudaFreeHost(sv->h_stage[b]);
    if (sv->ev[b]) cudaEventDestroy(sv->ev[b]);
  }
  if (sv->stream) cudaStreamSynchronize(sv->stream);
  if (sv->pool) cudaMemPoolDestroy(sv->pool);
  if (sv->h_table) cudaFreeHost(sv->h_table);
  if (sv->d_table) cudaFree(sv->d_table);
  if (sv->d_counter) cudaFree(sv->d_counter);
  if (sv->stream) cudaStreamDestroy(sv->stream);
  delete sv;
}

}  // extern "C"
