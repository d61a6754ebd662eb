// Serving loop: requests (graph + queries) arrive at any time; each is analysed and factored
// by a worker thread, admitted by device-memory footprint, and then swept together with every
// other admitted request by continuous batching: one persistent launch per step carries the
// next etree level of every active request, requests join at the next step after their
// factor is ready and leave after their last level.  A request's arithmetic is exactly that
// of peers_query, so its result is the same alone and in the mix, bit for bit.
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
  size_t pos = 0;
  int32_t slot = -1;
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
  int64_t next_ticket = 1;
  std::map<int64_t, std::shared_ptr<Request>> reqs;
  std::deque<std::shared_ptr<Request>> pending;    // waiting for a worker
  std::deque<std::shared_ptr<Request>> factored;   // ready to join the sweep
  int64_t used_bytes = 0, peak_bytes = 0;
  int32_t admitted = 0;                             // factored + active
  std::vector<std::thread> workers;
  std::thread device_thread;
  // device thread state
  cudaStream_t stream = nullptr;
  peers::SweepArgs *d_table = nullptr;
  std::vector<char> slot_used;
  SweepItem *d_items[2] = {nullptr, nullptr};
  SweepItem *h_items[2] = {nullptr, nullptr};
  int64_t items_cap[2] = {0, 0};
  int *d_counter = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  // statistics
  std::vector<double> latencies;
  int64_t completed = 0, failed = 0, queries = 0, steps = 0, launches = 0;
  Clock::time_point t_first, t_last;
  bool any_submit = false;
  std::string fatal;
};

namespace {

constexpr int32_t kTableSlots = 16384;

void release_device(Request &r) {
  if (r.d_scratch) cudaFree(r.d_scratch);
  if (r.d_R) cudaFree(r.d_R);
  r.d_scratch = r.d_R = nullptr;
  if (r.num) peers_free_numeric(r.num);
  r.num = nullptr;
}

// Worker: analyse, wait for room under the memory budget, factor, allocate the sweep's
// per-request scratch, hand the request to the device thread.
void worker_main(peers_server *sv) {
  cudaSetDevice(sv->device);
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
        rc = peers_factor(ctx, r->sym, nullptr, &r->num);
        if (rc != PEERS_OK) r->err = peers_last_error();
      }
      if (rc == PEERS_OK) {
        const int64_t sc = S.carry_slots * (int64_t(S.nbmax) + 1);
        if (cudaMalloc(&r->d_scratch, sizeof(double) * std::max<int64_t>(1, sc)) != cudaSuccess ||
            cudaMalloc(&r->d_R, sizeof(double) * std::max<int64_t>(1, S.nq)) != cudaSuccess) {
          cudaGetLastError();
          rc = PEERS_ENOMEM;
          r->err = "device allocation of the request's sweep scratch";
        } else if (S.nq > 0 &&
                   cudaMemsetAsync(r->d_R, 0, sizeof(double) * S.nq, ctx->stream) != cudaSuccess) {
          rc = PEERS_ECUDA;
          r->err = "clearing the request's results";
        }
        cudaStreamSynchronize(ctx->stream);
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
    } else {
      r->err = peers_last_error();
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (rc != PEERS_OK) {
      release_device(*r);
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

int ensure_items(peers_server *sv, int b, int64_t n) {
  if (n <= sv->items_cap[b]) return PEERS_OK;
  const int64_t cap = std::max<int64_t>(n, 2 * sv->items_cap[b]);
  if (sv->d_items[b]) cudaFree(sv->d_items[b]);
  if (sv->h_items[b]) cudaFreeHost(sv->h_items[b]);
  sv->d_items[b] = nullptr;
  sv->h_items[b] = nullptr;
  sv->items_cap[b] = 0;
  if (cudaMalloc(&sv->d_items[b], sizeof(SweepItem) * cap) != cudaSuccess ||
      cudaMallocHost(&sv->h_items[b], sizeof(SweepItem) * cap) != cudaSuccess) {
    cudaGetLastError();
    return PEERS_ENOMEM;
  }
  sv->items_cap[b] = cap;
  return PEERS_OK;
}

int64_t step_cost(const Symbolic &S, const SweepItem &it) {
  if (it.kind == 2) return it.nq;
  const int64_t nc = peers::sn_nc(S, it.s), N = nc + S.nb[it.s], cols = nc - it.j0;
  return int64_t(it.nq) * cols * (N - it.j0 - cols / 2);
}

// Fills buffer b with the next step of every active request; returns the item count and the
// launch's shared memory.
int64_t prepare_step(peers_server *sv, int b, std::vector<std::shared_ptr<Request>> &active,
                     int64_t *smem_out, std::string &err) {
  std::vector<std::pair<int64_t, SweepItem>> step;
  int64_t smem = 1024;
  for (auto &r : active) {
    if (r->pos >= r->steps.size()) continue;
    const ReqStep &st = r->steps[r->pos];
    const Symbolic &S = r->sym->S;
    const int32_t g = r->slot + st.wave;
    if (!st.combine) {
      const SweepItem *src = S.waves[st.wave].items.data();
      for (int64_t k = st.i0; k < st.i1; ++k) {
        SweepItem it = src[k];
        it.g = g;
        step.push_back({step_cost(S, it), it});
        smem = std::max(smem, peers::sweep_smem_bytes(peers::sn_nc(S, it.s) + S.nb[it.s], it.nq));
      }
    } else {
      for (int64_t k = st.k0; k < st.k1; k += 4096) {
        SweepItem it{};
        it.kind = 2;
        it.q0 = static_cast<int32_t>(k);
        it.nq = static_cast<int32_t>(std::min<int64_t>(4096, st.k1 - k));
        it.g = g;
        step.push_back({it.nq, it});
      }
    }
  }
  std::stable_sort(step.begin(), step.end(),
                   [](const auto &x, const auto &y) { return x.first > y.first; });
  const int64_t n = static_cast<int64_t>(step.size());
  if (n == 0) return 0;
  if (ensure_items(sv, b, n) != PEERS_OK) {
    err = "device allocation of the step's work list";
    return -1;
  }
  for (int64_t i = 0; i < n; ++i) sv->h_items[b][i] = step[i].second;
  *smem_out = smem;
  return n;
}

void device_main(peers_server *sv) {
  cudaSetDevice(sv->device);
  std::vector<std::shared_ptr<Request>> active;
  std::vector<std::shared_ptr<Request>> finishing[2];
  int64_t pending_n[2] = {0, 0};
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
        sv->cv.wait(lk, [&] { return sv->stop || !sv->factored.empty(); });
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
      while (!sv->factored.empty()) {
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
        std::vector<peers::SweepArgs> blocks;
        const Symbolic &S = r->sym->S;
        for (const auto &W : S.waves) {
          peers::SweepArgs a = sweep_args_of(r->num, S);
          a.carry = r->d_scratch;
          a.racc = r->d_scratch + S.carry_slots * int64_t(S.nbmax);
          a.R = r->d_R;
          a.wave_base = W.q_begin;
          blocks.push_back(a);
        }
        if (!blocks.empty())
          cudaMemcpyAsync(sv->d_table + base, blocks.data(),
                          sizeof(peers::SweepArgs) * blocks.size(), cudaMemcpyHostToDevice,
                          sv->stream);
        if (r->steps.empty()) {   // nothing to walk (no queries or only u == v)
          finishing[cur].push_back(r);
        } else {
          active.push_back(r);
        }
      }
    }
    // 2. prepare and launch step `cur`
    int64_t smem = 0;
    const int64_t n = prepare_step(sv, cur, active, &smem, err);
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
      sv->steps++;
      sv->launches++;
    }
    // requests whose last step this is retire when the step completes
    std::vector<std::shared_ptr<Request>> still;
    for (auto &r : active) {
      if (r->pos < r->steps.size()) r->pos++;
      if (r->pos >= r->steps.size()) finishing[cur].push_back(r);
      else still.push_back(r);
    }
    active.swap(still);
    for (auto &r : finishing[cur]) {
      const int64_t nq = r->sym->S.nq;
      r->R.resize(static_cast<size_t>(nq));
      if (nq > 0)
        cudaMemcpyAsync(r->R.data(), r->d_R, sizeof(double) * nq, cudaMemcpyDeviceToHost,
                        sv->stream);
    }
    cudaEventRecord(sv->ev[cur], sv->stream);
    in_flight[cur] = true;
    pending_n[cur] = n;
    // 3. retire the previous step's finished requests once it has completed
    const int prev = cur ^ 1;
    if (in_flight[prev]) {
      const cudaError_t e = cudaEventSynchronize(sv->ev[prev]);
      in_flight[prev] = false;
      if (e != cudaSuccess) {
        fail_all(std::string("sweep step failed: ") + cudaGetErrorString(e));
        continue;
      }
      std::lock_guard<std::mutex> lk(sv->mu);
      for (auto &r : finishing[prev]) {
        r->t_done = Clock::now();
        for (int32_t k = 0; k < static_cast<int32_t>(r->sym->S.waves.size()); ++k)
          sv->slot_used[r->slot + k] = 0;
        release_device(*r);
        sv->used_bytes -= r->footprint;
        sv->admitted--;
        r->done = true;
        sv->completed++;
        sv->queries += r->sym->S.nq;
        sv->latencies.push_back(std::chrono::duration<double>(r->t_done - r->t_submit).count());
        sv->t_last = r->t_done;
      }
      finishing[prev].clear();
      sv->cv.notify_all();
    }
    (void)pending_n;
    cur ^= 1;
    if (active.empty() && !in_flight[cur] && !in_flight[cur ^ 1] && finishing[0].empty() &&
        finishing[1].empty())
      continue;
    if (active.empty() && in_flight[cur ^ 1]) {
      // nothing new to launch: drain the last step before sleeping
      const int last = cur ^ 1;
      const cudaError_t e = cudaEventSynchronize(sv->ev[last]);
      in_flight[last] = false;
      std::lock_guard<std::mutex> lk(sv->mu);
      if (e != cudaSuccess) sv->fatal = cudaGetErrorString(e);
      for (auto &r : finishing[last]) {
        r->t_done = Clock::now();
        for (int32_t k = 0; k < static_cast<int32_t>(r->sym->S.waves.size()); ++k)
          sv->slot_used[r->slot + k] = 0;
        release_device(*r);
        sv->used_bytes -= r->footprint;
        sv->admitted--;
        r->done = true;
        if (e != cudaSuccess) {
          r->status = PEERS_ECUDA;
          sv->failed++;
        } else {
          sv->completed++;
          sv->queries += r->sym->S.nq;
          sv->latencies.push_back(std::chrono::duration<double>(r->t_done - r->t_submit).count());
          sv->t_last = r->t_done;
        }
      }
      finishing[last].clear();
      sv->cv.notify_all();
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
  cudaSetDevice(device);
  sv->slot_used.assign(kTableSlots, 0);
  if (cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&sv->d_table, sizeof(peers::SweepArgs) * kTableSlots) != cudaSuccess ||
      cudaMalloc(&sv->d_counter, sizeof(int) * 2) != cudaSuccess ||
      cudaEventCreateWithFlags(&sv->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&sv->ev[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    peers_server_destroy(sv);
    return peers_fail(PEERS_ECUDA, "server device setup failed");
  }
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
  return PEERS_OK;
}

void peers_server_destroy(peers_server *sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto &t : sv->workers)
    if (t.joinable()) t.join();
  sv->cv.notify_all();
  if (sv->device_thread.joinable()) sv->device_thread.join();
  cudaSetDevice(sv->device);
  for (auto &kv : sv->reqs) {
    release_device(*kv.second);
    if (kv.second->sym) peers_free_symbolic(kv.second->sym);
  }
  for (int b = 0; b < 2; ++b) {
    if (sv->d_items[b]) cudaFree(sv->d_items[b]);
    if (sv->h_items[b]) cudaFreeHost(sv->h_items[b]);
    if (sv->ev[b]) cudaEventDestroy(sv->ev[b]);
  }
  if (sv->d_table) cudaFree(sv->d_table);
  if (sv->d_counter) cudaFree(sv->d_counter);
  if (sv->stream) cudaStreamDestroy(sv->stream);
  delete sv;
}

}  // extern "C"
