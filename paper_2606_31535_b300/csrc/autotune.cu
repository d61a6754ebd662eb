// Tile-shape autotuner for the sweep: how many queries one CTA carries through a supernode.
//
// Larger tiles reuse each panel value for more queries but hold more shared memory per CTA,
// which lowers the number of CTAs an SM can keep resident to hide barriers and load
// latency; the best trade-off depends on the front size.  For each front-size class the
// tuner times every candidate cap on the heaviest supernodes of that class of the actual
// plan (real panels, the resident factor), keeps the fastest, re-tiles the plan and writes
// the choice into a small cache file keyed by GPU name and class, so later runs on the same
// kind of GPU skip the measurements.  Re-tiling never changes a query's arithmetic (column
// blocks stay aligned), so results are identical under any tile choice.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "device.cuh"
#include "handles.h"
#include "internal.h"
#include "peers.h"

namespace {

using peers::kBlock;
using peers::SweepItem;


int64_t items_fma(const Symbolic &S, int32_t s, int32_t j0) {
  const int64_t nc = peers::sn_nc(S, s), N = nc + S.nb[s];
  int64_t f = 0;
  for (int64_t J = j0; J < nc; J += kBlock) {
    const int64_t bw = std::min<int64_t>(kBlock, nc - J);
    f += bw * (bw - 1) / 2 + (N - J - bw) * bw + bw;
  }
  return f;
}

// Items of the first wave for supernodes `sns`, tiled with cap `cap`; at most limit[i]
// queries of each of supernode i's sources are taken (the same ones for every cap).
std::vector<SweepItem> tile_items(const Symbolic &S, const std::vector<int32_t> &sns,
                                  const std::vector<int64_t> &limit, int32_t cap) {
  const peers::SweepWave &W = S.waves[0];
  std::vector<SweepItem> out;
  for (size_t i = 0; i < sns.size(); ++i) {
    const int32_t p = sns[i];
    const int64_t N = peers::sn_nc(S, p) + S.nb[p];
    const int64_t tile = peers::sweep_tile(S, N, cap);
    auto emit = [&](int32_t src, int64_t b, int64_t e) {
      b = std::max(b, W.q_begin);
      e = std::min(e, W.q_end);
      e = std::min(e, b + limit[i]);
      for (int64_t q = b; q < e; q += tile) {
        SweepItem it{};
        it.s = p;
        it.src = src;
        it.q0 = static_cast<int32_t>(q);
        it.nq = static_cast<int32_t>(std::min<int64_t>(tile, e - q));
        const int32_t j0 = src >= 0 ? S.rmap[S.rows_off[src]] : S.qa[q];
        it.j0 = (j0 / kBlock) * kBlock;
        out.push_back(it);
      }
    };
    for (int32_t c = S.child_ptr[p]; c < S.child_ptr[p + 1]; ++c) {
      const int32_t ch = S.child_list[c];
      emit(ch, S.qbeg[S.fdesc[ch]], S.qbeg[ch + 1]);
    }
    emit(-1, S.qbeg[p], S.qbeg[p + 1]);
  }
  return out;
}

std::map<std::string, int32_t> read_cache(const char *path) {
  std::map<std::string, int32_t> m;
  if (!path) return m;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    const size_t bar = line.rfind('|');
    if (bar == std::string::npos) continue;
    try {
      m[line.substr(0, bar)] = std::stoi(line.substr(bar + 1));
    } catch (...) {
    }
  }
  return m;
}

void write_cache(const char *path, const std::map<std::string, int32_t> &m) {
  if (!path) return;
  std::ofstream out(path, std::ios::trunc);
  for (const auto &kv : m) out << kv.first << '|' << kv.second << '\n';
}

int tune(peers_ctx *ctx, peers_symbolic *sym, peers_numeric *num, const char *cache_path,
         int32_t caps[4], double gain[4], std::string &err) {
  Symbolic &S = sym->S;
  DEVICE_SCOPE(ctx->device);
  cudaDeviceProp prop;
  CUDA_TRY(cudaGetDeviceProperties(&prop, ctx->device));
  auto cache = read_cache(cache_path);
  for (int c = 0; c < peers::kSizeClasses; ++c) {
    caps[c] = S.qcap[c];
    gain[c] = 1.0;
  }
  if (S.waves.empty() || S.nsorted == 0) return PEERS_OK;
  int rc = ensure_carry(num, S, err);
  if (rc != PEERS_OK) return rc;
  double *d_R = nullptr;
  SweepItem *d_items = nullptr;
  CUDA_TRY(cudaMalloc(&d_R, sizeof(double) * std::max<int64_t>(1, S.nq)));
  // work per supernode in the first wave (queries through it x FMAs per query)
  std::vector<std::vector<std::pair<int64_t, int32_t>>> by_class(peers::kSizeClasses);
  for (int32_t p = 0; p < S.nsuper; ++p) {
    const int64_t q = std::min(S.qbeg[p + 1], S.waves[0].q_end) -
                      std::max(S.qbeg[S.fdesc[p]], S.waves[0].q_begin);
    if (q <= 0 || S.spill[p]) continue;   // fronts in global memory keep the full tile
    const int64_t N = peers::sn_nc(S, p) + S.nb[p];
    by_class[peers::size_class(N)].push_back({q * items_fma(S, p, 0), p});
  }
  peers::SweepArgs a = sweep_args_of(num, S);
  a.carry = num->carry;
  a.racc = num->racc;
  a.R = d_R;
  a.wave_base = S.waves[0].q_begin;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int32_t candidates[] = {1, 2, 4, 8, 16, 32};
  int64_t cap_items = 0;
  rc = PEERS_OK;
  for (int c = 0; c < peers::kSizeClasses && rc == PEERS_OK; ++c) {
    const std::string key = std::string(prop.name) + "|class" + std::to_string(c);
    auto hit = cache.find(key);
    if (hit != cache.end()) {
      caps[c] = hit->second;
      continue;
    }
    auto &v = by_class[c];
    if (v.empty()) continue;
    std::sort(v.begin(), v.end(), std::greater<>());
    // heaviest supernodes of the class, about 3e10 FMAs (about 50 ms) per timing run: a
    // supernode with more work than its share contributes only its first queries per source
    std::vector<int32_t> sns;
    std::vector<int64_t> limit;
    const int64_t budget = int64_t(30e9);
    int64_t acc = 0;
    for (auto &x : v) {
      const int32_t p = x.second;
      const int64_t per_q = std::max<int64_t>(1, items_fma(S, p, 0));
      const int64_t nsrc = S.child_ptr[p + 1] - S.child_ptr[p] + 1;
      const int64_t take_q = std::max<int64_t>(64 * nsrc, (budget - acc) / per_q);
      sns.push_back(p);
      limit.push_back(std::max<int64_t>(64, take_q / nsrc));
      acc += std::min(x.first, take_q * per_q);
      if (acc >= budget || sns.size() >= 4096) break;
    }
    double best_t = 1e30, default_t = 0;
    int32_t best = caps[c];
    std::vector<int64_t> seen;
    const int64_t default_sig =
        static_cast<int64_t>(tile_items(S, sns, limit, peers::kQMax).size());
    for (int32_t cand : candidates) {
      std::vector<SweepItem> items = tile_items(S, sns, limit, cand);
      // skip caps that tile exactly like an earlier one
      int64_t sig = static_cast<int64_t>(items.size());
      if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
      seen.push_back(sig);
      int64_t smem = 0;
      for (auto &it : items)
        smem = std::max(smem, peers::sweep_smem_bytes(peers::sn_nc(S, it.s) + S.nb[it.s], it.nq));
      if (static_cast<int64_t>(items.size()) > cap_items) {
        if (d_items) cudaFree(d_items);
        cap_items = static_cast<int64_t>(items.size());
        if (cudaMalloc(&d_items, sizeof(SweepItem) * cap_items) != cudaSuccess) {
          cudaGetLastError();
          rc = PEERS_ENOMEM;
          err = "autotune work list";
          break;
        }
      }
      cudaMemcpyAsync(d_items, items.data(), sizeof(SweepItem) * items.size(),
                      cudaMemcpyHostToDevice, ctx->stream);
      double t = 1e30;
      for (int rep = 0; rep < 4 && rc == PEERS_OK; ++rep) {
        cudaEventRecord(e0, ctx->stream);
        rc = peers::run_items(d_items, static_cast<int64_t>(items.size()), a, smem, ctx->stream,
                              err);
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) t = std::min(t, double(ms));
      }
      if (sig == default_sig) default_t = t;   // the tiling of the largest tiles
      if (t < best_t) {
        best_t = t;
        best = cand;
      }
    }
    caps[c] = best;
    gain[c] = default_t > 0 ? default_t / best_t : 1.0;
    cache[key] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (d_items) cudaFree(d_items);
  cudaFree(d_R);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (rc != PEERS_OK) return rc;
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return PEERS_ECUDA;
  }
  write_cache(cache_path, cache);
  rc = peers::build_sweep_plan(S, caps, err);
  if (rc != PEERS_OK) return rc;
  return refresh_tiles(ctx, S, num, err);
}

}  // namespace

extern "C" {

int peers_retile(peers_ctx *ctx, peers_symbolic *sym, peers_numeric *num, const int32_t qcap[4]) {
  if (!ctx || !sym || !num || !qcap) return peers_fail(PEERS_EINVAL, "null argument");
  if (num->sym != sym) return peers_fail(PEERS_EINVAL, "numeric handle belongs to another plan");
  std::string err;
  forget_route_plans(sym);
  int rc = peers::build_sweep_plan(sym->S, qcap, err);
  if (rc == PEERS_OK) rc = refresh_tiles(ctx, sym->S, num, err);
  return rc == PEERS_OK ? rc : peers_fail(rc, err);
}

int peers_autotune(peers_ctx *ctx, peers_symbolic *sym, peers_numeric *num,
                   const char *cache_path, int32_t qcap_out[4], double gain_out[4]) {
  if (!ctx || !sym || !num) return peers_fail(PEERS_EINVAL, "null argument");
  if (num->sym != sym) return peers_fail(PEERS_EINVAL, "numeric handle belongs to another plan");
  int32_t caps[4];
  double gain[4];
  std::string err;
  forget_route_plans(sym);
  int rc = tune(ctx, sym, num, cache_path, caps, gain, err);
  if (rc != PEERS_OK) return peers_fail(rc, err);
  for (int c = 0; c < 4; ++c) {
    if (qcap_out) qcap_out[c] = caps[c];
    if (gain_out) gain_out[c] = gain[c];
  }
  return PEERS_OK;
}

}  // extern "C"
