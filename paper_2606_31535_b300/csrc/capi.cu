// C ABI of the PEERS library (declared in include/peers.h): handles, status codes, device
// memory of the factor and of the sweep, and the calls that drive the kernels.
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

namespace {

thread_local std::string g_error;

int fail(int status, const std::string &msg) {
  g_error = msg;
  return status;
}

}  // namespace

int peers_fail(int status, const std::string &msg) { return fail(status, msg); }

int peers::check_device_result(int device, const void *p, std::string &err) {
  if (!p) return PEERS_OK;
  cudaPointerAttributes at{};
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    err = std::string("result pointer: ") + cudaGetErrorString(e);
    return PEERS_EINVAL;
  }
  if (at.type == cudaMemoryTypeManaged) return PEERS_OK;
  if (at.type != cudaMemoryTypeDevice || at.device != device) {
    err = "the result pointer is not device memory of the context's device (flag "
          "PEERS_OUT_DEVICE)";
    return PEERS_EINVAL;
  }
  return PEERS_OK;
}

namespace {

template <class T>
int dalloc(peers_numeric *num, T **p, int64_t count, std::string &err) {
  *p = nullptr;
  if (count <= 0) return PEERS_OK;
  void *q = nullptr;
  const size_t bytes = sizeof(T) * static_cast<size_t>(count);
  cudaError_t e = num->pool ? cudaMallocFromPoolAsync(&q, bytes, num->pool, num->pool_stream)
                            : cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    err = "cudaMalloc of " + std::to_string(sizeof(T) * count) + " bytes: " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PEERS_ENOMEM : PEERS_ECUDA;
  }
  num->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return PEERS_OK;
}

template <class T, class Alloc>
int upload(peers_numeric *num, T **p, const std::vector<T, Alloc> &v, cudaStream_t st,
           std::string &err) {
  int rc = dalloc(num, p, static_cast<int64_t>(v.size()), err);
  if (rc != PEERS_OK || v.empty()) return rc;
  CUDA_TRY(cudaMemcpyAsync(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  num->h2d_bytes += static_cast<int64_t>(sizeof(T) * v.size());
  return PEERS_OK;
}

void dfree(peers_numeric *num, void *p) {
  auto it = std::find(num->allocs.begin(), num->allocs.end(), p);
  if (it != num->allocs.end()) {
    if (num->pool)
      cudaFreeAsync(p, num->pool_stream);
    else
      cudaFree(p);
    num->allocs.erase(it);
  }
}

#define TRY(x)                      \
  do {                              \
    int rc_ = (x);                  \
    if (rc_ != PEERS_OK) return rc_; \
  } while (0)

// The tile-dependent part of the sweep plan: work items of every wave and the two-branch
// walk's steps (replaced after a re-tiling).
int upload_tiles(peers_numeric *num, const Symbolic &S, cudaStream_t st, std::string &err) {
  for (void *p : {static_cast<void *>(num->items), static_cast<void *>(num->ldesc),
                  static_cast<void *>(num->two_user), static_cast<void *>(num->two_a),
                  static_cast<void *>(num->two_b)})
    if (p) dfree(num, p);
  num->items = nullptr;
  num->ldesc = nullptr;
  num->two_user = nullptr;
  num->two_a = num->two_b = nullptr;
  std::vector<SweepItem> all;
  num->wave_item_off.clear();
  for (const auto &W : S.waves) {
    num->wave_item_off.push_back(static_cast<int64_t>(all.size()));
    all.insert(all.end(), W.items.begin(), W.items.end());
  }
  TRY(upload(num, &num->items, all, st, err));
  TRY(upload(num, &num->ldesc, S.ldesc, st, err));
  TRY(upload(num, &num->two_user, S.two_user, st, err));
  TRY(upload(num, &num->two_a, S.two_a, st, err));
  TRY(upload(num, &num->two_b, S.two_b, st, err));
  // the carry buffer and the front scratch are sized by the plan's waves and tiles: drop
  // them, the next query re-allocates
  if (num->carry) dfree(num, num->carry);
  if (num->racc) dfree(num, num->racc);
  if (num->spill) dfree(num, num->spill);
  if (num->spill_counter) dfree(num, num->spill_counter);
  num->carry = num->racc = num->spill = nullptr;
  num->spill_counter = nullptr;
  return PEERS_OK;
}

int factor_impl(peers_ctx *ctx, const peers_symbolic *sym, const double *w, peers_numeric *num,
                std::string &err) {
  const Symbolic &S = sym->S;
  cudaStream_t st = ctx->stream;
  DEVICE_SCOPE(ctx->device);
  num->device = ctx->device;
  num->sym = sym;
  // structure shared by the factorization and the sweep
  TRY(upload(num, &num->first, S.first, st, err));
  TRY(upload(num, &num->nb, S.nb, st, err));
  TRY(upload(num, &num->rmap, S.rmap, st, err));
  TRY(upload(num, &num->panel_off, S.panel_off, st, err));
  TRY(upload(num, &num->tinv_off, S.tinv_off, st, err));
  TRY(upload(num, &num->rows_off, S.rows_off, st, err));
  TRY(dalloc(num, &num->panel, S.panel_total, err));
  TRY(dalloc(num, &num->tinv, S.tinv_total, err));
  TRY(dalloc(num, &num->d, S.nr, err));
  TRY(dalloc(num, &num->dinv, S.nr, err));
  TRY(dalloc(num, &num->status, 2, err));
  CUDA_TRY(cudaMemsetAsync(num->status, 0, 2 * sizeof(int), st));
  // factorization-only data (freed below)
  std::vector<double> vals;
  peers::assembly_values(S, w ? w : S.w0.data(), vals);
  peers::FactorDevice D{};
  int64_t *u_off = nullptr, *a_dest = nullptr, *trail_prefix = nullptr;
  int32_t *fac_sn = nullptr, *fuse_sn = nullptr, *child_ptr = nullptr, *child_list = nullptr;
  int32_t *ea_pairs = nullptr;
  double *a_val = nullptr, *U = nullptr;
  int *status = nullptr;
  TRY(upload(num, &u_off, S.u_off, st, err));
  TRY(upload(num, &a_dest, S.a_dest, st, err));
  TRY(upload(num, &a_val, vals, st, err));
  TRY(upload(num, &trail_prefix, S.trail_prefix, st, err));
  TRY(upload(num, &fac_sn, S.fac_sn, st, err));
  TRY(upload(num, &fuse_sn, S.fuse_sn, st, err));
  TRY(upload(num, &child_ptr, S.child_ptr, st, err));
  TRY(upload(num, &child_list, S.child_list, st, err));
  TRY(upload(num, &ea_pairs, S.ea_pairs, st, err));
  TRY(dalloc(num, &U, std::max<int64_t>(S.u_total, 1), err));
  TRY(dalloc(num, &status, 2, err));
  D.args = peers::FactorArgs{num->panel, U, num->tinv, num->d, num->dinv, num->first, num->nb,
                             num->rmap, num->panel_off, num->tinv_off, u_off, num->rows_off,
                             status, S.panel_total};
  D.a_dest = a_dest;
  D.a_val = a_val;
  D.fac_sn = fac_sn;
  D.fuse_sn = fuse_sn;
  D.child_ptr = child_ptr;
  D.child_list = child_list;
  D.ea_pairs = ea_pairs;
  D.trail_prefix = trail_prefix;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ctx->timing) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  int64_t launches = 0;
  int rc = peers::run_factor(S, D, st, ctx_lanes(ctx), &launches, err);
  ctx->stats.factor_launches = launches;
  if (ctx->timing) {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ctx->stats.factor_s = ms * 1e-3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  for (void *p : {static_cast<void *>(u_off), static_cast<void *>(a_dest),
                  static_cast<void *>(a_val), static_cast<void *>(trail_prefix),
                  static_cast<void *>(fac_sn), static_cast<void *>(fuse_sn),
                  static_cast<void *>(child_ptr), static_cast<void *>(child_list),
                  static_cast<void *>(ea_pairs),
                  static_cast<void *>(U), static_cast<void *>(status)})
    dfree(num, p);
  if (rc != PEERS_OK) return rc;
  // sweep plan
  TRY(upload(num, &num->qa, S.qa, st, err));
  TRY(upload(num, &num->qb, S.qb, st, err));
  TRY(upload(num, &num->qorig, S.qorig, st, err));
  TRY(upload_tiles(num, S, st, err));
  CUDA_TRY(cudaStreamSynchronize(st));
  ctx->stats.h2d_bytes = num->h2d_bytes;
  ctx->stats.d2h_bytes = 2 * sizeof(int);
  return PEERS_OK;
}

}  // namespace

int factor_from_pool(peers_ctx *ctx, const peers_symbolic *sym, const double *w,
                     cudaMemPool_t pool, peers_numeric **out, std::string &err) {
  *out = nullptr;
  auto *num = new (std::nothrow) peers_numeric;
  if (!num) {
    err = "host allocation";
    return PEERS_ENOMEM;
  }
  num->pool = pool;
  num->pool_stream = ctx->stream;
  const int rc = factor_impl(ctx, sym, w, num, err);
  if (rc != PEERS_OK) {
    peers_free_numeric(num);
    return rc;
  }
  *out = num;
  return PEERS_OK;
}

int check_bounds_flag(int *d_status, cudaStream_t stream, const char *what, std::string &err) {
#if defined(PEERS_BOUNDS) && PEERS_BOUNDS
  if (!d_status) return PEERS_OK;
  int h[2] = {0, 0};
  CUDA_TRY(cudaMemcpyAsync(h, d_status, sizeof(h), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(h), stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  if (h[0] == peers::kErrBounds) {
    err = std::string(what) + ": out-of-bounds access skipped at source line " + std::to_string(h[1]);
    return PEERS_ECUDA;
  }
#else
  (void)d_status;
  (void)stream;
  (void)what;
  (void)err;
#endif
  return PEERS_OK;
}

const peers::Lanes *ctx_lanes(peers_ctx *ctx) {
  if (ctx->lanes_ready) return &ctx->lanes;
  peers::Lanes L{};
  int least = 0, greatest = 0;
  bool ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
            cudaStreamCreateWithPriority(&L.top, cudaStreamNonBlocking, greatest) == cudaSuccess &&
            cudaStreamCreateWithPriority(&L.top1, cudaStreamNonBlocking, greatest) == cudaSuccess &&
            cudaEventCreateWithFlags(&L.start, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&L.top_done, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < peers::kLanes && ok; ++i)
    ok = cudaStreamCreateWithFlags(&L.stream[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&L.done[i], cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i <= peers::kLanes && ok; ++i) {
    ok = cudaStreamCreateWithPriority(&L.chain[i], cudaStreamNonBlocking, greatest) == cudaSuccess &&
         cudaStreamCreateWithFlags(&L.upd[i], cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t *e : {&L.ev_start[i], &L.ev_panel[i], &L.ev_rest[i], &L.ev_chain[i],
                           &L.ev_upd[i]})
      ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    return nullptr;
  }
  ctx->lanes = L;
  ctx->lanes_ready = true;
  return &ctx->lanes;
}

int ensure_carry(peers_numeric *num, const Symbolic &S, std::string &err) {
  if (!num->carry && S.carry_slots > 0) {
    TRY(dalloc(num, &num->carry, std::max<int64_t>(1, S.carry_slots * S.nbmax), err));
    TRY(dalloc(num, &num->racc, S.carry_slots, err));
  }
  if (!num->spill && S.spill_stride > 0) {
    TRY(dalloc(num, &num->spill, int64_t(peers::kSpillGrid) * S.spill_stride, err));
    TRY(dalloc(num, &num->spill_counter, std::max<int64_t>(1, S.nlevels), err));
  }
  return PEERS_OK;
}

int refresh_tiles(peers_ctx *ctx, const Symbolic &S, peers_numeric *num, std::string &err) {
  DEVICE_SCOPE(ctx->device);
  TRY(upload_tiles(num, S, ctx->stream, err));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return PEERS_OK;
}

namespace {

int query_impl(peers_ctx *ctx, const peers_symbolic *sym, peers_numeric *num, double *R,
               int flags, std::string &err) {
  const Symbolic &S = sym->S;
  cudaStream_t st = ctx->stream;
  DEVICE_SCOPE(ctx->device);
  const bool host_out = !(flags & PEERS_OUT_DEVICE);
  if (!host_out && S.nq > 0) TRY(peers::check_device_result(ctx->device, R, err));
  TRY(ensure_carry(num, S, err));
  double *Rout = R;
  if (host_out) {
    if (!num->Rdev && S.nq > 0) TRY(dalloc(num, &num->Rdev, S.nq, err));
    Rout = num->Rdev;
  }
  if (S.nq > 0) CUDA_TRY(cudaMemsetAsync(Rout, 0, sizeof(double) * S.nq, st));
  peers::SweepArgs a{};
  a.panel = num->panel;
  a.tinv = num->tinv;
  a.dinv = num->dinv;
  a.first = num->first;
  a.nb = num->nb;
  a.rmap = num->rmap;
  a.panel_off = num->panel_off;
  a.tinv_off = num->tinv_off;
  a.rows_off = num->rows_off;
  a.qa = num->qa;
  a.qb = num->qb;
  a.qorig = num->qorig;
  a.ldesc = num->ldesc;
  a.carry = num->carry;
  a.racc = num->racc;
  a.R = Rout;
  a.nbmax = S.nbmax;
  a.spill = num->spill;
  a.spill_stride = S.spill_stride;
  a.spill_counter = num->spill_counter;
  a.status = num->status;
  a.carry_slots = S.carry_slots;
  a.nq = S.nq;
  a.nldesc = static_cast<int64_t>(S.ldesc.size());
  std::vector<cudaEvent_t> ev;
  if (ctx->timing) {
    ev.resize(2 * static_cast<size_t>(S.nlevels));
    for (auto &e : ev) cudaEventCreate(&e);
    ctx->level_ms.assign(static_cast<size_t>(S.nlevels), 0.0);
    ctx->stats.sweep_s = ctx->stats.max_launch_s = 0;
  }
  int64_t launches = 0;
  for (size_t w = 0; w < S.waves.size() && S.nsorted + S.nq_two > 0; ++w) {
    const peers::SweepWave &W = S.waves[w];
    TRY(peers::run_sweep_wave(S, W, num->items + num->wave_item_off[w], a, st,
                              ctx->timing ? ev.data() : nullptr, &launches, err));
    if (W.two_end > W.two_begin) {
      peers::SweepArgs c = a;
      c.wave_base = W.q_begin;
      TRY(peers::run_two_branch_combine(c, num->two_user, num->two_a, num->two_b, W.two_begin,
                                        W.two_end, st, &launches, err));
    }
    if (ctx->timing) {
      CUDA_TRY(cudaStreamSynchronize(st));
      for (int32_t l = 0; l < S.nlevels; ++l) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ev[2 * l], ev[2 * l + 1]);
        ctx->level_ms[l] += ms;
        ctx->stats.sweep_s += ms * 1e-3;
        ctx->stats.max_launch_s = std::max(ctx->stats.max_launch_s, ms * 1e-3);
      }
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  ctx->stats.sweep_launches = launches;
  ctx->stats.d2h_bytes = 0;
  ctx->stats.h2d_bytes = 0;
  if (host_out && S.nq > 0) {
    CUDA_TRY(cudaMemcpyAsync(R, Rout, sizeof(double) * S.nq, cudaMemcpyDeviceToHost, st));
    ctx->stats.d2h_bytes = static_cast<int64_t>(sizeof(double)) * S.nq;
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  CUDA_TRY(cudaGetLastError());
  return check_bounds_flag(num->status, st, "peers_query", err);
}

}  // namespace

extern "C" {

const char *peers_strerror(int status) {
  switch (status) {
    case PEERS_OK: return "ok";
    case PEERS_EINVAL: return "invalid argument";
    case PEERS_ENOTCONNECTED: return "graph is not connected";
    case PEERS_ENOTSPD: return "matrix is not positive definite";
    case PEERS_ENOMEM: return "out of memory";
    case PEERS_ECUDA: return "CUDA error";
    case PEERS_ETIMEOUT: return "device wait timed out";
    case PEERS_ENOTREADY: return "not ready";
    default: return "unknown status";
  }
}

const char *peers_last_error(void) { return g_error.c_str(); }

const char *peers_version(void) { return "peers-b300 0.1 (sm_103a, FP64)"; }

int peers_create(peers_ctx **out, int device, void *cuda_stream) {
  if (!out) return fail(PEERS_EINVAL, "null output pointer");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PEERS_ECUDA, std::string("cudaGetDeviceCount: ") + cudaGetErrorString(e));
  }
  if (device < 0 || device >= count) return fail(PEERS_EINVAL, "no such CUDA device");
  auto *ctx = new (std::nothrow) peers_ctx;
  if (!ctx) return fail(PEERS_ENOMEM, "host allocation");
  ctx->device = device;
  peers::DeviceGuard guard(device);
  e = guard.status();
  if (e == cudaSuccess) {
    if (cuda_stream) {
      ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = e == cudaSuccess;
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return fail(PEERS_ECUDA, std::string("stream setup: ") + cudaGetErrorString(e));
  }
  *out = ctx;
  return PEERS_OK;
}

void peers_destroy(peers_ctx *ctx) {
  if (!ctx) return;
  {
    peers::DeviceGuard guard(ctx->device);
    if (ctx->lanes_ready) {
      for (int i = 0; i < peers::kLanes; ++i) {
        cudaStreamDestroy(ctx->lanes.stream[i]);
        cudaEventDestroy(ctx->lanes.done[i]);
      }
      cudaEventDestroy(ctx->lanes.start);
      cudaEventDestroy(ctx->lanes.top_done);
      for (int i = 0; i <= peers::kLanes; ++i) {
        cudaStreamDestroy(ctx->lanes.chain[i]);
        cudaStreamDestroy(ctx->lanes.upd[i]);
        for (cudaEvent_t e : {ctx->lanes.ev_start[i], ctx->lanes.ev_panel[i],
                              ctx->lanes.ev_rest[i], ctx->lanes.ev_chain[i], ctx->lanes.ev_upd[i]})
          cudaEventDestroy(e);
      }
      cudaStreamDestroy(ctx->lanes.top);
      cudaStreamDestroy(ctx->lanes.top1);
    }
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  }
  delete ctx;
}

int peers_analyze(peers_ctx *ctx, int64_t n, const int64_t *indptr, const int32_t *indices,
                  const double *w, int32_t ground, int64_t nq, const int32_t *qu,
                  const int32_t *qv, const double *coords, int dim, const peers_options *opt,
                  peers_symbolic **out) {
  (void)ctx;
  if (!out) return fail(PEERS_EINVAL, "null output pointer");
  *out = nullptr;
  peers_options o{};
  if (opt) o = *opt;
  auto *sym = new (std::nothrow) peers_symbolic;
  if (!sym) return fail(PEERS_ENOMEM, "host allocation");
  std::string err;
  int rc;
  try {
    rc = peers::analyze(sym->S, n, indptr, indices, w, ground, nq, qu, qv, coords, dim, o, err);
  } catch (const std::bad_alloc &) {
    rc = PEERS_ENOMEM;
    err = "host allocation during analysis";
  }
  if (rc != PEERS_OK) {
    delete sym;
    return fail(rc, err);
  }
  *out = sym;
  return PEERS_OK;
}

int peers_symbolic_info(const peers_symbolic *sym, peers_info *info) {
  if (!sym || !info) return fail(PEERS_EINVAL, "null argument");
  const Symbolic &S = sym->S;
  std::memset(info, 0, sizeof(*info));
  info->n = S.n;
  info->n_reduced = S.nr;
  info->nnz_a = S.nnz_lower;
  info->nnz_l = S.panel_total;
  info->nsuper = S.nsuper;
  info->levels = S.nlevels;
  for (int32_t s = 0; s < S.nsuper; ++s) {
    info->max_nc = std::max<int64_t>(info->max_nc, peers::sn_nc(S, s));
    info->max_nb = std::max<int64_t>(info->max_nb, S.nb[s]);
  }
  info->nq = S.nq;
  info->nq_trivial = S.nq_trivial;
  info->nq_two_branch = S.nq_two;
  info->walk_entries = S.walk_entries;
  info->walk_fma = S.walk_fma;
  info->factor_fma = S.factor_fma;
  info->device_bytes = peers_footprint_bytes(sym);
  info->t_order = S.t_order;
  info->t_symbolic = S.t_symbolic;
  info->t_queries = S.t_queries;
  for (char x : S.spill) info->nsuper_spilled += x ? 1 : 0;
  info->front_bytes = S.front_bytes;
  info->lanes = S.nlanes;
  info->split_blocks = 0;
  if (!S.one_stream)
    for (int64_t off : S.split_off) info->split_blocks += off >= 0 ? 1 : 0;
  return PEERS_OK;
}

int64_t peers_num_queries(const peers_symbolic *sym) { return sym ? sym->S.nq : -1; }

int64_t peers_footprint_bytes(const peers_symbolic *sym) {
  if (!sym) return -1;
  const Symbolic &S = sym->S;
  int64_t items = 0;
  for (const auto &W : S.waves) items += static_cast<int64_t>(W.items.size());
  // resident factor + sweep scratch + results, plus the factorization's transient update
  // matrices and assembly arrays (freed when peers_factor returns)
  return 8 * (S.panel_total + S.tinv_total + 2 * S.nr + S.carry_slots * (S.nbmax + 1) + S.nq) +
         8 * int64_t(peers::kSpillGrid) * S.spill_stride + 4 * int64_t(S.nlevels) +
         8 * (S.u_total + 2 * static_cast<int64_t>(S.a_dest.size())) +
         4 * (3 * int64_t(S.nsuper) + static_cast<int64_t>(S.rmap.size()) + 2 * S.nsorted) +
         8 * (3 * int64_t(S.nsuper) + S.nsorted) + static_cast<int64_t>(sizeof(SweepItem)) * items;
}

int peers_symbolic_export(const peers_symbolic *sym, int32_t *perm, int32_t *sn_first,
                          int32_t *sn_parent, int32_t *sn_nb, int32_t *sn_level) {
  if (!sym) return fail(PEERS_EINVAL, "null argument");
  const Symbolic &S = sym->S;
  if (perm) std::copy(S.perm.begin(), S.perm.end(), perm);
  if (sn_first) std::copy(S.first.begin(), S.first.end(), sn_first);
  if (sn_parent) std::copy(S.parent.begin(), S.parent.end(), sn_parent);
  if (sn_nb) std::copy(S.nb.begin(), S.nb.end(), sn_nb);
  if (sn_level) std::copy(S.level.begin(), S.level.end(), sn_level);
  return PEERS_OK;
}

void peers_free_symbolic(peers_symbolic *sym) { delete sym; }

int peers_factor(peers_ctx *ctx, const peers_symbolic *sym, const double *w, peers_numeric **out) {
  if (!out) return fail(PEERS_EINVAL, "null output pointer");
  *out = nullptr;
  if (!ctx || !sym) return fail(PEERS_EINVAL, "null context or plan");
  if (w) {
    for (int64_t p = 0; p < sym->S.nnz_csr; ++p)
      if (!(w[p] > 0.0) || w[p] == INFINITY)
        return fail(PEERS_EINVAL, "conductance must be positive and finite");
  }
  auto *num = new (std::nothrow) peers_numeric;
  if (!num) return fail(PEERS_ENOMEM, "host allocation");
  std::string err;
  int rc = factor_impl(ctx, sym, w, num, err);
  if (rc != PEERS_OK) {
    peers_free_numeric(num);
    return fail(rc, err);
  }
  *out = num;
  return PEERS_OK;
}

int peers_numeric_diag(peers_ctx *ctx, const peers_numeric *num, double *d_host) {
  if (!ctx || !num || !d_host) return fail(PEERS_EINVAL, "null argument");
  std::string err;
  auto run = [&]() -> int {
    DEVICE_SCOPE(num->device);
    CUDA_TRY(cudaMemcpyAsync(d_host, num->d, sizeof(double) * num->sym->S.nr,
                             cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return PEERS_OK;
  };
  int rc = run();
  return rc == PEERS_OK ? rc : fail(rc, err);
}

void peers_free_numeric(peers_numeric *num) {
  if (!num) return;
  if (!num->allocs.empty()) {
    peers::DeviceGuard guard(num->device);
    for (void *p : num->allocs) {
      if (num->pool)
        cudaFreeAsync(p, num->pool_stream);
      else
        cudaFree(p);
    }
  }
  delete num;
}

int peers_query(peers_ctx *ctx, const peers_symbolic *sym, const peers_numeric *num, double *R,
                int flags) {
  if (!ctx || !sym || !num || (!R && sym->S.nq > 0)) return fail(PEERS_EINVAL, "null argument");
  if (num->sym != sym) return fail(PEERS_EINVAL, "numeric handle belongs to another plan");
  if (num->device != ctx->device) return fail(PEERS_EINVAL, "context on another device");
  std::string err;
  int rc = query_impl(ctx, sym, const_cast<peers_numeric *>(num), R, flags, err);
  return rc == PEERS_OK ? rc : fail(rc, err);
}

int peers_query_noalloc(peers_ctx *ctx, const peers_symbolic *sym, const peers_numeric *num,
                        double *R_device) {
  if (!ctx || !sym || !num || (!R_device && sym->S.nq > 0))
    return fail(PEERS_EINVAL, "null argument");
  if (num->sym != sym) return fail(PEERS_EINVAL, "numeric handle belongs to another plan");
  if (num->device != ctx->device) return fail(PEERS_EINVAL, "context on another device");
  const Symbolic &S = sym->S;
  peers::SweepArgs a{};
  a.panel = num->panel;
  a.tinv = num->tinv;
  a.dinv = num->dinv;
  a.first = num->first;
  a.nb = num->nb;
  a.rmap = num->rmap;
  a.panel_off = num->panel_off;
  a.tinv_off = num->tinv_off;
  a.rows_off = num->rows_off;
  a.qa = num->qa;
  a.qb = num->qb;
  a.qorig = num->qorig;
  a.ldesc = num->ldesc;
  a.nbmax = S.nbmax;
  a.status = num->status;
  a.carry_slots = S.carry_slots;
  a.nq = S.nq;
  a.nldesc = static_cast<int64_t>(S.ldesc.size());
  std::string err;
  int64_t launches = 0;
  int rc = peers::query_noalloc(ctx->stream, ctx->device, S, a, num->items,
                                num->wave_item_off.data(), num->two_user, num->two_a,
                                num->two_b, R_device, &launches, err);
  if (rc == PEERS_OK) rc = check_bounds_flag(num->status, ctx->stream, "peers_query_noalloc", err);
  if (rc != PEERS_OK) return fail(rc, err);
  ctx->stats.sweep_launches = launches;
  ctx->stats.h2d_bytes = 0;
  ctx->stats.d2h_bytes = 0;
  return PEERS_OK;
}

int peers_set_timing(peers_ctx *ctx, int enable) {
  if (!ctx) return fail(PEERS_EINVAL, "null context");
  ctx->timing = enable != 0;
  return PEERS_OK;
}

int peers_last_stats(const peers_ctx *ctx, peers_stats *out) {
  if (!ctx || !out) return fail(PEERS_EINVAL, "null argument");
  *out = ctx->stats;
  return PEERS_OK;
}

int peers_fp64_peak(peers_ctx *ctx, double tflops[3]) {
  if (!ctx || !tflops) return fail(PEERS_EINVAL, "null argument");
  std::string err;
  auto run = [&]() -> int {
    DEVICE_SCOPE(ctx->device);
    return peers::fp64_peak(ctx->stream, tflops, err);
  };
  int rc = run();
  return rc == PEERS_OK ? rc : fail(rc, err);
}

int peers_fp64_mma_shapes(peers_ctx *ctx, double tflops[4]) {
  if (!ctx || !tflops) return fail(PEERS_EINVAL, "null argument");
  std::string err;
  auto run = [&]() -> int {
    DEVICE_SCOPE(ctx->device);
    return peers::fp64_mma_shapes(ctx->stream, tflops, err);
  };
  int rc = run();
  return rc == PEERS_OK ? rc : fail(rc, err);
}

int64_t peers_last_level_times(const peers_ctx *ctx, double *ms, int64_t cap) {
  if (!ctx) return fail(PEERS_EINVAL, "null context");
  if (cap > 0 && !ms) return fail(PEERS_EINVAL, "null output array with a positive capacity");
  const int64_t nl = static_cast<int64_t>(ctx->level_ms.size());
  for (int64_t i = 0; i < std::min(nl, cap); ++i) ms[i] = ctx->level_ms[i];
  return nl;
}

}  // extern "C"
