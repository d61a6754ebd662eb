// Definitions of the C-ABI handles (library-internal; shared by capi.cu and batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <mutex>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "peers.h"

using peers::SweepItem;
using peers::Symbolic;

struct peers_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // lane streams and events (created on first use, see ctx_lanes)
  peers::Lanes lanes{};
  bool lanes_ready = false;
  bool timing = false;
  peers_stats stats{};
  std::vector<double> level_ms;
};

struct peers_symbolic {
  Symbolic S;
  // Host plans of the block-inverse and selected-inversion routes, built by their first call
  // and reused by later ones (blockinv.cu).  They read the query slots, which a rebuild of the
  // sweep plan rewrites, so peers_retile and peers_autotune drop them (forget_route_plans).
  mutable std::mutex route_mu;
  mutable std::shared_ptr<const void> blockinv_plan, selinv_plan;
  mutable int selinv_sms = 0;
};

inline void forget_route_plans(peers_symbolic *sym) {
  std::lock_guard<std::mutex> lock(sym->route_mu);
  sym->blockinv_plan.reset();
  sym->selinv_plan.reset();
  sym->selinv_sms = 0;
}

struct peers_numeric {
  int device = 0;
  const peers_symbolic *sym = nullptr;   // not owned; must outlive this handle
  std::vector<void *> allocs;
  // Stream-ordered allocation (the server's requests): when `pool` is set, every buffer of the
  // handle comes from that memory pool on `pool_stream` and is returned to it on
  // `pool_stream`, so that neither allocating nor freeing synchronises the device.  The owner
  // may point pool_stream at another stream before freeing the handle.
  cudaMemPool_t pool = nullptr;
  cudaStream_t pool_stream = nullptr;
  int64_t h2d_bytes = 0;   // bytes uploaded while building this handle
  // factor
  double *panel = nullptr, *tinv = nullptr, *d = nullptr, *dinv = nullptr;
  int32_t *first = nullptr, *nb = nullptr, *rmap = nullptr;
  int64_t *panel_off = nullptr, *tinv_off = nullptr, *rows_off = nullptr;
  // sweep plan
  int32_t *qa = nullptr, *qb = nullptr;
  int64_t *qorig = nullptr;
  SweepItem *items = nullptr;
  peers::SweepDesc *ldesc = nullptr;
  int64_t *two_user = nullptr;
  int32_t *two_a = nullptr, *two_b = nullptr;
  std::vector<int64_t> wave_item_off;
  double *carry = nullptr, *racc = nullptr, *Rdev = nullptr;
  double *spill = nullptr;        // kSpillGrid x spill_stride front scratch (if the plan spills)
  int *spill_counter = nullptr;   // one work counter per level
  int *status = nullptr;          // error flag of the sweep kernels (2 ints; bounds checks)
  // device copy of the selected inversion's plan and its working buffers, made by the first
  // peers_query_selinv on this factor and reused while the plan is the same (blockinv.cu);
  // route_mu serialises the calls that use it
  std::mutex route_mu;
  std::shared_ptr<void> selinv_dev;
};


// Argument block of the sweep kernels for one factored plan (scratch and R left unset).
inline peers::SweepArgs sweep_args_of(const peers_numeric *num, const Symbolic &S) {
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
  a.two_user = num->two_user;
  a.two_a = num->two_a;
  a.two_b = num->two_b;
  a.nbmax = S.nbmax;
  a.spill = num->spill;
  a.spill_stride = S.spill_stride;
  a.spill_counter = num->spill_counter;
  a.status = num->status;
  a.carry_slots = S.carry_slots;
  a.nq = S.nq;
  a.nldesc = static_cast<int64_t>(S.ldesc.size());
  return a;
}

// The context's lane streams (created on the first call that needs them, on the context's
// device, which must be current); nullptr if they cannot be created, in which case callers
// run everything on the context's stream (capi.cu).
const peers::Lanes *ctx_lanes(peers_ctx *ctx);

// Records a failure message for peers_last_error and returns the status.
int peers_fail(int status, const std::string &msg);

// peers_factor with every device buffer of the new handle taken from `pool` on the context's
// stream (stream-ordered; see peers_numeric::pool).  Returns a PEERS_* status (capi.cu).
int factor_from_pool(peers_ctx *ctx, const peers_symbolic *sym, const double *w,
                     cudaMemPool_t pool, peers_numeric **out, std::string &err);

// Bounds-checked build only: reads and clears a kernel error flag (2 ints) after the work on
// `stream`, and turns a recorded out-of-bounds access into PEERS_ECUDA with its source line.
// The regular build returns PEERS_OK without touching the device (capi.cu).
int check_bounds_flag(int *d_status, cudaStream_t stream, const char *what, std::string &err);

// Allocates the sweep's carry buffer of a factored plan if it has none (capi.cu).
int ensure_carry(peers_numeric *num, const Symbolic &S, std::string &err);
// Re-uploads the tile-dependent sweep plan after build_sweep_plan (capi.cu).
int refresh_tiles(peers_ctx *ctx, const Symbolic &S, peers_numeric *num, std::string &err);
