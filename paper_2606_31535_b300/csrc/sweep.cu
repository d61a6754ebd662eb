// The implicit-inverse query sweep (PEERS §III, Theorem 3): for each query (s, t),
//     R_st = sum_k y_k^2 / d_k,   L y = e_s - e_t          (eq. 16-18, L D L^T form),
// evaluated by walking the elimination-tree path on which y is non-zero (Lemma 1), one
// supernode at a time, never forming L^{-1}.
//
// For a graph edge the two endpoints' paths coincide above the lower endpoint, so each query
// starts in the supernode s0 holding its lower endpoint (the other endpoint is a row of that
// supernode's front) and walks to the root.  At supernode s with columns C (n_c) and
// below-diagonal rows B (n_b) the query's front x (n_c + n_b values) is processed as
//     y   = T^{-1} x[C]          T = unit-lower diagonal block of L on C
//     r  += sum_k y_k^2 / d_k
//     x[B] -= P y                 P = L[B, C]
// and x[B] moves into the parent's front through the relative row map.  Queries that pass
// through the same supernode form a tile of up to kQMax right-hand sides handled by one CTA,
// so every panel value fetched is used once per query of the tile.
//
// The triangular solve is blocked by kBlock columns: y_J = inv(T_JJ) x_J with the diagonal
// block's inverse precomputed by the factorization, then one rank-kBlock update of every row
// below the block.  Blocks start at fixed multiples of kBlock, so the arithmetic of a query
// (and its rounding) depends only on its own path, never on the other queries of its tile.
// The path is FP64 arithmetic bound (about 2 flops per 8-byte panel entry per query).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "device.cuh"
#include "internal.h"

namespace peers {

constexpr int kSweepThreads = 256;

// One work item (see SweepItem) by one CTA of kSweepThreads threads.  SPILL: the tile's
// fronts X live in this CTA's slice of the global scratch a.spill (fronts too large for
// shared memory); Y and T stay in shared memory.  The arithmetic is the same either way.
template <bool SPILL>
__device__ __forceinline__ void sweep_item(const SweepItem &it, const SweepArgs &a,
                                           double *smem) {
  if (it.kind == 2) {   // combine two-branch sums (multi-graph launches)
    for (int64_t k = it.q0 + threadIdx.x; k < int64_t(it.q0) + it.nq; k += kSweepThreads) {
      const int64_t sa = int64_t(a.two_a[k]) - a.wave_base, sb = int64_t(a.two_b[k]) - a.wave_base;
      if (!PEERS_IN(sa, a.carry_slots, a.status)) continue;
      double r = a.racc[sa];
      if (a.two_b[k] >= 0 && PEERS_IN(sb, a.carry_slots, a.status)) r += a.racc[sb];
      if (PEERS_IN(a.two_user[k], a.nq, a.status)) a.R[a.two_user[k]] = r;
    }
    return;
  }
  const int32_t s = it.s, Q = it.nq;
  const int32_t f = a.first[s], nc = a.first[s + 1] - f, nbv = a.nb[s], N = nc + nbv;
  const int QP = static_cast<int>(sweep_qstride(Q));
  const int nch = (Q + 3) / 4;
  double *X = SPILL ? a.spill + int64_t(blockIdx.x) * a.spill_stride
                    : smem;            // N x QP   the tile's fronts, row-major
  double *Y = SPILL ? smem : X + int64_t(N) * QP;   // kBlock x QP   y of the current block
  double *T = Y + kBlock * QP;         // kBlock x QP   y^2 / d of the current block
  const int tid = threadIdx.x;
  const int32_t j0 = it.j0;
  const int64_t NX = int64_t(N) * QP;   // doubles of the tile's fronts
#if defined(PEERS_BOUNDS) && PEERS_BOUNDS
  // the tile must fit its launch: fronts and y blocks in shared memory, or the fronts in this
  // CTA's slice of the global scratch
  if (!(SPILL ? PEERS_IN(NX - 1, a.spill_stride, a.status) &&
                    PEERS_IN(int64_t(blockIdx.x), kSpillGrid, a.status) &&
                    PEERS_IN(2 * kBlock * QP - 1, dynamic_smem_doubles(), a.status)
              : PEERS_IN(NX + 2 * kBlock * QP - 1, dynamic_smem_doubles(), a.status)) ||
      !PEERS_IN(int64_t(it.q0) - (it.kind == 1 ? 0 : a.wave_base) + Q - 1,
                it.kind == 1 ? a.nldesc : a.carry_slots, a.status))
    return;
  const int64_t cbase = a.panel_off[s], cext = a.panel_off[s + 1] - a.panel_off[s];
  const int64_t tbase = a.tinv_off[s], text = a.tinv_off[s + 1] - a.tinv_off[s];
#endif

  for (int64_t idx = int64_t(j0) * QP + tid; idx < NX; idx += kSweepThreads)
    X[idx] = 0.0;
  __syncthreads();
  if (it.kind == 1) {
    // two-branch walk steps: per entry its own source (child carry or seed) ...
    const int warp = tid / 32, lane = tid % 32;
    for (int q = warp; q < Q; q += kSweepThreads / 32) {
      const SweepDesc d = a.ldesc[it.q0 + q];
      const int64_t sa = int64_t(d.a) - a.wave_base;
      if (!PEERS_IN(sa, a.carry_slots, a.status)) continue;
      if (d.src_a >= 0) {
        const int32_t nbc = a.nb[d.src_a];
        const int32_t *rm = a.rmap + a.rows_off[d.src_a];
        for (int32_t t = lane; t < nbc; t += 32)
          if (PEERS_IN(t, a.nbmax, a.status) && PEERS_IN(int64_t(rm[t]) * QP + q, NX, a.status))
            X[rm[t] * QP + q] = a.carry[sa * a.nbmax + t];
      } else if (lane == 0) {
        if (a.qa[d.a] >= 0 && PEERS_IN(int64_t(a.qa[d.a]) * QP + q, NX, a.status))
          X[a.qa[d.a] * QP + q] = 1.0;
        if (a.qb[d.a] >= 0 && PEERS_IN(int64_t(a.qb[d.a]) * QP + q, NX, a.status))
          X[a.qb[d.a] * QP + q] = -1.0;
      }
    }
    __syncthreads();
    // ... plus, where the two branches merge, the other branch's carry or the -1 seed
    for (int q = warp; q < Q; q += kSweepThreads / 32) {
      const SweepDesc d = a.ldesc[it.q0 + q];
      if (d.b >= 0) {
        const int64_t sb = int64_t(d.b) - a.wave_base;
        const int32_t nbc = a.nb[d.src_b];
        const int32_t *rm = a.rmap + a.rows_off[d.src_b];
        if (!PEERS_IN(sb, a.carry_slots, a.status)) continue;
        for (int32_t t = lane; t < nbc; t += 32)
          if (PEERS_IN(t, a.nbmax, a.status) && PEERS_IN(int64_t(rm[t]) * QP + q, NX, a.status))
            X[rm[t] * QP + q] += a.carry[sb * a.nbmax + t];
      } else if (d.seed_b >= 0 && lane == 0) {
        if (PEERS_IN(int64_t(d.seed_b) * QP + q, NX, a.status)) X[d.seed_b * QP + q] -= 1.0;
      }
    }
  } else if (it.src >= 0) {
    // queries arriving from child src: scatter its carried B-part into this front
    const int32_t nbc = a.nb[it.src];
    const int32_t *rm = a.rmap + a.rows_off[it.src];
    const double *cin = a.carry + (int64_t(it.q0) - a.wave_base) * a.nbmax;
    for (int32_t idx = tid; idx < Q * nbc; idx += kSweepThreads) {
      const int32_t q = idx / nbc, t = idx - q * nbc;
      if (PEERS_IN(t, a.nbmax, a.status) && PEERS_IN(int64_t(rm[t]) * QP + q, NX, a.status))
        X[rm[t] * QP + q] = cin[int64_t(q) * a.nbmax + t];
    }
  } else {
    // queries starting here: e_lo - e_hi in local rows (eq. 4: no -1 when hi is the ground)
    for (int32_t q = tid; q < Q; q += kSweepThreads) {
      const int32_t qa = a.qa[it.q0 + q], qb = a.qb[it.q0 + q];
      if (qa >= 0 && PEERS_IN(int64_t(qa) * QP + q, NX, a.status)) X[qa * QP + q] = 1.0;
      if (qb >= 0 && PEERS_IN(int64_t(qb) * QP + q, NX, a.status)) X[qb * QP + q] = -1.0;
    }
  }

  double r = 0.0;   // owned by thread q < Q
  const double *panel = a.panel + a.panel_off[s];
  const double *tinv = a.tinv + a.tinv_off[s];
  for (int32_t J = j0; J < nc; J += kBlock) {
    const int32_t bw = min(kBlock, nc - J);
    __syncthreads();
    // y_J = inv(T_JJ) x_J and its y^2 / d terms
    const double *TI = tinv + int64_t(J / kBlock) * kBlock * kBlock;
#if defined(PEERS_BOUNDS) && PEERS_BOUNDS
    // this block's inverse and panel columns lie inside the supernode's stored extents
    if (!PEERS_IN(int64_t(J / kBlock) * kBlock * kBlock + bw * bw - 1, text, a.status) ||
        !PEERS_IN(int64_t(J + bw) * N - 1, cext, a.status))
      break;
#endif
    for (int u = tid; u < bw * Q; u += kSweepThreads) {
      const int k = u / Q, q = u - k * Q;
      double acc = X[(J + k) * QP + q];
      for (int j = 0; j < k; ++j) acc = fma(TI[k * bw + j], X[(J + j) * QP + q], acc);
      Y[k * QP + q] = acc;
      T[k * QP + q] = acc * acc * a.dinv[f + J + k];
    }
    __syncthreads();
    if (tid < Q)
      for (int k = 0; k < bw; ++k) r += T[k * QP + tid];
    // rows below the block: x_i -= sum_k L[i, J+k] y_k
    const double *PJ = panel + int64_t(J) * N;
    const int32_t rows = N - J - bw;
    const int32_t units = rows * nch;
    for (int32_t u = tid; u < units; u += kSweepThreads) {
      const int32_t i = J + bw + u / nch;
      const int c = u - (u / nch) * nch;
      // x_i -= l_k y_k, one fused multiply-add per term, in k order (the update of x_i
      // starts from x_i itself, so no separate subtraction is needed)
      double *xi = X + int64_t(i) * QP + c * 4;
      const double2 x01 = *reinterpret_cast<const double2 *>(xi);
      const double2 x23 = *reinterpret_cast<const double2 *>(xi + 2);
      double acc0 = x01.x, acc1 = x01.y, acc2 = x23.x, acc3 = x23.y;
      const double *yk = Y + c * 4;
      if (bw == kBlock) {
#pragma unroll 8
        for (int k = 0; k < kBlock; ++k) {
          const double l = -PJ[int64_t(k) * N + i];
          const double2 y01 = *reinterpret_cast<const double2 *>(yk + k * QP);
          const double2 y23 = *reinterpret_cast<const double2 *>(yk + k * QP + 2);
          acc0 = fma(l, y01.x, acc0);
          acc1 = fma(l, y01.y, acc1);
          acc2 = fma(l, y23.x, acc2);
          acc3 = fma(l, y23.y, acc3);
        }
      } else {
        for (int k = 0; k < bw; ++k) {
          const double l = -PJ[int64_t(k) * N + i];
          const double2 y01 = *reinterpret_cast<const double2 *>(yk + k * QP);
          const double2 y23 = *reinterpret_cast<const double2 *>(yk + k * QP + 2);
          acc0 = fma(l, y01.x, acc0);
          acc1 = fma(l, y01.y, acc1);
          acc2 = fma(l, y23.x, acc2);
          acc3 = fma(l, y23.y, acc3);
        }
      }
      const int qn = Q - c * 4;
      xi[0] = acc0;
      if (qn > 1) xi[1] = acc1;
      if (qn > 2) xi[2] = acc2;
      if (qn > 3) xi[3] = acc3;
    }
  }
  __syncthreads();
  if (it.kind == 1) {
    // two-branch steps keep their running sum in slot a; the combine kernel writes R
    const int warp = tid / 32, lane = tid % 32;
    for (int q = warp; q < Q; q += kSweepThreads / 32) {
      const int64_t sa = int64_t(a.ldesc[it.q0 + q].a) - a.wave_base;
      if (!PEERS_IN(sa, a.carry_slots, a.status)) continue;
      for (int32_t t = lane; t < nbv; t += 32)
        if (PEERS_IN(t, a.nbmax, a.status)) a.carry[sa * a.nbmax + t] = X[(nc + t) * QP + q];
    }
    if (tid < Q) {
      const SweepDesc d = a.ldesc[it.q0 + tid];
      double tot = r;
      if (d.src_a >= 0) tot += a.racc[int64_t(d.a) - a.wave_base];
      if (d.b >= 0 && PEERS_IN(int64_t(d.b) - a.wave_base, a.carry_slots, a.status))
        tot += a.racc[int64_t(d.b) - a.wave_base];
      if (PEERS_IN(int64_t(d.a) - a.wave_base, a.carry_slots, a.status))
        a.racc[int64_t(d.a) - a.wave_base] = tot;
    }
    return;
  }
  if (nbv > 0) {
    double *cout = a.carry + (int64_t(it.q0) - a.wave_base) * a.nbmax;
    for (int32_t idx = tid; idx < Q * nbv; idx += kSweepThreads) {
      const int32_t q = idx / nbv, t = idx - q * nbv;
      if (PEERS_IN(t, a.nbmax, a.status)) cout[int64_t(q) * a.nbmax + t] = X[(nc + t) * QP + q];
    }
  }
  if (tid < Q) {
    const int64_t slot = int64_t(it.q0) + tid;
    const double prev = it.src >= 0 ? a.racc[slot - a.wave_base] : 0.0;
    const double tot = prev + r;
    if (nbv > 0)
      a.racc[slot - a.wave_base] = tot;
    else if (PEERS_IN(a.qorig[slot], a.nq, a.status))
      a.R[a.qorig[slot]] = tot;
  }
}

__global__ void __launch_bounds__(kSweepThreads) k_sweep(const SweepItem *__restrict__ items,
                                                         SweepArgs a) {
  extern __shared__ double smem[];
  sweep_item<false>(items[blockIdx.x], a, smem);
}

// The items of a level whose fronts do not fit shared memory: a persistent grid of at most
// kSpillGrid CTAs pulling items (largest first) through *counter, each CTA working on its own
// front scratch.
__global__ void __launch_bounds__(kSweepThreads) k_sweep_spill(const SweepItem *__restrict__ items,
                                                               int64_t nitems, SweepArgs a,
                                                               int *counter) {
  extern __shared__ double smem[];
  __shared__ int next;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    __syncthreads();
    const int64_t i = next;
    __syncthreads();
    if (i >= nitems) break;
    sweep_item<true>(items[i], a, smem);
    __syncthreads();
  }
}

// Persistent multi-graph launch: as many CTAs as fit on the GPU, each pulling items (sorted
// largest first) until the level's list is exhausted.  Items of different graphs, and of
// different requests of a server, share one launch.
__global__ void __launch_bounds__(kSweepThreads) k_sweep_multi(const SweepItem *__restrict__ items,
                                                               int64_t nitems,
                                                               const SweepArgs *__restrict__ table,
                                                               int *counter) {
  extern __shared__ double smem[];
  __shared__ int next;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    __syncthreads();
    const int64_t i = next;
    __syncthreads();
    if (i >= nitems) break;
    const SweepItem it = items[i];
    sweep_item<false>(it, table[it.g], smem);
    __syncthreads();
  }
}

// Raises a kernel's dynamic shared-memory limit on the current device to at least `bytes`.
// The limit only ever grows, so launches configured earlier stay valid; the check and the
// raise happen under one lock, so a thread needing less can never lower the limit after a
// thread needing more has raised it (sweeps may run from several host threads).
std::mutex g_smem_lock;

int raise_smem_limit(const void *kernel, int *configured, int64_t bytes, std::string &err) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    err = "device index out of range";
    return PEERS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_smem_lock);
  if (bytes > configured[dev]) {
    CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(bytes)));
    configured[dev] = static_cast<int>(bytes);
  }
  return PEERS_OK;
}

template <class K>
int ensure_smem(K kernel, int *configured, int64_t bytes, std::string &err) {
  return raise_smem_limit(reinterpret_cast<const void *>(kernel), configured, bytes, err);
}
int g_sweep_smem[64] = {};
int g_multi_smem[64] = {};

int multi_step_grid(int64_t smem, int64_t nitems, int64_t *grid, std::string &err) {
  int rc = ensure_smem(k_sweep_multi, g_multi_smem, smem, err);
  if (rc != PEERS_OK) return rc;
  int dev = 0, sms = 0, per_sm = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_multi, kSweepThreads,
                                                         static_cast<size_t>(smem)));
  *grid = std::min<int64_t>(nitems, int64_t(std::max(per_sm, 1)) * sms);
  return PEERS_OK;
}

int run_multi_step(const SweepItem *items, int64_t nitems, const SweepArgs *table, int *counter,
                   int64_t smem, int64_t grid, cudaStream_t stream, std::string &err) {
  if (grid <= 0 || nitems <= 0) return PEERS_OK;
  k_sweep_multi<<<static_cast<unsigned>(grid), kSweepThreads, smem, stream>>>(items, nitems,
                                                                             table, counter);
  CUDA_TRY(cudaGetLastError());
  return PEERS_OK;
}


int run_sweep_wave(const Symbolic &S, const SweepWave &W, const SweepItem *d_items,
                   const SweepArgs &args, cudaStream_t stream, cudaEvent_t *events,
                   int64_t *launches, std::string &err) {
  int64_t need = 0;
  for (int64_t b : W.level_smem) need = std::max(need, b);
  int rc = ensure_smem(k_sweep, g_sweep_smem, need, err);
  if (rc != PEERS_OK) return rc;
  SweepArgs a = args;
  a.wave_base = W.q_begin;
  int64_t nspill_total = 0;
  for (int64_t x : W.level_nspill) nspill_total += x;
  if (nspill_total > 0) {
    if (!a.spill || !a.spill_counter) {
      err = "the plan keeps fronts in global memory but no front scratch was given";
      return PEERS_EINVAL;
    }
    CUDA_TRY(cudaMemsetAsync(a.spill_counter, 0, sizeof(int) * S.nlevels, stream));
  }
  for (int32_t l = 0; l < S.nlevels; ++l) {
    const int64_t i0 = W.level_ptr[l], i1 = W.level_ptr[l + 1];
    const int64_t ns = W.level_nspill.empty() ? 0 : W.level_nspill[l];
    if (events) CUDA_TRY(cudaEventRecord(events[2 * l], stream));
    if (ns > 0) {
      const unsigned grid = static_cast<unsigned>(std::min<int64_t>(ns, kSpillGrid));
      k_sweep_spill<<<grid, kSweepThreads, W.level_spill_smem[l], stream>>>(
          d_items + i0, ns, a, a.spill_counter + l);
      ++*launches;
      CUDA_TRY(cudaGetLastError());
    }
    if (i1 > i0 + ns) {
      k_sweep<<<static_cast<unsigned>(i1 - i0 - ns), kSweepThreads, W.level_smem[l], stream>>>(
          d_items + i0 + ns, a);
      ++*launches;
      CUDA_TRY(cudaGetLastError());
    }
    if (events) CUDA_TRY(cudaEventRecord(events[2 * l + 1], stream));
  }
  return PEERS_OK;
}

int run_items(const SweepItem *d_items, int64_t n, const SweepArgs &args, int64_t smem,
              cudaStream_t stream, std::string &err) {
  int rc = ensure_smem(k_sweep, g_sweep_smem, smem, err);
  if (rc != PEERS_OK) return rc;
  if (n <= 0) return PEERS_OK;
  k_sweep<<<static_cast<unsigned>(n), kSweepThreads, smem, stream>>>(d_items, args);
  CUDA_TRY(cudaGetLastError());
  return PEERS_OK;
}

__global__ void k_two_branch_combine(const int64_t *__restrict__ user, const int32_t *__restrict__ sa,
                                     const int32_t *__restrict__ sb, int64_t k0, int64_t k1,
                                     SweepArgs a) {
  const int64_t k = k0 + blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k >= k1) return;
  double r = a.racc[int64_t(sa[k]) - a.wave_base];
  if (sb[k] >= 0) r += a.racc[int64_t(sb[k]) - a.wave_base];
  a.R[user[k]] = r;
}

int run_two_branch_combine(const SweepArgs &args, const int64_t *two_user, const int32_t *two_a,
                           const int32_t *two_b, int64_t k0, int64_t k1, cudaStream_t stream,
                           int64_t *launches, std::string &err) {
  if (k1 <= k0) return PEERS_OK;
  const unsigned blocks = static_cast<unsigned>((k1 - k0 + 255) / 256);
  k_two_branch_combine<<<blocks, 256, 0, stream>>>(two_user, two_a, two_b, k0, k1, args);
  ++*launches;
  CUDA_TRY(cudaGetLastError());
  return PEERS_OK;
}

}  // namespace peers
