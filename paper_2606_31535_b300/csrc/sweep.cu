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

#include "device.cuh"
#include "internal.h"

namespace peers {

constexpr int kSweepThreads = 256;

__global__ void __launch_bounds__(kSweepThreads) k_sweep(const SweepItem *__restrict__ items,
                                                         SweepArgs a) {
  extern __shared__ double smem[];
  const SweepItem it = items[blockIdx.x];
  const int32_t s = it.s, Q = it.nq;
  const int32_t f = a.first[s], nc = a.first[s + 1] - f, nbv = a.nb[s], N = nc + nbv;
  const int QP = static_cast<int>(sweep_qstride(Q));
  const int nch = (Q + 3) / 4;
  double *X = smem;                    // N x QP   the tile's fronts, row-major
  double *Y = X + int64_t(N) * QP;     // kBlock x QP   y of the current block
  double *T = Y + kBlock * QP;         // kBlock x QP   y^2 / d of the current block
  const int tid = threadIdx.x;
  const int32_t j0 = it.j0;

  for (int64_t idx = int64_t(j0) * QP + tid; idx < int64_t(N) * QP; idx += kSweepThreads)
    X[idx] = 0.0;
  __syncthreads();
  if (it.src >= 0) {
    // queries arriving from child src: scatter its carried B-part into this front
    const int32_t nbc = a.nb[it.src];
    const int32_t *rm = a.rmap + a.rows_off[it.src];
    const double *cin = a.carry + (int64_t(it.q0) - a.wave_base) * a.nbmax;
    for (int32_t idx = tid; idx < Q * nbc; idx += kSweepThreads) {
      const int32_t q = idx / nbc, t = idx - q * nbc;
      X[rm[t] * QP + q] = cin[int64_t(q) * a.nbmax + t];
    }
  } else {
    // queries starting here: e_lo - e_hi in local rows (eq. 4: no -1 when hi is the ground)
    for (int32_t q = tid; q < Q; q += kSweepThreads) {
      X[a.qa[it.q0 + q] * QP + q] = 1.0;
      const int32_t b = a.qb[it.q0 + q];
      if (b >= 0) X[b * QP + q] = -1.0;
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
      double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
      const double *yk = Y + c * 4;
      if (bw == kBlock) {
#pragma unroll 8
        for (int k = 0; k < kBlock; ++k) {
          const double l = PJ[int64_t(k) * N + i];
          const double2 y01 = *reinterpret_cast<const double2 *>(yk + k * QP);
          const double2 y23 = *reinterpret_cast<const double2 *>(yk + k * QP + 2);
          acc0 = fma(l, y01.x, acc0);
          acc1 = fma(l, y01.y, acc1);
          acc2 = fma(l, y23.x, acc2);
          acc3 = fma(l, y23.y, acc3);
        }
      } else {
        for (int k = 0; k < bw; ++k) {
          const double l = PJ[int64_t(k) * N + i];
          const double2 y01 = *reinterpret_cast<const double2 *>(yk + k * QP);
          const double2 y23 = *reinterpret_cast<const double2 *>(yk + k * QP + 2);
          acc0 = fma(l, y01.x, acc0);
          acc1 = fma(l, y01.y, acc1);
          acc2 = fma(l, y23.x, acc2);
          acc3 = fma(l, y23.y, acc3);
        }
      }
      double *xi = X + int64_t(i) * QP + c * 4;
      const int qn = Q - c * 4;
      xi[0] -= acc0;
      if (qn > 1) xi[1] -= acc1;
      if (qn > 2) xi[2] -= acc2;
      if (qn > 3) xi[3] -= acc3;
    }
  }
  __syncthreads();
  if (nbv > 0) {
    double *cout = a.carry + (int64_t(it.q0) - a.wave_base) * a.nbmax;
    for (int32_t idx = tid; idx < Q * nbv; idx += kSweepThreads) {
      const int32_t q = idx / nbv, t = idx - q * nbv;
      cout[int64_t(q) * a.nbmax + t] = X[(nc + t) * QP + q];
    }
  }
  if (tid < Q) {
    const int64_t slot = int64_t(it.q0) + tid;
    const double prev = it.src >= 0 ? a.racc[slot - a.wave_base] : 0.0;
    const double tot = prev + r;
    if (nbv > 0)
      a.racc[slot - a.wave_base] = tot;
    else
      a.R[a.qorig[slot]] = tot;
  }
}

int run_sweep_wave(const Symbolic &S, const SweepWave &W, const SweepItem *d_items,
                   const SweepArgs &args, cudaStream_t stream, cudaEvent_t *events,
                   std::string &err) {
  static int configured_smem = 0;   // per process; the kernel's limit only grows
  int64_t need = 0;
  for (int64_t b : W.level_smem) need = std::max(need, b);
  if (need > configured_smem) {
    CUDA_TRY(cudaFuncSetAttribute(k_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(need)));
    configured_smem = static_cast<int>(need);
  }
  SweepArgs a = args;
  a.wave_base = W.q_begin;
  for (int32_t l = 0; l < S.nlevels; ++l) {
    const int64_t i0 = W.level_ptr[l], i1 = W.level_ptr[l + 1];
    if (events) CUDA_TRY(cudaEventRecord(events[2 * l], stream));
    if (i1 > i0) {
      k_sweep<<<static_cast<unsigned>(i1 - i0), kSweepThreads, W.level_smem[l], stream>>>(
          d_items + i0, a);
      CUDA_TRY(cudaGetLastError());
    }
    if (events) CUDA_TRY(cudaEventRecord(events[2 * l + 1], stream));
  }
  return PEERS_OK;
}

}  // namespace peers
