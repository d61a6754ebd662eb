// Numeric supernodal L D L^T of the grounded Laplacian on the GPU (multifrontal).
//
// PEERS computes the factor first (Alg. 8 step 1; T_Chol in Table II) and then walks it;
// the paper leaves the factorization to a library.  Here it runs level by level over the
// supernodal elimination tree: every supernode of a level is independent (its children are
// all finished), so one launch covers the whole level.  Per level:
//   1. extend-add: the children's update matrices U_c are scattered into the parent's panel
//      and update matrix, one launch per child rank so that no two CTAs add to the same entry
//      and the summation order is fixed (deterministic, no atomics);
//   2. for each 32-column block J of the level's supernodes, right-looking:
//        k_diag_block   L_JJ D_J L_JJ^T of the diagonal block (one warp), d, 1/d, and the
//                       inverse of the unit-lower L_JJ used by the sweep;
//        k_panel_rows   L[i, J] = F[i, J] L_JJ^{-T} D_J^{-1} for every row below the block;
//        k_trailing     F[i, j] -= sum_k L[i, k] d_k L[j, k] over the trailing lower triangle
//                       (remaining panel columns and the update matrix), 64 x 64 tiles.
// FP64 throughout (DFMA; on this part the FP64 mma.sync path is not faster than DFMA).
#include <cuda_runtime.h>

#include <algorithm>

#include <mutex>

#include "device.cuh"
#include "internal.h"

namespace peers {

// panel[dest[e]] = val[e]: the entries of L_r (off-diagonals -w, diagonals = degrees).
__global__ void k_assemble(const int64_t *__restrict__ dest, const double *__restrict__ val,
                           int64_t cnt, double *__restrict__ panel, int64_t panel_total,
                           int *status) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < cnt;
       e += int64_t(gridDim.x) * blockDim.x)
    if (PEERS_IN(dest[e], panel_total, status)) panel[dest[e]] = val[e];
}

// One CTA per (pair, chunk of 8 child columns).  pairs = (parent, child) interleaved.
__global__ void __launch_bounds__(256) k_extend_add(const int32_t *__restrict__ pairs,
                                                    FactorArgs a) {
  const int32_t p = pairs[2 * blockIdx.x], c = pairs[2 * blockIdx.x + 1];
  const int32_t nbc = a.nb[c];
  const int32_t j0 = blockIdx.y * 8;
  if (j0 >= nbc) return;
  const int32_t j1 = min(nbc, j0 + 8);
  const int32_t ncp = a.first[p + 1] - a.first[p], nbp = a.nb[p], Np = ncp + nbp;
  const int32_t *rm = a.rmap + a.rows_off[c];
  const double *Uc = a.U + a.u_off[c];
  double *Pp = a.panel + a.panel_off[p];
  double *Up = a.U + a.u_off[p];
#if defined(PEERS_BOUNDS) && PEERS_BOUNDS
  const int64_t pext = a.panel_off[p + 1] - a.panel_off[p], uext = a.u_off[p + 1] - a.u_off[p];
  if (!PEERS_IN(int64_t(nbc) * nbc - 1, a.u_off[c + 1] - a.u_off[c], a.status) ||
      !PEERS_IN(nbc - 1, a.rows_off[c + 1] - a.rows_off[c], a.status))
    return;
#endif
  // each thread gathers kEaRows entries of a column before adding them, so that enough
  // loads are in flight to cover the memory latency
  constexpr int kEaRows = 4;
  for (int32_t j = j0; j < j1; ++j) {
    const int32_t rj = rm[j];
    const bool to_panel = rj < ncp;
    for (int32_t i0 = j + threadIdx.x; i0 < nbc; i0 += kEaRows * blockDim.x) {
      double v[kEaRows];
      int64_t dst[kEaRows];
#pragma unroll
      for (int u = 0; u < kEaRows; ++u) {
        const int32_t i = i0 + u * blockDim.x;
        dst[u] = -1;
        v[u] = 0.0;
        if (i >= nbc) continue;
        v[u] = Uc[int64_t(j) * nbc + i];
        const int32_t ri = rm[i];
        if (to_panel) {
          if (PEERS_IN(int64_t(rj) * Np + ri, pext, a.status)) dst[u] = int64_t(rj) * Np + ri;
        } else if (PEERS_IN(int64_t(rj - ncp) * nbp + (ri - ncp), uext, a.status) &&
                   PEERS_IN(ri - ncp, nbp, a.status)) {
          dst[u] = int64_t(rj - ncp) * nbp + (ri - ncp);
        }
      }
      double *base = to_panel ? Pp : Up;
      double old[kEaRows];
#pragma unroll
      for (int u = 0; u < kEaRows; ++u) old[u] = dst[u] >= 0 ? base[dst[u]] : 0.0;
#pragma unroll
      for (int u = 0; u < kEaRows; ++u)
        if (dst[u] >= 0) base[dst[u]] = old[u] + v[u];
    }
  }
}

// Row r and column c <= r of entry e of a lower triangle listed row by row.
__device__ __forceinline__ void tri_entry(int e, int &r, int &c) {
  r = static_cast<int>((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
  if ((r + 1) * (r + 2) / 2 <= e) ++r;
  if (r * (r + 1) / 2 > e) --r;
  c = e - r * (r + 1) / 2;
}

// Dense L D L^T of the bw x bw lower block A (shared memory, A[i][j] = row i, column j)
// without pivoting (L_r is SPD): afterwards A holds L below the diagonal (unit diagonal
// implied) and d on it.  Step k scales column k by 1/d_k and forms -(L[i][k] d_k) once per
// row, then every (i, j) with k < j <= i takes A[i][j] -= (L[i][k] d_k) L[j][k]; the entries
// of the step's triangle are dealt to all threads of the CTA.
__device__ void ldlt_block(double (*A)[kBlock + 1], int bw, int *status, int col0) {
  __shared__ double cneg[kBlock];
  for (int k = 0; k < bw; ++k) {
    const double dk = A[k][k];
    if (threadIdx.x == 0 && !(dk > 0.0 && dk < INFINITY)) flag_error(status, kErrNotSpd, col0 + k);
    for (int i = k + 1 + threadIdx.x; i < bw; i += blockDim.x) {
      const double l = A[i][k] / dk;
      A[i][k] = l;
      cneg[i] = -(l * dk);
    }
    __syncthreads();
    const int m = bw - k - 1;
    for (int e = threadIdx.x; e < m * (m + 1) / 2; e += blockDim.x) {
      int r, c;
      tri_entry(e, r, c);
      const int i = k + 1 + r, j = k + 1 + c;
      A[i][j] = fma(cneg[i], A[j][k], A[i][j]);
    }
    __syncthreads();
  }
}

// X = the inverse of the unit-lower L held below the diagonal of A, by column sweeps: X
// starts as the identity and step k takes X[i][j] -= L[i][k] X[k][j] for i > k >= j.  Every
// entry adds its terms in increasing k, as row-by-row substitution does.
__device__ void unit_lower_inverse(const double (*A)[kBlock + 1], double (*X)[kBlock + 1],
                                   int bw) {
  for (int e = threadIdx.x; e < kBlock * kBlock; e += blockDim.x) {
    const int i = e / kBlock, j = e % kBlock;
    X[i][j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = 0; k + 1 < bw; ++k) {
    const int rows = bw - k - 1, cols = k + 1;
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int i = k + 1 + e / cols, j = e % cols;
      X[i][j] = fma(-A[i][k], X[k][j], X[i][j]);
    }
    __syncthreads();
  }
}

// Row i of the panel below the diagonal block: w = F[i, J] L_JJ^{-T}, then L[i, J] = w / d,
// taken as w times the stored 1/d, from the block's inverse X: w_k = sum_{j <= k} F[i][j]
// X[k][j].  The columns k of a row are independent sums, dealt to kPanelSplit threads
// (k = q, q + kPanelSplit, ...).  A thread walks j once and adds F[i][j] to every one of its
// sums that still takes it, so its dependent chain is one row long, not the sum of its
// columns' lengths; each w_k still adds its terms in increasing j.
constexpr int kPanelSplit = 4;
__device__ __forceinline__ void panel_row_from_inverse(const double *Frow, int64_t fstride,
                                                       const double (*X)[kBlock + 1],
                                                       const double *rd, int bw, int q,
                                                       double *Lrow, int64_t lstride) {
  constexpr int M = kBlock / kPanelSplit;
  double w[M];
#pragma unroll
  for (int m = 0; m < M; ++m) w[m] = 0.0;
  // segment sg: the j taken by the sums m >= sg only (k_m = q + kPanelSplit m >= j)
#pragma unroll
  for (int sg = 0; sg < M; ++sg) {
    const int jb = sg == 0 ? 0 : q + kPanelSplit * (sg - 1) + 1;
    const int je = min(q + kPanelSplit * sg, bw - 1);
    for (int j = jb; j <= je; ++j) {
      const double fj = Frow[j * fstride];
#pragma unroll
      for (int m = sg; m < M; ++m)
        if (q + kPanelSplit * m < bw) w[m] = fma(fj, X[q + kPanelSplit * m][j], w[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int k = q + kPanelSplit * m;
    if (k < bw) Lrow[k * lstride] = w[m] * rd[k];
  }
}

// Diagonal block J of each active supernode: dense L D L^T without pivoting, its d and 1/d,
// and the inverse of the unit-lower block (used by the panel rows and the sweep).  One CTA
// of 256 threads per supernode.
__global__ void __launch_bounds__(256) k_diag_block(const int32_t *__restrict__ sns, int32_t J,
                                                    FactorArgs a) {
  __shared__ double A[kBlock][kBlock + 1];
  __shared__ double X[kBlock][kBlock + 1];
  const int32_t s = sns[blockIdx.x];
  const int32_t f = a.first[s], nc = a.first[s + 1] - f, N = nc + a.nb[s];
  const int32_t c0 = J * kBlock, bw = min(kBlock, nc - c0);
  double *P = a.panel + a.panel_off[s];
  // the block's panel columns and inverse lie inside the supernode's stored extents
  if (!PEERS_IN(int64_t(c0 + bw) * N - 1, a.panel_off[s + 1] - a.panel_off[s], a.status) ||
      !PEERS_IN(int64_t(J) * kBlock * kBlock + bw * bw - 1, a.tinv_off[s + 1] - a.tinv_off[s],
                a.status))
    return;
  for (int e = threadIdx.x; e < kBlock * kBlock; e += blockDim.x) {
    const int i = e % kBlock, j = e / kBlock;   // consecutive threads read down a column
    A[i][j] = (i < bw && j < bw && i >= j) ? P[int64_t(c0 + j) * N + c0 + i] : 0.0;
  }
  __syncthreads();
  ldlt_block(A, bw, a.status, f + c0);
  // write L_JJ (strict lower), d (the diagonal slot keeps d), 1/d
  for (int e = threadIdx.x; e < bw * bw; e += blockDim.x) {
    const int i = e % bw, j = e / bw;
    if (i >= j) P[int64_t(c0 + j) * N + c0 + i] = A[i][j];
  }
  if (threadIdx.x < bw) {
    const double dk = A[threadIdx.x][threadIdx.x];
    a.d[f + c0 + threadIdx.x] = dk;
    a.dinv[f + c0 + threadIdx.x] = 1.0 / dk;
  }
  unit_lower_inverse(A, X, bw);
  double *T = a.tinv + a.tinv_off[s] + int64_t(J) * kBlock * kBlock;
  for (int e = threadIdx.x; e < bw * bw; e += blockDim.x) {
    const int i = e / bw, j = e % bw;
    T[i * bw + j] = j <= i ? X[i][j] : 0.0;
  }
}

// Rows below the diagonal block: L[i, c0+k] = w_k / d_k, w = F[i, J] L_JJ^{-T}, from the
// block's inverse formed by k_diag_block.  grid = (active supernode, chunk of 32 rows); the
// 32 rows of a chunk are staged in shared memory and each row's columns are shared by
// kPanelSplit warps.
__global__ void __launch_bounds__(kBlock * kPanelSplit) k_panel_rows(const int32_t *__restrict__ sns,
                                                                     int32_t J, FactorArgs a) {
  __shared__ double X[kBlock][kBlock + 1];
  __shared__ double Fr[kBlock][kBlock + 1];   // Fr[j][r]: column j of the chunk's row r
  __shared__ double rd[kBlock];
  const int32_t s = sns[blockIdx.x];
  const int32_t f = a.first[s], nc = a.first[s + 1] - f, N = nc + a.nb[s];
  const int32_t c0 = J * kBlock, bw = min(kBlock, nc - c0);
  const int32_t r0 = c0 + bw + blockIdx.y * kBlock;
  if (r0 >= N) return;
  double *P = a.panel + a.panel_off[s];
  if (!PEERS_IN(int64_t(c0 + bw) * N - 1, a.panel_off[s + 1] - a.panel_off[s], a.status)) return;
  const double *T = a.tinv + a.tinv_off[s] + int64_t(J) * kBlock * kBlock;
  for (int e = threadIdx.x; e < kBlock * kBlock; e += blockDim.x) {
    const int i = e / kBlock, j = e % kBlock;
    X[i][j] = (i < bw && j < bw) ? T[i * bw + j] : 0.0;
    const int r = e % kBlock, c = e / kBlock;   // coalesced down each panel column
    Fr[c][r] = (c < bw && r0 + r < N) ? P[int64_t(c0 + c) * N + r0 + r] : 0.0;
  }
  if (threadIdx.x < kBlock) rd[threadIdx.x] = threadIdx.x < bw ? a.dinv[f + c0 + threadIdx.x] : 1.0;
  __syncthreads();
  const int r = threadIdx.x % kBlock, q = threadIdx.x / kBlock;
  if (r0 + r < N)
    panel_row_from_inverse(&Fr[0][r], kBlock + 1, X, rd, bw, q, P + int64_t(c0) * N + r0 + r, N);
}

// Trailing update of block J: F[i, j] -= sum_k L[i, c0+k] d_k L[j, c0+k] for t0 <= j <= i < N,
// t0 = c0 + bw.  Column j < nc lives in the panel, j >= nc in the update matrix U_s.
// TS x TS tiles (TS = 64, or 32 for launches with few tiles, so that their work spreads over
// more SMs); 16 x 16 threads, (TS/16)^2 outputs each.  Every output sums over k in the same
// order whatever TS is.  kTrailAll updates every column after block J.  A split block runs
// three parts instead: kTrailNext, block J + 1's columns (one column of tiles per supernode,
// TS = 32); kTrailPanelRest, the panel's columns after block J + 1 (the tiles of that column
// range that reach the diagonal or below it); kTrailU, the update matrix's triangle.
constexpr int kTrailAll = 0, kTrailNext = 1, kTrailPanelRest = 2, kTrailU = 3;

// acc[u][v] += sum_k Li[k][tx + 16u] Lj[k][ty + 16v] over the sub-blocks u < NU, v < NV
// (and, for a tile on the diagonal, v <= u); NU, NV and DIAG are compile-time so that no
// multiply-add is issued for a skipped sub-block.
template <int TS, int NU, int NV, bool DIAG>
__device__ __forceinline__ void trail_fma_n(const double (*Li)[TS], const double (*Lj)[TS],
                                            int bw, int tx, int ty, double (*acc)[TS / 16]) {
  constexpr int U = TS / 16;
  for (int k = 0; k < bw; ++k) {
    double li[U], lj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      li[u] = u < NU ? Li[k][tx + 16 * u] : 0.0;
      lj[u] = u < NV ? Lj[k][ty + 16 * u] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < NU; ++u)
#pragma unroll
      for (int v = 0; v < (DIAG ? (u + 1 < NV ? u + 1 : NV) : NV); ++v)
        acc[u][v] = fma(li[u], lj[v], acc[u][v]);
  }
}
#define PEERS_TRAIL_FMA(NU_, NV_)                                              \
  if (nu == NU_ && nv == NV_) {                                                \
    trail_fma_n<TS, NU_, NV_, DIAG>(Li, Lj, bw, tx, ty, acc);                  \
    return;                                                                    \
  }
template <int TS, bool DIAG>
__device__ __forceinline__ void trail_fma(const double (*Li)[TS], const double (*Lj)[TS], int bw,
                                          int nu, int nv, int tx, int ty, double (*acc)[TS / 16]) {
  if constexpr (TS == 32) {
    PEERS_TRAIL_FMA(1, 1) PEERS_TRAIL_FMA(1, 2) PEERS_TRAIL_FMA(2, 1)
  } else {
    PEERS_TRAIL_FMA(1, 1) PEERS_TRAIL_FMA(1, 2) PEERS_TRAIL_FMA(1, 3) PEERS_TRAIL_FMA(1, 4)
    PEERS_TRAIL_FMA(2, 1) PEERS_TRAIL_FMA(2, 2) PEERS_TRAIL_FMA(2, 3) PEERS_TRAIL_FMA(2, 4)
    PEERS_TRAIL_FMA(3, 1) PEERS_TRAIL_FMA(3, 2) PEERS_TRAIL_FMA(3, 3) PEERS_TRAIL_FMA(3, 4)
    PEERS_TRAIL_FMA(4, 1) PEERS_TRAIL_FMA(4, 2) PEERS_TRAIL_FMA(4, 3)
  }
  trail_fma_n<TS, TS / 16, TS / 16, DIAG>(Li, Lj, bw, tx, ty, acc);
}
#undef PEERS_TRAIL_FMA

template <int TS, int MODE>
__global__ void __launch_bounds__(256) k_trailing(const int32_t *__restrict__ sns, int32_t J,
                                                  const int64_t *__restrict__ prefix, int32_t na,
                                                  FactorArgs a) {
  constexpr int U = TS / 16;
  __shared__ double Li[kBlock][TS];
  __shared__ double Lj[kBlock][TS];
  // locate the supernode of this tile
  const int64_t t = blockIdx.x;
  int32_t lo = 0, hi = na;   // prefix[lo] <= t < prefix[hi]
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) / 2;
    if (prefix[mid] <= t) lo = mid; else hi = mid;
  }
  const int32_t s = sns[lo];
  const int64_t lt = t - prefix[lo];
  const int32_t f = a.first[s], nc = a.first[s + 1] - f, nbv = a.nb[s], N = nc + nbv;
  const int32_t c0 = J * kBlock, bw = min(kBlock, nc - c0);
  // the part's first column (and row) and its column limit
  const int32_t base = MODE == kTrailPanelRest ? min(nc, c0 + 2 * kBlock)
                       : MODE == kTrailU       ? nc
                                               : c0 + bw;
  const int32_t clim = MODE == kTrailNext ? min(nc, base + kBlock)
                       : MODE == kTrailPanelRest ? nc
                                                 : N;
  int64_t ti = lt, tj = 0;
  if (MODE == kTrailPanelRest) {   // column tj holds the row tiles tj .. (N - base) / TS
    const int64_t T = (N - base + TS - 1) / TS;
    int64_t rem = lt;
    while (tj < T && rem >= T - tj) { rem -= T - tj; ++tj; }
    ti = tj + rem;
  } else if (MODE != kTrailNext) {
    ti = static_cast<int64_t>((sqrt(8.0 * double(lt) + 1.0) - 1.0) * 0.5);
    while (ti * (ti + 1) / 2 > lt) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= lt) ++ti;
    tj = lt - ti * (ti + 1) / 2;
  }
  const int32_t R0 = base + int32_t(ti) * TS, C0 = base + int32_t(tj) * TS;
  const double *P = a.panel + a.panel_off[s];
#if defined(PEERS_BOUNDS) && PEERS_BOUNDS
  const int64_t pext = a.panel_off[s + 1] - a.panel_off[s], uext = a.u_off[s + 1] - a.u_off[s];
  if (!PEERS_IN(int64_t(c0 + bw) * N - 1, pext, a.status)) return;
#endif
  for (int idx = threadIdx.x; idx < kBlock * TS; idx += blockDim.x) {
    const int k = idx / TS, r = idx % TS;
    const bool kin = k < bw;
    Li[k][r] = (kin && R0 + r < N) ? P[int64_t(c0 + k) * N + R0 + r] : 0.0;
    Lj[k][r] = (kin && C0 + r < clim) ? P[int64_t(c0 + k) * N + C0 + r] * a.d[f + c0 + k] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[U][U] = {};
  // sub-blocks of 16 x 16 outputs that no write keeps get no multiply-adds: on a tile of the
  // diagonal those with u < v (wholly above it), on the last row of tiles those whose 16 rows
  // all lie at or beyond N, on the last column of tiles those whose 16 columns all lie at or
  // beyond the part's column limit
  const int nu = min(U, (N - R0 + 15) / 16), nv = min(U, (clim - C0 + 15) / 16);
  if (R0 == C0)
    trail_fma<TS, true>(Li, Lj, bw, nu, nv, tx, ty, acc);
  else
    trail_fma<TS, false>(Li, Lj, bw, nu, nv, tx, ty, acc);
  double *Pw = a.panel + a.panel_off[s];
  double *Uw = a.U + a.u_off[s];
#pragma unroll
  for (int v = 0; v < U; ++v) {
    const int32_t j = C0 + ty + 16 * v;
    if (j >= clim) continue;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int32_t i = R0 + tx + 16 * u;
      if (i >= N || i < j) continue;
      if (j < nc) {
        if (PEERS_IN(int64_t(j) * N + i, pext, a.status)) Pw[int64_t(j) * N + i] -= acc[u][v];
      } else if (PEERS_IN(int64_t(j - nc) * nbv + (i - nc), uext, a.status)) {
        Uw[int64_t(j - nc) * nbv + (i - nc)] -= acc[u][v];
      }
    }
  }
}

// A whole supernode of one column block (n_c <= kBlock) whose front has at most kFactorFuseN
// rows, by one CTA in shared memory.  The front F (N x N, column-major, ld = N) is filled from
// the panel's assembled entries and the children's update matrices, added child by child in
// child order (the order of the per-rank k_extend_add launches); then the operations of
// k_diag_block, k_panel_rows and k_trailing run in their order on F, and the panel, d, 1/d,
// the diagonal-block inverse and the update matrix are written back.  The results are those
// of the blocked kernels bit for bit; the small supernodes of the lower levels just need one
// launch per level instead of four or more.
__global__ void __launch_bounds__(256) k_factor_small(const int32_t *__restrict__ sns,
                                                      const int32_t *__restrict__ child_ptr,
                                                      const int32_t *__restrict__ child_list,
                                                      FactorArgs a) {
  extern __shared__ double sm_fac[];
  __shared__ double A[kBlock][kBlock + 1];
  __shared__ double X[kBlock][kBlock + 1];
  __shared__ double dk[kBlock];
  __shared__ double rd[kBlock];
  const int32_t s = sns[blockIdx.x];
  const int32_t f = a.first[s], nc = a.first[s + 1] - f, nbv = a.nb[s], N = nc + nbv;
  const int bw = nc;   // one column block
  double *F = sm_fac;
  double *P = a.panel + a.panel_off[s];
  const int tid = threadIdx.x;
  // the front fits the launch's shared memory; panel, inverse and update matrix their extents
  if (!PEERS_IN(int64_t(N) * N - 1, dynamic_smem_doubles(), a.status) ||
      !PEERS_IN(int64_t(N) * nc - 1, a.panel_off[s + 1] - a.panel_off[s], a.status) ||
      !PEERS_IN(int64_t(nc) * nc - 1, a.tinv_off[s + 1] - a.tinv_off[s], a.status) ||
      !(nbv == 0 || PEERS_IN(int64_t(nbv) * nbv - 1, a.u_off[s + 1] - a.u_off[s], a.status)))
    return;
  for (int idx = tid; idx < N * N; idx += blockDim.x) F[idx] = idx / N < nc ? P[idx] : 0.0;
  __syncthreads();
  for (int32_t c = child_ptr[s]; c < child_ptr[s + 1]; ++c) {
    const int32_t ch = child_list[c];
    const int32_t nbc = a.nb[ch];
    const int32_t *rm = a.rmap + a.rows_off[ch];
    const double *Uc = a.U + a.u_off[ch];
    for (int idx = tid; idx < nbc * nbc; idx += blockDim.x) {
      const int j = idx / nbc, i = idx - j * nbc;
      if (i >= j && PEERS_IN(idx, a.u_off[ch + 1] - a.u_off[ch], a.status) &&
          PEERS_IN(int64_t(rm[j]) * N + rm[i], int64_t(N) * N, a.status))
        F[rm[j] * N + rm[i]] += Uc[idx];
    }
    __syncthreads();
  }
  // diagonal block: L_JJ D_J L_JJ^T and its inverse (k_diag_block's operations)
  for (int e = tid; e < kBlock * kBlock; e += blockDim.x) {
    const int i = e % kBlock, j = e / kBlock;
    A[i][j] = (i < bw && j < bw && i >= j) ? F[j * N + i] : 0.0;
  }
  __syncthreads();
  ldlt_block(A, bw, a.status, f);
  for (int e = tid; e < bw * bw; e += blockDim.x) {
    const int i = e % bw, j = e / bw;
    if (i >= j) P[int64_t(j) * N + i] = A[i][j];
  }
  if (tid < bw) {
    const double d = A[tid][tid];
    dk[tid] = d;
    rd[tid] = 1.0 / d;
    a.d[f + tid] = d;
    a.dinv[f + tid] = rd[tid];
  }
  unit_lower_inverse(A, X, bw);
  {
    double *T = a.tinv + a.tinv_off[s];
    for (int e = tid; e < bw * bw; e += blockDim.x) {
      const int i = e / bw, j = e % bw;
      T[i * bw + j] = j <= i ? X[i][j] : 0.0;
    }
  }
  // rows below the block (k_panel_rows' operations), written to the panel and read back
  const int rows = N - bw;
  for (int e = tid; e < rows * kPanelSplit; e += blockDim.x) {
    const int i = bw + e % rows, q = e / rows;
    panel_row_from_inverse(F + i, N, X, rd, bw, q, P + i, N);
  }
  __syncthreads();
  for (int e = tid; e < rows * bw; e += blockDim.x) {
    const int i = bw + e % rows, k = e / rows;
    F[k * N + i] = P[int64_t(k) * N + i];
  }
  __syncthreads();
  // trailing update of the update matrix: F[i, j] -= sum_k L[i, k] (L[j, k] d_k) (k_trailing)
  double *Uw = a.U + a.u_off[s];
  // the lower triangle (ii >= jj) only, dealt to the threads entry by entry
  for (int e = tid; e < nbv * (nbv + 1) / 2; e += blockDim.x) {
    int ii, jj;
    tri_entry(e, ii, jj);
    const int i = nc + ii, j = nc + jj;
    double acc = 0.0;
    for (int k = 0; k < bw; ++k) acc = fma(F[k * N + i], F[k * N + j] * dk[k], acc);
    Uw[int64_t(jj) * nbv + ii] = F[j * N + i] - acc;
  }
}

// Every kernel of the factorization asks for the largest shared-memory carveout, so that an SM
// running one of them can take the others' CTAs without a reconfiguration: the lanes' and the
// split groups' streams run different kernels side by side.  Once per device.
static int set_factor_carveout(std::string &err) {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    err = "device index out of range";
    return PEERS_EINVAL;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return PEERS_OK;
  const void *ks[] = {
      reinterpret_cast<const void *>(k_assemble),
      reinterpret_cast<const void *>(k_extend_add),
      reinterpret_cast<const void *>(k_diag_block),
      reinterpret_cast<const void *>(k_panel_rows),
      reinterpret_cast<const void *>(k_factor_small),
      reinterpret_cast<const void *>(k_trailing<32, kTrailAll>),
      reinterpret_cast<const void *>(k_trailing<64, kTrailAll>),
      reinterpret_cast<const void *>(k_trailing<32, kTrailNext>),
      reinterpret_cast<const void *>(k_trailing<32, kTrailPanelRest>),
      reinterpret_cast<const void *>(k_trailing<64, kTrailPanelRest>),
      reinterpret_cast<const void *>(k_trailing<32, kTrailU>),
      reinterpret_cast<const void *>(k_trailing<64, kTrailU>)};
  for (const void *k : ks)
    CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared));
  done[dev] = true;
  return PEERS_OK;
}

// Host driver: the full factorization on `stream`, with the lanes' subtrees on the lane
// streams when `lanes` is given (see kLanes).  Returns a PEERS_* status.
int run_factor(const Symbolic &S, const FactorDevice &D, cudaStream_t stream, const Lanes *lanes,
               int64_t *launches, std::string &err) {
  FactorArgs a = D.args;
  if (S.one_stream) lanes = nullptr;
  {
    const int rc = set_factor_carveout(err);
    if (rc != PEERS_OK) return rc;
  }
  CUDA_TRY(cudaMemsetAsync(a.panel, 0, sizeof(double) * S.panel_total, stream));
  if (S.u_total > 0) CUDA_TRY(cudaMemsetAsync(a.U, 0, sizeof(double) * S.u_total, stream));
  CUDA_TRY(cudaMemsetAsync(a.status, 0, sizeof(int) * 2, stream));
  {
    const int64_t cnt = static_cast<int64_t>(S.a_dest.size());
    const int blocks = static_cast<int>(std::min<int64_t>((cnt + 255) / 256, 148 * 16));
    if (cnt > 0) {
      k_assemble<<<blocks, 256, 0, stream>>>(D.a_dest, D.a_val, cnt, a.panel, S.panel_total,
                                             a.status);
      ++*launches;
    }
    CUDA_TRY(cudaGetLastError());
  }
  {
    int64_t smem = 0;
    for (int32_t s : S.fuse_sn) {
      const int64_t N = sn_nc(S, s) + S.nb[s];
      smem = std::max(smem, 8 * N * N);
    }
    static int fuse_smem[64] = {};   // limit set so far, per device
    const int rc = raise_smem_limit(reinterpret_cast<const void *>(k_factor_small), fuse_smem,
                                    smem, err);
    if (rc != PEERS_OK) return rc;
  }
  // the lanes start once the panels are assembled; the top part starts once they are done
  const bool forked = lanes && S.nlanes > 0;
  if (forked) {
    CUDA_TRY(cudaEventRecord(lanes->start, stream));
    for (int L = 0; L < S.nlanes; ++L) CUDA_TRY(cudaStreamWaitEvent(lanes->stream[L], lanes->start, 0));
  }
  bool joined = !forked;
  auto join = [&]() -> int {
    for (int L = 0; L < S.nlanes; ++L) {
      CUDA_TRY(cudaEventRecord(lanes->done[L], lanes->stream[L]));
      CUDA_TRY(cudaStreamWaitEvent(stream, lanes->done[L], 0));
    }
    joined = true;
    return PEERS_OK;
  };
  for (const FactorGroup &G : S.fgroups) {
    if (G.lane < 0 && !joined) {
      const int rc = join();
      if (rc != PEERS_OK) return rc;
    }
    const cudaStream_t st = (G.lane >= 0 && forked) ? lanes->stream[G.lane] : stream;
    const int32_t *sns = D.fac_sn + G.fac_b;
    // 0. supernodes factored whole, one CTA each
    if (G.fuse_e > G.fuse_b) {
      int64_t smem = 0;
      for (int32_t i = G.fuse_b; i < G.fuse_e; ++i) {
        const int64_t N = sn_nc(S, S.fuse_sn[i]) + S.nb[S.fuse_sn[i]];
        smem = std::max(smem, 8 * N * N);
      }
      k_factor_small<<<static_cast<unsigned>(G.fuse_e - G.fuse_b), 256, smem, st>>>(
          D.fuse_sn + G.fuse_b, D.child_ptr, D.child_list, a);
      ++*launches;
      CUDA_TRY(cudaGetLastError());
    }
    // 1. extend-add of the blocked supernodes' children, one launch per child rank
    for (int64_t r = G.ea_b; r < G.ea_e; ++r) {
      const int64_t p0 = S.ea_off[r], p1 = S.ea_off[r + 1];
      if (p1 <= p0) continue;
      int32_t maxnb = 0;
      for (int64_t q = p0; q < p1; ++q) maxnb = std::max(maxnb, S.nb[S.ea_pairs[2 * q + 1]]);
      if (maxnb == 0) continue;
      dim3 grid(static_cast<unsigned>(p1 - p0), static_cast<unsigned>((maxnb + 7) / 8));
      k_extend_add<<<grid, 256, 0, st>>>(D.ea_pairs + 2 * p0, a);
      ++*launches;
      CUDA_TRY(cudaGetLastError());
    }
    // 2. right-looking column blocks
    auto factor_block = [&](int32_t J, cudaStream_t bs) -> int {
      const int32_t na = static_cast<int32_t>(S.trail_na[G.trail_base + J]);
      k_diag_block<<<na, 256, 0, bs>>>(sns, J, a);
      ++*launches;
      CUDA_TRY(cudaGetLastError());
      int32_t maxrows = 0;
      for (int32_t i = 0; i < na; ++i) {
        const int32_t s = S.fac_sn[G.fac_b + i];
        const int32_t nc = sn_nc(S, s), N = nc + S.nb[s];
        maxrows = std::max(maxrows, N - std::min(nc, (J + 1) * kBlock));
      }
      if (maxrows > 0) {
        dim3 grid(static_cast<unsigned>(na), static_cast<unsigned>((maxrows + kBlock - 1) / kBlock));
        k_panel_rows<<<grid, kBlock * kPanelSplit, 0, bs>>>(sns, J, a);
        ++*launches;
        CUDA_TRY(cudaGetLastError());
      }
      return PEERS_OK;
    };
    // one part of block J's update (kTrail*) on stream `ts_`
    auto trailing = [&](int32_t J, int mode, cudaStream_t ts_) -> int {
      const int64_t tp = G.trail_base + J;
      const int32_t na = static_cast<int32_t>(S.trail_na[tp]);
      const int32_t nn = static_cast<int32_t>(S.next_na[tp]);
      int64_t off = S.trail_off[tp];
      int32_t cnt = na, ts = S.trail_ts[tp];
      if (mode == kTrailNext) { off = S.split_off[tp]; cnt = nn; ts = kTile / 2; }
      if (mode == kTrailPanelRest) { off = S.split_off[tp] + nn + 1; ts = S.pr_ts[tp]; }
      if (mode == kTrailU) { off = S.split_off[tp] + nn + na + 2; ts = S.up_ts[tp]; }
      const int64_t ntiles = S.trail_prefix[off + cnt];
      if (ntiles <= 0) return PEERS_OK;
      const unsigned g = static_cast<unsigned>(ntiles);
      const int64_t *pre = D.trail_prefix + off;
      if (mode == kTrailNext)
        k_trailing<32, kTrailNext><<<g, 256, 0, ts_>>>(sns, J, pre, cnt, a);
      else if (mode == kTrailPanelRest && ts == 32)
        k_trailing<32, kTrailPanelRest><<<g, 256, 0, ts_>>>(sns, J, pre, cnt, a);
      else if (mode == kTrailPanelRest)
        k_trailing<64, kTrailPanelRest><<<g, 256, 0, ts_>>>(sns, J, pre, cnt, a);
      else if (mode == kTrailU && ts == 32)
        k_trailing<32, kTrailU><<<g, 256, 0, ts_>>>(sns, J, pre, cnt, a);
      else if (mode == kTrailU)
        k_trailing<64, kTrailU><<<g, 256, 0, ts_>>>(sns, J, pre, cnt, a);
      else if (ts == 32)
        k_trailing<32, kTrailAll><<<g, 256, 0, ts_>>>(sns, J, pre, cnt, a);
      else
        k_trailing<64, kTrailAll><<<g, 256, 0, ts_>>>(sns, J, pre, cnt, a);
      ++*launches;
      CUDA_TRY(cudaGetLastError());
      return PEERS_OK;
    };
    int rc = PEERS_OK;
    if (!G.split || !lanes) {
      for (int32_t J = 0; J < G.nblocks; ++J) {
        if (S.trail_na[G.trail_base + J] == 0) continue;
        if ((rc = factor_block(J, st)) != PEERS_OK) return rc;
        if ((rc = trailing(J, kTrailAll, st)) != PEERS_OK) return rc;
      }
      continue;
    }
    // A split group: the chain (block J's diagonal block and panel rows, then block J + 1's
    // columns) on a stream of the device's highest priority; the panel's remaining columns on
    // the group's own stream; the update matrix on a third stream, off the chain.  Block
    // J + 1's columns are updated after the panel rest of block J - 1 (both write them), and
    // every part of block J starts once its panel rows are done.  The group's stream joins the
    // other two at its end.  Each entry still takes its updates in increasing J.
    const int li = G.lane >= 0 && forked ? G.lane : kLanes;
    const cudaStream_t cs = lanes->chain[li], us = lanes->upd[li];
    CUDA_TRY(cudaEventRecord(lanes->ev_start[li], st));
    CUDA_TRY(cudaStreamWaitEvent(cs, lanes->ev_start[li], 0));
    CUDA_TRY(cudaStreamWaitEvent(us, lanes->ev_start[li], 0));
    for (int32_t J = 0; J < G.nblocks; ++J) {
      if (S.trail_na[G.trail_base + J] == 0) break;
      if (J == 0 && (rc = factor_block(0, cs)) != PEERS_OK) return rc;
      CUDA_TRY(cudaEventRecord(lanes->ev_panel[li], cs));
      if (J > 0) CUDA_TRY(cudaStreamWaitEvent(cs, lanes->ev_rest[li], 0));
      if ((rc = trailing(J, kTrailNext, cs)) != PEERS_OK) return rc;
      CUDA_TRY(cudaStreamWaitEvent(st, lanes->ev_panel[li], 0));
      if ((rc = trailing(J, kTrailPanelRest, st)) != PEERS_OK) return rc;
      CUDA_TRY(cudaEventRecord(lanes->ev_rest[li], st));
      CUDA_TRY(cudaStreamWaitEvent(us, lanes->ev_panel[li], 0));
      if ((rc = trailing(J, kTrailU, us)) != PEERS_OK) return rc;
      if (J + 1 < G.nblocks && S.trail_na[G.trail_base + J + 1] > 0 &&
          (rc = factor_block(J + 1, cs)) != PEERS_OK)
        return rc;
    }
    CUDA_TRY(cudaEventRecord(lanes->ev_chain[li], cs));
    CUDA_TRY(cudaEventRecord(lanes->ev_upd[li], us));
    CUDA_TRY(cudaStreamWaitEvent(st, lanes->ev_chain[li], 0));
    CUDA_TRY(cudaStreamWaitEvent(st, lanes->ev_upd[li], 0));
  }
  if (!joined) {
    const int rc = join();
    if (rc != PEERS_OK) return rc;
  }
  int status[2] = {0, 0};
  CUDA_TRY(cudaMemcpyAsync(status, a.status, sizeof(status), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  if (status[0] == kErrNotSpd) {
    err = "non-positive pivot at elimination position " + std::to_string(status[1]);
    return PEERS_ENOTSPD;
  }
  if (status[0] == kErrBounds) {
    err = "peers_factor: out-of-bounds access skipped at source line " + std::to_string(status[1]);
    return PEERS_ECUDA;
  }
  return PEERS_OK;
}

}  // namespace peers
