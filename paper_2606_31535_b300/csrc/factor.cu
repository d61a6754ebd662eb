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

#include "device.cuh"
#include "internal.h"

namespace peers {

// panel[dest[e]] = val[e]: the entries of L_r (off-diagonals -w, diagonals = degrees).
__global__ void k_assemble(const int64_t *__restrict__ dest, const double *__restrict__ val,
                           int64_t cnt, double *__restrict__ panel) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < cnt;
       e += int64_t(gridDim.x) * blockDim.x)
    panel[dest[e]] = val[e];
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
  for (int32_t j = j0; j < j1; ++j) {
    const int32_t rj = rm[j];
    for (int32_t i = j + threadIdx.x; i < nbc; i += blockDim.x) {
      const double v = Uc[int64_t(j) * nbc + i];
      const int32_t ri = rm[i];
      if (rj < ncp)
        Pp[int64_t(rj) * Np + ri] += v;
      else
        Up[int64_t(rj - ncp) * nbp + (ri - ncp)] += v;
    }
  }
}

// Diagonal block J of each active supernode: dense L D L^T without pivoting (L_r is SPD),
// then the inverse of the unit-lower block for the sweep.  One CTA (one warp) per supernode.
__global__ void __launch_bounds__(32) k_diag_block(const int32_t *__restrict__ sns, int32_t J,
                                                   FactorArgs a) {
  __shared__ double A[kBlock][kBlock + 1];
  __shared__ double X[kBlock][kBlock + 1];
  const int32_t s = sns[blockIdx.x];
  const int32_t f = a.first[s], nc = a.first[s + 1] - f, N = nc + a.nb[s];
  const int32_t c0 = J * kBlock, bw = min(kBlock, nc - c0);
  double *P = a.panel + a.panel_off[s];
  const int lane = threadIdx.x;
  for (int j = 0; j < bw; ++j)
    A[lane][j] = (lane < bw && lane >= j) ? P[int64_t(c0 + j) * N + c0 + lane] : 0.0;
  __syncwarp();
  for (int k = 0; k < bw; ++k) {
    const double dk = A[k][k];
    if (lane == 0 && !(dk > 0.0 && dk < INFINITY)) flag_error(a.status, kErrNotSpd, f + c0 + k);
    if (lane > k && lane < bw) A[lane][k] = A[lane][k] / dk;
    __syncwarp();
    if (lane > k && lane < bw) {
      const double lk = A[lane][k] * dk;
      for (int j = k + 1; j <= lane; ++j) A[lane][j] = fma(-lk, A[j][k], A[lane][j]);
    }
    __syncwarp();
  }
  // write L_JJ (strict lower), d (diagonal slot keeps d), 1/d
  if (lane < bw) {
    for (int j = 0; j < lane; ++j) P[int64_t(c0 + j) * N + c0 + lane] = A[lane][j];
    const double dk = A[lane][lane];
    P[int64_t(c0 + lane) * N + c0 + lane] = dk;
    a.d[f + c0 + lane] = dk;
    a.dinv[f + c0 + lane] = 1.0 / dk;
  }
  // inverse of the unit-lower L_JJ, column `lane`: X[i][lane] for i >= lane
  if (lane < bw) {
    X[lane][lane] = 1.0;
    for (int i = lane + 1; i < bw; ++i) {
      double t = 0.0;
      for (int k = lane; k < i; ++k) t = fma(A[i][k], X[k][lane], t);
      X[i][lane] = -t;
    }
  }
  __syncwarp();
  double *T = a.tinv + a.tinv_off[s] + int64_t(J) * kBlock * kBlock;
  for (int i = 0; i < bw; ++i)
    if (lane < bw) T[i * bw + lane] = lane <= i ? X[i][lane] : 0.0;
}

// Rows below the diagonal block: L[i, c0+k] = w_k / d_k with w L_JJ^T = F[i, J] (forward
// substitution along the row).  grid = (active supernode, chunk of 128 rows).
__global__ void __launch_bounds__(128) k_panel_rows(const int32_t *__restrict__ sns, int32_t J,
                                                    FactorArgs a) {
  __shared__ double Ls[kBlock][kBlock + 1];
  __shared__ double dk[kBlock];
  const int32_t s = sns[blockIdx.x];
  const int32_t f = a.first[s], nc = a.first[s + 1] - f, N = nc + a.nb[s];
  const int32_t c0 = J * kBlock, bw = min(kBlock, nc - c0);
  const int32_t r0 = c0 + bw + blockIdx.y * blockDim.x;
  if (r0 >= N) return;
  double *P = a.panel + a.panel_off[s];
  for (int idx = threadIdx.x; idx < kBlock * kBlock; idx += blockDim.x) {
    const int i = idx / kBlock, j = idx % kBlock;
    Ls[i][j] = (i < bw && j < i) ? P[int64_t(c0 + j) * N + c0 + i] : 0.0;
  }
  if (threadIdx.x < kBlock) dk[threadIdx.x] = threadIdx.x < bw ? a.d[f + c0 + threadIdx.x] : 1.0;
  __syncthreads();
  const int32_t i = r0 + threadIdx.x;
  if (i >= N) return;
  double w[kBlock];
#pragma unroll
  for (int k = 0; k < kBlock; ++k) w[k] = k < bw ? P[int64_t(c0 + k) * N + i] : 0.0;
#pragma unroll
  for (int k = 0; k < kBlock; ++k) {
    double t = w[k];
#pragma unroll
    for (int j = 0; j < k; ++j) t = fma(-w[j], Ls[k][j], t);
    w[k] = t;
  }
#pragma unroll
  for (int k = 0; k < kBlock; ++k)
    if (k < bw) P[int64_t(c0 + k) * N + i] = w[k] / dk[k];
}

// Trailing update of block J: F[i, j] -= sum_k L[i, c0+k] d_k L[j, c0+k] for t0 <= j <= i < N,
// t0 = c0 + bw.  Column j < nc lives in the panel, j >= nc in the update matrix U_s.
__global__ void __launch_bounds__(256) k_trailing(const int32_t *__restrict__ sns, int32_t J,
                                                  const int64_t *__restrict__ prefix, int32_t na,
                                                  FactorArgs a) {
  __shared__ double Li[kBlock][kTile];
  __shared__ double Lj[kBlock][kTile];
  // locate the supernode of this tile
  const int64_t t = blockIdx.x;
  int32_t lo = 0, hi = na;   // prefix[lo] <= t < prefix[hi]
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) / 2;
    if (prefix[mid] <= t) lo = mid; else hi = mid;
  }
  const int32_t s = sns[lo];
  const int64_t lt = t - prefix[lo];
  int64_t ti = static_cast<int64_t>((sqrt(8.0 * double(lt) + 1.0) - 1.0) * 0.5);
  while (ti * (ti + 1) / 2 > lt) --ti;
  while ((ti + 1) * (ti + 2) / 2 <= lt) ++ti;
  const int64_t tj = lt - ti * (ti + 1) / 2;
  const int32_t f = a.first[s], nc = a.first[s + 1] - f, nbv = a.nb[s], N = nc + nbv;
  const int32_t c0 = J * kBlock, bw = min(kBlock, nc - c0), t0 = c0 + bw;
  const int32_t R0 = t0 + int32_t(ti) * kTile, C0 = t0 + int32_t(tj) * kTile;
  const double *P = a.panel + a.panel_off[s];
  for (int idx = threadIdx.x; idx < kBlock * kTile; idx += blockDim.x) {
    const int k = idx / kTile, r = idx % kTile;
    const bool kin = k < bw;
    Li[k][r] = (kin && R0 + r < N) ? P[int64_t(c0 + k) * N + R0 + r] : 0.0;
    Lj[k][r] = (kin && C0 + r < N) ? P[int64_t(c0 + k) * N + C0 + r] * a.d[f + c0 + k] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int k = 0; k < bw; ++k) {
    double li[4], lj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { li[u] = Li[k][tx + 16 * u]; lj[u] = Lj[k][ty + 16 * u]; }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fma(li[u], lj[v], acc[u][v]);
  }
  double *Pw = a.panel + a.panel_off[s];
  double *Uw = a.U + a.u_off[s];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int32_t j = C0 + ty + 16 * v;
    if (j >= N) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int32_t i = R0 + tx + 16 * u;
      if (i >= N || i < j) continue;
      if (j < nc)
        Pw[int64_t(j) * N + i] -= acc[u][v];
      else
        Uw[int64_t(j - nc) * nbv + (i - nc)] -= acc[u][v];
    }
  }
}

// Host driver: the full factorization on `stream`.  Returns a PEERS_* status.
int run_factor(const Symbolic &S, const FactorDevice &D, cudaStream_t stream, int64_t *launches,
               std::string &err, cudaEvent_t *level_events) {
  FactorArgs a = D.args;
  CUDA_TRY(cudaMemsetAsync(a.panel, 0, sizeof(double) * S.panel_total, stream));
  if (S.u_total > 0) CUDA_TRY(cudaMemsetAsync(a.U, 0, sizeof(double) * S.u_total, stream));
  CUDA_TRY(cudaMemsetAsync(a.status, 0, sizeof(int) * 2, stream));
  {
    const int64_t cnt = static_cast<int64_t>(S.a_dest.size());
    const int blocks = static_cast<int>(std::min<int64_t>((cnt + 255) / 256, 148 * 16));
    if (cnt > 0) {
      k_assemble<<<blocks, 256, 0, stream>>>(D.a_dest, D.a_val, cnt, a.panel);
      ++*launches;
    }
    CUDA_TRY(cudaGetLastError());
  }
  if (level_events) CUDA_TRY(cudaEventRecord(level_events[0], stream));
  for (int32_t l = 0; l < S.nlevels; ++l) {
    const int32_t *sns = D.level_sn + S.level_ptr[l];
    // 1. extend-add of the children, one launch per child rank
    for (int64_t r = S.ea_base[l]; r < S.ea_base[l + 1]; ++r) {
      const int64_t p0 = S.ea_off[r], p1 = S.ea_off[r + 1];
      if (p1 <= p0) continue;
      int32_t maxnb = 0;
      for (int64_t q = p0; q < p1; ++q) maxnb = std::max(maxnb, S.nb[S.ea_pairs[2 * q + 1]]);
      if (maxnb == 0) continue;
      dim3 grid(static_cast<unsigned>(p1 - p0), static_cast<unsigned>((maxnb + 7) / 8));
      k_extend_add<<<grid, 256, 0, stream>>>(D.ea_pairs + 2 * p0, a);
      ++*launches;
      CUDA_TRY(cudaGetLastError());
    }
    // 2. right-looking column blocks
    for (int32_t J = 0; J < S.level_nblocks[l]; ++J) {
      const int64_t tp = S.trail_base[l] + J;
      const int32_t na = static_cast<int32_t>(S.trail_na[tp]);
      if (na == 0) continue;
      k_diag_block<<<na, 32, 0, stream>>>(sns, J, a);
      ++*launches;
      CUDA_TRY(cudaGetLastError());
      int32_t maxrows = 0;
      for (int32_t i = 0; i < na; ++i) {
        const int32_t s = S.level_sn[S.level_ptr[l] + i];
        const int32_t nc = sn_nc(S, s), N = nc + S.nb[s];
        maxrows = std::max(maxrows, N - std::min(nc, (J + 1) * kBlock));
      }
      if (maxrows > 0) {
        dim3 grid(static_cast<unsigned>(na), static_cast<unsigned>((maxrows + 127) / 128));
        k_panel_rows<<<grid, 128, 0, stream>>>(sns, J, a);
        ++*launches;
        CUDA_TRY(cudaGetLastError());
      }
      const int64_t ntiles = S.trail_prefix[S.trail_off[tp] + na];
      if (ntiles > 0) {
        k_trailing<<<static_cast<unsigned>(ntiles), 256, 0, stream>>>(
            sns, J, D.trail_prefix + S.trail_off[tp], na, a);
        ++*launches;
        CUDA_TRY(cudaGetLastError());
      }
    }
    if (level_events) CUDA_TRY(cudaEventRecord(level_events[l + 1], stream));
  }
  int status[2] = {0, 0};
  CUDA_TRY(cudaMemcpyAsync(status, a.status, sizeof(status), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  if (status[0] == kErrNotSpd) {
    err = "non-positive pivot at elimination position " + std::to_string(status[1]);
    return PEERS_ENOTSPD;
  }
  return PEERS_OK;
}

}  // namespace peers
