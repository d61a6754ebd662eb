// Implicit inverse by elimination-tree blocks: the entries of Z = L^{-1} that the paper's
// row-wise traversal visits (§III-A/C, eq. 11; Lemma 1: Z[i, j] != 0 only for i an etree
// ancestor of j), computed block by block on the GPU and then combined per query:
//     R_st = sum_i (Z[i, s] - Z[i, t])^2 / d_i                  (eq. 12, eq. 18).
//
// Layout.  For supernode t with columns C_t, its block Z[P_t, C_t] holds the rows of the
// ancestor path P_t = C_t ++ C_parent ++ ... ++ C_root, column-major with ld = |P_t|.  Every
// non-zero of Z lives in exactly one block, and the block of an ancestor a of t occupies the
// last |P_a| rows of P_t (a suffix), which makes every gather a plain offset.
//
// Recurrence (from Z L = I, the column form of eq. 11):
//     Z[C_t, C_t]   = T_t^{-1}                          (unit-lower diagonal block of L)
//     Z[P_par, C_t] = -Z[P_par, B_t] * M_t,   M_t = L[B_t, C_t] * T_t^{-1}
// where column b of Z[P_par, B_t] is the block column of b's own supernode, zero above its
// suffix (a staircase: a row tile only needs the leading columns of B_t).  Phase 1 forms
// T_t^{-1} and M_t for every supernode at once; phase 2 walks the tree top-down, one launch
// per depth, every block of a depth from the (finished) blocks of its ancestors.  The query
// pass then reads, per query, the two stored columns along their paths.
//
// Work is sum_t |P_parent(t)| * n_b(t) * n_c(t) FMAs minus the staircase zeros, about 30x
// less than walking every query (the paper's Thm 4 order of work), for nnz(Z) of device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "device.cuh"
#include "handles.h"
#include "internal.h"
#include "peers.h"

namespace peers {
namespace {

constexpr int kT = 64;        // GEMM output tile (rows and columns)
constexpr int kK = 32;        // GEMM inner chunk
constexpr int kGemmThreads = 256;

struct BiArgs {
  const double *panel, *tinv, *dinv;
  const int32_t *first, *nb, *rows;
  const int64_t *panel_off, *tinv_off, *rows_off;
  const int64_t *zoff, *moff;      // block offsets of Z and M per supernode
  const int32_t *plen;             // |P_t|
  const int32_t *parent;
  const int32_t *gstart;           // per B_t entry: first row of its column within P_parent
  const int64_t *gsrc;             // per B_t entry: offset of its column in Z
  double *Z, *M;
  int *status;                     // error flag (bounds-checked build)
  int64_t ztotal, nq;              // extents of Z and of the results
};

// ---------------------------------------------------------------- phase 1a: T_t^{-1}

// One CTA per (supernode, 32-column block J, 8-column slice of it): those columns of T_t^{-1}
// by block forward substitution, X_I = inv(T_II) (E_IJ - sum_{J<=K<I} T_IK X_K), written to
// Z[C_t, cols].  A thread owns one row of a 32 x 8 output block: the warp's 32 rows read T
// coalesced, and the X_K value they share is one broadcast load.  Slicing J four ways cuts the
// longest CTA (the root's first block, whose substitution runs down all of C) to a quarter.
constexpr int kDiagSlice = 8;
constexpr int kDiagSlices = kBlock / kDiagSlice;

__global__ void __launch_bounds__(kBlock * kDiagSlice) k_bi_diag(const int32_t *__restrict__ sns,
                                                                 const int32_t *__restrict__ blk,
                                                                 BiArgs a) {
  __shared__ double Ti[kBlock][kBlock + 1];
  __shared__ double acc[kBlock][kDiagSlice + 1];
  const int32_t t = sns[blockIdx.x];
  const int32_t J = blk[blockIdx.x] / kDiagSlices, sl = blk[blockIdx.x] % kDiagSlices;
  const int32_t nc = a.first[t + 1] - a.first[t], N = nc + a.nb[t];
  const int32_t ld = a.plen[t];
  const double *P = a.panel + a.panel_off[t];
  double *Zt = a.Z + a.zoff[t];
  // the supernode's panel, block inverses and block of Z hold what this CTA touches
  if (!PEERS_IN(int64_t(nc) * N - 1, a.panel_off[t + 1] - a.panel_off[t], a.status) ||
      !PEERS_IN(int64_t(nc - 1) * ld + nc - 1, a.zoff[t + 1] - a.zoff[t], a.status) ||
      !PEERS_IN(a.tinv_off[t + 1] - a.tinv_off[t] - 1, a.tinv_off[t + 1] - a.tinv_off[t], a.status))
    return;
  const int c0 = J * kBlock;                        // the block's first column
  const int s0 = c0 + sl * kDiagSlice;              // this slice's first column
  const int sw = min(kDiagSlice, nc - s0);          // columns in the slice
  const int nblk = (nc + kBlock - 1) / kBlock;
  const int i = threadIdx.x % kBlock, j = threadIdx.x / kBlock;
  for (int I = J; I < nblk; ++I) {
    const int r0 = I * kBlock, bwI = min(kBlock, nc - r0);
    // acc = E_IJ - sum_K T[I rows, K cols] X_K   (X_K = Z[K rows, slice], already written)
    double s = 0.0;
    if (i < bwI && j < sw) {
      s = (r0 + i == s0 + j) ? 1.0 : 0.0;
      const double *Tp = P + r0 + i;
      const double *Xp = Zt + int64_t(s0 + j) * ld;
      // X[k, s0 + j] is zero above the slice's own rows (k < s0 + j): start there
      int k = s0 + j;
      for (; k + 4 <= r0; k += 4) {
        const double t0 = Tp[int64_t(k) * N], t1 = Tp[int64_t(k + 1) * N];
        const double t2 = Tp[int64_t(k + 2) * N], t3 = Tp[int64_t(k + 3) * N];
        const double x0 = Xp[k], x1 = Xp[k + 1], x2 = Xp[k + 2], x3 = Xp[k + 3];
        s = fma(-t0, x0, s);
        s = fma(-t1, x1, s);
        s = fma(-t2, x2, s);
        s = fma(-t3, x3, s);
      }
      for (; k < r0; ++k) s = fma(-Tp[int64_t(k) * N], Xp[k], s);
    }
    acc[i][j] = s;
    const double *TI = a.tinv + a.tinv_off[t] + int64_t(I) * kBlock * kBlock;
    for (int e = threadIdx.x; e < kBlock * kBlock; e += blockDim.x) {
      const int ii = e / kBlock, jj = e % kBlock;
      Ti[ii][jj] = (ii < bwI && jj < bwI) ? TI[ii * bwI + jj] : 0.0;
    }
    __syncthreads();
    if (i < bwI && j < sw) {
      double y = 0.0;
      for (int k = 0; k <= i; ++k) y = fma(Ti[i][k], acc[k][j], y);
      Zt[int64_t(s0 + j) * ld + r0 + i] = y;
    }
    __syncthreads();
  }
}

// Phase 1 for supernodes of at most 32 columns (one diagonal block): Z[C_t, C_t] is the
// block inverse the factorization already formed, and M_t = L[B_t, C_t] T_t^{-1} takes one
// row per thread.  grid = (supernode, chunk of 256 rows of B_t).
__global__ void __launch_bounds__(256) k_bi_small(const int32_t *__restrict__ sns,
                                                  const int32_t *__restrict__ chunk, BiArgs a) {
  __shared__ double Ti[kBlock][kBlock + 1];
  const int32_t t = sns[blockIdx.x], ch = chunk[blockIdx.x];
  const int32_t nc = a.first[t + 1] - a.first[t], nbv = a.nb[t], N = nc + nbv;
  const double *TI = a.tinv + a.tinv_off[t];
  if (!PEERS_IN(int64_t(nc) * nc - 1, a.tinv_off[t + 1] - a.tinv_off[t], a.status) ||
      !PEERS_IN(int64_t(nc) * N - 1, a.panel_off[t + 1] - a.panel_off[t], a.status) ||
      !PEERS_IN(int64_t(nc - 1) * a.plen[t] + nc - 1, a.zoff[t + 1] - a.zoff[t], a.status) ||
      !(nbv == 0 || PEERS_IN(int64_t(nbv) * nc - 1, a.moff[t + 1] - a.moff[t], a.status)))
    return;
  for (int e = threadIdx.x; e < kBlock * kBlock; e += blockDim.x) {
    const int i = e / kBlock, j = e % kBlock;
    Ti[i][j] = (i < nc && j < nc) ? TI[i * nc + j] : 0.0;
  }
  __syncthreads();
  if (ch == 0) {
    double *Zt = a.Z + a.zoff[t];
    const int32_t ld = a.plen[t];
    for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
      const int i = e % nc, j = e / nc;
      Zt[int64_t(j) * ld + i] = Ti[i][j];
    }
  }
  const int i = ch * 256 + threadIdx.x;
  if (i >= nbv) return;
  const double *P = a.panel + a.panel_off[t];
  double p[kBlock];
#pragma unroll
  for (int k = 0; k < kBlock; ++k) p[k] = k < nc ? P[int64_t(k) * N + nc + i] : 0.0;
  double *Mrow = a.M + a.moff[t] + int64_t(i) * nc;
#pragma unroll
  for (int c = 0; c < kBlock; ++c) {
    if (c >= nc) break;
    double m = 0.0;
#pragma unroll
    for (int k = 0; k < kBlock; ++k)
      if (k >= c) m = fma(p[k], Ti[k][c], m);
    Mrow[c] = m;
  }
}

// ---------------------------------------------------------------- GEMM tiles

// Tile descriptor: supernode, row tile, column tile.
struct Tile {
  int32_t t, r, c, pad;
};

// ---------------------------------------------------------------- row-per-thread products
//
// out(i, c) = (+/-) sum_{k = kb}^{ke-1} A[k * lda + i] * B(k, c) for the rows i of one chunk
// and the columns [c0, c0 + W) of one chunk: one row per thread with its W sums in registers,
// B staged in shared memory kRowsK rows at a time, A read coalesced across the warp.  The
// products on this path are tall and narrow (hundreds to thousands of rows, a few to a few
// tens of columns), where square tiles would spend most of their multiply-adds on padding.
// Each sum runs in increasing k, so a result does not depend on the chunking.
// Tile = (block, row chunk, c0, W).
constexpr int kRowsMaxThreads = 128;
constexpr int kRowsK = 64;
constexpr int kRowsMaxW = 64;

struct RowsGemm {
  const double *A;
  int64_t lda;            // A[k * lda + i]
  const double *B;
  int64_t bk, bc;         // B(k, c) = B[k * bk + c * bc]
  double *out;
  int64_t oi, oc;         // out(i, c) = out[i * oi + c * oc]
  int32_t nrows, kb, ke, ncols;
  bool negate;
  // extents of A, B and out from their pointers, and the error flag (bounds-checked build)
  int64_t a_ext, b_ext, o_ext;
  int *status;
};

template <int W>
__device__ __forceinline__ void rows_gemm(const RowsGemm &g, int r, int c0, int rows, double *Ms) {
  const int wn = min(W, g.ncols - c0);
  const int i = r * rows + threadIdx.x;
#if defined(PEERS_BOUNDS) && PEERS_BOUNDS
  // the largest index of each operand this tile reads or writes lies inside its extent
  if (g.ke > g.kb && g.nrows > 0 &&
      (!PEERS_IN(int64_t(g.ke - 1) * g.lda + g.nrows - 1, g.a_ext, g.status) ||
       !PEERS_IN(int64_t(g.ke - 1) * g.bk + int64_t(g.ncols - 1) * g.bc, g.b_ext, g.status) ||
       !PEERS_IN(int64_t(g.nrows - 1) * g.oi + int64_t(g.ncols - 1) * g.oc, g.o_ext, g.status)))
    return;
#endif
  double acc[W];
#pragma unroll
  for (int c = 0; c < W; ++c) acc[c] = 0.0;
  for (int k0 = g.kb; k0 < g.ke; k0 += kRowsK) {
    const int kn = min(kRowsK, g.ke - k0);
    for (int e = threadIdx.x; e < kRowsK * W; e += rows) {
      // read B along whichever of its two dimensions is contiguous
      int kk, c;
      if (g.bk == 1) { c = e / kRowsK; kk = e - c * kRowsK; }
      else { kk = e / W; c = e - kk * W; }
      Ms[kk * W + c] = (kk < kn && c < wn) ? g.B[int64_t(k0 + kk) * g.bk + int64_t(c0 + c) * g.bc]
                                           : 0.0;
    }
    __syncthreads();
    if (i < g.nrows) {
      const double *Ak = g.A + int64_t(k0) * g.lda + i;
      int kk = 0;
      // four loads in flight before their multiply-adds (narrow chunks are latency bound)
      for (; kk + 4 <= kn; kk += 4) {
        const double g0 = Ak[int64_t(kk) * g.lda], g1 = Ak[int64_t(kk + 1) * g.lda];
        const double g2 = Ak[int64_t(kk + 2) * g.lda], g3 = Ak[int64_t(kk + 3) * g.lda];
        const double *m = Ms + kk * W;
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = fma(g0, m[c], acc[c]);
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = fma(g1, m[W + c], acc[c]);
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = fma(g2, m[2 * W + c], acc[c]);
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = fma(g3, m[3 * W + c], acc[c]);
      }
      for (; kk < kn; ++kk) {
        const double a0 = Ak[int64_t(kk) * g.lda];
#pragma unroll
        for (int c = 0; c < W; ++c) acc[c] = fma(a0, Ms[kk * W + c], acc[c]);
      }
    }
    __syncthreads();
  }
  if (i < g.nrows) {
#pragma unroll
    for (int c = 0; c < W; ++c)
      if (c < wn) g.out[int64_t(i) * g.oi + int64_t(c0 + c) * g.oc] = g.negate ? -acc[c] : acc[c];
  }
}

// Chunk widths, in three groups compiled as separate kernels so that narrow chunks are not
// held to the register count of the widest: group 0 = 1..8, group 1 = 12..32, group 2 = 48..64.
inline int rows_width(int32_t cols) {
  constexpr int kW[] = {1, 2, 4, 8, 12, 16, 24, 32, 48, 64};
  for (int w : kW)
    if (cols <= w) return w;
  return kRowsMaxW;
}
inline int rows_group(int w) { return w <= 8 ? 0 : w <= 32 ? 1 : 2; }
__host__ __device__ constexpr int rows_group_width(int g) { return g == 0 ? 8 : g == 1 ? 32 : kRowsMaxW; }

template <int G>
__device__ __forceinline__ void rows_gemm_dispatch(const RowsGemm &g, const Tile &tl, int rows,
                                                   double *Ms) {
  if (G == 0) {
    switch (tl.pad) {
      case 1: rows_gemm<1>(g, tl.r, tl.c, rows, Ms); break;
      case 2: rows_gemm<2>(g, tl.r, tl.c, rows, Ms); break;
      case 4: rows_gemm<4>(g, tl.r, tl.c, rows, Ms); break;
      default: rows_gemm<8>(g, tl.r, tl.c, rows, Ms); break;
    }
  } else if (G == 1) {
    switch (tl.pad) {
      case 12: rows_gemm<12>(g, tl.r, tl.c, rows, Ms); break;
      case 16: rows_gemm<16>(g, tl.r, tl.c, rows, Ms); break;
      case 24: rows_gemm<24>(g, tl.r, tl.c, rows, Ms); break;
      default: rows_gemm<32>(g, tl.r, tl.c, rows, Ms); break;
    }
  } else {
    if (tl.pad == 48) rows_gemm<48>(g, tl.r, tl.c, rows, Ms);
    else rows_gemm<64>(g, tl.r, tl.c, rows, Ms);
  }
}

// Phase 1b: M_t = L[B_t, C_t] * Z[C_t, C_t] (row-major n_b x n_c) by the row-per-thread
// product.  Z[C_t, C_t] = T_t^{-1} is lower triangular, so a column chunk starting at c0 only
// needs k >= c0 (the entries above the diagonal are stored zeros).
constexpr int kMRows = 64;
// Column chunk of M's tiles: 16 rather than the widest 64, so that a tile (64 x 16 over up to
// n_c terms) holds its SM for a short time; the tiles of a low-priority stream then do not
// keep the critical path's launches waiting for long.
constexpr int kMWidth = 16;
template <int G>
__global__ void __launch_bounds__(kRowsMaxThreads) k_bi_m(const Tile *__restrict__ tiles, BiArgs a) {
  __shared__ double Ms[kRowsK * rows_group_width(G)];
  const Tile tl = tiles[blockIdx.x];
  const int32_t t = tl.t;
  const int32_t nc = a.first[t + 1] - a.first[t], nbv = a.nb[t], N = nc + nbv;
  RowsGemm g;
  g.A = a.panel + a.panel_off[t] + nc;
  g.lda = N;
  g.B = a.Z + a.zoff[t];
  g.bk = 1;
  g.bc = a.plen[t];
  g.out = a.M + a.moff[t];
  g.oi = nc;
  g.oc = 1;
  g.nrows = nbv;
  g.kb = tl.c;
  g.ke = nc;
  g.ncols = nc;
  g.negate = false;
  g.a_ext = a.panel_off[t + 1] - a.panel_off[t] - nc;
  g.b_ext = a.zoff[t + 1] - a.zoff[t];
  g.o_ext = a.moff[t + 1] - a.moff[t];
  g.status = a.status;
  rows_gemm_dispatch<G>(g, tl, kMRows, Ms);
}

// The tiles of M_t for every wide supernode, grouped by width, the largest products first
// (the launch's last wave then holds only small ones).
inline void m_tiles_of(const Symbolic &S, const std::vector<int32_t> &wide,
                       std::vector<Tile> &tiles, std::vector<int64_t> &ptr) {
  std::vector<Tile> grp[3];
  for (int32_t t : wide) {
    const int32_t nc = sn_nc(S, t), nbv = S.nb[t];
    for (int32_t r = 0; r * kMRows < nbv; ++r)
      for (int32_t c0 = 0; c0 < nc; c0 += kMWidth) {
        const int w = rows_width(std::min(kMWidth, nc - c0));
        grp[rows_group(w)].push_back({t, r, c0, w});
      }
  }
  tiles.clear();
  ptr.assign(1, 0);
  for (auto &g : grp) {
    std::stable_sort(g.begin(), g.end(), [&](const Tile &x, const Tile &y) {
      return int64_t(sn_nc(S, x.t) - x.c) * x.pad > int64_t(sn_nc(S, y.t) - y.c) * y.pad;
    });
    tiles.insert(tiles.end(), g.begin(), g.end());
    ptr.push_back(static_cast<int64_t>(tiles.size()));
  }
}

template <int G>
int launch_m(const Tile *d_tiles, const std::vector<int64_t> &ptr, const BiArgs &a,
             cudaStream_t st, int64_t *launches, std::string &err) {
  const int64_t n = ptr[G + 1] - ptr[G];
  if (n <= 0) return PEERS_OK;
  k_bi_m<G><<<static_cast<unsigned>(n), kMRows, 0, st>>>(d_tiles + ptr[G], a);
  ++*launches;
  CUDA_TRY(cudaGetLastError());
  return PEERS_OK;
}
int launch_m_all(const Tile *d_tiles, const std::vector<int64_t> &ptr, const BiArgs &a,
                 cudaStream_t st, int64_t *launches, std::string &err) {
  int rc = launch_m<0>(d_tiles, ptr, a, st, launches, err);
  if (rc == PEERS_OK) rc = launch_m<1>(d_tiles, ptr, a, st, launches, err);
  if (rc == PEERS_OK) rc = launch_m<2>(d_tiles, ptr, a, st, launches, err);
  return rc;
}

// ---------------------------------------------------------------- T^{-1} by doubling
//
// For a wide supernode (n_c > kBlock) the inverse X = T^{-1} of its unit-lower diagonal block
// is built from the factor's 32 x 32 diagonal-block inverses by doubling.  At level l (blocks
// of s = 32 * 2^l columns) each pair of adjacent inverted diagonal blocks A = T[a, a] and
// C = T[c, c] (c = a + s) with coupling B = T[c, a] gives the inverse of the 2s block:
//     X[c, a] = -C^{-1} (B A^{-1}),
// formed by two row-per-thread products, W = B A^{-1} (A^{-1} lower triangular: only
// k >= col contributes) and then X[c, a] = -C^{-1} W (C^{-1} lower triangular: k <= row).
// The pairs of one level, over every wide supernode of a list, share one launch per product,
// so the critical path is log2(n_c / 32) levels of well-filled launches rather than one
// CTA's block substitution down all n_c rows.  W is kept in a buffer laid out like X.
struct TinvTile {
  int32_t t;          // supernode
  int32_t a0, c0;     // first columns of A and of C
  int32_t ha, hc;     // their widths
  int32_t r;          // row chunk of the product (rows of C, kTinvRows each)
  int32_t col0, w;    // first column (of A) of the tile and its width (rows_width)
};
constexpr int kTinvRows = 32;
constexpr int kTinvWidth = 8;    // columns per doubling tile (short CTAs, many per SM)
// Supernodes at least this wide form T^{-1} by doubling; narrower ones by k_bi_diag's block
// substitution, whose single launch beats the doubling's launch chain there.
constexpr int32_t kTinvDoubling = 1024;

// X's 32 x 32 diagonal blocks from the factor's block inverses.  grid = (supernode, block).
__global__ void __launch_bounds__(256) k_tinv_base(const int32_t *__restrict__ sns,
                                                   const int32_t *__restrict__ blk, BiArgs a) {
  const int32_t t = sns[blockIdx.x], J = blk[blockIdx.x];
  const int32_t nc = a.first[t + 1] - a.first[t], ld = a.plen[t];
  const int32_t c0 = J * kBlock, bw = min(kBlock, nc - c0);
  if (!PEERS_IN(int64_t(J) * kBlock * kBlock + bw * bw - 1, a.tinv_off[t + 1] - a.tinv_off[t],
                a.status) ||
      !PEERS_IN(int64_t(c0 + bw - 1) * ld + c0 + bw - 1, a.zoff[t + 1] - a.zoff[t], a.status))
    return;
  const double *TI = a.tinv + a.tinv_off[t] + int64_t(J) * kBlock * kBlock;
  double *X = a.Z + a.zoff[t];
  for (int e = threadIdx.x; e < bw * bw; e += blockDim.x) {
    const int i = e % bw, j = e / bw;
    X[int64_t(c0 + j) * ld + c0 + i] = i >= j ? TI[i * bw + j] : 0.0;
  }
}

// One product of a doubling level: PHASE 0 forms W = B A^{-1}, PHASE 1 forms
// X[c, a] = -C^{-1} W (see above), for the tile's rows and columns.
template <int G, int PHASE>
__global__ void __launch_bounds__(kRowsMaxThreads) k_tinv_gemm(const TinvTile *__restrict__ tiles,
                                                               BiArgs a, double *Wd) {
  __shared__ double Ms[kRowsK * rows_group_width(G)];
  const TinvTile tl = tiles[blockIdx.x];
  const int32_t t = tl.t;
  const int32_t nc = a.first[t + 1] - a.first[t], N = nc + a.nb[t];
  const int32_t ld = a.plen[t];
  double *X = a.Z + a.zoff[t];
  double *Wt = Wd + a.zoff[t];
  const int64_t xext = a.zoff[t + 1] - a.zoff[t];
  RowsGemm g;
  if (PHASE == 0) {
    g.A = a.panel + a.panel_off[t] + int64_t(tl.a0) * N + tl.c0;
    g.lda = N;
    g.B = X + int64_t(tl.a0) * ld + tl.a0;
    g.kb = tl.col0;
    g.ke = tl.ha;
    g.negate = false;
    g.a_ext = a.panel_off[t + 1] - a.panel_off[t] - (int64_t(tl.a0) * N + tl.c0);
  } else {
    g.A = X + int64_t(tl.c0) * ld + tl.c0;
    g.lda = ld;
    g.B = Wt + int64_t(tl.a0) * ld + tl.c0;
    g.kb = 0;
    g.ke = min(tl.hc, (tl.r + 1) * kTinvRows);
    g.negate = true;
    g.a_ext = xext - (int64_t(tl.c0) * ld + tl.c0);
  }
  g.bk = 1;
  g.bc = ld;
  g.out = (PHASE == 0 ? Wt : X) + int64_t(tl.a0) * ld + tl.c0;
  g.oi = 1;
  g.oc = ld;
  g.nrows = tl.hc;
  g.ncols = tl.ha;
  g.b_ext = xext - (int64_t(tl.a0) * ld + (PHASE == 0 ? tl.a0 : tl.c0));
  g.o_ext = xext - (int64_t(tl.a0) * ld + tl.c0);
  g.status = a.status;
  rows_gemm_dispatch<G>(g, Tile{t, tl.r, tl.col0, tl.w}, kTinvRows, Ms);
}

// The doubling plan of a list of wide supernodes: base blocks, then per level the tiles of
// both products, grouped by width group (ptr: per level, 3 groups + 1 entries).
struct TinvPlan {
  std::vector<int32_t> base_sn, base_blk;
  std::vector<TinvTile> tiles;
  std::vector<std::vector<int64_t>> level_ptr;   // per level: 4 offsets into tiles
};

inline void tinv_plan_of(const Symbolic &S, const std::vector<int32_t> &wide, TinvPlan &T,
                         std::vector<TinvTile> &all) {
  for (int32_t t : wide)
    for (int32_t J = 0; J * kBlock < sn_nc(S, t); ++J) {
      T.base_sn.push_back(t);
      T.base_blk.push_back(J);
    }
  for (int32_t s = kBlock;; s *= 2) {
    std::vector<TinvTile> grp[3];
    bool any = false;
    for (int32_t t : wide) {
      const int32_t nc = sn_nc(S, t);
      for (int32_t a0 = 0; a0 + s < nc; a0 += 2 * s) {
        any = true;
        const int32_t c0 = a0 + s, ha = s, hc = std::min(s, nc - c0);
        for (int32_t r = 0; r * kTinvRows < hc; ++r)
          for (int32_t col0 = 0; col0 < ha; col0 += kTinvWidth) {
            const int w = rows_width(std::min(kTinvWidth, ha - col0));
            grp[rows_group(w)].push_back({t, a0, c0, ha, hc, r, col0, w});
          }
      }
    }
    if (!any) break;
    std::vector<int64_t> ptr;
    ptr.push_back(static_cast<int64_t>(all.size()));
    for (auto &g : grp) {
      all.insert(all.end(), g.begin(), g.end());
      ptr.push_back(static_cast<int64_t>(all.size()));
    }
    T.level_ptr.push_back(ptr);
  }
}

template <int PHASE>
int launch_tinv_level(const TinvTile *d_tiles, const std::vector<int64_t> &ptr, const BiArgs &a,
                      double *Wd, cudaStream_t st, int64_t *launches, std::string &err) {
  for (int g = 0; g < 2; ++g) {   // widths never exceed 32: groups 0 and 1
    const int64_t n = ptr[g + 1] - ptr[g];
    if (n <= 0) continue;
    if (g == 0)
      k_tinv_gemm<0, PHASE><<<static_cast<unsigned>(n), kTinvRows, 0, st>>>(d_tiles + ptr[g], a, Wd);
    else
      k_tinv_gemm<1, PHASE><<<static_cast<unsigned>(n), kTinvRows, 0, st>>>(d_tiles + ptr[g], a, Wd);
    ++*launches;
    CUDA_TRY(cudaGetLastError());
  }
  return PEERS_OK;
}

// Phase 2: Z[P_par, C_t] = -Z[P_par, B_t] * M_t for the supernodes of one depth, in tiles of
// TS x TS (TS = 16, 32 or 64 in Tile.pad, chosen per depth so that the launch has enough
// CTAs).  Row tile r covers rows [TS r, TS r + TS) of P_par; only the columns of B_t whose
// staircase starts above the tile's last row contribute (a prefix of B_t, found by binary
// search).  Every output sums over k in increasing order whatever TS is.
template <int TS>
__device__ __forceinline__ void bi_z_tile(const Tile &tl, const BiArgs &a, double *As, double *Bs,
                                          int32_t *sst, int64_t *ssrc, int32_t *kend_s) {
  constexpr int U = TS / 16;
  const int32_t t = tl.t;
  const int32_t nc = a.first[t + 1] - a.first[t], nbv = a.nb[t];
  const int32_t ldt = a.plen[t], lp = ldt - nc;   // |P_par|
  const int R0 = tl.r * TS, C0 = tl.c * TS;
  const int32_t *gs = a.gstart + a.rows_off[t];
  const int64_t *gsrc = a.gsrc + a.rows_off[t];
  if (threadIdx.x == 0) {   // first B_t column whose staircase starts at or below row R0+TS
    int lo = 0, hi = nbv;
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (gs[mid] < R0 + TS) lo = mid + 1; else hi = mid;
    }
    *kend_s = lo;
  }
  __syncthreads();
  const int32_t kend = *kend_s;
  const double *Mt = a.M + a.moff[t];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[U][U] = {};
  for (int k0 = 0; k0 < kend; k0 += kK) {
    if (threadIdx.x < kK) {
      const int kk = k0 + threadIdx.x;
      sst[threadIdx.x] = kk < kend ? gs[kk] : INT32_MAX;
      ssrc[threadIdx.x] = kk < kend ? gsrc[kk] : 0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kK * TS; e += kGemmThreads) {
      const int k = e / TS, r = e - (e / TS) * TS;
      const int kk = k0 + k;
      double g = 0.0, m = 0.0;
      if (kk < kend) {
        const int row = R0 + r;
        const int32_t st = sst[k];
        if (row < lp && row >= st && PEERS_IN(ssrc[k] + (row - st), a.ztotal, a.status))
          g = a.Z[ssrc[k] + (row - st)];
        if (C0 + r < nc) m = Mt[int64_t(kk) * nc + C0 + r];
      }
      As[k * TS + r] = g;
      Bs[k * TS + r] = m;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kK; ++k) {
      double av[U], bv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) { av[u] = As[k * TS + tx + 16 * u]; bv[u] = Bs[k * TS + ty + 16 * u]; }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
  double *Zt = a.Z + a.zoff[t];
#pragma unroll
  for (int v = 0; v < U; ++v) {
    const int j = C0 + ty + 16 * v;
    if (j >= nc) continue;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = R0 + tx + 16 * u;
      if (i < lp && PEERS_IN(int64_t(j) * ldt + nc + i, a.zoff[t + 1] - a.zoff[t], a.status))
        Zt[int64_t(j) * ldt + nc + i] = -acc[u][v];
    }
  }
}

__global__ void __launch_bounds__(kGemmThreads) k_bi_z(const Tile *__restrict__ tiles, BiArgs a) {
  __shared__ double As[kK * kT];
  __shared__ double Bs[kK * kT];
  __shared__ int32_t sst[kK];
  __shared__ int64_t ssrc[kK];
  __shared__ int32_t kend_s;
  const Tile tl = tiles[blockIdx.x];
  switch (tl.pad) {
    case 16: bi_z_tile<16>(tl, a, As, Bs, sst, ssrc, &kend_s); break;
    case 32: bi_z_tile<32>(tl, a, As, Bs, sst, ssrc, &kend_s); break;
    default: bi_z_tile<kT>(tl, a, As, Bs, sst, ssrc, &kend_s); break;
  }
}

// Phase 2 for narrow supernodes (n_c <= NC): one output row of Z[P_par, C_t] per thread, all
// n_c columns in registers; rows of M_t and the staircase of B_t staged in shared memory.
constexpr int kNarrowRows = 256;
constexpr int kNarrowK = 64;

template <int NC>
__device__ __forceinline__ void bi_z_narrow(const Tile &tl, const BiArgs &a, double *sm) {
  double *Ms = sm;                                              // kNarrowK x NC
  int32_t *gss = reinterpret_cast<int32_t *>(Ms + kNarrowK * NC);   // kNarrowK
  int64_t *gsr = reinterpret_cast<int64_t *>(gss + kNarrowK);       // kNarrowK
  __shared__ int32_t kend_s;
  const int32_t t = tl.t;
  const int32_t nc = a.first[t + 1] - a.first[t], nbv = a.nb[t];
  const int32_t ldt = a.plen[t], lp = ldt - nc;
  const int R0 = tl.r * kNarrowRows;
  const int32_t *gs = a.gstart + a.rows_off[t];
  const int64_t *gsrc = a.gsrc + a.rows_off[t];
  if (threadIdx.x == 0) {
    int lo = 0, hi = nbv;
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (gs[mid] < R0 + kNarrowRows) lo = mid + 1; else hi = mid;
    }
    kend_s = lo;
  }
  __syncthreads();
  const int32_t kend = kend_s;
  const double *Mt = a.M + a.moff[t];
  const int i = R0 + threadIdx.x;
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int k0 = 0; k0 < kend; k0 += kNarrowK) {
    const int kn = min(kNarrowK, kend - k0);
    for (int e = threadIdx.x; e < kNarrowK * NC; e += blockDim.x) {
      const int kk = e / NC, c = e % NC;
      Ms[e] = (kk < kn && c < nc) ? Mt[int64_t(k0 + kk) * nc + c] : 0.0;
    }
    for (int kk = threadIdx.x; kk < kNarrowK; kk += blockDim.x) {
      gss[kk] = kk < kn ? gs[k0 + kk] : INT32_MAX;
      gsr[kk] = kk < kn ? gsrc[k0 + kk] : 0;
    }
    __syncthreads();
    if (i < lp) {
      // the chunk's columns that reach row i: a prefix, since later columns start further
      // down (the staircase); their Z entries are loaded four at a time, so that several
      // loads are in flight before their multiply-adds, which keep increasing kk per column
      int lo = 0, hi = kn;
      while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (gss[mid] <= i) lo = mid + 1; else hi = mid;
      }
      const int kv = lo;
      auto zval = [&](int kk) -> double {
        const int64_t z = gsr[kk] + (i - gss[kk]);
        return PEERS_IN(z, a.ztotal, a.status) ? a.Z[z] : 0.0;
      };
      int kk = 0;
      for (; kk + 4 <= kv; kk += 4) {
        const double g0 = zval(kk), g1 = zval(kk + 1), g2 = zval(kk + 2), g3 = zval(kk + 3);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fma(g0, Ms[kk * NC + c], acc[c]);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fma(g1, Ms[(kk + 1) * NC + c], acc[c]);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fma(g2, Ms[(kk + 2) * NC + c], acc[c]);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fma(g3, Ms[(kk + 3) * NC + c], acc[c]);
      }
      for (; kk < kv; ++kk) {
        const double g = zval(kk);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fma(g, Ms[kk * NC + c], acc[c]);
      }
    }
    __syncthreads();
  }
  if (i < lp) {
    double *Zt = a.Z + a.zoff[t];
#pragma unroll
    for (int c = 0; c < NC; ++c)
      if (c < nc && PEERS_IN(int64_t(c) * ldt + nc + i, a.zoff[t + 1] - a.zoff[t], a.status))
        Zt[int64_t(c) * ldt + nc + i] = -acc[c];
  }
}

// Narrow tiles of one depth; Tile.pad selects the register width.  Two kernels, so that the
// narrowest chunks are not held to the register count of the widest: group 0 = 1, 2, 4, 8
// columns, group 1 = 12, 16, 24, 32.
template <int G>
__global__ void __launch_bounds__(kNarrowRows) k_bi_z_narrow(const Tile *__restrict__ tiles,
                                                             BiArgs a) {
  extern __shared__ double sm[];
  const Tile tl = tiles[blockIdx.x];
  if (G == 0) {
    switch (tl.pad) {
      case 1: bi_z_narrow<1>(tl, a, sm); break;
      case 2: bi_z_narrow<2>(tl, a, sm); break;
      case 4: bi_z_narrow<4>(tl, a, sm); break;
      default: bi_z_narrow<8>(tl, a, sm); break;
    }
  } else {
    switch (tl.pad) {
      case 12: bi_z_narrow<12>(tl, a, sm); break;
      case 16: bi_z_narrow<16>(tl, a, sm); break;
      case 24: bi_z_narrow<24>(tl, a, sm); break;
      default: bi_z_narrow<32>(tl, a, sm); break;
    }
  }
}

inline int narrow_width(int32_t nc) {
  return nc <= 1 ? 1 : nc <= 2 ? 2 : nc <= 4 ? 4 : nc <= 8 ? 8 : nc <= 12 ? 12
         : nc <= 16 ? 16 : nc <= 24 ? 24 : 32;
}
constexpr size_t narrow_smem(int group) {
  return size_t(kNarrowK) * (group == 0 ? 8 : 32) * 8 + kNarrowK * 4 + kNarrowK * 8;
}

// ---------------------------------------------------------------- query pass

struct BiQuery {
  int32_t s1, j1;   // supernode and local column of the first endpoint's Z column
  int32_t s2, j2;   // the second (s2 = -1: none, the pair touches the ground)
  int64_t out;      // index in R
};

// One warp per query: R = sum over P_s1 \ P_m of z1^2/d + over P_s2 \ P_m of z2^2/d + over
// P_m of (z1 - z2)^2/d, m = the lowest common supernode of s1 and s2 (s2 itself for an edge).
// A column z_s of Z holds the rows of the path P_s in order, supernode after supernode, so the
// three sums run over contiguous row ranges: the branch of s1 is z1[0, L1), that of s2 is
// z2[0, L2), and the common part pairs z1[L1 + c] with z2[L2 + c] (L = plen[s] - plen[m]).
// The warp first walks each path once into a list of (first column, start row) per
// supernode in shared memory; then every lane takes rows k = lane, lane + 32, ... and loads
// four rows' entries before their multiply-adds, so that the column's loads overlap instead
// of waiting one supernode at a time.  Paths longer than kQueryPath supernodes take the
// supernode-by-supernode walk.
constexpr int kQueryPath = 128;
constexpr int kQueryWarps = 8;   // warps per CTA (256 threads)

// The path of s up to (not including) stop: per supernode its first column and start row.
__device__ __forceinline__ int bi_path_list(const BiArgs &a, int32_t s, int32_t stop,
                                            int32_t *seg_f, int32_t *seg_o, int lane) {
  int n = 0;
  for (int32_t x = s; x != stop && x >= 0; x = a.parent[x]) {
    if (n == kQueryPath) return -1;
    if (lane == 0) {
      seg_f[n] = a.first[x];
      seg_o[n] = a.plen[s] - a.plen[x];
    }
    ++n;
  }
  __syncwarp();
  return n;
}

// sum over rows k in [k0, k1) of (za[k] - zb[k - shift])^2 * dinv[col(k)] (zb = nullptr: no
// zb term), col(k) = seg_f[i] + k - seg_o[i] for the path segment i holding row k (relative
// to the list's base row `base`).
__device__ __forceinline__ double bi_rows_sum(const BiArgs &a, const double *za, const double *zb,
                                              int64_t shift, int32_t k0, int32_t k1,
                                              const int32_t *seg_f, const int32_t *seg_o,
                                              int nseg, int32_t base, int lane) {
  double acc = 0.0;
  int i = 0;   // segment of the lane's current row, advancing with it
  auto term = [&](int32_t k, double &v, int32_t &col) {
    while (i + 1 < nseg && seg_o[i + 1] + base <= k) ++i;
    col = seg_f[i] + (k - base - seg_o[i]);
    v = za[k] - (zb ? zb[k - shift] : 0.0);
  };
  int32_t k = k0 + lane;
  for (; k + 96 < k1; k += 128) {
    double v0, v1, v2, v3;
    int32_t c0, c1, c2, c3;
    term(k, v0, c0);
    term(k + 32, v1, c1);
    term(k + 64, v2, c2);
    term(k + 96, v3, c3);
    acc = fma(v0 * v0, a.dinv[c0], acc);
    acc = fma(v1 * v1, a.dinv[c1], acc);
    acc = fma(v2 * v2, a.dinv[c2], acc);
    acc = fma(v3 * v3, a.dinv[c3], acc);
  }
  for (; k < k1; k += 32) {
    double v;
    int32_t c;
    term(k, v, c);
    acc = fma(v * v, a.dinv[c], acc);
  }
  return acc;
}

__global__ void __launch_bounds__(32 * kQueryWarps) k_bi_query(const BiQuery *__restrict__ qs,
                                                                int64_t nq, BiArgs a, double *R) {
  __shared__ int32_t seg_f[kQueryWarps][2][kQueryPath];
  __shared__ int32_t seg_o[kQueryWarps][2][kQueryPath];
  const int64_t w = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32, wl = threadIdx.x / 32;
  if (w >= nq) return;
  const BiQuery q = qs[w];
  const double *z1 = a.Z + a.zoff[q.s1] + int64_t(q.j1) * a.plen[q.s1];
  const double *z2 = q.s2 >= 0 ? a.Z + a.zoff[q.s2] + int64_t(q.j2) * a.plen[q.s2] : nullptr;
  // the merge supernode: walk both paths up by plen
  int32_t m = -1;
  if (q.s2 >= 0) {
    int32_t xs = q.s1, ys = q.s2;
    while (xs != ys && xs >= 0 && ys >= 0) {
      if (a.plen[xs] >= a.plen[ys]) xs = a.parent[xs]; else ys = a.parent[ys];
    }
    m = (xs == ys) ? xs : -1;
  }
  const int n1 = bi_path_list(a, q.s1, -1, seg_f[wl][0], seg_o[wl][0], lane);
  const int n2 = q.s2 >= 0 ? bi_path_list(a, q.s2, m, seg_f[wl][1], seg_o[wl][1], lane) : 0;
  double acc = 0.0;
  if (n1 >= 0 && n2 >= 0) {
    const int32_t p1 = a.plen[q.s1];
    const int32_t pm = m >= 0 ? a.plen[m] : 0;
    const int32_t L1 = q.s2 >= 0 ? p1 - pm : p1;
    // s1's branch (all of P_s1 when the query touches the ground)
    acc += bi_rows_sum(a, z1, nullptr, 0, 0, L1, seg_f[wl][0], seg_o[wl][0], n1, 0, lane);
    if (q.s2 >= 0) {
      const int32_t p2 = a.plen[q.s2], L2 = p2 - pm;
      acc += bi_rows_sum(a, z2, nullptr, 0, 0, L2, seg_f[wl][1], seg_o[wl][1], n2, 0, lane);
      // common part: rows [L1, p1) of z1 against rows [L2, p2) of z2, on s1's list
      acc += bi_rows_sum(a, z1, z2, int64_t(L1) - L2, L1, p1, seg_f[wl][0], seg_o[wl][0], n1,
                         0, lane);
    }
  } else {   // a path longer than the lists: supernode by supernode
    int32_t x = q.s1, y = q.s2;
    if (y >= 0) {
      for (; x != m; x = a.parent[x]) {
        const int32_t f = a.first[x], nc = a.first[x + 1] - f;
        const int64_t off = a.plen[q.s1] - a.plen[x];
        for (int k = lane; k < nc; k += 32) {
          const double v = z1[off + k];
          acc = fma(v * v, a.dinv[f + k], acc);
        }
      }
      for (; y != m; y = a.parent[y]) {
        const int32_t f = a.first[y], nc = a.first[y + 1] - f;
        const int64_t off = a.plen[q.s2] - a.plen[y];
        for (int k = lane; k < nc; k += 32) {
          const double v = z2[off + k];
          acc = fma(v * v, a.dinv[f + k], acc);
        }
      }
    }
    for (; x != -1; x = a.parent[x]) {
      const int32_t f = a.first[x], nc = a.first[x + 1] - f;
      const int64_t o1 = a.plen[q.s1] - a.plen[x];
      const int64_t o2 = q.s2 >= 0 ? a.plen[q.s2] - a.plen[x] : 0;
      for (int k = lane; k < nc; k += 32) {
        const double v = z1[o1 + k] - (q.s2 >= 0 ? z2[o2 + k] : 0.0);
        acc = fma(v * v, a.dinv[f + k], acc);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0 && PEERS_IN(q.out, a.nq, a.status)) R[q.out] = acc;
}

// ================================================================ selected inversion
//
// Sigma = L_r^{-1} on the pattern of L (Takahashi's recurrences in supernodal L D L^T form),
// top-down by depth.  For supernode s with T = L[C,C], P = L[B,C], M = P T^{-1}, Zd = T^{-1}:
//     Sigma[B,B] = the parent's inverse front restricted to B (a gather through rmap)
//     Sigma[B,C] = -Sigma[B,B] M
//     Sigma[C,C] = Zd^T D_C^{-1} Zd - M^T Sigma[B,C]
// The inverse front F(s) = Sigma[rows(s), rows(s)] (column-major) is all a query starting at s
// needs: R = F[a,a] + F[b,b] - 2 F[b,a] (eq. 2 with L_r^{-1} = Sigma).  Sigma is symmetric and
// only the lower triangle of F is formed (its B,B block in full, as the product's operand);
// every read of a front takes entry (max(i,j), min(i,j)).

struct SiArgs {
  const double *dinv;
  const int32_t *first, *nb, *rmap, *parent;
  const int64_t *rows_off;
  const double *Zd;       // T^{-1} per supernode, n_c x n_c column-major
  const int64_t *doff;
  const double *M;        // n_b x n_c row-major per supernode
  const int64_t *moff;
  const int64_t *foff;    // offset of F(s) in F (each lane's region alternates by depth)
  double *F;              // inverse fronts
  int *status;            // error flag (bounds-checked build)
  int64_t fbuf, nq;       // extents of F and of the results
};

// Sigma[B,B] of each supernode of this depth from its parent's front.  grid = (supernode,
// chunk of 8 columns of B).
__global__ void __launch_bounds__(256) k_si_gather(const int32_t *__restrict__ sns, SiArgs a) {
  const int32_t s = sns[blockIdx.x];
  const int32_t p = a.parent[s];
  const int32_t nc = a.first[s + 1] - a.first[s], nbv = a.nb[s], N = nc + nbv;
  const int32_t Np = a.first[p + 1] - a.first[p] + a.nb[p];
  const int32_t j0 = blockIdx.y * 8;
  if (j0 >= nbv) return;
  const int32_t *rm = a.rmap + a.rows_off[s];
  const double *Fp = a.F + a.foff[p];
  double *F = a.F + a.foff[s];
  if (!PEERS_IN(a.foff[s] + int64_t(N) * N - 1, a.fbuf, a.status) ||
      !PEERS_IN(a.foff[p] + int64_t(Np) * Np - 1, a.fbuf, a.status))
    return;
  for (int32_t j = j0; j < min(nbv, j0 + 8); ++j) {
    const int32_t rj = rm[j];
    for (int32_t i = threadIdx.x; i < nbv; i += blockDim.x) {
      const int32_t ri = rm[i];
      if (PEERS_IN(max(ri, rj), Np, a.status))
        F[int64_t(nc + j) * N + nc + i] = Fp[int64_t(min(ri, rj)) * Np + max(ri, rj)];
    }
  }
}

// Sigma[B,C] = -Sigma[B,B] M by the row-per-thread product (rows_gemm): A = Sigma[B,B] (the
// front's B,B block, column-major), B = M (row-major n_b x n_c), out = the front's B,C block.
template <int G>
__global__ void __launch_bounds__(kRowsMaxThreads) k_si_bc(const Tile *__restrict__ tiles,
                                                           SiArgs a, int rows) {
  __shared__ double Ms[kRowsK * rows_group_width(G)];
  const Tile tl = tiles[blockIdx.x];
  const int32_t s = tl.t;
  const int32_t nc = a.first[s + 1] - a.first[s], nbv = a.nb[s], N = nc + nbv;
  double *F = a.F + a.foff[s];
  RowsGemm g;
  g.A = F + int64_t(nc) * N + nc;
  g.lda = N;
  g.B = a.M + a.moff[s];
  g.bk = nc;
  g.bc = 1;
  g.out = F + nc;
  g.oi = 1;
  g.oc = N;
  g.nrows = nbv;
  g.kb = 0;
  g.ke = nbv;
  g.ncols = nc;
  g.negate = true;
  g.a_ext = a.fbuf - (a.foff[s] + int64_t(nc) * N + nc);
  g.b_ext = a.moff[s + 1] - a.moff[s];
  g.o_ext = a.fbuf - (a.foff[s] + nc);
  g.status = a.status;
  rows_gemm_dispatch<G>(g, tl, rows, Ms);
}

// Sigma[C,C] = Zd^T D^{-1} Zd - M^T Sigma[B,C], lower triangle: tiles (r >= c) of TS x TS over
// n_c x n_c, TS = 16, 32 or 64 following n_c (Tile.pad); 16 x 16 threads, (TS/16)^2 outputs each.
template <int TS>
__device__ __forceinline__ void si_cc_tile(const Tile &tl, const SiArgs &a, double *As,
                                           double *Bs) {
  constexpr int U = TS / 16;
  const int32_t s = tl.t;
  const int32_t f = a.first[s], nc = a.first[s + 1] - f, nbv = a.nb[s], N = nc + nbv;
  double *F = a.F + a.foff[s];
  const double *Zd = a.Zd + a.doff[s];
  const double *M = a.M + a.moff[s];
  const int R0 = tl.r * TS, C0 = tl.c * TS;
  if (!PEERS_IN(a.foff[s] + int64_t(N) * N - 1, a.fbuf, a.status) ||
      !PEERS_IN(int64_t(nc) * nc - 1, a.doff[s + 1] - a.doff[s], a.status) ||
      !(nbv == 0 || PEERS_IN(int64_t(nbv) * nc - 1, a.moff[s + 1] - a.moff[s], a.status)))
    return;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[U][U] = {};
  // Zd^T D^{-1} Zd: Zd[k, i] Zd[k, j] is non-zero only for k >= max(i, j)
  const int kstart = (max(R0, C0) / kK) * kK;
  for (int k0 = kstart; k0 < nc + nbv; k0 += kK) {
    // consecutive threads take consecutive k where the source is contiguous in k (Zd's
    // columns, the front's B,C block) and consecutive rows where it is contiguous in rows (M)
    for (int e = threadIdx.x; e < kK * TS; e += kGemmThreads) {
      const int r = e / kK, k = e - (e / kK) * kK;
      const int kk = k0 + k;
      double y = 0.0;
      if (kk < nc) {
        if (C0 + r < nc) y = Zd[int64_t(C0 + r) * nc + kk];
      } else if (kk < nc + nbv) {
        if (C0 + r < nc) y = -F[int64_t(C0 + r) * N + kk];
      }
      Bs[k * TS + r] = y;
    }
    if (k0 + kK <= nc) {
      for (int e = threadIdx.x; e < kK * TS; e += kGemmThreads) {
        const int r = e / kK, k = e - (e / kK) * kK;
        const int kk = k0 + k;
        As[k * TS + r] = R0 + r < nc ? Zd[int64_t(R0 + r) * nc + kk] * a.dinv[f + kk] : 0.0;
      }
    } else {
      for (int e = threadIdx.x; e < kK * TS; e += kGemmThreads) {
        const int k = e / TS, r = e - (e / TS) * TS;
        const int kk = k0 + k;
        double x = 0.0;
        if (kk < nc) {
          if (R0 + r < nc) x = Zd[int64_t(R0 + r) * nc + kk] * a.dinv[f + kk];
        } else if (kk < nc + nbv) {
          if (R0 + r < nc) x = M[int64_t(kk - nc) * nc + R0 + r];
        }
        As[k * TS + r] = x;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kK; ++k) {
      double av[U], bv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) { av[u] = As[k * TS + tx + 16 * u]; bv[u] = Bs[k * TS + ty + 16 * u]; }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int v = 0; v < U; ++v) {
    const int j = C0 + ty + 16 * v;
    if (j >= nc) continue;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = R0 + tx + 16 * u;
      if (i < nc && i >= j) F[int64_t(j) * N + i] = acc[u][v];
    }
  }
}

__global__ void __launch_bounds__(kGemmThreads) k_si_cc(const Tile *__restrict__ tiles, SiArgs a) {
  __shared__ double As[kK * kT];
  __shared__ double Bs[kK * kT];
  const Tile tl = tiles[blockIdx.x];
  switch (tl.pad) {
    case 16: si_cc_tile<16>(tl, a, As, Bs); break;
    case 32: si_cc_tile<32>(tl, a, As, Bs); break;
    default: si_cc_tile<64>(tl, a, As, Bs); break;
  }
}

inline int cc_tile(int32_t nc) { return nc <= 16 ? 16 : nc <= 32 ? 32 : kT; }

struct SiQuery {
  int32_t s, a, b, pad;   // start supernode, local rows of lo and hi in its front (b = -1: none)
  int64_t out;
};

// A whole small supernode (n_c <= 32 columns, front N <= 64 rows) in one CTA: M from the
// factor's diagonal-block inverse, Sigma[B,B] gathered from the parent's front, Sigma[B,C],
// Sigma[C,C], the front written for the children, and the supernode's own queries answered.
constexpr int kSiSmallN = 64;
struct SiSmallArgs {
  const double *panel, *tinv;
  const int64_t *panel_off, *tinv_off;
  const int64_t *qbeg, *qorig;
  const int32_t *qa, *qb;
  double *R;
};

__global__ void __launch_bounds__(256) k_si_small(const int32_t *__restrict__ sns, SiArgs a,
                                                  SiSmallArgs b) {
  extern __shared__ double sm_si[];
  const int32_t s = sns[blockIdx.x];
  const int32_t f = a.first[s], nc = a.first[s + 1] - f, nbv = a.nb[s], N = nc + nbv;
  double *F = sm_si;            // N x N
  double *Ti = F + N * N;       // nc x nc
  double *Mm = Ti + nc * nc;    // nbv x nc
  double *dv = Mm + nbv * nc;   // nc
  const int32_t p = a.parent[s];
  const int tid = threadIdx.x;
  const double *TI = b.tinv + b.tinv_off[s];
  if (!PEERS_IN(int64_t(N) * N + nc * nc + nbv * nc + nc - 1, dynamic_smem_doubles(), a.status) ||
      !PEERS_IN(a.foff[s] + int64_t(N) * N - 1, a.fbuf, a.status) ||
      !PEERS_IN(int64_t(nc) * nc - 1, b.tinv_off[s + 1] - b.tinv_off[s], a.status) ||
      !PEERS_IN(int64_t(nc) * N - 1, b.panel_off[s + 1] - b.panel_off[s], a.status))
    return;
  for (int e = tid; e < nc * nc; e += blockDim.x) Ti[e] = TI[e];
  for (int e = tid; e < nc; e += blockDim.x) dv[e] = a.dinv[f + e];
  if (p >= 0) {
    const int32_t Np = a.first[p + 1] - a.first[p] + a.nb[p];
    const int32_t *rm = a.rmap + a.rows_off[s];
    const double *Fp = a.F + a.foff[p];
    for (int e = tid; e < nbv * nbv; e += blockDim.x) {
      const int i = e % nbv, j = e / nbv;
      const int32_t ri = rm[i], rj = rm[j];
      if (PEERS_IN(max(ri, rj), Np, a.status) &&
          PEERS_IN(a.foff[p] + int64_t(Np) * Np - 1, a.fbuf, a.status))
        F[(nc + j) * N + nc + i] = Fp[int64_t(min(ri, rj)) * Np + max(ri, rj)];
    }
  }
  __syncthreads();
  // M[i][c] = sum_{k >= c} P[i][k] T^{-1}[k][c]
  const double *P = b.panel + b.panel_off[s];
  for (int e = tid; e < nbv * nc; e += blockDim.x) {
    const int i = e / nc, c = e % nc;
    double m = 0.0;
    for (int k = c; k < nc; ++k) m = fma(P[int64_t(k) * N + nc + i], Ti[k * nc + c], m);
    Mm[i * nc + c] = m;
  }
  __syncthreads();
  // Sigma[B,C] = -Sigma[B,B] M
  for (int e = tid; e < nbv * nc; e += blockDim.x) {
    const int i = e % nbv, j = e / nbv;
    double acc = 0.0;
    for (int k = 0; k < nbv; ++k) acc = fma(F[(nc + k) * N + nc + i], Mm[k * nc + j], acc);
    F[j * N + nc + i] = -acc;
    F[(nc + i) * N + j] = -acc;
  }
  __syncthreads();
  // Sigma[C,C] = T^{-T} D^{-1} T^{-1} - M^T Sigma[B,C]
  for (int e = tid; e < nc * nc; e += blockDim.x) {
    const int i = e % nc, j = e / nc;
    double acc = 0.0;
    for (int k = max(i, j); k < nc; ++k) acc = fma(Ti[k * nc + i] * dv[k], Ti[k * nc + j], acc);
    for (int k = 0; k < nbv; ++k) acc = fma(-Mm[k * nc + i], F[j * N + nc + k], acc);
    F[j * N + i] = acc;
  }
  __syncthreads();
  double *Fg = a.F + a.foff[s];
  for (int e = tid; e < N * N; e += blockDim.x) Fg[e] = F[e];
  for (int64_t q = b.qbeg[s] + tid; q < b.qbeg[s + 1]; q += blockDim.x) {
    const int32_t qa = b.qa[q], qb = b.qb[q];
    if (!PEERS_IN(qa, N, a.status) || (qb >= 0 && !PEERS_IN(qb, N, a.status)) ||
        !PEERS_IN(b.qorig[q], a.nq, a.status))
      continue;
    double r = F[qa * N + qa];
    if (qb >= 0) r += F[qb * N + qb] - 2.0 * F[min(qa, qb) * N + max(qa, qb)];
    b.R[b.qorig[q]] = r;
  }
}

__global__ void k_si_query(const SiQuery *__restrict__ qs, int64_t nq, SiArgs args, double *R) {
  const int64_t k = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (k >= nq) return;
  const SiQuery q = qs[k];
  const int32_t N = args.first[q.s + 1] - args.first[q.s] + args.nb[q.s];
  const double *F = args.F + args.foff[q.s];
  if (!PEERS_IN(q.a, N, args.status) || (q.b >= 0 && !PEERS_IN(q.b, N, args.status)) ||
      !PEERS_IN(q.out, args.nq, args.status) ||
      !PEERS_IN(args.foff[q.s] + int64_t(N) * N - 1, args.fbuf, args.status))
    return;
  double r = F[int64_t(q.a) * N + q.a];
  if (q.b >= 0) r += F[int64_t(q.b) * N + q.b] - 2.0 * F[int64_t(min(q.a, q.b)) * N + max(q.a, q.b)];
  R[q.out] = r;
}

}  // namespace

// ---------------------------------------------------------------- host plan

struct BlockInvPlan {
  std::vector<int32_t> plen, depth, parent;
  std::vector<int64_t> zoff, moff;
  int64_t ztotal = 0, mtotal = 0;
  std::vector<int32_t> gstart;
  std::vector<int64_t> gsrc;
  std::vector<int32_t> diag_sn, diag_blk;          // phase 1a CTAs (wide supernodes)
  std::vector<int32_t> small_sn, small_chunk;      // phase 1 CTAs of narrow supernodes
  std::vector<Tile> m_tiles;                       // phase 1b tiles, by width group
  std::vector<int64_t> m_ptr;
  std::vector<Tile> z_tiles;                       // phase 2 tiles, grouped by depth
  std::vector<int64_t> z_ptr;                      // depth d: z_tiles[z_ptr[d] .. z_ptr[d+1])
  std::vector<Tile> n_tiles;                       // phase 2 narrow tiles (n_c <= 32)
  std::vector<int64_t> n_ptr;                      // 2 width groups per depth
  std::vector<BiQuery> queries;
  int64_t gemm_fma = 0;                            // phase-2 FMAs with the staircase
};

int blockinv_plan(const Symbolic &S, BlockInvPlan &B, std::string &err) {
  const int32_t ns = S.nsuper;
  B.plen.assign(ns, 0);
  B.depth.assign(ns, 0);
  B.parent = S.parent;
  int32_t maxd = 0;
  for (int32_t t = ns - 1; t >= 0; --t) {
    const int32_t p = S.parent[t];
    B.plen[t] = sn_nc(S, t) + (p >= 0 ? B.plen[p] : 0);
    B.depth[t] = p >= 0 ? B.depth[p] + 1 : 0;
    maxd = std::max(maxd, B.depth[t]);
  }
  B.zoff.assign(ns + 1, 0);
  B.moff.assign(ns + 1, 0);
  for (int32_t t = 0; t < ns; ++t) {
    B.zoff[t + 1] = B.zoff[t] + int64_t(B.plen[t]) * sn_nc(S, t);
    B.moff[t + 1] = B.moff[t] + int64_t(S.nb[t]) * sn_nc(S, t);
  }
  B.ztotal = B.zoff[ns];
  B.mtotal = B.moff[ns];
  // staircase of each B_t column inside P_parent, and where its Z column lives
  B.gstart.assign(S.rows.size(), 0);
  B.gsrc.assign(S.rows.size(), 0);
  B.gemm_fma = 0;
  for (int32_t t = 0; t < ns; ++t) {
    const int32_t p = S.parent[t];
    if (p < 0) continue;
    for (int64_t k = S.rows_off[t]; k < S.rows_off[t + 1]; ++k) {
      const int32_t b = S.rows[k];
      const int32_t a = S.col2sn[b];
      B.gstart[k] = B.plen[p] - B.plen[a];
      B.gsrc[k] = B.zoff[a] + int64_t(b - S.first[a]) * B.plen[a];
      B.gemm_fma += int64_t(B.plen[a]) * sn_nc(S, t);
    }
  }
  // phase 1 work
  B.diag_sn.clear();
  B.diag_blk.clear();
  B.m_tiles.clear();
  B.small_sn.clear();
  B.small_chunk.clear();
  std::vector<int32_t> wide;
  for (int32_t t = 0; t < ns; ++t) {
    const int32_t nc = sn_nc(S, t), nbv = S.nb[t];
    if (nc <= kBlock) {   // one diagonal block: its inverse already exists
      for (int32_t ch = 0; ch == 0 || ch * 256 < nbv; ++ch) {
        B.small_sn.push_back(t);
        B.small_chunk.push_back(ch);
      }
      continue;
    }
    for (int32_t J = 0; J * kBlock < nc; ++J)
      for (int32_t sl = 0; sl < kDiagSlices && J * kBlock + sl * kDiagSlice < nc; ++sl) {
        B.diag_sn.push_back(t);
        B.diag_blk.push_back(J * kDiagSlices + sl);
      }
    wide.push_back(t);
  }
  m_tiles_of(S, wide, B.m_tiles, B.m_ptr);
  // phase 2 tiles by depth: square tiles for wide supernodes, one row per thread for narrow
  // ones (at most 32 columns)
  std::vector<std::vector<Tile>> per(maxd + 1), pern(2 * (maxd + 1));   // pern: 2 groups per depth
  std::vector<std::vector<int32_t>> wide_by_depth(maxd + 1);
  for (int32_t t = 0; t < ns; ++t) {
    const int32_t nc = sn_nc(S, t), lp = B.plen[t] - nc;
    if (lp == 0 || S.nb[t] == 0) continue;
    if (nc <= 32) {
      const int w = narrow_width(nc);
      for (int32_t r = 0; r * kNarrowRows < lp; ++r)
        pern[2 * B.depth[t] + (w <= 8 ? 0 : 1)].push_back({t, r, 0, w});
    } else {
      wide_by_depth[B.depth[t]].push_back(t);
    }
  }
  // wide tiles: per depth, the largest tile (64, 32, 16) that still gives the launch at least
  // 256 CTAs per SM of a 148-SM B300 (few large tiles leave most SMs idle at the top levels;
  // at pdn1m 16 per SM took the pass 1.30 s, 64 per SM 1.21 s, 128 1.16 s, 256 1.11 s)
  constexpr int64_t kTargetCtas = 148 * 256;
  for (int32_t d = 0; d <= maxd; ++d) {
    int ts = kT;
    for (; ts > 16; ts /= 2) {
      int64_t ctas = 0;
      for (int32_t t : wide_by_depth[d])
        ctas += int64_t((B.plen[t] - sn_nc(S, t) + ts - 1) / ts) * ((sn_nc(S, t) + ts - 1) / ts);
      if (ctas >= kTargetCtas) break;
    }
    for (int32_t t : wide_by_depth[d]) {
      const int32_t nc = sn_nc(S, t), lp = B.plen[t] - nc;
      for (int32_t r = 0; r * ts < lp; ++r)
        for (int32_t c = 0; c * ts < nc; ++c) per[d].push_back({t, r, c, ts});
    }
  }
  B.z_tiles.clear();
  B.z_ptr.assign(1, 0);
  B.n_tiles.clear();
  B.n_ptr.assign(1, 0);
  for (int32_t d = 0; d <= maxd; ++d) {
    B.z_tiles.insert(B.z_tiles.end(), per[d].begin(), per[d].end());
    B.z_ptr.push_back(static_cast<int64_t>(B.z_tiles.size()));
    for (int g = 0; g < 2; ++g) {
      B.n_tiles.insert(B.n_tiles.end(), pern[2 * d + g].begin(), pern[2 * d + g].end());
      B.n_ptr.push_back(static_cast<int64_t>(B.n_tiles.size()));
    }
  }
  // queries: the plan's single-path slots and two-branch pairs
  B.queries.clear();
  B.queries.reserve(static_cast<size_t>(S.nsorted + S.nq_two));
  for (int32_t s = 0; s < ns; ++s) {
    for (int64_t q = S.qbeg[s]; q < S.qbeg[s + 1]; ++q) {
      BiQuery bq{};
      bq.s1 = s;
      bq.j1 = S.qa[q];
      bq.out = S.qorig[q];
      const int32_t b = S.qb[q];
      if (b < 0) {
        bq.s2 = -1;
      } else {
        const int32_t nc = sn_nc(S, s);
        const int32_t hi = b < nc ? S.first[s] + b : S.rows[S.rows_off[s] + (b - nc)];
        bq.s2 = S.col2sn[hi];
        bq.j2 = hi - S.first[bq.s2];
      }
      B.queries.push_back(bq);
    }
  }
  for (int64_t k = 0; k < S.nq_two; ++k) {
    BiQuery bq{};
    bq.s1 = S.col2sn[S.two_lo[k]];
    bq.j1 = S.two_lo[k] - S.first[bq.s1];
    bq.s2 = S.col2sn[S.two_hi[k]];
    bq.j2 = S.two_hi[k] - S.first[bq.s2];
    bq.out = S.two_idx[k];
    B.queries.push_back(bq);
  }
  (void)err;
  return PEERS_OK;
}

// lanes (optional): a depth's narrow launches run on two of the lanes' streams beside its
// square-tile launch on `st`, so that each fills the others' partial last waves; the three
// write disjoint blocks of Z and read only shallower depths' blocks.
int blockinv_run(const Symbolic &S, const BlockInvPlan &B, const BiArgs &base, Tile *d_mt,
                 Tile *d_zt, Tile *d_nt, int32_t *d_dsn, int32_t *d_dblk, int32_t *d_ssn,
                 int32_t *d_sch, BiQuery *d_q, double *R,
                 cudaStream_t st, const Lanes *lanes, int64_t *launches,
                 std::vector<cudaEvent_t> *ev, std::string &err) {
  BiArgs a = base;
  auto mark = [&]() {
    if (ev) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      cudaEventRecord(e, st);
      ev->push_back(e);
    }
  };
  mark();
  if (S.nq > 0) CUDA_TRY(cudaMemsetAsync(R, 0, sizeof(double) * S.nq, st));
  // entries above each block's diagonal are zero and are never written by the kernels
  if (B.ztotal > 0) CUDA_TRY(cudaMemsetAsync(a.Z, 0, sizeof(double) * B.ztotal, st));
  if (!B.small_sn.empty()) {
    k_bi_small<<<static_cast<unsigned>(B.small_sn.size()), 256, 0, st>>>(d_ssn, d_sch, a);
    ++*launches;
    CUDA_TRY(cudaGetLastError());
  }
  if (!B.diag_sn.empty()) {
    k_bi_diag<<<static_cast<unsigned>(B.diag_sn.size()), kBlock * kDiagSlice, 0, st>>>(d_dsn, d_dblk, a);
    ++*launches;
    CUDA_TRY(cudaGetLastError());
  }
  mark();
  {
    const int rc = launch_m_all(d_mt, B.m_ptr, a, st, launches, err);
    if (rc != PEERS_OK) return rc;
  }
  mark();
  for (size_t d = 0; d + 1 < B.z_ptr.size(); ++d) {
    const int64_t n = B.z_ptr[d + 1] - B.z_ptr[d];
    const int64_t n0 = B.n_ptr[2 * d + 1] - B.n_ptr[2 * d];
    const int64_t n1 = B.n_ptr[2 * d + 2] - B.n_ptr[2 * d + 1];
    const bool fork = lanes && (n > 0) + (n0 > 0) + (n1 > 0) > 1;
    const cudaStream_t s0 = fork ? lanes->stream[0] : st, s1 = fork ? lanes->stream[1] : st;
    if (fork) {
      CUDA_TRY(cudaEventRecord(lanes->start, st));
      CUDA_TRY(cudaStreamWaitEvent(s0, lanes->start, 0));
      CUDA_TRY(cudaStreamWaitEvent(s1, lanes->start, 0));
    }
    if (n > 0) {
      k_bi_z<<<static_cast<unsigned>(n), kGemmThreads, 0, st>>>(d_zt + B.z_ptr[d], a);
      ++*launches;
      CUDA_TRY(cudaGetLastError());
    }
    if (n0 > 0) {
      k_bi_z_narrow<0><<<static_cast<unsigned>(n0), kNarrowRows, narrow_smem(0), s0>>>(
          d_nt + B.n_ptr[2 * d], a);
      ++*launches;
      CUDA_TRY(cudaGetLastError());
    }
    if (n1 > 0) {
      k_bi_z_narrow<1><<<static_cast<unsigned>(n1), kNarrowRows, narrow_smem(1), s1>>>(
          d_nt + B.n_ptr[2 * d + 1], a);
      ++*launches;
      CUDA_TRY(cudaGetLastError());
    }
    if (fork) {
      CUDA_TRY(cudaEventRecord(lanes->done[0], s0));
      CUDA_TRY(cudaEventRecord(lanes->done[1], s1));
      CUDA_TRY(cudaStreamWaitEvent(st, lanes->done[0], 0));
      CUDA_TRY(cudaStreamWaitEvent(st, lanes->done[1], 0));
    }
    if (n > 0 || n0 > 0 || n1 > 0) mark();
  }
  const int64_t nq = static_cast<int64_t>(B.queries.size());
  if (nq > 0) {
    const unsigned blocks = static_cast<unsigned>((nq * 32 + 255) / 256);
    k_bi_query<<<blocks, 256, 0, st>>>(d_q, nq, a, R);
    ++*launches;
    CUDA_TRY(cudaGetLastError());
  }
  mark();
  return PEERS_OK;
}

// ---------------------------------------------------------------- selected inversion plan

// One group of the selected inversion: the supernodes of one tree depth in one lane (lane -1:
// the part above the lanes' subtrees, on the context's stream), with the ranges of its
// launches in the plan's lists.
struct SiGroup {
  int32_t lane = -1, depth = 0;
  int64_t fused_b = 0, fused_e = 0, fused_smem = 0;   // whole small supernodes
  int64_t gather_b = 0, gather_e = 0;
  int32_t gather_ych = 0;                              // column chunks of the largest B
  int64_t bc_ptr[4] = {0, 0, 0, 0};                    // Sigma[B,C] tiles, three width groups
  int32_t bc_rows = 0;                                 // rows per Sigma[B,C] CTA
  int64_t cc_b = 0, cc_e = 0;
  int64_t q_b = 0, q_e = 0;
};

// Phase 1 (T^{-1} and M) of one lane's supernodes, or of one depth of the top part
// (lane -1), whose groups wait for it.
struct SiPhase1 {
  int32_t lane = -1, depth = 0;
  int64_t small_b = 0, small_e = 0;             // narrow supernodes (k_bi_small)
  int64_t diag_b = 0, diag_e = 0;               // wide: T^{-1} by substitution (k_bi_diag)
  int64_t base_b = 0, base_e = 0;               // wide: X's diagonal blocks (k_tinv_base)
  std::vector<std::vector<int64_t>> tlevels;    // wide: doubling levels, into tinv_tiles
  std::vector<int64_t> m_ptr;                   // 4 entries into m_tiles
};

struct SelInvPlan {
  std::vector<int32_t> ncs;                        // n_c per supernode (ld of Zd)
  std::vector<int64_t> doff, moff;
  int64_t dtotal = 0, mtotal = 0;
  std::vector<int64_t> foff;                       // offset of F(s) in the fronts buffer
  int64_t fbuf = 0;                                // doubles of the fronts buffer
  int32_t nlanes = 0;
  std::vector<SiGroup> groups;                     // top part by depth, then lanes by depth
  std::vector<SiPhase1> phase1;                    // top part by depth, then per lane
  std::vector<int32_t> gather_sn;
  std::vector<Tile> bc, cc;
  std::vector<SiQuery> queries;
  std::vector<int32_t> fused_sn;                   // whole small supernodes
  std::vector<int32_t> small_sn, small_chunk, diag_sn, diag_blk, tbase_sn, tbase_blk;
  std::vector<TinvTile> tinv_tiles;
  std::vector<Tile> m_tiles;
  int64_t fma = 0;
};

// sms: the device's multiprocessor count (sizes the launches).
int selinv_plan(const Symbolic &S, SelInvPlan &P, int sms, std::string &err) {
  if (S.nq_two > 0) {
    err = "the selected inverse covers pairs inside the pattern of L (every graph edge and "
          "every pair touching the ground); this plan lists " + std::to_string(S.nq_two) +
          " other pairs: use peers_query or peers_query_blockinv";
    return PEERS_EINVAL;
  }
  const int32_t ns = S.nsuper;
  const int32_t nl = S.nlanes;
  P.nlanes = nl;
  int32_t maxd = 0;
  for (int32_t t = 0; t < ns; ++t) maxd = std::max(maxd, S.depth[t]);
  P.ncs.resize(ns);
  P.doff.assign(ns + 1, 0);
  P.moff.assign(ns + 1, 0);
  P.foff.assign(ns, 0);
  P.fma = 0;
  // members of each (lane, depth) group; fronts of a lane alternate between two regions by
  // depth parity (a depth reads only its parents' fronts, one depth up)
  std::vector<std::vector<std::vector<int32_t>>> members(
      nl + 1, std::vector<std::vector<int32_t>>(maxd + 1));
  std::vector<std::vector<int64_t>> fsize(nl + 1, std::vector<int64_t>(maxd + 1, 0));
  for (int32_t t = 0; t < ns; ++t) {
    const int64_t nc = sn_nc(S, t), nbv = S.nb[t], N = nc + nbv;
    P.ncs[t] = static_cast<int32_t>(nc);
    P.doff[t + 1] = P.doff[t] + nc * nc;
    P.moff[t + 1] = P.moff[t] + nbv * nc;
    const int32_t L = S.lane_of[t] + 1, d = S.depth[t];
    members[L][d].push_back(t);
    P.foff[t] = fsize[L][d];
    fsize[L][d] += N * N;
    // useful multiply-adds: Sigma[B,C] (n_b^2 n_c), the lower triangle of Sigma[C,C] (the
    // T^{-T} D^{-1} T^{-1} part over k >= max(i, j), and M^T Sigma[B,C]), M = P T^{-1} over
    // k >= c, and T^{-1} itself where it is formed here (n_c > kBlock)
    P.fma += nbv * nbv * nc + nc * (nc + 1) * (nc + 2) / 6 + nbv * nc * (nc + 1) / 2 +
             nbv * nc * (nc + 1) / 2 + (nc > kBlock ? nc * (nc - 1) * (nc - 2) / 6 : 0);
  }
  // region bases: (lane, parity) -> offset
  std::vector<int64_t> base(2 * (nl + 1), 0);
  P.fbuf = 0;
  for (int32_t L = 0; L <= nl; ++L)
    for (int par = 0; par < 2; ++par) {
      int64_t mx = 0;
      for (int32_t d = par; d <= maxd; d += 2) mx = std::max(mx, fsize[L][d]);
      base[2 * L + par] = P.fbuf;
      P.fbuf += mx;
    }
  for (int32_t t = 0; t < ns; ++t)
    P.foff[t] += base[2 * (S.lane_of[t] + 1) + (S.depth[t] & 1)];
  P.dtotal = P.doff[ns];
  P.mtotal = P.moff[ns];
  auto fused = [&](int32_t t) {
    return sn_nc(S, t) <= kBlock && sn_nc(S, t) + S.nb[t] <= kSiSmallN;
  };
  // phase 1 (T^{-1} and M) as in the block inverse, for the supernodes not fused: the top
  // part depth by depth (each depth's groups wait only for their own phase 1, so the deeper
  // ones overlap the top of the tree), then each lane's supernodes
  P.phase1.clear();
  std::vector<std::pair<int32_t, int32_t>> p1keys;   // (lane, depth or -1 for all)
  for (int32_t d = 0; d <= maxd; ++d)
    if (!members[0][d].empty()) p1keys.push_back({-1, d});
  for (int32_t L = 0; L < nl; ++L) p1keys.push_back({L, -1});
  for (const auto &key : p1keys) {
    SiPhase1 ph;
    ph.lane = key.first;
    ph.depth = key.second;
    std::vector<int32_t> wide, doubling;
    ph.small_b = static_cast<int64_t>(P.small_sn.size());
    ph.diag_b = static_cast<int64_t>(P.diag_sn.size());
    for (int32_t t = 0; t < ns; ++t) {
      if (S.lane_of[t] != key.first || (key.second >= 0 && S.depth[t] != key.second) || fused(t))
        continue;
      const int32_t nc = sn_nc(S, t), nbv = S.nb[t];
      if (nc <= kBlock) {
        for (int32_t ch = 0; ch == 0 || ch * 256 < nbv; ++ch) {
          P.small_sn.push_back(t);
          P.small_chunk.push_back(ch);
        }
        continue;
      }
      wide.push_back(t);
      if (nc >= kTinvDoubling) {
        doubling.push_back(t);
        continue;
      }
      for (int32_t J = 0; J * kBlock < nc; ++J)
        for (int32_t sl = 0; sl < kDiagSlices && J * kBlock + sl * kDiagSlice < nc; ++sl) {
          P.diag_sn.push_back(t);
          P.diag_blk.push_back(J * kDiagSlices + sl);
        }
    }
    ph.small_e = static_cast<int64_t>(P.small_sn.size());
    ph.diag_e = static_cast<int64_t>(P.diag_sn.size());
    {
      TinvPlan T;
      tinv_plan_of(S, doubling, T, P.tinv_tiles);
      ph.base_b = static_cast<int64_t>(P.tbase_sn.size());
      P.tbase_sn.insert(P.tbase_sn.end(), T.base_sn.begin(), T.base_sn.end());
      P.tbase_blk.insert(P.tbase_blk.end(), T.base_blk.begin(), T.base_blk.end());
      ph.base_e = static_cast<int64_t>(P.tbase_sn.size());
      ph.tlevels = std::move(T.level_ptr);
    }
    std::vector<Tile> mt;
    std::vector<int64_t> mp;
    m_tiles_of(S, wide, mt, mp);
    const int64_t off = static_cast<int64_t>(P.m_tiles.size());
    P.m_tiles.insert(P.m_tiles.end(), mt.begin(), mt.end());
    for (int64_t x : mp) ph.m_ptr.push_back(off + x);
    P.phase1.push_back(std::move(ph));
  }
  // groups: the top part depth by depth, then the lanes, depth by depth
  for (int32_t L = 0; L <= nl; ++L) {
    // every launch is sized as if alone, for at least 64 CTAs per SM: the lanes overlap, but a
    // launch of few one-warp CTAs leaves the FP64 units of its SMs half idle (two to three
    // warps per SM sub-partition keep them busy), and many short CTAs end a launch with a
    // short partial wave (at pdn1m 16 per SM took 189 ms, 32 took 180 ms, 64 took 179 ms)
    const int64_t target_ctas = int64_t(std::max(sms, 1)) * 64;
    for (int32_t d = 0; d <= maxd; ++d) {
      const std::vector<int32_t> &mem = members[L][d];
      if (mem.empty()) continue;
      SiGroup G;
      G.lane = L - 1;
      G.depth = d;
      G.fused_b = static_cast<int64_t>(P.fused_sn.size());
      G.gather_b = static_cast<int64_t>(P.gather_sn.size());
      int32_t ych = 0;
      int64_t fsm = 0;
      for (int32_t t : mem) {
        if (fused(t)) {
          P.fused_sn.push_back(t);
          const int64_t nc = sn_nc(S, t), nbv = S.nb[t], N = nc + nbv;
          fsm = std::max(fsm, 8 * (N * N + nc * nc + nbv * nc + nc));
          continue;
        }
        const int32_t nbv = S.nb[t];
        if (nbv > 0) {
          P.gather_sn.push_back(t);
          ych = std::max(ych, (nbv + 7) / 8);
        }
      }
      G.fused_e = static_cast<int64_t>(P.fused_sn.size());
      G.fused_smem = fsm;
      G.gather_e = static_cast<int64_t>(P.gather_sn.size());
      G.gather_ych = ych;
      // Sigma[C,C] tiles: the largest tile (64, 32, 16; never wider than n_c needs) that still
      // gives the launch many CTAs, as for Sigma[B,C]
      int cc_cap = kT;
      for (; cc_cap > 16; cc_cap /= 2) {
        int64_t ctas = 0;
        for (int32_t t : mem) {
          if (fused(t)) continue;
          const int64_t nt = (sn_nc(S, t) + std::min(cc_cap, cc_tile(sn_nc(S, t))) - 1) /
                             std::min(cc_cap, cc_tile(sn_nc(S, t)));
          ctas += nt * (nt + 1) / 2;
        }
        if (ctas >= target_ctas) break;
      }
      G.cc_b = static_cast<int64_t>(P.cc.size());
      for (int32_t t : mem) {
        if (fused(t)) continue;
        const int32_t nc = sn_nc(S, t);
        const int ts = std::min(cc_cap, cc_tile(nc));
        for (int32_t r = 0; r * ts < nc; ++r)
          for (int32_t c = 0; c <= r; ++c) P.cc.push_back({t, r, c, ts});
      }
      G.cc_e = static_cast<int64_t>(P.cc.size());
      // Sigma[B,C] chunks: the widest chunks and tallest CTAs that still give the launch
      // target_ctas CTAs, else the narrowest (down to 2 columns).  FP64 issue is so slow that a
      // few warps with W independent multiply-adds keep an SM sub-partition's unit busy, so
      // small CTAs lose little; a launch of few large CTAs loses up to half its time to the
      // last, partial wave, and one of few one-warp CTAs leaves the FP64 units idle (measured
      // at pdn1m: adding the 4- and 2-column options took the pass from 189 to 181 ms).
      constexpr int kOpts[][2] = {{128, 64}, {64, 64}, {64, 32}, {32, 32}, {32, 16}, {32, 8},
                                  {32, 4}, {32, 2}};
      constexpr int kNOpts = sizeof(kOpts) / sizeof(kOpts[0]);
      int opt = 0;
      for (; opt < kNOpts - 1; ++opt) {
        const int rows = kOpts[opt][0], wcap = kOpts[opt][1];
        int64_t ctas = 0;
        for (int32_t t : mem) {
          if (fused(t) || S.nb[t] == 0) continue;
          ctas += int64_t((S.nb[t] + rows - 1) / rows) * ((sn_nc(S, t) + wcap - 1) / wcap);
        }
        if (ctas >= target_ctas) break;
      }
      const int rows = kOpts[opt][0], wcap = kOpts[opt][1];
      std::vector<Tile> bcg[3];
      for (int32_t t : mem) {
        if (fused(t) || S.nb[t] == 0) continue;
        const int32_t nc = sn_nc(S, t), nbv = S.nb[t];
        for (int32_t r = 0; r * rows < nbv; ++r)
          for (int32_t c0 = 0; c0 < nc; c0 += wcap) {
            const int w = rows_width(std::min(wcap, nc - c0));
            bcg[rows_group(w)].push_back({t, r, c0, w});
          }
      }
      G.bc_rows = rows;
      G.bc_ptr[0] = static_cast<int64_t>(P.bc.size());
      for (int g = 0; g < 3; ++g) {
        P.bc.insert(P.bc.end(), bcg[g].begin(), bcg[g].end());
        G.bc_ptr[g + 1] = static_cast<int64_t>(P.bc.size());
      }
      G.q_b = static_cast<int64_t>(P.queries.size());
      for (int32_t t : mem) {
        if (fused(t)) continue;   // answered inside the fused kernel
        for (int64_t q = S.qbeg[t]; q < S.qbeg[t + 1]; ++q)
          P.queries.push_back({t, S.qa[q], S.qb[q], 0, S.qorig[q]});
      }
      G.q_e = static_cast<int64_t>(P.queries.size());
      P.groups.push_back(G);
    }
  }
  return PEERS_OK;
}

// The route plans of a symbolic handle, built on first use and kept with it (the selected
// inversion's plan also depends on the device's SM count, so it is rebuilt for another one).
int cached_blockinv_plan(const peers_symbolic *sym, std::shared_ptr<const BlockInvPlan> &out,
                         std::string &err) {
  std::lock_guard<std::mutex> lock(sym->route_mu);
  if (!sym->blockinv_plan) {
    auto p = std::make_shared<BlockInvPlan>();
    const int rc = blockinv_plan(sym->S, *p, err);
    if (rc != PEERS_OK) return rc;
    sym->blockinv_plan = p;
  }
  out = std::static_pointer_cast<const BlockInvPlan>(sym->blockinv_plan);
  return PEERS_OK;
}

int cached_selinv_plan(const peers_symbolic *sym, int sms, std::shared_ptr<const SelInvPlan> &out,
                       std::string &err) {
  std::lock_guard<std::mutex> lock(sym->route_mu);
  if (!sym->selinv_plan || (sms > 0 && sym->selinv_sms != sms)) {
    auto p = std::make_shared<SelInvPlan>();
    const int rc = selinv_plan(sym->S, *p, sms > 0 ? sms : 148, err);
    if (rc != PEERS_OK) return rc;
    sym->selinv_plan = p;
    sym->selinv_sms = sms > 0 ? sms : 148;
  }
  out = std::static_pointer_cast<const SelInvPlan>(sym->selinv_plan);
  return PEERS_OK;
}

}  // namespace peers

// ---------------------------------------------------------------- C ABI

namespace {

int bi_query(peers_ctx *ctx, const peers_symbolic *sym, peers_numeric *num, double *R, int flags,
             std::string &err) {
  const Symbolic &S = sym->S;
  cudaStream_t st = ctx->stream;
  DEVICE_SCOPE(ctx->device);
  std::shared_ptr<const peers::BlockInvPlan> plan;
  int rc = peers::cached_blockinv_plan(sym, plan, err);
  if (rc != PEERS_OK) return rc;
  const peers::BlockInvPlan &B = *plan;
  std::vector<void *> mem;
  auto cleanup = [&]() {
    for (void *p : mem) cudaFree(p);
  };
  auto alloc = [&](void **p, size_t bytes) -> int {
    *p = nullptr;
    if (bytes == 0) bytes = 8;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      err = "cudaMalloc of " + std::to_string(bytes) + " bytes for the block inverse: " +
            cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? PEERS_ENOMEM : PEERS_ECUDA;
    }
    mem.push_back(*p);
    return PEERS_OK;
  };
  auto up = [&](void **p, const void *src, size_t bytes) -> int {
    int r = alloc(p, bytes);
    if (r != PEERS_OK) return r;
    if (bytes && cudaMemcpyAsync(*p, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      err = "upload for the block inverse";
      return PEERS_ECUDA;
    }
    return PEERS_OK;
  };
  peers::BiArgs a{};
  void *p = nullptr;
  rc = alloc(&p, sizeof(double) * B.ztotal);
  if (rc) { cleanup(); return rc; }
  a.Z = static_cast<double *>(p);
  rc = alloc(&p, sizeof(double) * B.mtotal);
  if (rc) { cleanup(); return rc; }
  a.M = static_cast<double *>(p);
  void *dz = nullptr, *dm = nullptr, *dpl = nullptr, *dpar = nullptr, *dgs = nullptr,
       *dgsrc = nullptr, *dmt = nullptr, *dzt = nullptr, *dnt = nullptr, *ddsn = nullptr,
       *ddblk = nullptr, *dssn = nullptr, *dsch = nullptr,
       *dq = nullptr, *drows = nullptr, *dout = nullptr;
  if ((rc = up(&dz, B.zoff.data(), sizeof(int64_t) * B.zoff.size())) ||
      (rc = up(&dm, B.moff.data(), sizeof(int64_t) * B.moff.size())) ||
      (rc = up(&dpl, B.plen.data(), sizeof(int32_t) * B.plen.size())) ||
      (rc = up(&dpar, B.parent.data(), sizeof(int32_t) * B.parent.size())) ||
      (rc = up(&dgs, B.gstart.data(), sizeof(int32_t) * B.gstart.size())) ||
      (rc = up(&dgsrc, B.gsrc.data(), sizeof(int64_t) * B.gsrc.size())) ||
      (rc = up(&dmt, B.m_tiles.data(), sizeof(peers::Tile) * B.m_tiles.size())) ||
      (rc = up(&dzt, B.z_tiles.data(), sizeof(peers::Tile) * B.z_tiles.size())) ||
      (rc = up(&dnt, B.n_tiles.data(), sizeof(peers::Tile) * B.n_tiles.size())) ||
      (rc = up(&ddsn, B.diag_sn.data(), sizeof(int32_t) * B.diag_sn.size())) ||
      (rc = up(&ddblk, B.diag_blk.data(), sizeof(int32_t) * B.diag_blk.size())) ||
      (rc = up(&dssn, B.small_sn.data(), sizeof(int32_t) * B.small_sn.size())) ||
      (rc = up(&dsch, B.small_chunk.data(), sizeof(int32_t) * B.small_chunk.size())) ||
      (rc = up(&dq, B.queries.data(), sizeof(peers::BiQuery) * B.queries.size())) ||
      (rc = up(&drows, S.rows.data(), sizeof(int32_t) * S.rows.size()))) {
    cleanup();
    return rc;
  }
  a.panel = num->panel;
  a.tinv = num->tinv;
  a.dinv = num->dinv;
  a.first = num->first;
  a.nb = num->nb;
  a.rows = static_cast<int32_t *>(drows);
  a.panel_off = num->panel_off;
  a.tinv_off = num->tinv_off;
  a.rows_off = num->rows_off;
  a.zoff = static_cast<int64_t *>(dz);
  a.moff = static_cast<int64_t *>(dm);
  a.plen = static_cast<int32_t *>(dpl);
  a.parent = static_cast<int32_t *>(dpar);
  a.gstart = static_cast<int32_t *>(dgs);
  a.gsrc = static_cast<int64_t *>(dgsrc);
  a.status = num->status;
  a.ztotal = B.ztotal;
  a.nq = S.nq;
  double *Rdev = R;
  const bool host_out = !(flags & PEERS_OUT_DEVICE);
  if (host_out) {
    rc = alloc(&dout, sizeof(double) * std::max<int64_t>(1, S.nq));
    if (rc) { cleanup(); return rc; }
    Rdev = static_cast<double *>(dout);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ctx->timing) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  int64_t launches = 0;
  std::vector<cudaEvent_t> ev;
  rc = peers::blockinv_run(S, B, a, static_cast<peers::Tile *>(dmt),
                           static_cast<peers::Tile *>(dzt), static_cast<peers::Tile *>(dnt),
                           static_cast<int32_t *>(ddsn), static_cast<int32_t *>(ddblk),
                           static_cast<int32_t *>(dssn), static_cast<int32_t *>(dsch),
                           static_cast<peers::BiQuery *>(dq),
                           Rdev, st, S.one_stream ? nullptr : ctx_lanes(ctx), &launches,
                           ctx->timing ? &ev : nullptr, err);
  if (ctx->timing) {
    // per phase: diagonal inverses, M, one entry per depth of Z blocks, query pass
    cudaStreamSynchronize(st);
    ctx->level_ms.clear();
    for (size_t i = 0; i + 1 < ev.size(); ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      ctx->level_ms.push_back(ms);
    }
    for (auto e : ev) cudaEventDestroy(e);
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
  ctx->stats.sweep_launches = launches;
  ctx->stats.h2d_bytes = 0;
  ctx->stats.d2h_bytes = 0;
  if (rc == PEERS_OK && host_out && S.nq > 0) {
    if (cudaMemcpyAsync(R, Rdev, sizeof(double) * S.nq, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess) {
      rc = PEERS_ECUDA;
      err = "result copy";
    }
    ctx->stats.d2h_bytes = int64_t(sizeof(double)) * S.nq;
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (rc == PEERS_OK && e != cudaSuccess) {
    rc = PEERS_ECUDA;
    err = cudaGetErrorString(e);
  }
  if (rc == PEERS_OK) rc = check_bounds_flag(num->status, st, "peers_query_blockinv", err);
  cleanup();
  return rc;
}

// Device buffers of one call, freed together (unless released to a longer-lived owner).
struct DevMem {
  std::vector<void *> ptrs;
  std::string *err;
  explicit DevMem(std::string *e) : err(e) {}
  ~DevMem() {
    for (void *p : ptrs) cudaFree(p);
  }
  std::vector<void *> release() {
    std::vector<void *> out;
    out.swap(ptrs);
    return out;
  }
  template <class T>
  int alloc(T **p, int64_t count) {
    void *q = nullptr;
    const size_t bytes = sizeof(T) * static_cast<size_t>(std::max<int64_t>(1, count));
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *err = "cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? PEERS_ENOMEM : PEERS_ECUDA;
    }
    ptrs.push_back(q);
    *p = static_cast<T *>(q);
    return PEERS_OK;
  }
  template <class T>
  int upload(T **p, const std::vector<T> &v, cudaStream_t st) {
    int rc = alloc(p, static_cast<int64_t>(v.size()));
    if (rc != PEERS_OK || v.empty()) return rc;
    if (cudaMemcpyAsync(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st) !=
        cudaSuccess) {
      *err = "upload";
      return PEERS_ECUDA;
    }
    return PEERS_OK;
  }
};

#define RC_TRY(x)                   \
  do {                              \
    int rc_ = (x);                  \
    if (rc_ != PEERS_OK) return rc_; \
  } while (0)

// The selected inversion's plan on the device and its working buffers for one factor: made
// by the first call and kept with the numeric handle while the plan stays the same, so that
// repeated calls neither allocate nor upload.
struct SiDevice {
  std::shared_ptr<const peers::SelInvPlan> plan;
  int device = 0;
  std::vector<void *> ptrs;
  double *Zd = nullptr, *Wd = nullptr, *M = nullptr, *F = nullptr, *Rdev = nullptr;
  int32_t *ncs = nullptr, *gsn = nullptr, *ssn = nullptr, *sch = nullptr, *dsn = nullptr,
          *dblk = nullptr, *tbs = nullptr, *tbb = nullptr, *fsn = nullptr, *par = nullptr;
  int64_t *doff = nullptr, *moff = nullptr, *foff = nullptr, *qbeg = nullptr;
  peers::Tile *bc = nullptr, *cc = nullptr, *mt = nullptr;
  peers::TinvTile *tt = nullptr;
  peers::SiQuery *qs = nullptr;
  ~SiDevice() {
    peers::DeviceGuard guard(device);
    for (void *p : ptrs) cudaFree(p);
  }
};

int si_device(peers_ctx *ctx, const Symbolic &S, const std::shared_ptr<const peers::SelInvPlan> &plan,
              std::shared_ptr<SiDevice> &out, std::string &err) {
  const peers::SelInvPlan &P = *plan;
  const cudaStream_t st = ctx->stream;
  auto d = std::make_shared<SiDevice>();
  d->plan = plan;
  d->device = ctx->device;
  DevMem mem(&err);
  RC_TRY(mem.alloc(&d->Zd, P.dtotal));
  RC_TRY(mem.alloc(&d->Wd, P.dtotal));
  RC_TRY(mem.alloc(&d->M, P.mtotal));
  RC_TRY(mem.alloc(&d->F, P.fbuf));
  RC_TRY(mem.alloc(&d->Rdev, S.nq));
  RC_TRY(mem.upload(&d->ncs, P.ncs, st));
  RC_TRY(mem.upload(&d->doff, P.doff, st));
  RC_TRY(mem.upload(&d->moff, P.moff, st));
  RC_TRY(mem.upload(&d->foff, P.foff, st));
  RC_TRY(mem.upload(&d->gsn, P.gather_sn, st));
  RC_TRY(mem.upload(&d->bc, P.bc, st));
  RC_TRY(mem.upload(&d->cc, P.cc, st));
  RC_TRY(mem.upload(&d->qs, P.queries, st));
  RC_TRY(mem.upload(&d->ssn, P.small_sn, st));
  RC_TRY(mem.upload(&d->sch, P.small_chunk, st));
  RC_TRY(mem.upload(&d->dsn, P.diag_sn, st));
  RC_TRY(mem.upload(&d->dblk, P.diag_blk, st));
  RC_TRY(mem.upload(&d->tbs, P.tbase_sn, st));
  RC_TRY(mem.upload(&d->tbb, P.tbase_blk, st));
  RC_TRY(mem.upload(&d->tt, P.tinv_tiles, st));
  RC_TRY(mem.upload(&d->mt, P.m_tiles, st));
  RC_TRY(mem.upload(&d->fsn, P.fused_sn, st));
  RC_TRY(mem.upload(&d->qbeg, S.qbeg, st));
  std::vector<int32_t> parent_host(S.parent);
  RC_TRY(mem.upload(&d->par, parent_host, st));
  CUDA_TRY(cudaStreamSynchronize(st));   // the host vectors above must outlive their copies
  d->ptrs = mem.release();
  out = d;
  return PEERS_OK;
}

int si_query(peers_ctx *ctx, const peers_symbolic *sym, peers_numeric *num, double *R, int flags,
             std::string &err) {
  const Symbolic &S = sym->S;
  cudaStream_t st = ctx->stream;
  DEVICE_SCOPE(ctx->device);
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  std::shared_ptr<const peers::SelInvPlan> plan;
  RC_TRY(peers::cached_selinv_plan(sym, sms, plan, err));
  const peers::SelInvPlan &P = *plan;
  const peers::Lanes *lanes = P.nlanes > 0 ? ctx_lanes(ctx) : nullptr;
  std::lock_guard<std::mutex> route_lock(num->route_mu);
  std::shared_ptr<SiDevice> dev = std::static_pointer_cast<SiDevice>(num->selinv_dev);
  if (!dev || dev->plan != plan) {
    num->selinv_dev.reset();
    RC_TRY(si_device(ctx, S, plan, dev, err));
    num->selinv_dev = dev;
  }
  double *Zd = dev->Zd, *Wd = dev->Wd, *M = dev->M, *F = dev->F, *Rdev = R;
  int32_t *ncs = dev->ncs, *gsn = dev->gsn, *ssn = dev->ssn, *sch = dev->sch, *dsn = dev->dsn,
          *dblk = dev->dblk, *tbs = dev->tbs, *tbb = dev->tbb, *fsn = dev->fsn, *par = dev->par;
  int64_t *doff = dev->doff, *moff = dev->moff, *foff = dev->foff, *qbeg = dev->qbeg;
  peers::Tile *bc = dev->bc, *cc = dev->cc, *mt = dev->mt;
  peers::TinvTile *tt = dev->tt;
  peers::SiQuery *qs = dev->qs;
  const bool host_out = !(flags & PEERS_OUT_DEVICE);
  if (host_out) Rdev = dev->Rdev;
  {
    int64_t need = 0;
    for (const peers::SiGroup &G : P.groups) need = std::max(need, G.fused_smem);
    static int si_small_smem[64] = {};   // limit set so far, per device
    RC_TRY(peers::raise_smem_limit(reinterpret_cast<const void *>(peers::k_si_small),
                                   si_small_smem, need, err));
  }
  // the part above the lanes (phase 1 and depths) runs on the high-priority top stream
  const cudaStream_t ts = lanes ? lanes->top : st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<cudaEvent_t> ev;
  auto mark = [&](cudaStream_t on) {
    if (ctx->timing) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      cudaEventRecord(e, on);
      ev.push_back(e);
    }
  };
  if (ctx->timing) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  int64_t launches = 0;
  if (S.nq > 0) CUDA_TRY(cudaMemsetAsync(Rdev, 0, sizeof(double) * S.nq, st));
  CUDA_TRY(cudaMemsetAsync(Zd, 0, sizeof(double) * std::max<int64_t>(1, P.dtotal), st));
  // the lanes start here (their phase 1 needs nothing of the top part)
  const int nl = lanes ? P.nlanes : 0;
  if (nl > 0) {
    CUDA_TRY(cudaEventRecord(lanes->start, st));
    CUDA_TRY(cudaStreamWaitEvent(ts, lanes->start, 0));
    for (int L = 0; L < nl; ++L) CUDA_TRY(cudaStreamWaitEvent(lanes->stream[L], lanes->start, 0));
  }
  auto stream_of = [&](int32_t lane) { return (lane >= 0 && nl > 0) ? lanes->stream[lane] : ts; };
  peers::BiArgs b{};
  b.panel = num->panel;
  b.tinv = num->tinv;
  b.dinv = num->dinv;
  b.first = num->first;
  b.nb = num->nb;
  b.panel_off = num->panel_off;
  b.tinv_off = num->tinv_off;
  b.rows_off = num->rows_off;
  b.zoff = doff;
  b.moff = moff;
  b.plen = ncs;
  b.Z = Zd;
  b.M = M;
  b.status = num->status;
  b.ztotal = P.dtotal;
  b.nq = S.nq;
  // phase 1: T^{-1} (into Zd, ld = n_c) and M, by the block inverse's kernels: the top part's
  // depth by depth on the second top stream (each depth's event releases its groups), the
  // lanes' on their own streams
  const cudaStream_t ts1 = lanes ? lanes->top1 : st;
  if (nl > 0) CUDA_TRY(cudaStreamWaitEvent(ts1, lanes->start, 0));
  std::vector<cudaEvent_t> p1_done(P.phase1.size(), nullptr);
  struct EventsGuard {
    std::vector<cudaEvent_t> &v;
    ~EventsGuard() {
      for (cudaEvent_t e : v)
        if (e) cudaEventDestroy(e);
    }
  } p1_guard{p1_done};
  std::vector<int32_t> p1_of_depth;
  bool lanes_released = false;
  for (size_t k = 0; k < P.phase1.size(); ++k) {
    const peers::SiPhase1 &ph = P.phase1[k];
    const cudaStream_t ls = ph.lane >= 0 ? stream_of(ph.lane) : ts1;
    if (ph.lane >= 0 && !lanes_released && k > 0 && p1_done[k - 1]) {
      // the lanes' phase 1 starts once the top part's is done: the top part is the critical
      // path, and its short launches would otherwise queue behind the lanes' long CTAs
      // (stream priorities order the CTAs waiting for an SM, they do not preempt running ones)
      for (int L = 0; L < nl; ++L)
        CUDA_TRY(cudaStreamWaitEvent(lanes->stream[L], p1_done[k - 1], 0));
      lanes_released = true;
    }
    if (ph.small_e > ph.small_b) {
      peers::k_bi_small<<<static_cast<unsigned>(ph.small_e - ph.small_b), 256, 0, ls>>>(
          ssn + ph.small_b, sch + ph.small_b, b);
      ++launches;
    }
    if (ph.diag_e > ph.diag_b) {
      peers::k_bi_diag<<<static_cast<unsigned>(ph.diag_e - ph.diag_b),
                         peers::kBlock * peers::kDiagSlice, 0, ls>>>(dsn + ph.diag_b,
                                                                     dblk + ph.diag_b, b);
      ++launches;
    }
    if (ph.base_e > ph.base_b) {
      peers::k_tinv_base<<<static_cast<unsigned>(ph.base_e - ph.base_b), 256, 0, ls>>>(
          tbs + ph.base_b, tbb + ph.base_b, b);
      ++launches;
    }
    for (const auto &lv : ph.tlevels) {
      RC_TRY(peers::launch_tinv_level<0>(tt, lv, b, Wd, ls, &launches, err));
      RC_TRY(peers::launch_tinv_level<1>(tt, lv, b, Wd, ls, &launches, err));
    }
    RC_TRY(peers::launch_m_all(mt, ph.m_ptr, b, ls, &launches, err));
    CUDA_TRY(cudaGetLastError());
    if (ph.lane < 0 && ts1 != ts) {
      CUDA_TRY(cudaEventCreateWithFlags(&p1_done[k], cudaEventDisableTiming));
      CUDA_TRY(cudaEventRecord(p1_done[k], ts1));
      if (p1_of_depth.size() <= size_t(ph.depth)) p1_of_depth.resize(ph.depth + 1, -1);
      p1_of_depth[ph.depth] = static_cast<int32_t>(k);
    }
  }
  // phase 2: top-down by depth, the top part first, then every lane on its own stream
  peers::SiArgs a{};
  a.dinv = num->dinv;
  a.first = num->first;
  a.nb = num->nb;
  a.rmap = num->rmap;
  a.rows_off = num->rows_off;
  a.Zd = Zd;
  a.doff = doff;
  a.M = M;
  a.moff = moff;
  a.foff = foff;
  a.parent = par;
  a.F = F;
  a.status = num->status;
  a.fbuf = P.fbuf;
  a.nq = S.nq;
  peers::SiSmallArgs sb{};
  sb.panel = num->panel;
  sb.tinv = num->tinv;
  sb.panel_off = num->panel_off;
  sb.tinv_off = num->tinv_off;
  sb.qbeg = qbeg;
  sb.qorig = num->qorig;
  sb.qa = num->qa;
  sb.qb = num->qb;
  sb.R = Rdev;
  bool top_done = nl == 0;
  for (const peers::SiGroup &G : P.groups) {
    if (G.lane >= 0 && !top_done) {
      // the lanes' first depth reads the top part's last fronts
      CUDA_TRY(cudaEventRecord(lanes->top_done, ts));
      for (int L = 0; L < nl; ++L)
        CUDA_TRY(cudaStreamWaitEvent(lanes->stream[L], lanes->top_done, 0));
      top_done = true;
    }
    const cudaStream_t gs = stream_of(G.lane);
    if (G.lane < 0 && size_t(G.depth) < p1_of_depth.size() && p1_of_depth[G.depth] >= 0)
      CUDA_TRY(cudaStreamWaitEvent(gs, p1_done[p1_of_depth[G.depth]], 0));
    if (G.fused_e > G.fused_b) {
      peers::k_si_small<<<static_cast<unsigned>(G.fused_e - G.fused_b), 256, G.fused_smem, gs>>>(
          fsn + G.fused_b, a, sb);
      ++launches;
    }
    if (G.gather_e > G.gather_b) {
      dim3 grid(static_cast<unsigned>(G.gather_e - G.gather_b),
                static_cast<unsigned>(G.gather_ych));
      peers::k_si_gather<<<grid, 256, 0, gs>>>(gsn + G.gather_b, a);
      ++launches;
    }
    for (int g = 0; g < 3; ++g) {
      const int64_t b0 = G.bc_ptr[g], b1 = G.bc_ptr[g + 1];
      if (b1 <= b0) continue;
      const unsigned n = static_cast<unsigned>(b1 - b0);
      const int rows = G.bc_rows;
      if (g == 0) peers::k_si_bc<0><<<n, rows, 0, gs>>>(bc + b0, a, rows);
      if (g == 1) peers::k_si_bc<1><<<n, rows, 0, gs>>>(bc + b0, a, rows);
      if (g == 2) peers::k_si_bc<2><<<n, rows, 0, gs>>>(bc + b0, a, rows);
      ++launches;
    }
    if (G.cc_e > G.cc_b) {
      peers::k_si_cc<<<static_cast<unsigned>(G.cc_e - G.cc_b), peers::kGemmThreads, 0, gs>>>(
          cc + G.cc_b, a);
      ++launches;
    }
    if (G.q_e > G.q_b) {
      peers::k_si_query<<<static_cast<unsigned>((G.q_e - G.q_b + 255) / 256), 256, 0, gs>>>(
          qs + G.q_b, G.q_e - G.q_b, a, Rdev);
      ++launches;
    }
    CUDA_TRY(cudaGetLastError());
    if (G.lane < 0) mark(ts);
  }
  if (nl > 0) {
    CUDA_TRY(cudaEventRecord(lanes->top_done, ts));
    CUDA_TRY(cudaStreamWaitEvent(st, lanes->top_done, 0));
    CUDA_TRY(cudaEventRecord(lanes->top_done, ts1));
    CUDA_TRY(cudaStreamWaitEvent(st, lanes->top_done, 0));
    for (int L = 0; L < nl; ++L) {
      CUDA_TRY(cudaEventRecord(lanes->done[L], lanes->stream[L]));
      CUDA_TRY(cudaStreamWaitEvent(st, lanes->done[L], 0));
    }
    mark(st);
  }
  if (ctx->timing) {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ctx->stats.sweep_s = ms * 1e-3;
    // each depth of the top part (with the wait for its phase 1, which runs beside the
    // depths above it), and the lanes' subtrees (concurrent streams) as one entry
    ctx->level_ms.clear();
    cudaEventElapsedTime(&ms, e0, ev[0]);
    ctx->level_ms.push_back(ms);
    for (size_t i = 0; i + 1 < ev.size(); ++i) {
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      ctx->level_ms.push_back(ms);
    }
    for (auto e : ev) cudaEventDestroy(e);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  ctx->stats.sweep_launches = launches;
  ctx->stats.h2d_bytes = 0;
  ctx->stats.d2h_bytes = 0;
  if (host_out && S.nq > 0) {
    CUDA_TRY(cudaMemcpyAsync(R, Rdev, sizeof(double) * S.nq, cudaMemcpyDeviceToHost, st));
    ctx->stats.d2h_bytes = int64_t(sizeof(double)) * S.nq;
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  return check_bounds_flag(num->status, st, "peers_query_selinv", err);
}

}  // namespace

extern "C" {

int64_t peers_blockinv_bytes(const peers_symbolic *sym) {
  if (!sym) return -1;
  std::shared_ptr<const peers::BlockInvPlan> plan;
  std::string err;
  if (peers::cached_blockinv_plan(sym, plan, err) != PEERS_OK) return -1;
  const peers::BlockInvPlan &B = *plan;
  return 8 * (B.ztotal + B.mtotal) + 12 * static_cast<int64_t>(B.gstart.size()) +
         16 * static_cast<int64_t>(B.z_tiles.size() + B.n_tiles.size() + B.m_tiles.size()) +
         24 * static_cast<int64_t>(B.queries.size());
}

int64_t peers_blockinv_fma(const peers_symbolic *sym) {
  if (!sym) return -1;
  std::shared_ptr<const peers::BlockInvPlan> plan;
  std::string err;
  if (peers::cached_blockinv_plan(sym, plan, err) != PEERS_OK) return -1;
  return plan->gemm_fma;
}

int peers_query_selinv(peers_ctx *ctx, const peers_symbolic *sym, const peers_numeric *num,
                       double *R, int flags) {
  if (!ctx || !sym || !num || (!R && sym->S.nq > 0)) return peers_fail(PEERS_EINVAL, "null argument");
  if (num->sym != sym) return peers_fail(PEERS_EINVAL, "numeric handle belongs to another plan");
  if (num->device != ctx->device) return peers_fail(PEERS_EINVAL, "context on another device");
  std::string err;
  int rc = PEERS_OK;
  if ((flags & PEERS_OUT_DEVICE) && sym->S.nq > 0) {
    peers::DeviceGuard guard(ctx->device);
    rc = peers::check_device_result(ctx->device, R, err);
  }
  if (rc == PEERS_OK) rc = si_query(ctx, sym, const_cast<peers_numeric *>(num), R, flags, err);
  return rc == PEERS_OK ? rc : peers_fail(rc, err);
}

int64_t peers_selinv_fma(const peers_symbolic *sym) {
  if (!sym) return -1;
  // the work does not depend on the SM count: any cached plan (or one for 148 SMs) serves
  std::shared_ptr<const peers::SelInvPlan> plan;
  std::string err;
  if (peers::cached_selinv_plan(sym, 0, plan, err) != PEERS_OK) return -1;
  return plan->fma;
}

int peers_query_blockinv(peers_ctx *ctx, const peers_symbolic *sym, const peers_numeric *num,
                         double *R, int flags) {
  if (!ctx || !sym || !num || (!R && sym->S.nq > 0)) return peers_fail(PEERS_EINVAL, "null argument");
  if (num->sym != sym) return peers_fail(PEERS_EINVAL, "numeric handle belongs to another plan");
  if (num->device != ctx->device) return peers_fail(PEERS_EINVAL, "context on another device");
  std::string err;
  int rc = PEERS_OK;
  if ((flags & PEERS_OUT_DEVICE) && sym->S.nq > 0) {
    peers::DeviceGuard guard(ctx->device);
    rc = peers::check_device_result(ctx->device, R, err);
  }
  if (rc == PEERS_OK) rc = bi_query(ctx, sym, const_cast<peers_numeric *>(num), R, flags, err);
  return rc == PEERS_OK ? rc : peers_fail(rc, err);
}

}  // extern "C"
