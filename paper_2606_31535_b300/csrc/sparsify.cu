// Spectral sparsification by effective resistances (PEERS §II-B, Alg. 1): q edges are drawn
// with probability proportional to w_e R_e and each draw adds w_e / (q p_e) to its edge.
//
// The draws are made bit-reproducible: every score w_e R_e is quantised once, in FP64, to an
// integer weight k_e = floor(w_e R_e * S) with S = floor(2^62 / m) / max_e(w_e R_e), so the
// cumulative weights are exact int64 sums (no rounding order) and p_e = k_e / K.  Draw i, with
// the caller's uniform u_i in [0, 1), picks the first edge whose cumulative weight exceeds
// floor(u_i K).  Counts are integer atomics, so the result does not depend on thread order.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "device.cuh"
#include "handles.h"
#include "internal.h"
#include "peers.h"

namespace peers {
namespace {

constexpr int kScanBlock = 1024;

__global__ void k_sp_score_max(const double *__restrict__ w, const double *__restrict__ R,
                               int64_t m, unsigned long long *bits_max) {
  // max over non-negative doubles == max over their bit patterns as unsigned integers
  unsigned long long best = 0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < m;
       e += int64_t(gridDim.x) * blockDim.x) {
    const double s = w[e] * R[e];
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(s > 0 ? s : 0.0));
    best = b > best ? b : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, best, o);
    best = x > best ? x : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(bits_max, best);
}

// k_e = floor(w_e R_e * S); block sums of k.
__global__ void k_sp_quantise(const double *__restrict__ w, const double *__restrict__ R,
                              int64_t m, const unsigned long long *bits_max, double scale_num,
                              long long *k, long long *block_sum) {
  __shared__ long long part[kScanBlock / 32];
  const double smax = __longlong_as_double(static_cast<long long>(*bits_max));
  const double S = smax > 0 ? scale_num / smax : 0.0;
  const int64_t e = blockIdx.x * int64_t(kScanBlock) + threadIdx.x;
  long long v = 0;
  if (e < m) {
    const double s = w[e] * R[e];
    v = s > 0 ? static_cast<long long>(floor(s * S)) : 0;
    k[e] = v;
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x / 32] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int i = 0; i < kScanBlock / 32; ++i) t += part[i];
    block_sum[blockIdx.x] = t;
  }
}

// Exclusive scan of the block sums in one CTA (sequential over chunks; exact integers).
__global__ void k_sp_scan_blocks(long long *block_sum, int64_t nb, long long *total) {
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    long long v = i < nb ? block_sum[i] : 0;
    // inclusive warp scan, then across warps
    __shared__ long long warp_tot[32];
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x / 32] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      long long t = threadIdx.x < blockDim.x / 32 ? warp_tot[threadIdx.x] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, t, o);
        if (threadIdx.x >= o) t += y;
      }
      warp_tot[threadIdx.x] = t;
    }
    __syncthreads();
    const long long before = (threadIdx.x >= 32 ? warp_tot[threadIdx.x / 32 - 1] : 0) + x - v;
    if (i < nb) block_sum[i] = carry + before;   // exclusive
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += before + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Inclusive cumulative weights: C_e = (exclusive block offset) + inclusive scan within block.
__global__ void k_sp_cumulate(long long *k, int64_t m, const long long *block_off) {
  __shared__ long long warp_tot[kScanBlock / 32];
  const int64_t e = blockIdx.x * int64_t(kScanBlock) + threadIdx.x;
  long long v = e < m ? k[e] : 0;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) >= o) x += y;
  }
  if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x / 32] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    long long t = warp_tot[threadIdx.x];
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (threadIdx.x >= o) t += y;
    }
    warp_tot[threadIdx.x] = t;
  }
  __syncthreads();
  const long long incl = (threadIdx.x >= 32 ? warp_tot[threadIdx.x / 32 - 1] : 0) + x;
  if (e < m) k[e] = block_off[blockIdx.x] + incl;
}

// Draw i: the first edge whose cumulative weight exceeds floor(u_i K).
__global__ void k_sp_draw(const long long *__restrict__ C, int64_t m, const double *__restrict__ u,
                          int64_t q, const long long *total, unsigned long long *count) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= q) return;
  const long long K = *total;
  if (K <= 0) return;
  long long t = static_cast<long long>(floor(u[i] * static_cast<double>(K)));
  if (t >= K) t = K - 1;
  if (t < 0) t = 0;
  int64_t lo = 0, hi = m;   // first index with C > t
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (C[mid] > t) hi = mid; else lo = mid + 1;
  }
  if (lo < m) atomicAdd(count + lo, 1ull);
}

// weight_e = count_e * w_e / (q p_e) with p_e = k_e / K (k_e recovered from the cumulative).
__global__ void k_sp_weights(const long long *__restrict__ C, const double *__restrict__ w,
                             int64_t m, int64_t q, const long long *total,
                             const unsigned long long *count, double *weight) {
  const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= m) return;
  const long long ke = C[e] - (e > 0 ? C[e - 1] : 0);
  const unsigned long long c = count[e];
  weight[e] = (c == 0 || ke == 0)
                  ? 0.0
                  : static_cast<double>(c) * w[e] * static_cast<double>(*total) /
                        (static_cast<double>(q) * static_cast<double>(ke));
}

}  // namespace
}  // namespace peers

extern "C" int peers_sparsify(peers_ctx *ctx, int64_t m, const double *w, const double *R,
                              int64_t q, const double *u, int64_t *count, double *weight) {
  if (!ctx || m < 1 || q < 0 || !w || !R || (!u && q > 0) || !count || !weight)
    return peers_fail(PEERS_EINVAL, "null argument or empty edge set");
  std::string err;
  auto run = [&]() -> int {
    DEVICE_SCOPE(ctx->device);
    cudaStream_t st = ctx->stream;
    const int64_t nb = (m + peers::kScanBlock - 1) / peers::kScanBlock;
    long long *C = nullptr, *bsum = nullptr, *total = nullptr;
    unsigned long long *bits = nullptr;
    CUDA_TRY(cudaMalloc(&C, sizeof(long long) * m));
    cudaError_t e = cudaMalloc(&bsum, sizeof(long long) * nb);
    if (e == cudaSuccess) e = cudaMalloc(&total, sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&bits, sizeof(unsigned long long));
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(C);
      cudaFree(bsum);
      cudaFree(total);
      err = "sparsify scratch";
      return PEERS_ENOMEM;
    }
    const double scale_num = std::floor(std::ldexp(1.0, 62) / static_cast<double>(m));
    cudaMemsetAsync(bits, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(count, 0, sizeof(int64_t) * m, st);
    peers::k_sp_score_max<<<148 * 4, 256, 0, st>>>(w, R, m, bits);
    peers::k_sp_quantise<<<static_cast<unsigned>(nb), peers::kScanBlock, 0, st>>>(
        w, R, m, bits, scale_num, C, bsum);
    peers::k_sp_scan_blocks<<<1, 1024, 0, st>>>(bsum, nb, total);
    peers::k_sp_cumulate<<<static_cast<unsigned>(nb), peers::kScanBlock, 0, st>>>(C, m, bsum);
    if (q > 0)
      peers::k_sp_draw<<<static_cast<unsigned>((q + 255) / 256), 256, 0, st>>>(
          C, m, u, q, total, reinterpret_cast<unsigned long long *>(count));
    peers::k_sp_weights<<<static_cast<unsigned>((m + 255) / 256), 256, 0, st>>>(
        C, w, m, q, total, reinterpret_cast<const unsigned long long *>(count), weight);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(C);
    cudaFree(bsum);
    cudaFree(total);
    cudaFree(bits);
    if (e != cudaSuccess) {
      err = cudaGetErrorString(e);
      return PEERS_ECUDA;
    }
    return PEERS_OK;
  };
  const int rc = run();
  return rc == PEERS_OK ? rc : peers_fail(rc, err);
}
