// FP64 throughput of the device, measured with register-only kernels: the sweep's roofline
// denominator.  Three figures: DFMA on the CUDA cores, mma.sync m8n8k4 f64 (the FP64 tensor
// path), and both issued at once by alternate warps of one kernel.  The third says whether
// the two draw on separate hardware (it would then approach the sum of the first two) or on
// one FP64 unit (it stays near the larger of the two).  A second probe times every shape of
// the f64 mma.sync (m8n8k4, m16n8k4, m16n8k8, m16n8k16): the larger shapes carry more
// multiply-adds per instruction, so they would show an FP64 tensor rate that the smallest
// shape's issue rate hides.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "device.cuh"

namespace peers {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kDfmaChains = 8;   // independent accumulators per thread
constexpr int kDfmaDepth = 8;    // FMAs per chain per iteration
constexpr int kMmaChains = 8;    // independent m8n8k4 accumulators per warp

__device__ __forceinline__ void dmma_m8n8k4(double &d0, double &d1, double x, double y) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(x), "d"(y));
}

// MODE 0: every warp runs DFMA chains; 1: every warp runs m8n8k4 chains; 2: even warps DFMA,
// odd warps m8n8k4.
template <int MODE>
__global__ void __launch_bounds__(kPeakThreads) k_fp64_peak(double *out, int iters, double b,
                                                            double c) {
  const bool mma = MODE == 1 || (MODE == 2 && ((threadIdx.x >> 5) & 1));
  double acc[2 * kMmaChains];
#pragma unroll
  for (int i = 0; i < 2 * kMmaChains; ++i) acc[i] = threadIdx.x + i;
  if (mma) {
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int j = 0; j < kMmaChains; ++j) dmma_m8n8k4(acc[2 * j], acc[2 * j + 1], b, c);
    }
  } else {
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int d = 0; d < kDfmaDepth; ++d)
#pragma unroll
        for (int j = 0; j < kDfmaChains; ++j) acc[j] = fma(acc[j], b, c);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 2 * kMmaChains; ++i) s += acc[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The larger f64 mma.sync shapes (sm_90 and later).  Fragments per thread: m16n8k4 A 2, B 1,
// C/D 4; m16n8k8 A 4, B 2, C/D 4; m16n8k16 A 8, B 4, C/D 4 doubles.
__device__ __forceinline__ void dmma_m16n8k4(double (&d)[4], double a, double b) {
  asm volatile(
      "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};\n"
      : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
      : "d"(a), "d"(a), "d"(b));
}
__device__ __forceinline__ void dmma_m16n8k8(double (&d)[4], double a, double b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
      : "d"(a), "d"(a), "d"(a), "d"(a), "d"(b), "d"(b));
}
__device__ __forceinline__ void dmma_m16n8k16(double (&d)[4], double a, double b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
      : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
      : "d"(a), "d"(a), "d"(a), "d"(a), "d"(a), "d"(a), "d"(a), "d"(a), "d"(b), "d"(b),
        "d"(b), "d"(b));
}

// SHAPE 1: m16n8k4, 2: m16n8k8, 3: m16n8k16; kMmaChains independent accumulators per warp.
template <int SHAPE>
__global__ void __launch_bounds__(kPeakThreads) k_fp64_mma_shape(double *out, int iters,
                                                                 double a, double b) {
  double acc[kMmaChains][4];
#pragma unroll
  for (int j = 0; j < kMmaChains; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[j][i] = threadIdx.x + j + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kMmaChains; ++j) {
      if (SHAPE == 1) dmma_m16n8k4(acc[j], a, b);
      else if (SHAPE == 2) dmma_m16n8k8(acc[j], a, b);
      else dmma_m16n8k16(acc[j], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kMmaChains; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) s += acc[j][i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// flops one warp does per iteration
constexpr double kDfmaWarpFlops = 2.0 * 32 * kDfmaChains * kDfmaDepth;
constexpr double kMmaWarpFlops = 2.0 * 8 * 8 * 4 * kMmaChains;

template <int MODE>
int time_mode(cudaStream_t stream, double *out, int blocks, int iters, double *tflops,
              std::string &err) {
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  // the MMA chains start from 1.0 * 1.0 products; the DFMA chains stay near their start values
  const double b = MODE == 1 ? 1.0 : 1.0000001, c = MODE == 1 ? 1.0 : 1e-9;
  float best = 0.0f;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, stream);
    k_fp64_peak<MODE><<<blocks, kPeakThreads, 0, stream>>>(out, iters, b, c);
    cudaEventRecord(e1, stream);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms > 0.0f) best = best == 0.0f ? ms : std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return PEERS_ECUDA;
  }
  const double warps = double(blocks) * (kPeakThreads / 32);
  const double per_iter = MODE == 0 ? warps * kDfmaWarpFlops
                          : MODE == 1 ? warps * kMmaWarpFlops
                                      : warps / 2 * (kDfmaWarpFlops + kMmaWarpFlops);
  *tflops = best > 0.0f ? per_iter * iters / (double(best) * 1e9) : 0.0;
  return PEERS_OK;
}

// Best-of-3 TFLOP/s of k_fp64_mma_shape<SHAPE> (after one untimed launch).
template <int SHAPE>
int time_shape(cudaStream_t stream, double *out, int blocks, int iters, double *tflops,
               std::string &err) {
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float best = 0.0f;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, stream);
    k_fp64_mma_shape<SHAPE><<<blocks, kPeakThreads, 0, stream>>>(out, iters, 1.0, 1.0);
    cudaEventRecord(e1, stream);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms > 0.0f) best = best == 0.0f ? ms : std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return PEERS_ECUDA;
  }
  const double k = SHAPE == 1 ? 4 : SHAPE == 2 ? 8 : 16;
  const double warp_flops = 2.0 * 16 * 8 * k * kMmaChains;
  const double warps = double(blocks) * (kPeakThreads / 32);
  *tflops = best > 0.0f ? warps * warp_flops * iters / (double(best) * 1e9) : 0.0;
  return PEERS_OK;
}

}  // namespace

int fp64_mma_shapes(cudaStream_t stream, double out4[4], std::string &err) {
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 4;
  double *out = nullptr;
  CUDA_TRY(cudaMalloc(&out, sizeof(double) * blocks * kPeakThreads));
  int rc = time_mode<1>(stream, out, blocks, 1024, &out4[0], err);
  if (rc == PEERS_OK) rc = time_shape<1>(stream, out, blocks, 512, &out4[1], err);
  if (rc == PEERS_OK) rc = time_shape<2>(stream, out, blocks, 256, &out4[2], err);
  if (rc == PEERS_OK) rc = time_shape<3>(stream, out, blocks, 128, &out4[3], err);
  cudaFree(out);
  return rc;
}

int fp64_peak(cudaStream_t stream, double out3[3], std::string &err) {
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 4;
  double *out = nullptr;
  CUDA_TRY(cudaMalloc(&out, sizeof(double) * blocks * kPeakThreads));
  int rc = time_mode<0>(stream, out, blocks, 512, &out3[0], err);
  if (rc == PEERS_OK) rc = time_mode<1>(stream, out, blocks, 1024, &out3[1], err);
  if (rc == PEERS_OK) rc = time_mode<2>(stream, out, blocks, 768, &out3[2], err);
  cudaFree(out);
  return rc;
}

}  // namespace peers
