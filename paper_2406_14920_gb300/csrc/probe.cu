// Peak arithmetic probe: the FP64 DFMA and FP32 FFMA rates this GPU sustains,
// the denominators of the ALU roofline of the ERI kernels (which are bound by
// those pipes, not by HBM).  Each thread runs CHAINS independent fused
// multiply-add chains (enough to hide the pipe latency) for a fixed number of
// iterations; the grid fills every SM with several resident blocks.  The
// result is stored once per thread so the compiler cannot drop the chains.
#include <cuda_runtime.h>

#include "../../include/eri.h"

namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kBlock) k_fma_probe(int iters, T a, T b, T* out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int probe(int iters, cudaStream_t s, double* tflops) {
  int dev = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ERI_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ERI_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_probe<T>, kBlock, 0) != cudaSuccess) return ERI_ECUDA;
  const int grid = nsm * (occ > 0 ? occ : 1);
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)grid * kBlock) != cudaSuccess) return ERI_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = ERI_OK;
  float ms = 0.0f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = ERI_ECUDA;
  if (rc == ERI_OK) {
    // x <- x * a + b with |a| < 1 stays finite for any iteration count
    k_fma_probe<T><<<grid, kBlock, 0, s>>>(iters / 8 + 1, T(0.999), T(1e-3), out);  // warm-up
    cudaEventRecord(e0, s);
    k_fma_probe<T><<<grid, kBlock, 0, s>>>(iters, T(0.999), T(1e-3), out);
    cudaEventRecord(e1, s);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.0f)
      rc = ERI_ECUDA;
  }
  if (rc == ERI_OK) *tflops = 2.0 * kChains * (double)iters * grid * kBlock / (ms * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

}  // namespace

extern "C" int eri_peak_probe(int32_t precision, int32_t iters, double* tflops, void* stream) {
  if (!tflops || iters < 1 || (precision != ERI_FP64 && precision != ERI_MIXED)) return ERI_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  return precision == ERI_FP64 ? probe<double>(iters, s, tflops) : probe<float>(iters, s, tflops);
}
