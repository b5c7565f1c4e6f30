// Measured arithmetic roof of the GPU: fused multiply-add throughput in FP64 and FP32.
//
// The paper has no counterpart.  The solver's kernels are bound by HBM bandwidth when the
// state streams in FP32, and by the FP64 pipe (or by issue) when it lives on chip or runs in
// FP64; the roofline fraction of those kernels is reported against the rate this kernel
// measures on the same GPU, at whatever clock the GPU runs (no clock is set here).
//
// Every thread runs BQ_PEAK_CHAINS independent dependent chains a <- a * b + c, unrolled so
// that the loop counter costs a small fraction of an issue slot per FMA; the grid holds
// several CTAs of 256 threads per SM so that the chains' latency is hidden.
#include <cuda_runtime.h>

#include "bq.h"

#define BQ_PEAK_CHAINS 16
#define BQ_PEAK_UNROLL 8
#define BQ_PEAK_THREADS 256
#define BQ_PEAK_CTAS_PER_SM 4

namespace {

// written only if a chain ever reaches -1, which the host's arguments rule out; it keeps the
// chains from being removed without giving the kernel an output buffer
__device__ double g_peak_sink;

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(BQ_PEAK_THREADS) k_fma_peak(long long iters, T b, T c) {
  T a[BQ_PEAK_CHAINS];
#pragma unroll
  for (int i = 0; i < BQ_PEAK_CHAINS; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < BQ_PEAK_UNROLL; ++u)
#pragma unroll
      for (int i = 0; i < BQ_PEAK_CHAINS; ++i) a[i] = fma_t<T>(a[i], b, c);
  }
  T s = (T)0;
#pragma unroll
  for (int i = 0; i < BQ_PEAK_CHAINS; ++i) s += a[i];
  // never true for the arguments the host passes: every chain starts in [0, 0.3] and moves
  // towards c / (1 - b) = 1
  if (s == (T)-1.0) g_peak_sink = (double)s;
}

template <typename T>
int run_peak(long long iters, double* fma_per_s, cudaStream_t st) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BQ_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return BQ_ECUDA;
  const int grid = nsm * BQ_PEAK_CTAS_PER_SM;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return BQ_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return BQ_ECUDA; }
  int rc = BQ_OK;
  k_fma_peak<T><<<grid, BQ_PEAK_THREADS, 0, st>>>(1, (T)0.9999999, (T)1e-7);  // warm-up
  cudaEventRecord(e0, st);
  k_fma_peak<T><<<grid, BQ_PEAK_THREADS, 0, st>>>(iters, (T)0.9999999, (T)1e-7);
  cudaEventRecord(e1, st);
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
    rc = BQ_ECUDA;
  } else {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double n_fma = (double)grid * BQ_PEAK_THREADS * BQ_PEAK_CHAINS * BQ_PEAK_UNROLL * (double)iters;
    *fma_per_s = ms > 0.f ? n_fma / (ms * 1e-3) : 0.0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace

extern "C" int bq_fma_peak(int dtype, int64_t iters, double* fma_per_s, void* stream) {
  if (!fma_per_s || iters < 1 || (dtype != BQ_F64 && dtype != BQ_F32)) return BQ_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  return dtype == BQ_F64 ? run_peak<double>((long long)iters, fma_per_s, st)
                         : run_peak<float>((long long)iters, fma_per_s, st);
}
