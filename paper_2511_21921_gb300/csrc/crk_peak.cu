// crk_peak.cu -- FMA-chain microbenchmarks: the FP32 and FP64 arithmetic rates
// of the GPU the library runs on, measured with the same clocks and power
// state as the pair sweeps.  The pair sweeps are bound by the FP32 pipes, so
// their roofline denominator is the FP32 FMA rate; the FP64 rate explains why
// the mixed-precision path avoids FP64 in its inner loops.
//
// Every thread runs ILP independent chains x <- x a + b (one fused multiply-add
// = 2 flops each); a, b are runtime values, so nothing folds, and the chains
// converge to b / (1 - a) instead of overflowing.  The grid fills every SM
// with 8 blocks of 256 threads.
#include <cuda_runtime.h>

#include "crk.h"

namespace {

constexpr int kPeakIlp = 8;
constexpr int kPeakUnroll = 16;
constexpr int kPeakBlock = 256;
constexpr int kPeakBlocksPerSm = 8;

__device__ __forceinline__ float fma_(float x, float a, float b) { return fmaf(x, a, b); }
__device__ __forceinline__ double fma_(double x, double a, double b) { return fma(x, a, b); }

template <class T>
__global__ void __launch_bounds__(kPeakBlock) k_fma_chain(int iters, T a, T b, T* out) {
  T x[kPeakIlp];
#pragma unroll
  for (int k = 0; k < kPeakIlp; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kPeakIlp; ++k) x[k] = fma_(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kPeakIlp; ++k) s += x[k];
  // never true for the values above; keeps every chain live
  if (s == T(-1)) out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T> crk_status run(cudaStream_t st, int iters, double* fps, double* ms_out) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return CRK_ECUDA;
  const unsigned grid = (unsigned)(sms * kPeakBlocksPerSm);
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * grid * kPeakBlock) != cudaSuccess) return CRK_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  crk_status rc = CRK_OK;
  double best = 0.0, best_ms = 0.0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = CRK_ECUDA;
  } else {
    const T a = T(0.9999), b = T(1e-4);
    k_fma_chain<T><<<grid, kPeakBlock, 0, st>>>(iters, a, b, out);  // warm-up
    for (int rep = 0; rep < 3 && rc == CRK_OK; ++rep) {
      cudaEventRecord(e0, st);
      k_fma_chain<T><<<grid, kPeakBlock, 0, st>>>(iters, a, b, out);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
          !(ms > 0.f)) {
        rc = CRK_ECUDA;
        break;
      }
      const double flops =
          2.0 * (double)grid * kPeakBlock * (double)iters * kPeakUnroll * kPeakIlp;
      const double r = flops / (ms * 1e-3);
      if (r > best) best = r, best_ms = ms;
    }
  }
  if (rc == CRK_OK && cudaGetLastError() != cudaSuccess) rc = CRK_ECUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc == CRK_OK) {
    *fps = best;
    if (ms_out) *ms_out = best_ms;
  }
  return rc;
}

}  // namespace

extern "C" crk_status crk_alu_peak(crk_stream_t stream, int32_t fp64, int32_t iters,
                                   double* flops_per_s, double* ms) {
  if (!flops_per_s || iters <= 0 || (fp64 != 0 && fp64 != 1)) return CRK_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return fp64 ? run<double>(st, iters, flops_per_s, ms) : run<float>(st, iters, flops_per_s, ms);
}
