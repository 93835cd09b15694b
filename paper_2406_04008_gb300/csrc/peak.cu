// collage_fp32_peak: the FP32 FMA throughput of the current device, measured.
//
// The distance kernel's roofline is the FP32 pipe (nothing on the path is a dense contraction), and
// the device's copy bandwidth and tensor-core peaks say nothing about it.  This kernel runs eight
// independent FMA chains per thread at full occupancy; the rate it reaches is the denominator the
// benchmark reports the distance kernel against.
#include "collage.h"
#include "internal.h"

namespace collage {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float* out, int iters, float m, float c) {
  float a[kPeakChains];
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) a[i] = (float)threadIdx.x * 1e-3f + (float)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kPeakChains; ++i) a[i] = fmaf(a[i], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) s += a[i];
  if (s == -1.0f) out[blockIdx.x] = s;  // never taken for m, c near (1, 0): keeps the chains live
}

}  // namespace collage

extern "C" collage_status collage_fp32_peak(void* stream, float* h_tflops) {
  using namespace collage;
  if (!h_tflops) return COLLAGE_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak, kPeakThreads, 0) != cudaSuccess)
    return COLLAGE_ERR_CUDA;
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  const int iters = 4096;
  float* out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  collage_status st = COLLAGE_OK;
  if (cudaMalloc(&out, sizeof(float) * grid) != cudaSuccess) return COLLAGE_ERR_OOM;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) st = COLLAGE_ERR_CUDA;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && st == COLLAGE_OK; ++rep) {  // the first launch is a warm-up
    cudaEventRecord(a, s);
    k_fma_peak<<<grid, kPeakThreads, 0, s>>>(out, iters, 0.9999999f, 1e-7f);
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) {
      st = COLLAGE_ERR_CUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    if (rep > 0 && ms < best) best = ms;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  if (st) return st;
  const double flops = 2.0 * (double)grid * kPeakThreads * iters * kPeakUnroll * kPeakChains;
  *h_tflops = (float)(flops / (best * 1e-3) / 1e12);
  return COLLAGE_OK;
}
