// FP64 throughput probes: the denominators of the FP64 roofline that the plain (DFMA) path and the
// split-BF16 emulation are compared against.  Not part of Algorithm 1.
//
//   which = 0: DFMA on the CUDA cores (fma.rn.f64), 8 independent chains per thread;
//   which = 1: DMMA on the tensor cores (mma.sync m8n8k4 f64), 4 independent accumulators per warp.
// Grid: 4 blocks of 256 threads per SM.  Timed with CUDA events around one launch after a warm-up
// launch; flops counted as 2 per FMA.
#include <cuda_runtime.h>

#include "../../include/chase_gb300.h"
#include "common.cuh"

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 4;

// written only when a result equals an impossible value: keeps every chain's result live
__device__ double g_peak_sink;

__global__ void __launch_bounds__(PEAK_THREADS) dfma_probe_kernel(int iters, double seed) {
  double a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = seed + 1e-3 * (threadIdx.x + j);
  const double b = 0.999999, c = 1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == 12345.678) g_peak_sink = s;
}

__global__ void __launch_bounds__(PEAK_THREADS) dmma_probe_kernel(int iters, double seed) {
  double av = seed + 1e-3 * threadIdx.x, bv = 0.5 - 1e-4 * threadIdx.x;
  double c[4][2];
#pragma unroll
  for (int j = 0; j < 4; ++j) c[j][0] = c[j][1] = 0.0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                     : "+d"(c[j][0]), "+d"(c[j][1])
                     : "d"(av), "d"(bv));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) s += c[j][0] + c[j][1];
  if (s == 12345.678) g_peak_sink = s;
}

}  // namespace

extern "C" chase_status chase_measure_fp64_peak(int which, double* tflops_out, double* ms_out) {
  if (!tflops_out || (which != 0 && which != 1)) return CHASE_ERR_ARG;
  try {
    int dev = 0, sms = 0;
    CHASE_CUDA(cudaGetDevice(&dev));
    CHASE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * PEAK_BLOCKS_PER_SM;
    const int iters = which == 0 ? 4096 : 2048;
    cudaStream_t st = nullptr;
    CHASE_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CHASE_CUDA(cudaEventCreate(&e0));
    CHASE_CUDA(cudaEventCreate(&e1));
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
      CHASE_CUDA(cudaEventRecord(e0, st));
      if (which == 0)
        dfma_probe_kernel<<<blocks, PEAK_THREADS, 0, st>>>(iters, 1.0);
      else
        dmma_probe_kernel<<<blocks, PEAK_THREADS, 0, st>>>(iters, 1.0);
      CHASE_CHECK_LAUNCH();
      CHASE_CUDA(cudaEventRecord(e1, st));
      CHASE_CUDA(cudaEventSynchronize(e1));
      CHASE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    const double threads = (double)blocks * PEAK_THREADS;
    // DFMA: 16 x 8 FMAs per thread and iteration; DMMA: 16 m8n8k4 MMAs (256 FMAs each) per warp and iteration
    const double fmas = which == 0 ? threads * iters * 16.0 * 8.0 : (threads / 32.0) * iters * 16.0 * 256.0;
    *tflops_out = 2.0 * fmas / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
  } catch (const chase::Error& e) {
    return (chase_status)e.status;
  }
  return CHASE_OK;
}
