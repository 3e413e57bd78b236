// Throughput probes (not part of Algorithm 1):
//  - FP64: the denominators of the FP64 roofline that the plain (DFMA) path and the split-BF16 emulation are
//    compared against;
//  - tcgen05 issue rate: cycles per MMA of the split-product kernel's issue pattern, alone and with the
//    synchronisation the kernel needs (commits, distinct operand tiles, barrier checks), which bounds it.
//
//   which = 0: DFMA on the CUDA cores (fma.rn.f64), 8 independent chains per thread;
//   which = 1: DMMA on the tensor cores (mma.sync m8n8k4 f64), 4 independent accumulators per warp.
// Grid: 4 blocks of 256 threads per SM.  Timed with CUDA events around one launch after a warm-up
// launch; flops counted as 2 per FMA.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "tcgen05.cuh"

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

// ---------------------------------------------------------------- tcgen05 issue-rate probe
// One CTA per SM; one thread issues `iters` repetitions of the FP64 filter's per-k-block pattern: 7 left slices
// t (descending), per slice two left planes x two K-steps x the right slices u with t + u <= 6, MMA M = 128,
// width N, K = 16 (28 pairs, 112 MMAs).  Operands are zero; only time matters.  VAR bits: 1 a tcgen05.commit
// after each slice, 2 a distinct left tile per slice, 4 an mbarrier test (already complete) before each slice,
// 8 no A-collector hints.  Accumulator of a pair: level t + u modulo the accumulators that fit 512 columns.
namespace {

constexpr int PROBE_S = 7;
constexpr int PROBE_THREADS = 128;

template <int COL, int N>
__device__ __forceinline__ void probe_mma(uint32_t d, uint64_t a, uint64_t b) {
  chase::oz::mma_bf16_c<COL>(d, a, b, chase::oz::idesc_bf16(128, N), 1u);
}

template <int N, int VAR>
__global__ void __launch_bounds__(PROBE_THREADS) mma_issue_probe_kernel(int iters, unsigned long long* cycles, int* err) {
  constexpr int NACC = 512 / N < 6 ? 512 / N : 6;
  constexpr int A_BYTES = (VAR & 2) ? PROBE_S * 16384 : 16384;
  extern __shared__ __align__(1024) unsigned char probe_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)probe_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm;
  unsigned char* sB = sm + A_BYTES;  // PROBE_S slices x N rows x 64 bytes
  __shared__ __align__(8) uint64_t bar_done, bar_commit, bar_ready;
  __shared__ uint32_t tslot;
  for (int i = threadIdx.x; i < (A_BYTES + PROBE_S * N * 64) / 16; i += blockDim.x)
    ((uint4*)sm)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    chase::oz::mbar_init(chase::oz::smem_u32(&bar_done), 1);
    chase::oz::mbar_init(chase::oz::smem_u32(&bar_commit), (1u << 20) - 1);  // never completes: commits only arrive
    chase::oz::mbar_init(chase::oz::smem_u32(&bar_ready), 1);
    chase::oz::mbar_arrive(chase::oz::smem_u32(&bar_ready));  // phase 0 complete: the tests below succeed at once
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(chase::oz::smem_u32(&tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  chase::oz::fence_before();
  __syncthreads();
  chase::oz::fence_after();
  const uint32_t tmem = tslot;
  if (threadIdx.x == 32) {
    const uint64_t bd = chase::oz::sw64_desc(chase::oz::smem_u32(sB));
    const long long c0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int t = PROBE_S - 1; t >= 0; --t) {
        if (VAR & 4) {
          uint32_t ok = 0;
          for (int g = 0; !ok && g < (1 << 20); ++g) ok = chase::oz::mbar_try(chase::oz::smem_u32(&bar_ready), 0);
          chase::oz::fence_after();
        }
        const uint64_t ad = chase::oz::sw64_desc(chase::oz::smem_u32(sA + ((VAR & 2) ? t * 16384 : 0)));
#pragma unroll
        for (int pl = 0; pl < 2; ++pl) {
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t a = ad + (uint64_t)((pl * 8192) >> 4) + (uint64_t)(ks * 2);
            const int cnt = PROBE_S - t;
#pragma unroll
            for (int i = 0; i < PROBE_S; ++i) {
              if (i >= cnt) continue;
              const int u = cnt - 1 - i;
              const uint32_t d = tmem + (uint32_t)(((t + u) % NACC) * N);
              const uint64_t b = bd + (uint64_t)((u * N * 64) >> 4) + (uint64_t)(ks * 2);
              if ((VAR & 8) || cnt == 1) probe_mma<0, N>(d, a, b);
              else if (i == 0) probe_mma<1, N>(d, a, b);
              else if (i == cnt - 1) probe_mma<3, N>(d, a, b);
              else probe_mma<2, N>(d, a, b);
            }
          }
        }
        if (VAR & 1) chase::oz::mma_commit(chase::oz::smem_u32(&bar_commit));
      }
    }
    chase::oz::mma_commit(chase::oz::smem_u32(&bar_done));
    const unsigned long long t0 = chase::oz::globaltimer();
    while (!chase::oz::mbar_try(chase::oz::smem_u32(&bar_done), 0)) {
      if (chase::oz::globaltimer() - t0 > 2000000000ull) {
        atomicOr(err, 1);
        break;
      }
    }
    cycles[blockIdx.x] = (unsigned long long)(clock64() - c0);
  }
  chase::oz::fence_before();
  __syncthreads();
  chase::oz::fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

template <int N, int VAR> static double run_issue_probe(int sms) {
  constexpr int A_BYTES = (VAR & 2) ? PROBE_S * 16384 : 16384;
  int smem = A_BYTES + PROBE_S * N * 64 + 1024;
  if (smem < 120 * 1024) smem = 120 * 1024;  // one CTA (and one 512-column TMEM allocation) per SM
  CHASE_CUDA(cudaFuncSetAttribute(mma_issue_probe_kernel<N, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  unsigned long long* d_cyc = nullptr;
  int* d_err = nullptr;
  CHASE_CUDA(cudaMalloc(&d_cyc, sms * sizeof(unsigned long long)));
  CHASE_CUDA(cudaMalloc(&d_err, sizeof(int)));
  CHASE_CUDA(cudaMemset(d_err, 0, sizeof(int)));
  const int iters = 400;
  mma_issue_probe_kernel<N, VAR><<<sms, PROBE_THREADS, smem>>>(8, d_cyc, d_err);  // warm-up
  CHASE_CHECK_LAUNCH();
  mma_issue_probe_kernel<N, VAR><<<sms, PROBE_THREADS, smem>>>(iters, d_cyc, d_err);
  CHASE_CHECK_LAUNCH();
  std::vector<unsigned long long> h(sms);
  int herr = 0;
  CHASE_CUDA(cudaMemcpy(h.data(), d_cyc, sms * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  CHASE_CUDA(cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost));
  cudaFree(d_cyc);
  cudaFree(d_err);
  CHASE_REQUIRE(herr == 0, CHASE_ERR_TIMEOUT, "issue-rate probe: completion wait hit its limit");
  double avg = 0.0;
  for (auto v : h) avg += (double)v;
  return avg / sms / ((double)iters * 112.0);
}

}  // namespace

extern "C" chase_status chase_measure_mma_issue(int n_cols, int variant, double* cycles_per_mma) {
  if (!cycles_per_mma) return CHASE_ERR_ARG;
  try {
    int dev = 0, sms = 0, major = 0, minor = 0;
    CHASE_CUDA(cudaGetDevice(&dev));
    CHASE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CHASE_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
    CHASE_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
    if (!(major == 10 && minor == 3)) return CHASE_ERR_UNSUPPORTED;
    double c = -1.0;
    if (variant == 0) {
      switch (n_cols) {
        case 16: c = run_issue_probe<16, 0>(sms); break;
        case 32: c = run_issue_probe<32, 0>(sms); break;
        case 64: c = run_issue_probe<64, 0>(sms); break;
        case 80: c = run_issue_probe<80, 0>(sms); break;
        case 96: c = run_issue_probe<96, 0>(sms); break;
        case 128: c = run_issue_probe<128, 0>(sms); break;
        case 256: c = run_issue_probe<256, 0>(sms); break;
        default: return CHASE_ERR_ARG;
      }
    } else {
      if (n_cols != 80) return CHASE_ERR_ARG;
      switch (variant) {
        case 1: c = run_issue_probe<80, 1>(sms); break;
        case 2: c = run_issue_probe<80, 2>(sms); break;
        case 3: c = run_issue_probe<80, 3>(sms); break;
        case 7: c = run_issue_probe<80, 7>(sms); break;
        case 8: c = run_issue_probe<80, 8>(sms); break;
        default: return CHASE_ERR_ARG;
      }
    }
    *cycles_per_mma = c;
  } catch (const chase::Error& e) {
    return (chase_status)e.status;
  }
  return CHASE_OK;
}
