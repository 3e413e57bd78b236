// Dense Hermitian eigensolve that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is already
// reserved by a framework's caching allocator or by its own arena, or code that
// must not allocate (allocation can fail under memory pressure and
// cudaMalloc/cudaFree synchronize the device).  For them this file provides one
// entry point that runs the parallel cyclic Jacobi eigensolver of the
// Rayleigh-Ritz quotient using a fixed scratch array that lives in the
// library's own device memory, reserved when the library is loaded onto a
// device and kept until the process exits.
//
// Limits and sharing rules:
//   * k <= CHASE_HEEVJ_NOALLOC_KMAX (256); larger k is rejected with
//     CHASE_ERR_ARG.
//   * Every call, on every stream, uses the same scratch array on a device.
//     Calls that overlap on the GPU race and give wrong results: serialise them
//     (one stream, or events).  The array keeps the previous call's contents;
//     the solver writes every scratch value it reads, so nothing needs clearing.
//   * Host code cannot use the array's symbol as a device address.  The first
//     call in each CUDA context (normally one per device: the primary context)
//     looks up the array's device address with cudaGetSymbolAddress while that
//     context is current and caches it by context, so a context created later
//     on the same device (after cudaDeviceReset, or a caller's own context)
//     gets its own lookup; make the first call in a context before capturing
//     any stream into a CUDA graph.
#include <cuda.h>

#include <mutex>

#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int KMAX = CHASE_HEEVJ_NOALLOC_KMAX;
// G copy (k*k) + unsorted Z (k*k) + rotation records (3k scalars) + a little slack,
// in complex scalars; plus doubles (eigenvalues k, partial sums 2k+2) and ints (k).
constexpr size_t SCALARS = 2 * (size_t)KMAX * KMAX + 3 * (size_t)KMAX + 16;
constexpr size_t SCRATCH_BYTES = SCALARS * 16 + (3 * (size_t)KMAX + 16) * 8 + (size_t)KMAX * 4 + 256;

__device__ __align__(256) unsigned char g_heevj_scratch[SCRATCH_BYTES];

// (context, address) pairs; a context's module, and with it the array, lives as long as the context
constexpr int MAX_CONTEXTS = 64;
std::mutex g_mu;
CUcontext g_ctx[MAX_CONTEXTS] = {};
void* g_addr[MAX_CONTEXTS] = {};
int g_used = 0;

// cuCtxGetCurrent through the runtime's driver entry-point query, so that the library does not link
// the driver library (it loads on machines without a GPU driver)
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)p;
  });
  return fn;
}

template <typename T>
void run(const T* G, int64_t ldg, int k, double* w_host, T* Z, int64_t ldz, cudaStream_t st, unsigned char* base) {
  T* Gw = (T*)base;                               // k*k working copy of G (destroyed)
  T* work = Gw + (size_t)k * k;                   // k*k + 3k + 8 scalars for the solver
  double* w = (double*)(base + SCALARS * 16);     // k eigenvalues
  double* dwork = w + KMAX;                       // 2k + 2 partial sums
  int* iwork = (int*)(dwork + 2 * KMAX + 16);     // k permutation entries
  chase::copy_cols<T>(st, k, k, G, ldg, Gw, k);
  chase::heev_jacobi<T>(st, k, Gw, k, w, Z, ldz, work, (int64_t)k * k + 3 * (int64_t)k + 8, dwork, iwork, 1e-14, 60);
  CHASE_CUDA(cudaMemcpyAsync(w_host, w, k * sizeof(double), cudaMemcpyDeviceToHost, st));
  CHASE_CUDA(cudaStreamSynchronize(st));
}

}  // namespace

extern "C" chase_status chase_heevj_noalloc(const void* G_dev, int64_t ldg, int k, chase_dtype dtype,
                                            double* w_host, void* Z_dev, int64_t ldz, void* stream) {
  // sizes beyond the scratch array are rejected before any device work
  if (!G_dev || !Z_dev || !w_host || k < 1 || k > KMAX || ldg < k || ldz < k ||
      (dtype != CHASE_R64 && dtype != CHASE_C128))
    return CHASE_ERR_ARG;
  try {
    CtxGetCurrentFn get_ctx = ctx_get_current();
    if (!get_ctx) return CHASE_ERR_CUDA;
    CUcontext cur = nullptr;
    if (get_ctx(&cur) != CUDA_SUCCESS) return CHASE_ERR_CUDA;
    if (cur == nullptr) {
      // no context yet: the runtime's symbol lookup creates the device's primary context
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_heevj_scratch) != cudaSuccess) return CHASE_ERR_CUDA;
      if (get_ctx(&cur) != CUDA_SUCCESS || cur == nullptr) return CHASE_ERR_CUDA;
    }
    unsigned char* base = nullptr;
    {
      std::lock_guard<std::mutex> lock(g_mu);
      for (int i = 0; i < g_used && !base; ++i)
        if (g_ctx[i] == cur) base = (unsigned char*)g_addr[i];
      if (!base) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_heevj_scratch);
        if (e != cudaSuccess) return CHASE_ERR_CUDA;
        // a full table (more than 64 contexts in one process) overwrites its first entry
        const int slot = g_used < MAX_CONTEXTS ? g_used++ : 0;
        g_ctx[slot] = cur;
        g_addr[slot] = p;
        base = (unsigned char*)p;
      }
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == CHASE_C128)
      run<double2>((const double2*)G_dev, ldg, k, w_host, (double2*)Z_dev, ldz, st, base);
    else
      run<double>((const double*)G_dev, ldg, k, w_host, (double*)Z_dev, ldz, st, base);
  } catch (const chase::Error& e) {
    return (chase_status)e.status;
  } catch (const std::exception&) {
    return CHASE_ERR_CUDA;
  }
  return CHASE_OK;
}
