// Shared device helpers: scalar traits for real (double) and complex (double2)
// FP64 arithmetic, error handling, launch helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <string>

namespace chase {

// ---------------------------------------------------------------- scalar traits
template <typename T> struct S;

template <> struct S<double> {
  static constexpr bool cplx = false;
  __host__ __device__ static inline double zero() { return 0.0; }
  __host__ __device__ static inline double one() { return 1.0; }
  __host__ __device__ static inline double conj(double a) { return a; }
  __host__ __device__ static inline double mul(double a, double b) { return a * b; }
  __host__ __device__ static inline double fma(double a, double b, double c) { return ::fma(a, b, c); }
  // c + conj(a) * b
  __host__ __device__ static inline double fmac(double a, double b, double c) { return ::fma(a, b, c); }
  __host__ __device__ static inline double add(double a, double b) { return a + b; }
  __host__ __device__ static inline double sub(double a, double b) { return a - b; }
  __host__ __device__ static inline double scale(double a, double s) { return a * s; }
  __host__ __device__ static inline double abs2(double a) { return a * a; }
  __host__ __device__ static inline double re(double a) { return a; }
  __host__ __device__ static inline double im(double) { return 0.0; }
  __host__ __device__ static inline double make(double r, double) { return r; }
};

template <> struct S<double2> {
  static constexpr bool cplx = true;
  __host__ __device__ static inline double2 zero() { return make_double2(0.0, 0.0); }
  __host__ __device__ static inline double2 one() { return make_double2(1.0, 0.0); }
  __host__ __device__ static inline double2 conj(double2 a) { return make_double2(a.x, -a.y); }
  __host__ __device__ static inline double2 mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
  }
  __host__ __device__ static inline double2 fma(double2 a, double2 b, double2 c) {
    c.x = ::fma(a.x, b.x, c.x);
    c.x = ::fma(-a.y, b.y, c.x);
    c.y = ::fma(a.x, b.y, c.y);
    c.y = ::fma(a.y, b.x, c.y);
    return c;
  }
  __host__ __device__ static inline double2 fmac(double2 a, double2 b, double2 c) {
    c.x = ::fma(a.x, b.x, c.x);
    c.x = ::fma(a.y, b.y, c.x);
    c.y = ::fma(a.x, b.y, c.y);
    c.y = ::fma(-a.y, b.x, c.y);
    return c;
  }
  __host__ __device__ static inline double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
  __host__ __device__ static inline double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
  __host__ __device__ static inline double2 scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
  __host__ __device__ static inline double abs2(double2 a) { return a.x * a.x + a.y * a.y; }
  __host__ __device__ static inline double re(double2 a) { return a.x; }
  __host__ __device__ static inline double im(double2 a) { return a.y; }
  __host__ __device__ static inline double2 make(double r, double i) { return make_double2(r, i); }
};

// ---------------------------------------------------------------- errors
struct Error {
  int status;
  std::string msg;
};

#define CHASE_CUDA(call)                                                                         \
  do {                                                                                           \
    cudaError_t _e = (call);                                                                     \
    if (_e != cudaSuccess)                                                                       \
      throw ::chase::Error{6, std::string(#call) + ": " + cudaGetErrorString(_e)};              \
  } while (0)

// every kernel launch of the library is followed by CHASE_CHECK_LAUNCH(), which also counts it
extern std::atomic<long long> g_kernel_launches;
#define CHASE_CHECK_LAUNCH()                        \
  do {                                              \
    ::chase::g_kernel_launches.fetch_add(1);        \
    CHASE_CUDA(cudaGetLastError());                 \
  } while (0)

#define CHASE_REQUIRE(cond, code, text)                                                          \
  do {                                                                                           \
    if (!(cond)) throw ::chase::Error{(code), std::string(text)};                                \
  } while (0)

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// warp-level FP64 sum
__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace chase
