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

// single-precision traits (FP32 first pass of the Rayleigh-Ritz eigensolve); scalars are doubles
// at the interface and rounded to float
template <> struct S<float> {
  static constexpr bool cplx = false;
  __host__ __device__ static inline float zero() { return 0.0f; }
  __host__ __device__ static inline float one() { return 1.0f; }
  __host__ __device__ static inline float conj(float a) { return a; }
  __host__ __device__ static inline float mul(float a, float b) { return a * b; }
  __host__ __device__ static inline float fma(float a, float b, float c) { return ::fmaf(a, b, c); }
  __host__ __device__ static inline float fmac(float a, float b, float c) { return ::fmaf(a, b, c); }
  __host__ __device__ static inline float add(float a, float b) { return a + b; }
  __host__ __device__ static inline float sub(float a, float b) { return a - b; }
  // scaled in double: s itself may lie outside the float range (1/|g| for a denormal g)
  __host__ __device__ static inline float scale(float a, double s) { return (float)((double)a * s); }
  __host__ __device__ static inline double abs2(float a) { return (double)a * (double)a; }
  __host__ __device__ static inline double re(float a) { return a; }
  __host__ __device__ static inline double im(float) { return 0.0; }
  __host__ __device__ static inline float make(double r, double) { return (float)r; }
};

template <> struct S<float2> {
  static constexpr bool cplx = true;
  __host__ __device__ static inline float2 zero() { return make_float2(0.0f, 0.0f); }
  __host__ __device__ static inline float2 one() { return make_float2(1.0f, 0.0f); }
  __host__ __device__ static inline float2 conj(float2 a) { return make_float2(a.x, -a.y); }
  __host__ __device__ static inline float2 mul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
  }
  __host__ __device__ static inline float2 fma(float2 a, float2 b, float2 c) {
    c.x = ::fmaf(a.x, b.x, c.x);
    c.x = ::fmaf(-a.y, b.y, c.x);
    c.y = ::fmaf(a.x, b.y, c.y);
    c.y = ::fmaf(a.y, b.x, c.y);
    return c;
  }
  __host__ __device__ static inline float2 fmac(float2 a, float2 b, float2 c) {
    c.x = ::fmaf(a.x, b.x, c.x);
    c.x = ::fmaf(a.y, b.y, c.x);
    c.y = ::fmaf(a.x, b.y, c.y);
    c.y = ::fmaf(-a.y, b.x, c.y);
    return c;
  }
  __host__ __device__ static inline float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
  __host__ __device__ static inline float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
  __host__ __device__ static inline float2 scale(float2 a, double s) {
    return make_float2((float)((double)a.x * s), (float)((double)a.y * s));
  }
  __host__ __device__ static inline double abs2(float2 a) {
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
  }
  __host__ __device__ static inline double re(float2 a) { return a.x; }
  __host__ __device__ static inline double im(float2 a) { return a.y; }
  __host__ __device__ static inline float2 make(double r, double i) { return make_float2((float)r, (float)i); }
};

// the single-precision type used for the first pass of a FP64 type
template <typename T> struct Lowp;
template <> struct Lowp<double> { using type = float; };
template <> struct Lowp<double2> { using type = float2; };

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

// Wall-clock limit of the bounded grid-barrier waits of the Jacobi sweep kernel (nanoseconds).  Two
// seconds unless a test shortens it through chase_set_wait_limit_ns (0 restores the default).
extern std::atomic<unsigned long long> g_wait_limit_ns;
inline unsigned long long grid_wait_limit_ns() {
  const unsigned long long v = g_wait_limit_ns.load();
  return v ? v : 2000000000ull;
}

// warp-level FP64 sum
__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace chase
