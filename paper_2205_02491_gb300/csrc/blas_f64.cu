// FP64 (DFMA) dense kernels: tiled GEMM with a fused epilogue and split-K,
// column reductions, column permutations, blocked Cholesky and right TRSM.
//
// These are the FP64-exact building blocks of Algorithm 1 (QR via Cholesky-QR,
// Rayleigh-Ritz projection and back-transform, residual norms) and the
// reference path of the Chebyshev filter product.  On GB300 FP64 runs on the
// CUDA cores only (about 1.2 TFLOP/s), so the large products of the
// production path go through the split-BF16 tensor-core kernels instead.
#include "common.cuh"
#include "kernels.h"

namespace chase {

// ============================================================== GEMM
constexpr int GB_M = 64, GB_N = 64;

template <typename T> struct GK { static constexpr int BK = 8; };
template <> struct GK<double> { static constexpr int BK = 16; };

template <typename T>
__device__ inline void epi_store(const Epi& e, int64_t i, int64_t j, T acc) {
  using s = S<T>;
  T v = s::scale(acc, e.alpha);
  if (e.Y) {
    double g = e.gamma * (e.ycol ? e.ycol[j] : 1.0);
    v = s::add(v, s::scale(((const T*)e.Y)[i + j * e.ldy], g));
  }
  if (e.Z) v = s::add(v, s::scale(((const T*)e.Z)[i + j * e.ldz], e.beta));
  ((T*)e.C)[i + j * e.ldc] = v;
}

template <typename T, int OPA, int OPB>
__global__ void __launch_bounds__(256) gemm_f64_kernel(int64_t M, int64_t N, int64_t K, const T* __restrict__ A,
                                                       int64_t lda, const T* __restrict__ B, int64_t ldb, Epi epi,
                                                       T* __restrict__ work, int64_t kchunk) {
  using s = S<T>;
  constexpr int BK = GK<T>::BK;
  __shared__ T As[BK][GB_M + 1];
  __shared__ T Bs[BK][GB_N + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = (int64_t)blockIdx.x * GB_M, n0 = (int64_t)blockIdx.y * GB_N;
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = min(K, kb + kchunk);
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = s::zero();

  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
    // A tile: BM x BK
#pragma unroll
    for (int t = tid; t < GB_M * BK; t += 256) {
      int i, kk;
      if (OPA == OP_N) { i = t % GB_M; kk = t / GB_M; } else { kk = t % BK; i = t / BK; }
      int64_t gi = m0 + i, gk = k0 + kk;
      T v = s::zero();
      if (gi < M && gk < ke) v = (OPA == OP_N) ? A[gi + gk * lda] : s::conj(A[gk + gi * lda]);
      As[kk][i] = v;
    }
#pragma unroll
    for (int t = tid; t < GB_N * BK; t += 256) {
      int j, kk;
      if (OPB == OP_N) { kk = t % BK; j = t / BK; } else { j = t % GB_N; kk = t / GB_N; }
      int64_t gj = n0 + j, gk = k0 + kk;
      T v = s::zero();
      if (gj < N && gk < ke) v = (OPB == OP_N) ? B[gk + gj * ldb] : s::conj(B[gj + gk * ldb]);
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = s::fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int64_t i = m0 + ty + 16 * r, j = n0 + tx + 16 * c;
      if (i < M && j < N) {
        if (work)
          work[(int64_t)blockIdx.z * M * N + i + j * M] = acc[r][c];
        else
          epi_store<T>(epi, i, j, acc[r][c]);
      }
    }
}

template <typename T>
__global__ void splitk_reduce_kernel(int64_t M, int64_t N, int nsplit, const T* __restrict__ work, Epi epi) {
  using s = S<T>;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  T acc = s::zero();
  for (int z = 0; z < nsplit; ++z) acc = s::add(acc, work[(int64_t)z * M * N + idx]);
  epi_store<T>(epi, idx % M, idx / M, acc);
}

template <typename T>
void gemm_f64(cudaStream_t st, Op opA, Op opB, int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, const T* B,
              int64_t ldb, const Epi& epi, T* work, int64_t work_elems) {
  if (M <= 0 || N <= 0) return;
  constexpr int BK = GK<T>::BK;
  int64_t tiles = (int64_t)ceil_div(M, GB_M) * ceil_div(N, GB_N);
  int nsplit = 1;
  if (K > 0) {
    int64_t want = (2 * 152 + tiles - 1) / tiles;  // aim for >= 2 waves of blocks
    int64_t maxsplit = K / (8 * BK);
    nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(want, std::min<int64_t>(maxsplit, 64)));
    if (work == nullptr || work_elems < nsplit * M * N) nsplit = 1;
  }
  int64_t kchunk = K > 0 ? ((K + nsplit - 1) / nsplit + BK - 1) / BK * BK : BK;
  if (K <= 0) {
    // C = epilogue with acc = 0
    nsplit = 1;
  }
  dim3 grid(ceil_div(M, GB_M), ceil_div(N, GB_N), nsplit);
  T* w = nsplit > 1 ? work : nullptr;
#define LAUNCH(OA, OB) gemm_f64_kernel<T, OA, OB><<<grid, 256, 0, st>>>(M, N, std::max<int64_t>(K, 0), A, lda, B, ldb, epi, w, kchunk)
  if (opA == OP_N && opB == OP_N) LAUNCH(OP_N, OP_N);
  else if (opA == OP_C && opB == OP_N) LAUNCH(OP_C, OP_N);
  else if (opA == OP_N && opB == OP_C) LAUNCH(OP_N, OP_C);
  else LAUNCH(OP_C, OP_C);
#undef LAUNCH
  CHASE_CHECK_LAUNCH();
  if (nsplit > 1) {
    splitk_reduce_kernel<T><<<ceil_div(M * N, 256), 256, 0, st>>>(M, N, nsplit, work, epi);
    CHASE_CHECK_LAUNCH();
  }
}

// ============================================================== column reductions
template <typename T>
__global__ void colnorms_kernel(int64_t n, const T* __restrict__ X, int64_t ldx, double* out) {
  using s = S<T>;
  const T* x = X + (int64_t)blockIdx.x * ldx;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += s::abs2(x[i]);
  __shared__ double red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(v);
  }
}

template <typename T> void colnorms(cudaStream_t st, int64_t n, int k, const T* X, int64_t ldx, double* out) {
  if (k <= 0) return;
  colnorms_kernel<T><<<k, 256, 0, st>>>(n, X, ldx, out);
  CHASE_CHECK_LAUNCH();
}

template <typename T>
__global__ void colmaxabs_kernel(int64_t n, const T* __restrict__ X, int64_t ldx, double* out) {
  using s = S<T>;
  const T* x = X + (int64_t)blockIdx.x * ldx;
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    T v = x[i];
    m = fmax(m, fmax(fabs(s::re(v)), fabs(s::im(v))));
  }
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) out[blockIdx.x] = v;
  }
}

template <typename T> void colmaxabs(cudaStream_t st, int64_t n, int k, const T* X, int64_t ldx, double* out) {
  if (k <= 0) return;
  colmaxabs_kernel<T><<<k, 256, 0, st>>>(n, X, ldx, out);
  CHASE_CHECK_LAUNCH();
}

template <typename T>
__global__ void fro_partial_kernel(int64_t n, int k, const T* __restrict__ X, int64_t ldx, double* out) {
  // one block per column: sum |x|^2 ; then summed in column order by a single thread
  using s = S<T>;
  const T* x = X + (int64_t)blockIdx.x * ldx;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += s::abs2(x[i]);
  __shared__ double red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
  }
}

__global__ void sum_kernel(int k, const double* in, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < k; i += 32) acc += in[i];
  acc = warp_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

template <typename T> void fro_norm2(cudaStream_t st, int64_t n, int k, const T* X, int64_t ldx, double* out) {
  // out[0] = ||X||_F^2 ; out[1..k] scratch
  fro_partial_kernel<T><<<k, 256, 0, st>>>(n, k, X, ldx, out + 1);
  CHASE_CHECK_LAUNCH();
  sum_kernel<<<1, 32, 0, st>>>(k, out + 1, out);
  CHASE_CHECK_LAUNCH();
}

// ============================================================== column moves
template <typename T>
__global__ void permute_cols_kernel(int64_t n, const T* __restrict__ src, int64_t lds, T* __restrict__ dst,
                                    int64_t ldd, const int* __restrict__ perm) {
  int a = blockIdx.y;
  int p = perm ? perm[a] : a;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i + a * ldd] = src[i + p * lds];
}

template <typename T>
void permute_cols(cudaStream_t st, int64_t n, int k, const T* src, int64_t lds, T* dst, int64_t ldd, const int* perm) {
  if (k <= 0 || n <= 0) return;
  dim3 grid(std::min<unsigned>(ceil_div(n, 256), 64), k);
  permute_cols_kernel<T><<<grid, 256, 0, st>>>(n, src, lds, dst, ldd, perm);
  CHASE_CHECK_LAUNCH();
}

template <typename T>
void copy_cols(cudaStream_t st, int64_t n, int k, const T* src, int64_t lds, T* dst, int64_t ldd) {
  if (k <= 0 || n <= 0) return;
  CHASE_CUDA(cudaMemcpy2DAsync(dst, ldd * sizeof(T), src, lds * sizeof(T), n * sizeof(T), k,
                               cudaMemcpyDeviceToDevice, st));
}

template <typename T>
__global__ void scale_cols_kernel(int64_t n, T* X, int64_t ldx, const double* s, int invert) {
  int a = blockIdx.y;
  double f = s[a];
  if (invert) f = (f > 0.0) ? 1.0 / f : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    X[i + a * ldx] = S<T>::scale(X[i + a * ldx], f);
}

template <typename T> void scale_cols(cudaStream_t st, int64_t n, int k, T* X, int64_t ldx, const double* s, int invert) {
  if (k <= 0 || n <= 0) return;
  dim3 grid(std::min<unsigned>(ceil_div(n, 256), 64), k);
  scale_cols_kernel<T><<<grid, 256, 0, st>>>(n, X, ldx, s, invert);
  CHASE_CHECK_LAUNCH();
}

template <typename T>
__global__ void add_diag_kernel(int k, T* G, int64_t ldg, const double* shift_dev, double shift) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  double sh = shift + (shift_dev ? *shift_dev : 0.0);
  T v = G[i + i * ldg];
  G[i + i * ldg] = S<T>::make(S<T>::re(v) + sh, 0.0);
}

template <typename T> void add_diag(cudaStream_t st, int k, T* G, int64_t ldg, const double* shift_dev, double shift) {
  add_diag_kernel<T><<<ceil_div(k, 256), 256, 0, st>>>(k, G, ldg, shift_dev, shift);
  CHASE_CHECK_LAUNCH();
}

template <typename T> __global__ void hermitianize_kernel(int k, T* G, int64_t ldg) {
  int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 32 + threadIdx.y;
  if (i >= k || j >= k || i < j) return;
  using s = S<T>;
  if (i == j) {
    G[i + i * ldg] = s::make(s::re(G[i + i * ldg]), 0.0);
    return;
  }
  T a = G[i + j * ldg], b = s::conj(G[j + i * ldg]);
  T m = s::scale(s::add(a, b), 0.5);
  G[i + j * ldg] = m;
  G[j + i * ldg] = s::conj(m);
}

template <typename T> void hermitianize(cudaStream_t st, int k, T* G, int64_t ldg) {
  dim3 grid(ceil_div(k, 32), ceil_div(k, 32));
  hermitianize_kernel<T><<<grid, dim3(32, 32), 0, st>>>(k, G, ldg);
  CHASE_CHECK_LAUNCH();
}

// ============================================================== Cholesky and TRSM
constexpr int CB = 32;  // block size of the blocked Cholesky / TRSM

// Unblocked Cholesky of one CB x CB diagonal block in shared memory (lower).  A pivot that is not finite,
// or <= floor, marks the factorisation failed (info), except in detection mode (dep != null): there a
// finite pivot <= floor marks its column numerically dependent on the columns before it (dep[1 + col],
// count in dep[0]); the column gets a unit pivot and a zero column below it, so it drops out of the
// trailing update and the factorisation of the other columns goes on.
template <typename T>
__global__ void potrf_diag_kernel(int nb, T* G, int64_t ldg, int* info, int col0, double floor, int* dep) {
  using s = S<T>;
  __shared__ T a[CB][CB + 1];
  __shared__ int bad;
  __shared__ int dep_sh[CB];
  int i = threadIdx.x, j = threadIdx.y;  // element (i, j)
  if (i == 0 && j == 0) bad = 0;
  if (j == 0 && i < CB) dep_sh[i] = 0;
  if (i < nb && j < nb) a[i][j] = G[i + j * ldg];
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    if (i == c && j == c) {
      double d = s::re(a[c][c]);
      if (!isfinite(d)) {
        bad = 1;
        d = 1.0;
      } else if (!(d > floor)) {
        if (dep) dep_sh[c] = 1;
        else bad = 1;
        d = 1.0;
      }
      a[c][c] = s::make(sqrt(d), 0.0);
    }
    __syncthreads();
    double piv = s::re(a[c][c]);
    if (j == c && i > c && i < nb) a[i][c] = dep_sh[c] ? s::zero() : s::scale(a[i][c], 1.0 / piv);
    __syncthreads();
    if (i > c && j > c && i < nb && j <= i) a[i][j] = s::sub(a[i][j], s::mul(a[i][c], s::conj(a[j][c])));
    __syncthreads();
  }
  if (i < nb && j < nb) G[i + j * ldg] = (j <= i) ? a[i][j] : s::zero();
  if (i == 0 && j == 0 && bad && info) atomicMax(info, col0 + 1);
  if (dep && j == 0 && i < nb && dep_sh[i]) {
    dep[1 + col0 + i] = 1;
    atomicAdd(&dep[0], 1);
  }
}

// X(rows x nb) <- X L^{-H} with L the nb x nb lower block (row-parallel forward substitution).  dep
// (nullable): dependent-column flags of the block's columns, whose results are set to zero.
template <typename T>
__global__ void trsm_rows_kernel(int64_t rows, int nb, T* X, int64_t ldx, const T* L, int64_t ldl,
                                 const int* dep) {
  using s = S<T>;
  __shared__ T l[CB][CB + 1];
  for (int t = threadIdx.x; t < CB * CB; t += blockDim.x) {
    int i = t % CB, j = t / CB;
    l[i][j] = (i < nb && j < nb && j <= i) ? L[i + j * ldl] : s::zero();
  }
  __syncthreads();
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  T q[CB];
#pragma unroll
  for (int j = 0; j < CB; ++j) {
    if (j < nb) {
      T v = X[r + j * ldx];
#pragma unroll
      for (int m = 0; m < CB; ++m)
        if (m < j) v = s::sub(v, s::mul(q[m], s::conj(l[j][m])));
      q[j] = (dep && dep[j]) ? s::zero() : s::scale(v, 1.0 / s::re(l[j][j]));
    }
  }
#pragma unroll
  for (int j = 0; j < CB; ++j)
    if (j < nb) X[r + j * ldx] = q[j];
}

template <typename T>
void potrf_lower(cudaStream_t st, int k, T* G, int64_t ldg, int* info, T* work, int64_t work_elems,
                 double pivot_floor, int* dep) {
  for (int j0 = 0; j0 < k; j0 += CB) {
    int nb = std::min(CB, k - j0);
    T* Gjj = G + j0 + (int64_t)j0 * ldg;
    potrf_diag_kernel<T><<<1, dim3(CB, CB), 0, st>>>(nb, Gjj, ldg, info, j0, pivot_floor, dep);
    CHASE_CHECK_LAUNCH();
    int rest = k - j0 - nb;
    if (rest <= 0) break;
    T* P = G + (j0 + nb) + (int64_t)j0 * ldg;  // panel below the diagonal block
    trsm_rows_kernel<T><<<ceil_div(rest, 128), 128, 0, st>>>(rest, nb, P, ldg, Gjj, ldg,
                                                             dep ? dep + 1 + j0 : nullptr);
    CHASE_CHECK_LAUNCH();
    // trailing update  G22 -= P P^H
    T* G22 = G + (j0 + nb) + (int64_t)(j0 + nb) * ldg;
    Epi e;
    e.C = G22;
    e.ldc = ldg;
    e.alpha = -1.0;
    e.Z = G22;
    e.ldz = ldg;
    e.beta = 1.0;
    gemm_f64<T>(st, OP_N, OP_C, rest, rest, nb, P, ldg, P, ldg, e, work, work_elems);
  }
}

template <typename T>
void trsm_right_lh(cudaStream_t st, int64_t n, int k, T* X, int64_t ldx, const T* L, int64_t ldl, T* work,
                   int64_t work_elems) {
  for (int j0 = 0; j0 < k; j0 += CB) {
    int nb = std::min(CB, k - j0);
    T* Xb = X + (int64_t)j0 * ldx;
    const T* Ljj = L + j0 + (int64_t)j0 * ldl;
    trsm_rows_kernel<T><<<ceil_div(n, 128), 128, 0, st>>>(n, nb, Xb, ldx, Ljj, ldl, nullptr);
    CHASE_CHECK_LAUNCH();
    int rest = k - j0 - nb;
    if (rest <= 0) break;
    // X[:, j0+nb:] -= Xb * L[j0+nb:, j0:j0+nb]^H
    T* Xr = X + (int64_t)(j0 + nb) * ldx;
    Epi e;
    e.C = Xr;
    e.ldc = ldx;
    e.alpha = -1.0;
    e.Z = Xr;
    e.ldz = ldx;
    e.beta = 1.0;
    gemm_f64<T>(st, OP_N, OP_C, n, rest, nb, Xb, ldx, L + (j0 + nb) + (int64_t)j0 * ldl, ldl, e, work, work_elems);
  }
}

// ============================================================== triangular inverse
// Inverse of one CB x CB lower-triangular diagonal block in place (one block per CTA).
template <typename T> __global__ void trtri_diag_kernel(int k, T* L, int64_t ldl) {
  using s = S<T>;
  __shared__ T a[CB][CB + 1];
  __shared__ T x[CB][CB + 1];
  const int j0 = blockIdx.x * CB;
  const int nb = min(CB, k - j0);
  const int i = threadIdx.x, j = threadIdx.y;
  T* Lb = L + j0 + (int64_t)j0 * ldl;
  if (i < nb && j < nb) a[i][j] = (j <= i) ? Lb[i + (int64_t)j * ldl] : s::zero();
  __syncthreads();
  // column j of the inverse by forward substitution (thread row 0 of each column does it)
  if (i == 0 && j < nb) {
    for (int r = 0; r < nb; ++r) {
      T v = (r == j) ? s::one() : s::zero();
      for (int m = j; m < r; ++m) v = s::sub(v, s::mul(a[r][m], x[m][j]));
      // divide by the (real, positive) diagonal
      x[r][j] = (r < j) ? s::zero() : s::scale(v, 1.0 / s::re(a[r][r]));
    }
  }
  __syncthreads();
  if (i < nb && j < nb) Lb[i + (int64_t)j * ldl] = (j <= i) ? x[i][j] : s::zero();
}

template <typename T> __global__ void zero_upper_kernel(int k, T* G, int64_t ldg) {
  int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 32 + threadIdx.y;
  if (i < k && j < k && i < j) G[i + (int64_t)j * ldg] = S<T>::zero();
}

template <typename T> void zero_upper(cudaStream_t st, int k, T* G, int64_t ldg) {
  zero_upper_kernel<T><<<dim3(ceil_div(k, 32), ceil_div(k, 32)), dim3(32, 32), 0, st>>>(k, G, ldg);
  CHASE_CHECK_LAUNCH();
}

template <typename T> void trtri_diag(cudaStream_t st, int k, T* L, int64_t ldl) {
  trtri_diag_kernel<T><<<ceil_div(k, CB), dim3(CB, CB), 0, st>>>(k, L, ldl);
  CHASE_CHECK_LAUNCH();
}

// ============================================================== generator
template <typename T>
__global__ void generate_wy_kernel(T* A, int64_t n, int64_t lda, const double* __restrict__ lam,
                                   const T* __restrict__ U, const T* __restrict__ B, const T* __restrict__ D, int k) {
  // A_ij = lam_i d_ij - lam_j sum_a B_ia conj(U_ja) - lam_i sum_a U_ia conj(B_ja) + sum_a D_ia conj(B_ja)
  // computed for i >= j and mirrored so A is exactly Hermitian.
  using s = S<T>;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t j = (int64_t)blockIdx.y;
  if (i >= n || i < j) return;
  T t1 = s::zero(), t2 = s::zero(), t3 = s::zero();
  for (int a = 0; a < k; ++a) {
    T bja = B[j + a * n];
    t1 = s::fma(B[i + a * n], s::conj(U[j + a * n]), t1);
    t2 = s::fma(U[i + a * n], s::conj(bja), t2);
    t3 = s::fma(D[i + a * n], s::conj(bja), t3);
  }
  T v = s::sub(s::sub(t3, s::scale(t1, lam[j])), s::scale(t2, lam[i]));
  if (i == j) {
    A[i + i * lda] = s::make(s::re(v) + lam[i], 0.0);
  } else {
    A[i + j * lda] = v;
    A[j + i * lda] = s::conj(v);
  }
}

template <typename T>
void generate_wy(cudaStream_t st, T* A, int64_t n, int64_t lda, const double* lam, const T* U, const T* B, const T* D,
                 int k) {
  // grid.y = columns (<= 2^31-1 OK for n up to 65535 per launch dimension limit): split if needed
  for (int64_t j0 = 0; j0 < n; j0 += 65535) {
    int64_t nj = std::min<int64_t>(65535, n - j0);
    (void)nj;
  }
  CHASE_REQUIRE(n <= 65535, 1, "generator supports n <= 65535");
  dim3 grid(ceil_div(n, 256), n);
  generate_wy_kernel<T><<<grid, 256, 0, st>>>(A, n, lda, lam, U, B, D, k);
  CHASE_CHECK_LAUNCH();
}

// ============================================================== Householder QR building blocks
// Reflector of one column segment x (length m): alpha = -ph ||x|| with ph = x0/|x0| (1 for x0 = 0),
// v = x - alpha e1 written over x, H = I - tau v v^H with tau = 2/||v||^2 (0 for x = 0), so H x = alpha e1.
template <typename T>
__global__ void __launch_bounds__(1024) householder_vec_kernel(int64_t m, T* x, T* alpha, double* tau) {
  using s = S<T>;
  __shared__ double red[32];
  double ss = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) ss += s::abs2(x[i]);
  ss = warp_sum(ss);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    const T x0 = x[0];
    const double a0 = sqrt(s::abs2(x0));
    const double nrm = sqrt(t);
    const T ph = a0 > 0.0 ? s::scale(x0, 1.0 / a0) : s::one();
    alpha[0] = s::scale(ph, -nrm);
    const T v0 = s::scale(ph, a0 + nrm);
    const double vv = t - a0 * a0 + (a0 + nrm) * (a0 + nrm);
    tau[0] = vv > 0.0 ? 2.0 / vv : 0.0;
    x[0] = v0;
  }
}

// X (m x ncols, ld ldx) <- (I - tau v v^H) X, one block per column.
template <typename T>
__global__ void householder_apply_kernel(int64_t m, const T* __restrict__ v, T* X, int64_t ldx, const double* tau) {
  using s = S<T>;
  __shared__ double red_re[32], red_im[32];
  __shared__ T w_sh;
  T* x = X + (int64_t)blockIdx.x * ldx;
  T acc = s::zero();
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) acc = s::fmac(v[i], x[i], acc);  // conj(v) x
  double re = warp_sum(s::re(acc)), im = warp_sum(s::im(acc));
  if ((threadIdx.x & 31) == 0) {
    red_re[threadIdx.x >> 5] = re;
    red_im[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tr += red_re[w];
      ti += red_im[w];
    }
    w_sh = s::scale(s::make(tr, ti), tau[0]);
  }
  __syncthreads();
  const T w = w_sh;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) x[i] = s::sub(x[i], s::mul(v[i], w));
}

// Panel reflectors with explicit zeros: V[i, j] = Xp[i, j] for i >= j, 0 above (m x pb, ld ldv).
template <typename T>
__global__ void reflector_panel_kernel(int64_t m, const T* __restrict__ Xp, int64_t ldx, T* V, int64_t ldv) {
  const int j = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    V[i + (int64_t)j * ldv] = i < j ? S<T>::zero() : Xp[i + (int64_t)j * ldx];
}

// Compact-WY factor of H_1 ... H_pb = I - V Tm V^H (forward, column-wise): Tm upper triangular, Tm_jj = tau_j,
// Tm(0:j, j) = -tau_j Tm(0:j, 0:j) Gv(0:j, j) with Gv = V^H V (pb x pb, ld pb).  One thread.
template <typename T>
__global__ void householder_T_kernel(int pb, const T* __restrict__ Gv, const double* __restrict__ tau, T* Tm,
                                     int64_t ldt) {
  using s = S<T>;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int j = 0; j < pb; ++j) {
    for (int i = 0; i < j; ++i) {
      T acc = s::zero();
      for (int l = i; l < j; ++l) acc = s::add(acc, s::mul(Tm[i + (int64_t)l * ldt], Gv[l + (int64_t)j * pb]));
      Tm[i + (int64_t)j * ldt] = s::scale(acc, -tau[j]);
    }
    Tm[j + (int64_t)j * ldt] = s::make(tau[j], 0.0);
    for (int i = j + 1; i < pb; ++i) Tm[i + (int64_t)j * ldt] = s::zero();
  }
}

template <typename T> __global__ void identity_rect_kernel(int64_t n, int k, T* Q, int64_t ldq) {
  const int j = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Q[i + (int64_t)j * ldq] = (i == j) ? S<T>::one() : S<T>::zero();
}

template <typename T> void householder_vec(cudaStream_t st, int64_t m, T* x, T* alpha, double* tau) {
  householder_vec_kernel<T><<<1, 1024, 0, st>>>(m, x, alpha, tau);
  CHASE_CHECK_LAUNCH();
}
template <typename T>
void householder_apply(cudaStream_t st, int64_t m, const T* v, T* X, int64_t ldx, int ncols, const double* tau) {
  if (ncols <= 0) return;
  householder_apply_kernel<T><<<ncols, 256, 0, st>>>(m, v, X, ldx, tau);
  CHASE_CHECK_LAUNCH();
}
template <typename T> void reflector_panel(cudaStream_t st, int64_t m, int pb, const T* Xp, int64_t ldx, T* V, int64_t ldv) {
  dim3 grid(std::min<unsigned>(ceil_div(m, 256), 64), pb);
  reflector_panel_kernel<T><<<grid, 256, 0, st>>>(m, Xp, ldx, V, ldv);
  CHASE_CHECK_LAUNCH();
}
template <typename T> void householder_T(cudaStream_t st, int pb, const T* Gv, const double* tau, T* Tm, int64_t ldt) {
  householder_T_kernel<T><<<1, 32, 0, st>>>(pb, Gv, tau, Tm, ldt);
  CHASE_CHECK_LAUNCH();
}
template <typename T> void identity_rect(cudaStream_t st, int64_t n, int k, T* Q, int64_t ldq) {
  dim3 grid(std::min<unsigned>(ceil_div(n, 256), 64), k);
  identity_rect_kernel<T><<<grid, 256, 0, st>>>(n, k, Q, ldq);
  CHASE_CHECK_LAUNCH();
}

// ============================================================== seeded Hermitian perturbation
// Counter-based Gaussian: SplitMix64 (Steele, Lea & Flood 2014) as a hash of (seed, counter), two 53-bit
// uniforms per draw, Box-Muller.  G_ij (complex) uses counter 2 (i + j n) and 2 (i + j n) + 1; real uses one
// normal.  A += eps * s * (G + G^H)/2 with s = 1/sqrt(2n) (complex) or 1/sqrt(2n) * sqrt(2) (real), the
// semicircle-edge estimate of 1/||(G+G^H)/2||_2.
__device__ inline unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ inline double2 normal_pair(unsigned long long seed, unsigned long long ctr) {
  unsigned long long a = splitmix64(seed ^ splitmix64(2 * ctr));
  unsigned long long b = splitmix64(seed ^ splitmix64(2 * ctr + 1));
  double u1 = ((double)(a >> 11) + 1.0) * 1.1102230246251565e-16;  // (0, 1]
  double u2 = (double)(b >> 11) * 1.1102230246251565e-16;           // [0, 1)
  double r = sqrt(-2.0 * log(u1));
  double t = 6.283185307179586 * u2;
  return make_double2(r * cos(t), r * sin(t));
}

template <typename T>
__global__ void perturb_kernel(T* A, int64_t n, int64_t lda, double eps, unsigned long long seed) {
  using s = S<T>;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t j = blockIdx.y;
  if (i >= n || i < j) return;
  const double sc = s::cplx ? eps / sqrt(2.0 * (double)n) : eps / sqrt(2.0 * (double)n);
  double2 gij = normal_pair(seed, (unsigned long long)(i + j * n));
  double2 gji = normal_pair(seed, (unsigned long long)(j + i * n));
  if (s::cplx) {
    // G = (x + i y)/sqrt(2): h_ij = (G_ij + conj(G_ji))/2
    double hr = 0.5 * 0.7071067811865476 * (gij.x + gji.x);
    double hi = 0.5 * 0.7071067811865476 * (gij.y - gji.y);
    if (i == j) hi = 0.0;
    T d = s::make(sc * hr, sc * hi);
    A[i + j * lda] = s::add(A[i + j * lda], d);
    if (i != j) A[j + i * lda] = s::add(A[j + i * lda], s::conj(d));
  } else {
    double h = 0.5 * (gij.x + gji.x);
    T d = s::make(sc * h, 0.0);
    A[i + j * lda] = s::add(A[i + j * lda], d);
    if (i != j) A[j + i * lda] = s::add(A[j + i * lda], d);
  }
}

template <typename T> void perturb(cudaStream_t st, T* A, int64_t n, int64_t lda, double eps, unsigned long long seed) {
  CHASE_REQUIRE(n <= 65535, 1, "perturbation supports n <= 65535");
  dim3 grid(ceil_div(n, 256), (unsigned)n);
  perturb_kernel<T><<<grid, 256, 0, st>>>(A, n, lda, eps, seed);
  CHASE_CHECK_LAUNCH();
}

// Seeded start vectors: X[i + j ldx] = the counter-based normal of counter i + j rows ((x + i y)/sqrt(2) complex,
// x real), the same generator as above.
template <typename T>
__global__ void fill_normal_kernel(T* X, int64_t rows, int64_t ldx, unsigned long long seed) {
  using s = S<T>;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= rows) return;
  const double2 g = normal_pair(seed, (unsigned long long)(i + j * rows));
  X[i + j * ldx] = s::cplx ? s::make(0.7071067811865476 * g.x, 0.7071067811865476 * g.y) : s::make(g.x, 0.0);
}

template <typename T> void fill_normal(cudaStream_t st, T* X, int64_t rows, int cols, int64_t ldx, unsigned long long seed) {
  if (rows <= 0 || cols <= 0) return;
  CHASE_REQUIRE(cols <= 65535, 1, "fill_normal: too many columns");
  dim3 grid(ceil_div(rows, 256), (unsigned)cols);
  fill_normal_kernel<T><<<grid, 256, 0, st>>>(X, rows, ldx, seed);
  CHASE_CHECK_LAUNCH();
}

// ============================================================== instantiations
#define INST(T)                                                                                                   \
  template void gemm_f64<T>(cudaStream_t, Op, Op, int64_t, int64_t, int64_t, const T*, int64_t, const T*, int64_t, \
                            const Epi&, T*, int64_t);                                                            \
  template void colnorms<T>(cudaStream_t, int64_t, int, const T*, int64_t, double*);                              \
  template void colmaxabs<T>(cudaStream_t, int64_t, int, const T*, int64_t, double*);                             \
  template void fro_norm2<T>(cudaStream_t, int64_t, int, const T*, int64_t, double*);                             \
  template void permute_cols<T>(cudaStream_t, int64_t, int, const T*, int64_t, T*, int64_t, const int*);          \
  template void copy_cols<T>(cudaStream_t, int64_t, int, const T*, int64_t, T*, int64_t);                         \
  template void scale_cols<T>(cudaStream_t, int64_t, int, T*, int64_t, const double*, int);                       \
  template void add_diag<T>(cudaStream_t, int, T*, int64_t, const double*, double);                               \
  template void hermitianize<T>(cudaStream_t, int, T*, int64_t);                                                  \
  template void potrf_lower<T>(cudaStream_t, int, T*, int64_t, int*, T*, int64_t, double, int*);                   \
  template void householder_vec<T>(cudaStream_t, int64_t, T*, T*, double*);                                      \
  template void householder_apply<T>(cudaStream_t, int64_t, const T*, T*, int64_t, int, const double*);            \
  template void reflector_panel<T>(cudaStream_t, int64_t, int, const T*, int64_t, T*, int64_t);                   \
  template void householder_T<T>(cudaStream_t, int, const T*, const double*, T*, int64_t);                         \
  template void identity_rect<T>(cudaStream_t, int64_t, int, T*, int64_t);                                         \
  template void trsm_right_lh<T>(cudaStream_t, int64_t, int, T*, int64_t, const T*, int64_t, T*, int64_t);        \
  template void generate_wy<T>(cudaStream_t, T*, int64_t, int64_t, const double*, const T*, const T*, const T*, int); \
  template void zero_upper<T>(cudaStream_t, int, T*, int64_t);                                                    \
  template void trtri_diag<T>(cudaStream_t, int, T*, int64_t);                                                   \
  template void perturb<T>(cudaStream_t, T*, int64_t, int64_t, double, unsigned long long);                      \
  template void fill_normal<T>(cudaStream_t, T*, int64_t, int, int64_t, unsigned long long);
INST(double)
INST(double2)
#undef INST
// single-precision first pass of the Rayleigh-Ritz eigensolve
template void permute_cols<float>(cudaStream_t, int64_t, int, const float*, int64_t, float*, int64_t, const int*);
template void permute_cols<float2>(cudaStream_t, int64_t, int, const float2*, int64_t, float2*, int64_t, const int*);

}  // namespace chase
