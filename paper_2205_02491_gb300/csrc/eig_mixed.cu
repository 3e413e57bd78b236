// Helpers of the mixed-precision Rayleigh-Ritz eigensolve (Algorithm 1, line 6).
//
// The quotient G is first diagonalised by the parallel Jacobi solver in FP32 (58x
// the FP64 rate on GB300).  Its eigenvectors Z are then refined in FP64-class
// arithmetic: with Z orthonormal and G' = Z^H G Z, the first-order correction
// Z <- Z (I + X), X_pq = G'_pq / (d_q - d_p) for well separated d = diag(G'),
// converges quadratically (three steps take the FP32 pass, stopped at its rounding floor, to FP64 accuracy).
// Pairs closer than omega (clusters) are left to an exact FP64 Jacobi on each
// cluster's block of G', one block per cluster.
#include "common.cuh"
#include "kernels.h"

namespace chase {

template <typename A, typename B> __device__ inline B cvt(A a);
template <> __device__ inline float cvt<double, float>(double a) { return (float)a; }
template <> __device__ inline double cvt<float, double>(float a) { return (double)a; }
template <> __device__ inline float2 cvt<double2, float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ inline double2 cvt<float2, double2>(float2 a) { return make_double2(a.x, a.y); }

template <typename T, typename F>
__global__ void convert_kernel(int k, const T* in, int64_t ldi, F* out, int64_t ldo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i < k) out[i + (int64_t)j * ldo] = cvt<T, F>(in[i + (int64_t)j * ldi]);
}

template <typename T, typename F> void convert_mat(cudaStream_t st, int k, const T* in, int64_t ldi, F* out, int64_t ldo) {
  convert_kernel<T, F><<<dim3(ceil_div(k, 256), k), 256, 0, st>>>(k, in, ldi, out, ldo);
  CHASE_CHECK_LAUNCH();
}

template <typename T>
__global__ void correction_kernel(int k, const T* Gp, int64_t ldg, T* X, int64_t ldx, double omega) {
  using s = S<T>;
  int p = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (p >= k) return;
  T v = s::zero();
  if (p != q) {
    const double dp = s::re(Gp[p + (int64_t)p * ldg]), dq = s::re(Gp[q + (int64_t)q * ldg]);
    const double gap = dq - dp;
    if (fabs(gap) > omega) v = s::scale(Gp[p + (int64_t)q * ldg], 1.0 / gap);
  }
  X[p + (int64_t)q * ldx] = v;
}

template <typename T>
void eig_correction(cudaStream_t st, int k, const T* Gp, int64_t ldg, T* X, int64_t ldx, double omega) {
  correction_kernel<T><<<dim3(ceil_div(k, 128), k), 128, 0, st>>>(k, Gp, ldg, X, ldx, omega);
  CHASE_CHECK_LAUNCH();
}

template <typename T> __global__ void diag_real_kernel(int k, const T* G, int64_t ldg, double* d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) d[i] = S<T>::re(G[i + (int64_t)i * ldg]);
}

template <typename T> void diag_real(cudaStream_t st, int k, const T* G, int64_t ldg, double* d) {
  diag_real_kernel<T><<<ceil_div(k, 256), 256, 0, st>>>(k, G, ldg, d);
  CHASE_CHECK_LAUNCH();
}

// One CTA per cluster [s, s+c), c <= CMAX: cyclic Jacobi on the block of G', eigenvalues to w[s..s+c),
// then Z[:, s:s+c] <- Z[:, s:s+c] U in place, row by row.
constexpr int CMAX = 32;
template <typename T>
__global__ void cluster_kernel(int k, const int* cl, const T* Gp, int64_t ldg, T* Z, int64_t ldz, double* w,
                               int* status) {
  using s = S<T>;
  const int start = cl[2 * blockIdx.x], c = cl[2 * blockIdx.x + 1];
  __shared__ T B[CMAX][CMAX + 1];
  __shared__ T U[CMAX][CMAX + 1];
  __shared__ T jpp, jpq, jqp, jqq;
  __shared__ int cont;
  for (int t = threadIdx.x; t < c * c; t += blockDim.x) {
    int i = t % c, j = t / c;
    B[i][j] = Gp[(start + i) + (int64_t)(start + j) * ldg];
    U[i][j] = (i == j) ? s::one() : s::zero();
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) {
      double fro = 0.0, off = 0.0;
      for (int i = 0; i < c; ++i)
        for (int j = 0; j < c; ++j) {
          double a = s::abs2(B[i][j]);
          fro += a;
          if (i != j) off += a;
        }
      cont = (sqrt(off) > 1e-15 * sqrt(fro)) && fro > 0.0;
    }
    __syncthreads();
    if (!cont) break;
    for (int p = 0; p < c - 1; ++p)
      for (int q = p + 1; q < c; ++q) {
        if (threadIdx.x == 0) {
          T g = B[p][q];
          double ag = sqrt(s::abs2(g));
          if (ag == 0.0) {
            jpp = s::one();
            jpq = s::zero();
            jqp = s::zero();
            jqq = s::one();
          } else {
            double z = (s::re(B[q][q]) - s::re(B[p][p])) / (2.0 * ag);
            double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
            double cc = 1.0 / sqrt(1.0 + t * t), sn = t * cc;
            T ph = s::scale(s::conj(g), 1.0 / ag);
            jpp = s::make(cc, 0.0);
            jpq = s::make(sn, 0.0);
            jqp = s::scale(ph, -sn);
            jqq = s::scale(ph, cc);
          }
        }
        __syncthreads();
        int i = threadIdx.x;
        if (i < c) {  // columns p, q of B and U
          T bp = B[i][p], bq = B[i][q];
          B[i][p] = s::add(s::mul(bp, jpp), s::mul(bq, jqp));
          B[i][q] = s::add(s::mul(bp, jpq), s::mul(bq, jqq));
          T up = U[i][p], uq = U[i][q];
          U[i][p] = s::add(s::mul(up, jpp), s::mul(uq, jqp));
          U[i][q] = s::add(s::mul(up, jpq), s::mul(uq, jqq));
        }
        __syncthreads();
        if (i < c) {  // rows p, q of B
          T rp = B[p][i], rq = B[q][i];
          B[p][i] = s::add(s::mul(s::conj(jpp), rp), s::mul(s::conj(jqp), rq));
          B[q][i] = s::add(s::mul(s::conj(jpq), rp), s::mul(s::conj(jqq), rq));
        }
        __syncthreads();
        if (i == 0) {
          B[p][q] = s::zero();
          B[q][p] = s::zero();
          B[p][p] = s::make(s::re(B[p][p]), 0.0);
          B[q][q] = s::make(s::re(B[q][q]), 0.0);
        }
        __syncthreads();
      }
  }
  if (threadIdx.x == 0 && sweep >= 40) atomicMax(status, 1);
  for (int i = threadIdx.x; i < c; i += blockDim.x) w[start + i] = s::re(B[i][i]);
  __syncthreads();
  // Z[:, start:start+c] <- Z[:, start:start+c] U
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    T row[CMAX];
#pragma unroll
    for (int j = 0; j < CMAX; ++j)
      if (j < c) row[j] = Z[r + (int64_t)(start + j) * ldz];
#pragma unroll
    for (int j = 0; j < CMAX; ++j) {
      if (j >= c) continue;
      T acc = s::zero();
#pragma unroll
      for (int m = 0; m < CMAX; ++m)
        if (m < c) acc = s::fma(row[m], U[m][j], acc);
      Z[r + (int64_t)(start + j) * ldz] = acc;
    }
  }
}

template <typename T>
void cluster_eig(cudaStream_t st, int k, int nclusters, const int* cl, const T* Gp, int64_t ldg, T* Z, int64_t ldz,
                 double* w, T* scratch, int* status) {
  (void)scratch;
  if (nclusters <= 0) return;
  cluster_kernel<T><<<nclusters, 128, 0, st>>>(k, cl, Gp, ldg, Z, ldz, w, status);
  CHASE_CHECK_LAUNCH();
}

template <typename T> __global__ void rank_kernel(int k, const double* w, double* wout, int* perm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  double wi = w[i];
  int rank = 0;
  for (int j = 0; j < k; ++j) rank += (w[j] < wi) || (w[j] == wi && j < i);
  wout[rank] = wi;
  perm[rank] = i;
}

template <typename T>
void sort_pairs(cudaStream_t st, int k, double* w, T* Z, int64_t ldz, T* tmp, double* wtmp, int* perm) {
  rank_kernel<T><<<ceil_div(k, 128), 128, 0, st>>>(k, w, wtmp, perm);
  CHASE_CHECK_LAUNCH();
  permute_cols<T>(st, k, k, Z, ldz, tmp, k, perm);
  copy_cols<T>(st, k, k, tmp, k, Z, ldz);
  CHASE_CUDA(cudaMemcpyAsync(w, wtmp, k * sizeof(double), cudaMemcpyDeviceToDevice, st));
}

#define INST(T)                                                                                                  \
  template void eig_correction<T>(cudaStream_t, int, const T*, int64_t, T*, int64_t, double);                     \
  template void cluster_eig<T>(cudaStream_t, int, int, const int*, const T*, int64_t, T*, int64_t, double*, T*,   \
                               int*);                                                                            \
  template void diag_real<T>(cudaStream_t, int, const T*, int64_t, double*);                                     \
  template void sort_pairs<T>(cudaStream_t, int, double*, T*, int64_t, T*, double*, int*);
INST(double)
INST(double2)
#undef INST
template void convert_mat<double, float>(cudaStream_t, int, const double*, int64_t, float*, int64_t);
template void convert_mat<float, double>(cudaStream_t, int, const float*, int64_t, double*, int64_t);
template void convert_mat<double2, float2>(cudaStream_t, int, const double2*, int64_t, float2*, int64_t);
template void convert_mat<float2, double2>(cudaStream_t, int, const float2*, int64_t, double2*, int64_t);

}  // namespace chase
