// Lanczos spectral-bound estimation (Algorithm 1, line 2) on the device.
//
// All runs advance together: a multi-vector HEMV (A times one vector per run,
// FP64 DFMA with A streamed once per step, or the caller's FP64-class split
// tensor-core product for large n), the three-term update, one classical
// Gram-Schmidt reorthogonalisation against the run's basis, normalisation.  The
// tridiagonal T of each run is diagonalised by a single-block cyclic Jacobi
// (same rotation as the Rayleigh-Ritz solver), and one thread computes
// b_sup = max(theta_max + |beta_last|), mu_1 = min theta_min, theta_max and the
// density-of-states quantile mu_ne = smallest pooled Ritz value whose
// cumulative weight (1/runs) sum tau_j^2 reaches ne/n, clamped into
// (mu_1, b_sup) by 1e-3 of the spectral span.
#include "common.cuh"
#include "kernels.h"

namespace chase {

constexpr int LZ_MAXR = 8;      // runs
constexpr int LZ_MAXS = 64;     // steps
constexpr int HEMV_ROWS = 256;
constexpr int HEMV_COLS = 256;  // column chunk per block

// part[c][r][i] = sum_{j in chunk c} A[i,j] X[j,r]
template <typename T, int R>
__global__ void __launch_bounds__(HEMV_ROWS) hemv_multi_kernel(int64_t n, const T* __restrict__ A, int64_t lda,
                                                                const T* __restrict__ X, int64_t ldx, T* part) {
  using s = S<T>;
  __shared__ T xs[HEMV_COLS][R];
  int64_t j0 = (int64_t)blockIdx.y * HEMV_COLS;
  int nj = (int)(n - j0 < HEMV_COLS ? n - j0 : HEMV_COLS);
  for (int t = threadIdx.x; t < HEMV_COLS * R; t += blockDim.x) {
    int j = t / R, r = t % R;
    xs[j][r] = j < nj ? X[(j0 + j) + (int64_t)r * ldx] : s::zero();
  }
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * HEMV_ROWS + threadIdx.x;
  if (i >= n) return;
  T acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = s::zero();
  const T* a = A + i + j0 * lda;
  for (int j = 0; j < nj; ++j) {
    T v = a[(int64_t)j * lda];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = s::fma(v, xs[j][r], acc[r]);
  }
#pragma unroll
  for (int r = 0; r < R; ++r) part[((int64_t)blockIdx.y * R + r) * n + i] = acc[r];
}

template <typename T>
__global__ void hemv_reduce_kernel(int64_t n, int R, int nchunk, const T* __restrict__ part, T* Y, int64_t ldy) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * R) return;
  int r = (int)(idx / n);
  int64_t i = idx % n;
  T acc = S<T>::zero();
  for (int c = 0; c < nchunk; ++c) acc = S<T>::add(acc, part[((int64_t)c * R + r) * n + i]);
  Y[i + r * ldy] = acc;
}

// d[r][i] = sum_rows conj(Vb_r[:, i]) w_r, i < m ; block (chunk, run) partials
constexpr int DOT_CHUNKS = 64;
template <typename T>
__global__ void basis_dots_kernel(int64_t n, int m, int steps, const T* __restrict__ Vb, const T* __restrict__ W,
                                  T* part) {
  using s = S<T>;
  int r = blockIdx.y, c = blockIdx.x;
  int64_t per = (n + DOT_CHUNKS - 1) / DOT_CHUNKS;
  int64_t i0 = c * per, i1 = (i0 + per < n ? i0 + per : n);
  const T* V = Vb + (int64_t)r * n * steps;
  const T* w = W + (int64_t)r * n;
  __shared__ T red[32][LZ_MAXS];
  for (int col = 0; col < m; ++col) {
    T acc = s::zero();
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc = s::fmac(V[i + (int64_t)col * n], w[i], acc);
    // block reduce (fixed order)
    double re = warp_sum(s::re(acc)), im = warp_sum(s::im(acc));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][col] = s::make(re, im);
  }
  __syncthreads();
  for (int col = threadIdx.x; col < m; col += blockDim.x) {
    T acc = s::zero();
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) acc = s::add(acc, red[wv][col]);
    part[((int64_t)r * DOT_CHUNKS + c) * LZ_MAXS + col] = acc;
  }
}

template <typename T> __global__ void dots_reduce_kernel(int runs, int m, const T* part, T* d) {
  int r = blockIdx.x, col = threadIdx.x;
  if (col >= m) return;
  T acc = S<T>::zero();
  for (int c = 0; c < DOT_CHUNKS; ++c) acc = S<T>::add(acc, part[((int64_t)r * DOT_CHUNKS + c) * LZ_MAXS + col]);
  d[r * LZ_MAXS + col] = acc;
}

// w_r -= sum_{i<m} coef[r][i] Vb_r[:, i]
template <typename T>
__global__ void basis_update_kernel(int64_t n, int m, int steps, const T* __restrict__ Vb, T* W, const T* __restrict__ coef) {
  using s = S<T>;
  int r = blockIdx.y;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T* V = Vb + (int64_t)r * n * steps;
  T acc = W[(int64_t)r * n + i];
  for (int col = 0; col < m; ++col) {
    T cf = coef[r * LZ_MAXS + col];
    acc = s::sub(acc, s::mul(V[i + (int64_t)col * n], cf));
  }
  W[(int64_t)r * n + i] = acc;
}

// three-term coefficients: alpha_j = Re d[j]; coef = {.., beta_{j-1} at j-1, alpha_j at j}
template <typename T>
__global__ void lanczos_coef3_kernel(int runs, int j, const T* d, T* coef, double* alpha, const double* beta) {
  int r = threadIdx.x;
  if (r >= runs) return;
  double a = S<T>::re(d[r * LZ_MAXS + j]);
  alpha[r * LZ_MAXS + j] = a;
  for (int i = 0; i < LZ_MAXS; ++i) coef[r * LZ_MAXS + i] = S<T>::zero();
  coef[r * LZ_MAXS + j] = S<T>::make(a, 0.0);
  if (j > 0) coef[r * LZ_MAXS + j - 1] = S<T>::make(beta[r * LZ_MAXS + j - 1], 0.0);
}

// beta_j = ||w||; if more steps follow, basis[:, j+1] = w / beta_j
template <typename T>
__global__ void lanczos_norm_kernel(int64_t n, int steps, int j, const T* __restrict__ W, T* Vb, double* beta) {
  using s = S<T>;
  int r = blockIdx.x;
  const T* w = W + (int64_t)r * n;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += s::abs2(w[i]);
  __shared__ double red[32];
  __shared__ double bsh;
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) {
      bsh = sqrt(v);
      beta[r * LZ_MAXS + j] = bsh;
    }
  }
  __syncthreads();
  if (j + 1 < steps) {
    double inv = bsh > 0.0 ? 1.0 / bsh : 0.0;
    T* v = Vb + (int64_t)r * n * steps + (int64_t)(j + 1) * n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v[i] = s::scale(w[i], inv);
  }
}

// basis[:, 0] = L0[:, r] / ||L0[:, r]||
template <typename T> __global__ void lanczos_start_kernel(int64_t n, int steps, const T* __restrict__ L0, T* Vb) {
  using s = S<T>;
  int r = blockIdx.x;
  const T* x = L0 + (int64_t)r * n;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += s::abs2(x[i]);
  __shared__ double red[32];
  __shared__ double inv;
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) inv = 1.0 / sqrt(v);
  }
  __syncthreads();
  T* v0 = Vb + (int64_t)r * n * steps;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v0[i] = s::scale(x[i], inv);
}

// Cyclic Jacobi on the run's tridiagonal T (real symmetric, steps <= 64), one block per run.
// Output theta ascending and tau2 = squared first components of the eigenvectors.
__global__ void tridiag_jacobi_kernel(int steps, const double* alpha, const double* beta, double* theta,
                                      double* tau2, int* status) {
  int r = blockIdx.x;
  int k = steps;
  __shared__ double G[LZ_MAXS][LZ_MAXS + 1];
  __shared__ double Z[LZ_MAXS][LZ_MAXS + 1];
  __shared__ double rc, rs, rph;
  __shared__ int cont;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int i = t % k, j = t / k;
    double v = 0.0;
    if (i == j) v = alpha[r * LZ_MAXS + i];
    else if (i == j + 1) v = beta[r * LZ_MAXS + j];
    else if (j == i + 1) v = beta[r * LZ_MAXS + i];
    G[i][j] = v;
    Z[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) {
      double fro = 0.0, off = 0.0;
      for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
          fro += G[i][j] * G[i][j];
          if (i != j) off += G[i][j] * G[i][j];
        }
      cont = (k > 1) && (sqrt(off) > 1e-15 * sqrt(fro)) && fro > 0.0;
    }
    __syncthreads();
    if (!cont) break;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        if (threadIdx.x == 0) {
          double g = G[p][q];
          double ag = fabs(g);
          if (ag == 0.0) {
            rc = 1.0;
            rs = 0.0;
            rph = 1.0;
          } else {
            double z = (G[q][q] - G[p][p]) / (2.0 * ag);
            double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
            rc = 1.0 / sqrt(1.0 + t * t);
            rs = t * rc;
            rph = g > 0 ? 1.0 : -1.0;
          }
        }
        __syncthreads();
        double c = rc, sn = rs, ph = rph;
        if (sn != 0.0) {
          double Jpp = c, Jpq = sn, Jqp = -sn * ph, Jqq = c * ph;
          int i = threadIdx.x;
          if (i < k) {
            double cp = G[i][p], cq = G[i][q];
            G[i][p] = cp * Jpp + cq * Jqp;
            G[i][q] = cp * Jpq + cq * Jqq;
          }
          __syncthreads();
          if (i < k) {
            double rp = G[p][i], rq = G[q][i];
            G[p][i] = Jpp * rp + Jqp * rq;
            G[q][i] = Jpq * rp + Jqq * rq;
          }
          __syncthreads();
          if (i == 0) {
            G[p][q] = 0.0;
            G[q][p] = 0.0;
          }
          if (i < k) {
            double zp = Z[i][p], zq = Z[i][q];
            Z[i][p] = zp * Jpp + zq * Jqp;
            Z[i][q] = zp * Jpq + zq * Jqq;
          }
        }
        __syncthreads();
      }
  }
  if (threadIdx.x == 0 && sweep >= 60) atomicMax(status, 1);
  // ascending (stable) order of the diagonal
  int i = threadIdx.x;
  if (i < k) {
    double wi = G[i][i];
    int rank = 0;
    for (int j = 0; j < k; ++j) rank += (G[j][j] < wi) || (G[j][j] == wi && j < i);
    theta[r * LZ_MAXS + rank] = wi;
    tau2[r * LZ_MAXS + rank] = Z[0][i] * Z[0][i];
  }
}

// b_sup, mu_1, mu_ne (DoS quantile), theta_max
__global__ void lanczos_bounds_kernel(int runs, int steps, int64_t n, int ne, const double* theta, const double* tau2,
                                      const double* beta, double* out4) {
  if (threadIdx.x != 0) return;
  double b_sup = -1e308, mu1 = 1e308, tmax = -1e308;
  for (int r = 0; r < runs; ++r) {
    b_sup = fmax(b_sup, theta[r * LZ_MAXS + steps - 1] + fabs(beta[r * LZ_MAXS + steps - 1]));
    mu1 = fmin(mu1, theta[r * LZ_MAXS]);
    tmax = fmax(tmax, theta[r * LZ_MAXS + steps - 1]);
  }
  // stable selection through the pooled (theta, weight) list in ascending theta
  int total = runs * steps;
  double target = (double)ne / (double)n;
  double acc = 0.0;
  double mu_ne = -1e308;
  double last_t = -1e308;
  int last_idx = -1;
  for (int cnt = 0; cnt < total; ++cnt) {
    // next element in (theta, index) order after (last_t, last_idx)
    double best_t = 1e308;
    int best = -1;
    for (int idx = 0; idx < total; ++idx) {
      int r = idx / steps, j = idx % steps;
      double t = theta[r * LZ_MAXS + j];
      bool after = (t > last_t) || (t == last_t && idx > last_idx);
      bool better = (t < best_t) || (t == best_t && idx < best);
      if (after && (best < 0 || better)) {
        best_t = t;
        best = idx;
      }
    }
    int r = best / steps, j = best % steps;
    acc += tau2[r * LZ_MAXS + j] / runs;
    last_t = best_t;
    last_idx = best;
    mu_ne = best_t;
    if (acc >= target) break;
  }
  double span = b_sup - mu1;
  double lo = mu1 + 1e-3 * span, hi = b_sup - 1e-3 * span;
  mu_ne = fmin(fmax(mu_ne, lo), hi);
  out4[0] = b_sup;
  out4[1] = mu1;
  out4[2] = mu_ne;
  out4[3] = tmax;
}

template <typename T>
void lanczos(cudaStream_t st, const T* A, int64_t n, int64_t lda, int ne, const T* L0, int runs, int steps,
             double* out4, T* work, int64_t work_elems, double* dwork, const MatvecFn<T>* matvec) {
  CHASE_REQUIRE(runs >= 1 && runs <= LZ_MAXR, 1, "lanczos: 1 <= runs <= 8");
  CHASE_REQUIRE(steps >= 1 && steps <= LZ_MAXS && steps <= n, 1, "lanczos: 1 <= steps <= min(64, n)");
  int64_t nchunk = ceil_div(n, HEMV_COLS);
  // workspace (scalars): basis runs*steps*n | W runs*n | part max(nchunk*runs*n, runs*DOT_CHUNKS*LZ_MAXS)
  //                      | d runs*LZ_MAXS | coef runs*LZ_MAXS
  int64_t need_part = std::max<int64_t>(nchunk * runs * n, (int64_t)runs * DOT_CHUNKS * LZ_MAXS);
  int64_t need = (int64_t)runs * steps * n + runs * n + need_part + 2 * runs * LZ_MAXS;
  CHASE_REQUIRE(work_elems >= need, 2, "lanczos: workspace too small");
  T* Vb = work;
  T* W = Vb + (int64_t)runs * steps * n;
  T* part = W + (int64_t)runs * n;
  T* d = part + need_part;
  T* coef = d + runs * LZ_MAXS;
  // dwork: alpha, beta, theta, tau2 (runs*LZ_MAXS each) + status
  double* alpha = dwork;
  double* beta = alpha + LZ_MAXR * LZ_MAXS;
  double* theta = beta + LZ_MAXR * LZ_MAXS;
  double* tau2 = theta + LZ_MAXR * LZ_MAXS;
  int* status = reinterpret_cast<int*>(tau2 + LZ_MAXR * LZ_MAXS);
  CHASE_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));

  lanczos_start_kernel<T><<<runs, 256, 0, st>>>(n, steps, L0, Vb);
  CHASE_CHECK_LAUNCH();
  // the j-th basis vectors of all runs are not contiguous: gather them into a (n x runs) block
  // by using the HEMV input stride: basis vector j of run r sits at Vb + r*n*steps + j*n, so the
  // "ldx" between runs is n*steps.
  for (int j = 0; j < steps; ++j) {
    const T* X = Vb + (int64_t)j * n;
    if (matvec) {
      (*matvec)(X, n * steps, W);
    } else {
      dim3 g1(ceil_div(n, HEMV_ROWS), nchunk);
      switch (runs) {
#define CASE(R) case R: hemv_multi_kernel<T, R><<<g1, HEMV_ROWS, 0, st>>>(n, A, lda, X, n * steps, part); break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
      }
      CHASE_CHECK_LAUNCH();
      hemv_reduce_kernel<T><<<ceil_div(n * runs, 256), 256, 0, st>>>(n, runs, (int)nchunk, part, W, n);
      CHASE_CHECK_LAUNCH();
    }
    int m = j + 1;
    // alpha_j and the three-term update
    basis_dots_kernel<T><<<dim3(DOT_CHUNKS, runs), 256, 0, st>>>(n, m, steps, Vb, W, part);
    CHASE_CHECK_LAUNCH();
    dots_reduce_kernel<T><<<runs, LZ_MAXS, 0, st>>>(runs, m, part, d);
    CHASE_CHECK_LAUNCH();
    lanczos_coef3_kernel<T><<<1, 32, 0, st>>>(runs, j, d, coef, alpha, beta);
    CHASE_CHECK_LAUNCH();
    basis_update_kernel<T><<<dim3(ceil_div(n, 256), runs), 256, 0, st>>>(n, m, steps, Vb, W, coef);
    CHASE_CHECK_LAUNCH();
    // one full classical Gram-Schmidt pass against the run's basis
    basis_dots_kernel<T><<<dim3(DOT_CHUNKS, runs), 256, 0, st>>>(n, m, steps, Vb, W, part);
    CHASE_CHECK_LAUNCH();
    dots_reduce_kernel<T><<<runs, LZ_MAXS, 0, st>>>(runs, m, part, d);
    CHASE_CHECK_LAUNCH();
    basis_update_kernel<T><<<dim3(ceil_div(n, 256), runs), 256, 0, st>>>(n, m, steps, Vb, W, d);
    CHASE_CHECK_LAUNCH();
    lanczos_norm_kernel<T><<<runs, 256, 0, st>>>(n, steps, j, W, Vb, beta);
    CHASE_CHECK_LAUNCH();
  }
  tridiag_jacobi_kernel<<<runs, LZ_MAXS, 0, st>>>(steps, alpha, beta, theta, tau2, status);
  CHASE_CHECK_LAUNCH();
  lanczos_bounds_kernel<<<1, 32, 0, st>>>(runs, steps, n, ne, theta, tau2, beta, out4);
  CHASE_CHECK_LAUNCH();
}

template void lanczos<double>(cudaStream_t, const double*, int64_t, int64_t, int, const double*, int, int, double*,
                              double*, int64_t, double*, const MatvecFn<double>*);
template void lanczos<double2>(cudaStream_t, const double2*, int64_t, int64_t, int, const double2*, int, int, double*,
                               double2*, int64_t, double*, const MatvecFn<double2>*);

}  // namespace chase
