// Adjoint of the partial eigendecomposition (lambda, V) = lowest eigenpairs of a real
// symmetric A (the differentiation form beside Algorithm 1; the paper has no
// backward).  With S the set of converged (locked) pairs, gbar and Vbar padded by
// zeros outside the returned nev pairs:
//   Abar = V_S (diag(gbar_S) + F o (V_S^T Vbar_S)) V_S^T + X V^T,
//   F_ij = 1/(lambda_j - lambda_i) (i != j, 0 on the diagonal),
// and column x_j of X solves P (A - lambda_j I) P x_j = -P vbar_j on range(P),
// P = I - V_S V_S^T, by MINRES (Paige & Saunders), all nev columns at once: one
// A-times-block product per iteration (split tensor-core products) and one block
// per column for the recurrences.  Abar is symmetrised at the end.
#include "common.cuh"
#include "kernels.h"

namespace chase {

// inner(i, j) for i < l, j < nev: (i == j ? gl_j : 0) + F_ij M_ij
__global__ void adj_inner_kernel(int l, int nev, const double* lam, const double* M, int64_t ldm, const double* gl,
                                 double* inner, int64_t ldi) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= l || j >= nev) return;
  double v = 0.0;
  if (i == j) {
    v = gl ? gl[j] : 0.0;
  } else if (M) {
    v = M[i + (int64_t)j * ldm] / (lam[j] - lam[i]);
  }
  inner[i + (int64_t)j * ldi] = v;
}

struct MinresState {
  double beta1, beta, oldb, dbar, epsln, phibar, cs, sn;
  int done, itn;
};

// y = b (stored in R1 and R2), v = b / ||b||, scalars; one block per column
__global__ void minres_init_kernel(int64_t n, const double* B, int64_t ldb, double* R1, double* R2, double* Vv,
                                   double* X, double* W, double* W2, MinresState* st, double tol) {
  int j = blockIdx.x;
  const double* b = B + (int64_t)j * ldb;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += b[i] * b[i];
  __shared__ double red[32];
  __shared__ double nb;
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    nb = sqrt(s);
    MinresState m;
    m.beta1 = nb;
    m.beta = nb;
    m.oldb = 0.0;
    m.dbar = 0.0;
    m.epsln = 0.0;
    m.phibar = nb;
    m.cs = -1.0;
    m.sn = 0.0;
    m.done = (nb == 0.0) ? 1 : 0;
    m.itn = 0;
    st[j] = m;
  }
  __syncthreads();
  const double inv = nb > 0.0 ? 1.0 / nb : 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t o = i + (int64_t)j * n;
    R1[o] = b[i];
    R2[o] = b[i];
    Vv[o] = b[i] * inv;
    X[o] = 0.0;
    W[o] = 0.0;
    W2[o] = 0.0;
  }
}

__device__ inline double block_sum(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;  // valid in thread 0
}

// One MINRES iteration after Y = P (A - lambda_j I) v (one block per column).
// In place: R1 <- new r2 (= y), Wold1 <- new w, Vv <- next v; the host rotates buffer roles.
__global__ void minres_update_kernel(int64_t n, const double* __restrict__ Y, double* R1, const double* R2,
                                     double* Vv, double* Wn /* in: w1, out: new w */, const double* Wc /* w */,
                                     double* X, MinresState* st, double tol) {
  const int j = blockIdx.x;
  __shared__ double red[32];
  __shared__ double sh[8];
  __shared__ int skip;
  if (threadIdx.x == 0) skip = st[j].done;
  __syncthreads();
  if (skip) return;
  const int64_t off = (int64_t)j * n;
  const MinresState m0 = st[j];
  const double kr1 = (m0.itn >= 1) ? m0.beta / m0.oldb : 0.0;  // y -= (beta/oldb) r1 from the 2nd iteration on
  // pass 1: alfa = v . (Y - kr1 r1)
  double d = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) d += Vv[off + i] * (Y[off + i] - kr1 * R1[off + i]);
  double alfa = block_sum(d, red);
  if (threadIdx.x == 0) sh[0] = alfa;
  __syncthreads();
  alfa = sh[0];
  const double ka = alfa / m0.beta;
  // pass 2: y = Y - kr1 r1 - ka r2 (written over r1), ||y||^2
  double q = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double y = Y[off + i] - kr1 * R1[off + i] - ka * R2[off + i];
    R1[off + i] = y;
    q += y * y;
  }
  double yy = block_sum(q, red);
  if (threadIdx.x == 0) {
    MinresState m = m0;
    m.oldb = m.beta;
    m.beta = sqrt(yy);
    const double oldeps = m.epsln;
    const double delta = m.cs * m.dbar + m.sn * alfa;
    const double gbar = m.sn * m.dbar - m.cs * alfa;
    m.epsln = m.sn * m.beta;
    m.dbar = -m.cs * m.beta;
    double gamma = hypot(gbar, m.beta);
    if (gamma < 1e-300) gamma = 1e-300;
    m.cs = gbar / gamma;
    m.sn = m.beta / gamma;
    const double phi = m.cs * m.phibar;
    m.phibar = m.sn * m.phibar;
    m.itn += 1;
    if (m.phibar <= tol * m.beta1 || m.beta == 0.0) m.done = 1;
    st[j] = m;
    sh[1] = oldeps;
    sh[2] = delta;
    sh[3] = gamma;
    sh[4] = phi;
    sh[5] = m.beta > 0.0 ? 1.0 / m.beta : 0.0;
  }
  __syncthreads();
  const double oldeps = sh[1], delta = sh[2], ginv = 1.0 / sh[3], phi = sh[4], binv = sh[5];
  // pass 3: w = (v - oldeps w1 - delta w2)/gamma over w1; x += phi w; v <- y / beta
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double w = (Vv[off + i] - oldeps * Wn[off + i] - delta * Wc[off + i]) * ginv;
    Wn[off + i] = w;
    X[off + i] += phi * w;
    Vv[off + i] = R1[off + i] * binv;
  }
}

__global__ void count_done_kernel(int nev, const MinresState* st, int* out) {
  int c = 0;
  for (int j = threadIdx.x; j < nev; j += 32) c += st[j].done;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (threadIdx.x == 0) *out = c;
}

__global__ void add_kernel(int64_t count, double* a, const double* b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) a[i] += b[i];
}

void adj_inner(cudaStream_t st, int l, int nev, const double* lam, const double* M, int64_t ldm, const double* gl,
               double* inner, int64_t ldi) {
  adj_inner_kernel<<<dim3(ceil_div(l, 128), nev), 128, 0, st>>>(l, nev, lam, M, ldm, gl, inner, ldi);
  CHASE_CHECK_LAUNCH();
}

void minres_init(cudaStream_t st, int64_t n, int nev, const double* B, int64_t ldb, double* R1, double* R2,
                 double* Vv, double* X, double* W, double* W2, void* state, double tol) {
  minres_init_kernel<<<nev, 256, 0, st>>>(n, B, ldb, R1, R2, Vv, X, W, W2, (MinresState*)state, tol);
  CHASE_CHECK_LAUNCH();
}

void minres_update(cudaStream_t st, int64_t n, int nev, const double* Y, double* R1, const double* R2, double* Vv,
                   double* Wn, const double* Wc, double* X, void* state, double tol) {
  minres_update_kernel<<<nev, 256, 0, st>>>(n, Y, R1, R2, Vv, Wn, Wc, X, (MinresState*)state, tol);
  CHASE_CHECK_LAUNCH();
}

void minres_count_done(cudaStream_t st, int nev, const void* state, int* out) {
  count_done_kernel<<<1, 32, 0, st>>>(nev, (const MinresState*)state, out);
  CHASE_CHECK_LAUNCH();
}

void add_inplace(cudaStream_t st, int64_t count, double* a, const double* b) {
  add_kernel<<<ceil_div(count, 256), 256, 0, st>>>(count, a, b);
  CHASE_CHECK_LAUNCH();
}

size_t minres_state_bytes(int nev) { return (size_t)nev * sizeof(MinresState); }

}  // namespace chase
