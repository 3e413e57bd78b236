// Deflation & locking, bound update, degree optimisation and degree sort
// (Algorithm 1, lines 8-14) for the k active Ritz pairs, in one block.
//
// Inputs: ritz[0..k) ascending, res[0..k) absolute residual norms,
// thresh = tol * ||A||_est.  bounds[] = {b_sup, mu_1, mu_ne, c, e, locked_min}.
// Readings (the paper gives no formulas): prefix locking; mu_1 = min(locked,
// active), mu_ne = max(active remaining); degree m = ceil(ln(res/thresh)/ln rho)
// + extra with rho = |t| + sqrt(t^2-1), t = (lambda - c)/e, clamped to
// [1, maxdeg] (|t| <= 1 or rho <= 1+1e-12 gives maxdeg); stable sort by
// (m, lambda).
#include "common.cuh"
#include "kernels.h"

namespace chase {

__global__ void bookkeeping_kernel(int k, const double* __restrict__ ritz, const double* __restrict__ res,
                                   double thresh, double* bounds, int maxdeg, int extra_deg, int* out_lock,
                                   int* out_deg, int* out_perm, double* out_ritz, double* out_res, int* mtmp) {
  __shared__ int p_sh;
  __shared__ double c_sh, e_sh;
  if (threadIdx.x == 0) {
    int p = 0;
    while (p < k && res[p] <= thresh) ++p;
    p_sh = p;
    double b_sup = bounds[0];
    double lmin = bounds[5];
    for (int a = 0; a < p; ++a) lmin = fmin(lmin, ritz[a]);
    double mu1 = lmin;
    for (int a = p; a < k; ++a) mu1 = fmin(mu1, ritz[a]);
    double mu_ne = bounds[2];
    if (k - p > 0) {
      mu_ne = ritz[p];
      for (int a = p; a < k; ++a) mu_ne = fmax(mu_ne, ritz[a]);
    }
    double c = 0.5 * (b_sup + mu_ne), e = 0.5 * (b_sup - mu_ne);
    bounds[1] = mu1;
    bounds[2] = mu_ne;
    bounds[3] = c;
    bounds[4] = e;
    bounds[5] = lmin;
    c_sh = c;
    e_sh = e;
    *out_lock = p;
  }
  __syncthreads();
  const int p = p_sh;
  const int kr = k - p;
  const double c = c_sh, e = e_sh;
  for (int a = threadIdx.x; a < kr; a += blockDim.x) {
    double w = ritz[p + a];
    double t = (w - c) / e;
    int m;
    if (fabs(t) <= 1.0) {
      m = maxdeg;
    } else {
      double rho = fabs(t) + sqrt(t * t - 1.0);
      if (rho <= 1.0 + 1e-12) {
        m = maxdeg;
      } else {
        double ratio = res[p + a] / thresh;
        m = ratio > 0.0 ? (int)ceil(log(ratio) / log(rho)) + extra_deg : 1;
        m = min(max(m, 1), maxdeg);
      }
    }
    mtmp[a] = m;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < kr; a += blockDim.x) {
    int ma = mtmp[a];
    double wa = ritz[p + a];
    int rank = 0;
    for (int b = 0; b < kr; ++b) {
      int mb = mtmp[b];
      double wb = ritz[p + b];
      rank += (mb < ma) || (mb == ma && (wb < wa || (wb == wa && b < a)));
    }
    out_deg[rank] = ma;
    out_perm[rank] = p + a;
    out_ritz[rank] = wa;
    out_res[rank] = res[p + a];
  }
}

void bookkeeping(cudaStream_t st, int k, const double* ritz, const double* res, double thresh, double b_sup,
                 double* bounds, int maxdeg, int extra_deg, int* out_lock, int* out_deg, int* out_perm,
                 double* out_ritz, double* out_res, int* scratch) {
  (void)b_sup;
  bookkeeping_kernel<<<1, 1024, 0, st>>>(k, ritz, res, thresh, bounds, maxdeg, extra_deg, out_lock, out_deg, out_perm,
                                         out_ritz, out_res, scratch);
  CHASE_CHECK_LAUNCH();
}

}  // namespace chase
