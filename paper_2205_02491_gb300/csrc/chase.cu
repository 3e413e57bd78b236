// ChASE driver (Algorithm 1) on one GPU and the C ABI declared in
// include/chase_gb300.h.
//
// Device-resident loop: the start block, the locked prefix and the active
// block share one n x ne buffer V (locked columns [0, l), active [l, ne)); two
// more n x ne buffers hold the filter's ping-pong partner / Ritz vectors (T1)
// and A Q (T2).  Per outer iteration the host reads one small status record
// (locked count, degrees, bounds) to size the next filter launches; nothing
// else crosses the host-device boundary (the paper does one transfer per
// iteration too, Section "Offloading Selected Routines to GPUs").
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "kernels.h"
#include "oz.h"

using namespace chase;

namespace chase {
std::atomic<long long> g_kernel_launches{0};
std::atomic<unsigned long long> g_wait_limit_ns{0};
}

struct chase_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  chase_dtype dtype = CHASE_C128;
  chase_opts opts{};
  int64_t n_max = 0;
  int ne_max = 0;
  size_t esz = 16;  // scalar size
  // workspace
  void* V = nullptr;
  void* T1 = nullptr;
  void* T2 = nullptr;
  void* G = nullptr;
  void* Z = nullptr;
  void* work = nullptr;
  int64_t work_elems = 0;
  double* dwork = nullptr;
  int64_t dwork_elems = 0;
  int* iwork = nullptr;
  double* ritz = nullptr;
  double* res = nullptr;
  double* ritz2 = nullptr;
  double* res2 = nullptr;
  double* lam_locked = nullptr;
  double* bounds = nullptr;
  double* eigvals = nullptr;
  double* lam_sorted = nullptr;  // all locked eigenvalues of the last solve, ascending
  int l_final = 0;               // locked pairs of the last solve
  double* bwd = nullptr;         // adjoint work: 9 blocks n x nev (allocated on first backward)
  void* a_stage = nullptr;       // device copy of a host A (allocated on the first solve given one)
  size_t a_stage_bytes = 0;
  void* l0_stage = nullptr;      // device copy of host Lanczos start vectors (n_max x 8)
  size_t bwd_bytes = 0;
  int* deg = nullptr;
  int* perm = nullptr;
  int* info = nullptr;
  int* status_dev = nullptr;
  int* qr_dep = nullptr;             // Cholesky-QR dependent-column flags (count, then ne_max flags)
  void* hh = nullptr;                // Householder QR scratch: 3 x 32 x ne_max + ne_max + 1024 scalars
  oz::Workspace ozw{};
  // result state
  bool have_result = false;
  int64_t n = 0;
  int nev = 0, nex = 0;
  chase_stats_t stats{};
  std::string err;
  cudaEvent_t ev[8] = {};
  // batched solves: opts.batch_workers - 1 more contexts, each with its own stream
  std::vector<chase_ctx*> workers;
  // grouped batched solves: one context per problem (sized to it, own stream), kept between calls
  std::vector<chase_ctx*> slots;
  cudaStream_t filter_stream = nullptr;  // stream of the grouped filter launches
};

namespace {

struct Timer {
  cudaStream_t st;
  cudaEvent_t a, b;
  double* acc;
  Timer(chase_ctx* c, int slot, double* acc_) : st(c->stream), a(c->ev[2 * slot]), b(c->ev[2 * slot + 1]), acc(acc_) {
    CHASE_CUDA(cudaEventRecord(a, st));
  }
  void stop() {
    CHASE_CUDA(cudaEventRecord(b, st));
    CHASE_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    CHASE_CUDA(cudaEventElapsedTime(&ms, a, b));
    *acc += ms;
  }
};

bool verbose() {
  static const bool v = []() {
    const char* e = getenv("CHASE_VERBOSE");
    return e && e[0] && e[0] != '0';
  }();
  return v;
}

void filter_coeffs(double b_sup, double mu_1, double mu_ne, int mmax, double& c, double& e, std::vector<double>& al,
                   std::vector<double>& be) {
  // Scaled three-term recurrence (Eq. three-terms-recurrence) with gamma = c:
  // Y_1 = (sigma_1/e)(A - cI)Y_0, Y_{s+1} = (2 sigma_{s+1}/e)(A - cI)Y_s - sigma_s sigma_{s+1} Y_{s-1},
  // sigma_1 = e/(mu_1 - c), sigma_{s+1} = 1/(2/sigma_1 - sigma_s).
  c = 0.5 * (b_sup + mu_ne);
  e = 0.5 * (b_sup - mu_ne);
  double sigma1 = e / (mu_1 - c);
  al.assign(mmax + 1, 0.0);
  be.assign(mmax + 1, 0.0);
  double sigma = sigma1;
  if (mmax >= 1) al[1] = sigma1 / e;
  for (int s = 1; s < mmax; ++s) {
    double sn = 1.0 / (2.0 / sigma1 - sigma);
    al[s + 1] = 2.0 * sn / e;
    be[s + 1] = -sigma * sn;
    sigma = sn;
  }
}

template <typename T> __global__ void gather_odd_kernel(int64_t n, const int* deg, T* V, int64_t ldv, const T* Y1, int64_t ldy) {
  int a = blockIdx.y;
  if ((deg[a] & 1) == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    V[i + a * ldv] = Y1[i + a * ldy];
}

__global__ void fill_int_kernel(int n, int* x, int v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}

__global__ void init_bounds_kernel(const double* lz4, double* bounds) {
  bounds[0] = lz4[0];
  bounds[1] = lz4[1];
  bounds[2] = lz4[2];
  bounds[3] = 0.5 * (lz4[0] + lz4[2]);
  bounds[4] = 0.5 * (lz4[0] - lz4[2]);
  bounds[5] = 1e308;
}

__global__ void nan_check_kernel(int64_t n, int k, const double* X, int64_t ldx, int* flag) {
  // X viewed as doubles: n rows (already scaled by scalar width) x k columns
  int a = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(X[i + a * ldx])) atomicOr(flag, 1);
}

// rank-sort the l locked eigenvalues, output first nev ascending and the permutation
__global__ void final_sort_kernel(int l, int nev, const double* lam, double* out, double* all, int* perm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= l) return;
  double wi = lam[i];
  int rank = 0;
  for (int j = 0; j < l; ++j) rank += (lam[j] < wi) || (lam[j] == wi && j < i);
  perm[rank] = i;
  all[rank] = wi;
  if (rank < nev) out[rank] = wi;
}

// MINRES helpers for the adjoint (real symmetric) ------------------------------------------
struct MinresScalars {
  double beta1, beta, oldb, dbar, epsln, phibar, cs, sn, alfa, phi, gamma, delta, oldeps, shift;
  int active;
};

}  // namespace

// =====================================================================================
template <typename T> struct Solver {
  chase_ctx* c;
  explicit Solver(chase_ctx* ctx) : c(ctx) {}
  T* V() { return (T*)c->V; }
  T* T1() { return (T*)c->T1; }
  T* T2() { return (T*)c->T2; }
  T* Gb() { return (T*)c->G; }
  T* Zb() { return (T*)c->Z; }
  T* W() { return (T*)c->work; }
  cudaStream_t st() { return c->stream; }

  void check_nan(const T* X, int64_t n, int k, int64_t ld, const char* what) {
    CHASE_CUDA(cudaMemsetAsync(c->status_dev, 0, sizeof(int), st()));
    int64_t rows = n * (int64_t)(sizeof(T) / sizeof(double));
    dim3 grid(std::min<unsigned>(ceil_div(rows, 256), 64), k);
    nan_check_kernel<<<grid, 256, 0, st()>>>(rows, k, (const double*)X, ld * (int64_t)(sizeof(T) / sizeof(double)),
                                             c->status_dev);
    CHASE_CHECK_LAUNCH();
    int flag = 0;
    CHASE_CUDA(cudaMemcpyAsync(&flag, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost, st()));
    CHASE_CUDA(cudaStreamSynchronize(st()));
    CHASE_REQUIRE(flag == 0, CHASE_ERR_NAN, std::string("non-finite values in ") + what);
  }

  // C(n x k) = A(n x n) * B(n x k) with epilogue, in the given filter arithmetic.
  void hemm(const T* A, int64_t n, int64_t lda, const T* B, int64_t ldb, int k, const Epi& e, int mode) {
    CHASE_REQUIRE(mode == CHASE_FP64_NATIVE || oz::available(), CHASE_ERR_UNSUPPORTED,
                  "the split tensor-core products need an sm_103 device; only CHASE_FP64_NATIVE runs here");
    if (mode == CHASE_FP64_NATIVE) {
      gemm_f64<T>(st(), OP_N, OP_N, n, k, n, A, lda, B, ldb, e, W(), c->work_elems);
    } else {
      oz::prepare_A<T>(st(), c->ozw, A, n, lda, mode);  // cached per A within a call
      oz::hemm<T>(st(), c->ozw, A, n, lda, B, ldb, k, e, mode);
    }
  }

  // C = op(A) op(B) with FP64 accuracy: split tensor-core products for large shapes, DFMA for
  // small ones (and always in the native mode).  Split products may write C over an operand.
  bool use_split(int mode, int64_t M, int64_t N, int64_t K) {
    if (mode == CHASE_FP64_NATIVE || !oz::available()) return false;
    double mflop = (S<T>::cplx ? 8.0 : 2.0) * (double)M * (double)N * (double)K * 1e-6;
    return mflop >= (double)c->opts.native_below_mflop;
  }
  // force_split: the split tensor-core product whatever the size (for the skinny products of a long loop,
  // which split along K where DFMA tiles stay latency-bound)
  void gemm(Op opA, const T* A, int64_t lda, Op opB, const T* B, int64_t ldb, int64_t M, int64_t N, int64_t K,
            const Epi& e, int mode, bool force_split = false) {
    if ((force_split && mode != CHASE_FP64_NATIVE && oz::available()) || use_split(mode, M, N, K))
      oz::gemm<T>(st(), c->ozw, opA, A, lda, opB, B, ldb, M, N, K, e, CHASE_FP64);
    else
      gemm_f64<T>(st(), opA, opB, M, N, K, A, lda, B, ldb, e, W(), c->work_elems);
  }

  // L (k x k lower, diagonal CB-blocks already inverted) -> L^{-1} by recursive halving:
  // [[A, 0], [B, C]]^{-1} = [[A^-1, 0], [-C^-1 B A^-1, C^-1]].  tmp: k*k/4 scalars.
  void trtri_combine(T* L, int64_t ld, int k, T* tmp, int mode) {
    if (k <= 32) return;
    int k1 = ((k / 2 + 31) / 32) * 32;
    if (k1 >= k) k1 = k - 32;
    const int k2 = k - k1;
    trtri_combine(L, ld, k1, tmp, mode);
    trtri_combine(L + k1 + (int64_t)k1 * ld, ld, k2, tmp, mode);
    T* B = L + k1;
    Epi e1;
    e1.C = tmp;
    e1.ldc = k2;
    gemm(OP_N, B, ld, OP_N, L, ld, k2, k1, k1, e1, mode);  // tmp = B A^-1
    Epi e2;
    e2.C = B;
    e2.ldc = ld;
    e2.alpha = -1.0;
    gemm(OP_N, L + k1 + (int64_t)k1 * ld, ld, OP_N, tmp, k2, k2, k1, k2, e2, mode);  // B = -C^-1 tmp
  }

  // Y_s (n x k, ld n) <- Q with Y_s = Q R (Cholesky-QR2 with column equilibration) and Y_p <- Y_p R^{-1}:
  // both iterates of the three-term recurrence take the same right factor, so the recurrence goes on
  // and the filtered block keeps its span.  Returns false (both blocks rescaled consistently, otherwise
  // as they were after the last completed pass) when a Cholesky factorisation fails.
  bool orthonormalize_pair(T* Ys, T* Yp, int64_t n, int k) {
    T* Gm = Gb();
    for (int pass = 0; pass < 2; ++pass) {
      colnorms<T>(st(), n, k, Ys, n, c->dwork);
      scale_cols<T>(st(), n, k, Ys, n, c->dwork, 1);
      scale_cols<T>(st(), n, k, Yp, n, c->dwork, 1);
      Epi e;
      e.C = Gm;
      e.ldc = k;
      gemm(OP_C, Ys, n, OP_N, Ys, n, k, k, n, e, CHASE_FP64);
      hermitianize<T>(st(), k, Gm, k);
      CHASE_CUDA(cudaMemsetAsync(c->info, 0, sizeof(int), st()));
      potrf_lower<T>(st(), k, Gm, k, c->info, W(), c->work_elems);
      int info = 0;
      CHASE_CUDA(cudaMemcpyAsync(&info, c->info, sizeof(int), cudaMemcpyDeviceToHost, st()));
      CHASE_CUDA(cudaStreamSynchronize(st()));
      if (info != 0) return false;
      if (use_split(CHASE_FP64, n, k, k)) {
        zero_upper<T>(st(), k, Gm, k);
        trtri_diag<T>(st(), k, Gm, k);
        trtri_combine(Gm, k, k, Zb(), CHASE_FP64);
        for (T* X : {Ys, Yp}) {
          Epi q;
          q.C = X;
          q.ldc = n;
          gemm(OP_N, X, n, OP_C, Gm, k, n, k, k, q, CHASE_FP64);
        }
      } else {
        trsm_right_lh<T>(st(), n, k, Ys, n, Gm, k, W(), c->work_elems);
        trsm_right_lh<T>(st(), n, k, Yp, n, Gm, k, W(), c->work_elems);
      }
    }
    return true;
  }

  // ------------------------------------------------------------ Algorithm 1, line 4
  // Filter the k columns of Y0 (ld n) in place; T1 (ld n) is the ping-pong partner.
  // deg_host non-decreasing; deg_dev the same on the device.
  // reorth: when every column has the same degree (the first outer iteration) and the filter would
  // amplify the component along mu_1 by more than 1e7 over the damped interval, the iterate is
  // orthonormalised (with the previous one carried along) every s_split steps, keeping each stretch's
  // amplification below 1e7.  In exact arithmetic the filtered span is unchanged; it keeps the block
  // within reach of the Cholesky-QR of line 5 (a Householder QR copes with any conditioning, a
  // Cholesky-QR only with about 1e8).
  int64_t filter(const T* A, int64_t n, int64_t lda, T* Y0, T* Y1, int k, const int* deg_host, const int* deg_dev,
                 double b_sup, double mu_1, double mu_ne, int mode, bool reorth = false) {
    if (k <= 0) return 0;
    int mmax = deg_host[k - 1];
    double cc, ee;
    std::vector<double> al, be;
    filter_coeffs(b_sup, mu_1, mu_ne, mmax, cc, ee, al, be);
    int s_split = mmax + 1;
    if (reorth && k >= 2 && deg_host[0] == mmax) {
      const double t1 = std::fabs((mu_1 - cc) / ee);
      const double rho = t1 > 1.0 ? t1 + std::sqrt(t1 * t1 - 1.0) : 1.0;
      if (rho > 1.0 + 1e-12) s_split = std::max(1, (int)std::floor(std::log(1e7) / std::log(rho)));
    }
    T* B[2] = {Y0, Y1};
    int f = 0;
    int64_t mv = 0;
    for (int s = 1; s <= mmax; ++s) {
      while (f < k && deg_host[f] < s) ++f;
      int cols = k - f;
      if (cols <= 0) break;
      mv += cols;
      T* out = B[s & 1] + (int64_t)f * n;
      const T* in = B[(s - 1) & 1] + (int64_t)f * n;
      Epi e;
      e.C = out;
      e.ldc = n;
      e.alpha = al[s];
      e.Y = in;
      e.ldy = n;
      e.gamma = -al[s] * cc;
      if (s >= 2) {
        e.Z = out;
        e.ldz = n;
        e.beta = be[s];
      }
      hemm(A, n, lda, in, n, cols, e, mode);
      c->stats.filter_launches++;
      if (s % s_split == 0 && s < mmax && orthonormalize_pair(B[s & 1], B[(s - 1) & 1], n, k))
        c->stats.filter_reorth++;
    }
    dim3 grid(std::min<unsigned>(ceil_div(n, 256), 64), k);
    gather_odd_kernel<T><<<grid, 256, 0, st()>>>(n, deg_dev, Y0, n, Y1, n);
    CHASE_CHECK_LAUNCH();
    return mv;
  }

  // ------------------------------------------------------------ Householder QR (line 5, ill-conditioned blocks)
  // X (n x k, ld ldx) <- Q of X = Q R by blocked Householder QR (panels of 32 reflectors, compact-WY
  // trailing updates and Q formation through FP64-class products).  Unlike Cholesky-QR it keeps every
  // direction of X down to rounding, whatever the conditioning (the paper's QR is a Householder geqrf).
  // Scratch: T1 (reflectors, n x k), T2 (Q), hh (panel factors and products), dwork (tau).
  void householder_qr(T* X, int64_t n, int k, int64_t ldx) {
    constexpr int NB = 32;
    T* Vx = T1();
    T* Q = T2();
    T* Tw = (T*)c->hh;               // NB x k: the panels' compact-WY factors
    T* alpha = Tw + (int64_t)NB * k; // k
    T* Gv = alpha + k;               // NB x NB
    T* W1 = Gv + NB * NB;            // NB x k
    T* W2 = W1 + (int64_t)NB * k;    // NB x k
    double* tau = c->dwork;
    for (int j0 = 0; j0 < k; j0 += NB) {
      const int pb = std::min(NB, k - j0);
      const int64_t m = n - j0;
      for (int j = 0; j < pb; ++j) {
        const int col = j0 + j;
        T* x = X + col + (int64_t)col * ldx;
        householder_vec<T>(st(), n - col, x, alpha + col, tau + col);
        householder_apply<T>(st(), n - col, x, x + ldx, ldx, pb - j - 1, tau + col);
      }
      T* Vp = Vx + j0 + (int64_t)j0 * n;  // the panel's reflectors, rows j0.., ld n
      reflector_panel<T>(st(), m, pb, X + j0 + (int64_t)j0 * ldx, ldx, Vp, n);
      Epi eg;
      eg.C = Gv;
      eg.ldc = pb;
      gemm(OP_C, Vp, n, OP_N, Vp, n, pb, pb, m, eg, CHASE_FP64);
      T* Tp = Tw + (int64_t)j0 * NB;
      householder_T<T>(st(), pb, Gv, tau + j0, Tp, NB);
      const int rest = k - j0 - pb;
      if (rest > 0) {
        // X(j0:, j0+pb:) <- (I - V Tp^H V^H) X(j0:, j0+pb:)
        T* Xt = X + j0 + (int64_t)(j0 + pb) * ldx;
        Epi e1;
        e1.C = W1;
        e1.ldc = NB;
        gemm(OP_C, Vp, n, OP_N, Xt, ldx, pb, rest, m, e1, CHASE_FP64);
        Epi e2;
        e2.C = W2;
        e2.ldc = NB;
        gemm(OP_C, Tp, NB, OP_N, W1, NB, pb, rest, pb, e2, CHASE_FP64);
        Epi e3;
        e3.C = Xt;
        e3.ldc = ldx;
        e3.alpha = -1.0;
        e3.Z = Xt;
        e3.ldz = ldx;
        e3.beta = 1.0;
        gemm(OP_N, Vp, n, OP_N, W2, NB, m, rest, pb, e3, CHASE_FP64);
      }
    }
    // Q = H_1 ... H_k [I; 0], panels applied last to first
    identity_rect<T>(st(), n, k, Q, n);
    for (int j0 = ((k - 1) / NB) * NB; j0 >= 0; j0 -= NB) {
      const int pb = std::min(NB, k - j0);
      const int64_t m = n - j0;
      const int cols = k - j0;
      T* Vp = Vx + j0 + (int64_t)j0 * n;
      T* Tp = Tw + (int64_t)j0 * NB;
      T* Qt = Q + j0 + (int64_t)j0 * n;
      Epi e1;
      e1.C = W1;
      e1.ldc = NB;
      gemm(OP_C, Vp, n, OP_N, Qt, n, pb, cols, m, e1, CHASE_FP64);
      Epi e2;
      e2.C = W2;
      e2.ldc = NB;
      gemm(OP_N, Tp, NB, OP_N, W1, NB, pb, cols, pb, e2, CHASE_FP64);
      Epi e3;
      e3.C = Qt;
      e3.ldc = n;
      e3.alpha = -1.0;
      e3.Z = Qt;
      e3.ldz = n;
      e3.beta = 1.0;
      gemm(OP_N, Vp, n, OP_N, W2, NB, m, cols, pb, e3, CHASE_FP64);
    }
    copy_cols<T>(st(), n, k, Q, n, X, ldx);
  }

  // ------------------------------------------------------------ Algorithm 1, line 5
  // X (n x k, ld ldx) <- orthonormal basis of span(X) orthogonal to Y (n x l, ld ldy, orthonormal).
  void qr(const T* Y, int64_t ldy, int l, T* X, int64_t ldx, int64_t n, int k, int qr_mode) {
    if (k <= 0) return;
    T* Gm = Gb();
    // one block classical Gram-Schmidt pass against the locked columns: X -= Y (Y^H X)
    const int pm = qr_mode;
    auto project = [&]() {
      if (l <= 0) return;
      Epi e;
      e.C = Gm;
      e.ldc = l;
      gemm(OP_C, Y, ldy, OP_N, X, ldx, l, k, n, e, pm);
      Epi u;
      u.C = X;
      u.ldc = ldx;
      u.alpha = -1.0;
      u.Z = X;
      u.ldz = ldx;
      u.beta = 1.0;
      gemm(OP_N, Y, ldy, OP_N, Gm, l, n, k, l, u, pm);
    };
    project();
    // column equilibration (does not change the span)
    colnorms<T>(st(), n, k, X, ldx, c->dwork);
    scale_cols<T>(st(), n, k, X, ldx, c->dwork, 1);
    // dep (nullable): detection mode of the Cholesky factorisation; returns false with *ndep > 0 when it
    // found numerically dependent columns (X is then left unchanged)
    int ndep = 0;
    auto chol_pass = [&](double shift_factor, int* dep = nullptr) -> bool {
      Epi e;
      e.C = Gm;
      e.ldc = k;
      gemm(OP_C, X, ldx, OP_N, X, ldx, k, k, n, e, pm);
      hermitianize<T>(st(), k, Gm, k);
      if (shift_factor > 0.0) {
        fro_norm2<T>(st(), n, k, X, ldx, c->dwork);
        double tr = 0.0;
        CHASE_CUDA(cudaMemcpyAsync(&tr, c->dwork, sizeof(double), cudaMemcpyDeviceToHost, st()));
        CHASE_CUDA(cudaStreamSynchronize(st()));
        double shift = shift_factor * ((double)n * k + (double)k * (k + 1)) * 1.1102230246251565e-16 * tr;
        add_diag<T>(st(), k, Gm, k, nullptr, shift);
      }
      CHASE_CUDA(cudaMemsetAsync(c->info, 0, sizeof(int), st()));
      // detection: the columns have unit norm, so the Gram matrix has a unit diagonal and a pivot below
      // 8 (k + sqrt(n)) u lies within the rounding error of the Gram matrix and its factorisation: that
      // column is numerically in the span of the columns before it
      const double floor_dep = 8.0 * ((double)k + std::sqrt((double)n)) * 1.1102230246251565e-16;
      if (dep) CHASE_CUDA(cudaMemsetAsync(dep, 0, (size_t)(k + 1) * sizeof(int), st()));
      potrf_lower<T>(st(), k, Gm, k, c->info, W(), c->work_elems, dep ? floor_dep : 0.0, dep);
      int hinfo[2] = {0, 0};
      CHASE_CUDA(cudaMemcpyAsync(&hinfo[0], c->info, sizeof(int), cudaMemcpyDeviceToHost, st()));
      if (dep) CHASE_CUDA(cudaMemcpyAsync(&hinfo[1], dep, sizeof(int), cudaMemcpyDeviceToHost, st()));
      CHASE_CUDA(cudaStreamSynchronize(st()));
      ndep = hinfo[1];
      if (hinfo[0] != 0 || ndep > 0) return false;
      if (use_split(pm, n, k, k)) {
        // X <- X L^{-H} as one product with the explicit triangular inverse (written over X)
        zero_upper<T>(st(), k, Gm, k);
        trtri_diag<T>(st(), k, Gm, k);
        trtri_combine(Gm, k, k, Zb(), pm);
        Epi q;
        q.C = X;
        q.ldc = ldx;
        gemm(OP_N, X, ldx, OP_C, Gm, k, n, k, k, q, pm);
      } else {
        trsm_right_lh<T>(st(), n, k, X, ldx, Gm, k, W(), c->work_elems);
      }
      return true;
    };
    // Cholesky-QR2 with a projection before each pass, so the final basis is orthogonal to the
    // locked columns to rounding even when X was ill-conditioned.  A filtered block can be numerically
    // rank deficient for a Cholesky-QR (eigen-directions amplified beyond about 1e8 over others): the
    // first pass then finds columns whose remainder after the columns before them is within the
    // rounding of the Gram matrix.  Such a block goes to the Householder QR, which keeps those
    // directions down to rounding; its basis is then projected against the locked columns once more and
    // re-orthonormalised by Cholesky-QR2 (now well conditioned).
    bool ok = chol_pass(0.0, c->qr_dep);
    if (!ok && ndep > 0) {
      c->stats.qr_householder++;
      householder_qr(X, n, k, ldx);
      project();
      colnorms<T>(st(), n, k, X, ldx, c->dwork);
      scale_cols<T>(st(), n, k, X, ldx, c->dwork, 1);
      ok = chol_pass(0.0);
    }
    if (ok) {
      project();
      ok = chol_pass(0.0);
    }
    if (!ok) {
      // shifted Cholesky-QR3 (Fukaya et al.): one shifted pass, then Cholesky-QR2
      c->stats.qr_fallbacks++;
      colnorms<T>(st(), n, k, X, ldx, c->dwork);
      scale_cols<T>(st(), n, k, X, ldx, c->dwork, 1);
      project();
      ok = chol_pass(11.0);
      if (ok) {
        project();
        ok = chol_pass(0.0);
      }
      if (ok) {
        project();
        ok = chol_pass(0.0);
      }
    }
    CHASE_REQUIRE(ok, CHASE_ERR_QR_BREAKDOWN, "Cholesky-QR breakdown after the shifted fallback");
  }

  // ------------------------------------------------------------ Rayleigh-Ritz eigensolve
  // Z (k x k, orthonormal columns) <- Z L^{-H} with G_z = Z^H Z = L L^H.  Returns false if not SPD.
  bool orthonormalize_small(T* Z, int k, T* Gm, T* tmp) {
    Epi e;
    e.C = Gm;
    e.ldc = k;
    gemm(OP_C, Z, k, OP_N, Z, k, k, k, k, e, CHASE_FP64);
    hermitianize<T>(st(), k, Gm, k);
    CHASE_CUDA(cudaMemsetAsync(c->info, 0, sizeof(int), st()));
    potrf_lower<T>(st(), k, Gm, k, c->info, W(), c->work_elems);
    int info = 0;
    CHASE_CUDA(cudaMemcpyAsync(&info, c->info, sizeof(int), cudaMemcpyDeviceToHost, st()));
    CHASE_CUDA(cudaStreamSynchronize(st()));
    if (info != 0) return false;
    if (use_split(CHASE_FP64, k, k, k)) {
      zero_upper<T>(st(), k, Gm, k);
      trtri_diag<T>(st(), k, Gm, k);
      trtri_combine(Gm, k, k, tmp, CHASE_FP64);
      Epi q;
      q.C = Z;
      q.ldc = k;
      gemm(OP_N, Z, k, OP_C, Gm, k, k, k, k, q, CHASE_FP64);
    } else {
      trsm_right_lh<T>(st(), k, k, Z, k, Gm, k, W(), c->work_elems);
    }
    return true;
  }

  // Eigenpairs of the Hermitian G = Gb() (k x k): FP32 parallel Jacobi, two first-order refinement
  // steps in FP64-class products, exact FP64 Jacobi on clusters closer than omega.  Ascending
  // eigenvalues to w (device), eigenvectors to Zb().  scratch: 3 k*k scalars.  Returns false when a
  // step cannot be completed (the caller then uses the FP64 Jacobi solver).
  // verbose-mode probe: report non-finite entries of a device block
  void dbg_finite(const void* X, int64_t rows, int cols, int64_t ld, size_t esz, const char* what) {
    if (!verbose()) return;
    CHASE_CUDA(cudaMemsetAsync(c->status_dev, 0, sizeof(int), st()));
    int64_t r = rows * (int64_t)(esz / sizeof(double));
    dim3 grid(std::min<unsigned>(ceil_div(r, 256), 64), cols);
    nan_check_kernel<<<grid, 256, 0, st()>>>(r, cols, (const double*)X, ld * (int64_t)(esz / sizeof(double)),
                                             c->status_dev);
    CHASE_CHECK_LAUNCH();
    int flag = 0;
    CHASE_CUDA(cudaMemcpyAsync(&flag, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost, st()));
    CHASE_CUDA(cudaStreamSynchronize(st()));
    if (flag) fprintf(stderr, "[chase] non-finite values in %s (%lld x %d)\n", what, (long long)rows, cols);
  }

  bool eigh_mixed(int k, double* w, T* scratch) {
    using F = typename Lowp<T>::type;
    T* G = Gb();
    T* Z = Zb();
    T *Wk = scratch, *Gp = scratch + (size_t)k * k, *X = scratch + 2 * (size_t)k * k;
    F* Gf = (F*)W();
    F* Zf = Gf + (size_t)k * k;
    F* jw = Zf + (size_t)k * k;
    const int64_t jw_elems = (c->work_elems * (int64_t)sizeof(T)) / (int64_t)sizeof(F) - 2 * (int64_t)k * k;
    if (jw_elems < (int64_t)k * k + 3 * (int64_t)k + 8) return false;
    dbg_finite(G, k, k, k, sizeof(T), "G before the FP32 pass");
    convert_mat<T, F>(st(), k, G, k, Gf, k);
    try {
      // block Jacobi for quotients of a few blocks and more (its rounds scale with k / 32, not k); the scalar
      // cooperative sweep below that
      if (k >= 128 && jw_elems >= (int64_t)k * k + heev_block_workspace(k))
        c->stats.rr_sweeps += heev_block_jacobi<F>(st(), k, Gf, k, w, Zf, k, jw, jw_elems, c->dwork, c->iwork, 3e-6, 40);
      else
        c->stats.rr_sweeps += heev_jacobi<F>(st(), k, Gf, k, w, Zf, k, jw, jw_elems, c->dwork, c->iwork, 3e-6, 40,
                                             false, true);
    } catch (const Error& e) {
      // non-finite FP32 values: G itself is untouched and the FP64 solver takes over; a grid barrier
      // that hit its wait limit is reported as CHASE_ERR_TIMEOUT
      if (e.status != CHASE_ERR_NAN) throw;
      return false;
    }
    convert_mat<F, T>(st(), k, Zf, k, Z, k);
    dbg_finite(Z, k, k, k, sizeof(T), "Z after the FP32 pass");
    double ends[2];
    CHASE_CUDA(cudaMemcpyAsync(&ends[0], w, sizeof(double), cudaMemcpyDeviceToHost, st()));
    CHASE_CUDA(cudaMemcpyAsync(&ends[1], w + (k - 1), sizeof(double), cudaMemcpyDeviceToHost, st()));
    CHASE_CUDA(cudaStreamSynchronize(st()));
    const double scale = std::max(std::fabs(ends[0]), std::fabs(ends[1]));
    if (!(scale > 0.0) || !std::isfinite(scale)) return false;
    const double omega = 1e-5 * scale;
    // three first-order corrections: the FP32 pass stops at its rounding floor (up to about 1e-4 relative
    // off-diagonal norm for large k), which quadratic convergence takes to FP64 level in three steps
    for (int it = 0; it < 4; ++it) {
      if (!orthonormalize_small(Z, k, Gp, X)) return false;
      Epi e1;
      e1.C = Wk;
      e1.ldc = k;
      gemm(OP_N, G, k, OP_N, Z, k, k, k, k, e1, CHASE_FP64);  // G Z
      Epi e2;
      e2.C = Gp;
      e2.ldc = k;
      gemm(OP_C, Z, k, OP_N, Wk, k, k, k, k, e2, CHASE_FP64);  // G' = Z^H G Z
      hermitianize<T>(st(), k, Gp, k);
      dbg_finite(Gp, k, k, k, sizeof(T), "G' in the refinement");
      if (it == 3) break;
      eig_correction<T>(st(), k, Gp, k, X, k, omega);
      Epi e3;
      e3.C = Wk;
      e3.ldc = k;
      e3.Y = Z;
      e3.ldy = k;
      e3.gamma = 1.0;
      gemm(OP_N, Z, k, OP_N, X, k, k, k, k, e3, CHASE_FP64);  // Z (I + X)
      copy_cols<T>(st(), k, k, Wk, k, Z, k);
    }
    // eigenvalues: diagonal of G', clusters solved exactly
    diag_real<T>(st(), k, Gp, k, w);
    std::vector<double> d(k);
    CHASE_CUDA(cudaMemcpyAsync(d.data(), w, k * sizeof(double), cudaMemcpyDeviceToHost, st()));
    CHASE_CUDA(cudaStreamSynchronize(st()));
    std::vector<int> cl;
    for (int i = 0; i < k;) {
      int j = i + 1;
      while (j < k && std::fabs(d[j] - d[j - 1]) <= omega) ++j;
      if (j - i > 1) {
        if (j - i > 32) return false;
        cl.push_back(i);
        cl.push_back(j - i);
      }
      i = j;
    }
    const int ncl = (int)cl.size() / 2;
    c->stats.rr_clusters += ncl;
    if (ncl > 0) {
      CHASE_CUDA(cudaMemcpyAsync(c->iwork, cl.data(), cl.size() * sizeof(int), cudaMemcpyHostToDevice, st()));
      CHASE_CUDA(cudaMemsetAsync(c->status_dev, 0, sizeof(int), st()));
      cluster_eig<T>(st(), k, ncl, c->iwork, Gp, k, Z, k, w, nullptr, c->status_dev);
    }
    sort_pairs<T>(st(), k, w, Z, k, Wk, c->dwork + 8, c->iwork + k);
    return true;
  }

  // ------------------------------------------------------------ Algorithm 1, lines 6-7
  // Q (n x k, ld n) orthonormal.  Out: Q <- Ritz vectors, ritz[k] ascending (device), res[k] (device).
  // Uses T2 (A Q) and Tv (n x k scratch, ld n).
  void rayleigh_ritz(const T* A, int64_t n, int64_t lda, T* Q, T* Wb, T* Tv, int k, double* ritz, double* res, int mode) {
    if (k <= 0) return;
    Epi e;
    e.C = Wb;
    e.ldc = n;
    int rmode = (mode == CHASE_FP64_NATIVE) ? CHASE_FP64_NATIVE : CHASE_FP64;
    hemm(A, n, lda, Q, n, k, e, rmode);                       // W = A Q
    Epi g;
    g.C = Gb();
    g.ldc = k;
    gemm(OP_C, Q, n, OP_N, Wb, n, k, k, n, g, rmode);  // G = Q^H W
    hermitianize<T>(st(), k, Gb(), k);
    dbg_finite(Gb(), k, k, k, sizeof(T), "the Rayleigh quotient");
    dbg_finite(Wb, n, k, n, sizeof(T), "A Q");
    // FP32 Jacobi + FP64-class refinement for large quotients (scratch: the Ritz-vector buffer, unused
    // until the back-transform); the FP64 Jacobi otherwise and as the fallback
    bool done = false;
    if (rmode != CHASE_FP64_NATIVE && k >= 64 && n >= 3 * (int64_t)k) {
      done = eigh_mixed(k, ritz, Tv);  // leaves G intact, so the fallback below can still use it
      if (!done) {
        c->stats.rr_fallbacks++;
        if (verbose()) fprintf(stderr, "[chase] mixed eigensolve fell back to FP64 Jacobi (k=%d)\n", k);
      }
    }
    if (!done) {
      T* jw = (T*)c->work;  // Jacobi workspace (k*k + 3k + 8 scalars)
      c->stats.rr_sweeps += heev_jacobi<T>(st(), k, Gb(), k, ritz, Zb(), k, jw, c->work_elems, c->dwork, c->iwork, 1e-14, 60);
    }
    Epi v;
    v.C = Tv;
    v.ldc = n;
    gemm(OP_N, Q, n, OP_N, Zb(), k, n, k, k, v, rmode);  // Vhat = Q Z
    Epi r;
    r.C = Q;
    r.ldc = n;
    r.Y = Tv;
    r.ldy = n;
    r.gamma = -1.0;
    r.ycol = ritz;
    gemm(OP_N, Wb, n, OP_N, Zb(), k, n, k, k, r, rmode);  // R = W Z - Vhat diag(ritz)
    colnorms<T>(st(), n, k, Q, n, res);
    copy_cols<T>(st(), n, k, Tv, n, Q, n);
  }

  // ------------------------------------------------------------ adjoint (real symmetric)
  // Abar = V_S (diag(gl) + F o (V_S^T Vbar)) V_nev^T + X V_nev^T, symmetrised (see adjoint.cu).
  void backward(const T* A, int64_t lda, const double* gl, const T* gV, int64_t ldg, T* gA, int64_t ldga, double tol,
                int maxit) {
    const int64_t n = c->n;
    const int nev = c->nev, l = c->l_final;
    CHASE_REQUIRE(l >= nev && nev >= 1, CHASE_ERR_STATE, "no converged pairs to differentiate");
    CHASE_REQUIRE(gA && ldga >= n && lda >= n && (gV == nullptr || ldg >= n), CHASE_ERR_ARG, "bad backward arguments");
    CHASE_REQUIRE(tol > 0.0 && maxit >= 1, CHASE_ERR_ARG, "bad MINRES tolerance or iteration cap");
    const size_t need = 9 * (size_t)n * nev * sizeof(T) + minres_state_bytes(nev) + 256;
    if (c->bwd_bytes < need) {
      if (c->bwd) CHASE_CUDA(cudaFree(c->bwd));
      c->bwd = nullptr;
      c->bwd_bytes = 0;
      CHASE_CUDA(cudaMalloc(&c->bwd, need));
      c->bwd_bytes = need;
    }
    T* base = (T*)c->bwd;
    const int64_t blk = n * nev;
    T *Tb = base, *Bb = base + blk, *Vv = base + 2 * blk, *Yb = base + 3 * blk, *R1 = base + 4 * blk,
      *R2 = base + 5 * blk, *Wa = base + 6 * blk, *Wb = base + 7 * blk, *X = base + 8 * blk;
    void* state = (void*)(base + 9 * blk);
    const T* Vs = T1();              // locked eigenvectors, ascending (n x l, ld n)
    const double* lam = c->lam_sorted;
    T* M = Gb();                     // V_S^T Vbar (l x nev)
    T* inner = Zb();                 // l x nev
    oz::invalidate(c->ozw);
    if (gV) {
      Epi e;
      e.C = M;
      e.ldc = l;
      gemm(OP_C, Vs, n, OP_N, gV, ldg, l, nev, n, e, CHASE_FP64);
    }
    adj_inner(st(), l, nev, lam, gV ? (const double*)M : nullptr, l, gl, (double*)inner, l);
    Epi et;
    et.C = Tb;
    et.ldc = n;
    gemm(OP_N, Vs, n, OP_N, inner, l, n, nev, l, et, CHASE_FP64);  // T = V_S inner
    if (gV) {
      // right-hand sides -P vbar = V_S M - Vbar
      Epi eb;
      eb.C = Bb;
      eb.ldc = n;
      eb.Y = gV;
      eb.ldy = ldg;
      eb.gamma = -1.0;
      gemm(OP_N, Vs, n, OP_N, M, l, n, nev, l, eb, CHASE_FP64);
      minres_init(st(), n, nev, (const double*)Bb, n, (double*)R1, (double*)R2, (double*)Vv, (double*)X,
                  (double*)Wa, (double*)Wb, state, tol);
      T* Mp = Gb();
      T *r1 = R1, *r2 = R2, *wc = Wa, *wn = Wb;  // wc: w_{t-1}, wn: w_{t-2}
      int it = 0;
      for (; it < maxit; ++it) {
        Epi ea;
        ea.C = Yb;
        ea.ldc = n;
        ea.Y = Vv;
        ea.ldy = n;
        ea.gamma = -1.0;
        ea.ycol = lam;
        hemm(A, n, lda, Vv, n, nev, ea, CHASE_FP64);  // Y = A v - lambda_j v
        Epi ep;
        ep.C = Mp;
        ep.ldc = l;
        gemm(OP_C, Vs, n, OP_N, Yb, n, l, nev, n, ep, CHASE_FP64, true);
        Epi eu;
        eu.C = Yb;
        eu.ldc = n;
        eu.alpha = -1.0;
        eu.Z = Yb;
        eu.ldz = n;
        eu.beta = 1.0;
        gemm(OP_N, Vs, n, OP_N, Mp, l, n, nev, l, eu, CHASE_FP64, true);  // Y -= V_S (V_S^T Y)
        minres_update(st(), n, nev, (const double*)Yb, (double*)r1, (const double*)r2, (double*)Vv, (double*)wn,
                      (const double*)wc, (double*)X, state, tol);
        std::swap(r1, r2);
        std::swap(wc, wn);
        if (it % 10 == 9) {
          minres_count_done(st(), nev, state, c->status_dev);
          int done = 0;
          CHASE_CUDA(cudaMemcpyAsync(&done, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost, st()));
          CHASE_CUDA(cudaStreamSynchronize(st()));
          if (done == nev) break;
        }
      }
      c->stats.minres_iterations = it + 1;
      add_inplace(st(), blk, (double*)Tb, (const double*)X);
    }
    // Abar = (T + X) V_nev^T, then (Abar + Abar^T)/2
    Epi ga;
    ga.C = gA;
    ga.ldc = ldga;
    gemm_f64<T>(st(), OP_N, OP_C, n, n, nev, Tb, n, Vs, n, ga, W(), c->work_elems);
    hermitianize<T>(st(), (int)n, gA, ldga);
    CHASE_CUDA(cudaStreamSynchronize(st()));
    CHASE_REQUIRE(oz::read_flags(st(), c->ozw) == 0, CHASE_ERR_TIMEOUT, "a tensor-core product hit its wait limit");
  }

  // ------------------------------------------------------------ Algorithm 1
  // Host state of one solve between the stages of an outer iteration (a batched solve keeps one per
  // problem and runs the stages of all problems in lockstep).
  struct Run {
    const T* A = nullptr;
    int64_t n = 0, lda = 0;
    int nev = 0, nex = 0, ne = 0, mode = 0, deg = 0;
    double thresh = 0.0, norm_est = 0.0, b_sup = 0.0, mu_1 = 0.0, mu_ne = 0.0;
    std::vector<int> m;  // degrees of the active columns (non-decreasing)
    int l = 0, it = 0;
    bool lowp = false;
    double lowp_floor = 0.0, prev_minres = 1e308;
    std::vector<int> degbuf;
    std::vector<double> resbuf, reslock;
    int k() const { return ne - l; }
    bool done(int maxiter) const { return l >= nev || it >= maxiter; }
    int fmode() const { return (mode == CHASE_FP64_NATIVE) ? CHASE_FP64_NATIVE : (lowp ? mode : CHASE_FP64); }
  };

  // Validation, NaN checks, Lanczos bounds (line 2), start block and initial degrees (line 1).
  void begin(Run& R, const T* A, int64_t n, int64_t lda, int nev, int nex, double tol, int deg, int mode, const T* V0,
             const T* L0) {
    const int ne = nev + nex;
    CHASE_REQUIRE(n >= 1 && n <= c->n_max, CHASE_ERR_ARG, "n out of range for this context");
    CHASE_REQUIRE(nev >= 1 && nex >= 0 && ne <= c->ne_max && ne <= n, CHASE_ERR_ARG, "nev/nex out of range");
    CHASE_REQUIRE(lda >= n, CHASE_ERR_ARG, "lda < n");
    CHASE_REQUIRE(tol > 0.0 && deg >= 1 && deg <= c->opts.maxdeg, CHASE_ERR_ARG, "tol or deg out of range");
    CHASE_REQUIRE(A && V0 && L0, CHASE_ERR_ARG, "null A, V0 or L0");
    CHASE_REQUIRE(mode >= CHASE_FP64 && mode <= CHASE_BF16x6, CHASE_ERR_ARG, "unknown mode");
    CHASE_REQUIRE(mode == CHASE_FP64_NATIVE || oz::available(), CHASE_ERR_UNSUPPORTED,
                  "the FP64 and split-BF16 modes need the tensor-core kernels (sm_103); use CHASE_FP64_NATIVE");
    c->have_result = false;
    c->stats = chase_stats_t{};
    oz::invalidate(c->ozw);  // A may hold new values at the same address
    chase_stats_t& S = c->stats;
    check_nan(A, n, (int)n, lda, "A");
    check_nan(V0, n, ne, n, "V0");
    const int runs = c->opts.lanczos_runs, steps = std::min<int>(c->opts.lanczos_steps, (int)n);
    // Lanczos (line 2)
    {
      Timer t(c, 1, &S.ms_lanczos);
      // large problems: the Lanczos matvecs use the FP64-class split tensor-core product (the digit
      // planes of A are then reused by the filter); small ones and the native mode use DFMA
      MatvecFn<T> mv = [&](const T* X, int64_t ldx, T* Wout) {
        Epi e;
        e.C = Wout;
        e.ldc = n;
        hemm(A, n, lda, X, ldx, runs, e, CHASE_FP64);
      };
      const bool lz_split = runs <= c->ne_max && use_split(mode == CHASE_FP64_NATIVE ? CHASE_FP64_NATIVE : CHASE_FP64,
                                                           n, runs, n);
      lanczos<T>(st(), A, n, lda, ne, L0, runs, steps, c->dwork, W(), c->work_elems, c->dwork + 8,
                 lz_split ? &mv : nullptr);
      init_bounds_kernel<<<1, 1, 0, st()>>>(c->dwork, c->bounds);
      CHASE_CHECK_LAUNCH();
      t.stop();
    }
    double hb[6];
    CHASE_CUDA(cudaMemcpyAsync(hb, c->dwork, 4 * sizeof(double), cudaMemcpyDeviceToHost, st()));
    CHASE_CUDA(cudaStreamSynchronize(st()));
    R = Run{};
    R.A = A;
    R.n = n;
    R.lda = lda;
    R.nev = nev;
    R.nex = nex;
    R.ne = ne;
    R.mode = mode;
    R.deg = deg;
    R.b_sup = hb[0];
    R.mu_1 = hb[1];
    R.mu_ne = hb[2];
    const double theta_max = hb[3];
    S.b_sup = R.b_sup;
    S.mu_1 = R.mu_1;
    S.mu_ne = R.mu_ne;
    R.norm_est = std::max(std::fabs(R.mu_1), std::fabs(theta_max));
    S.norm_est = R.norm_est;
    R.thresh = tol * R.norm_est;
    CHASE_REQUIRE(std::isfinite(R.b_sup) && std::isfinite(R.mu_1) && std::isfinite(R.mu_ne), CHASE_ERR_NAN,
                  "non-finite Lanczos bounds");
    copy_cols<T>(st(), n, ne, V0, n, V(), n);
    R.m.assign(ne, deg);
    fill_int_kernel<<<ceil_div(ne, 256), 256, 0, st()>>>(ne, c->deg, deg);
    CHASE_CHECK_LAUNCH();
    // mixed modes: bulk filter in split-BF16 while it still makes progress; switch to FP64 for the rest
    // once the smallest unconverged relative residual reaches the bulk precision floor or stops falling
    // by at least a factor 4 per iteration
    R.lowp = (mode == CHASE_BF16x3 || mode == CHASE_BF16x6);
    R.lowp_floor = (mode == CHASE_BF16x3) ? 1e-3 : 3e-5;
    R.degbuf.assign(ne, 0);
    R.resbuf.assign(ne, 0.0);
    R.reslock.assign(ne, 0.0);
  }

  // Line 4 of one outer iteration (the filter of the active block), timed.
  void filter_stage(Run& R) {
    chase_stats_t& S = c->stats;
    const int k = R.k();
    T* Vact = V() + (int64_t)R.l * R.n;
    T* T1act = T1() + (int64_t)R.l * R.n;
    Timer t(c, 1, &S.ms_filter);
    if (oz::available()) oz::timing_begin(c->ozw);
    int64_t mv = filter(R.A, R.n, R.lda, Vact, T1act, k, R.m.data(), c->deg, R.b_sup, R.mu_1, R.mu_ne, R.fmode(), true);
    if (oz::available()) {
      int nl = 0;
      double ms = oz::timing_collect(c->ozw, &nl);
      if (R.lowp) {
        S.ms_filter_kernel_lowp += ms;
      } else {
        S.ms_filter_kernel += ms;
        S.filter_kernel_launches += nl;
      }
    }
    count_matvecs(R, mv);
    t.stop();
  }

  void count_matvecs(Run& R, int64_t mv) {
    chase_stats_t& S = c->stats;
    S.matvecs += mv;
    if (R.lowp) {
      S.matvecs_lowp += mv;
      S.lowp_iterations++;
    }
  }

  // Lines 5-14 of one outer iteration: QR, Rayleigh-Ritz, residuals, locking, bounds, degrees, sort.
  void after_filter(Run& R) {
    chase_stats_t& S = c->stats;
    const int64_t n = R.n;
    const int k = R.k();
    T* Vact = V() + (int64_t)R.l * n;
    T* T1act = T1() + (int64_t)R.l * n;
    T* T2act = T2() + (int64_t)R.l * n;
    const int fmode = R.fmode();
    {
      Timer t(c, 1, &S.ms_qr);
      qr(V(), n, R.l, Vact, n, n, k, R.mode == CHASE_FP64_NATIVE ? CHASE_FP64_NATIVE : CHASE_FP64);
      t.stop();
    }
    {
      Timer t(c, 1, &S.ms_rr);
      rayleigh_ritz(R.A, n, R.lda, Vact, T2act, T1act, k, c->ritz, c->res, fmode);
      t.stop();
    }
    {
      Timer t(c, 1, &S.ms_resid);
      struct {
        int lock;
        int pad;
        double bnd[6];
      } hstat;
      bookkeeping(st(), k, c->ritz, c->res, R.thresh, R.b_sup, c->bounds, c->opts.maxdeg, c->opts.extra_deg,
                  c->status_dev, c->deg, c->perm, c->ritz2, c->res2, c->iwork);
      CHASE_CUDA(cudaMemcpyAsync(&hstat.lock, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost, st()));
      CHASE_CUDA(cudaMemcpyAsync(hstat.bnd, c->bounds, 6 * sizeof(double), cudaMemcpyDeviceToHost, st()));
      CHASE_CUDA(cudaMemcpyAsync(R.degbuf.data(), c->deg, k * sizeof(int), cudaMemcpyDeviceToHost, st()));
      CHASE_CUDA(cudaMemcpyAsync(R.resbuf.data(), c->res2, k * sizeof(double), cudaMemcpyDeviceToHost, st()));
      CHASE_CUDA(cudaMemcpyAsync(R.reslock.data(), c->res, k * sizeof(double), cudaMemcpyDeviceToHost, st()));
      CHASE_CUDA(cudaStreamSynchronize(st()));
      CHASE_REQUIRE(oz::read_flags(st(), c->ozw) == 0, CHASE_ERR_TIMEOUT, "a tensor-core product hit its wait limit");
      const int p = hstat.lock;
      for (int a = 0; a < p; ++a) S.max_resid = std::max(S.max_resid, R.reslock[a] / R.norm_est);
      // lock: Ritz values of the converged prefix, then reorder the remaining active columns
      if (p > 0)
        CHASE_CUDA(cudaMemcpyAsync(c->lam_locked + R.l, c->ritz, p * sizeof(double), cudaMemcpyDeviceToDevice, st()));
      const int kr = k - p;
      if (kr > 0) {
        permute_cols<T>(st(), n, kr, Vact, n, T1act, n, c->perm);
        copy_cols<T>(st(), n, kr, T1act, n, Vact + (int64_t)p * n, n);
      }
      // the device degree array must follow the new active block (it starts at l + p)
      R.l += p;
      R.mu_1 = hstat.bnd[1];
      R.mu_ne = hstat.bnd[2];
      R.m.assign(R.degbuf.begin(), R.degbuf.begin() + kr);
      if (verbose()) {
        double mr = 0.0, mn = 1e308;
        for (int a = 0; a < kr; ++a) {
          mr = std::max(mr, R.resbuf[a] / R.norm_est);
          mn = std::min(mn, R.resbuf[a] / R.norm_est);
        }
        fprintf(stderr, "[chase] it=%d mode=%d k=%d locked=%d(+%d) mu1=%.6g mune=%.6g res[min,max]=%.3e,%.3e deg[0,last]=%d,%d fallbacks=%d ms[filter,qr,rr,resid]=%.1f,%.1f,%.1f,%.1f\n",
                R.it, fmode, k, R.l, p, R.mu_1, R.mu_ne, mn, mr, kr ? R.m[0] : 0, kr ? R.m[kr - 1] : 0, S.qr_fallbacks,
                S.ms_filter, S.ms_qr, S.ms_rr, S.ms_resid);
      }
      if (R.lowp) {
        double minres = 1e308;
        for (int a = 0; a < kr; ++a) minres = std::min(minres, R.resbuf[a] / R.norm_est);
        if (kr == 0 || minres <= R.lowp_floor || minres > 0.25 * R.prev_minres ||
            R.it >= c->opts.maxiter - c->opts.nfinal)
          R.lowp = false;
        R.prev_minres = minres;
      }
      t.stop();
    }
  }

  // Result of the solve: NOCONV check, the nev smallest locked pairs ascending, warm-start block.
  void finish(Run& R) {
    chase_stats_t& S = c->stats;
    const int64_t n = R.n;
    S.iterations = R.it;
    S.locked = R.l;
    CHASE_REQUIRE(R.l >= R.nev, CHASE_ERR_NOCONV, "maxiter reached before nev pairs converged");
    final_sort_kernel<<<ceil_div(R.l, 128), 128, 0, st()>>>(R.l, R.nev, c->lam_locked, c->eigvals, c->lam_sorted, c->perm);
    CHASE_CHECK_LAUNCH();
    // T1 = [locked pairs ascending | remaining active block]: the first nev columns are the
    // eigenvectors, the whole block is a warm start for a nearby problem
    permute_cols<T>(st(), n, R.l, V(), n, T1(), n, c->perm);
    if (R.ne > R.l) copy_cols<T>(st(), n, R.ne - R.l, V() + (int64_t)R.l * n, n, T1() + (int64_t)R.l * n, n);
    c->n = n;
    c->nev = R.nev;
    c->nex = R.nex;
    c->l_final = R.l;
    c->have_result = true;
  }

  void solve(const T* A, int64_t n, int64_t lda, int nev, int nex, double tol, int deg, int mode, const T* V0,
             const T* L0) {
    Run R;
    c->stats = chase_stats_t{};
    Timer ttot(c, 0, &c->stats.ms_total);
    begin(R, A, n, lda, nev, nex, tol, deg, mode, V0, L0);
    while (!R.done(c->opts.maxiter)) {
      ++R.it;
      filter_stage(R);
      after_filter(R);
    }
    // on NOCONV the timers still record: finish() throws after the iteration count is stored
    c->stats.ms_total = 0.0;
    ttot.stop();
    finish(R);
  }
};

// =====================================================================================
static chase_status fail(chase_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return (chase_status)code;
}

#define API_BEGIN(ctx) \
  if (!(ctx)) return CHASE_ERR_ARG; \
  try {                           \
    CHASE_CUDA(cudaSetDevice((ctx)->device));
#define API_END(ctx)                                                             \
  }                                                                              \
  catch (const chase::Error& e) {                                                \
    return fail((ctx), e.status, e.msg);                                         \
  }                                                                              \
  catch (const std::bad_alloc&) {                                                \
    return fail((ctx), CHASE_ERR_OOM, "host allocation failed");                 \
  }                                                                              \
  catch (const std::exception& e) {                                              \
    return fail((ctx), CHASE_ERR_CUDA, e.what());                                \
  }                                                                              \
  (ctx)->err.clear();                                                            \
  return CHASE_OK;

template <typename T>
static void filter_api(chase_ctx* c, const T* A, int64_t n, int64_t lda, T* V, int64_t ldv, int k, const int* deg,
                       double b_sup, double mu_1, double mu_ne, int mode) {
  Solver<T> s(c);
  oz::invalidate(c->ozw);
  // work on the context's V/T1 buffers (ld n), copy in/out
  copy_cols<T>(c->stream, n, k, V, ldv, s.V(), n);
  std::vector<int> d(deg, deg + k);
  CHASE_CUDA(cudaMemcpyAsync(c->deg, d.data(), k * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  s.filter(A, n, lda, s.V(), s.T1(), k, d.data(), c->deg, b_sup, mu_1, mu_ne, mode);
  copy_cols<T>(c->stream, n, k, s.V(), n, V, ldv);
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
}

template <typename T>
static void rr_api(chase_ctx* c, const T* A, int64_t n, int64_t lda, T* Q, int64_t ldq, int k, double* ritz_host,
                   double* res_host) {
  Solver<T> s(c);
  oz::invalidate(c->ozw);
  copy_cols<T>(c->stream, n, k, Q, ldq, s.V(), n);
  s.rayleigh_ritz(A, n, lda, s.V(), s.T2(), s.T1(), k, c->ritz, c->res, CHASE_FP64);
  copy_cols<T>(c->stream, n, k, s.V(), n, Q, ldq);
  if (ritz_host) CHASE_CUDA(cudaMemcpyAsync(ritz_host, c->ritz, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (res_host) CHASE_CUDA(cudaMemcpyAsync(res_host, c->res, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
}

template <typename T>
static void heevj_api(chase_ctx* c, const T* G, int64_t ldg, int k, double* w_host, T* Z, int64_t ldz) {
  T* Gw = (T*)c->G;
  copy_cols<T>(c->stream, k, k, G, ldg, Gw, k);
  heev_jacobi<T>(c->stream, k, Gw, k, c->ritz, Z, ldz, (T*)c->work, c->work_elems, c->dwork, c->iwork, 1e-14, 60);
  CHASE_CUDA(cudaMemcpyAsync(w_host, c->ritz, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
}

extern "C" {

void chase_default_opts(chase_opts* o) {
  if (!o) return;
  o->maxdeg = 36;
  o->lanczos_steps = 25;
  o->lanczos_runs = 4;
  o->maxiter = 30;
  o->extra_deg = 2;
  o->nfinal = 1;
  o->oz_slices = 7;
  o->native_below_mflop = 2000;
  o->batch_workers = 1;
  o->batch_grouped = 1;
}

static int64_t lanczos_elems(int64_t n, int runs, int steps) {
  int64_t nchunk = (n + 255) / 256;
  int64_t part = std::max<int64_t>(nchunk * runs * n, (int64_t)runs * 64 * 64);
  return (int64_t)runs * steps * n + runs * n + part + 2 * runs * 64;
}

static int64_t work_elems_for(int64_t n, int ne, const chase_opts& o) {
  // FP64 Jacobi: ne^2 + 3 ne + 8 scalars; FP32 first pass: 3 ne^2 + 3 ne + 8 half-size scalars
  int64_t jac = 2 * (int64_t)ne * ne + 3 * (int64_t)ne + 16;
  int64_t lz = lanczos_elems(n, o.lanczos_runs, std::min<int>(o.lanczos_steps, (int)n));
  int64_t split = 2 * 1024 * 1024;
  return std::max(std::max(jac, lz), split);
}

int64_t chase_workspace_bytes(int64_t n_max, int ne_max, chase_dtype dtype, const chase_opts* opts) {
  chase_opts o;
  chase_default_opts(&o);
  if (opts) o = *opts;
  int64_t esz = dtype == CHASE_C128 ? 16 : 8;
  int64_t b = 3 * n_max * ne_max * esz + 2 * (int64_t)ne_max * ne_max * esz + work_elems_for(n_max, ne_max, o) * esz;
  b += (3 * 32 * (int64_t)ne_max + ne_max + 1024) * esz;  // Householder QR scratch
  b += oz::workspace_bytes(n_max, ne_max, dtype == CHASE_C128, o.oz_slices);
  return b;
}

chase_status chase_create(chase_ctx** out, int64_t n_max, int ne_max, chase_dtype dtype, const chase_opts* opts,
                          void* stream) {
  if (!out) return CHASE_ERR_ARG;
  *out = nullptr;
  if (n_max < 1 || ne_max < 1 || ne_max > n_max || (dtype != CHASE_R64 && dtype != CHASE_C128)) return CHASE_ERR_ARG;
  chase_ctx* c = new (std::nothrow) chase_ctx();
  if (!c) return CHASE_ERR_OOM;
  chase_default_opts(&c->opts);
  if (opts) c->opts = *opts;
  if (c->opts.maxdeg < 1 || c->opts.lanczos_runs < 1 || c->opts.lanczos_runs > 8 || c->opts.lanczos_steps < 1 ||
      c->opts.lanczos_steps > 64 || c->opts.maxiter < 1 || c->opts.oz_slices < 6 || c->opts.oz_slices > 7 ||
      c->opts.native_below_mflop < 0 || c->opts.batch_workers < 1 || c->opts.batch_workers > 32 ||
      c->opts.batch_grouped < 0 || c->opts.batch_grouped > 1) {
    delete c;
    return CHASE_ERR_ARG;
  }
  c->dtype = dtype;
  c->n_max = n_max;
  c->ne_max = ne_max;
  c->esz = dtype == CHASE_C128 ? 16 : 8;
  try {
    CHASE_CUDA(cudaGetDevice(&c->device));
    // NULL is the legacy default stream (the one a framework's default stream maps to), so work
    // enqueued by the caller on it before a call is ordered before the call's kernels
    c->stream = (cudaStream_t)stream;
    for (auto& e : c->ev) CHASE_CUDA(cudaEventCreate(&e));
    size_t freeb = 0, totb = 0;
    CHASE_CUDA(cudaMemGetInfo(&freeb, &totb));
    const int nctx = c->opts.batch_grouped ? 1 : c->opts.batch_workers;
    int64_t need = chase_workspace_bytes(n_max, ne_max, dtype, &c->opts) * (int64_t)nctx;
    if ((size_t)need + (64ull << 20) > freeb) {
      c->err = "workspace of " + std::to_string(need) + " bytes does not fit in free device memory";
      chase_destroy(c);
      return CHASE_ERR_OOM;
    }
    size_t blk = (size_t)n_max * ne_max * c->esz;
    CHASE_CUDA(cudaMalloc(&c->V, blk));
    CHASE_CUDA(cudaMalloc(&c->T1, blk));
    CHASE_CUDA(cudaMalloc(&c->T2, blk));
    CHASE_CUDA(cudaMalloc(&c->G, (size_t)ne_max * ne_max * c->esz));
    CHASE_CUDA(cudaMalloc(&c->Z, (size_t)ne_max * ne_max * c->esz));
    c->work_elems = work_elems_for(n_max, ne_max, c->opts);
    CHASE_CUDA(cudaMalloc(&c->work, (size_t)c->work_elems * c->esz));
    c->dwork_elems = 8 + 5 * 8 * 64 + 4 * (int64_t)ne_max + 16;
    CHASE_CUDA(cudaMalloc(&c->dwork, c->dwork_elems * sizeof(double)));
    CHASE_CUDA(cudaMalloc(&c->iwork, (size_t)(2 * ne_max + 16) * sizeof(int)));
    CHASE_CUDA(cudaMalloc(&c->ritz, ne_max * sizeof(double)));
    CHASE_CUDA(cudaMalloc(&c->res, ne_max * sizeof(double)));
    CHASE_CUDA(cudaMalloc(&c->ritz2, ne_max * sizeof(double)));
    CHASE_CUDA(cudaMalloc(&c->res2, ne_max * sizeof(double)));
    CHASE_CUDA(cudaMalloc(&c->lam_locked, ne_max * sizeof(double)));
    CHASE_CUDA(cudaMalloc(&c->eigvals, ne_max * sizeof(double)));
    CHASE_CUDA(cudaMalloc(&c->lam_sorted, ne_max * sizeof(double)));
    CHASE_CUDA(cudaMalloc(&c->bounds, 8 * sizeof(double)));
    CHASE_CUDA(cudaMalloc(&c->deg, ne_max * sizeof(int)));
    CHASE_CUDA(cudaMalloc(&c->perm, ne_max * sizeof(int)));
    CHASE_CUDA(cudaMalloc(&c->info, sizeof(int)));
    CHASE_CUDA(cudaMalloc(&c->status_dev, 4 * sizeof(int)));
    CHASE_CUDA(cudaMalloc(&c->qr_dep, (size_t)(ne_max + 1) * sizeof(int)));
    CHASE_CUDA(cudaMalloc(&c->hh, (size_t)(3 * 32 * (size_t)ne_max + ne_max + 1024) * c->esz));
    oz::create(c->ozw, n_max, ne_max, dtype == CHASE_C128, c->opts.oz_slices);
    // workers of batched solves: same sizes and options, one non-blocking stream each
    chase_opts wo = c->opts;
    wo.batch_workers = 1;
    for (int w = 1; w < nctx; ++w) {
      cudaStream_t ws = nullptr;
      CHASE_CUDA(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
      chase_ctx* wc = nullptr;
      chase_status st = chase_create(&wc, n_max, ne_max, dtype, &wo, ws);
      if (st != CHASE_OK) {
        cudaStreamDestroy(ws);
        throw chase::Error{(int)st, "creating a batch worker failed"};
      }
      wc->own_stream = true;
      c->workers.push_back(wc);
    }
  } catch (const chase::Error& e) {
    chase_destroy(c);
    return (chase_status)e.status;
  }
  *out = c;
  return CHASE_OK;
}

void chase_destroy(chase_ctx* c) {
  if (!c) return;
  for (chase_ctx* w : c->workers) chase_destroy(w);
  c->workers.clear();
  for (chase_ctx* w : c->slots) chase_destroy(w);
  c->slots.clear();
  if (c->filter_stream) {
    cudaStreamSynchronize(c->filter_stream);
    cudaStreamDestroy(c->filter_stream);
    c->filter_stream = nullptr;
  }
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  void* ptrs[] = {c->V, c->T1, c->T2, c->G, c->Z, c->work, c->dwork, c->iwork, c->ritz, c->res, c->ritz2, c->res2,
                  c->lam_locked, c->eigvals, c->lam_sorted, c->bwd, c->bounds, c->deg, c->perm, c->info,
                  c->status_dev, c->qr_dep, c->hh, c->a_stage, c->l0_stage};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  oz::destroy(c->ozw);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* chase_last_error(const chase_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t chase_kernel_launch_count(void) { return (int64_t)chase::g_kernel_launches.load(); }

void chase_set_wait_limit_ns(uint64_t ns) { chase::g_wait_limit_ns.store((unsigned long long)ns); }

// true for memory the device cannot be handed directly as a kernel argument of this library:
// pageable or pinned host allocations (copied to the device first)
static bool is_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // an unknown pointer is plain host memory
    return true;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

chase_status chase_solve(chase_ctx* c, const void* A, int64_t n, int64_t lda, int nev, int nex, double tol, int deg,
                         int mode, const void* V0, const void* L0) {
  API_BEGIN(c)
  CHASE_REQUIRE(A, CHASE_ERR_ARG, "null A");
  CHASE_REQUIRE(n >= 1 && n <= c->n_max && lda >= n, CHASE_ERR_ARG, "n or lda out of range for this context");
  CHASE_REQUIRE(nev >= 1 && nex >= 0 && nev + nex <= c->ne_max, CHASE_ERR_ARG, "nev/nex out of range");
  // start vectors the caller leaves to the library: seeded counter-based normals (see the header)
  if (!V0) {
    // the filter partner buffer is free until the first filter step (V0 is read before it)
    if (c->dtype == CHASE_C128)
      fill_normal<double2>(c->stream, (double2*)c->T1, n, nev + nex, n, CHASE_SEED_V0);
    else
      fill_normal<double>(c->stream, (double*)c->T1, n, nev + nex, n, CHASE_SEED_V0);
    V0 = c->T1;
  }
  if (!L0) {
    if (!c->l0_stage) CHASE_CUDA(cudaMalloc(&c->l0_stage, (size_t)c->n_max * 8 * c->esz));
    if (c->dtype == CHASE_C128)
      fill_normal<double2>(c->stream, (double2*)c->l0_stage, n, c->opts.lanczos_runs, n, CHASE_SEED_L0);
    else
      fill_normal<double>(c->stream, (double*)c->l0_stage, n, c->opts.lanczos_runs, n, CHASE_SEED_L0);
    L0 = c->l0_stage;
  }
  // host inputs: copied to the device on the context's stream (pinned memory: DMA at link speed)
  const size_t esz = c->esz;
  if (is_host_ptr(A)) {
    const size_t need = (size_t)n * (size_t)n * esz;
    if (c->a_stage_bytes < need) {
      if (c->a_stage) CHASE_CUDA(cudaFree(c->a_stage));
      c->a_stage = nullptr;
      c->a_stage_bytes = 0;
      size_t freeb = 0, totb = 0;
      CHASE_CUDA(cudaMemGetInfo(&freeb, &totb));
      CHASE_REQUIRE(need + (64ull << 20) <= freeb, CHASE_ERR_OOM, "no device memory for a copy of the host A");
      CHASE_CUDA(cudaMalloc(&c->a_stage, need));
      c->a_stage_bytes = need;
    }
    if (lda == n)
      CHASE_CUDA(cudaMemcpyAsync(c->a_stage, A, need, cudaMemcpyHostToDevice, c->stream));
    else
      CHASE_CUDA(cudaMemcpy2DAsync(c->a_stage, n * esz, A, lda * esz, n * esz, n, cudaMemcpyHostToDevice, c->stream));
    A = c->a_stage;
    lda = n;
  }
  if (is_host_ptr(V0)) {
    // the filter partner buffer is free until the first filter step (V0 is read before it)
    CHASE_CUDA(cudaMemcpyAsync(c->T1, V0, (size_t)n * (nev + nex) * esz, cudaMemcpyHostToDevice, c->stream));
    V0 = c->T1;
  }
  if (is_host_ptr(L0)) {
    if (!c->l0_stage) CHASE_CUDA(cudaMalloc(&c->l0_stage, (size_t)c->n_max * 8 * esz));
    CHASE_CUDA(cudaMemcpyAsync(c->l0_stage, L0, (size_t)n * c->opts.lanczos_runs * esz, cudaMemcpyHostToDevice,
                               c->stream));
    L0 = c->l0_stage;
  }
  if (c->dtype == CHASE_C128)
    Solver<double2>(c).solve((const double2*)A, n, lda, nev, nex, tol, deg, mode, (const double2*)V0, (const double2*)L0);
  else
    Solver<double>(c).solve((const double*)A, n, lda, nev, nex, tol, deg, mode, (const double*)V0, (const double*)L0);
  API_END(c)
}

chase_status chase_eigvals(chase_ctx* c, double* out, int on_device) {
  API_BEGIN(c)
  CHASE_REQUIRE(c->have_result, CHASE_ERR_STATE, "no solve result");
  CHASE_REQUIRE(out, CHASE_ERR_ARG, "null output");
  CHASE_CUDA(cudaMemcpyAsync(out, c->eigvals, c->nev * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
  API_END(c)
}

chase_status chase_eigvecs(chase_ctx* c, void* out, int64_t ldv, int on_device) {
  API_BEGIN(c)
  CHASE_REQUIRE(c->have_result, CHASE_ERR_STATE, "no solve result");
  CHASE_REQUIRE(out && ldv >= c->n, CHASE_ERR_ARG, "bad output");
  CHASE_CUDA(cudaMemcpy2DAsync(out, ldv * c->esz, c->T1, c->n * c->esz, c->n * c->esz, c->nev,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
  API_END(c)
}

chase_status chase_stats(const chase_ctx* c, chase_stats_t* out) {
  if (!c || !out) return CHASE_ERR_ARG;
  *out = c->stats;
  return CHASE_OK;
}

chase_status chase_lanczos(chase_ctx* c, const void* A, int64_t n, int64_t lda, int ne, const void* L0, int runs,
                           int steps, double* out_host) {
  API_BEGIN(c)
  CHASE_REQUIRE(A && L0 && out_host && n >= 1 && n <= c->n_max && lda >= n && ne >= 1, CHASE_ERR_ARG, "bad args");
  CHASE_REQUIRE(runs >= 1 && runs <= 8 && steps >= 1 && steps <= 64 && steps <= n, CHASE_ERR_ARG, "bad runs/steps");
  if (c->dtype == CHASE_C128)
    lanczos<double2>(c->stream, (const double2*)A, n, lda, ne, (const double2*)L0, runs, steps, c->dwork,
                     (double2*)c->work, c->work_elems, c->dwork + 8);
  else
    lanczos<double>(c->stream, (const double*)A, n, lda, ne, (const double*)L0, runs, steps, c->dwork,
                    (double*)c->work, c->work_elems, c->dwork + 8);
  CHASE_CUDA(cudaMemcpyAsync(out_host, c->dwork, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
  API_END(c)
}


chase_status chase_filter(chase_ctx* c, const void* A, int64_t n, int64_t lda, void* V, int64_t ldv, int ncols,
                          const int* deg_host, double b_sup, double mu_1, double mu_ne, int mode) {
  API_BEGIN(c)
  CHASE_REQUIRE(A && V && deg_host && n >= 1 && n <= c->n_max && lda >= n && ldv >= n && ncols >= 0 &&
                    ncols <= c->ne_max,
                CHASE_ERR_ARG, "bad args");
  CHASE_REQUIRE(mode >= CHASE_FP64 && mode <= CHASE_BF16x6, CHASE_ERR_ARG, "unknown mode");
  for (int a = 0; a < ncols; ++a) {
    CHASE_REQUIRE(deg_host[a] >= 1 && deg_host[a] <= 1000, CHASE_ERR_ARG, "degree out of range");
    CHASE_REQUIRE(a == 0 || deg_host[a] >= deg_host[a - 1], CHASE_ERR_ARG, "degrees must be non-decreasing");
  }
  if (c->dtype == CHASE_C128)
    filter_api<double2>(c, (const double2*)A, n, lda, (double2*)V, ldv, ncols, deg_host, b_sup, mu_1, mu_ne, mode);
  else
    filter_api<double>(c, (const double*)A, n, lda, (double*)V, ldv, ncols, deg_host, b_sup, mu_1, mu_ne, mode);
  API_END(c)
}

chase_status chase_qr(chase_ctx* c, void* X, int64_t n, int64_t ldx, int ncols, int nlocked) {
  API_BEGIN(c)
  CHASE_REQUIRE(X && n >= 1 && n <= c->n_max && ldx >= n && nlocked >= 0 && ncols >= nlocked && ncols <= c->ne_max &&
                    ncols <= n,
                CHASE_ERR_ARG, "bad args");
  if (c->dtype == CHASE_C128) {
    double2* x = (double2*)X;
    Solver<double2>(c).qr(x, ldx, nlocked, x + nlocked * ldx, ldx, n, ncols - nlocked, CHASE_FP64);
  } else {
    double* x = (double*)X;
    Solver<double>(c).qr(x, ldx, nlocked, x + nlocked * ldx, ldx, n, ncols - nlocked, CHASE_FP64);
  }
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
  API_END(c)
}


chase_status chase_rayleigh_ritz(chase_ctx* c, const void* A, int64_t n, int64_t lda, void* Q, int64_t ldq, int ncols,
                                 double* ritz_host, double* resid_host) {
  API_BEGIN(c)
  CHASE_REQUIRE(A && Q && n >= 1 && n <= c->n_max && lda >= n && ldq >= n && ncols >= 1 && ncols <= c->ne_max,
                CHASE_ERR_ARG, "bad args");
  if (c->dtype == CHASE_C128)
    rr_api<double2>(c, (const double2*)A, n, lda, (double2*)Q, ldq, ncols, ritz_host, resid_host);
  else
    rr_api<double>(c, (const double*)A, n, lda, (double*)Q, ldq, ncols, ritz_host, resid_host);
  API_END(c)
}


chase_status chase_heevj(chase_ctx* c, const void* G, int64_t ldg, int k, double* w_host, void* Z, int64_t ldz) {
  API_BEGIN(c)
  CHASE_REQUIRE(G && Z && w_host && k >= 1 && k <= c->ne_max && ldg >= k && ldz >= k, CHASE_ERR_ARG, "bad args");
  if (c->dtype == CHASE_C128)
    heevj_api<double2>(c, (const double2*)G, ldg, k, w_host, (double2*)Z, ldz);
  else
    heevj_api<double>(c, (const double*)G, ldg, k, w_host, (double*)Z, ldz);
  API_END(c)
}

chase_status chase_hemm(chase_ctx* c, const void* A, int64_t n, int64_t lda, const void* B, int64_t ldb, int ncols,
                        void* C, int64_t ldc, int mode) {
  API_BEGIN(c)
  CHASE_REQUIRE(A && B && C && n >= 1 && n <= c->n_max && lda >= n && ldb >= n && ldc >= n && ncols >= 1 &&
                    ncols <= c->ne_max,
                CHASE_ERR_ARG, "bad args");
  CHASE_REQUIRE(mode >= CHASE_FP64 && mode <= CHASE_BF16x6, CHASE_ERR_ARG, "unknown mode");
  Epi e;
  e.C = C;
  e.ldc = ldc;
  oz::invalidate(c->ozw);
  if (c->dtype == CHASE_C128)
    Solver<double2>(c).hemm((const double2*)A, n, lda, (const double2*)B, ldb, ncols, e, mode);
  else
    Solver<double>(c).hemm((const double*)A, n, lda, (const double*)B, ldb, ncols, e, mode);
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
  CHASE_REQUIRE(oz::read_flags(c->stream, c->ozw) == 0, CHASE_ERR_TIMEOUT, "a tensor-core product hit its wait limit");
  API_END(c)
}

chase_status chase_generate(chase_ctx* c, void* A, int64_t n, int64_t lda, const double* lam, const void* U,
                            const void* B, const void* D, int k) {
  API_BEGIN(c)
  CHASE_REQUIRE(A && lam && U && B && D && n >= 1 && lda >= n && k >= 0, CHASE_ERR_ARG, "bad args");
  if (c->dtype == CHASE_C128)
    generate_wy<double2>(c->stream, (double2*)A, n, lda, lam, (const double2*)U, (const double2*)B, (const double2*)D, k);
  else
    generate_wy<double>(c->stream, (double*)A, n, lda, lam, (const double*)U, (const double*)B, (const double*)D, k);
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
  API_END(c)
}

chase_status chase_perturb(chase_ctx* c, void* A, int64_t n, int64_t lda, double eps, uint64_t seed) {
  API_BEGIN(c)
  CHASE_REQUIRE(A && n >= 1 && lda >= n, CHASE_ERR_ARG, "bad args");
  if (c->dtype == CHASE_C128)
    perturb<double2>(c->stream, (double2*)A, n, lda, eps, (unsigned long long)seed);
  else
    perturb<double>(c->stream, (double*)A, n, lda, eps, (unsigned long long)seed);
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
  API_END(c)
}

// One problem of a batch on context c (its stream): solve, then hand back the eigenvalues and
// the next start block (eigenvectors ascending followed by the rest of the search block).
static void solve_one_of_batch(chase_ctx* c, const void* A, int64_t n, int nev, int nex, double tol, int deg, int mode,
                               void* Vd, const void* L0, double* eigvals, chase_stats_t* stats) {
  const int ne = nev + nex;
  if (c->dtype == CHASE_C128) {
    Solver<double2>(c).solve((const double2*)A, n, n, nev, nex, tol, deg, mode, (const double2*)Vd,
                             (const double2*)L0);
    copy_cols<double2>(c->stream, n, ne, (const double2*)c->T1, n, (double2*)Vd, n);
  } else {
    Solver<double>(c).solve((const double*)A, n, n, nev, nex, tol, deg, mode, (const double*)Vd, (const double*)L0);
    copy_cols<double>(c->stream, n, ne, (const double*)c->T1, n, (double*)Vd, n);
  }
  CHASE_CUDA(cudaMemcpyAsync(eigvals, c->eigvals, nev * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
  if (stats) *stats = c->stats;
}

}  // extern "C"

// Runs fn(i) for i in [0, count) on up to `threads` host threads (each with the context's device
// current); the first exception is rethrown after every thread has finished.
template <typename Fn> static void parallel_for(int device, int threads, int count, Fn fn) {
  std::atomic<int> next{0};
  std::mutex mu;
  int err_status = CHASE_OK;
  std::string err_msg;
  auto run = [&]() {
    if (cudaSetDevice(device) != cudaSuccess) {
      std::lock_guard<std::mutex> lock(mu);
      if (err_status == CHASE_OK) {
        err_status = CHASE_ERR_CUDA;
        err_msg = "cudaSetDevice failed in a batch thread";
      }
      return;
    }
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= count) return;
      try {
        fn(i);
      } catch (const chase::Error& e) {
        std::lock_guard<std::mutex> lock(mu);
        if (err_status == CHASE_OK) {
          err_status = e.status;
          err_msg = e.msg;
        }
      } catch (const std::exception& e) {
        std::lock_guard<std::mutex> lock(mu);
        if (err_status == CHASE_OK) {
          err_status = CHASE_ERR_CUDA;
          err_msg = e.what();
        }
      }
    }
  };
  const int nt = std::max(1, std::min(threads, count));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(run);
  run();
  for (auto& t : pool) t.join();
  CHASE_REQUIRE(err_status == CHASE_OK, err_status, err_msg);
}

// Grouped batched solve: every problem runs Algorithm 1 in its own context (sized to it, own stream),
// and the problems advance in lockstep by outer iteration.  The filter (line 4) of all problems is one
// grouped split-product launch per degree step over every problem's tiles (a device-side list of
// (problem, tile) blocks in the launch's parameter block) on the batch context's stream; the other
// stages (Lanczos, QR, Rayleigh-Ritz, residuals, locking, degrees) run per problem on its stream, on
// opts.batch_workers host threads.
template <typename T>
static void solve_batched_grouped(chase_ctx* c, int nprob, const void* const* A, const int64_t* n, const int* nev,
                                  const int* nex, double tol, int deg, int mode, void* const* Vd, const void* const* L0,
                                  double* const* eigvals, chase_stats_t* stats_host) {
  constexpr bool CPLX = S<T>::cplx;
  // per-problem contexts, created on first use and kept while they are large enough
  chase_opts so = c->opts;
  so.batch_workers = 1;
  so.batch_grouped = 0;
  if ((int)c->slots.size() < nprob) c->slots.resize(nprob, nullptr);
  for (int p = 0; p < nprob; ++p) {
    chase_ctx*& sl = c->slots[p];
    const int ne = nev[p] + nex[p];
    if (sl && (sl->n_max < n[p] || sl->ne_max < ne)) {
      chase_destroy(sl);
      sl = nullptr;
    }
    if (!sl) {
      cudaStream_t ws = nullptr;
      CHASE_CUDA(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
      chase_status st = chase_create(&sl, n[p], ne, c->dtype, &so, ws);
      if (st != CHASE_OK) {
        cudaStreamDestroy(ws);
        sl = nullptr;
        throw chase::Error{(int)st, "creating the workspace of batch problem " + std::to_string(p) + " failed"};
      }
      sl->own_stream = true;
    }
  }
  // the grouped filter launches run on a stream of their own (measured: giving the problem streams a
  // higher priority only slowed the filter, with no gain in the overlap)
  if (!c->filter_stream) CHASE_CUDA(cudaStreamCreateWithFlags(&c->filter_stream, cudaStreamNonBlocking));
  cudaStream_t fs = c->filter_stream;
  // inputs the caller enqueued on the batch context's stream must be complete before the problem streams
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
  std::vector<typename Solver<T>::Run> R(nprob);
  std::vector<char> failed(nprob, 0);
  int err_status = CHASE_OK;
  std::string err_msg;
  auto fail_problem = [&](int p, const chase::Error& e) {
    failed[p] = 1;
    if (err_status == CHASE_OK) {
      err_status = e.status;
      err_msg = "problem " + std::to_string(p) + ": " + e.msg;
    }
  };
  const int threads = c->opts.batch_workers;
  // Lanczos bounds, start blocks, initial degrees
  {
    std::mutex mu;
    parallel_for(c->device, threads, nprob, [&](int p) {
      try {
        Solver<T>(c->slots[p]).begin(R[p], (const T*)A[p], n[p], n[p], nev[p], nex[p], tol, deg, mode, (const T*)Vd[p],
                                     (const T*)L0[p]);
      } catch (const chase::Error& e) {
        std::lock_guard<std::mutex> lock(mu);
        fail_problem(p, e);
      }
    });
  }
  c->stats = chase_stats_t{};
  oz::invalidate(c->ozw);
  // two cohorts of about equal filter work (n^3 per problem), whose stages alternate: while one cohort's
  // grouped filter runs on the batch stream, the other cohort's QR / Rayleigh-Ritz / bookkeeping run on
  // their own streams, so the latency-bound per-problem stages overlap the tensor-core launches
  std::vector<int> order(nprob);
  for (int p = 0; p < nprob; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  std::vector<int> cohort[2];
  double work[2] = {0.0, 0.0};
  for (int p : order) {
    const int h = work[0] <= work[1] ? 0 : 1;
    cohort[h].push_back(p);
    work[h] += (double)n[p] * (double)n[p] * (double)n[p];
  }
  std::vector<cudaEvent_t> evs;  // destroyed at the end (a destroyed event that a stream still waits on is fine)
  auto event = [&](unsigned flags) {
    cudaEvent_t e = nullptr;
    CHASE_CUDA(cudaEventCreateWithFlags(&e, flags));
    evs.push_back(e);
    return e;
  };
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> filter_times;
  struct FilterPlan {
    int p;
    double cc;
    std::vector<double> al, be;
    int f = 0;
    int64_t mv = 0;
  };
  auto active_of = [&](int h) {
    std::vector<int> a;
    for (int p : cohort[h])
      if (!failed[p] && !R[p].done(c->opts.maxiter)) a.push_back(p);
    return a;
  };
  // line 4 for every active problem of a cohort, enqueued on the batch stream: one grouped launch per
  // degree step (and arithmetic); returns without waiting for the device
  auto enqueue_filter = [&](const std::vector<int>& active) {
    cudaEvent_t t0 = event(cudaEventDefault), t1 = event(cudaEventDefault);
    std::vector<FilterPlan> plans;
    int smax = 0;
    for (int p : active) {
      chase_ctx* sc = c->slots[p];
      ++R[p].it;
      cudaEvent_t e = event(cudaEventDisableTiming);
      CHASE_CUDA(cudaEventRecord(e, sc->stream));
      CHASE_CUDA(cudaStreamWaitEvent(fs, e, 0));
      if (R[p].k() <= 0) continue;
      FilterPlan fp;
      fp.p = p;
      double ee;
      const int mmax = R[p].m[R[p].k() - 1];
      filter_coeffs(R[p].b_sup, R[p].mu_1, R[p].mu_ne, mmax, fp.cc, ee, fp.al, fp.be);
      smax = std::max(smax, mmax);
      plans.push_back(std::move(fp));
    }
    CHASE_CUDA(cudaEventRecord(t0, fs));
    // the digit planes of A: computed once per solve (cached in the problem's workspace)
    for (FilterPlan& fp : plans) oz::prepare_A<T>(fs, c->slots[fp.p]->ozw, R[fp.p].A, R[fp.p].n, R[fp.p].lda,
                                                  CHASE_FP64);
    std::vector<oz::ProductOp> ops_hi, ops_lo;
    for (int sstep = 1; sstep <= smax; ++sstep) {
      ops_hi.clear();
      ops_lo.clear();
      for (FilterPlan& fp : plans) {
        auto& r = R[fp.p];
        chase_ctx* sc = c->slots[fp.p];
        const int k = r.k();
        while (fp.f < k && r.m[fp.f] < sstep) ++fp.f;
        const int cols = k - fp.f;
        if (cols <= 0) continue;
        fp.mv += cols;
        T* Vact = (T*)sc->V + (int64_t)r.l * r.n;
        T* T1act = (T*)sc->T1 + (int64_t)r.l * r.n;
        T* Bb[2] = {Vact, T1act};
        T* out = Bb[sstep & 1] + (int64_t)fp.f * r.n;
        const T* in = Bb[(sstep - 1) & 1] + (int64_t)fp.f * r.n;
        const int fmode = r.fmode();
        oz::split_right<T>(fs, sc->ozw, fmode, in, r.n, cols, r.n);
        Epi e;
        e.C = out;
        e.ldc = r.n;
        e.alpha = fp.al[sstep];
        e.Y = in;
        e.ldy = r.n;
        e.gamma = -fp.al[sstep] * fp.cc;
        if (sstep >= 2) {
          e.Z = out;
          e.ldz = r.n;
          e.beta = fp.be[sstep];
        }
        oz::ProductOp op{sc->ozw.a_planes, sc->ozw.a_scale, sc->ozw.slices, sc->ozw.b_planes, sc->ozw.b_scale,
                         r.n, cols, r.n, e, c->ozw.group_m};
        (fmode == CHASE_FP64 ? ops_hi : ops_lo).push_back(op);
        sc->stats.filter_launches++;
      }
      if (!ops_hi.empty()) oz::launch_group<CPLX>(fs, c->ozw, CHASE_FP64, ops_hi.data(), (int)ops_hi.size());
      // the low-precision problems of one batch share its mode
      if (!ops_lo.empty()) oz::launch_group<CPLX>(fs, c->ozw, mode, ops_lo.data(), (int)ops_lo.size());
    }
    for (FilterPlan& fp : plans) {
      auto& r = R[fp.p];
      chase_ctx* sc = c->slots[fp.p];
      const int k = r.k();
      T* Vact = (T*)sc->V + (int64_t)r.l * r.n;
      T* T1act = (T*)sc->T1 + (int64_t)r.l * r.n;
      dim3 grid(std::min<unsigned>(ceil_div(r.n, 256), 64), k);
      gather_odd_kernel<T><<<grid, 256, 0, fs>>>(r.n, sc->deg, Vact, r.n, T1act, r.n);
      CHASE_CHECK_LAUNCH();
      Solver<T>(sc).count_matvecs(r, fp.mv);
    }
    CHASE_CUDA(cudaEventRecord(t1, fs));
    filter_times.emplace_back(t0, t1);
    cudaEvent_t done_f = event(cudaEventDisableTiming);
    CHASE_CUDA(cudaEventRecord(done_f, fs));
    for (int p : active) CHASE_CUDA(cudaStreamWaitEvent(c->slots[p]->stream, done_f, 0));
  };
  // lines 5-14 per problem of a cohort, on the host threads (each problem on its own stream)
  auto after = [&](const std::vector<int>& active) {
    std::mutex mu;
    parallel_for(c->device, threads, (int)active.size(), [&](int i) {
      const int p = active[i];
      try {
        Solver<T>(c->slots[p]).after_filter(R[p]);
      } catch (const chase::Error& e) {
        std::lock_guard<std::mutex> lock(mu);
        fail_problem(p, e);
      }
    });
  };
  try {
    std::vector<int> act[2] = {active_of(0), active_of(1)};
    for (int h = 0; h < 2; ++h)
      if (!act[h].empty()) enqueue_filter(act[h]);
    for (int h = 0; !act[0].empty() || !act[1].empty(); h ^= 1) {
      if (act[h].empty()) continue;
      after(act[h]);
      act[h] = active_of(h);
      if (!act[h].empty()) enqueue_filter(act[h]);
    }
    CHASE_CUDA(cudaStreamSynchronize(fs));
    for (auto& t : filter_times) {
      float ms = 0.f;
      CHASE_CUDA(cudaEventElapsedTime(&ms, t.first, t.second));
      c->stats.ms_filter += ms;
    }
    CHASE_REQUIRE(oz::read_flags(fs, c->ozw) == 0, CHASE_ERR_TIMEOUT,
                  "a grouped tensor-core product hit its wait limit");
  } catch (...) {
    cudaStreamSynchronize(fs);
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    throw;
  }
  for (cudaEvent_t e : evs) cudaEventDestroy(e);
  // results: eigenvalues, eigenvectors followed by the rest of the search block (next start block)
  {
    std::mutex mu;
    parallel_for(c->device, threads, nprob, [&](int p) {
      if (failed[p]) return;
      chase_ctx* sc = c->slots[p];
      try {
        Solver<T>(sc).finish(R[p]);
        const int ne = nev[p] + nex[p];
        copy_cols<T>(sc->stream, n[p], ne, (const T*)sc->T1, n[p], (T*)Vd[p], n[p]);
        CHASE_CUDA(cudaMemcpyAsync(eigvals[p], sc->eigvals, nev[p] * sizeof(double), cudaMemcpyDeviceToDevice,
                                   sc->stream));
        CHASE_CUDA(cudaStreamSynchronize(sc->stream));
      } catch (const chase::Error& e) {
        std::lock_guard<std::mutex> lock(mu);
        fail_problem(p, e);
      }
      if (stats_host) stats_host[p] = sc->stats;
    });
  }
  CHASE_REQUIRE(err_status == CHASE_OK, err_status, err_msg);
}

extern "C" {

chase_status chase_solve_batched(chase_ctx* c, int nprob, const void* const* A, const int64_t* n, const int* nev,
                                 const int* nex, double tol, int deg, int mode, void* const* Vd, const void* const* L0,
                                 double* const* eigvals, chase_stats_t* stats_host) {
  API_BEGIN(c)
  CHASE_REQUIRE(nprob >= 0 && A && n && nev && nex && Vd && L0 && eigvals, CHASE_ERR_ARG, "bad args");
  for (int p = 0; p < nprob; ++p)
    CHASE_REQUIRE(n[p] >= 1 && n[p] <= c->n_max && nev[p] >= 1 && nex[p] >= 0 && nev[p] + nex[p] <= c->ne_max,
                  CHASE_ERR_ARG, "problem " + std::to_string(p) + " exceeds the context's sizes");
  if (c->opts.batch_grouped && mode != CHASE_FP64_NATIVE && oz::available()) {
    if (c->dtype == CHASE_C128)
      solve_batched_grouped<double2>(c, nprob, A, n, nev, nex, tol, deg, mode, Vd, L0, eigvals, stats_host);
    else
      solve_batched_grouped<double>(c, nprob, A, n, nev, nex, tol, deg, mode, Vd, L0, eigvals, stats_host);
  } else if (c->workers.empty()) {
    for (int p = 0; p < nprob; ++p)
      solve_one_of_batch(c, A[p], n[p], nev[p], nex[p], tol, deg, mode, Vd[p], L0[p], eigvals[p],
                         stats_host ? &stats_host[p] : nullptr);
  } else {
    // inputs the caller enqueued on the context's stream must be complete before the workers'
    // non-blocking streams read them
    CHASE_CUDA(cudaStreamSynchronize(c->stream));
    std::vector<int> order(nprob);
    for (int p = 0; p < nprob; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
    std::atomic<int> next{0};
    std::atomic<bool> failed{false};
    int err_status = CHASE_OK;
    std::string err_msg;
    std::mutex err_mu;
    auto record = [&](int status, const std::string& msg) {
      std::lock_guard<std::mutex> lock(err_mu);
      if (err_status == CHASE_OK) {
        err_status = status;
        err_msg = msg;
      }
      failed.store(true);
    };
    auto run = [&](chase_ctx* wc) {
      if (cudaSetDevice(wc->device) != cudaSuccess) {
        record(CHASE_ERR_CUDA, "cudaSetDevice failed in a batch worker");
        return;
      }
      for (;;) {
        if (failed.load()) return;
        const int i = next.fetch_add(1);
        if (i >= nprob) return;
        const int p = order[i];
        try {
          solve_one_of_batch(wc, A[p], n[p], nev[p], nex[p], tol, deg, mode, Vd[p], L0[p], eigvals[p],
                             stats_host ? &stats_host[p] : nullptr);
        } catch (const chase::Error& e) {
          record(e.status, "problem " + std::to_string(p) + ": " + e.msg);
        } catch (const std::exception& e) {
          record(CHASE_ERR_CUDA, "problem " + std::to_string(p) + ": " + e.what());
        }
      }
    };
    std::vector<std::thread> threads;
    threads.reserve(c->workers.size());
    for (chase_ctx* wc : c->workers) threads.emplace_back(run, wc);
    run(c);
    for (auto& t : threads) t.join();
    CHASE_REQUIRE(err_status == CHASE_OK, err_status, err_msg);
  }
  CHASE_CUDA(cudaStreamSynchronize(c->stream));
  API_END(c)
}

chase_status chase_backward(chase_ctx* c, const void* A, int64_t lda, const double* gl, const void* gV, int64_t ldg,
                            void* gA, int64_t ldga, double minres_tol, int minres_maxit) {
  API_BEGIN(c)
  CHASE_REQUIRE(c->dtype == CHASE_R64, CHASE_ERR_UNSUPPORTED, "backward implemented for real symmetric problems");
  CHASE_REQUIRE(c->have_result, CHASE_ERR_STATE, "no solve result");
  CHASE_REQUIRE(A != nullptr, CHASE_ERR_ARG, "null A");
  Timer t(c, 0, &c->stats.ms_backward);
  Solver<double>(c).backward((const double*)A, lda, gl, (const double*)gV, ldg, (double*)gA, ldga, minres_tol,
                             minres_maxit);
  t.stop();
  API_END(c)
}

}  // extern "C"
