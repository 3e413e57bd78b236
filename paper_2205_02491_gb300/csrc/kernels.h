// Internal launch interface of the FP64 kernels (host side).  Not part of the C ABI.
#pragma once
#include <functional>
#include <cuda_runtime.h>
#include <stdint.h>

namespace chase {

enum Op { OP_N = 0, OP_C = 1 };  // OP_C: conjugate transpose (transpose for real)

// Epilogue of a product:  C = alpha*acc + gamma*ycol[j]*Y + beta*Z  (Y, Z optional; Z may alias C).
struct Epi {
  void* C = nullptr;
  int64_t ldc = 0;
  double alpha = 1.0;
  const void* Y = nullptr;
  int64_t ldy = 0;
  double gamma = 0.0;
  const double* ycol = nullptr;  // per-column factor on Y (device), optional
  const void* Z = nullptr;
  int64_t ldz = 0;
  double beta = 0.0;
};

// C(MxN) = op(A) op(B) with epilogue, FP64 DFMA.  work: >= ksplit*M*N scalars when ksplit > 1.
template <typename T>
void gemm_f64(cudaStream_t st, Op opA, Op opB, int64_t M, int64_t N, int64_t K, const T* A, int64_t lda,
              const T* B, int64_t ldb, const Epi& epi, T* work, int64_t work_elems);

template <typename T> void colnorms(cudaStream_t st, int64_t n, int k, const T* X, int64_t ldx, double* out);
template <typename T> void colmaxabs(cudaStream_t st, int64_t n, int k, const T* X, int64_t ldx, double* out);
template <typename T>
void permute_cols(cudaStream_t st, int64_t n, int k, const T* src, int64_t lds, T* dst, int64_t ldd, const int* perm);
template <typename T> void scale_cols(cudaStream_t st, int64_t n, int k, T* X, int64_t ldx, const double* s, int invert);
template <typename T>
void copy_cols(cudaStream_t st, int64_t n, int k, const T* src, int64_t lds, T* dst, int64_t ldd);

// Cholesky G = L L^H (lower, in place, k x k).  info: device int, set > 0 on a non-finite pivot or one
// <= pivot_floor.  dep (nullable, k + 1 ints, zeroed by the caller): detection mode, where a finite pivot
// <= pivot_floor marks its column as numerically dependent (dep[1 + j] = 1, dep[0] counts them) instead
// of failing; such a column is decoupled (unit pivot, zero below it) and the factorisation goes on.
template <typename T>
void potrf_lower(cudaStream_t st, int k, T* G, int64_t ldg, int* info, T* work, int64_t work_elems,
                 double pivot_floor = 0.0, int* dep = nullptr);
// Householder QR building blocks (blas_f64.cu): reflector of a column segment (v over x, alpha, real tau),
// application of one reflector to ncols columns, the panel's reflectors with explicit zeros, the
// compact-WY factor Tm of a panel from Gv = V^H V, and Q = [I; 0].
template <typename T> void householder_vec(cudaStream_t st, int64_t m, T* x, T* alpha, double* tau);
template <typename T>
void householder_apply(cudaStream_t st, int64_t m, const T* v, T* X, int64_t ldx, int ncols, const double* tau);
template <typename T> void reflector_panel(cudaStream_t st, int64_t m, int pb, const T* Xp, int64_t ldx, T* V, int64_t ldv);
template <typename T> void householder_T(cudaStream_t st, int pb, const T* Gv, const double* tau, T* Tm, int64_t ldt);
template <typename T> void identity_rect(cudaStream_t st, int64_t n, int k, T* Q, int64_t ldq);

// X <- X L^{-H} (right solve with the lower Cholesky factor), X n x k.
template <typename T>
void trsm_right_lh(cudaStream_t st, int64_t n, int k, T* X, int64_t ldx, const T* L, int64_t ldl, T* work,
                   int64_t work_elems);
template <typename T> void zero_upper(cudaStream_t st, int k, T* G, int64_t ldg);
// inverts every CB x CB diagonal block of the lower-triangular L in place (CB = 32)
template <typename T> void trtri_diag(cudaStream_t st, int k, T* L, int64_t ldl);
template <typename T> void add_diag(cudaStream_t st, int k, T* G, int64_t ldg, const double* shift_dev, double shift);
template <typename T> void hermitianize(cudaStream_t st, int k, T* G, int64_t ldg);
template <typename T> void fro_norm2(cudaStream_t st, int64_t n, int k, const T* X, int64_t ldx, double* out);

// Parallel cyclic Jacobi: G (k x k, destroyed) -> w ascending, Z.  Returns sweeps used; throws on cap.
template <typename T>
int heev_jacobi(cudaStream_t st, int k, T* G, int64_t ldg, double* w, T* Z, int64_t ldz, T* work,
                int64_t work_elems, double* dwork, int* iwork, double tol, int max_sweeps,
                bool require_convergence = true, bool persistent = false);

// Two-sided block Jacobi (blocks of 32, one CTA per block pair per round) for the FP32 first pass of the
// mixed eigensolve: G (k x k, destroyed) -> w ascending, Z.  work: k*k + heev_block_workspace(k) scalars.
// Returns the sweeps used (the cap is not an error: the FP64 refinement follows).
int heev_block_workspace(int k);
template <typename F>
int heev_block_jacobi(cudaStream_t st, int k, F* G, int64_t ldg, double* w, F* Z, int64_t ldz, F* work,
                      int64_t work_elems, double* dwork, int* iwork, double tol, int max_sweeps);

// mixed-precision eigensolve helpers (eig_mixed.cu)
template <typename T, typename F> void convert_mat(cudaStream_t st, int k, const T* in, int64_t ldi, F* out, int64_t ldo);
template <typename T>
void eig_correction(cudaStream_t st, int k, const T* Gp, int64_t ldg, T* X, int64_t ldx, double omega);
template <typename T>
void cluster_eig(cudaStream_t st, int k, int nclusters, const int* cl /* start,size pairs (device) */, const T* Gp,
                 int64_t ldg, T* Z, int64_t ldz, double* w, T* scratch, int* status);
template <typename T> void diag_real(cudaStream_t st, int k, const T* G, int64_t ldg, double* d);
template <typename T>
void sort_pairs(cudaStream_t st, int k, double* w, T* Z, int64_t ldz, T* tmp, double* wtmp, int* perm);

// Lanczos bounds (Algorithm 1, line 2).  out4 (device) = {b_sup, mu_1, mu_ne, theta_max}.
// matvec (nullable): W (n x runs, ld n) = A X (X: n x runs, ld ldx) on stream st, replacing the
// DFMA multi-vector HEMV (used with the FP64-class split tensor-core products).
template <typename T> using MatvecFn = std::function<void(const T* X, int64_t ldx, T* W)>;
template <typename T>
void lanczos(cudaStream_t st, const T* A, int64_t n, int64_t lda, int ne, const T* L0, int runs, int steps,
             double* out4, T* work, int64_t work_elems, double* dwork, const MatvecFn<T>* matvec = nullptr);

// Input generator from compact-WY factors.
template <typename T>
void generate_wy(cudaStream_t st, T* A, int64_t n, int64_t lda, const double* lam, const T* U, const T* B,
                 const T* D, int k);

// A += eps * H(seed), H a counter-based seeded Hermitian Gaussian scaled to spectral norm about 1.
template <typename T>
void perturb(cudaStream_t st, T* A, int64_t n, int64_t lda, double eps, unsigned long long seed);

// X (rows x cols, ld ldx) <- seeded counter-based normals (SplitMix64 + Box-Muller; complex: (x + i y)/sqrt(2)),
// counter i + j rows: the library's start block and Lanczos start vectors when the caller passes none
template <typename T> void fill_normal(cudaStream_t st, T* X, int64_t rows, int cols, int64_t ldx, unsigned long long seed);

// Bookkeeping (Algorithm 1, lines 8-14) on the device.  See chase.cu for the layout of `bk`.
void bookkeeping(cudaStream_t st, int k, const double* ritz, const double* res, double thresh, double b_sup,
                 double* bounds, int maxdeg, int extra_deg, int* out_lock, int* out_deg, int* out_perm,
                 double* out_ritz, double* out_res, int* scratch);

// adjoint helpers (adjoint.cu)
void adj_inner(cudaStream_t st, int l, int nev, const double* lam, const double* M, int64_t ldm, const double* gl,
               double* inner, int64_t ldi);
void minres_init(cudaStream_t st, int64_t n, int nev, const double* B, int64_t ldb, double* R1, double* R2,
                 double* Vv, double* X, double* W, double* W2, void* state, double tol);
void minres_update(cudaStream_t st, int64_t n, int nev, const double* Y, double* R1, const double* R2, double* Vv,
                   double* Wn, const double* Wc, double* X, void* state, double tol);
void minres_count_done(cudaStream_t st, int nev, const void* state, int* out);
void add_inplace(cudaStream_t st, int64_t count, double* a, const double* b);
size_t minres_state_bytes(int nev);

}  // namespace chase
