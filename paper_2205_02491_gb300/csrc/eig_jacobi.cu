// Dense Hermitian eigensolver of the Rayleigh-Ritz quotient (Algorithm 1,
// line 6) on the device: parallel cyclic two-sided Jacobi in FP64.
//
// Ordering: round-robin tournament on kp = k rounded up to even indices; each
// of the kp-1 rounds of a sweep rotates kp/2 disjoint pairs at once.  A round
// is two launches: rotation parameters for every pair (from the 2x2 blocks of
// the current G), then an in-place update of G (2x2 blocks of J^H G J) and of
// Z (Z J).  For each pair the 2x2 block [[a, g], [conj g, b]] is made real by
// the phase D = diag(1, conj(g)/|g|) and zeroed by the real rotation with
// t = sign(z)/(|z| + sqrt(1+z^2)), z = (b-a)/(2|g|).
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace chase {

template <typename T> struct Rot {
  int partner;  // index paired with this one in the current round (-1: none)
  T self;       // J[x][x]
  T other;      // J[partner][x]
};

__device__ inline void round_pair(int r, int idx, int kp, int& a, int& b) {
  int m = kp - 1;
  if (idx == 0) {
    a = r;
    b = kp - 1;
  } else {
    a = (r + idx) % m;
    b = (r - idx + m) % m;
  }
}

// rotation parameters of pair idx of round r.  The device functions take plain (not __restrict__)
// pointers: inside the persistent sweep kernel G and the rotations are written by other blocks
// between barriers, so their loads must not go through the non-coherent read-only path.
template <typename T>
__device__ __forceinline__ void jacobi_params(int k, int kp, int r, int idx, const T* G, int64_t ldg, Rot<T>* rot) {
  using s = S<T>;
  int a, b;
  round_pair(r, idx, kp, a, b);
  int p = min(a, b), q = max(a, b);
  if (q >= k) {  // dummy index for odd k
    if (p < k) rot[p] = Rot<T>{-1, s::one(), s::zero()};
    return;
  }
  T g = G[p + (int64_t)q * ldg];
  double ag = sqrt(s::abs2(g));
  if (!(ag > 1e-300)) {
    rot[p] = Rot<T>{q, s::one(), s::zero()};
    rot[q] = Rot<T>{p, s::one(), s::zero()};
    return;
  }
  double ap = s::re(G[p + (int64_t)p * ldg]), bq = s::re(G[q + (int64_t)q * ldg]);
  double z = (bq - ap) / (2.0 * ag);
  double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
  double c = 1.0 / sqrt(1.0 + t * t);
  double sn = t * c;
  T ph = s::scale(s::conj(g), 1.0 / ag);  // conj(g)/|g|
  // J = [[c, sn], [-sn*ph, c*ph]] on columns (p, q)
  rot[p] = Rot<T>{q, s::make(c, 0.0), s::scale(ph, -sn)};  // J[p][p], J[q][p]
  rot[q] = Rot<T>{p, s::scale(ph, c), s::make(sn, 0.0)};   // J[q][q], J[p][q]
}

template <typename T>
__global__ void jacobi_params_kernel(int k, int kp, int r, const T* __restrict__ G, int64_t ldg, Rot<T>* rot) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kp / 2) return;
  jacobi_params<T>(k, kp, r, idx, G, ldg, rot);
}

// G <- J^H G J, one thread per (row pair, column pair) 2x2 block (in place).  Split into a load
// and a compute/store half so that the persistent sweep can keep several blocks' loads in flight.
template <typename T> struct GItem {
  int rows[2], cols[2];
  bool diag;  // i1 == i2: the rotated pair's own 2x2 block
  T in[2][2], js[2], jo[2], ks[2], ko[2];
};

template <typename T>
__device__ __forceinline__ void g_load(int k, int kp, int r, int i1, int i2, const T* G, int64_t ldg,
                                       const Rot<T>* rot, GItem<T>& it) {
  using s = S<T>;
  round_pair(r, i1, kp, it.rows[0], it.rows[1]);
  round_pair(r, i2, kp, it.cols[0], it.cols[1]);
  it.diag = i1 == i2;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v)
      it.in[u][v] = (it.rows[u] < k && it.cols[v] < k) ? G[it.rows[u] + (int64_t)it.cols[v] * ldg] : s::zero();
  // coefficients: J[x][x] and J[partner(x)][x]
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    if (it.rows[u] < k) {
      Rot<T> rr = rot[it.rows[u]];
      it.js[u] = rr.self;
      it.jo[u] = rr.partner >= 0 ? rr.other : s::zero();
    } else {
      it.js[u] = s::one();
      it.jo[u] = s::zero();
    }
    if (it.cols[u] < k) {
      Rot<T> rc = rot[it.cols[u]];
      it.ks[u] = rc.self;
      it.ko[u] = rc.partner >= 0 ? rc.other : s::zero();
    } else {
      it.ks[u] = s::one();
      it.ko[u] = s::zero();
    }
  }
}

template <typename T>
__device__ __forceinline__ void g_store(int k, T* G, int64_t ldg, const GItem<T>& it) {
  using s = S<T>;
  // column update: C[u][v] = in[u][v] J[v][v] + in[u][v'] J[v'][v]
  T cu[2][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) cu[u][v] = s::add(s::mul(it.in[u][v], it.ks[v]), s::mul(it.in[u][1 - v], it.ko[v]));
  // row update: out[u][v] = conj(J[u][u]) C[u][v] + conj(J[u'][u]) C[u'][v]
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      if (it.rows[u] >= k || it.cols[v] >= k) continue;
      T o = s::add(s::mul(s::conj(it.js[u]), cu[u][v]), s::mul(s::conj(it.jo[u]), cu[1 - u][v]));
      if (it.rows[u] == it.cols[v]) o = s::make(s::re(o), 0.0);
      if (it.diag && u != v) o = s::zero();  // the rotated pair's off-diagonal entry
      G[it.rows[u] + (int64_t)it.cols[v] * ldg] = o;
    }
}

template <typename T>
__device__ __forceinline__ void jacobi_apply_g(int k, int kp, int r, int i1, int i2, T* G, int64_t ldg,
                                               const Rot<T>* rot) {
  GItem<T> it;
  g_load<T>(k, kp, r, i1, i2, G, ldg, rot, it);
  g_store<T>(k, G, ldg, it);
}

template <typename T>
__global__ void jacobi_apply_g_kernel(int k, int kp, int r, T* G, int64_t ldg, const Rot<T>* __restrict__ rot) {
  int i1 = blockIdx.x * blockDim.x + threadIdx.x;  // row pair index
  int i2 = blockIdx.y * blockDim.y + threadIdx.y;  // column pair index
  int half = kp / 2;
  if (i1 >= half || i2 >= half) return;
  jacobi_apply_g<T>(k, kp, r, i1, i2, G, ldg, rot);
}

// Z <- Z J (rows i, column pairs), in place; load / compute-store halves as for G.
template <typename T> struct ZItem {
  int a, b;
  T za, zb, as, ao, bs, bo;
};

template <typename T>
__device__ __forceinline__ bool z_load(int k, int kp, int r, int i, int pi, const T* Z, int64_t ldz,
                                       const Rot<T>* rot, ZItem<T>& it) {
  round_pair(r, pi, kp, it.a, it.b);
  if (it.a >= k || it.b >= k) return false;
  const Rot<T> ra = rot[it.a], rb = rot[it.b];
  it.as = ra.self;
  it.ao = ra.other;
  it.bs = rb.self;
  it.bo = rb.other;
  it.za = Z[i + (int64_t)it.a * ldz];
  it.zb = Z[i + (int64_t)it.b * ldz];
  return true;
}

template <typename T> __device__ __forceinline__ void z_store(int i, T* Z, int64_t ldz, const ZItem<T>& it) {
  using s = S<T>;
  Z[i + (int64_t)it.a * ldz] = s::add(s::mul(it.za, it.as), s::mul(it.zb, it.ao));
  Z[i + (int64_t)it.b * ldz] = s::add(s::mul(it.zb, it.bs), s::mul(it.za, it.bo));
}

template <typename T>
__device__ __forceinline__ void jacobi_apply_z(int k, int kp, int r, int i, int pi, T* Z, int64_t ldz,
                                               const Rot<T>* rot) {
  ZItem<T> it;
  if (z_load<T>(k, kp, r, i, pi, Z, ldz, rot, it)) z_store<T>(i, Z, ldz, it);
}

template <typename T>
__global__ void jacobi_apply_z_kernel(int k, int kp, int r, T* Z, int64_t ldz, const Rot<T>* __restrict__ rot) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int pi = blockIdx.y;
  if (i >= k) return;
  jacobi_apply_z<T>(k, kp, r, i, pi, Z, ldz, rot);
}

// ---------------------------------------------------------------- persistent sweep
// One cooperative launch runs all kp-1 rounds of a sweep: rotation parameters, then the G and Z
// updates, separated by grid-wide barriers (all blocks are co-resident under a cooperative
// launch).  Every barrier wait is bounded by a wall-clock limit; on expiry, or when another block
// has flagged an error, the block sets/keeps the error flag and returns.
constexpr int SWEEP_THREADS = 256;  // up to four blocks per SM (measured faster than one 1024-thread block)
// barrier words, each in its own 32-byte sector so that the pollers of the generation word do not
// contend with the arrival atomics
constexpr int BAR_COUNT = 0, BAR_GEN = 8, BAR_ERR = 16, BAR_WORDS = 17;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bar[BAR_COUNT]: arrivals, bar[BAR_GEN]: generation, bar[BAR_ERR]: error flag (all zero at launch);
// wait_ns: wall-clock limit of one wait
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned long long wait_ns) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vb = bar;
    int ok = vb[BAR_ERR] == 0u;
    if (ok) {
      const unsigned gen = vb[BAR_GEN];
      __threadfence();
      if (atomicAdd(&bar[BAR_COUNT], 1u) == nblocks - 1) {
        atomicExch(&bar[BAR_COUNT], 0u);
        __threadfence();
        atomicAdd(&bar[BAR_GEN], 1u);
      } else {
        const unsigned long long t0 = gtimer();
        while (vb[BAR_GEN] == gen) {
          if (vb[BAR_ERR] != 0u) {
            ok = 0;
            break;
          }
          if (gtimer() - t0 > wait_ns) {
            atomicOr(&bar[BAR_ERR], 1u);
            ok = 0;
            break;
          }
          __nanosleep(100);
        }
      }
      __threadfence();
    }
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

template <typename T>
__global__ void __launch_bounds__(SWEEP_THREADS, 4) jacobi_sweep_kernel(int k, int kp, T* G, int64_t ldg, T* Z,
                                                                        int64_t ldz, Rot<T>* rot, unsigned* bar,
                                                                        unsigned long long wait_ns) {
  const int half = kp / 2;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int64_t ng = (int64_t)half * half, nz = (int64_t)k * half;
  for (int r = 0; r < kp - 1; ++r) {
    for (int64_t idx = tid; idx < half; idx += nthr) jacobi_params<T>(k, kp, r, (int)idx, G, ldg, rot);
    if (!grid_barrier(bar, gridDim.x, wait_ns)) return;
    for (int64_t x = tid; x < ng; x += nthr) jacobi_apply_g<T>(k, kp, r, (int)(x % half), (int)(x / half), G, ldg, rot);
    for (int64_t x = tid; x < nz; x += nthr) jacobi_apply_z<T>(k, kp, r, (int)(x % k), (int)(x / k), Z, ldz, rot);
    if (!grid_barrier(bar, gridDim.x, wait_ns)) return;
  }
}

// co-resident blocks of SWEEP_THREADS threads for the sweep kernel (0: no cooperative launch)
template <typename T> static int sweep_grid() {
  static const int nb = []() {
    int dev = 0, sms = 0, per = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jacobi_sweep_kernel<T>, SWEEP_THREADS, 0) != cudaSuccess)
      return 0;
    return sms * std::min(per, 4);
  }();
  return nb;
}

template <typename T> __global__ void set_identity_kernel(int k, T* Z, int64_t ldz) {
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i < k) Z[i + (int64_t)j * ldz] = (i == j) ? S<T>::one() : S<T>::zero();
}

// off^2 and fro^2 of G: per-column partials then an ordered sum (deterministic)
template <typename T> __global__ void offdiag_partial_kernel(int k, const T* __restrict__ G, int64_t ldg, double* part) {
  using s = S<T>;
  int j = blockIdx.x;
  double off = 0.0, tot = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double v = s::abs2(G[i + (int64_t)j * ldg]);
    tot += v;
    if (i != j) off += v;
  }
  __shared__ double r1[32], r2[32];
  off = warp_sum(off);
  tot = warp_sum(tot);
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = off;
    r2[threadIdx.x >> 5] = tot;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double a = threadIdx.x < (blockDim.x >> 5) ? r1[threadIdx.x] : 0.0;
    double b = threadIdx.x < (blockDim.x >> 5) ? r2[threadIdx.x] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x == 0) {
      part[2 * j] = a;
      part[2 * j + 1] = b;
    }
  }
}

__global__ void offdiag_sum_kernel(int k, const double* part, double* out) {
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < k; j += 32) {
    a += part[2 * j];
    b += part[2 * j + 1];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

// eigenvalues from the diagonal, ascending rank (stable), permutation
template <typename T>
__global__ void diag_rank_kernel(int k, const T* __restrict__ G, int64_t ldg, double* w, int* perm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  double wi = S<T>::re(G[i + (int64_t)i * ldg]);
  int rank = 0;
  for (int j = 0; j < k; ++j) {
    double wj = S<T>::re(G[j + (int64_t)j * ldg]);
    rank += (wj < wi) || (wj == wi && j < i);
  }
  w[rank] = wi;
  perm[rank] = i;
}

template <typename T>
int heev_jacobi(cudaStream_t st, int k, T* G, int64_t ldg, double* w, T* Z, int64_t ldz, T* work, int64_t work_elems,
                double* dwork, int* iwork, double tol, int max_sweeps, bool require_convergence, bool persistent) {
  // work: k*k scalars for the unsorted Z plus Rot array; dwork: 2k+2 doubles; iwork: k ints
  CHASE_REQUIRE(work_elems >= (int64_t)k * k + 3 * (int64_t)k + 8, 2, "heev_jacobi: workspace too small");
  if (k <= 0) return 0;
  T* Zu = work;
  Rot<T>* rot = reinterpret_cast<Rot<T>*>(work + (int64_t)k * k);
  int kp = k + (k & 1);
  set_identity_kernel<T><<<dim3(ceil_div(k, 256), k), 256, 0, st>>>(k, Zu, k);
  CHASE_CHECK_LAUNCH();
  double* part = dwork + 2;
  double hstat[2];
  int sweeps = 0;
  bool done = false;
  // one cooperative launch per sweep; the barrier words live in iwork[0, BAR_WORDS) (k >= 64 ints;
  // overwritten by the final ranking only after the sweeps)
  // grid sized by the work of a round (about 4 rotation updates per thread), at most the co-resident
  // maximum: small quotients take few SMs, which leaves room for other streams' kernels
  int coop_grid = (persistent && k >= 64) ? sweep_grid<T>() : 0;
  if (coop_grid > 0) {
    const int64_t items = (int64_t)(kp / 2) * (kp / 2) + (int64_t)k * (kp / 2);
    coop_grid = (int)std::max<int64_t>(1, std::min<int64_t>(coop_grid, ceil_div(items, 4 * SWEEP_THREADS)));
  }
  unsigned* bar = reinterpret_cast<unsigned*>(iwork);
  unsigned bar_err = 0;
  for (; sweeps <= max_sweeps; ++sweeps) {
    offdiag_partial_kernel<T><<<k, 128, 0, st>>>(k, G, ldg, part);
    CHASE_CHECK_LAUNCH();
    offdiag_sum_kernel<<<1, 32, 0, st>>>(k, part, dwork);
    CHASE_CHECK_LAUNCH();
    CHASE_CUDA(cudaMemcpyAsync(hstat, dwork, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (coop_grid > 0 && sweeps > 0)
      CHASE_CUDA(cudaMemcpyAsync(&bar_err, bar + BAR_ERR, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CHASE_CUDA(cudaStreamSynchronize(st));
    CHASE_REQUIRE(bar_err == 0, 8, "heev_jacobi: a grid barrier of the sweep kernel hit its wait limit");
    CHASE_REQUIRE(isfinite(hstat[0]) && isfinite(hstat[1]), 5, "heev_jacobi: non-finite matrix");
    if (sqrt(hstat[0]) <= tol * sqrt(hstat[1]) || k == 1) {
      done = true;
      break;
    }
    if (sweeps == max_sweeps) break;
    int half = kp / 2;
    dim3 gblk(16, 16), ggrid(ceil_div(half, 16), ceil_div(half, 16));
    dim3 zgrid(ceil_div(k, 128), half);
    if (coop_grid > 0) {
      CHASE_CUDA(cudaMemsetAsync(bar, 0, BAR_WORDS * sizeof(unsigned), st));
      int kk = k, kpp = kp;
      int64_t ldgg = ldg, ldzz = k;
      T* Gp = G;
      T* Zp = Zu;
      Rot<T>* rp = rot;
      unsigned long long wait_ns = grid_wait_limit_ns();
      void* args[] = {&kk, &kpp, &Gp, &ldgg, &Zp, &ldzz, &rp, &bar, &wait_ns};
      CHASE_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_sweep_kernel<T>, dim3(coop_grid), dim3(SWEEP_THREADS),
                                             args, 0, st));
      CHASE_CHECK_LAUNCH();
    } else {
      for (int r = 0; r < kp - 1; ++r) {
        jacobi_params_kernel<T><<<ceil_div(half, 128), 128, 0, st>>>(k, kp, r, G, ldg, rot);
        CHASE_CHECK_LAUNCH();
        jacobi_apply_g_kernel<T><<<ggrid, gblk, 0, st>>>(k, kp, r, G, ldg, rot);
        CHASE_CHECK_LAUNCH();
        jacobi_apply_z_kernel<T><<<zgrid, 128, 0, st>>>(k, kp, r, Zu, k, rot);
        CHASE_CHECK_LAUNCH();
      }
    }
  }
  CHASE_REQUIRE(done || !require_convergence, 8, "heev_jacobi: sweep cap reached without convergence");
  diag_rank_kernel<T><<<ceil_div(k, 128), 128, 0, st>>>(k, G, ldg, w, iwork);
  CHASE_CHECK_LAUNCH();
  permute_cols<T>(st, k, k, Zu, k, Z, ldz, iwork);
  return sweeps;
}

// ---------------------------------------------------------------- block Jacobi (FP32 first pass)
// Two-sided block Jacobi: the indices are cut into blocks of BJ_B; a round-robin tournament over the
// blocks pairs them, and each round reduces every pair's 2 BJ_B x 2 BJ_B principal submatrix
// S = G[IJ, IJ] in shared memory (one sweep of parallel cyclic Jacobi, one CTA per pair, accumulating the
// rotations in U), then applies U to the whole matrix: G[:, IJ] <- G[:, IJ] U and Z[:, IJ] <- Z[:, IJ] U,
// then G[IJ, :] <- U^H G[IJ, :].
// A sweep has (blocks - 1) rounds instead of the scalar method's (k - 1), each doing dense
// (k x 64) x (64 x 64) updates, so the round count (and its launch and synchronisation cost) falls by
// the block width while the arithmetic per sweep stays 4 k^3 multiply-adds.
constexpr int BJ_B = 32;          // block width
constexpr int BJ_M = 2 * BJ_B;    // subproblem order
constexpr int BJ_LD = BJ_M + 1;   // padded shared-memory row length
constexpr int BJ_SOLVE_THREADS = 1024;
constexpr int BJ_UPD_THREADS = 256;
constexpr int BJ_TILE = 64;       // rows (columns) of G or Z per update CTA

// global index of local index l of block pair (I, J)
__device__ __forceinline__ int bj_global(int I, int J, int l) {
  return l < BJ_B ? I * BJ_B + l : J * BJ_B + (l - BJ_B);
}

// realness of a diagonal entry without a round trip through double
__device__ __forceinline__ void bj_real(float& a) {}
__device__ __forceinline__ void bj_real(float2& a) { a.y = 0.0f; }

template <typename F>
__global__ void __launch_bounds__(BJ_SOLVE_THREADS) bj_solve_kernel(int k, int nbp, int r, const F* G, int64_t ldg,
                                                                     F* Ubuf, int inner_sweeps) {
  using s = S<F>;
  extern __shared__ __align__(16) unsigned char bj_smem[];
  F* Sm = reinterpret_cast<F*>(bj_smem);  // S[l][m] at Sm[l * BJ_LD + m]
  F* Um = Sm + BJ_M * BJ_LD;              // U[l][m] at Um[l * BJ_LD + m]
  __shared__ F rself[BJ_M], rother[BJ_M];
  const int nb = (k + BJ_B - 1) / BJ_B;
  int I, J;
  round_pair(r, blockIdx.x, nbp, I, J);
  if (I >= nb || J >= nb) return;  // paired with the padding block: nothing to do this round
  const int tid = threadIdx.x;
  for (int e = tid; e < BJ_M * BJ_M; e += blockDim.x) {
    const int l = e % BJ_M, m = e / BJ_M;
    const int gl = bj_global(I, J, l), gm = bj_global(I, J, m);
    Sm[l * BJ_LD + m] = (gl < k && gm < k) ? G[gl + (int64_t)gm * ldg] : s::zero();
    Um[l * BJ_LD + m] = (l == m) ? s::one() : s::zero();
  }
  __syncthreads();
  for (int sw = 0; sw < inner_sweeps; ++sw) {
    for (int rr = 0; rr < BJ_M - 1; ++rr) {
      if (tid < BJ_M / 2) {
        int a, b;
        round_pair(rr, tid, BJ_M, a, b);
        const int p = min(a, b), q = max(a, b);
        const bool valid = bj_global(I, J, q) < k && bj_global(I, J, p) < k;
        const F g = Sm[p * BJ_LD + q];
        // parameters in FP64 (32 threads, a few operations per round): FP32 parameters raise the pass's
        // rounding floor above what the FP64 corrections that follow can absorb for close eigenvalues
        const double ag = sqrt(s::abs2(g));
        const double app = s::re(Sm[p * BJ_LD + p]), aqq = s::re(Sm[q * BJ_LD + q]);
        if (!valid || !(ag > 1e-30)) {
          rself[p] = s::one();
          rother[p] = s::zero();
          rself[q] = s::one();
          rother[q] = s::zero();
        } else {
          const double z = (aqq - app) / (2.0 * ag);
          const double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
          const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
          const F ph = s::scale(s::conj(g), 1.0 / ag);  // conj(g)/|g|
          // J = [[c, sn], [-sn ph, c ph]] on (p, q): J[p][p], J[q][p] for p; J[q][q], J[p][q] for q
          rself[p] = s::make(c, 0.0);
          rother[p] = s::scale(ph, -sn);
          rself[q] = s::scale(ph, c);
          rother[q] = s::make(sn, 0.0);
        }
      }
      __syncthreads();
      // S <- J^H S J on every (row pair, column pair) 2x2 block, U <- U J; each item owns its entries
      for (int it = tid; it < (BJ_M / 2) * (BJ_M / 2); it += blockDim.x) {
        const int i1 = it % (BJ_M / 2), i2 = it / (BJ_M / 2);
        int rows[2], cols[2];
        round_pair(rr, i1, BJ_M, rows[0], rows[1]);
        round_pair(rr, i2, BJ_M, cols[0], cols[1]);
        F in[2][2], cu[2][2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) in[u][v] = Sm[rows[u] * BJ_LD + cols[v]];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v)
            cu[u][v] = s::add(s::mul(in[u][v], rself[cols[v]]), s::mul(in[u][1 - v], rother[cols[v]]));
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            F o = s::add(s::mul(s::conj(rself[rows[u]]), cu[u][v]), s::mul(s::conj(rother[rows[u]]), cu[1 - u][v]));
            if (rows[u] == cols[v]) bj_real(o);
            if (i1 == i2 && u != v) o = s::zero();
            Sm[rows[u] * BJ_LD + cols[v]] = o;
          }
      }
      for (int it = tid; it < BJ_M * (BJ_M / 2); it += blockDim.x) {
        const int i = it % BJ_M, pi = it / BJ_M;
        int a, b;
        round_pair(rr, pi, BJ_M, a, b);
        const F ua = Um[i * BJ_LD + a], ub = Um[i * BJ_LD + b];
        Um[i * BJ_LD + a] = s::add(s::mul(ua, rself[a]), s::mul(ub, rother[a]));
        Um[i * BJ_LD + b] = s::add(s::mul(ub, rself[b]), s::mul(ua, rother[b]));
      }
      __syncthreads();
    }
  }
  F* U = Ubuf + (int64_t)blockIdx.x * BJ_M * BJ_M;
  for (int e = tid; e < BJ_M * BJ_M; e += blockDim.x) {
    const int l = e % BJ_M, m = e / BJ_M;
    U[l + m * BJ_M] = Um[l * BJ_LD + m];
  }
}

// X[:, IJ] <- X[:, IJ] U for a tile of BJ_TILE rows (X = G for blockIdx.z == 0, Z for 1)
template <typename F>
__global__ void __launch_bounds__(BJ_UPD_THREADS) bj_cols_kernel(int k, int nbp, int r, F* G, int64_t ldg, F* Z,
                                                                  int64_t ldz, const F* __restrict__ Ubuf) {
  using s = S<F>;
  extern __shared__ __align__(16) unsigned char bj_smem[];
  F* Us = reinterpret_cast<F*>(bj_smem);   // BJ_M x BJ_LD
  F* Xs = Us + BJ_M * BJ_LD;               // BJ_TILE x BJ_LD
  const int nb = (k + BJ_B - 1) / BJ_B;
  int I, J;
  round_pair(r, blockIdx.y, nbp, I, J);
  if (I >= nb || J >= nb) return;
  F* X = blockIdx.z == 0 ? G : Z;
  const int64_t ldx = blockIdx.z == 0 ? ldg : ldz;
  const int r0 = blockIdx.x * BJ_TILE;
  const F* U = Ubuf + (int64_t)blockIdx.y * BJ_M * BJ_M;
  const int tid = threadIdx.x;
  for (int e = tid; e < BJ_M * BJ_M; e += blockDim.x) Us[(e % BJ_M) * BJ_LD + e / BJ_M] = U[e];
  for (int e = tid; e < BJ_TILE * BJ_M; e += blockDim.x) {
    const int i = e % BJ_TILE, l = e / BJ_TILE;
    const int gi = r0 + i, gl = bj_global(I, J, l);
    Xs[i * BJ_LD + l] = (gi < k && gl < k) ? X[gi + (int64_t)gl * ldx] : s::zero();
  }
  __syncthreads();
  // thread: one row, BJ_M / 4 columns (c = cq + 4 j)
  const int i = tid % BJ_TILE, cq = tid / BJ_TILE;
  F acc[BJ_M / 4];
#pragma unroll
  for (int j = 0; j < BJ_M / 4; ++j) acc[j] = s::zero();
  for (int m = 0; m < BJ_M; ++m) {
    const F xv = Xs[i * BJ_LD + m];
#pragma unroll
    for (int j = 0; j < BJ_M / 4; ++j) acc[j] = s::fma(xv, Us[m * BJ_LD + cq + 4 * j], acc[j]);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < BJ_M / 4; ++j) Xs[i * BJ_LD + cq + 4 * j] = acc[j];
  __syncthreads();
  for (int e = tid; e < BJ_TILE * BJ_M; e += blockDim.x) {
    const int ii = e % BJ_TILE, l = e / BJ_TILE;
    const int gi = r0 + ii, gl = bj_global(I, J, l);
    if (gi < k && gl < k) X[gi + (int64_t)gl * ldx] = Xs[ii * BJ_LD + l];
  }
}

// G[IJ, :] <- U^H G[IJ, :] for a tile of BJ_TILE columns
template <typename F>
__global__ void __launch_bounds__(BJ_UPD_THREADS) bj_rows_kernel(int k, int nbp, int r, F* G, int64_t ldg,
                                                                  const F* __restrict__ Ubuf) {
  using s = S<F>;
  extern __shared__ __align__(16) unsigned char bj_smem[];
  F* Us = reinterpret_cast<F*>(bj_smem);   // BJ_M x BJ_LD
  F* Xs = Us + BJ_M * BJ_LD;               // Xs[l][j]: row l of the pair, column c0 + j (BJ_M x BJ_LD)
  const int nb = (k + BJ_B - 1) / BJ_B;
  int I, J;
  round_pair(r, blockIdx.y, nbp, I, J);
  if (I >= nb || J >= nb) return;
  const int c0 = blockIdx.x * BJ_TILE;
  const F* U = Ubuf + (int64_t)blockIdx.y * BJ_M * BJ_M;
  const int tid = threadIdx.x;
  for (int e = tid; e < BJ_M * BJ_M; e += blockDim.x) Us[(e % BJ_M) * BJ_LD + e / BJ_M] = U[e];
  for (int e = tid; e < BJ_M * BJ_TILE; e += blockDim.x) {
    const int l = e % BJ_M, j = e / BJ_M;
    const int gl = bj_global(I, J, l), gj = c0 + j;
    Xs[l * BJ_LD + j] = (gl < k && gj < k) ? G[gl + (int64_t)gj * ldg] : s::zero();
  }
  __syncthreads();
  // thread: one column j, BJ_M / 4 rows (l = lq + 4 q); out[l][j] = sum_m conj(U[m][l]) X[m][j]
  const int j = tid % BJ_TILE, lq = tid / BJ_TILE;
  F acc[BJ_M / 4];
#pragma unroll
  for (int q = 0; q < BJ_M / 4; ++q) acc[q] = s::zero();
  for (int m = 0; m < BJ_M; ++m) {
    const F xv = Xs[m * BJ_LD + j];
#pragma unroll
    for (int q = 0; q < BJ_M / 4; ++q) acc[q] = s::fma(s::conj(Us[m * BJ_LD + lq + 4 * q]), xv, acc[q]);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < BJ_M / 4; ++q) Xs[(lq + 4 * q) * BJ_LD + j] = acc[q];
  __syncthreads();
  for (int e = tid; e < BJ_M * BJ_TILE; e += blockDim.x) {
    const int l = e % BJ_M, jj = e / BJ_M;
    const int gl = bj_global(I, J, l), gj = c0 + jj;
    if (gl < k && gj < k) G[gl + (int64_t)gj * ldg] = Xs[l * BJ_LD + jj];
  }
}

template <typename F> static size_t bj_smem_bytes() { return (size_t)2 * BJ_M * BJ_LD * sizeof(F); }

int heev_block_workspace(int k) {
  const int nb = (k + BJ_B - 1) / BJ_B;
  const int nbp = nb + (nb & 1);
  return nbp / 2 * BJ_M * BJ_M;
}

template <typename F>
int heev_block_jacobi(cudaStream_t st, int k, F* G, int64_t ldg, double* w, F* Z, int64_t ldz, F* work,
                      int64_t work_elems, double* dwork, int* iwork, double tol, int max_sweeps) {
  const int nb = (k + BJ_B - 1) / BJ_B;
  const int nbp = nb + (nb & 1);
  const int npairs = nbp / 2;
  CHASE_REQUIRE(k >= 1 && work_elems >= (int64_t)k * k + heev_block_workspace(k), 2,
                "heev_block_jacobi: workspace too small");
  F* Zu = work;
  F* Ubuf = work + (int64_t)k * k;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, []() {
    const int b = (int)bj_smem_bytes<F>();
    attr = cudaFuncSetAttribute(bj_solve_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (attr == cudaSuccess) attr = cudaFuncSetAttribute(bj_cols_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (attr == cudaSuccess) attr = cudaFuncSetAttribute(bj_rows_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  });
  CHASE_CUDA(attr);
  set_identity_kernel<F><<<dim3(ceil_div(k, 256), k), 256, 0, st>>>(k, Zu, k);
  CHASE_CHECK_LAUNCH();
  double* part = dwork + 2;
  double hstat[2];
  double prev_off = 0.0;
  int sweeps = 0;
  const int tiles = ceil_div(k, BJ_TILE);
  for (; sweeps <= max_sweeps; ++sweeps) {
    offdiag_partial_kernel<F><<<k, 128, 0, st>>>(k, G, ldg, part);
    CHASE_CHECK_LAUNCH();
    offdiag_sum_kernel<<<1, 32, 0, st>>>(k, part, dwork);
    CHASE_CHECK_LAUNCH();
    CHASE_CUDA(cudaMemcpyAsync(hstat, dwork, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CHASE_CUDA(cudaStreamSynchronize(st));
    CHASE_REQUIRE(isfinite(hstat[0]) && isfinite(hstat[1]), 5, "heev_block_jacobi: non-finite matrix");
    if (sqrt(hstat[0]) <= tol * sqrt(hstat[1]) || k == 1 || sweeps == max_sweeps) break;
    // FP32 floor: the 64-term updates leave off-diagonal rounding that can exceed tol for large k; once a sweep
    // no longer quarters the off-diagonal norm below 1e-5 relative, the FP64 refinement takes over.  Its
    // first-order corrections converge quadratically in (off-diagonal / gap): 1e-5 keeps that ratio near 0.05
    // for relative gaps of 2e-4 (the Table 2 Geometric spectrum), where three corrections reach FP64 level
    if (sweeps >= 2 && hstat[0] > 0.0625 * prev_off && sqrt(hstat[0]) <= 1e-5 * sqrt(hstat[1])) break;
    prev_off = hstat[0];
    for (int r = 0; r < nbp - 1; ++r) {
      bj_solve_kernel<F><<<npairs, BJ_SOLVE_THREADS, bj_smem_bytes<F>(), st>>>(k, nbp, r, G, ldg, Ubuf, 1);
      CHASE_CHECK_LAUNCH();
      bj_cols_kernel<F><<<dim3(tiles, npairs, 2), BJ_UPD_THREADS, bj_smem_bytes<F>(), st>>>(k, nbp, r, G, ldg, Zu, k,
                                                                                          Ubuf);
      CHASE_CHECK_LAUNCH();
      bj_rows_kernel<F><<<dim3(tiles, npairs), BJ_UPD_THREADS, bj_smem_bytes<F>(), st>>>(k, nbp, r, G, ldg, Ubuf);
      CHASE_CHECK_LAUNCH();
    }
  }
  diag_rank_kernel<F><<<ceil_div(k, 128), 128, 0, st>>>(k, G, ldg, w, iwork);
  CHASE_CHECK_LAUNCH();
  permute_cols<F>(st, k, k, Zu, k, Z, ldz, iwork);
  return sweeps;
}

template int heev_block_jacobi<float>(cudaStream_t, int, float*, int64_t, double*, float*, int64_t, float*, int64_t,
                                      double*, int*, double, int);
template int heev_block_jacobi<float2>(cudaStream_t, int, float2*, int64_t, double*, float2*, int64_t, float2*,
                                       int64_t, double*, int*, double, int);

template int heev_jacobi<double>(cudaStream_t, int, double*, int64_t, double*, double*, int64_t, double*, int64_t,
                                 double*, int*, double, int, bool, bool);
template int heev_jacobi<double2>(cudaStream_t, int, double2*, int64_t, double*, double2*, int64_t, double2*, int64_t,
                                  double*, int*, double, int, bool, bool);
template int heev_jacobi<float>(cudaStream_t, int, float*, int64_t, double*, float*, int64_t, float*, int64_t, double*,
                                int*, double, int, bool, bool);
template int heev_jacobi<float2>(cudaStream_t, int, float2*, int64_t, double*, float2*, int64_t, float2*, int64_t,
                                 double*, int*, double, int, bool, bool);

}  // namespace chase
