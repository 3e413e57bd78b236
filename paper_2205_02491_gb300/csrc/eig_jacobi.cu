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

template int heev_jacobi<double>(cudaStream_t, int, double*, int64_t, double*, double*, int64_t, double*, int64_t,
                                 double*, int*, double, int, bool, bool);
template int heev_jacobi<double2>(cudaStream_t, int, double2*, int64_t, double*, double2*, int64_t, double2*, int64_t,
                                  double*, int*, double, int, bool, bool);
template int heev_jacobi<float>(cudaStream_t, int, float*, int64_t, double*, float*, int64_t, float*, int64_t, double*,
                                int*, double, int, bool, bool);
template int heev_jacobi<float2>(cudaStream_t, int, float2*, int64_t, double*, float2*, int64_t, float2*, int64_t,
                                 double*, int*, double, int, bool, bool);

}  // namespace chase
