// Split-BF16 products, host side and digit planes: the per-row / per-column power-of-two scales and the
// digit-plane split kernels of the operands, the workspace, the launch-configuration tuner, the K-split
// planning and the dispatch of products (single, grouped) to the tcgen05 kernel of oz_kernel.cuh, whose
// instantiations live in the oz_inst_*.cu units.  The digit arithmetic, the exact-level accumulation and
// the kernel's roles are described in oz_kernel.cuh.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "oz.h"
#include "oz_kernel.cuh"

namespace chase {
namespace oz {
// ---------------------------------------------------------------- split kernels
// Per-column power-of-two scale s = 2^e with max|re|,|im| = f 2^e, f in [0.5, 1).
template <typename T>
__global__ void col_scale_kernel(int64_t K, const T* __restrict__ X, int64_t ldx, double* scale) {
  const T* x = X + (int64_t)blockIdx.x * ldx;
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < K; i += blockDim.x) {
    T v = x[i];
    m = fmax(m, fmax(fabs(S<T>::re(v)), fabs(S<T>::im(v))));
  }
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmax(v, red[w]);
    int e = 0;
    if (v > 0.0 && isfinite(v)) frexp(v, &e);
    scale[blockIdx.x] = v > 0.0 ? ldexp(1.0, e) : 1.0;
  }
}

// Digits of one value: d_t = rint(r_t), r_0 = x/s * 2^7, r_{t+1} = (r_t - d_t) 2^8; plane stores d_t 2^-8t.
template <int NS> __device__ __forceinline__ void digits(double xs, __nv_bfloat16 (&out)[NS]) {
  double r = xs * 128.0;
  float sc = 1.0f;
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    double d = rint(r);
    out[t] = __float2bfloat16_rn((float)d * sc);
    r = (r - d) * 256.0;
    sc *= 0.00390625f;
  }
}

// Left-operand planes (K-major rows = conjugated columns of X when conj, else columns):
// plane (t, p), p in {re, im}.  Right-operand planes: p in {-im, re, im}.
// Real: one plane per slice.  Layout planes[(t*P + p) * ncols + col][Kpad].
template <typename T, int NS, int KIND>
__global__ void split_cols_kernel(int64_t K, int64_t Kpad, int ncols, const T* __restrict__ X, int64_t ldx,
                                  const double* __restrict__ scale, int conj, __nv_bfloat16* planes) {
  constexpr bool CPLX = S<T>::cplx;
  const int col = blockIdx.y;
  const T* x = X + (int64_t)col * ldx;
  const double inv = 1.0 / scale[col];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
    T v = x[i];
    double re = S<T>::re(v) * inv;
    double im = (conj ? -S<T>::im(v) : S<T>::im(v)) * inv;
    __nv_bfloat16 dr[NS], di[NS];
    digits<NS>(re, dr);
    if (CPLX) digits<NS>(im, di);
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      if (!CPLX) {
        planes[((int64_t)t * ncols + col) * Kpad + i] = dr[t];
      } else if (KIND == 0) {
        planes[((int64_t)(t * 2 + 0) * ncols + col) * Kpad + i] = dr[t];
        planes[((int64_t)(t * 2 + 1) * ncols + col) * Kpad + i] = di[t];
      } else {
        planes[((int64_t)(t * 3 + 0) * ncols + col) * Kpad + i] = __hneg(di[t]);
        planes[((int64_t)(t * 3 + 1) * ncols + col) * Kpad + i] = dr[t];
        planes[((int64_t)(t * 3 + 2) * ncols + col) * Kpad + i] = di[t];
      }
    }
  }
}

// Per-row power-of-two scale of a column-major X (vector i = row i, K along columns).
template <typename T>
__global__ void row_scale_kernel(int64_t nvec, int64_t K, const T* __restrict__ X, int64_t ldx, double* scale) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvec) return;
  double m = 0.0;
  for (int64_t kk = 0; kk < K; ++kk) {
    T v = X[i + kk * ldx];
    m = fmax(m, fmax(fabs(S<T>::re(v)), fabs(S<T>::im(v))));
  }
  int e = 0;
  if (m > 0.0 && isfinite(m)) frexp(m, &e);
  scale[i] = m > 0.0 ? ldexp(1.0, e) : 1.0;
}

// Planes of the vectors i = rows of X (K along columns), via a 32x32 shared-memory transpose.
template <typename T, int NS, int KIND>
__global__ void split_rows_kernel(int64_t nvec, int64_t K, int64_t Kpad, const T* __restrict__ X, int64_t ldx,
                                  const double* __restrict__ scale, int conj, __nv_bfloat16* planes) {
  constexpr bool CPLX = S<T>::cplx;
  __shared__ T tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int64_t kk = k0 + r, i = i0 + threadIdx.x;
    tile[r][threadIdx.x] = (kk < K && i < nvec) ? X[i + kk * ldx] : S<T>::zero();
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int64_t i = i0 + r, kk = k0 + threadIdx.x;
    if (i >= nvec || kk >= K) continue;
    T v = tile[threadIdx.x][r];
    const double inv = 1.0 / scale[i];
    double re = S<T>::re(v) * inv;
    double im = (conj ? -S<T>::im(v) : S<T>::im(v)) * inv;
    __nv_bfloat16 dr[NS], di[NS];
    digits<NS>(re, dr);
    if (CPLX) digits<NS>(im, di);
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      if (!CPLX) {
        planes[((int64_t)t * nvec + i) * Kpad + kk] = dr[t];
      } else if (KIND == 0) {
        planes[((int64_t)(t * 2 + 0) * nvec + i) * Kpad + kk] = dr[t];
        planes[((int64_t)(t * 2 + 1) * nvec + i) * Kpad + kk] = di[t];
      } else {
        planes[((int64_t)(t * 3 + 0) * nvec + i) * Kpad + kk] = __hneg(di[t]);
        planes[((int64_t)(t * 3 + 1) * nvec + i) * Kpad + kk] = dr[t];
        planes[((int64_t)(t * 3 + 2) * nvec + i) * Kpad + kk] = di[t];
      }
    }
  }
}

// ---------------------------------------------------------------- host side
static int slices_for(int mode, int fp64_slices) {
  if (mode == 2) return 2;   // BF16x3
  if (mode == 3) return 3;   // BF16x6
  return fp64_slices;        // FP64
}


bool available() {
  // thread-safe one-time probe (batched solves call this from several host threads)
  static const bool ok = []() {
    int dev = 0, major = 0, minor = 0;
    return cudaGetDevice(&dev) == cudaSuccess &&
           cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) == cudaSuccess &&
           cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) == cudaSuccess && major == 10 &&
           minor == 3 && encode_fn() != nullptr;
  }();
  return ok;
}

static int64_t left_elems(int64_t n_max, int ne_max) {
  return std::max<int64_t>(n_max * kpad(ne_max), (int64_t)ne_max * kpad(n_max));
}

int64_t workspace_bytes(int64_t n_max, int ne_max, bool complex_, int slices) {
  int ap = complex_ ? 2 : 1, bp = complex_ ? 3 : 1;
  int64_t kp = kpad(n_max);
  int64_t a = (int64_t)slices * ap * n_max * kp * 2;
  int64_t l = (int64_t)slices * ap * left_elems(n_max, ne_max) * 2;
  int64_t b = (int64_t)slices * bp * ne_max * kp * 2;
  return a + l + b + (2 * n_max + 2 * ne_max) * 8 + 64 + (8ll << 20) * 8;
}

void create(Workspace& w, int64_t n_max, int ne_max, bool complex_, int slices) {
  w.n_max = n_max;
  w.ne_max = ne_max;
  w.complex_ = complex_;
  w.slices = slices;
  if (!available()) return;
  int ap = complex_ ? 2 : 1, bp = complex_ ? 3 : 1;
  int64_t kp = kpad(n_max);
  CHASE_CUDA(cudaMalloc(&w.a_planes, (size_t)slices * ap * n_max * kp * 2));
  CHASE_CUDA(cudaMalloc(&w.l_planes, (size_t)slices * ap * left_elems(n_max, ne_max) * 2));
  CHASE_CUDA(cudaMalloc(&w.b_planes, (size_t)slices * bp * ne_max * kp * 2));
  CHASE_CUDA(cudaMalloc(&w.a_scale, n_max * sizeof(double)));
  CHASE_CUDA(cudaMalloc(&w.l_scale, std::max<int64_t>(n_max, ne_max) * sizeof(double)));
  CHASE_CUDA(cudaMalloc(&w.b_scale, ne_max * sizeof(double)));
  CHASE_CUDA(cudaMalloc(&w.flags, 16 * sizeof(int)));
  CHASE_CUDA(cudaMemset(w.flags, 0, 16 * sizeof(int)));
  // partial sums of K-split products: up to about 4 waves of 128 x 40 complex tiles
  w.partial_elems = 8ll << 20;
  CHASE_CUDA(cudaMalloc(&w.partial, (size_t)w.partial_elems * sizeof(double)));
  w.ready = true;
}

void destroy(Workspace& w) {
  void* ps[] = {w.a_planes, w.l_planes, w.b_planes, w.a_scale, w.l_scale, w.b_scale, w.flags, w.partial};
  for (void* p : ps)
    if (p) cudaFree(p);
  for (auto& e : w.ev) cudaEventDestroy(e);
  for (auto& kv : w.tune)
    for (auto& e : kv.second.ev)
      if (e) cudaEventDestroy(e);
  w = Workspace{};
}

// Split nvec vectors of length K taken from a column-major X: by columns (vector = column,
// optionally conjugated) or by rows (vector = row).  kind 0: left-operand planes (re, im);
// kind 1: right-operand planes (-im, re, im).
template <typename T>
static void split(cudaStream_t st, int S_, int kind, bool by_rows, bool conj, const T* X, int64_t ld, int64_t nvec,
                  int64_t K, void* planes, double* scale) {
  const int64_t kp = kpad(K);
  if (!by_rows) {
    col_scale_kernel<T><<<(unsigned)nvec, 256, 0, st>>>(K, X, ld, scale);
    CHASE_CHECK_LAUNCH();
    dim3 grid(std::min<unsigned>(ceil_div(K, 256), 32), (unsigned)nvec);
#define SC(SS, KD) split_cols_kernel<T, SS, KD><<<grid, 256, 0, st>>>(K, kp, (int)nvec, X, ld, scale, conj ? 1 : 0, (__nv_bfloat16*)planes)
#define SWK(SS) if (kind == 0) SC(SS, 0); else SC(SS, 1);
    switch (S_) {
      case 2: SWK(2); break;
      case 3: SWK(3); break;
      case 6: SWK(6); break;
      case 7: SWK(7); break;
      default: CHASE_REQUIRE(false, 1, "unsupported slice count");
    }
#undef SWK
#undef SC
  } else {
    row_scale_kernel<T><<<ceil_div(nvec, 128), 128, 0, st>>>(nvec, K, X, ld, scale);
    CHASE_CHECK_LAUNCH();
    dim3 grid(ceil_div(K, 32), ceil_div(nvec, 32));
    CHASE_REQUIRE(grid.y <= 65535, 1, "split: too many vectors");
#define SR(SS, KD) split_rows_kernel<T, SS, KD><<<grid, dim3(32, 8), 0, st>>>(nvec, K, kp, X, ld, scale, conj ? 1 : 0, (__nv_bfloat16*)planes)
#define SWK(SS) if (kind == 0) SR(SS, 0); else SR(SS, 1);
    switch (S_) {
      case 2: SWK(2); break;
      case 3: SWK(3); break;
      case 6: SWK(6); break;
      case 7: SWK(7); break;
      default: CHASE_REQUIRE(false, 1, "unsupported slice count");
    }
#undef SWK
#undef SR
  }
  CHASE_CHECK_LAUNCH();
}

template <typename T>
void prepare_A(cudaStream_t st, Workspace& w, const T* A, int64_t n, int64_t lda, int mode) {
  CHASE_REQUIRE(w.ready, 9, "split products not initialised");
  // planes of all slices are nested: the S-slice split's first slices are the 2- and 3-slice splits
  if (w.a_src == (const void*)A && w.a_n == n && w.a_mode == w.slices) return;
  (void)mode;
  // A Hermitian: K-major row i of A = conjugate of column i of its column-major storage
  split<T>(st, w.slices, 0, false, true, A, lda, n, n, w.a_planes, w.a_scale);
  w.a_src = A;
  w.a_n = n;
  w.a_mode = w.slices;
}

void timing_begin(Workspace& w) {
  if (w.ev.empty()) {
    w.ev.resize(256);
    for (auto& e : w.ev) CHASE_CUDA(cudaEventCreate(&e));
  }
  w.ev_used = 0;
  w.timing = true;
}

double timing_collect(Workspace& w, int* launches) {
  double ms = 0.0;
  for (int i = 0; i + 1 < w.ev_used; i += 2) {
    CHASE_CUDA(cudaEventSynchronize(w.ev[i + 1]));
    float t = 0.f;
    CHASE_CUDA(cudaEventElapsedTime(&t, w.ev[i], w.ev[i + 1]));
    ms += t;
  }
  if (launches) *launches = w.ev_used / 2;
  w.ev_used = 0;
  w.timing = false;
  return ms;
}

void invalidate(Workspace& w) {
  w.a_src = nullptr;
  w.a_n = 0;
  w.a_mode = -1;
  if (w.flags) CHASE_CUDA(cudaMemset(w.flags, 0, 16 * sizeof(int)));  // a new call starts clean
}

// C(M x N) = L(M x K) R(K x N) from digit planes (left: rows = M vectors of length K, right:
// rows = N vectors of length K), split with l_slices_total / S slices respectively.
// ---------------------------------------------------------------- launch-configuration tuner
// Candidates per arithmetic: the FP64 kernels (NT fixed at 80 by TMEM) try the tile-order group sizes;
// the mixed kernels (one accumulator) also try the 256-column tile, which halves the instructions per
// unit of tensor work.
static const LaunchCfg kCandFP64[] = {{0, 2}, {0, 4}, {0, 8}, {0, 16}, {0, 32}};
static const LaunchCfg kCandMixed[] = {{128, 4}, {128, 16}, {256, 4}, {256, 16}};

static int log2_bucket(int64_t x) {
  int b = 0;
  while (x > 1) {
    x >>= 1;
    ++b;
  }
  return b;
}

// Size class of a launch: arithmetic, element type, grouped or not, and the log2 buckets of the shape.
static uint64_t tune_key(int S_, bool cplx, bool grouped, int64_t M, int64_t N, int64_t K) {
  return ((uint64_t)S_ << 56) | ((uint64_t)cplx << 55) | ((uint64_t)grouped << 54) |
         ((uint64_t)log2_bucket(M) << 36) | ((uint64_t)log2_bucket(N) << 18) | (uint64_t)log2_bucket(K);
}

// The configuration for the next launch of a size class.  Until every candidate has been timed, each
// launch takes the next candidate and gets an event pair (*ev_out); the first launch after that reads
// the times (one event synchronisation per size class and context) and keeps the fastest.
static LaunchCfg tune_pick(Workspace& w, uint64_t key, bool mixed, cudaEvent_t** ev_out) {
  const LaunchCfg* cand = mixed ? kCandMixed : kCandFP64;
  const int nc = mixed ? (int)(sizeof(kCandMixed) / sizeof(kCandMixed[0]))
                       : (int)(sizeof(kCandFP64) / sizeof(kCandFP64[0]));
  *ev_out = nullptr;
  if (!w.autotune) {
    LaunchCfg d = mixed ? LaunchCfg{128, w.group_m} : LaunchCfg{0, w.group_m};
    return d;
  }
  TuneEntry& t = w.tune[key];
  if (t.best >= 0) return cand[t.best];
  if (t.ev.empty()) {
    t.ev.resize(2 * nc, nullptr);
    for (auto& e : t.ev) CHASE_CUDA(cudaEventCreate(&e));
  }
  if (t.next < nc) {
    *ev_out = &t.ev[2 * t.next];
    return cand[t.next++];
  }
  float best_ms = 0.f;
  int best = 0;
  for (int i = 0; i < nc; ++i) {
    CHASE_CUDA(cudaEventSynchronize(t.ev[2 * i + 1]));
    float ms = 0.f;
    CHASE_CUDA(cudaEventElapsedTime(&ms, t.ev[2 * i], t.ev[2 * i + 1]));
    if (i == 0 || ms < best_ms) {
      best_ms = ms;
      best = i;
    }
  }
  t.best = best;
  return cand[best];
}

std::vector<std::pair<uint64_t, int>> tuned(const Workspace& w) {
  std::vector<std::pair<uint64_t, int>> out;
  for (const auto& kv : w.tune)
    if (kv.second.best >= 0) out.emplace_back(kv.first, kv.second.best);
  return out;
}

static int sm_count() {
  static const int n = []() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return 148;
    return sms;
  }();
  return n;
}

// A product with fewer output tiles than two per SM is split along K (slices of at least 384, multiples of
// 96, at most 16 of them, within the partial-sum buffer) so that its launch covers the GPU.
static void plan_ksplit(Workspace& w, ProductOp& op, int ncols_tile, bool cplx) {
  const int64_t tiles = (int64_t)ceil_div(op.N, ncols_tile) * (int64_t)ceil_div(op.M, BM);
  const int64_t want = 2 * (int64_t)sm_count();
  if (tiles >= want || op.K < 2 * 384 || !w.partial) return;
  int64_t ks = std::min<int64_t>({16, ceil_div(want, tiles), op.K / 384});
  const int64_t per = op.M * op.N * (cplx ? 2 : 1);
  ks = std::min<int64_t>(ks, w.partial_elems / std::max<int64_t>(1, per));
  if (ks <= 1) return;
  const int64_t klen = ((op.K + ks - 1) / ks + 95) / 96 * 96;
  op.klen = (int)klen;
  op.ksplit = (int)ceil_div(op.K, klen);
  op.part = w.partial;
  if (op.ksplit <= 1) {
    op.ksplit = 1;
    op.part = nullptr;
  }
}

template <int S, int NEX, bool CPLX, int NTT>
static void launch(cudaStream_t st, Workspace& w, const void* lpl, const double* lsc, int l_slices_total,
                   const void* rpl, const double* rsc, int64_t M, int64_t N, int64_t K, const Epi& e,
                   int group_m, cudaEvent_t* tune_ev) {
  ProductOp op{lpl, lsc, l_slices_total, rpl, rsc, M, N, K, e, group_m};
  plan_ksplit(w, op, Cfg<S, NEX, CPLX, NTT>::NCOLS, CPLX);
  launch_ops<S, NEX, CPLX, NTT, 1>(st, w, &op, 1, tune_ev);
}

template <bool CPLX>
static void dispatch(cudaStream_t st, Workspace& w, int S_, const void* lpl, const double* lsc, int l_slices_total,
                     int64_t M, int64_t N, int64_t K, const Epi& e) {
  CHASE_REQUIRE(K <= 65472, 1, "split products support K <= 65472 (int64 exact-level sums)");
  // a narrow right operand (up to 8 complex or 16 real columns: the Lanczos block) takes the N = 16 tile, so
  // the launch streams the left planes once without computing unused accumulator columns
  const bool narrow = N <= (CPLX ? 8 : 16);
  const void* rp = w.b_planes;
  const double* rs = w.b_scale;
  if (narrow && S_ >= 6) {
    // one column tile: the tile order is irrelevant
    if (S_ == 7) launch<7, 5, CPLX, 16>(st, w, lpl, lsc, l_slices_total, rp, rs, M, N, K, e, 1, nullptr);
    else launch<6, 5, CPLX, 16>(st, w, lpl, lsc, l_slices_total, rp, rs, M, N, K, e, 1, nullptr);
    return;
  }
  cudaEvent_t* ev = nullptr;
  const LaunchCfg cfg = tune_pick(w, tune_key(S_, CPLX, false, M, N, K), S_ <= 3, &ev);
  if (S_ == 7) launch<7, 5, CPLX, 80>(st, w, lpl, lsc, l_slices_total, rp, rs, M, N, K, e, cfg.group_m, ev);
  else if (S_ == 6) launch<6, 5, CPLX, 80>(st, w, lpl, lsc, l_slices_total, rp, rs, M, N, K, e, cfg.group_m, ev);
  else if (S_ == 3 && cfg.nt == 256) launch<3, 0, CPLX, 256>(st, w, lpl, lsc, l_slices_total, rp, rs, M, N, K, e, cfg.group_m, ev);
  else if (S_ == 3) launch<3, 0, CPLX, 128>(st, w, lpl, lsc, l_slices_total, rp, rs, M, N, K, e, cfg.group_m, ev);
  else if (cfg.nt == 256) launch<2, 0, CPLX, 256>(st, w, lpl, lsc, l_slices_total, rp, rs, M, N, K, e, cfg.group_m, ev);
  else launch<2, 0, CPLX, 128>(st, w, lpl, lsc, l_slices_total, rp, rs, M, N, K, e, cfg.group_m, ev);
}

template <typename T>
void split_right(cudaStream_t st, Workspace& w, int mode, const T* B, int64_t ldb, int k, int64_t n) {
  CHASE_REQUIRE(w.ready, 9, "split products not initialised");
  CHASE_REQUIRE(k <= w.ne_max && n <= w.n_max, 1, "split_right: size exceeds the workspace");
  split<T>(st, slices_for(mode, w.slices), 1, false, false, B, ldb, k, n, w.b_planes, w.b_scale);
}

template <bool CPLX>
void launch_group(cudaStream_t st, Workspace& w, int mode, const ProductOp* ops, int nops) {
  constexpr int G = 64;
  const int S_ = slices_for(mode, w.slices);
  std::vector<ProductOp> chunk;
  for (int q0 = 0; q0 < nops; q0 += G) {
    const int cnt = std::min(G, nops - q0);
    // size class of a grouped launch: its total work in row blocks x columns x K
    int64_t rows = 0, cols = 0, kk = 0;
    for (int q = q0; q < q0 + cnt; ++q) {
      CHASE_REQUIRE(ops[q].K <= 65472, 1, "split products support K <= 65472 (int64 exact-level sums)");
      rows += ops[q].M;
      cols = std::max(cols, ops[q].N);
      kk = std::max(kk, ops[q].K);
    }
    cudaEvent_t* ev = nullptr;
    const LaunchCfg cfg = tune_pick(w, tune_key(S_, CPLX, true, rows, cols, kk), S_ <= 3, &ev);
    chunk.assign(ops + q0, ops + q0 + cnt);
    for (auto& o : chunk) o.group_m = cfg.group_m;
    const ProductOp* cp = chunk.data();
    if (S_ == 7) launch_ops<7, 5, CPLX, 80, G>(st, w, cp, cnt, ev);
    else if (S_ == 6) launch_ops<6, 5, CPLX, 80, G>(st, w, cp, cnt, ev);
    else if (S_ == 3 && cfg.nt == 256) launch_ops<3, 0, CPLX, 256, G>(st, w, cp, cnt, ev);
    else if (S_ == 3) launch_ops<3, 0, CPLX, 128, G>(st, w, cp, cnt, ev);
    else if (cfg.nt == 256) launch_ops<2, 0, CPLX, 256, G>(st, w, cp, cnt, ev);
    else launch_ops<2, 0, CPLX, 128, G>(st, w, cp, cnt, ev);
  }
}

template <typename T>
void hemm(cudaStream_t st, Workspace& w, const T* A, int64_t n, int64_t lda, const T* B, int64_t ldb, int k,
          const Epi& e, int mode) {
  CHASE_REQUIRE(w.ready, 9, "split products not initialised");
  CHASE_REQUIRE(w.a_src == (const void*)A && w.a_n == n, 7, "prepare_A must precede hemm");
  CHASE_REQUIRE(k <= w.ne_max && n <= w.n_max, 1, "hemm size exceeds the workspace");
  const int S_ = slices_for(mode, w.slices);
  split<T>(st, S_, 1, false, false, B, ldb, k, n, w.b_planes, w.b_scale);
  dispatch<S<T>::cplx>(st, w, S_, w.a_planes, w.a_scale, w.slices, n, k, n, e);
}

template <typename T>
void gemm(cudaStream_t st, Workspace& w, Op opA, const T* A, int64_t lda, Op opB, const T* B, int64_t ldb, int64_t M,
          int64_t N, int64_t K, const Epi& e, int mode) {
  CHASE_REQUIRE(w.ready, 9, "split products not initialised");
  if (M <= 0 || N <= 0) return;
  CHASE_REQUIRE(N <= w.ne_max && M * kpad(K) <= left_elems(w.n_max, w.ne_max) && N * kpad(K) <= (int64_t)w.ne_max * kpad(w.n_max),
                1, "split product exceeds the workspace");
  const int S_ = slices_for(mode, w.slices);
  // left operand: OP_N rows of A (M x K), OP_C conjugated columns of A (K x M)
  split<T>(st, S_, 0, opA == OP_N, opA == OP_C, A, lda, M, K, w.l_planes, w.l_scale);
  // right operand: OP_N columns of B (K x N), OP_C conjugated rows of B (N x K)
  split<T>(st, S_, 1, opB == OP_C, opB == OP_C, B, ldb, N, K, w.b_planes, w.b_scale);
  dispatch<S<T>::cplx>(st, w, S_, w.l_planes, w.l_scale, S_, M, N, K, e);
}

int read_flags(cudaStream_t st, Workspace& w) {
  if (!w.ready) return 0;
  int f = 0;
  CHASE_CUDA(cudaMemcpyAsync(&f, w.flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  CHASE_CUDA(cudaStreamSynchronize(st));
  return f;
}

template void prepare_A<double>(cudaStream_t, Workspace&, const double*, int64_t, int64_t, int);
template void prepare_A<double2>(cudaStream_t, Workspace&, const double2*, int64_t, int64_t, int);
template void hemm<double>(cudaStream_t, Workspace&, const double*, int64_t, int64_t, const double*, int64_t, int,
                           const Epi&, int);
template void gemm<double>(cudaStream_t, Workspace&, Op, const double*, int64_t, Op, const double*, int64_t, int64_t,
                           int64_t, int64_t, const Epi&, int);
template void gemm<double2>(cudaStream_t, Workspace&, Op, const double2*, int64_t, Op, const double2*, int64_t, int64_t,
                            int64_t, int64_t, const Epi&, int);
template void hemm<double2>(cudaStream_t, Workspace&, const double2*, int64_t, int64_t, const double2*, int64_t, int,
                            const Epi&, int);
template void split_right<double>(cudaStream_t, Workspace&, int, const double*, int64_t, int, int64_t);
template void split_right<double2>(cudaStream_t, Workspace&, int, const double2*, int64_t, int, int64_t);
template void launch_group<false>(cudaStream_t, Workspace&, int, const ProductOp*, int);
template void launch_group<true>(cudaStream_t, Workspace&, int, const ProductOp*, int);

}  // namespace oz
}  // namespace chase
