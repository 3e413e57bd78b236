#pragma once
// Split-BF16 tensor-core products on sm_103a (tcgen05 + TMEM + TMA).
//
// Every FP64 operand is scaled by a power of two per row (left operand) or per
// column (right operand) to |x| <= 1 and split into S signed 8-bit digits,
// x = sum_t d_t 2^(-7-8t), d_t integer in [-128, 128].  Plane t stores
// d_t 2^(-8t) in bf16 (exact).  A product of plane t and plane u lands on level
// L = t + u with unit 2^(-8L); all products of one level share that grid, so a
// level's FP32 partial sum over a chunk of 96 K values is an exact integer
// (|sum| < 2^24: at most 10 products of magnitude <= 2^14 per K value).
//
//   FP64 mode (S = 7 by default, levels 0..6; S = 6 optional): levels 0..4
//   accumulate in their own TMEM accumulators (MMA N = 80) and are flushed
//   exactly every 96 K into one int64 register per output (units 2^-32, no
//   overflow for K <= 65472); the remaining levels share one FP32 accumulator over
//   the whole K.  Each tensor-core accumulation step truncates to about 24 bits
//   of the running sum (measured), so the error of a shared accumulator grows
//   with the number of steps times its magnitude; keeping five levels exact
//   leaves only terms below 2^-40 there.  The digits dropped after slice S-1 of each operand (and the
//   pairs beyond level S-1) leave a truncation below about 2^-8S relative to |row max| * |col max| per
//   product (S = 7: 2^-56, errors comparable to DFMA).
//   Mixed modes (S = 2: 3 products, S = 3: 6 products): one FP32 accumulator.
//
// Complex operands use real tiles: with B1 = [Yr | Yi] and B2 = [-Yi | Yr]
// (N = 2 x 40 columns in the FP64 modes, 2 x 64 or 2 x 128 in the mixed ones) one
// accumulator holds [Cr | Ci] = Ar B1 + Ai B2.  A is the Hermitian matrix of the eigenproblem, whose K-major
// rows are the conjugated columns of its column-major storage.
//
// Kernel roles (320 threads): warp 0 lane 0 issues TMA loads, warp 1 lane 0
// issues tcgen05.mma, warps 2..9 (2 groups of 4 warps covering the 4 TMEM lane
// quadrants, half of the accumulator columns each) run
// the exact-level flushes and the fused FP64 epilogue
//   C = alpha * acc + gamma * ycol[j] * Y + beta * Z.
// The MMA issuer's barrier checks and commits stall its MMA queue (a check costs
// about 200 cycles with the tensor pipe idle), so the FP64 kernels move the left
// slices in three groups per k-block (Cfg::GROUPED): 3 checks and 4 commits per
// 112 MMAs instead of one of each per slice.
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the CTA sets
// an error flag, drains its copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "oz.h"
#include "tcgen05.cuh"

namespace chase {
namespace oz {

constexpr int BM = 128;          // output rows per tile (TMEM lanes)
constexpr int BK = 32;           // K per k-block: 64 bytes of bf16 (64B swizzle atom)
constexpr int B_STAGES = 2;      // right-operand k-blocks (all slices)
constexpr int KB_PER_CHUNK = 3;  // exact levels flushed every 96 K
constexpr int NTHREADS = 320;   // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr int EPI_WARP0 = 2;
constexpr int EPI_WARPS = 8;
constexpr unsigned long long TIMEOUT_NS = 2000000000ull;

// NTT: accumulator width (MMA N).  80 for the FP64 modes (six accumulators share TMEM), 128 for the
// single-accumulator mixed modes, 16 for narrow right operands (a few columns: the Lanczos block).
template <int S, int NEX, bool CPLX, int NTT> struct Cfg {
  static constexpr int NT = NTT;
  static constexpr int AP = CPLX ? 2 : 1;          // left planes per slice (re, im)
  static constexpr int BP = CPLX ? 3 : 1;          // right planes per slice (-im, re, im)
  static constexpr int NCOLS = CPLX ? NT / 2 : NT; // output columns per tile
  static constexpr int BROWS = NCOLS;              // right-operand rows (N index) per plane box
  static constexpr int A_PLANE = BM * BK * 2;      // 8 KB
  static constexpr int A_SLOT = AP * A_PLANE;
  static constexpr int B_PLANE = BROWS * BK * 2;
  static constexpr int B_SLICE = BP * B_PLANE;
  static constexpr int B_BYTES = S * B_SLICE;                 // bytes landed per k-block
  static constexpr int B_STAGE = (B_BYTES + 1023) / 1024 * 1024;  // stage stride (1 KB aligned)
  static constexpr int SMEM_LIMIT = 232448 - 1024 - 256;
  static constexpr int A_FIT = (SMEM_LIMIT - B_STAGES * B_STAGE) / A_SLOT;
  // ring of left-operand slices (>= S): as deep as shared memory allows, at most 12 (the barrier area
  // holds 2 x 12 + 2 x B_STAGES + 3 mbarriers plus two words); narrow tiles, whose MMAs are short, need
  // the extra depth to keep the copies of the next k-block in flight
  static constexpr int A_SLOTS = A_FIT < 12 ? A_FIT : 12;
  // Grouped synchronisation (the FP64 kernels whose ring holds exactly one k-block, slot = processing index):
  // the first G0 slices in processing order (the smallest: 1 + 2 + 3 digit pairs for S = 7) travel with the
  // right operand on its barrier and are released together, so a k-block costs 1 + (S - G0) barrier checks
  // and 2 + (S - G0) commits instead of 1 + S and 1 + S.  Each barrier check of the issuing thread stalls the
  // MMA queue (measured: about 170 cycles), so fewer checks keep the tensor pipe fed.
  static constexpr bool GROUPED = (A_SLOTS == S) && (NEX > 0) && (S >= 6);
  static constexpr int G0 = GROUPED ? 3 : 0;
  // The later slices go in groups too (processing indices {3, 4} and {5, ..., S-1}): a group's slots are
  // loaded onto the barrier of its first slot and released together after its last slice.  A group's
  // refill is issued when its slots are released and needed one k-block later, after at least the
  // MMAs of the slices processed in between (60 or more), which covers the copy latency.  Without
  // grouping every slice is its own group.
  static constexpr int gfirst(int ti) { return !GROUPED ? ti : (ti < 3 ? 0 : (ti < 5 ? 3 : 5)); }
  static constexpr int glast(int ti) { return !GROUPED ? ti : (ti < 3 ? 2 : (ti < 5 ? 4 : S - 1)); }
  static constexpr int NACC = NEX + 1;
  static constexpr int TMEM_USED = NACC * NT;
  static constexpr int TMEM_COLS = TMEM_USED <= 128 ? 128 : (TMEM_USED <= 256 ? 256 : 512);
  static constexpr int EPI_COLS = NT / 2;          // accumulator columns per epilogue thread (2 groups)
  static constexpr int SMEM_OPS = B_STAGES * B_STAGE + A_SLOTS * A_SLOT;
  static constexpr int SMEM_BYTES = SMEM_OPS + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int MAXLEVEL = S - 1;
  static_assert(TMEM_USED <= 512, "TMEM");
  static_assert(SMEM_BYTES <= 232448, "shared memory");
  static_assert(A_SLOTS >= S, "a k-block's slices must fit in the ring");
  static_assert((2 * A_SLOTS + 2 * B_STAGES + 3) * 8 + 8 <= 256, "barrier area");
  static_assert(EPI_COLS % 8 == 0, "epilogue loads 8 columns at a time");
};

// ---------------------------------------------------------------- PTX helpers

// bounded wait: false on timeout or when another role aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_sh, int* err) {
  unsigned long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 255) {
      if (*abort_sh) return false;
      unsigned long long t = globaltimer();
      if (t0 == 0) t0 = t;
      else if (t - t0 > TIMEOUT_NS) {
        *abort_sh = 1;
        atomicOr(err, 1);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          dst),
      "l"((unsigned long long)map), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// collector hint COL as above; EN: enable_input_d as a compile-time constant (0 starts the accumulator)
template <int COL, int EN>
__device__ __forceinline__ void mma_bf16_ce(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc) {
  mma_bf16_c<COL>(tmem_d, adesc, bdesc, idesc, (uint32_t)EN);
}

__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// EPI_COLS consecutive accumulator columns of this thread's lane into r, without waiting: as few
// tcgen05.ld instructions as the width allows (32-column loads, then 8-column loads)
template <int COLS> __device__ __forceinline__ void tmem_ld_cols_nowait(uint32_t taddr, uint32_t* r) {
#pragma unroll
  for (int h = 0; h < COLS / 32; ++h) tmem_ld32_nowait(taddr + (uint32_t)(h * 32), &r[h * 32]);
#pragma unroll
  for (int h = (COLS / 32) * 4; h < COLS / 8; ++h) tmem_ld8_nowait(taddr + (uint32_t)(h * 8), &r[h * 8]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- kernel
struct EpiArgs {
  void* C;
  int64_t ldc;
  double alpha;
  const void* Y;
  int64_t ldy;
  double gamma;
  const double* ycol;
  const void* Z;
  int64_t ldz;
  double beta;
};

// Accumulator of digit level L: levels below NEX have their own (exact) accumulators, the rest share one.
__host__ __device__ constexpr int acc_of(int level, int nex) { return level < nex ? level : nex; }

// Issue order of one k-block's MMAs: slices t descending; per slice the left planes pl, the two K-steps ks
// and the right slices u descending over the pass's range (pass 0: all pairs; 1: inexact levels; 2: exact
// levels).  An MMA starts its accumulator (enable_input_d = 0) when it is the accumulator's first MMA in
// that order and the k-block restarts it: mode 0 = the first k-block (every accumulator), mode 1 = the
// first k-block of a later chunk (exact accumulators, whose first MMAs are in pass 2), mode 2 = neither.
// Evaluated on compile-time arguments only, so the issuer's per-MMA enable flags are constants.
template <int S, int NEX, int AP>
__host__ __device__ constexpr bool first_touch(int t, int pl, int ks, int u, int pass, int mode) {
  if (mode == 2) return false;
  const int a = acc_of(t + u, NEX);
  if (mode == 1 && a >= NEX) return false;
  for (int ti = 0; ti < S; ++ti) {
    const int tt = S - 1 - ti;
    int ulo = 0, uhi = S - 1 - tt;
    if (pass == 1) ulo = NEX - tt > 0 ? NEX - tt : 0;
    if (pass == 2 && NEX - 1 - tt < uhi) uhi = NEX - 1 - tt;
    for (int p = 0; p < AP; ++p)
      for (int k = 0; k < BK / 16; ++k)
        for (int uu = uhi; uu >= ulo; --uu) {
          if (tt == t && p == pl && k == ks && uu == u) return true;
          if (acc_of(tt + uu, NEX) == a) return false;
        }
  }
  return true;
}

// Parameters of one launch: G independent products (problems) C_p = L_p R_p, each with its own tensor maps,
// sizes, scales and epilogue.  The launch's tiles are the problems' tiles back to back: problem p owns
// blocks [tile_begin[p], tile_begin[p + 1]).  Passed as one __grid_constant__ parameter (the tensor maps
// must live in parameter, constant or global memory for TMA); G = 64 is about 24 KB.
// A product may also be split along K into ksplit slices of klen (a multiple of 96) for launches with
// few output tiles: each slice's CTA writes its FP64 partial sum to part (slice-major, column-major
// M x N, re/im interleaved for complex) and split_reduce_kernel adds the slices and applies the epilogue.
template <int G> struct GroupParams {
  CUtensorMap tmA[G];
  CUtensorMap tmB[G];
  EpiArgs ep[G];
  const double* a_scale[G];
  const double* b_scale[G];
  double* part[G];
  int M[G], N[G], K[G], group_m[G], ksplit[G], klen[G];
  int tile_begin[G + 1];
  int nprob;
};

// Tiles of one problem run in groups of group_m row blocks: inside a group the row block varies fastest,
// so the CTAs that are resident together share the right-operand column blocks (read from DRAM about
// once per group) and a few left-operand row blocks, instead of every row block re-streaming all
// right-operand planes.
template <int S, int NEX, bool CPLX, int NTT, int G>
// 168 registers: ten warps put three on some SM sub-partitions (16384 registers each)
__global__ void __maxnreg__(168) oz_gemm_kernel(const __grid_constant__ GroupParams<G> gp, int* err) {
  using Cf = Cfg<S, NEX, CPLX, NTT>;
  // this block's problem (a short scan of the parameter block's tile offsets)
  int prob = 0;
  if (G > 1)
    while (prob + 1 < gp.nprob && (int)blockIdx.x >= gp.tile_begin[prob + 1]) ++prob;
  const CUtensorMap& tmA = gp.tmA[prob];
  const CUtensorMap& tmB = gp.tmB[prob];
  const EpiArgs& ep = gp.ep[prob];
  const double* __restrict__ a_scale = gp.a_scale[prob];
  const double* __restrict__ b_scale = gp.b_scale[prob];
  const int M = gp.M[prob], N = gp.N[prob], group_m = gp.group_m[prob];
  const int ksplit = gp.ksplit[prob];
  double* __restrict__ part_out = gp.part[prob];
  int local_tile = (int)blockIdx.x - gp.tile_begin[prob];
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sB = smem;
  unsigned char* sA = smem + B_STAGES * Cf::B_STAGE;
  uint64_t* bars = (uint64_t*)(sA + Cf::A_SLOTS * Cf::A_SLOT);
  // barrier layout
  uint64_t* a_full = bars;                    // Cf::A_SLOTS
  uint64_t* a_empty = a_full + Cf::A_SLOTS;       // Cf::A_SLOTS
  uint64_t* b_full = a_empty + Cf::A_SLOTS;       // B_STAGES
  uint64_t* b_empty = b_full + B_STAGES;      // B_STAGES
  uint64_t* chunk_full = b_empty + B_STAGES;  // 1
  uint64_t* tmem_empty = chunk_full + 1;      // 1
  uint64_t* drain = tmem_empty + 1;           // 1
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_sh = (volatile int*)(tmem_slot + 1);

  // a CTA of a launch that already hit a wait limit does nothing
  if (*(volatile int*)err != 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_m = (M + BM - 1) / BM, num_n = (N + Cf::NCOLS - 1) / Cf::NCOLS;
  // K slice of this block (slice-major tile order; one slice unless the product is split along K)
  const int kslice = local_tile / (num_m * num_n);
  local_tile -= kslice * num_m * num_n;
  const int kbeg = kslice * gp.klen[prob];
  const int K = min(gp.K[prob] - kbeg, gp.klen[prob]);  // this slice's extent along K
  const int per_group = group_m * num_n;
  const int first_m = (local_tile / per_group) * group_m;
  const int gm = min(group_m, num_m - first_m);
  const int in_group = local_tile % per_group;
  const int m_tile = first_m + in_group % gm, n_tile = in_group / gm;
  const int m0 = m_tile * BM, n0 = n_tile * Cf::NCOLS;
  const int nkb = (K + BK - 1) / BK;
  const int nchunks = (nkb + KB_PER_CHUNK - 1) / KB_PER_CHUNK;

  if (threadIdx.x == 0) {
    for (int i = 0; i < Cf::A_SLOTS; ++i) {
      mbar_init(smem_u32(&a_full[i]), 1);
      mbar_init(smem_u32(&a_empty[i]), 1);
    }
    for (int i = 0; i < B_STAGES; ++i) {
      mbar_init(smem_u32(&b_full[i]), 1);
      mbar_init(smem_u32(&b_empty[i]), 1);
    }
    mbar_init(smem_u32(chunk_full), 1);
    mbar_init(smem_u32(tmem_empty), EPI_WARPS);
    mbar_init(smem_u32(drain), 1);
    *abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(Cf::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ TMA producer
    int a_iter = 0, b_issued = 0;
    bool ok = true;
    for (int kb = 0; kb < nkb && ok; ++kb) {
      const int k0 = kbeg + kb * BK;
      const int bs = kb % B_STAGES;
      if (!mbar_wait(smem_u32(&b_empty[bs]), ((kb / B_STAGES) & 1) ^ 1, abort_sh, err)) {
        ok = false;
        break;
      }
      ++b_issued;
      if (Cf::GROUPED) {
        // the leading G0 slices' slots are released together (on a_empty[0]) and refilled with this k-block's
        // right operand, all on b_full[bs]
        if (!mbar_wait(smem_u32(&a_empty[0]), (kb & 1) ^ 1, abort_sh, err)) {
          ok = false;
          break;
        }
        mbar_expect_tx(smem_u32(&b_full[bs]), Cf::B_BYTES + Cf::G0 * Cf::A_SLOT);
      } else {
        mbar_expect_tx(smem_u32(&b_full[bs]), Cf::B_BYTES);
      }
      // every slice and plane of the right operand's k-block in one copy (the box spans all S x BP planes,
      // landing plane-major exactly as the MMA descriptors expect)
      tma_load_3d(smem_u32(sB + bs * Cf::B_STAGE), &tmB, smem_u32(&b_full[bs]), k0, n0, 0);
      for (int ti = 0; ti < S; ++ti, ++a_iter) {
        const int t = S - 1 - ti;
        const int as = a_iter % Cf::A_SLOTS;
        if (ti < Cf::G0) {  // grouped: slot as == ti, already free
          tma_load_3d(smem_u32(sA + as * Cf::A_SLOT), &tmA, smem_u32(&b_full[bs]), k0, m0, t * Cf::AP);
          continue;
        }
        // a group's first slice waits for the group's release and announces all of its bytes
        const int fs = (a_iter - ti + Cf::gfirst(ti)) % Cf::A_SLOTS;  // slot of the group's first slice
        if (ti == Cf::gfirst(ti)) {
          if (!mbar_wait(smem_u32(&a_empty[as]), ((a_iter / Cf::A_SLOTS) & 1) ^ 1, abort_sh, err)) {
            ok = false;
            break;
          }
          mbar_expect_tx(smem_u32(&a_full[as]), (Cf::glast(ti) - ti + 1) * Cf::A_SLOT);
        }
        // both planes (re, im) of the slice in one copy
        tma_load_3d(smem_u32(sA + as * Cf::A_SLOT), &tmA, smem_u32(&a_full[fs]), k0, m0, t * Cf::AP);
      }
    }
    // drain: every issued copy must have landed before the CTA exits
    for (int i = 0; i < B_STAGES; ++i) {
      int uses = b_issued / B_STAGES + (i < b_issued % B_STAGES ? 1 : 0);
      if (uses > 0) {
        unsigned long long t0 = globaltimer();
        while (!mbar_try(smem_u32(&b_full[i]), (uses - 1) & 1) && globaltimer() - t0 < TIMEOUT_NS) {
        }
      }
    }
    for (int i = Cf::G0; i < Cf::A_SLOTS; ++i) {
      if (Cf::GROUPED && i != Cf::gfirst(i)) continue;  // grouped: only a group's first slot has copies on it
      int uses = a_iter / Cf::A_SLOTS + (i < a_iter % Cf::A_SLOTS ? 1 : 0);
      if (uses > 0) {
        unsigned long long t0 = globaltimer();
        while (!mbar_try(smem_u32(&a_full[i]), (uses - 1) & 1) && globaltimer() - t0 < TIMEOUT_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    constexpr uint32_t IDESC = idesc_bf16(BM, Cf::NT);
    int a_iter = 0;
    bool ok = true;
    // MMAs of slice t (all its pairs in `pass`), both K-steps, in the order first_touch walks.  Per A plane
    // and K-step, the MMAs over the right-operand slices u run back to back and share one A tile through the
    // collector buffer (fill, use..., lastuse).  After unrolling, t, pass and mode are constants, so levels,
    // accumulators, descriptor offsets, collector hints and enable flags all fold.
    auto issue_slice = [&](const int t, const int pass, const int mode, const uint64_t adesc, const uint64_t bdesc) {
      int ulo = 0, uhi = Cf::MAXLEVEL - t;  // u range: levels t + ulo .. t + uhi
      if (pass == 1) ulo = NEX - t > 0 ? NEX - t : 0;
      if (pass == 2 && NEX - 1 - t < uhi) uhi = NEX - 1 - t;
      if (uhi < ulo) return;
      const int cnt = uhi - ulo + 1;
#pragma unroll
      for (int pl = 0; pl < Cf::AP; ++pl) {
#pragma unroll
        for (int ks = 0; ks < BK / 16; ++ks) {
          const uint64_t ko = (uint64_t)(ks * 2);  // 32 bytes along K, in 16-byte units
          const uint64_t a = adesc + (uint64_t)((pl * Cf::A_PLANE) >> 4) + ko;
#pragma unroll
          for (int i = 0; i < S; ++i) {
            if (i >= cnt) continue;
            const int u = uhi - i;
            const int acc = acc_of(t + u, NEX);
            const uint32_t dt = tmem + (uint32_t)(acc * Cf::NT);
            const uint64_t bslice = bdesc + (uint64_t)((u * Cf::B_SLICE) >> 4);
            // complex: [Cr | Ci] += Ar [Yr | Yi] (planes 1, 2) + Ai [-Yi | Yr] (planes 0, 1)
            const uint64_t b = (CPLX && pl == 0 ? bslice + (uint64_t)(Cf::B_PLANE >> 4) : bslice) + ko;
            const bool st = first_touch<S, NEX, Cf::AP>(t, pl, ks, u, pass, mode);
            const int col = cnt == 1 ? 0 : (i == 0 ? 1 : (i == cnt - 1 ? 3 : 2));
            if (st) {
              if (col == 0) mma_bf16_ce<0, 0>(dt, a, b, IDESC);
              else if (col == 1) mma_bf16_ce<1, 0>(dt, a, b, IDESC);
              else if (col == 3) mma_bf16_ce<3, 0>(dt, a, b, IDESC);
              else mma_bf16_ce<2, 0>(dt, a, b, IDESC);
            } else {
              if (col == 0) mma_bf16_ce<0, 1>(dt, a, b, IDESC);
              else if (col == 1) mma_bf16_ce<1, 1>(dt, a, b, IDESC);
              else if (col == 3) mma_bf16_ce<3, 1>(dt, a, b, IDESC);
              else mma_bf16_ce<2, 1>(dt, a, b, IDESC);
            }
          }
        }
      }
    };
    // one pass over all slices (modes 0 and 2): slices in descending order, each slot released after its MMAs
    auto one_pass = [&](const int mode, const uint64_t bdesc) {
#pragma unroll
      for (int ti = 0; ti < S; ++ti) {
        const int as = (a_iter + ti) % Cf::A_SLOTS;
        const int fs = (a_iter + Cf::gfirst(ti)) % Cf::A_SLOTS;
        // the leading G0 slices arrived with the right operand; a later group is checked at its first slice
        if (ti >= Cf::G0 && ti == Cf::gfirst(ti)) {
          if (ok && !mbar_wait(smem_u32(&a_full[as]), ((a_iter + ti) / Cf::A_SLOTS) & 1, abort_sh, err)) ok = false;
          if (!ok) break;
          fence_after();
        }
        issue_slice(S - 1 - ti, 0, mode, sw64_desc(smem_u32(sA + as * Cf::A_SLOT)), bdesc);
        if (ti >= Cf::G0 && ti == Cf::glast(ti)) mma_commit(smem_u32(&a_empty[fs]));
        else if (ti == Cf::G0 - 1) mma_commit(smem_u32(&a_empty[0]));
      }
    };
    for (int kb = 0; kb < nkb && ok; ++kb) {
      const int bs = kb % B_STAGES;
      const int chunk = kb / KB_PER_CHUNK;
      const bool chunk_start = (kb % KB_PER_CHUNK) == 0;
      if (!mbar_wait(smem_u32(&b_full[bs]), (kb / B_STAGES) & 1, abort_sh, err)) {
        ok = false;
        break;
      }
      fence_after();
      const uint64_t bdesc = sw64_desc(smem_u32(sB + bs * Cf::B_STAGE));
      if (kb == 0) {
        one_pass(0, bdesc);
        if (!ok) break;
        a_iter += S;
      } else if (!(NEX > 0 && chunk_start)) {
        one_pass(2, bdesc);
        if (!ok) break;
        a_iter += S;
      } else {
        // first k-block of a chunk: every inexact pair of the k-block runs while the epilogue
        // flushes the exact accumulators of the previous chunk, then the exact pairs.  Slices
        // t >= NEX have no exact pairs (level t + u >= NEX): their slots are released at once.
#pragma unroll
        for (int ti = 0; ti < S; ++ti) {
          const int as = (a_iter + ti) % Cf::A_SLOTS;
          const int fs = (a_iter + Cf::gfirst(ti)) % Cf::A_SLOTS;
          if (ti >= Cf::G0 && ti == Cf::gfirst(ti)) {
            if (ok && !mbar_wait(smem_u32(&a_full[as]), ((a_iter + ti) / Cf::A_SLOTS) & 1, abort_sh, err)) ok = false;
            if (!ok) break;
            fence_after();
          }
          issue_slice(S - 1 - ti, 1, 1, sw64_desc(smem_u32(sA + as * Cf::A_SLOT)), bdesc);
          // a group whose last slice has no exact pairs is done after this pass
          if (S - 1 - Cf::glast(ti) >= NEX) {
            if (ti >= Cf::G0 && ti == Cf::glast(ti)) mma_commit(smem_u32(&a_empty[fs]));
            else if (ti == Cf::G0 - 1) mma_commit(smem_u32(&a_empty[0]));
          }
        }
        if (ok && !mbar_wait(smem_u32(tmem_empty), (chunk - 1) & 1, abort_sh, err)) ok = false;
        if (!ok) break;
        fence_after();
#pragma unroll
        for (int ti = 0; ti < S; ++ti) {
          if (S - 1 - ti >= NEX) continue;
          const int as = (a_iter + ti) % Cf::A_SLOTS;
          const int fs = (a_iter + Cf::gfirst(ti)) % Cf::A_SLOTS;
          issue_slice(S - 1 - ti, 2, 1, sw64_desc(smem_u32(sA + as * Cf::A_SLOT)), bdesc);
          if (ti >= Cf::G0 && ti == Cf::glast(ti)) mma_commit(smem_u32(&a_empty[fs]));
          else if (ti == Cf::G0 - 1) mma_commit(smem_u32(&a_empty[0]));
        }
        a_iter += S;
      }
      mma_commit(smem_u32(&b_empty[bs]));
      // exact levels: one commit per chunk (the epilogue consumes each before the next
      // chunk's exact MMAs start); single-accumulator modes: one commit at the end
      if ((NEX > 0 && (kb % KB_PER_CHUNK) == KB_PER_CHUNK - 1) || kb == nkb - 1) mma_commit(smem_u32(chunk_full));
    }
    // drain all MMAs before TMEM can be freed
    mma_commit(smem_u32(drain));
    unsigned long long t0 = globaltimer();
    while (!mbar_try(smem_u32(drain), 0) && globaltimer() - t0 < TIMEOUT_NS) {
    }
  } else if (warp >= EPI_WARP0) {
    // ------------------------------------------------------------ epilogue
    constexpr int EPI_COLS = Cf::EPI_COLS;
    const int ew = warp - EPI_WARP0;
    const int wg = ew >> 2;        // accumulator columns [EPI_COLS wg, EPI_COLS (wg + 1))
    const int q = warp & 3;        // TMEM lane quadrant
    const int row = q * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
    // exact levels 0..NEX-1 summed as one integer in units of level NEX-1's grid
    // (2^-32 for NEX = 5).  Per chunk |sum| <= 1.5 2^53, so K <= 65472 cannot overflow.
    long long acc64[NEX > 0 ? EPI_COLS : 1];
#pragma unroll
    for (int j = 0; j < (NEX > 0 ? EPI_COLS : 1); ++j) acc64[j] = 0;
    bool ok = true;
    const int nwait = NEX > 0 ? nchunks : 1;
    for (int ch = 0; ch < nwait; ++ch) {
      if (!mbar_wait(smem_u32(chunk_full), ch & 1, abort_sh, err)) {
        ok = false;
        break;
      }
      fence_after();
      if (NEX > 0) {
#pragma unroll
        for (int L = 0; L < (NEX > 0 ? NEX : 1); ++L) {
          // all columns of one level in flight, one wait
          uint32_t r[EPI_COLS];
          tmem_ld_cols_nowait<EPI_COLS>(lane_addr + (uint32_t)(L * Cf::NT + wg * EPI_COLS), r);
          tmem_wait_ld();
          const float sc = (float)(1ull << (8 * L));  // level L unit is 2^-8L
#pragma unroll
          for (int j = 0; j < EPI_COLS; ++j) {
            const long long iv = (long long)__float2int_rn(__uint_as_float(r[j]) * sc);
            acc64[j] += iv << (8 * (NEX - 1 - L));
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(tmem_empty));
      }
    }
    if (ok) {
      const int gi = m0 + row;
#pragma unroll
      for (int h = 0; h < EPI_COLS / 8; ++h) {
        uint32_t r[8];
        tmem_ld8(lane_addr + (uint32_t)(NEX * Cf::NT + wg * EPI_COLS + h * 8), r);
        if (gi >= M) continue;
        const double rs = a_scale[gi];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int j = h * 8 + jj;
          const int c = wg * EPI_COLS + j;
          int gj, part;
          if (CPLX) {
            gj = n0 + (c % Cf::NCOLS);
            part = c / Cf::NCOLS;
          } else {
            gj = n0 + c;
            part = 0;
          }
          if (gj >= N) continue;
          double v = (double)__uint_as_float(r[jj]);
          if (NEX > 0) v += (double)acc64[NEX > 0 ? j : 0] * 2.3283064365386963e-10;  // 2^-32
          v *= rs * b_scale[gj] * 6.103515625e-05;                                   // 2^-14
          const int comp = CPLX ? 2 : 1;
          if (ksplit > 1) {
            part_out[(((int64_t)kslice * N + gj) * M + gi) * comp + part] = v;
            continue;
          }
          double out = ep.alpha * v;
          if (ep.Y) {
            const double g = ep.gamma * (ep.ycol ? ep.ycol[gj] : 1.0);
            out += g * ((const double*)ep.Y)[(gi + (int64_t)gj * ep.ldy) * comp + part];
          }
          if (ep.Z) out += ep.beta * ((const double*)ep.Z)[(gi + (int64_t)gj * ep.ldz) * comp + part];
          ((double*)ep.C)[(gi + (int64_t)gj * ep.ldc) * comp + part] = out;
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cf::TMEM_COLS));
}

// C = alpha sum_s part[s] + gamma ycol Y + beta Z over the ksplit K slices (slice order fixed, so the
// result does not depend on scheduling).
template <bool CPLX>
__global__ void split_reduce_kernel(int M, int N, int ksplit, const double* __restrict__ part, EpiArgs ep) {
  constexpr int comp = CPLX ? 2 : 1;
  const int64_t total = (int64_t)M * N * comp;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int pt = (int)(idx % comp);
    const int64_t e = idx / comp;
    const int gi = (int)(e % M), gj = (int)(e / M);
    double v = 0.0;
    for (int ks = 0; ks < ksplit; ++ks) v += part[(int64_t)ks * total + idx];
    double out = ep.alpha * v;
    if (ep.Y) {
      const double g = ep.gamma * (ep.ycol ? ep.ycol[gj] : 1.0);
      out += g * ((const double*)ep.Y)[(gi + (int64_t)gj * ep.ldy) * comp + pt];
    }
    if (ep.Z) out += ep.beta * ((const double*)ep.Z)[(gi + (int64_t)gj * ep.ldz) * comp + pt];
    ((double*)ep.C)[(gi + (int64_t)gj * ep.ldc) * comp + pt] = out;
  }
}

// ---------------------------------------------------------------- launch
typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                             const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeFn)p;
  });
  return fn;
}

// box: BK (K) x box_rows x box_planes consecutive planes; a copy lands plane-major in shared memory
inline CUtensorMap make_map(const void* base, int64_t K, int64_t Kpad, int64_t rows, int planes, int box_rows,
                            int box_planes) {
  CUtensorMap m;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(Kpad * 2), (cuuint64_t)(Kpad * 2 * rows)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
  cuuint32_t es[3] = {1, 1, 1};
  EncodeFn fn = encode_fn();
  CHASE_REQUIRE(fn != nullptr, 9, "cuTensorMapEncodeTiled unavailable");
  CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CHASE_REQUIRE(r == CUDA_SUCCESS, 6, "cuTensorMapEncodeTiled failed");
  return m;
}

inline int64_t kpad(int64_t K) { return (K + 7) / 8 * 8; }

// Products of one launch: up to G of them, each C = L R from its digit planes (left: rows = M vectors of
// length K, split into l_slices_total slices of which the first S are used; right: rows = N vectors of
// length K, S slices).
template <int S, int NEX, bool CPLX, int NTT, int G>
void launch_ops(cudaStream_t st, Workspace& w, const ProductOp* ops, int nops, cudaEvent_t* tune_ev) {
  using Cf = Cfg<S, NEX, CPLX, NTT>;
  CHASE_REQUIRE(nops >= 1 && nops <= G, 1, "split product: bad number of products in one launch");
  const int ap = CPLX ? 2 : 1, bp = CPLX ? 3 : 1;
  // the parameter block is large for G > 1: build it in thread-local host memory
  static thread_local GroupParams<G> gp;
  int64_t tiles = 0;
  for (int q = 0; q < nops; ++q) {
    const ProductOp& o = ops[q];
    const int64_t kp = kpad(o.K);
    gp.tmA[q] = make_map(o.lpl, o.K, kp, o.M, o.l_slices_total * ap, BM, ap);
    gp.tmB[q] = make_map(o.rpl, o.K, kp, o.N, S * bp, Cf::BROWS, S * bp);
    const Epi& e = o.e;
    gp.ep[q] = EpiArgs{e.C, e.ldc, e.alpha, e.Y, e.ldy, e.gamma, e.ycol, e.Z, e.ldz, e.beta};
    gp.a_scale[q] = o.lsc;
    gp.b_scale[q] = o.rsc;
    gp.M[q] = (int)o.M;
    gp.N[q] = (int)o.N;
    gp.K[q] = (int)o.K;
    gp.group_m[q] = std::max(1, o.group_m);
    gp.ksplit[q] = std::max(1, o.ksplit);
    gp.klen[q] = o.ksplit > 1 ? o.klen : (int)o.K;
    gp.part[q] = o.part;
    gp.tile_begin[q] = (int)tiles;
    tiles += (int64_t)ceil_div(o.N, Cf::NCOLS) * (int64_t)ceil_div(o.M, BM) * gp.ksplit[q];
    CHASE_REQUIRE(tiles <= 0x7fffffff, 1, "split product: too many tiles");
  }
  gp.tile_begin[nops] = (int)tiles;
  gp.nprob = nops;
  if (tiles == 0) return;
  // once per instantiation, thread-safe (batched solves launch from several host threads)
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [&]() {
    attr_err = cudaFuncSetAttribute(oz_gemm_kernel<S, NEX, CPLX, NTT, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    Cf::SMEM_BYTES);
  });
  CHASE_CUDA(attr_err);
  const bool timed = w.timing && w.ev_used + 2 <= (int)w.ev.size();
  if (timed) CHASE_CUDA(cudaEventRecord(w.ev[w.ev_used], st));
  if (tune_ev) CHASE_CUDA(cudaEventRecord(tune_ev[0], st));
  oz_gemm_kernel<S, NEX, CPLX, NTT, G><<<(unsigned)tiles, NTHREADS, Cf::SMEM_BYTES, st>>>(gp, w.flags);
  CHASE_CHECK_LAUNCH();
  for (int q = 0; q < nops; ++q) {
    if (gp.ksplit[q] <= 1) continue;
    const int64_t total = ops[q].M * ops[q].N * (CPLX ? 2 : 1);
    split_reduce_kernel<CPLX><<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 4096), 256, 0, st>>>(
        (int)ops[q].M, (int)ops[q].N, gp.ksplit[q], ops[q].part, gp.ep[q]);
    CHASE_CHECK_LAUNCH();
  }
  if (tune_ev) CHASE_CUDA(cudaEventRecord(tune_ev[1], st));
  if (timed) {
    CHASE_CUDA(cudaEventRecord(w.ev[w.ev_used + 1], st));
    w.ev_used += 2;
  }
}

// The launches are instantiated in the oz_inst_*.cu units (compiled in parallel); every other unit sees
// them as external.
extern template void launch_ops<7, 5, true, 80, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<7, 5, true, 16, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<7, 5, true, 80, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<6, 5, true, 80, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<6, 5, true, 16, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<6, 5, true, 80, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<3, 0, true, 256, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<3, 0, true, 128, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<3, 0, true, 256, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<3, 0, true, 128, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<2, 0, true, 256, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<2, 0, true, 128, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<2, 0, true, 256, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<2, 0, true, 128, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<7, 5, false, 80, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<7, 5, false, 16, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<7, 5, false, 80, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<6, 5, false, 80, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<6, 5, false, 16, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<6, 5, false, 80, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<3, 0, false, 256, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<3, 0, false, 128, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<3, 0, false, 256, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<3, 0, false, 128, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<2, 0, false, 256, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<2, 0, false, 128, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<2, 0, false, 256, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
extern template void launch_ops<2, 0, false, 128, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);

}  // namespace oz
}  // namespace chase
