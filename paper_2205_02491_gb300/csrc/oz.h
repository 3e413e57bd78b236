// Split-BF16 tensor-core products (tcgen05) with FP64-accurate or mixed
// precision accumulation: the production path of the large HEMM/GEMM products.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <vector>

#include "kernels.h"

namespace chase {
namespace oz {

// Launch configuration of the split-product kernel chosen by measurement (see tune_pick in oz_gemm.cu):
// the tile width NT of the mixed modes (128 or 256 columns) and the tile-order group size.
struct LaunchCfg {
  int nt = 0;       // 0: the mode's fixed width
  int group_m = 8;
};

// One size class of the tuner: candidates are timed on consecutive launches of that class (the degree
// steps of a filter repeat one shape), then the fastest is kept for the context's lifetime.
struct TuneEntry {
  int next = 0;          // candidates launched so far
  int best = -1;         // index of the chosen candidate once every one has been timed
  std::vector<cudaEvent_t> ev;  // start/stop pair per candidate
};

struct Workspace {
  bool ready = false;
  bool complex_ = true;
  int slices = 6;
  int64_t n_max = 0;
  int ne_max = 0;
  void* a_planes = nullptr;   // bf16 digit planes of A
  void* b_planes = nullptr;   // bf16 digit planes of the right operand
  void* l_planes = nullptr;   // bf16 digit planes of a general left operand
  double* a_scale = nullptr;  // per-row power-of-two scale of A
  double* l_scale = nullptr;  // per-row scale of the general left operand
  double* b_scale = nullptr;  // per-column scale of the right operand
  int* flags = nullptr;       // device error flags of the bounded waits
  double* partial = nullptr;  // FP64 partial sums of products split along K
  int64_t partial_elems = 0;
  int group_m = 8;            // row blocks per tile group of the split-product launch order (untuned launches)
  bool autotune = true;       // choose LaunchCfg per size class by timing the candidates
  std::map<uint64_t, TuneEntry> tune;  // size class -> measurements and choice
  // optional CUDA-event timing of the product kernels (filter roofline)
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  const void* a_src = nullptr;  // A whose planes are cached
  int a_mode = -1;
  int64_t a_n = 0;
};

// One product C = L R of a grouped launch: digit planes and scales of both operands, sizes, epilogue and
// the tile-order group size.
struct ProductOp {
  const void* lpl;
  const double* lsc;
  int l_slices_total;
  const void* rpl;
  const double* rsc;
  int64_t M, N, K;
  Epi e;
  int group_m;
  int ksplit = 1;           // K slices (> 1: partial sums to `part`, then a reduction launch)
  int klen = 0;             // slice length along K (multiple of 96)
  double* part = nullptr;   // ksplit x M x N (x 2 complex) doubles
};

bool available();
int64_t workspace_bytes(int64_t n_max, int ne_max, bool complex_, int slices);
void create(Workspace& w, int64_t n_max, int ne_max, bool complex_, int slices);
void destroy(Workspace& w);
// the tuner's choices so far: (size-class key, candidate index) pairs, for reports
std::vector<std::pair<uint64_t, int>> tuned(const Workspace& w);
void invalidate(Workspace& w);
// start recording event pairs around every product kernel; collect returns (ms, launches)
void timing_begin(Workspace& w);
double timing_collect(Workspace& w, int* launches);
int read_flags(cudaStream_t st, Workspace& w);
// digit planes of the right operand B (n x k, ld ldb) into w's right-operand buffer, for the given mode
template <typename T>
void split_right(cudaStream_t st, Workspace& w, int mode, const T* B, int64_t ldb, int k, int64_t n);
// one launch (per 64 products) over the tiles of all the products; w supplies the error flags and timing.
// Every op's planes must have been split with the mode's slice count (left: at least that many slices).
template <bool CPLX> void launch_group(cudaStream_t st, Workspace& w, int mode, const ProductOp* ops, int nops);
template <typename T>
void prepare_A(cudaStream_t st, Workspace& w, const T* A, int64_t n, int64_t lda, int mode);
template <typename T>
void hemm(cudaStream_t st, Workspace& w, const T* A, int64_t n, int64_t lda, const T* B, int64_t ldb, int k,
          const Epi& e, int mode);
// C = op(A) op(B) (M x N, inner K) through split products; op(A) = A (M x K) or A^H (A: K x M),
// op(B) = B (K x N) or B^H (B: N x K).
template <typename T>
void gemm(cudaStream_t st, Workspace& w, Op opA, const T* A, int64_t lda, Op opB, const T* B, int64_t ldb, int64_t M,
          int64_t N, int64_t K, const Epi& e, int mode);

}  // namespace oz
}  // namespace chase
