// Placeholder for the tensor-core split products until the tcgen05 kernels land.
#include "common.cuh"
#include "oz.h"

namespace chase {
namespace oz {
bool available() { return false; }
int64_t workspace_bytes(int64_t, int, bool, int) { return 0; }
void create(Workspace& w, int64_t n_max, int ne_max, bool complex_, int slices) {
  w.n_max = n_max;
  w.ne_max = ne_max;
  w.complex_ = complex_;
  w.slices = slices;
}
void destroy(Workspace&) {}
template <typename T> void prepare_A(cudaStream_t, Workspace&, const T*, int64_t, int64_t, int) {
  throw Error{9, "tensor-core split products not available"};
}
template <typename T>
void hemm(cudaStream_t, Workspace&, const T*, int64_t, int64_t, const T*, int64_t, int, const Epi&, int) {
  throw Error{9, "tensor-core split products not available"};
}
template void prepare_A<double>(cudaStream_t, Workspace&, const double*, int64_t, int64_t, int);
template void prepare_A<double2>(cudaStream_t, Workspace&, const double2*, int64_t, int64_t, int);
template void hemm<double>(cudaStream_t, Workspace&, const double*, int64_t, int64_t, const double*, int64_t, int,
                           const Epi&, int);
template void hemm<double2>(cudaStream_t, Workspace&, const double2*, int64_t, int64_t, const double2*, int64_t, int,
                            const Epi&, int);
}  // namespace oz
}  // namespace chase
