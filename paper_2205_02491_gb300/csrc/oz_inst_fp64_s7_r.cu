// Split-product launches (kernel instantiations) for the FP64 modes, 7 slices, real operands: one unit per group so the
// kernels compile in parallel.
#include "oz_kernel.cuh"

namespace chase {
namespace oz {

template void launch_ops<7, 5, false, 80, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
template void launch_ops<7, 5, false, 16, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
template void launch_ops<7, 5, false, 80, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);

}  // namespace oz
}  // namespace chase
