// Split-product launches (kernel instantiations) for the mixed modes (2 or 3 slices), real operands: one unit per group so the
// kernels compile in parallel.
#include "oz_kernel.cuh"

namespace chase {
namespace oz {

template void launch_ops<3, 0, false, 256, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
template void launch_ops<3, 0, false, 128, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
template void launch_ops<3, 0, false, 256, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
template void launch_ops<3, 0, false, 128, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
template void launch_ops<2, 0, false, 256, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
template void launch_ops<2, 0, false, 128, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
template void launch_ops<2, 0, false, 256, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);
template void launch_ops<2, 0, false, 128, 64>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);

}  // namespace oz
}  // namespace chase
