// Split-product launches (kernel instantiations) for the FP64 modes, 7 slices, complex operands, 80-column tiles, one product per launch: one
// unit per instantiation of this (largest) group so the kernels compile in parallel.
#include "oz_kernel.cuh"

namespace chase {
namespace oz {

template void launch_ops<7, 5, true, 80, 1>(cudaStream_t, Workspace&, const ProductOp*, int, cudaEvent_t*);

}  // namespace oz
}  // namespace chase
