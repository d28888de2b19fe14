// TF32 instantiations of the tensor-core Chebyshev step kernel.
#include "tc_kernel.cuh"

namespace dg {
FilterKernel pick_kernel_tf32(int G, int T, int ACC, int layout) {
  return pick_shape<MODE_TF32>(G, T, ACC, layout);
}
}  // namespace dg
