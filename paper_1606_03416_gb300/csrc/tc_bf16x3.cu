// BF16X3 instantiations of the tensor-core Chebyshev step kernel.
#include "tc_kernel.cuh"

namespace dg {
FilterKernel pick_kernel_bf16x3(int G, int T, int ACC, int layout) {
  return pick_shape<MODE_BF16X3>(G, T, ACC, layout);
}
}  // namespace dg
