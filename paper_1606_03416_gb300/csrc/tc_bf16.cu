// BF16 instantiations of the tensor-core Chebyshev step kernel.
#include "tc_kernel.cuh"

namespace dg {
FilterKernel pick_kernel_bf16(int G, int T, int ACC, int layout) {
  return pick_shape<MODE_BF16>(G, T, ACC, layout);
}
}  // namespace dg
