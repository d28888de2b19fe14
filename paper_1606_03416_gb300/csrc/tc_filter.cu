// Tensor-core (tcgen05) Chebyshev filter: placeholder until the kernel lands.
#include "ctx.h"

namespace dg {

struct TcState {};

dgchefsi_status filter_tc(dgchefsi_ctx* ctx, int prec, const double*, double*, int64_t, int64_t, int, double, double,
                          double) {
  (void)ctx;
  return set_error(DGCHEFSI_ERR_UNSUPPORTED, "tensor-core precision %d not built", prec);
}

void tc_destroy(dgchefsi_ctx* ctx) {
  delete ctx->tc;
  ctx->tc = nullptr;
}

}  // namespace dg
