// moma_blas_wide.cu -- element-wise kernels for 512-, 768- and 1024-bit containers (16, 24 and
// 32 limbs), kept apart from the narrower widths so that the two halves compile in parallel.
#include "moma_blas_kern.cuh"
#include "moma_internal.hpp"

namespace moma {

moma_status launch_vec_wide(moma_ctx* ctx, int op, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                            const uint32_t* alpha_host, const moma_config& cfg, cudaStream_t st) {
  switch (ctx->L) {
    case 16: return dispatch_op<16>(ctx, op, n, a, b, c, alpha_host, cfg, st);
    case 24: return dispatch_op<24>(ctx, op, n, a, b, c, alpha_host, cfg, st);
    case 32: return dispatch_op<32>(ctx, op, n, a, b, c, alpha_host, cfg, st);
  }
  return MOMA_ERR_INVALID_ARG;
}

}  // namespace moma
