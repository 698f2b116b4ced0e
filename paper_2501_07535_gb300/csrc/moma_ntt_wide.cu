// moma_ntt_wide.cu -- transform pass kernels and twiddle generation for 512-, 768- and 1024-bit
// containers (16, 24 and 32 limbs), kept apart from the narrower widths so that the two halves
// compile in parallel.
#include "moma_internal.hpp"
#include "moma_ntt_pass.cuh"

namespace moma {

moma_status run_pass_wide(moma_ctx* ctx, const Plan* pl, const PassDesc& d, size_t count, const uint32_t* src,
                          const uint32_t* src2, uint32_t* dst, uint32_t flags, const moma_config& cfg,
                          cudaStream_t st) {
  switch (ctx->L) {
    case 16: return run_pass_for<16>(ctx, pl, d, count, src, src2, dst, flags, cfg, st);
    case 24: return run_pass_for<24>(ctx, pl, d, count, src, src2, dst, flags, cfg, st);
    case 32: return run_pass_for<32>(ctx, pl, d, count, src, src2, dst, flags, cfg, st);
  }
  return MOMA_ERR_UNSUPPORTED;
}

moma_status gen_table_wide(const moma_ctx* ctx, uint32_t* dst, uint64_t count, uint64_t D, uint64_t C, uint64_t S,
                           int logn, const std::vector<BigU>& pw, const BigU& init) {
  switch (ctx->L) {
    case 16: return gen_table<16>(ctx, dst, count, D, C, S, logn, pw, init);
    case 24: return gen_table<24>(ctx, dst, count, D, C, S, logn, pw, init);
    case 32: return gen_table<32>(ctx, dst, count, D, C, S, logn, pw, init);
  }
  return MOMA_ERR_UNSUPPORTED;
}

}  // namespace moma
