// moma_blas.cu -- element-wise modular BLAS (Sec. 2.1 Eq. 1, Sec. 2.3 axpy): schedules (product
// engine, vector width) and the dispatch over limb counts up to 384 bits.  The kernels are in
// moma_blas_kern.cuh; 512 bits and up dispatch in moma_blas_wide.cu.
#include "moma_blas_kern.cuh"
#include "moma_internal.hpp"

namespace moma {

// Largest vector width per L: keeps the two operand tiles (2*V*L words) near 64 registers.
int vec_max_width(int L) { return L <= 8 ? 4 : (L <= 12 ? 2 : 1); }

int vec_max_log_tile(int L) {
  switch (L) {
    case 2: return vec_staged_max_log_tile<2>();
    case 4: return vec_staged_max_log_tile<4>();
    case 8: return vec_staged_max_log_tile<8>();
    case 12: return vec_staged_max_log_tile<12>();
    case 16: return vec_staged_max_log_tile<16>();
    case 24: return vec_staged_max_log_tile<24>();
    case 32: return vec_staged_max_log_tile<32>();
  }
  return 0;
}

moma_config vec_config(const moma_ctx* ctx, int vec_op) {
  moma_config c = {0, 0, 0, 0, 0, 0};
  {
    std::lock_guard<std::mutex> g(ctx->lock);  // moma_ctx_set_config may write the map meanwhile
    auto it = ctx->configs.find(std::make_pair(MOMA_OP_ADD + vec_op, -1));
    if (it != ctx->configs.end()) c = it->second;
  }
  // Karatsuba (engine 3) measured at or above schoolbook for mulmod on GB300 from 64 to 768 bits
  // (1.00x at 256 bits up to 1.2x at 768 bits; 0.9x at 1024 bits, where carry chains are kept);
  // carry chains for the other ops
  if (c.engine == 0) c.engine = (vec_op == VEC_MUL && ctx->L <= 24) ? 3 : 1;
  // measured on GB300 at 2^24 elements: two elements per thread at 256 bits (the two products
  // interleave: 430 against 453 us for mulmod), one for mulmod from 384 bits up, two for additions
  // and axpy; narrow widths take the widest vectors
  if (c.vec_width == 0) {
    const int vm = vec_max_width(ctx->L);
    const int pref = ctx->L <= 4 ? 4 : ((vec_op == VEC_MUL && ctx->L > 8) ? 1 : 2);
    c.vec_width = pref < vm ? pref : vm;
  }
  // tile_log: 0 = direct vector loads; 8..10 = operands staged by bulk copies in tiles of
  // 2^tile_log elements (full-width contexts always load directly)
  if (ctx->mont) c.tile_log = 0;
  c.max_logr = 0;
  return c;
}

moma_status launch_vec_cfg(moma_ctx* ctx, int op, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                           const uint32_t* alpha_host, const moma_config& cfg, cudaStream_t st) {
  switch (ctx->L) {
    case 2: return dispatch_op<2>(ctx, op, n, a, b, c, alpha_host, cfg, st);
    case 4: return dispatch_op<4>(ctx, op, n, a, b, c, alpha_host, cfg, st);
    case 8: return dispatch_op<8>(ctx, op, n, a, b, c, alpha_host, cfg, st);
    case 12: return dispatch_op<12>(ctx, op, n, a, b, c, alpha_host, cfg, st);
    default: return launch_vec_wide(ctx, op, n, a, b, c, alpha_host, cfg, st);
  }
}

moma_status launch_vec(moma_ctx* ctx, int op, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                       const uint32_t* alpha_host, cudaStream_t st) {
  return launch_vec_cfg(ctx, op, n, a, b, c, alpha_host, vec_config(ctx, op), st);
}

}  // namespace moma
