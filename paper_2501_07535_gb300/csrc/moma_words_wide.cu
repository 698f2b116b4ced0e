// moma_words_wide.cu -- the word-level block probe for 512- and 768-bit contexts (1024 bits is
// not instantiated: its one kernel alone would double the library's build time).
#include "moma_words.cuh"

namespace moma {

moma_status run_words_wide(moma_ctx* ctx, int op, int engine, size_t n, const uint32_t* a, const uint32_t* b,
                           uint32_t* out, cudaStream_t st) {
  switch (ctx->L) {
    case 16: return run_words<16>(ctx, op, engine, n, a, b, out, st);
    case 24: return run_words<24>(ctx, op, engine, n, a, b, out, st);
  }
  return MOMA_ERR_UNSUPPORTED;
}

}  // namespace moma
