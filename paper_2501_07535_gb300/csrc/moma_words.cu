// moma_words.cu -- moma_word_probe: the word-level building blocks with their raw outputs
// (kernel in moma_words.cuh; 512 bits and up in moma_words_wide.cu).
#include "moma_words.cuh"

using namespace moma;

extern "C" moma_status moma_word_probe(moma_ctx* ctx, int op, int engine, size_t n, const uint32_t* a,
                                       const uint32_t* b, uint32_t* out, void* stream) {
  if (!ctx || !a || !b || !out) return MOMA_ERR_INVALID_ARG;
  if (op < MOMA_WORD_ADD || op > MOMA_WORD_BARRETT_FULL) return MOMA_ERR_INVALID_ARG;
  if (engine < 0 || engine > 3) return MOMA_ERR_INVALID_ARG;
  if (n == 0) return MOMA_OK;
  if (n > ((size_t)1 << 30)) return MOMA_ERR_SIZE;
  if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)out) & 3u) return MOMA_ERR_ALIGN;
  const bool needs_full = op == MOMA_WORD_MONT || op == MOMA_WORD_BARRETT_FULL;
  if (op >= MOMA_WORD_BARRETT && needs_full != ctx->mont) return MOMA_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  switch (ctx->L) {
    case 2: return run_words<2>(ctx, op, engine, n, a, b, out, st);
    case 4: return run_words<4>(ctx, op, engine, n, a, b, out, st);
    case 8: return run_words<8>(ctx, op, engine, n, a, b, out, st);
    case 12: return run_words<12>(ctx, op, engine, n, a, b, out, st);
    default: return run_words_wide(ctx, op, engine, n, a, b, out, st);
  }
}
