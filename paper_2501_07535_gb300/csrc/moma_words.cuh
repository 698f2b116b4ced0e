// moma_words.cuh -- the word-level building blocks of the multi-word arithmetic, one element per
// thread, with their raw outputs (before any final reduction), so that tests can check each
// block against plain integer arithmetic and against the bounds the method relies on:
//   - add_words / sub_words: the sum with its carry word and the difference with its borrow
//     (rules (addqdd), (adc), (subddd) of Table 1, the recursion of Sec. 3.2);
//   - the double-width product by each product engine (schoolbook carry chains, whole products,
//     Karatsuba; Sec. 2.2 Eq. muls / Eq. mulk, rule (mulqdd));
//   - the truncated high half of a product (the Barrett quotient estimate), exact or one less;
//   - Barrett reduction of a*b with the flag of its final correction (Sec. 3.1 Eq. barrett: one
//     correction suffices for a (W-4)-bit modulus);
//   - the fixed-multiplicand product before its corrections (a value in [0, 3q));
//   - the Montgomery product a b R^-1 mod q (full-width contexts);
//   - the word-based Barrett reduction of full-width contexts: r before its two subtractions
//     (L+1 words, below 4q) and the reduced product.
// moma_words.cu instantiates them up to 384 bits, moma_words_wide.cu from 512 bits.
#pragma once
#include "moma_consts.cuh"
#include "moma_internal.hpp"
#include "moma_limbs.cuh"

namespace moma {

template <int L>
struct WordArgs {
  const uint32_t* a;
  const uint32_t* b;
  uint32_t* out;  // [2L + 1][n]
  uint64_t n;
  int op, engine;
  uint32_t w[L], wp[L];  // MOMA_WORD_FIXED: the multiplicand b[0] and its companion
  ModK<L> k;
};

template <int L>
__global__ void __launch_bounds__(256) word_kernel(const __grid_constant__ WordArgs<L> p) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  uint32_t a[L], b[L], o[2 * L + 1];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    a[l] = p.a[i + (uint64_t)l * p.n];
    b[l] = p.b[i + (uint64_t)l * p.n];
  }
#pragma unroll
  for (int l = 0; l < 2 * L + 1; ++l) o[l] = 0u;
  switch (p.op) {
    case MOMA_WORD_ADD: {
      uint32_t c[L];
      add_words<L, false>(c, a, b);
      o[L] = carry_out();
#pragma unroll
      for (int l = 0; l < L; ++l) o[l] = c[l];
      break;
    }
    case MOMA_WORD_SUB: {
      uint32_t c[L];
      sub_words<L, false>(c, a, b);
      o[L] = borrow_mask() & 1u;
#pragma unroll
      for (int l = 0; l < L; ++l) o[l] = c[l];
      break;
    }
    case MOMA_WORD_MUL: {
      uint32_t t[2 * L];
      if (p.engine == 3) mul_full_k<L>(t, a, b);
      else if (p.engine == 2) mul_full_w<L>(t, a, b);
      else mul_full<L>(t, a, b);
#pragma unroll
      for (int l = 0; l < 2 * L; ++l) o[l] = t[l];
      break;
    }
    case MOMA_WORD_MUL_HI: {
      uint32_t h[L];
      if (p.engine == 2) mul_hi_trunc_w<L>(h, a, b);
      else mul_hi_trunc<L>(h, a, b);
#pragma unroll
      for (int l = 0; l < L; ++l) o[l] = h[l];
      break;
    }
    case MOMA_WORD_BARRETT: {
      uint32_t t[2 * L], c[L], s[L];
      mul_full<L>(t, a, b);
      const uint32_t fired = p.engine == 2 ? barrett_reduce<L, true>(c, s, t, p.k) : barrett_reduce<L, false>(c, s, t, p.k);
#pragma unroll
      for (int l = 0; l < L; ++l) o[l] = c[l];
      o[L] = fired;
      break;
    }
    case MOMA_WORD_FIXED: {
      uint32_t r[L];
      if (p.engine == 2) mulmod_fixed_lazy<L, 2>(r, a, p.w, p.wp, p.k);
      else mulmod_fixed_lazy<L, 1>(r, a, p.w, p.wp, p.k);
#pragma unroll
      for (int l = 0; l < L; ++l) o[l] = r[l];
      break;
    }
    case MOMA_WORD_BARRETT_FULL: {
      uint32_t t[2 * L], c[L], r[L + 1];
      if (p.engine == 3) mul_full_k<L>(t, a, b);
      else if (p.engine == 2) mul_full_w<L>(t, a, b);
      else mul_full<L>(t, a, b);
      barrett_reduce_full<L>(c, r, t, p.k);
#pragma unroll
      for (int l = 0; l <= L; ++l) o[l] = r[l];
#pragma unroll
      for (int l = 0; l < L; ++l) o[L + 1 + l] = c[l];
      break;
    }
    default: {  // MOMA_WORD_MONT
      uint32_t c[L];
      montmul<L>(c, a, b, p.k);
#pragma unroll
      for (int l = 0; l < L; ++l) o[l] = c[l];
    }
  }
#pragma unroll
  for (int l = 0; l < 2 * L + 1; ++l) p.out[i + (uint64_t)l * p.n] = o[l];
}

template <int L>
moma_status run_words(moma_ctx* ctx, int op, int engine, size_t n, const uint32_t* a, const uint32_t* b,
                             uint32_t* out, cudaStream_t st) {
  WordArgs<L> p;
  p.a = a;
  p.b = b;
  p.out = out;
  p.n = n;
  p.op = op;
  p.engine = engine;
  fill_modk<L>(ctx, p.k);
  for (int l = 0; l < L; ++l) p.w[l] = p.wp[l] = 0u;
  if (op == MOMA_WORD_FIXED) {  // the multiplicand is b[0]; its companion comes from the host
    uint32_t w0[L];
    for (int l = 0; l < L; ++l) {
      if (cudaMemcpy(&w0[l], b + (size_t)l * n, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return MOMA_ERR_CUDA;
    }
    const BigU w = BigU::from_words(w0, L);
    if (cmp(w, ctx->Q) >= 0) return MOMA_ERR_INVALID_ARG;
    for (int l = 0; l < L; ++l) p.w[l] = w0[l];
    companion(ctx, w, p.wp);
  }
  const unsigned blocks = (unsigned)((n + 255) / 256);
  word_kernel<L><<<blocks, 256, 0, st>>>(p);
  return cuda_status(cudaGetLastError());
}

}  // namespace moma

