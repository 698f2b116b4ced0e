// moma_consts.cuh -- the per-modulus constants of a context as the kernels receive them.
#pragma once
#include "moma_internal.hpp"
#include "moma_limbs.cuh"

namespace moma {

// Kernel-parameter copy of the context's constants (Barrett and, for full-width contexts,
// Montgomery fields).
template <int L>
inline void fill_modk(const moma_ctx* ctx, ModK<L>& k) {
  for (int i = 0; i < L; ++i) {
    k.q[i] = ctx->k.q[i];
    k.nq[i] = ctx->k.nq[i];
    k.mu[i] = ctx->k.mu[i];
    k.q2[i] = ctx->k.q2[i];
    k.q4[i] = ctx->k.q4[i];
    k.r2[i] = ctx->k.r2[i];
  }
  k.qinv = ctx->k.qinv;
  k.mu_hi = ctx->k.mu_hi;
  k.q2_hi = ctx->k.q2_hi;
}

}  // namespace moma
