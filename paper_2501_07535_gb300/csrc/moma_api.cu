// moma_api.cu -- the extern "C" entry points declared in include/moma.h.
//
// Argument checking and marshalling only; all arithmetic on vectors runs in the kernels
// of moma_blas.cu and moma_ntt.cu.  Host work here is per modulus (constants) or per call
// (scalar companions, plan look-up).
#include <new>

#include "moma_internal.hpp"

using namespace moma;

extern "C" {

const char* moma_status_string(moma_status s) {
  switch (s) {
    case MOMA_OK: return "MOMA_OK";
    case MOMA_ERR_INVALID_ARG: return "MOMA_ERR_INVALID_ARG";
    case MOMA_ERR_MODULUS: return "MOMA_ERR_MODULUS";
    case MOMA_ERR_SIZE: return "MOMA_ERR_SIZE";
    case MOMA_ERR_ALIGN: return "MOMA_ERR_ALIGN";
    case MOMA_ERR_OOM: return "MOMA_ERR_OOM";
    case MOMA_ERR_CUDA: return "MOMA_ERR_CUDA";
    case MOMA_ERR_TIMEOUT: return "MOMA_ERR_TIMEOUT";
    case MOMA_ERR_BUDGET: return "MOMA_ERR_BUDGET";
    case MOMA_ERR_UNSUPPORTED: return "MOMA_ERR_UNSUPPORTED";
  }
  return "MOMA_ERR_UNKNOWN";
}

// Common set-up of both context kinds.  mont: a full-width modulus reduced by Montgomery
// products (Sec. 5.2); otherwise a (W-4)-bit modulus with the Barrett constants of Sec. 3.1.
static moma_status ctx_create(const uint32_t* q, int bits, bool mont, moma_ctx** out) {
  if (!out) return MOMA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!q) return MOMA_ERR_INVALID_ARG;
  if (bits != 64 && bits != 128 && bits != 256 && bits != 384 && bits != 512 && bits != 768 && bits != 1024)
    return MOMA_ERR_INVALID_ARG;
  const int L = bits / 32;
  BigU Q = BigU::from_words(q, L);
  if (!Q.is_odd()) return MOMA_ERR_MODULUS;  // odd: needed by every reduction
  if (mont ? Q.bits() <= bits - 32 : Q.bits() != bits - 4) return MOMA_ERR_MODULUS;
  moma_ctx* c = new (std::nothrow) moma_ctx();
  if (!c) return MOMA_ERR_OOM;
  c->L = L;
  c->bits = bits;
  c->mont = mont;
  c->Q = Q;
  c->red = new Reducer(Q);
  c->k.L = L;
  BigU W = pow2(bits);
  BigU Q0, R0;
  divmod(W, Q, &Q0, &R0);
  Q.to_words(c->k.q, L);
  R0.to_words(c->k.R0, L);
  c->k.Q0 = Q0.word(0);
  if (mont) {
    c->red->mulmod(R0, R0).to_words(c->k.r2, L);  // R^2 mod q
    uint32_t inv = q[0];  // q^-1 mod 2^32 by Newton's iteration (q odd: q*q = 1 mod 8 to start)
    for (int i = 0; i < 5; ++i) inv *= 2u - q[0] * inv;
    c->k.qinv = 0u - inv;
    // word-based Barrett for products of two vectors: mu = floor(2^(64L) / q) (L+1 words),
    // 2^(32L) - q and 2q (L+1 words)
    BigU mu, q2 = add(Q, Q);
    divmod(pow2(2 * bits), Q, &mu, nullptr);
    sub(W, Q).to_words(c->k.nq, L);
    mu.to_words(c->k.mu, L);
    c->k.mu_hi = mu.word((size_t)L);
    q2.to_words(c->k.q2, L);
    c->k.q2_hi = q2.word((size_t)L);
  } else {
    const int B = bits - 4;
    BigU nq = sub(W, Q);
    BigU mu;
    divmod(pow2(2 * B + 3), Q, &mu, nullptr);  // Eq. mu with k = 2B+3
    BigU q2 = add(Q, Q);
    BigU q4 = add(q2, q2);
    nq.to_words(c->k.nq, L);
    mu.to_words(c->k.mu, L);
    q2.to_words(c->k.q2, L);
    q4.to_words(c->k.q4, L);
  }
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c->red;
    delete c;
    return MOMA_ERR_CUDA;
  }
  if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess) {
    delete c->red;
    delete c;
    return MOMA_ERR_OOM;
  }
  // the fixed scratch array of moma_ntt_fwd_noalloc is placed on this device now (module load),
  // not in that entry point's first call
  if (noalloc_prepare(c->device) != MOMA_OK) {
    cudaFree(c->d_status);
    delete c->red;
    delete c;
    return MOMA_ERR_CUDA;
  }
  cudaMemset(c->d_status, 0, sizeof(int));
  *out = c;
  return MOMA_OK;
}

moma_status moma_ctx_create(const uint32_t* q, int bits, moma_ctx** out) {
  return ctx_create(q, bits, false, out);
}

moma_status moma_ctx_create_full(const uint32_t* q, int bits, moma_ctx** out) {
  return ctx_create(q, bits, true, out);
}

int moma_ctx_is_full(const moma_ctx* ctx) { return ctx && ctx->mont ? 1 : 0; }

void moma_ctx_destroy(moma_ctx* ctx) {
  if (!ctx) return;
  for (auto& kv : ctx->plans) free_plan(kv.second);
  if (ctx->d_status) cudaFree(ctx->d_status);
  delete ctx->red;
  delete ctx;
}

int moma_ctx_limbs(const moma_ctx* ctx) { return ctx ? ctx->L : 0; }

size_t moma_ctx_device_bytes(const moma_ctx* ctx) {
  if (!ctx) return 0;
  std::lock_guard<std::mutex> g(ctx->lock);
  size_t b = sizeof(int);  // the status word
  for (const auto& kv : ctx->plans) b += kv.second->table_bytes;
  return b;
}

static int log2_exact(size_t n) {
  if (n == 0 || (n & (n - 1))) return -1;
  int k = 0;
  while (((size_t)1 << k) < n) ++k;
  return k;
}

moma_status moma_ctx_root(moma_ctx* ctx, size_t n, uint32_t* w_out) {
  if (!ctx || !w_out) return MOMA_ERR_INVALID_ARG;
  int lg = log2_exact(n);
  if (lg < 1 || lg > kMaxLogN) return MOMA_ERR_SIZE;
  moma_status st = ntt_prepare(ctx);
  if (st) return st;
  if (lg > ctx->two_adicity) return MOMA_ERR_SIZE;
  root_of_unity(ctx, lg).to_words(w_out, ctx->L);
  return MOMA_OK;
}

moma_status moma_ctx_sync_status(moma_ctx* ctx) {
  if (!ctx) return MOMA_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return MOMA_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MOMA_ERR_CUDA;
  if (v) cudaMemset(ctx->d_status, 0, sizeof(int));
  return (moma_status)v;
}

moma_status moma_ctx_set_wait_limit(moma_ctx* ctx, uint64_t ns) {
  if (!ctx || ns == 0) return MOMA_ERR_INVALID_ARG;
  ctx->wait_ns = ns;
  return MOMA_OK;
}

moma_status moma_ctx_inject_missing_copy(moma_ctx* ctx) {
  if (!ctx) return MOMA_ERR_INVALID_ARG;
  ctx->inject_missing_copy.store(1);
  return MOMA_OK;
}

static bool aligned4(const void* p) { return ((uintptr_t)p & 3u) == 0; }

static moma_status vec_call(moma_ctx* ctx, int op, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                            const uint32_t* alpha, void* stream) {
  if (!ctx) return MOMA_ERR_INVALID_ARG;
  if (n == 0) return MOMA_OK;
  if (!a || !b || !c || (op == VEC_AXPY && !alpha)) return MOMA_ERR_INVALID_ARG;
  if (!aligned4(a) || !aligned4(b) || !aligned4(c)) return MOMA_ERR_ALIGN;
  if (n > ((size_t)1 << 40)) return MOMA_ERR_SIZE;
  return launch_vec(ctx, op, n, a, b, c, alpha, (cudaStream_t)stream);
}

moma_status moma_vec_addmod(moma_ctx* ctx, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                            void* stream) {
  return vec_call(ctx, VEC_ADD, n, a, b, c, nullptr, stream);
}

moma_status moma_vec_submod(moma_ctx* ctx, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                            void* stream) {
  return vec_call(ctx, VEC_SUB, n, a, b, c, nullptr, stream);
}

moma_status moma_vec_mulmod(moma_ctx* ctx, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                            void* stream) {
  return vec_call(ctx, VEC_MUL, n, a, b, c, nullptr, stream);
}

moma_status moma_vec_axpymod(moma_ctx* ctx, size_t n, const uint32_t* alpha, const uint32_t* x, const uint32_t* y,
                             uint32_t* out, void* stream) {
  return vec_call(ctx, VEC_AXPY, n, x, y, out, alpha, stream);
}

static moma_status ntt_call(moma_ctx* ctx, size_t n, size_t count, bool inverse, const uint32_t* in, uint32_t* out,
                            void* stream) {
  if (!ctx || !in || !out) return MOMA_ERR_INVALID_ARG;
  if (!aligned4(in) || !aligned4(out)) return MOMA_ERR_ALIGN;
  int lg = log2_exact(n);
  if (lg < 1 || lg > kMaxLogN) return MOMA_ERR_SIZE;
  if (count > ((size_t)1 << 20)) return MOMA_ERR_SIZE;
  return launch_ntt(ctx, lg, count, inverse, in, out, (cudaStream_t)stream);
}

moma_status moma_ntt_fwd(moma_ctx* ctx, size_t n, const uint32_t* in, uint32_t* out, void* stream) {
  return ntt_call(ctx, n, 1, false, in, out, stream);
}

moma_status moma_ntt_inv(moma_ctx* ctx, size_t n, const uint32_t* in, uint32_t* out, void* stream) {
  return ntt_call(ctx, n, 1, true, in, out, stream);
}

moma_status moma_ntt_fwd_many(moma_ctx* ctx, size_t n, size_t count, const uint32_t* in, uint32_t* out,
                              void* stream) {
  return ntt_call(ctx, n, count, false, in, out, stream);
}

moma_status moma_ntt_inv_many(moma_ctx* ctx, size_t n, size_t count, const uint32_t* in, uint32_t* out,
                              void* stream) {
  return ntt_call(ctx, n, count, true, in, out, stream);
}

moma_status moma_polymul(moma_ctx* ctx, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c, void* stream) {
  if (!ctx || !a || !b || !c) return MOMA_ERR_INVALID_ARG;
  if (!aligned4(a) || !aligned4(b) || !aligned4(c)) return MOMA_ERR_ALIGN;
  int lg = log2_exact(n);
  if (lg < 1 || lg > kMaxLogN) return MOMA_ERR_SIZE;
  return launch_polymul(ctx, lg, a, b, c, (cudaStream_t)stream);
}

static moma_status nega_ntt_call(moma_ctx* ctx, size_t n, size_t count, bool inverse, const uint32_t* in,
                                 uint32_t* out, void* stream) {
  if (!ctx || !in || !out) return MOMA_ERR_INVALID_ARG;
  if (!aligned4(in) || !aligned4(out)) return MOMA_ERR_ALIGN;
  int lg = log2_exact(n);
  if (lg < 1 || lg > kMaxLogN) return MOMA_ERR_SIZE;
  if (count > ((size_t)1 << 20)) return MOMA_ERR_SIZE;
  return launch_ntt_cfg(ctx, lg, count, inverse, in, out,
                        ntt_config(ctx, inverse ? MOMA_OP_NTT_INV : MOMA_OP_NTT_FWD, lg, count), (cudaStream_t)stream,
                        true);
}

moma_status moma_ntt_fwd_negacyclic(moma_ctx* ctx, size_t n, size_t count, const uint32_t* in, uint32_t* out,
                                    void* stream) {
  return nega_ntt_call(ctx, n, count, false, in, out, stream);
}

moma_status moma_ntt_inv_negacyclic(moma_ctx* ctx, size_t n, size_t count, const uint32_t* in, uint32_t* out,
                                    void* stream) {
  return nega_ntt_call(ctx, n, count, true, in, out, stream);
}

moma_status moma_polymul_negacyclic(moma_ctx* ctx, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                                    void* stream) {
  if (!ctx || !a || !b || !c) return MOMA_ERR_INVALID_ARG;
  if (!aligned4(a) || !aligned4(b) || !aligned4(c)) return MOMA_ERR_ALIGN;
  int lg = log2_exact(n);
  if (lg < 1 || lg > kMaxLogN) return MOMA_ERR_SIZE;
  return launch_polymul_cfg(ctx, lg, a, b, c, ntt_config(ctx, MOMA_OP_POLYMUL, lg, 1), (cudaStream_t)stream, true);
}

}  // extern "C"
