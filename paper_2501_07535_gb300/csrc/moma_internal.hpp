// moma_internal.hpp -- context, plans and launcher declarations shared by the .cu files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/moma.h"
#include "moma_bigint.hpp"

namespace moma {

constexpr int kMaxL = 32;
constexpr int kMaxLogN = 24;

// Host copy of the per-modulus constants (device code receives ModK<L> by value).
struct HostConsts {
  int L = 0;
  uint32_t q[kMaxL] = {}, nq[kMaxL] = {}, mu[kMaxL] = {}, q2[kMaxL] = {}, q4[kMaxL] = {};
  uint32_t R0[kMaxL] = {};  // 2^(32L) mod q
  uint32_t Q0 = 0;          // floor(2^(32L) / q)  (between 16 and 31 for a W-4 bit q)
  uint32_t r2[kMaxL] = {};  // full-width contexts: 2^(64L) mod q
  uint32_t qinv = 0;        // full-width contexts: -q^-1 mod 2^32
  uint32_t mu_hi = 0;       // full-width contexts: word L of floor(2^(64L) / q)
  uint32_t q2_hi = 0;       // full-width contexts: word L of 2q
};

// One Stockham pass: radix 2^logR over groups of stride n/R, after logNs radix bits.
struct PassDesc {
  int logR = 0, logNs = 0, logG = 0;
  uint32_t* tw_pass = nullptr;  // [2L][tw_count], null when Ns == 1
  uint32_t* tw_int = nullptr;   // [2L][R/2]
  uint64_t tw_count = 0;
};

struct Plan {
  int logn = 0;
  bool inverse = false;
  bool negacyclic = false;
  int max_logr = 0;
  uint32_t* psi = nullptr;  // negacyclic: [n][2L] psi^e (forward) or n^-1 psi^-e (inverse)
  std::vector<PassDesc> passes;
  uint32_t* d_tables = nullptr;  // one allocation holding every table of the plan
  size_t table_bytes = 0;         // its size
  uint32_t scale[kMaxL] = {}, scalep[kMaxL] = {};  // n^-1 and its companion (inverse)
  int tile_log = 0;                                // log2 of the CTA tile (elements)
};

}  // namespace moma

struct moma_ctx {
  int L = 0;
  int bits = 0;
  bool mont = false;  // full-width modulus: Montgomery reduction, canonical values
  int device = 0;
  int num_sms = 0;
  moma::HostConsts k;
  moma::BigU Q;
  moma::Reducer* red = nullptr;  // host reductions mod q
  // transform state, filled on first use
  mutable std::mutex lock;  // guards plans, configs and the transform state
  int ntt_ready = 0;  // 0: not yet, 1: ok, -1: modulus not prime
  uint32_t g = 0;     // smallest quadratic non-residue
  int two_adicity = 0;
  // (logn, inverse, tile_log, max_logr, negacyclic) -> plan
  std::map<std::tuple<int, int, int, int, int>, moma::Plan*> plans;
  // schedule per (op, logn) for transforms, (op, -1) for BLAS; absent = defaults
  std::map<std::pair<int, int>, moma_config> configs;
  int* d_status = nullptr;  // device-side error word
  // bound of one wait of the staged BLAS kernels on a shared-memory stage (ns of global time)
  uint64_t wait_ns = 2000000000ull;
  // test hook: the next staged BLAS launch makes one wait run out (moma_ctx_inject_missing_copy)
  std::atomic<int> inject_missing_copy{0};
};

namespace moma {

// Status helpers
inline moma_status cuda_status(cudaError_t e) { return e == cudaSuccess ? MOMA_OK : MOMA_ERR_CUDA; }

// moma_blas.cu
enum VecOp { VEC_ADD = 0, VEC_SUB = 1, VEC_MUL = 2, VEC_AXPY = 3 };
int vec_max_width(int L);
int vec_max_log_tile(int L);  // largest staged tile (log2 elements) for L limbs, 0 if none
moma_config vec_config(const moma_ctx* ctx, int vec_op);  // effective (defaults filled)
moma_status launch_vec(moma_ctx* ctx, int op, size_t n, const uint32_t* a, const uint32_t* b,
                       uint32_t* c, const uint32_t* alpha_host, cudaStream_t st);
moma_status launch_vec_cfg(moma_ctx* ctx, int op, size_t n, const uint32_t* a, const uint32_t* b,
                           uint32_t* c, const uint32_t* alpha_host, const moma_config& cfg, cudaStream_t st);
// moma_blas_wide.cu: 512-, 768- and 1024-bit contexts
moma_status launch_vec_wide(moma_ctx* ctx, int op, size_t n, const uint32_t* a, const uint32_t* b,
                            uint32_t* c, const uint32_t* alpha_host, const moma_config& cfg, cudaStream_t st);

// moma_ntt.cu
int default_tile_log(int L);
int max_tile_log(int L);                 // shared-memory limit
// Effective schedule (defaults filled) for `count` transforms of 2^logn points in one call; count 0:
// the default for large batches (persistent batch tiles).
moma_config ntt_config(const moma_ctx* ctx, int op, int logn, size_t count = 0);
bool ntt_config_valid(int L, int logn, const moma_config& c);
moma_status ntt_prepare(moma_ctx* ctx);  // primality, generator (takes ctx->lock)
moma_status get_plan(moma_ctx* ctx, int logn, bool inverse, int tile_log, int max_logr, Plan** out,
                     bool negacyclic = false);
moma_status launch_ntt(moma_ctx* ctx, int logn, size_t count, bool inverse, const uint32_t* in,
                       uint32_t* out, cudaStream_t st);
moma_status launch_ntt_cfg(moma_ctx* ctx, int logn, size_t count, bool inverse, const uint32_t* in,
                           uint32_t* out, const moma_config& cfg, cudaStream_t st, bool negacyclic = false);
moma_status launch_polymul(moma_ctx* ctx, int logn, const uint32_t* a, const uint32_t* b,
                           uint32_t* c, cudaStream_t st);
moma_status launch_polymul_cfg(moma_ctx* ctx, int logn, const uint32_t* a, const uint32_t* b,
                               uint32_t* c, const moma_config& cfg, cudaStream_t st, bool negacyclic = false);
void free_plan(Plan* p);
// moma_ntt_wide.cu: passes and twiddle tables of 512-, 768- and 1024-bit contexts
moma_status run_pass_wide(moma_ctx* ctx, const Plan* pl, const PassDesc& d, size_t count, const uint32_t* src,
                          const uint32_t* src2, uint32_t* dst, uint32_t flags, const moma_config& cfg,
                          cudaStream_t st);
moma_status gen_table_wide(const moma_ctx* ctx, uint32_t* dst, uint64_t count, uint64_t D, uint64_t C, uint64_t S,
                           int logn, const std::vector<BigU>& pw, const BigU& init);
// Every pass of a plan with caller-provided intermediate buffers (s1, s2: count*L*n words each;
// s1 may be null for a one-pass plan, s2 for plans of up to two passes).
moma_status run_plan_buffers(moma_ctx* ctx, const Plan* pl, size_t count, const uint32_t* in, const uint32_t* in2,
                             uint32_t* out, const moma_config& cfg, uint32_t* s1, uint32_t* s2, cudaStream_t st);
// moma_words_wide.cu: the word-level block probe of 512- and 768-bit contexts
moma_status run_words_wide(moma_ctx* ctx, int op, int engine, size_t n, const uint32_t* a, const uint32_t* b,
                           uint32_t* out, cudaStream_t st);
// Existing plan or null; never builds one (no allocation).
Plan* find_plan(moma_ctx* ctx, int logn, bool inverse, int tile_log, int max_logr);
// moma_noalloc.cu: look up the device address of the fixed scratch array on device `dev`
// (current), once per device; called when a context is created.
moma_status noalloc_prepare(int dev);
BigU root_of_unity(moma_ctx* ctx, int logn);  // requires ntt_prepare()

// Shoup-style companion floor(w * 2^(32L) / q) for a host constant w < q.
void companion(const moma_ctx* ctx, const BigU& w, uint32_t* out);

}  // namespace moma
