// moma_ntt.cu -- forward/inverse cyclic NTT (Sec. 2.3 Eq. ntt) as Stockham radix-2^k passes.
//
// Pass p (radix R = 2^logR, after Ns = 2^logNs radix points already combined) computes,
// for every group j in [0, n/R) with k = j mod Ns,
//     v[r]  = in[j + r*n/R] * w_(Ns*R)^(r*k)          r = 0..R-1   (pre-twiddle)
//     V     = DFT_R(v)                                 (R-point NTT, w_R = w_n^(n/R))
//     out[(j-k)*R + k + s*Ns] = V[s]                   s = 0..R-1
// so that natural order is kept in and out (Stockham autosort).  One CTA owns G
// consecutive groups: it reads G-element runs of each of the R strided rows (coalesced),
// holds the [R][G] tile of every limb plane in shared memory, runs the R-point transform
// as logR in-place radix-2 decimation-in-frequency stages (butterfly (a, b) ->
// (a + b, (a - b) * w), one addmod, one submod, one mulmod: the butterfly of Sec. 5.3),
// and writes the outputs back in contiguous runs.  DIF leaves each group's outputs in
// bit-reversed position inside the tile; the store reads them through the bit reversal.
// Twiddles equal to 1 are not multiplied: the whole last DIF stage, the first butterfly of
// every block in the other stages, the k = 0 pre-twiddles and all of the first pass (Ns = 1).
//
// Values are kept lazily reduced inside a transform: every stage maps [0, 4q) to [0, 4q)
// (the 4-bit headroom of a (W-4)-bit modulus keeps 8q below 2^W), and the last pass makes
// its outputs canonical as it stores them.  Inputs must be canonical.
//
// Twiddles are in the reduction's domain: every table entry w carries its companion
// floor(w * 2^(32L) / q), so a twiddle multiplication needs no double-width product
// (mulmod_fixed).  Tables are built on the device once per (modulus, size, direction) and
// stored entry-major, [entry][w limbs | companion limbs], 16-byte aligned per entry.
#include <algorithm>

#include "moma_internal.hpp"
#include "moma_limbs.cuh"
#include "moma_ntt_pass.cuh"
#include "moma_ntt_tile.cuh"

namespace moma {

// Default schedule per width, the fastest measured on GB300 for 2^20-point transforms in
// batches (see the autotuner for other sizes): 128-thread CTAs on 2^10-element tiles with radix
// up to 2^5 through 384 bits (the 384-bit kernel capped at 102 registers), 256-thread CTAs on
// 2^11 tiles with radix 2^7 at 768 bits; the wide engine through 384 bits, carry chains above.
// The ends of the paper's width sweep: 2^12 tiles with radix up to 2^7 at 64 bits (three passes for
// 2^20 points: 10% faster than four); 2^9 tiles at 512 and 1024 bits, so
// that two of their CTAs (up to 255 registers per thread) fit an SM (1024 bits: 217 against 425 us
// for a 2^16-point transform with 2^10 tiles; 512 bits: 8% faster).
struct NttDefaults {
  int engine, tile_log, max_logr, threads, tight;
};
static NttDefaults ntt_defaults(int L) {
  switch (L) {
    case 2: return {2, 12, 7, 256, 0};
    case 4: return {2, 10, 5, 128, 0};
    case 8: return {2, 10, 5, 128, 0};
    case 12: return {2, 10, 5, 128, 1};
    case 16: return {1, 9, 5, 128, 0};
    case 24: return {1, 11, 7, 256, 0};
    default: return {1, 9, 5, 128, 0};
  }
}
int default_tile_log(int L) { return ntt_defaults(L).tile_log; }

// Calls with little work (count * n <= 2^19 points, 128 to 384 bits): 2^9-element tiles, so that
// the call has twice as many CTAs as with 2^10 tiles.  Up to 2^18 points 256-thread CTAs (two
// elements, one butterfly per thread per stage) and radix up to 2^6; at 2^19 points 128-thread CTAs
// with the register cap and radix up to 2^5.  Measured on GB300 for single transforms: 2^16 points
// 0.042 against 0.082 ms with the batch default at 256 bits, 0.059 against 0.119 ms at 384 bits,
// 0.037 against 0.058 ms at 128 bits; 2^18 points 3-22% faster; from 2^20 points the batch default
// is as fast or faster.
// At 768 bits (one 256-thread CTA per SM) a call of up to 2^16 points takes 2^9 tiles with radix up
// to 2^7 and one of 2^17 points 2^10 tiles with radix up to 2^6: a CTA's latency sets the time of
// such a call, and smaller tiles spread it over more SMs.  Measured on GB300: 2^12 points 0.110
// against 0.310 ms, 2^16 points 0.160 against 0.441 ms (also 2^12 x 16 transforms: 0.111 against
// 0.309 ms), 2^17 points 0.280 against 0.468 ms; from 2^18 points the 2^11 tiles are as fast or
// faster (within 5% either way up to 2^22).
static int work_log(int logn, size_t count) {  // ceil(log2(count * n)); -1 when count is unknown (0)
  if (count == 0) return -1;
  return logn + (count > 1 ? 64 - __builtin_clzll((unsigned long long)(count - 1)) : 0);
}
static bool small_work_default(int L, int logn, size_t count, NttDefaults& d) {
  const int wl = work_log(logn, count);
  if (wl < 0) return false;
  if (L == 4 || L == 8 || L == 12) {
    if (wl > 19) return false;
    d = wl <= 18 ? NttDefaults{2, 9, 6, 256, 0} : NttDefaults{2, 9, 5, 128, 1};
    return true;
  }
  if (L == 24) {
    if (wl > 17) return false;
    d = wl <= 16 ? NttDefaults{1, 9, 7, 256, 0} : NttDefaults{1, 10, 6, 256, 0};
    return true;
  }
  return false;
}

// Largest tile that fits the 227 KiB of shared memory one CTA may use.
int max_tile_log(int L) {
  int t = 5;
  while ((size_t)L * 4u << (t + 1) <= 227u * 1024u) ++t;
  return t;
}

moma_config ntt_config(const moma_ctx* ctx, int op, int logn, size_t count) {
  moma_config c = {0, 0, 0, 0, 0, 0};
  bool set = false;
  {
    std::lock_guard<std::mutex> g(ctx->lock);  // moma_ctx_set_config may write the map meanwhile
    auto it = ctx->configs.find(std::make_pair(op, logn));
    if (it != ctx->configs.end()) {
      c = it->second;
      set = true;
    }
  }
  NttDefaults d = ntt_defaults(ctx->L);
  if (!set && !ctx->mont) small_work_default(ctx->L, logn, count, d);
  if (c.engine == 0) c.engine = d.engine;
  if (c.tile_log == 0) c.tile_log = d.tile_log;
  if (c.max_logr == 0) c.max_logr = c.tile_log == d.tile_log ? d.max_logr : (c.tile_log > 6 ? c.tile_log - 5 : 1);
  if (c.cta_threads == 0) c.cta_threads = d.threads;
  if (!set && c.cta_threads <= 128) c.tight_regs = d.tight;
  c.vec_width = 0;
  return c;
}

bool ntt_config_valid(int L, int logn, const moma_config& c) {
  (void)logn;
  if (c.engine < 0 || c.engine > 2) return false;
  if (c.tile_log != 0 && (c.tile_log < 5 || c.tile_log > max_tile_log(L))) return false;
  if (c.max_logr < 0 || (c.max_logr != 0 && c.tile_log != 0 && c.max_logr > c.tile_log)) return false;
  if (c.cta_threads != 0 && c.cta_threads != 32 && c.cta_threads != 64 && c.cta_threads != 128 &&
      c.cta_threads != 256)
    return false;
  if (c.tight_regs != 0 && (c.tight_regs != 1 || c.cta_threads > 128)) return false;
  return true;
}

static moma_status gen_table_l(const moma_ctx* ctx, uint32_t* dst, uint64_t count, uint64_t D, uint64_t C,
                               uint64_t S, int logn, const std::vector<BigU>& pw, const BigU& init = BigU(1)) {
  switch (ctx->L) {
    case 2: return gen_table<2>(ctx, dst, count, D, C, S, logn, pw, init);
    case 4: return gen_table<4>(ctx, dst, count, D, C, S, logn, pw, init);
    case 8: return gen_table<8>(ctx, dst, count, D, C, S, logn, pw, init);
    case 12: return gen_table<12>(ctx, dst, count, D, C, S, logn, pw, init);
    default: return gen_table_wide(ctx, dst, count, D, C, S, logn, pw, init);
  }
}

// ------------------------------------------------------------------ host set-up

moma_status ntt_prepare(moma_ctx* ctx) {
  std::lock_guard<std::mutex> g(ctx->lock);
  if (ctx->ntt_ready) return ctx->ntt_ready > 0 ? MOMA_OK : MOMA_ERR_MODULUS;
  if (!probably_prime(ctx->Q)) {
    ctx->ntt_ready = -1;
    return MOMA_ERR_MODULUS;
  }
  BigU one(1), qm1 = sub(ctx->Q, one), half = shr(qm1, 1);
  uint32_t gg = 2;
  while (cmp(ctx->red->powmod(BigU(gg), half), qm1) != 0) ++gg;
  ctx->g = gg;
  int s = 0;
  while (!qm1.bit(s)) ++s;
  ctx->two_adicity = s;
  ctx->ntt_ready = 1;
  return MOMA_OK;
}

BigU root_of_unity(moma_ctx* ctx, int logn) {
  BigU one(1), qm1 = sub(ctx->Q, one);
  return ctx->red->powmod(BigU(ctx->g), shr(qm1, logn));  // g^((q-1)/n)
}

void companion(const moma_ctx* ctx, const BigU& w, uint32_t* out) {
  BigU quo;
  ctx->red->divmod_(shl(w, 32 * ctx->L), &quo, nullptr);  // w*2^W < 2^(2B+4) < 2^k
  quo.to_words(out, ctx->L);
}

void free_plan(Plan* p) {
  if (!p) return;
  if (p->d_tables) cudaFree(p->d_tables);
  delete p;
}

static void split_passes(int logn, int max_logr, std::vector<int>& out) {
  int P = (logn + max_logr - 1) / max_logr;
  if (P < 1) P = 1;
  out.clear();
  for (int i = 0; i < P; ++i) out.push_back(logn / P + (i < logn % P ? 1 : 0));
}

static moma_status build_plan(moma_ctx* ctx, int logn, bool inverse, int tile_log, int max_logr, bool nega,
                              Plan** out) {
  const int L = ctx->L;
  Plan* pl = new Plan();
  pl->logn = logn;
  pl->inverse = inverse;
  pl->negacyclic = nega;
  pl->tile_log = tile_log;
  pl->max_logr = max_logr;
  const int T = pl->tile_log;
  std::vector<int> radices;
  if (logn <= T) {
    radices.push_back(logn);
  } else {
    split_passes(logn, max_logr, radices);
  }
  BigU w = root_of_unity(ctx, logn);
  if (inverse) w = ctx->red->powmod(w, sub(pow2(logn), BigU(1)));  // w^(n-1) = w^-1
  std::vector<BigU> pw;
  BigU cur = w;
  for (int b = 0; b < logn; ++b) {
    pw.push_back(cur);
    cur = ctx->red->mulmod(cur, cur);
  }
  // table sizes
  uint64_t words = 0;
  int logNs = 0;
  for (int lr : radices) {
    PassDesc d;
    d.logR = lr;
    d.logNs = logNs;
    d.logG = std::min(T - lr, logn - lr);
    d.tw_count = logNs > 0 ? (((uint64_t)1 << lr) - 1) << logNs : 0;
    words += 2ull * L * (d.tw_count + ((uint64_t)1 << (lr - 1)));
    pl->passes.push_back(d);
    logNs += lr;
  }
  if (nega) words += 2ull * L * (1ull << logn);  // psi table, one entry per position
  if (cudaMalloc(&pl->d_tables, words * 4) != cudaSuccess) {
    delete pl;
    return MOMA_ERR_OOM;
  }
  pl->table_bytes = words * 4;
  uint32_t* ptr = pl->d_tables;
  const uint64_t n = 1ull << logn;
  for (auto& d : pl->passes) {
    const uint64_t R = 1ull << d.logR;
    d.tw_int = ptr;
    // internal: w_R^e = w_n^(e * n/R), e < R/2
    moma_status st = gen_table_l(ctx, ptr, R / 2, ~0ull >> 1, 1, n / R, logn, pw);
    if (st) { free_plan(pl); return st; }
    ptr += 2ull * L * (R / 2);
    if (d.tw_count) {
      d.tw_pass = ptr;
      // pass: entry (r-1)*Ns + k holds w_(Ns*R)^(r*k) = w_n^(r*k * n/(Ns*R))
      const uint64_t Ns = 1ull << d.logNs;
      st = gen_table_l(ctx, ptr, d.tw_count, Ns, 1, n / (Ns * R), logn, pw);
      if (st) { free_plan(pl); return st; }
      ptr += 2ull * L * d.tw_count;
    }
  }
  BigU ninv = sub(ctx->Q, shr(sub(ctx->Q, BigU(1)), logn));  // n^-1 = q - (q-1)/n
  if (inverse) {
    if (ctx->mont) {  // n^-1 R mod q (Montgomery form); no companion
      ctx->red->mulmod(ninv, BigU::from_words(ctx->k.R0, L)).to_words(pl->scale, L);
    } else {
      ninv.to_words(pl->scale, L);
      companion(ctx, ninv, pl->scalep);
    }
  }
  if (nega) {
    // psi = primitive 2n-th root (psi^2 = w_n); forward table psi^e, inverse n^-1 psi^-e, e < n
    BigU psi = root_of_unity(ctx, logn + 1);
    if (inverse) psi = ctx->red->powmod(psi, sub(pow2(logn + 1), BigU(1)));  // psi^(2n-1) = psi^-1
    std::vector<BigU> ppw;
    BigU c2 = psi;
    for (int b = 0; b < logn; ++b) {
      ppw.push_back(c2);
      c2 = ctx->red->mulmod(c2, c2);
    }
    pl->psi = ptr;
    moma_status st = gen_table_l(ctx, ptr, 1ull << logn, ~0ull >> 1, 1, 1, logn, ppw, inverse ? ninv : BigU(1));
    if (st) { free_plan(pl); return st; }
    ptr += 2ull * L * (1ull << logn);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    free_plan(pl);
    return MOMA_ERR_CUDA;
  }
  *out = pl;
  return MOMA_OK;
}

moma_status get_plan(moma_ctx* ctx, int logn, bool inverse, int tile_log, int max_logr, Plan** out, bool nega) {
  moma_status st = ntt_prepare(ctx);
  if (st) return st;
  if (logn > ctx->two_adicity || logn < 1 || logn > kMaxLogN) return MOMA_ERR_SIZE;
  if (nega && logn + 1 > ctx->two_adicity) return MOMA_ERR_SIZE;  // needs a 2n-th root
  if (logn <= tile_log) max_logr = 0;  // single pass: the split does not matter
  std::lock_guard<std::mutex> g(ctx->lock);
  auto key = std::make_tuple(logn, inverse ? 1 : 0, tile_log, max_logr, nega ? 1 : 0);
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) {
    *out = it->second;
    return MOMA_OK;
  }
  Plan* pl = nullptr;
  st = build_plan(ctx, logn, inverse, tile_log, max_logr, nega, &pl);
  if (st) return st;
  ctx->plans[key] = pl;
  *out = pl;
  return MOMA_OK;
}

static moma_status run_pass_l(moma_ctx* ctx, const Plan* pl, const PassDesc& d, size_t count, const uint32_t* src,
                              const uint32_t* src2, uint32_t* dst, uint32_t flags, const moma_config& cfg,
                              cudaStream_t st) {
  switch (ctx->L) {
    case 2: return run_pass_for<2>(ctx, pl, d, count, src, src2, dst, flags, cfg, st);
    case 4: return run_pass_for<4>(ctx, pl, d, count, src, src2, dst, flags, cfg, st);
    case 8: return run_pass_for<8>(ctx, pl, d, count, src, src2, dst, flags, cfg, st);
    case 12: return run_pass_for<12>(ctx, pl, d, count, src, src2, dst, flags, cfg, st);
    default: return run_pass_wide(ctx, pl, d, count, src, src2, dst, flags, cfg, st);
  }
}

// Flags of pass i of P: the first pass can fuse a pointwise product with a second operand
// (polymul) and, for the inverse, the n^-1 scaling; negacyclic plans apply psi at the first load
// (forward) or the last store (inverse, which also carries n^-1); the last pass stores canonical
// values.
static uint32_t pass_flags(const Plan* pl, size_t i, size_t P, bool pointwise) {
  uint32_t flags = (i + 1 == P) ? F_LAST : 0;
  if (i == 0 && pointwise) flags |= F_POINTWISE;
  if (i == 0 && pl->inverse && !pl->negacyclic) flags |= F_SCALE;
  if (i == 0 && pl->negacyclic && !pl->inverse) flags |= F_PSI_IN;
  if (i + 1 == P && pl->negacyclic && pl->inverse) flags |= F_PSI_OUT;
  return flags;
}

// Calls whose two passes run in one cluster launch: a two-pass plan at 128 to 384 bits (Barrett
// contexts) whose n/T tiles fit one portable cluster, with both tiles of a CTA in shared memory,
// and little work in the call: count * n up to 2^16 points at 128 bits, 2^15 at 256 and 384.
// Measured on GB300 (2^10..2^12 points, 1..16 transforms per call, 200 calls back to back): one
// 2^12-point transform 20.5 against 23.3 us per call at 256 bits, 12.3 against 16.9 us at 128
// bits, 32.8 against 35.5 us at 384 bits; sixteen 2^12-point transforms at 256 bits 28.8 against
// 24.5 us (slower: 128 CTAs in clusters of 8).  Most of the gain is host time (one launch, no
// intermediate buffers to allocate); replayed from a CUDA graph the two forms are within 3%.
static int pair_work_log(int L) { return L == 4 ? 16 : 15; }
static bool pair_cluster_ok(const moma_ctx* ctx, const Plan* pl, size_t count) {
  if (ctx->mont || pl->passes.size() != 2) return false;
  if (ctx->L != 4 && ctx->L != 8 && ctx->L != 12) return false;
  const PassDesc& d0 = pl->passes[0];
  const PassDesc& d1 = pl->passes[1];
  const int logT = d0.logR + d0.logG;
  if (d1.logR + d1.logG != logT || pl->logn <= logT) return false;
  if (pl->logn - logT > 3 || ((size_t)2 * ctx->L * 4u << logT) > kPairClusterMaxSmem) return false;  // 8 CTAs
  return count > 0 && count <= ((size_t)1 << pair_work_log(ctx->L)) >> pl->logn;
}

static moma_status run_pair_cluster_l(moma_ctx* ctx, const Plan* pl, size_t count, const uint32_t* in,
                                      const uint32_t* in2, uint32_t* out, const moma_config& cfg, cudaStream_t st) {
  const uint32_t f0 = pass_flags(pl, 0, 2, in2 != nullptr), f1 = pass_flags(pl, 1, 2, false);
  const int th = cfg.cta_threads;
  const bool wide = cfg.engine == 2;
  switch (ctx->L) {
    case 4:
      return wide ? run_pair_cluster<4, 2>(ctx, pl, count, in, in2, out, f0, f1, th, st)
                  : run_pair_cluster<4, 1>(ctx, pl, count, in, in2, out, f0, f1, th, st);
    case 8:
      return wide ? run_pair_cluster<8, 2>(ctx, pl, count, in, in2, out, f0, f1, th, st)
                  : run_pair_cluster<8, 1>(ctx, pl, count, in, in2, out, f0, f1, th, st);
    default:
      return wide ? run_pair_cluster<12, 2>(ctx, pl, count, in, in2, out, f0, f1, th, st)
                  : run_pair_cluster<12, 1>(ctx, pl, count, in, in2, out, f0, f1, th, st);
  }
}

// Run every pass of a plan: in -> [s1 -> s2 -> s1 ...] -> out, with caller-provided
// intermediate buffers (each count*L*n words; s1 unused for one pass, s2 for up to two; neither
// for a plan that runs in one cluster launch).
moma_status run_plan_buffers(moma_ctx* ctx, const Plan* pl, size_t count, const uint32_t* in, const uint32_t* in2,
                             uint32_t* out, const moma_config& cfg, uint32_t* s1, uint32_t* s2, cudaStream_t st) {
  if (pair_cluster_ok(ctx, pl, count)) return run_pair_cluster_l(ctx, pl, count, in, in2, out, cfg, st);
  const size_t P = pl->passes.size();
  moma_status rc = MOMA_OK;
  const uint32_t* src = in;
  for (size_t i = 0; i < P && rc == MOMA_OK; ++i) {
    uint32_t* dst = (i + 1 == P) ? out : ((i % 2 == 0) ? s1 : s2);
    rc = run_pass_l(ctx, pl, pl->passes[i], count, src, i == 0 ? in2 : nullptr, dst,
                    pass_flags(pl, i, P, in2 != nullptr), cfg, st);
    src = dst;
  }
  return rc;
}

// run_plan_buffers with intermediate buffers from the stream-ordered pool.
static moma_status run_plan(moma_ctx* ctx, const Plan* pl, size_t count, const uint32_t* in, const uint32_t* in2,
                            uint32_t* out, const moma_config& cfg, cudaStream_t st) {
  const size_t P = pair_cluster_ok(ctx, pl, count) ? 1 : pl->passes.size();  // intermediate buffers needed
  const size_t words = (size_t)ctx->L * ((size_t)1 << pl->logn) * count;
  uint32_t* s1 = nullptr;
  uint32_t* s2 = nullptr;
  if (P >= 2 && cudaMallocAsync(&s1, words * 4, st) != cudaSuccess) return MOMA_ERR_OOM;
  if (P >= 3 && cudaMallocAsync(&s2, words * 4, st) != cudaSuccess) {
    cudaFreeAsync(s1, st);
    return MOMA_ERR_OOM;
  }
  const moma_status rc = run_plan_buffers(ctx, pl, count, in, in2, out, cfg, s1, s2, st);
  if (s1) cudaFreeAsync(s1, st);
  if (s2) cudaFreeAsync(s2, st);
  return rc;
}

Plan* find_plan(moma_ctx* ctx, int logn, bool inverse, int tile_log, int max_logr) {
  if (logn <= tile_log) max_logr = 0;
  std::lock_guard<std::mutex> g(ctx->lock);
  auto it = ctx->plans.find(std::make_tuple(logn, inverse ? 1 : 0, tile_log, max_logr, 0));
  return it == ctx->plans.end() ? nullptr : it->second;
}

moma_status launch_ntt_cfg(moma_ctx* ctx, int logn, size_t count, bool inverse, const uint32_t* in, uint32_t* out,
                           const moma_config& cfg, cudaStream_t st, bool nega) {
  Plan* pl = nullptr;
  moma_status rc = get_plan(ctx, logn, inverse, cfg.tile_log, cfg.max_logr, &pl, nega);
  if (rc) return rc;
  if (count == 0) return MOMA_OK;
  return run_plan(ctx, pl, count, in, nullptr, out, cfg, st);
}

moma_status launch_ntt(moma_ctx* ctx, int logn, size_t count, bool inverse, const uint32_t* in, uint32_t* out,
                       cudaStream_t st) {
  return launch_ntt_cfg(ctx, logn, count, inverse, in, out,
                        ntt_config(ctx, inverse ? MOMA_OP_NTT_INV : MOMA_OP_NTT_FWD, logn, count), st);
}

moma_status launch_polymul_cfg(moma_ctx* ctx, int logn, const uint32_t* a, const uint32_t* b, uint32_t* c,
                               const moma_config& cfg, cudaStream_t st, bool nega) {
  Plan *fw = nullptr, *iv = nullptr;
  moma_status rc = get_plan(ctx, logn, false, cfg.tile_log, cfg.max_logr, &fw, nega);
  if (rc) return rc;
  rc = get_plan(ctx, logn, true, cfg.tile_log, cfg.max_logr, &iv, nega);
  if (rc) return rc;
  const size_t words = (size_t)ctx->L << logn;
  uint32_t* fa = nullptr;
  if (cudaMallocAsync(&fa, 2 * words * 4, st) != cudaSuccess) return MOMA_ERR_OOM;
  uint32_t* fb = fa + words;
  rc = run_plan(ctx, fw, 1, a, nullptr, fa, cfg, st);
  if (!rc) rc = run_plan(ctx, fw, 1, b, nullptr, fb, cfg, st);
  if (!rc) rc = run_plan(ctx, iv, 1, fa, fb, c, cfg, st);
  cudaFreeAsync(fa, st);
  return rc;
}

moma_status launch_polymul(moma_ctx* ctx, int logn, const uint32_t* a, const uint32_t* b, uint32_t* c,
                           cudaStream_t st) {
  return launch_polymul_cfg(ctx, logn, a, b, c, ntt_config(ctx, MOMA_OP_POLYMUL, logn, 1), st);
}

}  // namespace moma
