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
// The last DIF stage has twiddle 1 and no multiplication; the first pass has Ns = 1 and
// no pre-twiddles.
//
// Twiddles are in the reduction's domain: every table entry w carries its companion
// floor(w * 2^(32L) / q), so a twiddle multiplication needs no double-width product
// (mulmod_fixed).  Tables are built on the device once per (modulus, size, direction).
#include <algorithm>

#include "moma_internal.hpp"
#include "moma_limbs.cuh"

namespace moma {

constexpr int kNttThreads = 256;

// Default CTA tile (elements) per width: the tile takes L*T*4 bytes of shared memory.
int default_tile_log(int L) {
  switch (L) {
    case 4: return 12;   // 64 KiB
    case 8: return 11;   // 64 KiB
    case 12: return 11;  // 96 KiB
    default: return 10;
  }
}

// Largest tile that fits the 227 KiB of shared memory one CTA may use.
int max_tile_log(int L) {
  int t = 5;
  while ((size_t)L * 4u << (t + 1) <= 227u * 1024u) ++t;
  return t;
}

constexpr int kDefaultEngine = 1;

moma_config ntt_config(const moma_ctx* ctx, int op, int logn) {
  moma_config c = {0, 0, 0, 0};
  auto it = ctx->configs.find(std::make_pair(op, logn));
  if (it != ctx->configs.end()) c = it->second;
  if (c.engine == 0) c.engine = kDefaultEngine;
  if (c.tile_log == 0) c.tile_log = default_tile_log(ctx->L);
  if (c.max_logr == 0) c.max_logr = c.tile_log > 6 ? c.tile_log - 5 : 1;
  c.vec_width = 0;
  return c;
}

bool ntt_config_valid(int L, int logn, const moma_config& c) {
  (void)logn;
  if (c.engine < 0 || c.engine > 2) return false;
  if (c.tile_log != 0 && (c.tile_log < 5 || c.tile_log > max_tile_log(L))) return false;
  if (c.max_logr < 0 || (c.max_logr != 0 && c.tile_log != 0 && c.max_logr > c.tile_log)) return false;
  return true;
}

// XOR swizzle of a word index inside one limb plane of the tile: flips the low five
// bits by the next five, so that both row-wise and bit-reversed column-wise accesses
// spread over the 32 banks.  A bijection on every aligned block of 32 words.
__device__ __forceinline__ uint32_t swz(uint32_t x) { return x ^ ((x >> 5) & 31u); }

template <int L>
struct NttPassArgs {
  const uint32_t* src;
  const uint32_t* src2;  // pointwise second operand (fused polynomial product), else null
  uint32_t* dst;
  const uint32_t* tw_pass;
  const uint32_t* tw_int;
  uint64_t tw_count;
  uint64_t n;
  uint32_t logR, logG, logNs;
  uint32_t tiles_per_transform;
  uint32_t flags;  // 1: pre-twiddle, 2: multiply by sc at load, 4: pointwise product at load
  uint32_t sc[L], scp[L];
  ModK<L> k;
};

enum { F_PRETW = 1, F_SCALE = 2, F_POINTWISE = 4 };

template <int L, bool WIDE>
__global__ void __launch_bounds__(kNttThreads) ntt_pass_kernel(const __grid_constant__ NttPassArgs<L> p) {
  extern __shared__ uint32_t sm[];
  const uint32_t R = 1u << p.logR;
  const uint32_t G = 1u << p.logG;
  const uint32_t T = R << p.logG;
  const uint32_t tile = blockIdx.x;
  const uint64_t b = tile / p.tiles_per_transform;
  const uint64_t jb = tile - b * p.tiles_per_transform;
  const uint64_t base = b * (uint64_t)L * p.n;
  const uint64_t j0 = jb << p.logG;
  const uint64_t nR = p.n >> p.logR;
  const uint64_t ns_mask = (1ull << p.logNs) - 1;

  // ---- load (+ pointwise product, scaling, pre-twiddle) into the tile
  for (uint32_t e = threadIdx.x; e < T; e += kNttThreads) {
    const uint32_t r = e >> p.logG, g = e & (G - 1);
    const uint64_t j = j0 + g;
    const uint64_t idx = base + j + (uint64_t)r * nR;
    uint32_t v[L];
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = p.src[idx + (uint64_t)l * p.n];
    if (p.flags & F_POINTWISE) {
      uint32_t u[L], t[L];
#pragma unroll
      for (int l = 0; l < L; ++l) u[l] = p.src2[idx + (uint64_t)l * p.n];
      mulmod_barrett<L, WIDE>(t, v, u, p.k);
#pragma unroll
      for (int l = 0; l < L; ++l) v[l] = t[l];
    }
    if (p.flags & F_SCALE) {
      uint32_t t[L];
      mulmod_fixed<L, WIDE>(t, v, p.sc, p.scp, p.k);
#pragma unroll
      for (int l = 0; l < L; ++l) v[l] = t[l];
    }
    if ((p.flags & F_PRETW) && r != 0) {
      const uint64_t ti = (uint64_t)(r - 1) * (ns_mask + 1) + (j & ns_mask);
      uint32_t w[L], wp[L], t[L];
#pragma unroll
      for (int l = 0; l < L; ++l) {
        w[l] = __ldg(p.tw_pass + ti + (uint64_t)l * p.tw_count);
        wp[l] = __ldg(p.tw_pass + ti + (uint64_t)(L + l) * p.tw_count);
      }
      mulmod_fixed<L, WIDE>(t, v, w, wp, p.k);
#pragma unroll
      for (int l = 0; l < L; ++l) v[l] = t[l];
    }
    const uint32_t a = swz(e);  // e = r*G + g
#pragma unroll
    for (int l = 0; l < L; ++l) sm[l * T + a] = v[l];
  }
  __syncthreads();

  // ---- R-point transforms: logR radix-2 DIF stages, in place in the tile
  const uint32_t half_int = R >> 1;
#pragma unroll 1
  for (uint32_t s = 0; s < p.logR; ++s) {
    const uint32_t logh = p.logR - s - 1;
    const uint32_t h = 1u << logh;
    for (uint32_t bi = threadIdx.x; bi < (T >> 1); bi += kNttThreads) {
      const uint32_t g = bi & (G - 1), u = bi >> p.logG;
      const uint32_t i = u & (h - 1), blk = u >> logh;
      const uint32_t p0 = (blk << (logh + 1)) + i;
      const uint32_t a0 = swz((p0 << p.logG) + g), a1 = swz(((p0 + h) << p.logG) + g);
      uint32_t x0[L], x1[L], y0[L], d[L];
#pragma unroll
      for (int l = 0; l < L; ++l) {
        x0[l] = sm[l * T + a0];
        x1[l] = sm[l * T + a1];
      }
      addmod<L>(y0, x0, x1, p.k.q);
      submod<L>(d, x0, x1, p.k.q);
      if (logh != 0) {
        const uint32_t ti = i << s;  // w_(2h)^i = w_R^(i * R/(2h))
        uint32_t w[L], wp[L], y1[L];
#pragma unroll
        for (int l = 0; l < L; ++l) {
          w[l] = __ldg(p.tw_int + ti + l * half_int);
          wp[l] = __ldg(p.tw_int + ti + (L + l) * half_int);
        }
        mulmod_fixed<L, WIDE>(y1, d, w, wp, p.k);
#pragma unroll
        for (int l = 0; l < L; ++l) d[l] = y1[l];
      }
#pragma unroll
      for (int l = 0; l < L; ++l) {
        sm[l * T + a0] = y0[l];
        sm[l * T + a1] = d[l];
      }
    }
    __syncthreads();
  }

  // ---- store: output s of group j goes to (j-k)*R + k + s*Ns; consecutive threads take
  // consecutive addresses (k fastest, then s, then the Ns-blocks of the tile).
  const uint32_t logGl = p.logG < p.logNs ? p.logG : p.logNs;
  const uint32_t Gl = 1u << logGl;
  for (uint32_t e = threadIdx.x; e < T; e += kNttThreads) {
    const uint32_t gl = e & (Gl - 1);
    const uint32_t sp = (e >> logGl) & (R - 1);
    const uint32_t gh = e >> (logGl + p.logR);
    const uint32_t g = (gh << logGl) + gl;
    const uint64_t j = j0 + g;
    const uint64_t kk = j & ns_mask;
    const uint64_t addr = base + (j - kk) * R + kk + ((uint64_t)sp << p.logNs);
    const uint32_t pr = __brev(sp) >> (32 - p.logR);
    const uint32_t a = swz((pr << p.logG) + g);
#pragma unroll
    for (int l = 0; l < L; ++l) p.dst[addr + (uint64_t)l * p.n] = sm[l * T + a];
  }
}

// ------------------------------------------------------------------ twiddle tables
template <int L>
struct TwGenArgs {
  uint32_t* dst;
  uint64_t count;
  // exponent of entry idx: ((idx / D) + C) * (idx % D) * S  (mod n, all < n by construction)
  uint64_t D, C, S;
  uint32_t logn;
  uint32_t pw[kMaxLogN][L];  // w^(2^b)
  uint32_t R0[L];
  uint32_t Q0;
  ModK<L> k;
};

template <int L>
__global__ void __launch_bounds__(256) twiddle_gen_kernel(const __grid_constant__ TwGenArgs<L> p) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < p.count; idx += stride) {
    const uint64_t e = ((idx / p.D) + p.C) * (idx % p.D) * p.S & ((1ull << p.logn) - 1);
    uint32_t acc[L];
#pragma unroll
    for (int l = 0; l < L; ++l) acc[l] = l == 0 ? 1u : 0u;
    for (uint32_t bb = 0; bb < p.logn; ++bb) {
      if ((e >> bb) & 1) {
        uint32_t t[L];
        mulmod_barrett<L>(t, acc, p.pw[bb], p.k);
#pragma unroll
        for (int l = 0; l < L; ++l) acc[l] = t[l];
      }
    }
    // companion floor(w*2^W/q) = w*Q0 + floor(w*R0/q), with 2^W = Q0*q + R0
    uint32_t prod[2 * L], rem[L], quo[L];
    mul_full<L>(prod, acc, p.R0);
    const uint32_t corr = barrett_reduce<L>(rem, quo, prod, p.k);
    uint32_t wp[L];
    uint64_t c = corr;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      c += (uint64_t)acc[l] * p.Q0 + quo[l];
      wp[l] = (uint32_t)c;
      c >>= 32;
    }
#pragma unroll
    for (int l = 0; l < L; ++l) {
      p.dst[idx + (uint64_t)l * p.count] = acc[l];
      p.dst[idx + (uint64_t)(L + l) * p.count] = wp[l];
    }
  }
}

template <int L>
static void fill_modk(const moma_ctx* ctx, ModK<L>& k) {
  for (int i = 0; i < L; ++i) {
    k.q[i] = ctx->k.q[i];
    k.nq[i] = ctx->k.nq[i];
    k.mu[i] = ctx->k.mu[i];
    k.q2[i] = ctx->k.q2[i];
  }
}

template <int L>
static moma_status gen_table(const moma_ctx* ctx, uint32_t* dst, uint64_t count, uint64_t D, uint64_t C,
                             uint64_t S, int logn, const std::vector<BigU>& pw) {
  TwGenArgs<L> a;
  a.dst = dst;
  a.count = count;
  a.D = D;
  a.C = C;
  a.S = S;
  a.logn = (uint32_t)logn;
  for (int b = 0; b < kMaxLogN; ++b)
    for (int l = 0; l < L; ++l) a.pw[b][l] = b < logn ? pw[b].word(l) : 0u;
  for (int l = 0; l < L; ++l) a.R0[l] = ctx->k.R0[l];
  a.Q0 = ctx->k.Q0;
  fill_modk<L>(ctx, a.k);
  uint64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  twiddle_gen_kernel<L><<<(unsigned)blocks, 256>>>(a);
  return cuda_status(cudaGetLastError());
}

static moma_status gen_table_l(const moma_ctx* ctx, uint32_t* dst, uint64_t count, uint64_t D, uint64_t C,
                               uint64_t S, int logn, const std::vector<BigU>& pw) {
  switch (ctx->L) {
    case 4: return gen_table<4>(ctx, dst, count, D, C, S, logn, pw);
    case 8: return gen_table<8>(ctx, dst, count, D, C, S, logn, pw);
    case 12: return gen_table<12>(ctx, dst, count, D, C, S, logn, pw);
  }
  return MOMA_ERR_UNSUPPORTED;
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

static moma_status build_plan(moma_ctx* ctx, int logn, bool inverse, int tile_log, int max_logr, Plan** out) {
  const int L = ctx->L;
  Plan* pl = new Plan();
  pl->logn = logn;
  pl->inverse = inverse;
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
  if (cudaMalloc(&pl->d_tables, words * 4) != cudaSuccess) {
    delete pl;
    return MOMA_ERR_OOM;
  }
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
  if (inverse) {
    // n^-1 = q - (q-1)/n
    BigU ninv = sub(ctx->Q, shr(sub(ctx->Q, BigU(1)), logn));
    ninv.to_words(pl->scale, L);
    companion(ctx, ninv, pl->scalep);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    free_plan(pl);
    return MOMA_ERR_CUDA;
  }
  *out = pl;
  return MOMA_OK;
}

moma_status get_plan(moma_ctx* ctx, int logn, bool inverse, int tile_log, int max_logr, Plan** out) {
  moma_status st = ntt_prepare(ctx);
  if (st) return st;
  if (logn > ctx->two_adicity || logn < 1 || logn > kMaxLogN) return MOMA_ERR_SIZE;
  if (logn <= tile_log) max_logr = 0;  // single pass: the split does not matter
  std::lock_guard<std::mutex> g(ctx->lock);
  auto key = std::make_tuple(logn, inverse ? 1 : 0, tile_log, max_logr);
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) {
    *out = it->second;
    return MOMA_OK;
  }
  Plan* pl = nullptr;
  st = build_plan(ctx, logn, inverse, tile_log, max_logr, &pl);
  if (st) return st;
  ctx->plans[key] = pl;
  *out = pl;
  return MOMA_OK;
}

template <int L, bool WIDE>
static moma_status run_pass(moma_ctx* ctx, const Plan* pl, const PassDesc& d, size_t count, const uint32_t* src,
                            const uint32_t* src2, uint32_t* dst, uint32_t flags, cudaStream_t st) {
  NttPassArgs<L> a;
  a.src = src;
  a.src2 = src2;
  a.dst = dst;
  a.tw_pass = d.tw_pass;
  a.tw_int = d.tw_int;
  a.tw_count = d.tw_count;
  a.n = 1ull << pl->logn;
  a.logR = (uint32_t)d.logR;
  a.logG = (uint32_t)d.logG;
  a.logNs = (uint32_t)d.logNs;
  a.tiles_per_transform = (uint32_t)(a.n >> (d.logR + d.logG));
  a.flags = flags | (d.logNs > 0 ? F_PRETW : 0);
  for (int i = 0; i < L; ++i) {
    a.sc[i] = pl->scale[i];
    a.scp[i] = pl->scalep[i];
  }
  fill_modk<L>(ctx, a.k);
  const size_t smem = (size_t)L * 4u << (d.logR + d.logG);
  static bool attr_done = false;
  if (!attr_done) {
    if (cudaFuncSetAttribute(ntt_pass_kernel<L, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             L * 4 << max_tile_log(L)) != cudaSuccess)
      return MOMA_ERR_CUDA;
    attr_done = true;
  }
  const uint64_t grid = (uint64_t)count * a.tiles_per_transform;
  if (grid == 0) return MOMA_OK;
  if (grid > 0x7fffffffull) return MOMA_ERR_SIZE;
  ntt_pass_kernel<L, WIDE><<<(unsigned)grid, kNttThreads, smem, st>>>(a);
  return cuda_status(cudaGetLastError());
}

static moma_status run_pass_l(moma_ctx* ctx, const Plan* pl, const PassDesc& d, size_t count, const uint32_t* src,
                              const uint32_t* src2, uint32_t* dst, uint32_t flags, int engine, cudaStream_t st) {
  const bool wide = engine == 2;
  switch (ctx->L) {
    case 4: return wide ? run_pass<4, true>(ctx, pl, d, count, src, src2, dst, flags, st)
                        : run_pass<4, false>(ctx, pl, d, count, src, src2, dst, flags, st);
    case 8: return wide ? run_pass<8, true>(ctx, pl, d, count, src, src2, dst, flags, st)
                        : run_pass<8, false>(ctx, pl, d, count, src, src2, dst, flags, st);
    case 12: return wide ? run_pass<12, true>(ctx, pl, d, count, src, src2, dst, flags, st)
                         : run_pass<12, false>(ctx, pl, d, count, src, src2, dst, flags, st);
  }
  return MOMA_ERR_UNSUPPORTED;
}

// Run every pass of a plan: in -> [scratch1 -> scratch2 -> ...] -> out.  The first pass can
// fuse a pointwise product with src2 (polymul) and, for the inverse, the n^-1 scaling.
static moma_status run_plan(moma_ctx* ctx, const Plan* pl, size_t count, const uint32_t* in, const uint32_t* in2,
                            uint32_t* out, int engine, cudaStream_t st) {
  const size_t P = pl->passes.size();
  const size_t words = (size_t)ctx->L * ((size_t)1 << pl->logn) * count;
  uint32_t* s1 = nullptr;
  uint32_t* s2 = nullptr;
  if (P >= 2 && cudaMallocAsync(&s1, words * 4, st) != cudaSuccess) return MOMA_ERR_OOM;
  if (P >= 3 && cudaMallocAsync(&s2, words * 4, st) != cudaSuccess) {
    cudaFreeAsync(s1, st);
    return MOMA_ERR_OOM;
  }
  moma_status rc = MOMA_OK;
  const uint32_t* src = in;
  for (size_t i = 0; i < P && rc == MOMA_OK; ++i) {
    uint32_t* dst = (i + 1 == P) ? out : ((i % 2 == 0) ? s1 : s2);
    uint32_t flags = 0;
    if (i == 0 && in2) flags |= F_POINTWISE;
    if (i == 0 && pl->inverse) flags |= F_SCALE;
    rc = run_pass_l(ctx, pl, pl->passes[i], count, src, i == 0 ? in2 : nullptr, dst, flags, engine, st);
    src = dst;
  }
  if (s1) cudaFreeAsync(s1, st);
  if (s2) cudaFreeAsync(s2, st);
  return rc;
}

Plan* find_plan(moma_ctx* ctx, int logn, bool inverse, int tile_log, int max_logr) {
  if (logn <= tile_log) max_logr = 0;
  std::lock_guard<std::mutex> g(ctx->lock);
  auto it = ctx->plans.find(std::make_tuple(logn, inverse ? 1 : 0, tile_log, max_logr));
  return it == ctx->plans.end() ? nullptr : it->second;
}

moma_status run_plan_scratch(moma_ctx* ctx, const Plan* pl, const uint32_t* in, uint32_t* out, int engine,
                             uint32_t* s1, uint32_t* s2, cudaStream_t st) {
  const size_t P = pl->passes.size();
  moma_status rc = MOMA_OK;
  const uint32_t* src = in;
  for (size_t i = 0; i < P && rc == MOMA_OK; ++i) {
    uint32_t* dst = (i + 1 == P) ? out : ((i % 2 == 0) ? s1 : s2);
    const uint32_t flags = (i == 0 && pl->inverse) ? F_SCALE : 0;
    rc = run_pass_l(ctx, pl, pl->passes[i], 1, src, nullptr, dst, flags, engine, st);
    src = dst;
  }
  return rc;
}

moma_status launch_ntt_cfg(moma_ctx* ctx, int logn, size_t count, bool inverse, const uint32_t* in, uint32_t* out,
                           const moma_config& cfg, cudaStream_t st) {
  Plan* pl = nullptr;
  moma_status rc = get_plan(ctx, logn, inverse, cfg.tile_log, cfg.max_logr, &pl);
  if (rc) return rc;
  if (count == 0) return MOMA_OK;
  return run_plan(ctx, pl, count, in, nullptr, out, cfg.engine, st);
}

moma_status launch_ntt(moma_ctx* ctx, int logn, size_t count, bool inverse, const uint32_t* in, uint32_t* out,
                       cudaStream_t st) {
  return launch_ntt_cfg(ctx, logn, count, inverse, in, out,
                        ntt_config(ctx, inverse ? MOMA_OP_NTT_INV : MOMA_OP_NTT_FWD, logn), st);
}

moma_status launch_polymul_cfg(moma_ctx* ctx, int logn, const uint32_t* a, const uint32_t* b, uint32_t* c,
                               const moma_config& cfg, cudaStream_t st) {
  Plan *fw = nullptr, *iv = nullptr;
  moma_status rc = get_plan(ctx, logn, false, cfg.tile_log, cfg.max_logr, &fw);
  if (rc) return rc;
  rc = get_plan(ctx, logn, true, cfg.tile_log, cfg.max_logr, &iv);
  if (rc) return rc;
  const size_t words = (size_t)ctx->L << logn;
  uint32_t* fa = nullptr;
  if (cudaMallocAsync(&fa, 2 * words * 4, st) != cudaSuccess) return MOMA_ERR_OOM;
  uint32_t* fb = fa + words;
  rc = run_plan(ctx, fw, 1, a, nullptr, fa, cfg.engine, st);
  if (!rc) rc = run_plan(ctx, fw, 1, b, nullptr, fb, cfg.engine, st);
  if (!rc) rc = run_plan(ctx, iv, 1, fa, fb, c, cfg.engine, st);
  cudaFreeAsync(fa, st);
  return rc;
}

moma_status launch_polymul(moma_ctx* ctx, int logn, const uint32_t* a, const uint32_t* b, uint32_t* c,
                           cudaStream_t st) {
  return launch_polymul_cfg(ctx, logn, a, b, c, ntt_config(ctx, MOMA_OP_POLYMUL, logn), st);
}

}  // namespace moma
