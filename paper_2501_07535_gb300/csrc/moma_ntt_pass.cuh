// moma_ntt_pass.cuh -- the transform pass kernels, their launchers and the twiddle-table
// generator, as templates over the limb count.  moma_ntt.cu instantiates them for up to 384 bits,
// moma_ntt_wide.cu for 512 to 1024 bits (separate translation units compile in parallel).
#pragma once
#include <cooperative_groups.h>

#include <vector>

#include "moma_internal.hpp"
#include "moma_limbs.cuh"
#include "moma_ntt_tile.cuh"

namespace moma {

constexpr int kNttMaxThreads = 256;  // per CTA; the launch may use 32, 64, 128 or 256
constexpr int kPairClusterMaxCtas = 8;              // portable cluster size
constexpr size_t kPairClusterMaxSmem = 227 * 1024;  // both tiles of a CTA of the pair kernel

// Register cap: 85 per thread up to 384 bits (six 128-thread or three 256-thread CTAs per SM;
// measured 2-4% faster than 128); from 512 bits up the full 255.  TIGHT variants (at most 128
// threads per CTA) are compiled for 64 registers up to 256 bits, 102 at 384 bits and 170 at 768
// bits, without spills, for more resident CTAs.
// FE: the product form of the twiddle multiplications (mulmod_fixed_lazy; the schedule's engine).
template <int L, int FE, bool TIGHT>
__global__ void __launch_bounds__(TIGHT ? 128 : kNttMaxThreads,
                                  TIGHT ? (L <= 8 ? 8 : (L == 12 ? 5 : 3)) : (L <= 12 ? 3 : 1))
    ntt_pass_kernel(const __grid_constant__ NttPassArgs<L> p) {
  extern __shared__ __align__(16) uint32_t sm[];
  ntt_tile<L, FE>(p, blockIdx.x, sm);
}

// Full-width contexts: the same pass with Montgomery arithmetic (carry chains, canonical values).
template <int L>
__global__ void __launch_bounds__(kNttMaxThreads, L <= 12 ? 2 : 1)
    ntt_pass_mont_kernel(const __grid_constant__ NttPassArgs<L> p) {
  extern __shared__ __align__(16) uint32_t sm[];
  ntt_tile_impl<L, MontArith<L>>(p, blockIdx.x, sm);
}

// ------------------------------------------------------------------ two passes in one cluster
// A transform of two passes whose n/T tiles (T elements each) fit one thread-block cluster runs
// as one launch: CTA c of the cluster computes tile c of the first pass and stores every output
// straight into the shared memory of the CTA whose second-pass tile reads it (distributed shared
// memory); after a cluster barrier each CTA computes its second-pass tile from its own shared
// memory.  This saves the second launch and the round trip through global memory between the
// passes, which set the time of small transforms.

// First-pass outputs: position pos of the transform is read by the second pass as element
// (r, g) of tile c, with pos = j + r n/R1 and j = c G1 + g; it goes to slot r G1 + g of CTA c.
template <int L>
struct ClusterOut {
  uint32_t* smB;  // this CTA's second-pass tile; the peers' are mapped by cluster rank
  uint32_t lognR1, logG1, logT;
  __device__ __forceinline__ void put(const NttPassArgs<L>& p, uint64_t base, uint64_t pos,
                                      const uint32_t (&v)[L]) const {
    (void)p;
    (void)base;
    const uint32_t r = (uint32_t)(pos >> lognR1);
    const uint32_t j = (uint32_t)pos & ((1u << lognR1) - 1u);
    const uint32_t c = j >> logG1, g = j & ((1u << logG1) - 1u);
    uint32_t* dst = cooperative_groups::this_cluster().map_shared_rank(smB, c);
    tile_store<L>(dst, swz((r << logG1) | g, logT), v);
  }
};

// Second-pass inputs: already in this CTA's tile, at the slot the load would write (in place).
struct ClusterIn {
  template <int L>
  __device__ __forceinline__ void get(const NttPassArgs<L>& p, uint64_t base, uint64_t pos, uint32_t e,
                                      const uint32_t* sm, uint32_t logT, uint32_t (&v)[L]) const {
    (void)p;
    (void)base;
    (void)pos;
    tile_load<L>(sm, swz(e, logT), v);
  }
};

template <int L, int FE>
__global__ void __launch_bounds__(kNttMaxThreads, L <= 12 ? 3 : 1)
    ntt_pair_cluster_kernel(const __grid_constant__ NttPassArgs<L> p0, const __grid_constant__ NttPassArgs<L> p1) {
  extern __shared__ __align__(16) uint32_t sm[];
  namespace cg = cooperative_groups;
  const uint32_t logT = p0.logR + p0.logG;
  uint32_t* smA = sm;                        // first-pass tile
  uint32_t* smB = sm + ((size_t)L << logT);  // second-pass tile, written by the cluster's CTAs
  cg::cluster_group cluster = cg::this_cluster();
  cluster.sync();  // every CTA of the cluster runs before any of them writes a peer's shared memory
  const ClusterOut<L> to_peers{smB, (uint32_t)(63 - __clzll((long long)p1.n)) - p1.logR, p1.logG, logT};
  ntt_tile_impl<L, BarrettArith<L, FE>, GlobalIO, ClusterOut<L>>(p0, blockIdx.x, smA, GlobalIO(), to_peers);
  cluster.sync();  // the peers' stores into smB are complete and visible
  ntt_tile_impl<L, BarrettArith<L, FE>, ClusterIn, GlobalIO>(p1, blockIdx.x, smB, ClusterIn(), GlobalIO());
}

// ------------------------------------------------------------------ twiddle tables
template <int L>
struct TwGenArgs {
  uint32_t* dst;
  uint64_t count;
  // exponent of entry idx: ((idx / D) + C) * (idx % D) * S  (mod n, all < n by construction)
  uint64_t D, C, S;
  uint32_t logn;
  uint32_t pw[kMaxLogN + 1][L];  // w^(2^b)
  uint32_t init[L];              // start value of the product (1, or a constant factor)
  uint32_t R0[L];
  uint32_t Q0;
  ModK<L> k;
};

// MONT: full-width context; pw, init and the entries are in Montgomery form (x R mod q), the
// products are Montgomery products and the companion half of each entry is zero.
template <int L, bool MONT>
__global__ void __launch_bounds__(256) twiddle_gen_kernel(const __grid_constant__ TwGenArgs<L> p) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < p.count; idx += stride) {
    const uint64_t e = ((idx / p.D) + p.C) * (idx % p.D) * p.S & ((1ull << p.logn) - 1);
    uint32_t acc[L];
#pragma unroll
    for (int l = 0; l < L; ++l) acc[l] = p.init[l];
    for (uint32_t bb = 0; bb < p.logn; ++bb) {
      if ((e >> bb) & 1) {
        uint32_t t[L];
        if constexpr (MONT) montmul<L>(t, acc, p.pw[bb], p.k);
        else mulmod_barrett<L>(t, acc, p.pw[bb], p.k);
#pragma unroll
        for (int l = 0; l < L; ++l) acc[l] = t[l];
      }
    }
    if constexpr (MONT) {
#pragma unroll
      for (int l = 0; l < L; ++l) {
        p.dst[idx * 2 * L + l] = acc[l];
        p.dst[idx * 2 * L + L + l] = 0u;
      }
      continue;
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
      p.dst[idx * 2 * L + l] = acc[l];
      p.dst[idx * 2 * L + L + l] = wp[l];
    }
  }
}

template <int L>
moma_status gen_table(const moma_ctx* ctx, uint32_t* dst, uint64_t count, uint64_t D, uint64_t C,
                             uint64_t S, int logn, const std::vector<BigU>& pw, const BigU& init) {
  TwGenArgs<L> a;
  a.dst = dst;
  a.count = count;
  a.D = D;
  a.C = C;
  a.S = S;
  a.logn = (uint32_t)logn;
  // full-width contexts take the factors in Montgomery form: x R mod q, R = 2^(32L)
  auto form = [&](const BigU& x) { return ctx->mont ? ctx->red->mulmod(x, BigU::from_words(ctx->k.R0, L)) : x; };
  for (int b = 0; b <= kMaxLogN; ++b) {
    const BigU f = b < logn ? form(pw[b]) : BigU();
    for (int l = 0; l < L; ++l) a.pw[b][l] = f.word(l);
  }
  form(init).to_words(a.init, L);
  for (int l = 0; l < L; ++l) a.R0[l] = ctx->k.R0[l];
  a.Q0 = ctx->k.Q0;
  fill_modk<L>(ctx, a.k);
  uint64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (ctx->mont) twiddle_gen_kernel<L, true><<<(unsigned)blocks, 256>>>(a);
  else twiddle_gen_kernel<L, false><<<(unsigned)blocks, 256>>>(a);
  return cuda_status(cudaGetLastError());
}

template <int L, int FE, bool TIGHT>
moma_status run_pass(moma_ctx* ctx, const Plan* pl, const PassDesc& d, size_t count, const uint32_t* src,
                            const uint32_t* src2, uint32_t* dst, uint32_t flags, int threads, cudaStream_t st) {
  NttPassArgs<L> a;
  fill_pass_args<L>(ctx, pl, d, count, src, src2, dst, flags, a);
  const size_t smem = (size_t)L * 4u << (d.logR + d.logG);
  static std::atomic<uint64_t> attr_done{0};  // one bit per device: the attribute is per device
  const uint64_t dev_bit = 1ull << (ctx->device & 63);
  if (!(attr_done.load(std::memory_order_acquire) & dev_bit)) {
    if (cudaFuncSetAttribute(ntt_pass_kernel<L, FE, TIGHT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             L * 4 << max_tile_log(L)) != cudaSuccess)
      return MOMA_ERR_CUDA;
    attr_done.fetch_or(dev_bit, std::memory_order_release);
  }
  const uint64_t grid = (uint64_t)count * a.tiles_per_transform;
  if (grid == 0) return MOMA_OK;
  if (grid > 0x7fffffffull) return MOMA_ERR_SIZE;
  ntt_pass_kernel<L, FE, TIGHT><<<(unsigned)grid, threads, smem, st>>>(a);
  return cuda_status(cudaGetLastError());
}

template <int L>
moma_status run_pass_mont(moma_ctx* ctx, const Plan* pl, const PassDesc& d, size_t count, const uint32_t* src,
                                 const uint32_t* src2, uint32_t* dst, uint32_t flags, int threads, cudaStream_t st) {
  NttPassArgs<L> a;
  fill_pass_args<L>(ctx, pl, d, count, src, src2, dst, flags, a);
  const size_t smem = (size_t)L * 4u << (d.logR + d.logG);
  static std::atomic<uint64_t> attr_done{0};  // one bit per device: the attribute is per device
  const uint64_t dev_bit = 1ull << (ctx->device & 63);
  if (!(attr_done.load(std::memory_order_acquire) & dev_bit)) {
    if (cudaFuncSetAttribute(ntt_pass_mont_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             L * 4 << max_tile_log(L)) != cudaSuccess)
      return MOMA_ERR_CUDA;
    attr_done.fetch_or(dev_bit, std::memory_order_release);
  }
  const uint64_t grid = (uint64_t)count * a.tiles_per_transform;
  if (grid == 0) return MOMA_OK;
  if (grid > 0x7fffffffull) return MOMA_ERR_SIZE;
  ntt_pass_mont_kernel<L><<<(unsigned)grid, threads, smem, st>>>(a);
  return cuda_status(cudaGetLastError());
}

// Both passes of a two-pass plan in one cluster launch (see ntt_pair_cluster_kernel): count
// clusters of n/T CTAs.  f0, f1: the passes' flags.
template <int L, int FE>
moma_status run_pair_cluster(moma_ctx* ctx, const Plan* pl, size_t count, const uint32_t* src, const uint32_t* src2,
                             uint32_t* dst, uint32_t f0, uint32_t f1, int threads, cudaStream_t st) {
  NttPassArgs<L> a0, a1;
  fill_pass_args<L>(ctx, pl, pl->passes[0], count, src, src2, nullptr, f0, a0);
  fill_pass_args<L>(ctx, pl, pl->passes[1], count, nullptr, nullptr, dst, f1, a1);
  const int logT = pl->passes[0].logR + pl->passes[0].logG;
  const size_t smem = (size_t)2 * L * 4u << logT;
  static std::atomic<uint64_t> attr_done{0};
  const uint64_t dev_bit = 1ull << (ctx->device & 63);
  if (!(attr_done.load(std::memory_order_acquire) & dev_bit)) {
    if (cudaFuncSetAttribute(ntt_pair_cluster_kernel<L, FE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPairClusterMaxSmem) != cudaSuccess)
      return MOMA_ERR_CUDA;
    attr_done.fetch_or(dev_bit, std::memory_order_release);
  }
  const uint64_t grid = (uint64_t)count * a0.tiles_per_transform;
  if (grid == 0) return MOMA_OK;
  if (grid > 0x7fffffffull) return MOMA_ERR_SIZE;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)grid, 1, 1);
  lc.blockDim = dim3((unsigned)threads, 1, 1);
  lc.dynamicSmemBytes = smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = a0.tiles_per_transform;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  return cuda_status(cudaLaunchKernelEx(&lc, ntt_pair_cluster_kernel<L, FE>, a0, a1));
}

// One pass with the kernel the schedule picks: Montgomery for full-width contexts; otherwise the
// product form of the twiddle multiplications (engine 1 or 2: mulmod_fixed_lazy's FE) and the
// register cap.  From 512 bits up only carry chains are instantiated, except at 768 bits (engine 2
// and the capped variant); other settings fall back to carry chains.
template <int L>
moma_status run_pass_for(moma_ctx* ctx, const Plan* pl, const PassDesc& d, size_t count, const uint32_t* src,
                         const uint32_t* src2, uint32_t* dst, uint32_t flags, const moma_config& cfg,
                         cudaStream_t st) {
  if (ctx->mont) return run_pass_mont<L>(ctx, pl, d, count, src, src2, dst, flags, cfg.cta_threads, st);
  const int fe = cfg.engine;
  const int th = cfg.cta_threads;
  const bool tight = cfg.tight_regs != 0 && th <= 128;
  if constexpr (L <= 12) {
    if (fe == 2)
      return tight ? run_pass<L, 2, true>(ctx, pl, d, count, src, src2, dst, flags, th, st)
                   : run_pass<L, 2, false>(ctx, pl, d, count, src, src2, dst, flags, th, st);
    return tight ? run_pass<L, 1, true>(ctx, pl, d, count, src, src2, dst, flags, th, st)
                 : run_pass<L, 1, false>(ctx, pl, d, count, src, src2, dst, flags, th, st);
  } else if constexpr (L == 24) {
    if (tight) return run_pass<L, 1, true>(ctx, pl, d, count, src, src2, dst, flags, th, st);
    return fe == 2 ? run_pass<L, 2, false>(ctx, pl, d, count, src, src2, dst, flags, th, st)
                   : run_pass<L, 1, false>(ctx, pl, d, count, src, src2, dst, flags, th, st);
  } else {
    return run_pass<L, 1, false>(ctx, pl, d, count, src, src2, dst, flags, th, st);
  }
}

}  // namespace moma
