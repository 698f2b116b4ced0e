// moma_blas_kern.cuh -- the element-wise kernels and their launchers as templates over the limb
// count.  moma_blas.cu instantiates them for up to 384 bits, moma_blas_wide.cu for 512 to 1024 bits.
//
// Data are limb-major: plane l of a length-n vector is the contiguous run v[l*n .. l*n+n).
// A thread handles V consecutive elements per step and reads each of the L planes with
// one V-wide vector load (uint4 for V = 4), so every load of a warp is a coalesced
// 32*V-word run of one plane.  Grid-stride loop over a grid sized to fill every SM.
#pragma once
#include "moma_async.cuh"
#include "moma_consts.cuh"
#include "moma_internal.hpp"
#include "moma_limbs.cuh"

namespace moma {

template <int L>
struct VecArgs {
  const uint32_t* a;
  const uint32_t* b;
  uint32_t* c;
  uint64_t n;
  uint32_t alpha[L], alphap[L];  // axpy scalar and its companion floor(alpha*2^(32L)/q)
  ModK<L> k;
  // staged kernel only
  int* status;            // device status word of the context (MOMA_ERR_TIMEOUT)
  uint64_t wait_ns;       // bound of one wait on a stage's barrier
  uint32_t log_tile;      // elements per tile, log2 (a multiple of the CTA size)
  uint32_t inject;        // test hook: CTA 0 expects 16 bytes more than its first tile brings
};

template <int V>
struct VecT;
template <>
struct VecT<1> {
  using T = uint32_t;
  static __device__ __forceinline__ void split(const T& v, uint32_t* o) { o[0] = v; }
  static __device__ __forceinline__ T join(const uint32_t* o) { return o[0]; }
};
template <>
struct VecT<2> {
  using T = uint2;
  static __device__ __forceinline__ void split(const T& v, uint32_t* o) { o[0] = v.x; o[1] = v.y; }
  static __device__ __forceinline__ T join(const uint32_t* o) { return make_uint2(o[0], o[1]); }
};
template <>
struct VecT<4> {
  using T = uint4;
  static __device__ __forceinline__ void split(const T& v, uint32_t* o) {
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  static __device__ __forceinline__ T join(const uint32_t* o) { return make_uint4(o[0], o[1], o[2], o[3]); }
};

// ENG: 1 carry-chain rows, 2 whole-product (mad.wide) rows, 3 Karatsuba double-width product
// (Eq. mulk, carry-chain base) for mulmod; axpy's fixed-scalar product has no double-width
// product, so ENG 3 uses carry chains there.
// FULL: 0 a (W-4)-bit modulus (Barrett, Eq. barrett); 1 a full-width modulus, sums with their
// carry word, mulmod by the ENG product and the word-based Barrett reduction with an (L+1)-word
// constant; 2 a full-width modulus with mulmod as two Montgomery products.  In both full-width
// forms the axpy scalar arrives in Montgomery form (one Montgomery product gives alpha * x).
template <int L, int OP, int ENG, int FULL>
__device__ __forceinline__ void vec_apply(uint32_t (&z)[L], const uint32_t (&x)[L], const uint32_t (&y)[L],
                                          const VecArgs<L>& p) {
  if constexpr (FULL != 0) {
    if constexpr (OP == VEC_ADD) {
      addmod_full<L>(z, x, y, p.k.q);
    } else if constexpr (OP == VEC_SUB) {
      submod<L>(z, x, y, p.k.q);
    } else if constexpr (OP == VEC_MUL) {
      if constexpr (FULL == 2) mulmod_mont<L>(z, x, y, p.k);
      else mulmod_barrett_full<L, ENG>(z, x, y, p.k);
    } else {
      uint32_t ax[L];
      montmul<L>(ax, x, p.alpha, p.k);
      addmod_full<L>(z, ax, y, p.k.q);
    }
  } else if constexpr (OP == VEC_ADD) {
    addmod<L>(z, x, y, p.k.q);
  } else if constexpr (OP == VEC_SUB) {
    submod<L>(z, x, y, p.k.q);
  } else if constexpr (OP == VEC_MUL) {
    mulmod_barrett<L, ENG == 2, ENG == 3>(z, x, y, p.k);
  } else {
    uint32_t ax[L];
    mulmod_fixed<L, (ENG == 2 ? 2 : 1)>(ax, x, p.alpha, p.alphap, p.k);
    addmod<L>(z, ax, y, p.k.q);
  }
}

template <int L, int OP, int V, int ENG, int FULL = 0>
__global__ void __launch_bounds__(256) vec_kernel(const __grid_constant__ VecArgs<L> p) {
  using VT = typename VecT<V>::T;
  const uint64_t units = p.n / V;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += stride) {
    uint32_t x[V][L], y[V][L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      uint32_t tmp[V];
      VecT<V>::split(reinterpret_cast<const VT*>(p.a + (uint64_t)l * p.n)[u], tmp);
#pragma unroll
      for (int v = 0; v < V; ++v) x[v][l] = tmp[v];
      VecT<V>::split(reinterpret_cast<const VT*>(p.b + (uint64_t)l * p.n)[u], tmp);
#pragma unroll
      for (int v = 0; v < V; ++v) y[v][l] = tmp[v];
    }
    uint32_t z[V][L];
#pragma unroll
    for (int v = 0; v < V; ++v) vec_apply<L, OP, ENG, FULL>(z[v], x[v], y[v], p);
#pragma unroll
    for (int l = 0; l < L; ++l) {
      uint32_t tmp[V];
#pragma unroll
      for (int v = 0; v < V; ++v) tmp[v] = z[v][l];
      reinterpret_cast<VT*>(p.c + (uint64_t)l * p.n)[u] = VecT<V>::join(tmp);
    }
  }
}

// Kernel arguments common to both forms (constants, axpy scalar); MOMA_ERR_INVALID_ARG for a
// non-canonical scalar.
template <int L, int OP, int FULL>
moma_status fill_vec_args(moma_ctx* ctx, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                          const uint32_t* alpha_host, VecArgs<L>& p) {
  p.a = a;
  p.b = b;
  p.c = c;
  p.n = n;
  fill_modk<L>(ctx, p.k);
  for (int i = 0; i < L; ++i) {
    p.alpha[i] = 0;
    p.alphap[i] = 0;
  }
  if (OP == VEC_AXPY) {
    BigU al = BigU::from_words(alpha_host, L);
    if (cmp(al, ctx->Q) >= 0) return MOMA_ERR_INVALID_ARG;
    if (FULL != 0) {  // alpha R mod q: one Montgomery product gives alpha * x
      ctx->red->mulmod(al, BigU::from_words(ctx->k.R0, L)).to_words(p.alpha, L);
    } else {
      al.to_words(p.alpha, L);
      companion(ctx, al, p.alphap);
    }
  }
  p.status = ctx->d_status;
  p.wait_ns = ctx->wait_ns;
  p.log_tile = 0;
  p.inject = 0;
  return MOMA_OK;
}

template <int L, int OP, int V, int ENG, int FULL = 0>
moma_status run_vec(moma_ctx* ctx, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                           const uint32_t* alpha_host, cudaStream_t st) {
  VecArgs<L> p;
  moma_status rc = fill_vec_args<L, OP, FULL>(ctx, n, a, b, c, alpha_host, p);
  if (rc) return rc;
  // 256-thread CTAs (at 768 bits, where one such CTA fills an SM's registers, three CTAs of 128
  // threads measured 9% slower), as many per SM as fit
  static std::atomic<int> occ_cached{-1};  // per-instantiation occupancy, computed once
  int occ = occ_cached.load(std::memory_order_relaxed);
  if (occ < 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, vec_kernel<L, OP, V, ENG, FULL>, 256, 0) != cudaSuccess)
      return MOMA_ERR_CUDA;
    occ = o > 0 ? o : 1;
    occ_cached.store(occ, std::memory_order_relaxed);
  }
  const uint64_t units = n / V;
  uint64_t blocks = (units + 255) / 256;
  const uint64_t cap = (uint64_t)ctx->num_sms * (uint64_t)occ;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) return MOMA_OK;
  vec_kernel<L, OP, V, ENG, FULL><<<(unsigned)blocks, 256, 0, st>>>(p);
  return cuda_status(cudaGetLastError());
}

// Bulk copies need every plane of both operands to start on a 16-byte boundary.
inline bool vec_staged_ok(size_t n, const uint32_t* a, const uint32_t* b) {
  return n % 4 == 0 && (((uintptr_t)a | (uintptr_t)b) & 15u) == 0;
}

// ------------------------------------------------------------------ staged (bulk-copy) form
// The same element-wise operation with its operands brought into shared memory by the bulk-copy
// engine: a persistent grid, each CTA taking tiles of E = 256 U consecutive elements (U elements
// per thread, fixed per width by vec_staged_max_per_thread; log_tile = log2 E)
// (tiles blockIdx.x, blockIdx.x + gridDim.x, ...).  One thread issues, per tile, one
// cp.async.bulk per limb plane of each operand (2L copies of 4E bytes) into one of kVecStages
// shared-memory stages and arms the stage's mbarrier with the byte count; while the CTA computes
// tile k, the copies of tiles k+1 .. k+kVecStages-1 are in flight, so loads never stall the
// multiply pipe.  Every thread reads its elements' limbs from the stage (consecutive threads,
// consecutive words: no bank conflicts), the CTA synchronises (the stage may be refilled), and
// the results go straight to global memory (coalesced per plane).  Elements past the last whole
// tile take direct loads.  Needs 16-byte aligned operands and n a multiple of 4 (every plane
// starts on a 16-byte boundary).  A wait that runs out (wait_ns) records MOMA_ERR_TIMEOUT in the
// context's status word; the CTA then waits, bounded again, for its copies still in flight and
// returns.
constexpr int kVecStages = 3;
constexpr int kVecStagedThreads = 256;

template <int L>
__host__ __device__ constexpr uint32_t vec_stage_words(uint32_t E) {
  return 2u * L * E;
}

template <int L>
constexpr size_t vec_staged_smem(uint32_t log_tile) {
  return (size_t)kVecStages * vec_stage_words<L>(1u << log_tile) * 4u + kVecStages * sizeof(uint64_t);
}

// Elements per thread per tile, at most: 4 up to 128 bits, 2 at 256 bits, 1 at 384 bits (the
// operands of all of them are held in registers at once).  Wider containers are not staged: their
// products are bound by the multiply pipe, not by loads.
template <int L>
constexpr int vec_staged_max_per_thread() {
  return L <= 4 ? 4 : (L <= 8 ? 2 : (L <= 12 ? 1 : 0));
}

// Largest tile (log2 elements, 8..10) for L limbs; 0 if the width is not staged.  Every tile's
// stages fit the 227 KiB of shared memory a CTA may use.
template <int L>
constexpr int vec_staged_max_log_tile() {
  return vec_staged_max_per_thread<L>() == 4 ? 10
         : vec_staged_max_per_thread<L>() == 2 ? 9
         : vec_staged_max_per_thread<L>() == 1 ? 8
                                                : 0;
}
static_assert(vec_staged_smem<12>(8) <= 227u * 1024u && vec_staged_smem<8>(9) <= 227u * 1024u &&
                  vec_staged_smem<4>(10) <= 227u * 1024u,
              "staged tiles fit shared memory");

template <int L, int OP, int ENG, int FULL = 0>
__global__ void __launch_bounds__(kVecStagedThreads) vec_staged_kernel(const __grid_constant__ VecArgs<L> p) {
  extern __shared__ __align__(128) uint32_t sm[];
  constexpr int U = vec_staged_max_per_thread<L>();  // elements per thread per tile
  static_assert(U > 0, "width not staged");
  constexpr uint32_t E = (uint32_t)U * kVecStagedThreads;  // = 2^log_tile
  const uint32_t SW = vec_stage_words<L>(E);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kVecStages * SW);
  const uint32_t tid = threadIdx.x;
  const uint64_t ntiles = p.n >> p.log_tile;
  const uint64_t mine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  auto issue = [&](uint64_t k) {  // thread 0: tile k of this CTA into stage k % kVecStages
    const uint32_t s = (uint32_t)(k % kVecStages);
    const uint64_t off = (blockIdx.x + k * gridDim.x) << p.log_tile;
    uint32_t* dst = sm + s * SW;
    const uint32_t extra = (p.inject && blockIdx.x == 0 && k == 0) ? 16u : 0u;
    mbar_arrive_expect_tx(&bars[s], SW * 4u + extra);
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
      bulk_g2s(dst + l * E, p.a + (uint64_t)l * p.n + off, E * 4u, &bars[s]);
      bulk_g2s(dst + (L + l) * E, p.b + (uint64_t)l * p.n + off, E * 4u, &bars[s]);
    }
  };

  if (mine > 0) {
    if (tid == 0) {
      for (int s = 0; s < kVecStages; ++s) mbar_init(&bars[s], 1);
      fence_barrier_init();
      for (uint64_t k = 0; k < mine && k < (uint64_t)kVecStages; ++k) issue(k);
    }
    __syncthreads();
  }
#pragma unroll 1
  for (uint64_t k = 0; k < mine; ++k) {
    const uint32_t s = (uint32_t)(k % kVecStages);
    const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((k / kVecStages) & 1u), p.wait_ns);
    const uint32_t* st = sm + s * SW;
    uint32_t x[U][L], y[U][L];
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int l = 0; l < L; ++l) {
        x[u][l] = st[l * E + u * kVecStagedThreads + tid];
        y[u][l] = st[(L + l) * E + u * kVecStagedThreads + tid];
      }
    }
    // every thread has read stage s: it may be refilled; the timeout decision is CTA-wide
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        atomicExch(p.status, (int)MOMA_ERR_TIMEOUT);
        // copies still in flight target tiles k .. min(k + stages, mine) - 1: wait for them, bounded
        for (uint64_t j = k; j < mine && j < k + kVecStages; ++j)
          (void)mbar_wait_bounded(&bars[j % kVecStages], (uint32_t)((j / kVecStages) & 1u), p.wait_ns);
      }
      return;
    }
    if (tid == 0 && k + kVecStages < mine) issue(k + kVecStages);
    const uint64_t off = (blockIdx.x + k * gridDim.x) << p.log_tile;
    uint32_t z[U][L];  // the U elements are independent: their products interleave
#pragma unroll
    for (int u = 0; u < U; ++u) vec_apply<L, OP, ENG, FULL>(z[u], x[u], y[u], p);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t e = off + u * kVecStagedThreads + tid;
#pragma unroll
      for (int l = 0; l < L; ++l) p.c[(uint64_t)l * p.n + e] = z[u][l];
    }
  }
  // ragged tail: elements past the last whole tile, direct loads
  const uint64_t stride = (uint64_t)gridDim.x * kVecStagedThreads;
  for (uint64_t e = (ntiles << p.log_tile) + (uint64_t)blockIdx.x * kVecStagedThreads + tid; e < p.n; e += stride) {
    uint32_t x[L], y[L], z[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      x[l] = p.a[(uint64_t)l * p.n + e];
      y[l] = p.b[(uint64_t)l * p.n + e];
    }
    vec_apply<L, OP, ENG, FULL>(z, x, y, p);
#pragma unroll
    for (int l = 0; l < L; ++l) p.c[(uint64_t)l * p.n + e] = z[l];
  }
}

template <int L, int OP, int ENG, int FULL = 0>
moma_status run_vec_staged(moma_ctx* ctx, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                           const uint32_t* alpha_host, int log_tile, cudaStream_t st) {
  VecArgs<L> p;
  moma_status rc = fill_vec_args<L, OP, FULL>(ctx, n, a, b, c, alpha_host, p);
  if (rc) return rc;
  p.log_tile = (uint32_t)log_tile;
  p.inject = ctx->inject_missing_copy.exchange(0) ? 1u : 0u;
  const size_t smem = vec_staged_smem<L>((uint32_t)log_tile);
  auto kern = vec_staged_kernel<L, OP, ENG, FULL>;
  // the largest tile this kernel is launched with sets the shared-memory attribute; the attribute
  // and the occupancy are per device and tile size
  static std::atomic<uint64_t> attr_done[3] = {};
  static std::atomic<int> occ_cached[3][64] = {};
  constexpr int kMaxTile = vec_staged_max_log_tile<L>();
  const int ti = log_tile - 8;
  if (log_tile != kMaxTile) return MOMA_ERR_INVALID_ARG;  // the kernel's tile is fixed per width
  const int dev = ctx->device & 63;
  const uint64_t dev_bit = 1ull << dev;
  if (!(attr_done[ti].load(std::memory_order_acquire) & dev_bit)) {
    // the attribute is the largest tile's, so that every tile size stays launchable
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)vec_staged_smem<L>(kMaxTile)) != cudaSuccess)
      return MOMA_ERR_CUDA;
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, kVecStagedThreads, smem) != cudaSuccess)
      return MOMA_ERR_CUDA;
    occ_cached[ti][dev].store(o > 0 ? o : 1, std::memory_order_relaxed);
    attr_done[ti].fetch_or(dev_bit, std::memory_order_release);
  }
  const int occ = occ_cached[ti][dev].load(std::memory_order_relaxed);
  const uint64_t ntiles = (uint64_t)n >> log_tile;
  uint64_t blocks = (uint64_t)ctx->num_sms * (uint64_t)occ;
  if (ntiles < blocks) blocks = ntiles > 0 ? ntiles : 1;
  kern<<<(unsigned)blocks, kVecStagedThreads, smem, st>>>(p);
  return cuda_status(cudaGetLastError());
}

template <int L, int OP, int ENG>
moma_status dispatch_v(moma_ctx* ctx, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                              const uint32_t* alpha, int vw, int log_tile, cudaStream_t st) {
  constexpr int VM = L <= 8 ? 4 : (L <= 12 ? 2 : 1);
  const uintptr_t mis = (uintptr_t)a | (uintptr_t)b | (uintptr_t)c;
  if constexpr (vec_staged_max_per_thread<L>() > 0) {
    if (log_tile != 0 && vec_staged_ok(n, a, b))
      return run_vec_staged<L, OP, ENG>(ctx, n, a, b, c, alpha, log_tile, st);
  }
  if (VM >= 4 && vw >= 4 && n % 4 == 0 && (mis & 15) == 0)
    return run_vec<L, OP, (VM >= 4 ? 4 : 1), ENG>(ctx, n, a, b, c, alpha, st);
  if (VM >= 2 && vw >= 2 && n % 2 == 0 && (mis & 7) == 0)
    return run_vec<L, OP, (VM >= 2 ? 2 : 1), ENG>(ctx, n, a, b, c, alpha, st);
  return run_vec<L, OP, 1, ENG>(ctx, n, a, b, c, alpha, st);
}

template <int L>
moma_status dispatch_op(moma_ctx* ctx, int op, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                               const uint32_t* alpha, const moma_config& cfg, cudaStream_t st) {
  const int eng = cfg.engine;
  const int vw = cfg.vec_width;
  const int lt = cfg.tile_log;
  if (ctx->mont) {  // full-width modulus, one element per thread
    switch (op) {
      case VEC_ADD: return run_vec<L, VEC_ADD, 1, 1, 1>(ctx, n, a, b, c, alpha, st);
      case VEC_SUB: return run_vec<L, VEC_SUB, 1, 1, 1>(ctx, n, a, b, c, alpha, st);
      case VEC_MUL:
        return eng == 4   ? run_vec<L, VEC_MUL, 1, 1, 2>(ctx, n, a, b, c, alpha, st)
               : eng == 3 ? run_vec<L, VEC_MUL, 1, 3, 1>(ctx, n, a, b, c, alpha, st)
               : eng == 2 ? run_vec<L, VEC_MUL, 1, 2, 1>(ctx, n, a, b, c, alpha, st)
                          : run_vec<L, VEC_MUL, 1, 1, 1>(ctx, n, a, b, c, alpha, st);
      case VEC_AXPY: return run_vec<L, VEC_AXPY, 1, 1, 2>(ctx, n, a, b, c, alpha, st);
    }
    return MOMA_ERR_INVALID_ARG;
  }
  switch (op) {
    case VEC_ADD: return dispatch_v<L, VEC_ADD, 1>(ctx, n, a, b, c, alpha, vw, lt, st);
    case VEC_SUB: return dispatch_v<L, VEC_SUB, 1>(ctx, n, a, b, c, alpha, vw, lt, st);
    case VEC_MUL:
      return eng == 2 ? dispatch_v<L, VEC_MUL, 2>(ctx, n, a, b, c, alpha, vw, lt, st)
             : eng == 3 ? dispatch_v<L, VEC_MUL, 3>(ctx, n, a, b, c, alpha, vw, lt, st)
                        : dispatch_v<L, VEC_MUL, 1>(ctx, n, a, b, c, alpha, vw, lt, st);
    case VEC_AXPY:
      return eng == 2 ? dispatch_v<L, VEC_AXPY, 2>(ctx, n, a, b, c, alpha, vw, lt, st)
                      : dispatch_v<L, VEC_AXPY, 1>(ctx, n, a, b, c, alpha, vw, lt, st);
  }
  return MOMA_ERR_INVALID_ARG;
}

}  // namespace moma
