// moma_blas_kern.cuh -- the element-wise kernels and their launchers as templates over the limb
// count.  moma_blas.cu instantiates them for up to 384 bits, moma_blas_wide.cu for 512 to 1024 bits.
//
// Data are limb-major: plane l of a length-n vector is the contiguous run v[l*n .. l*n+n).
// A thread handles V consecutive elements per step and reads each of the L planes with
// one V-wide vector load (uint4 for V = 4), so every load of a warp is a coalesced
// 32*V-word run of one plane.  Grid-stride loop over a grid sized to fill every SM.
#pragma once
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
    for (int v = 0; v < V; ++v) {
      if constexpr (FULL != 0) {
        if constexpr (OP == VEC_ADD) {
          addmod_full<L>(z[v], x[v], y[v], p.k.q);
        } else if constexpr (OP == VEC_SUB) {
          submod<L>(z[v], x[v], y[v], p.k.q);
        } else if constexpr (OP == VEC_MUL) {
          if constexpr (FULL == 2) mulmod_mont<L>(z[v], x[v], y[v], p.k);
          else mulmod_barrett_full<L, ENG>(z[v], x[v], y[v], p.k);
        } else {
          uint32_t ax[L];
          montmul<L>(ax, x[v], p.alpha, p.k);
          addmod_full<L>(z[v], ax, y[v], p.k.q);
        }
      } else if constexpr (OP == VEC_ADD) {
        addmod<L>(z[v], x[v], y[v], p.k.q);
      } else if constexpr (OP == VEC_SUB) {
        submod<L>(z[v], x[v], y[v], p.k.q);
      } else if constexpr (OP == VEC_MUL) {
        mulmod_barrett<L, ENG == 2, ENG == 3>(z[v], x[v], y[v], p.k);
      } else {
        uint32_t ax[L];
        mulmod_fixed<L, ENG == 2>(ax, x[v], p.alpha, p.alphap, p.k);
        addmod<L>(z[v], ax, y[v], p.k.q);
      }
    }
#pragma unroll
    for (int l = 0; l < L; ++l) {
      uint32_t tmp[V];
#pragma unroll
      for (int v = 0; v < V; ++v) tmp[v] = z[v][l];
      reinterpret_cast<VT*>(p.c + (uint64_t)l * p.n)[u] = VecT<V>::join(tmp);
    }
  }
}

template <int L, int OP, int V, int ENG, int FULL = 0>
moma_status run_vec(moma_ctx* ctx, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                           const uint32_t* alpha_host, cudaStream_t st) {
  VecArgs<L> p;
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

template <int L, int OP, int ENG>
moma_status dispatch_v(moma_ctx* ctx, size_t n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                              const uint32_t* alpha, int vw, cudaStream_t st) {
  constexpr int VM = L <= 8 ? 4 : (L <= 12 ? 2 : 1);
  const uintptr_t mis = (uintptr_t)a | (uintptr_t)b | (uintptr_t)c;
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
    case VEC_ADD: return dispatch_v<L, VEC_ADD, 1>(ctx, n, a, b, c, alpha, vw, st);
    case VEC_SUB: return dispatch_v<L, VEC_SUB, 1>(ctx, n, a, b, c, alpha, vw, st);
    case VEC_MUL:
      return eng == 2 ? dispatch_v<L, VEC_MUL, 2>(ctx, n, a, b, c, alpha, vw, st)
             : eng == 3 ? dispatch_v<L, VEC_MUL, 3>(ctx, n, a, b, c, alpha, vw, st)
                        : dispatch_v<L, VEC_MUL, 1>(ctx, n, a, b, c, alpha, vw, st);
    case VEC_AXPY:
      return eng == 2 ? dispatch_v<L, VEC_AXPY, 2>(ctx, n, a, b, c, alpha, vw, st)
                      : dispatch_v<L, VEC_AXPY, 1>(ctx, n, a, b, c, alpha, vw, st);
  }
  return MOMA_ERR_INVALID_ARG;
}

}  // namespace moma
