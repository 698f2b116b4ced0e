// moma_ntt_tile.cuh -- one CTA tile of a Stockham NTT pass (device code shared by the
// per-pass kernels of moma_ntt.cu and the persistent batch kernel of moma_batch.cu).
#pragma once
#include "moma_consts.cuh"
#include "moma_internal.hpp"
#include "moma_limbs.cuh"

namespace moma {

// XOR swizzle of an element slot x of a tile of 2^logT slots: the low three bits are flipped by
// the top three.  Row-wise accesses (consecutive slots) stay a permutation of each aligned group
// of eight; the bit-reversed reads of the first passes (consecutive outputs come from slots that
// differ in their top bits) land on eight different low-bit patterns, i.e. different banks.
__device__ __forceinline__ uint32_t swz(uint32_t x, uint32_t logT) {
  return logT >= 6 ? x ^ ((x >> (logT - 3)) & 7u) : x;
}

// The tile is element-major: slot x holds the L limbs of one element in L/4 16-byte chunks.
// With an even chunk count the chunk index is flipped by bit 2 of the slot, so eight
// consecutive slots (one quarter-warp of 128-bit accesses) hit eight different bank groups.
template <int L>
__device__ __forceinline__ uint32_t chunk_of(uint32_t x, int c) {
  if constexpr ((L / 4) % 2 == 0) return (uint32_t)c ^ ((x >> 2) & 1u);
  else return (uint32_t)c;
}

// (A 64-bit container, L = 2, takes one 8-byte access per element instead.)
template <int L>
__device__ __forceinline__ void tile_load(const uint32_t* sm, uint32_t x, uint32_t (&v)[L]) {
  if constexpr (L % 4 != 0) {
    static_assert(L == 2, "limb counts are 2 or multiples of 4");
    const uint2 t = reinterpret_cast<const uint2*>(sm)[x];
    v[0] = t.x;
    v[1] = t.y;
    return;
  } else {
    const uint4* p = reinterpret_cast<const uint4*>(sm) + x * (L / 4);
#pragma unroll
    for (int c = 0; c < L / 4; ++c) {
      const uint4 t = p[chunk_of<L>(x, c)];
      v[4 * c] = t.x;
      v[4 * c + 1] = t.y;
      v[4 * c + 2] = t.z;
      v[4 * c + 3] = t.w;
    }
  }
}

template <int L>
__device__ __forceinline__ void tile_store(uint32_t* sm, uint32_t x, const uint32_t (&v)[L]) {
  if constexpr (L % 4 != 0) {
    reinterpret_cast<uint2*>(sm)[x] = make_uint2(v[0], v[1]);
  } else {
    uint4* p = reinterpret_cast<uint4*>(sm) + x * (L / 4);
#pragma unroll
    for (int c = 0; c < L / 4; ++c)
      p[chunk_of<L>(x, c)] = make_uint4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
  }
}

// One twiddle entry (value and companion) from an entry-major table, L/2 16-byte loads.
template <int L>
__device__ __forceinline__ void twiddle_load(const uint32_t* table, uint64_t entry, uint32_t (&w)[L],
                                             uint32_t (&wp)[L]) {
  if constexpr (L % 4 != 0) {  // L = 2: the whole entry is one 16-byte load
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(table + entry * 2 * L));
    w[0] = a.x;
    w[1] = a.y;
    wp[0] = a.z;
    wp[1] = a.w;
    return;
  }
  const uint4* p = reinterpret_cast<const uint4*>(table + entry * 2 * L);
#pragma unroll
  for (int c = 0; c < L / 4; ++c) {
    const uint4 a = __ldg(p + c), b = __ldg(p + L / 4 + c);
    w[4 * c] = a.x;
    w[4 * c + 1] = a.y;
    w[4 * c + 2] = a.z;
    w[4 * c + 3] = a.w;
    wp[4 * c] = b.x;
    wp[4 * c + 1] = b.y;
    wp[4 * c + 2] = b.z;
    wp[4 * c + 3] = b.w;
  }
}

template <int L>
struct NttPassArgs {
  const uint32_t* src;
  const uint32_t* src2;  // pointwise second operand (fused polynomial product), else null
  uint32_t* dst;
  const uint32_t* tw_pass;
  const uint32_t* tw_int;
  const uint32_t* psi;  // negacyclic pre/post factors, [n][2L] (F_PSI_IN / F_PSI_OUT)
  uint64_t tw_count;
  uint64_t n;
  uint32_t logR, logG, logNs;
  uint32_t tiles_per_transform;
  uint32_t flags;  // F_* below
  uint32_t sc[L], scp[L];
  ModK<L> k;
};

// F_PRETW: pre-twiddles (Ns > 1); F_SCALE: multiply by sc at load (n^-1 of the inverse);
// F_POINTWISE: product with src2 at load (fused polynomial product); F_LAST: canonical store;
// F_PSI_IN: multiply input position j by psi[j] at load (negacyclic forward);
// F_PSI_OUT: multiply output position j by psi[j] at the store (negacyclic inverse).
enum { F_PRETW = 1, F_SCALE = 2, F_POINTWISE = 4, F_LAST = 8, F_PSI_IN = 16, F_PSI_OUT = 32 };

// DIF butterfly on lazy values: a, b in [0, 4q) -> (a + b, (a - b) * w) both in [0, 4q).
// With MUL false the twiddle is 1.  FE: the product form of mulmod_fixed_lazy.
template <int L, int FE>
__device__ __forceinline__ void dif_butterfly_lazy(uint32_t (&a)[L], uint32_t (&b)[L], bool mul,
                                                   const uint32_t* table, uint32_t entry, const ModK<L>& k) {
  uint32_t x[L], d[L];
  add_words<L, false>(x, a, b);  // [0, 8q)
  cond_sub<L>(x, k.q4);           // [0, 4q)
  add_words<L, false>(d, a, k.q4);
  sub_words<L, false>(d, d, b);   // a + 4q - b in (0, 8q)
  if (mul) {
    uint32_t w[L], wp[L];
    twiddle_load<L>(table, entry, w, wp);
    mulmod_fixed_lazy<L, FE>(b, d, w, wp, k);  // [0, 3q)
  } else {
    cond_sub<L>(d, k.q4);
#pragma unroll
    for (int l = 0; l < L; ++l) b[l] = d[l];
  }
#pragma unroll
  for (int l = 0; l < L; ++l) a[l] = x[l];
}

// The modular arithmetic of a transform pass, by reduction.
// Barrett contexts (B = W - 4): lazy values in [0, 4q) inside a transform, twiddles with Barrett
// companions (mulmod_fixed_lazy with product form FE), canonical store at the end.
template <int L, int FE>
struct BarrettArith {
  static __device__ __forceinline__ void pointwise(uint32_t (&v)[L], const uint32_t (&u)[L], const ModK<L>& k) {
    uint32_t t[L];
    mulmod_barrett<L, FE == 2>(t, v, u, k);
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = t[l];
  }
  static __device__ __forceinline__ void mul_fixed(uint32_t (&v)[L], const uint32_t (&w)[L], const uint32_t (&wp)[L],
                                                   const ModK<L>& k) {
    uint32_t t[L];
    mulmod_fixed_lazy<L, FE>(t, v, w, wp, k);
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = t[l];
  }
  static __device__ __forceinline__ void butterfly(uint32_t (&a)[L], uint32_t (&b)[L], bool mul, const uint32_t* table,
                                                   uint32_t entry, const ModK<L>& k) {
    dif_butterfly_lazy<L, FE>(a, b, mul, table, entry, k);
  }
  static __device__ __forceinline__ void finish(uint32_t (&v)[L], const ModK<L>& k) {  // [0, 4q) -> [0, q)
    cond_sub<L>(v, k.q2);
    cond_sub<L>(v, k.q);
  }
};

// Full-width contexts (up to B = W): canonical values throughout, twiddles and constants in
// Montgomery form (w R mod q; the companion half of each table entry is unused), Montgomery
// products.  The pointwise product of two canonical values is exact (mulmod_mont).
template <int L>
struct MontArith {
  static __device__ __forceinline__ void pointwise(uint32_t (&v)[L], const uint32_t (&u)[L], const ModK<L>& k) {
    uint32_t t[L];
    mulmod_mont<L>(t, v, u, k);
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = t[l];
  }
  static __device__ __forceinline__ void mul_fixed(uint32_t (&v)[L], const uint32_t (&w)[L], const uint32_t (&wp)[L],
                                                   const ModK<L>& k) {
    (void)wp;
    uint32_t t[L];
    montmul<L>(t, v, w, k);
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = t[l];
  }
  static __device__ __forceinline__ void butterfly(uint32_t (&a)[L], uint32_t (&b)[L], bool mul, const uint32_t* table,
                                                   uint32_t entry, const ModK<L>& k) {
    uint32_t x[L], d[L];
    addmod_full<L>(x, a, b, k.q);
    submod<L>(d, a, b, k.q);
    if (mul) {
      uint32_t w[L], wp[L];
      twiddle_load<L>(table, entry, w, wp);
      montmul<L>(b, d, w, k);
    } else {
#pragma unroll
      for (int l = 0; l < L; ++l) b[l] = d[l];
    }
#pragma unroll
    for (int l = 0; l < L; ++l) a[l] = x[l];
  }
  static __device__ __forceinline__ void finish(uint32_t (&v)[L], const ModK<L>& k) {
    (void)v;
    (void)k;
  }
};

// Where a pass's tile elements come from and where its outputs go.  `base` is the transform's
// first word (b * L * n), `pos` the element's position in the transform, `e` its tile slot
// before the swizzle.  GlobalIO: the transform's buffers in global memory (every per-pass
// launch, the batch kernel, the first load and the last store of a fused transform), read with
// L2-only loads so that data written earlier in the same persistent launch by other SMs is never
// served from a stale L1 line.
struct GlobalIO {
  template <int L>
  __device__ __forceinline__ void get(const NttPassArgs<L>& p, uint64_t base, uint64_t pos, uint32_t e,
                                      const uint32_t* sm, uint32_t logT, uint32_t (&v)[L]) const {
    (void)e;
    (void)sm;
    (void)logT;
#pragma unroll
    for (int l = 0; l < L; ++l) v[l] = __ldcg(p.src + base + pos + (uint64_t)l * p.n);
  }
  template <int L>
  __device__ __forceinline__ void put(const NttPassArgs<L>& p, uint64_t base, uint64_t pos,
                                      const uint32_t (&v)[L]) const {
#pragma unroll
    for (int l = 0; l < L; ++l) p.dst[base + pos + (uint64_t)l * p.n] = v[l];
  }
};

// One CTA tile of one Stockham pass: `tile` indexes (transform, group block).  `sm` holds
// L*R*G words.  Elements come in through `in` and leave through `out` (GlobalIO for the
// per-pass kernels and the persistent batch kernel).
template <int L, class A, class IN = GlobalIO, class OUT = GlobalIO>
__device__ __forceinline__ void ntt_tile_impl(const NttPassArgs<L>& p, uint32_t tile, uint32_t* sm,
                                              const IN& in = IN(), const OUT& out = OUT()) {
  const uint32_t R = 1u << p.logR;
  const uint32_t G = 1u << p.logG;
  const uint32_t T = R << p.logG;
  const uint32_t logT = p.logR + p.logG;
  const uint64_t b = tile / p.tiles_per_transform;
  const uint64_t jb = tile - b * p.tiles_per_transform;
  const uint64_t base = b * (uint64_t)L * p.n;
  const uint64_t j0 = jb << p.logG;
  const uint64_t nR = p.n >> p.logR;
  const uint64_t ns_mask = (1ull << p.logNs) - 1;

  // ---- load (+ pointwise product, scaling, pre-twiddle) into the tile
  for (uint32_t e = threadIdx.x; e < T; e += blockDim.x) {
    const uint32_t r = e >> p.logG, g = e & (G - 1);
    const uint64_t j = j0 + g;
    const uint64_t pos = j + (uint64_t)r * nR;
    uint32_t v[L];
    in.get(p, base, pos, e, sm, logT, v);
    if (p.flags & F_POINTWISE) {
      uint32_t u[L];
#pragma unroll
      for (int l = 0; l < L; ++l) u[l] = __ldcg(p.src2 + base + pos + (uint64_t)l * p.n);
      A::pointwise(v, u, p.k);
    }
    if (p.flags & F_SCALE) A::mul_fixed(v, p.sc, p.scp, p.k);
    if (p.flags & F_PSI_IN) {
      uint32_t w[L], wp[L];
      twiddle_load<L>(p.psi, pos, w, wp);
      A::mul_fixed(v, w, wp, p.k);
    }
    if ((p.flags & F_PRETW) && r != 0 && (j & ns_mask) != 0) {
      const uint64_t ti = (uint64_t)(r - 1) * (ns_mask + 1) + (j & ns_mask);
      uint32_t w[L], wp[L];
      twiddle_load<L>(p.tw_pass, ti, w, wp);
      A::mul_fixed(v, w, wp, p.k);
    }
    tile_store<L>(sm, swz(e, logT), v);  // e = r*G + g
  }
  __syncthreads();

  // ---- R-point transforms: logR radix-2 DIF stages, in place in the tile
  const uint32_t logNT = 31u - (uint32_t)__clz(blockDim.x);
  const uint32_t logW = logNT > p.logG ? logNT - p.logG : 0u;
#pragma unroll 1
  for (uint32_t s = 0; s < p.logR; ++s) {
    const uint32_t logh = p.logR - s - 1;
    const uint32_t h = 1u << logh;
#pragma unroll 1
    for (uint32_t bi = threadIdx.x; bi < (T >> 1); bi += blockDim.x) {
      // butterfly row u of group g; the W = NT/G rows one pass of the CTA takes are rotated by
      // the pass index, so that every warp gets its share of the unit-twiddle (i = 0) rows
      const uint32_t g = bi & (G - 1), u0 = bi >> p.logG;
      const uint32_t uh = u0 >> logW, wm = (1u << logW) - 1;
      const uint32_t u = (uh << logW) | ((u0 + uh) & wm);
      const uint32_t i = u & (h - 1), blk = u >> logh;
      const uint32_t p0 = (blk << (logh + 1)) + i;
      const uint32_t a0 = swz((p0 << p.logG) + g, logT), a1 = swz(((p0 + h) << p.logG) + g, logT);
      uint32_t x0[L], x1[L];
      tile_load<L>(sm, a0, x0);
      tile_load<L>(sm, a1, x1);
      // twiddle w_(2h)^i = w_R^(i * R/(2h)); 1 for i = 0 and in the last stage (h = 1)
      A::butterfly(x0, x1, i != 0, p.tw_int, i << s, p.k);
      tile_store<L>(sm, a0, x0);
      tile_store<L>(sm, a1, x1);
    }
    __syncthreads();
  }

  // ---- store: output s of group j goes to (j-k)*R + k + s*Ns; consecutive threads take
  // consecutive addresses (k fastest, then s, then the Ns-blocks of the tile).
  const uint32_t logGl = p.logG < p.logNs ? p.logG : p.logNs;
  const uint32_t Gl = 1u << logGl;
  for (uint32_t e = threadIdx.x; e < T; e += blockDim.x) {
    const uint32_t gl = e & (Gl - 1);
    const uint32_t sp = (e >> logGl) & (R - 1);
    const uint32_t gh = e >> (logGl + p.logR);
    const uint32_t g = (gh << logGl) + gl;
    const uint64_t j = j0 + g;
    const uint64_t kk = j & ns_mask;
    const uint64_t pos = (j - kk) * R + kk + ((uint64_t)sp << p.logNs);
    const uint32_t pr = __brev(sp) >> (32 - p.logR);
    uint32_t v[L];
    tile_load<L>(sm, swz((pr << p.logG) + g, logT), v);
    if (p.flags & F_PSI_OUT) {  // Barrett: [0, 4q) -> [0, 3q)
      uint32_t w[L], wp[L];
      twiddle_load<L>(p.psi, pos, w, wp);
      A::mul_fixed(v, w, wp, p.k);
    }
    if (p.flags & F_LAST) A::finish(v, p.k);
    out.put(p, base, pos, v);
  }
}

template <int L, int FE>
__device__ __forceinline__ void ntt_tile(const NttPassArgs<L>& p, uint32_t tile, uint32_t* sm) {
  ntt_tile_impl<L, BarrettArith<L, FE>>(p, tile, sm);
}

// Host: fill the arguments of one pass (count transforms of length 2^logn).
template <int L>
inline void fill_pass_args(const moma_ctx* ctx, const Plan* pl, const PassDesc& d, size_t count,
                           const uint32_t* src, const uint32_t* src2, uint32_t* dst, uint32_t flags,
                           NttPassArgs<L>& a) {
  a.src = src;
  a.src2 = src2;
  a.dst = dst;
  a.tw_pass = d.tw_pass;
  a.tw_int = d.tw_int;
  a.psi = pl->psi;
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
  (void)count;
}

}  // namespace moma
