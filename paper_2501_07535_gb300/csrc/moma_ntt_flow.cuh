// moma_ntt_flow.cuh -- every Stockham pass of a transform call in one persistent launch, each tile
// waiting only for the tiles of the previous pass it reads (device code).
//
// With one pass per launch, a pass whose tiles fill one or two waves of resident CTAs leaves most
// SMs idle while its last partial wave runs, and the next pass cannot start before the launch ends.
// Here a resident grid takes (pass, tile) entries from a queue in pass order; a tile of pass p+1
// reads R*G elements written by a handful of pass-p tiles (its producers) and waits until exactly
// those have finished (a per-tile completion counter reaching its producer count), so the first
// tiles of pass p+1 start while pass p drains.  Within a pass, tiles are queued in the order in
// which the next pass first needs them (computed on the host from the Stockham index map), so the
// head of every pass depends on tiles that were queued early.
//
// Progress: a tile only waits for tiles earlier in the queue, which were claimed by running CTAs;
// the earliest unfinished tile has all its producers finished, so its CTA runs and every wait ends.
// Each wait is bounded all the same: past the limit it records MOMA_ERR_TIMEOUT in the context's
// status word and the tile is skipped (its results undefined); the kernel never hangs.
#pragma once
#include "moma_ntt_tile.cuh"

namespace moma {

constexpr int kFlowMaxPasses = 6;

template <int L>
struct FlowArgs {
  NttPassArgs<L> pass[kFlowMaxPasses];
  uint32_t npass;
  uint32_t count;                    // transforms of the call
  uint32_t total;                    // tiles of one transform, all passes
  uint32_t tiles[kFlowMaxPasses];    // tiles of one transform in pass p
  uint32_t base[kFlowMaxPasses];     // sum of tiles[q], q < p
  const uint32_t* order;             // [total]: order[base[p] + pos] = the pass-p tile queued at pos
  const uint32_t* req;               // [total]: producers of (p, tile); 0 in pass 0
  const uint32_t* cons_off;          // [total + 1]: consumers of (p, tile) in pass p+1 ...
  const uint32_t* cons_idx;          // ... cons_idx[cons_off[base[p]+tile] .. cons_off[base[p]+tile+1])
  uint32_t* ctr;                     // [count * total] completion counters, zero at launch
  uint32_t* head;                    // queue head, zero at launch
  int* status;
  uint64_t wait_polls;
};

__device__ __forceinline__ uint32_t flow_ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Queue entry e -> (pass, position in the pass, transform).  Entries run pass by pass; within a
// pass position-major over the transforms, so the queued-first tiles of every transform come first.
template <int L>
__device__ __forceinline__ void flow_decode(const FlowArgs<L>& a, uint32_t e, uint32_t& p, uint32_t& pos,
                                            uint32_t& t) {
  p = 0;
  while (p + 1 < a.npass && e >= a.count * a.base[p + 1]) ++p;
  const uint32_t q = e - a.count * a.base[p];
  pos = q / a.count;
  t = q - pos * a.count;
}

template <int L, class A>
__device__ __forceinline__ void ntt_flow_body(const FlowArgs<L>& a, uint32_t* sm) {
  __shared__ uint32_t s_e, s_skip;
  const uint32_t entries = a.count * a.total;
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t e = atomicAdd(a.head, 1u);
      s_e = e;
      s_skip = 0;
      if (e < entries) {
        uint32_t p, pos, t;
        flow_decode(a, e, p, pos, t);
        if (p > 0) {
          const uint32_t tile = __ldg(a.order + a.base[p] + pos);
          const uint32_t need = __ldg(a.req + a.base[p] + tile);
          const uint32_t* c = a.ctr + (uint64_t)t * a.total + a.base[p] + tile;
          uint64_t polls = 0;
          while (flow_ld_acquire(c) < need) {
            if (++polls > a.wait_polls) {
              atomicExch(a.status, (int)MOMA_ERR_TIMEOUT);
              s_skip = 1;
              break;
            }
            __nanosleep(64);
          }
        }
      }
    }
    __syncthreads();
    const uint32_t e = s_e;
    if (e >= entries) return;
    uint32_t p, pos, t;
    flow_decode(a, e, p, pos, t);
    const uint32_t tile = __ldg(a.order + a.base[p] + pos);
    if (!s_skip) ntt_tile_impl<L, A>(a.pass[p], t * a.tiles[p] + tile, sm);
    __syncthreads();  // every store of the tile is issued; every thread has read s_e and s_skip
    if (threadIdx.x == 0 && p + 1 < a.npass) {
      __threadfence();
      const uint32_t k0 = __ldg(a.cons_off + a.base[p] + tile), k1 = __ldg(a.cons_off + a.base[p] + tile + 1);
      uint32_t* c = a.ctr + (uint64_t)t * a.total + a.base[p + 1];
      for (uint32_t k = k0; k < k1; ++k) atomicAdd(c + __ldg(a.cons_idx + k), 1u);
    }
  }
}

template <int L, int FE>
__global__ void __launch_bounds__(256) ntt_flow_kernel(const __grid_constant__ FlowArgs<L> a) {
  extern __shared__ __align__(16) uint32_t sm[];
  ntt_flow_body<L, BarrettArith<L, FE>>(a, sm);
}

}  // namespace moma
