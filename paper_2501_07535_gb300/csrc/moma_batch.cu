// moma_batch.cu -- many transforms, cyclic products and vector ops of uneven sizes and mixed
// widths in one persistent launch.
//
// The paper runs many kernels concurrently by batching them (Sec. 5.1, "batch processing").
// Here a batch is decomposed into work tiles: one CTA tile of one Stockham pass of one
// transform (ntt_tile), or 2048 elements of one vector op.  Every tile belongs to a segment
// (one pass of one transform, or one vector op); segments are queued by level (the pass
// index, counting the forward passes of a cyclic product before its inverse) and a resident
// grid of CTAs takes tiles in queue order from a global counter.  A tile of pass p waits until
// every tile of pass p-1 of the same transform has finished (per-transform completion counters,
// release/acquire); the inverse of a cyclic product waits for both forward transforms.  Because
// a tile only waits for tiles that come earlier in the queue, and those were taken by CTAs that
// are resident and running, every wait ends.  Each wait is still bounded: past the limit the
// kernel records MOMA_ERR_TIMEOUT and skips the tile.
//
// Widths are mixed inside one launch: the CTA dispatches on the tile's limb count.  Products
// use whole mad.wide rows up to 256 bits and carry chains at 384 bits (the faster form of each
// width on GB300); results are identical either way.  Jobs at 512 bits and up and jobs over
// full-width moduli (Montgomery arithmetic) are not tiles of the persistent kernel (their registers
// and code would cut the occupancy of every other tile), nor are 64-bit jobs: they run with the
// per-call kernels right after it, on the same stream and inside the same CUDA graph.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "moma_internal.hpp"
#include "moma_limbs.cuh"
#include "moma_ntt_tile.cuh"

namespace moma {

constexpr int kBatchThreads = 128;
constexpr int kBatchMinBlocks = 5;      // register cap 102: five CTAs per SM where shared memory allows
constexpr int kBatchTileLog = 10;       // transform tiles of 2^10 elements
constexpr uint32_t kVecTile = 2048;     // elements per vector-op tile
constexpr uint64_t kDefaultWaitPolls = 1ull << 24;

enum : uint32_t { SEG_NTT = 0, SEG_VEC = 1 };

template <int L>
struct VecJobArgs {
  const uint32_t* a;
  const uint32_t* b;
  uint32_t* c;
  uint64_t n;
  uint32_t op;  // VecOp
  uint32_t alpha[L], alphap[L];
  ModK<L> k;
};

struct Seg {
  uint32_t kind, L;
  uint32_t first;   // first global tile of the segment
  uint32_t ntiles;
  uint32_t done_id;  // completion counter incremented by each tile
  uint32_t wait_id[2];
  uint32_t wait_count[2];  // wait until counter[wait_id] >= wait_count (0: no wait)
  const void* args;        // device copy of NttPassArgs<L> or VecJobArgs<L>
};

template <int L>
__device__ __forceinline__ void vec_tile(const VecJobArgs<L>& p, uint32_t tile) {
  const uint64_t begin = (uint64_t)tile * kVecTile;
  const uint64_t end = begin + kVecTile < p.n ? begin + kVecTile : p.n;
  for (uint64_t e = begin + threadIdx.x; e < end; e += blockDim.x) {
    uint32_t x[L], y[L], z[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      x[l] = __ldcg(p.a + e + (uint64_t)l * p.n);
      y[l] = __ldcg(p.b + e + (uint64_t)l * p.n);
    }
    switch (p.op) {
      case VEC_ADD: addmod<L>(z, x, y, p.k.q); break;
      case VEC_SUB: submod<L>(z, x, y, p.k.q); break;
      case VEC_MUL: mulmod_barrett<L, false>(z, x, y, p.k); break;
      default: {
        uint32_t ax[L];
        mulmod_fixed<L, 1>(ax, x, p.alpha, p.alphap, p.k);
        addmod<L>(z, ax, y, p.k.q);
      }
    }
#pragma unroll
    for (int l = 0; l < L; ++l) p.c[e + (uint64_t)l * p.n] = z[l];
  }
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// A CTA claims its next tile (one atomic, one look-up in the tile -> segment table) while it
// works on the current one, and waits for the next tile's dependencies right after publishing
// the current one.  Shared state is double-buffered by iteration parity.  Progress: the lowest
// unfinished tile depends only on finished tiles, and whichever resident CTA holds it (as its
// current or its claimed next tile) reaches it, so every wait ends.
__global__ void __launch_bounds__(kBatchThreads, kBatchMinBlocks)
    batch_kernel(const Seg* __restrict__ segs, const uint32_t* __restrict__ tile_seg, uint32_t total, uint32_t* ctr,
                 int* status, uint64_t wait_polls) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ uint32_t s_tile[2], s_seg[2], s_skip[2];
  auto claim = [&](int b) {  // thread 0
    const uint32_t t = atomicAdd(&ctr[0], 1u);
    s_tile[b] = t;
    s_seg[b] = t < total ? __ldg(tile_seg + t) : 0u;
  };
  auto wait_deps = [&](int b) {  // thread 0: bounded waits on the tile's dependency counters
    s_skip[b] = 0;
    if (s_tile[b] >= total) return;
    const Seg& sg = segs[s_seg[b]];
    for (int w = 0; w < 2; ++w) {
      if (sg.wait_count[w] == 0) continue;
      uint64_t polls = 0;
      while (ld_acquire(&ctr[1 + sg.wait_id[w]]) < sg.wait_count[w]) {
        if (++polls > wait_polls) {
          atomicExch(status, (int)MOMA_ERR_TIMEOUT);
          s_skip[b] = 1;
          break;
        }
        __nanosleep(128);
      }
    }
  };
  if (threadIdx.x == 0) {
    claim(0);
    wait_deps(0);
  }
  __syncthreads();
  for (int b = 0;; b ^= 1) {
    const uint32_t t = s_tile[b];
    if (t >= total) return;
    const uint32_t si = s_seg[b];
    const bool skip = s_skip[b] != 0;
    if (threadIdx.x == 0) claim(b ^ 1);
    const Seg sg = segs[si];
    if (!skip) {
      const uint32_t local = t - sg.first;
      if (sg.kind == SEG_NTT) {
        switch (sg.L) {
          case 4: ntt_tile<4, 2>(*static_cast<const NttPassArgs<4>*>(sg.args), local, sm); break;
          case 8: ntt_tile<8, 2>(*static_cast<const NttPassArgs<8>*>(sg.args), local, sm); break;
          case 12: ntt_tile<12, 1>(*static_cast<const NttPassArgs<12>*>(sg.args), local, sm); break;
        }
      } else {
        switch (sg.L) {
          case 4: vec_tile<4>(*static_cast<const VecJobArgs<4>*>(sg.args), local); break;
          case 8: vec_tile<8>(*static_cast<const VecJobArgs<8>*>(sg.args), local); break;
          case 12: vec_tile<12>(*static_cast<const VecJobArgs<12>*>(sg.args), local); break;
        }
      }
    }
    __syncthreads();  // every store of the tile is issued
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&ctr[1 + sg.done_id], 1u);
      wait_deps(b ^ 1);
    }
    __syncthreads();
  }
}

}  // namespace moma

using namespace moma;

// A 768-bit job of a batch, run with the per-call kernels after the persistent launch
// (transform intermediates in the batch's scratch: [s1 | s2 | fa | fb]; vector ops keep a copy
// of the axpy scalar).
struct BatchDeferred {
  int op = 0;
  size_t n = 0;
  std::vector<uint32_t> alpha;
  moma_ctx* ctx = nullptr;
  const moma::Plan* fwd = nullptr;
  const moma::Plan* inv = nullptr;
  const uint32_t* a = nullptr;
  const uint32_t* b = nullptr;
  uint32_t* out = nullptr;
  uint32_t* scratch = nullptr;
  size_t w = 0;
  moma_config cfg = {};
};

struct moma_batch {
  int device = 0;
  std::vector<BatchDeferred> deferred;
  int runs = 0;
  std::vector<Seg> segs;
  uint32_t total = 0;
  uint32_t ncounters = 0;
  size_t smem = 0;
  int grid = 0;
  uint64_t wait_polls = kDefaultWaitPolls;
  // one device block holds the small arrays below (filled by one copy at creation)
  uint8_t* d_block = nullptr;
  Seg* d_segs = nullptr;
  uint32_t* d_tile_seg = nullptr;  // segment index of every tile
  uint8_t* d_args = nullptr;
  uint32_t* d_ctr = nullptr;
  int* d_status = nullptr;
  uint32_t* d_scratch = nullptr;
  cudaEvent_t ready = nullptr;  // recorded after the creation's upload on the set-up stream
  bool ready_seen = false;      // the host has seen `ready` complete
  cudaGraphExec_t graph = nullptr;
  bool dirty = false;  // descriptors changed since upload
};

namespace {

// Per-device stream for batch set-up and tear-down: allocations and uploads are stream-ordered
// there (cudaMallocAsync / cudaFreeAsync), so creating or destroying a batch never waits for
// the work other streams have in flight.
cudaStream_t setup_stream(int dev) {
  static std::mutex lock;
  static cudaStream_t streams[64] = {};
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(lock);
  if (!streams[dev]) cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
  return streams[dev];
}

struct ArgBuf {
  std::vector<uint8_t> bytes;
  template <typename T>
  size_t put(const T& v) {
    size_t off = (bytes.size() + 15) & ~(size_t)15;
    bytes.resize(off + sizeof(T));
    memcpy(bytes.data() + off, &v, sizeof(T));
    return off;
  }
};

struct PendingSeg {
  int level, job, sub;
  Seg s;
  size_t arg_off;
};

template <int L>
void ntt_pass_args(const moma_ctx* ctx, const Plan* pl, size_t pass, const uint32_t* src, const uint32_t* src2,
                   uint32_t* dst, uint32_t flags, ArgBuf& ab, size_t* off, uint32_t* ntiles) {
  NttPassArgs<L> a;
  fill_pass_args<L>(ctx, pl, pl->passes[pass], 1, src, src2, dst, flags, a);
  *ntiles = a.tiles_per_transform;
  *off = ab.put(a);
}

template <int L>
size_t vec_args(const moma_ctx* ctx, const moma_job& j, ArgBuf& ab) {
  VecJobArgs<L> a;
  a.a = j.a;
  a.b = j.b;
  a.c = j.out;
  a.n = j.n;
  a.op = (uint32_t)(j.op - MOMA_OP_ADD);
  fill_modk<L>(ctx, a.k);
  for (int i = 0; i < L; ++i) {
    a.alpha[i] = 0;
    a.alphap[i] = 0;
  }
  if (j.op == MOMA_OP_AXPY) {
    BigU al = BigU::from_words(j.alpha, L);
    al.to_words(a.alpha, L);
    companion(ctx, al, a.alphap);
  }
  return ab.put(a);
}

moma_status pass_args_l(const moma_ctx* ctx, const Plan* pl, size_t pass, const uint32_t* src, const uint32_t* src2,
                        uint32_t* dst, uint32_t flags, ArgBuf& ab, size_t* off, uint32_t* ntiles) {
  switch (ctx->L) {
    case 4: ntt_pass_args<4>(ctx, pl, pass, src, src2, dst, flags, ab, off, ntiles); return MOMA_OK;
    case 8: ntt_pass_args<8>(ctx, pl, pass, src, src2, dst, flags, ab, off, ntiles); return MOMA_OK;
    case 12: ntt_pass_args<12>(ctx, pl, pass, src, src2, dst, flags, ab, off, ntiles); return MOMA_OK;
  }
  return MOMA_ERR_UNSUPPORTED;
}

// Jobs the persistent kernel runs as tiles: Barrett contexts of 128, 256 and 384 bits.  The others
// (64-bit containers, 512 bits and up, full-width moduli) run with the per-call kernels after it.
bool batch_tile_kind(const moma_ctx* ctx) { return !ctx->mont && (ctx->L == 4 || ctx->L == 8 || ctx->L == 12); }

int log2_n(size_t n) {
  if (n == 0 || (n & (n - 1))) return -1;
  int k = 0;
  while (((size_t)1 << k) < n) ++k;
  return k;
}

// Appends the segments of one transform (sub-job `sub` of job `job`) to `out`.
moma_status add_transform(const moma_ctx* ctx, const Plan* pl, int job, int sub, int level0, uint32_t counter,
                          const uint32_t* in, const uint32_t* in2, uint32_t* out, uint32_t* s1, uint32_t* s2,
                          const uint32_t wait_ids[2], const uint32_t wait_counts[2], ArgBuf& ab,
                          std::vector<PendingSeg>& segs, uint32_t* total_tiles) {
  const size_t P = pl->passes.size();
  const uint32_t* src = in;
  uint32_t before = 0;
  for (size_t i = 0; i < P; ++i) {
    uint32_t* dst = (i + 1 == P) ? out : ((i % 2 == 0) ? s1 : s2);
    uint32_t flags = (i + 1 == P) ? F_LAST : 0;
    if (i == 0 && in2) flags |= F_POINTWISE;
    if (i == 0 && pl->inverse) flags |= F_SCALE;
    PendingSeg ps;
    ps.level = level0 + (int)i;
    ps.job = job;
    ps.sub = sub;
    ps.s = Seg{};
    ps.s.kind = SEG_NTT;
    ps.s.L = (uint32_t)ctx->L;
    ps.s.done_id = counter;
    uint32_t nt = 0;
    moma_status rc = pass_args_l(ctx, pl, i, src, i == 0 ? in2 : nullptr, dst, flags, ab, &ps.arg_off, &nt);
    if (rc) return rc;
    ps.s.ntiles = nt;
    if (i == 0) {
      for (int w = 0; w < 2; ++w) {
        ps.s.wait_id[w] = wait_ids[w];
        ps.s.wait_count[w] = wait_counts[w];
      }
    } else {
      ps.s.wait_id[0] = counter;
      ps.s.wait_count[0] = before;
    }
    before += nt;
    segs.push_back(ps);
    src = dst;
  }
  *total_tiles = before;
  return MOMA_OK;
}

// CTAs of the persistent kernel that fit the device at once with `smem` bytes of shared memory
// each (every CTA resident: the dependency waits rely on it); the kernel attribute is set once
// per device and the occupancy kept per (device, shared memory size).  0 on a CUDA error.
int resident_grid(int dev, size_t smem) {
  static std::mutex lock;
  static uint64_t attr_done = 0;
  static std::map<std::pair<int, size_t>, int> grids;
  std::lock_guard<std::mutex> g(lock);
  const auto key = std::make_pair(dev, smem);
  const auto it = grids.find(key);
  if (it != grids.end()) return it->second;
  const uint64_t bit = 1ull << (dev & 63);
  if (!(attr_done & bit)) {
    if (cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(12 * 4 << kBatchTileLog)) !=
        cudaSuccess)
      return 0;
    attr_done |= bit;
  }
  int occ = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel, kBatchThreads, smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || occ <= 0)
    return 0;
  grids[key] = occ * sms;
  return occ * sms;
}

// Order work on `st` after the creation's upload: a stream wait on the event, or, while the
// caller captures `st` into a graph (an outside event cannot join it), a host wait, once.
moma_status wait_ready(moma_batch* b, cudaStream_t st) {
  if (b->ready_seen) return MOMA_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (st && cudaStreamIsCapturing(st, &cap) != cudaSuccess) return MOMA_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) {
    if (cudaEventSynchronize(b->ready) != cudaSuccess) return MOMA_ERR_CUDA;
    b->ready_seen = true;
    return MOMA_OK;
  }
  return cuda_status(cudaStreamWaitEvent(st, b->ready, 0));
}

}  // namespace

extern "C" moma_status moma_batch_create(const moma_job* jobs, int njobs, moma_batch** out) {
  if (!out) return MOMA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!jobs || njobs <= 0) return MOMA_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MOMA_ERR_CUDA;

  // validate and size the scratch
  size_t scratch_words = 0;
  std::vector<size_t> scratch_off(njobs, 0);
  std::vector<const Plan*> fwd(njobs, nullptr), inv(njobs, nullptr);
  for (int j = 0; j < njobs; ++j) {
    const moma_job& jb = jobs[j];
    moma_ctx* ctx = jb.ctx;
    if (!ctx || !jb.a || !jb.out) return MOMA_ERR_INVALID_ARG;
    if (ctx->device != dev) return MOMA_ERR_INVALID_ARG;
    const bool ntt = jb.op == MOMA_OP_NTT_FWD || jb.op == MOMA_OP_NTT_INV || jb.op == MOMA_OP_POLYMUL;
    if (!ntt && (jb.op < MOMA_OP_ADD || jb.op > MOMA_OP_AXPY)) return MOMA_ERR_INVALID_ARG;
    if ((jb.op == MOMA_OP_POLYMUL || (!ntt)) && !jb.b) return MOMA_ERR_INVALID_ARG;
    if (jb.op == MOMA_OP_AXPY && !jb.alpha) return MOMA_ERR_INVALID_ARG;
    if (((uintptr_t)jb.a | (uintptr_t)jb.out | (uintptr_t)jb.b) & 3u) return MOMA_ERR_ALIGN;
    if (!ntt) {
      if (jb.n == 0) return MOMA_ERR_SIZE;
      if (jb.op == MOMA_OP_AXPY && cmp(BigU::from_words(jb.alpha, ctx->L), ctx->Q) >= 0) return MOMA_ERR_INVALID_ARG;
      continue;
    }
    const int lg = log2_n(jb.n);
    if (lg < 1 || lg > kMaxLogN) return MOMA_ERR_SIZE;
    // jobs run with the per-call kernels (768 bits, full-width moduli) keep the schedule of a
    // per-call transform (one transform: the little-work default applies)
    const bool per_call = !batch_tile_kind(ctx);
    moma_config cfg = ntt_config(ctx, jb.op, lg, per_call ? 1 : 0);
    const int tl = per_call ? cfg.tile_log : std::min(cfg.tile_log, kBatchTileLog);
    const int rmax = per_call ? cfg.max_logr : std::min(cfg.max_logr, tl);
    Plan* pl = nullptr;
    moma_status rc;
    if (jb.op != MOMA_OP_NTT_INV) {
      rc = get_plan(ctx, lg, false, tl, rmax, &pl);
      if (rc) return rc;
      fwd[j] = pl;
    }
    if (jb.op != MOMA_OP_NTT_FWD) {
      rc = get_plan(ctx, lg, true, tl, rmax, &pl);
      if (rc) return rc;
      inv[j] = pl;
    }
    const size_t w = (size_t)ctx->L * jb.n;
    scratch_off[j] = scratch_words;
    // transforms: two ping-pong buffers; cyclic product: two more for the forward outputs
    scratch_words += (jb.op == MOMA_OP_POLYMUL ? 6 : 2) * w;
    scratch_words = (scratch_words + 63) & ~(size_t)63;
  }

  moma_batch* b = new (std::nothrow) moma_batch();
  if (!b) return MOMA_ERR_OOM;
  b->device = dev;
  cudaStream_t ss = setup_stream(dev);
  if (!ss) {
    delete b;
    return MOMA_ERR_CUDA;
  }
  if (scratch_words && cudaMallocAsync(&b->d_scratch, scratch_words * 4, ss) != cudaSuccess) {
    delete b;
    return MOMA_ERR_OOM;
  }

  ArgBuf ab;
  std::vector<PendingSeg> pend;
  uint32_t counter = 0;
  moma_status rc = MOMA_OK;
  for (int j = 0; j < njobs && rc == MOMA_OK; ++j) {
    const moma_job& jb = jobs[j];
    moma_ctx* ctx = jb.ctx;
    const uint32_t no_id[2] = {0, 0}, no_cnt[2] = {0, 0};
    uint32_t* base = b->d_scratch + scratch_off[j];
    const size_t w = (size_t)ctx->L * jb.n;
    if (!batch_tile_kind(ctx)) {  // 64, 512, 768, 1024 bits, full-width moduli: per-call kernels afterwards
      BatchDeferred d;
      d.op = jb.op;
      d.n = jb.n;
      if (jb.op == MOMA_OP_AXPY) d.alpha.assign(jb.alpha, jb.alpha + ctx->L);
      d.ctx = ctx;
      d.fwd = fwd[j];
      d.inv = inv[j];
      d.a = jb.a;
      d.b = jb.b;
      d.out = jb.out;
      d.scratch = base;
      d.w = w;
      if (jb.op <= MOMA_OP_POLYMUL) d.cfg = ntt_config(ctx, jb.op, log2_n(jb.n), 1);
      b->deferred.push_back(d);
    } else if (jb.op == MOMA_OP_NTT_FWD || jb.op == MOMA_OP_NTT_INV) {
      const Plan* pl = jb.op == MOMA_OP_NTT_FWD ? fwd[j] : inv[j];
      uint32_t tiles = 0;
      rc = add_transform(ctx, pl, j, 0, 0, counter++, jb.a, nullptr, jb.out, base, base + w, no_id, no_cnt, ab, pend,
                         &tiles);
    } else if (jb.op == MOMA_OP_POLYMUL) {
      uint32_t* fa = base + 2 * w;
      uint32_t* fb = base + 3 * w;
      const uint32_t ca = counter++, cb = counter++, cc = counter++;
      uint32_t ta = 0, tb = 0, tc = 0;
      rc = add_transform(ctx, fwd[j], j, 0, 0, ca, jb.a, nullptr, fa, base, base + w, no_id, no_cnt, ab, pend, &ta);
      if (!rc)
        rc = add_transform(ctx, fwd[j], j, 1, 0, cb, jb.b, nullptr, fb, base + 4 * w, base + 5 * w, no_id, no_cnt,
                           ab, pend, &tb);
      if (!rc) {
        const uint32_t ids[2] = {ca, cb}, cnts[2] = {ta, tb};
        rc = add_transform(ctx, inv[j], j, 2, (int)fwd[j]->passes.size(), cc, fa, fb, jb.out, base, base + w, ids,
                           cnts, ab, pend, &tc);
      }
    } else {
      PendingSeg ps;
      ps.level = 0;
      ps.job = j;
      ps.sub = 0;
      ps.s = Seg{};
      ps.s.kind = SEG_VEC;
      ps.s.L = (uint32_t)ctx->L;
      ps.s.done_id = counter++;
      ps.s.ntiles = (uint32_t)((jb.n + kVecTile - 1) / kVecTile);
      switch (ctx->L) {
        case 4: ps.arg_off = vec_args<4>(ctx, jb, ab); break;
        case 8: ps.arg_off = vec_args<8>(ctx, jb, ab); break;
        case 12: ps.arg_off = vec_args<12>(ctx, jb, ab); break;
        default: ps.arg_off = vec_args<24>(ctx, jb, ab); break;
      }
      pend.push_back(ps);
    }
  }
  if (rc) {
    moma_batch_destroy(b);
    return rc;
  }
  // queue order: level; within a level the segments with the most work (tiles x L^2) first, so that
  // the large transforms' passes end early in the level and their next pass never waits at the
  // level's end (measured 2.2% faster on the uneven 256-job batch than job order; ordering by the
  // levels left after the segment first gave 1.7%); then job and sub-transform
  std::stable_sort(pend.begin(), pend.end(), [](const PendingSeg& x, const PendingSeg& y) {
    const uint64_t wx = (uint64_t)x.s.ntiles * x.s.L * x.s.L, wy = (uint64_t)y.s.ntiles * y.s.L * y.s.L;
    if (x.level != y.level) return x.level < y.level;
    if (wx != wy) return wx > wy;
    return std::make_tuple(x.job, x.sub) < std::make_tuple(y.job, y.sub);
  });
  uint64_t total = 0;
  for (const auto& ps : pend) total += ps.s.ntiles;
  if (total >= 0xffffffffull) {
    moma_batch_destroy(b);
    return MOMA_ERR_SIZE;
  }
  // one device block: arguments | segments | tile -> segment map | status word | counters, each
  // part 256-byte aligned; everything before the counters is copied from one host image (the
  // counters are reset by every run)
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t o_segs = align(std::max<size_t>(ab.bytes.size(), 16));
  const size_t o_tseg = o_segs + align(std::max<size_t>(pend.size(), 1) * sizeof(Seg));
  const size_t o_stat = o_tseg + align(std::max<size_t>((size_t)total, 1) * 4);
  const size_t o_ctr = o_stat + 256;
  const size_t block_bytes = o_ctr + align((1 + (size_t)counter) * sizeof(uint32_t));
  if (cudaMallocAsync(&b->d_block, block_bytes, ss) != cudaSuccess) {
    moma_batch_destroy(b);
    return MOMA_ERR_OOM;
  }
  b->d_args = b->d_block;
  b->d_segs = reinterpret_cast<Seg*>(b->d_block + o_segs);
  b->d_tile_seg = reinterpret_cast<uint32_t*>(b->d_block + o_tseg);
  b->d_status = reinterpret_cast<int*>(b->d_block + o_stat);
  b->d_ctr = reinterpret_cast<uint32_t*>(b->d_block + o_ctr);
  std::vector<uint8_t> img(o_ctr, 0);  // the status word starts at 0
  uint32_t* tile_seg = reinterpret_cast<uint32_t*>(img.data() + o_tseg);
  uint64_t first = 0;
  for (const auto& ps : pend) {
    Seg sg = ps.s;
    sg.first = (uint32_t)first;
    sg.args = b->d_args + ps.arg_off;
    std::fill(tile_seg + first, tile_seg + first + sg.ntiles, (uint32_t)b->segs.size());
    first += sg.ntiles;
    b->segs.push_back(sg);
  }
  b->total = (uint32_t)total;
  b->ncounters = counter;
  memcpy(img.data(), ab.bytes.data(), ab.bytes.size());
  memcpy(img.data() + o_segs, b->segs.data(), b->segs.size() * sizeof(Seg));
  // a copy from pageable memory returns once the image is staged, so `img` may go out of scope;
  // runs wait for `ready` instead of the host waiting here
  if (cudaMemcpyAsync(b->d_block, img.data(), o_ctr, cudaMemcpyHostToDevice, ss) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(b->ready, ss) != cudaSuccess) {
    moma_batch_destroy(b);
    return MOMA_ERR_CUDA;
  }
  // shared memory: the largest transform tile of the batch
  size_t smem = 0;
  for (int j = 0; j < njobs; ++j)
    if (jobs[j].op <= MOMA_OP_POLYMUL && batch_tile_kind(jobs[j].ctx))
      smem = std::max(smem, (size_t)jobs[j].ctx->L * 4u << kBatchTileLog);
  b->smem = smem;
  const int grid = resident_grid(dev, smem);
  if (grid <= 0) {
    moma_batch_destroy(b);
    return MOMA_ERR_CUDA;
  }
  b->grid = grid;  // every CTA resident at once: the waits rely on it
  *out = b;
  return MOMA_OK;
}

static moma_status batch_launch(moma_batch* b, cudaStream_t st) {
  if (b->total > 0) {
    if (cudaMemsetAsync(b->d_ctr, 0, (1 + b->ncounters) * sizeof(uint32_t), st) != cudaSuccess) return MOMA_ERR_CUDA;
    batch_kernel<<<b->grid, kBatchThreads, b->smem, st>>>(b->d_segs, b->d_tile_seg, b->total, b->d_ctr, b->d_status,
                                                          b->wait_polls);
    const moma_status rc = cuda_status(cudaGetLastError());
    if (rc) return rc;
  }
  for (const BatchDeferred& d : b->deferred) {
    uint32_t* s1 = d.scratch;
    uint32_t* s2 = d.scratch + d.w;
    moma_status rc;
    if (d.op == MOMA_OP_NTT_FWD) {
      rc = run_plan_buffers(d.ctx, d.fwd, 1, d.a, nullptr, d.out, d.cfg, s1, s2, st);
    } else if (d.op == MOMA_OP_NTT_INV) {
      rc = run_plan_buffers(d.ctx, d.inv, 1, d.a, nullptr, d.out, d.cfg, s1, s2, st);
    } else if (d.op >= MOMA_OP_ADD) {
      rc = launch_vec(d.ctx, d.op - MOMA_OP_ADD, d.n, d.a, d.b, d.out, d.alpha.empty() ? nullptr : d.alpha.data(), st);
    } else {
      uint32_t* fa = d.scratch + 2 * d.w;
      uint32_t* fb = d.scratch + 3 * d.w;
      rc = run_plan_buffers(d.ctx, d.fwd, 1, d.a, nullptr, fa, d.cfg, s1, s2, st);
      if (!rc) rc = run_plan_buffers(d.ctx, d.fwd, 1, d.b, nullptr, fb, d.cfg, s1, s2, st);
      if (!rc) rc = run_plan_buffers(d.ctx, d.inv, 1, fa, fb, d.out, d.cfg, s1, s2, st);
    }
    if (rc) return rc;
  }
  return MOMA_OK;
}

extern "C" moma_status moma_batch_run(moma_batch* b, void* stream) {
  if (!b) return MOMA_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const moma_status wr = wait_ready(b, st);
  if (wr) return wr;
  if (b->dirty) {
    if (cudaMemcpyAsync(b->d_segs, b->segs.data(), b->segs.size() * sizeof(Seg), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return MOMA_ERR_CUDA;
    b->dirty = false;
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (st == nullptr || b->runs++ == 0 || cudaStreamIsCapturing(st, &cap) != cudaSuccess ||
      cap != cudaStreamCaptureStatusNone)
    return batch_launch(b, st);  // legacy stream, first run, or inside the caller's capture
  if (!b->graph) {
    // capture the counter reset and the persistent launch once, replay it afterwards
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MOMA_ERR_CUDA;
    moma_status rc = batch_launch(b, st);
    if (cudaStreamEndCapture(st, &g) != cudaSuccess || rc) {
      if (g) cudaGraphDestroy(g);
      return rc ? rc : MOMA_ERR_CUDA;
    }
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return MOMA_ERR_CUDA;
    b->graph = ex;
  }
  return cuda_status(cudaGraphLaunch(b->graph, st));
}

extern "C" moma_status moma_batch_sync_status(moma_batch* b) {
  if (!b) return MOMA_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return MOMA_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, b->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MOMA_ERR_CUDA;
  if (v) cudaMemset(b->d_status, 0, sizeof(int));
  return (moma_status)v;
}

extern "C" moma_status moma_batch_set_wait_limit(moma_batch* b, uint64_t polls) {
  if (!b || polls == 0) return MOMA_ERR_INVALID_ARG;
  b->wait_polls = polls;
  if (b->graph) {  // the limit is a launch argument: capture again on the next run
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return MOMA_OK;
}

extern "C" moma_status moma_batch_inject_missing_dependency(moma_batch* b) {
  if (!b || b->segs.empty()) return MOMA_ERR_INVALID_ARG;
  Seg& last = b->segs.back();
  last.wait_id[1] = last.done_id;  // waits for more of its own tiles than will ever finish
  last.wait_count[1] = 0xffffffffu;
  b->dirty = true;
  return MOMA_OK;
}

extern "C" void moma_batch_destroy(moma_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->ready) cudaEventDestroy(b->ready);
  cudaStream_t ss = setup_stream(b->device);
  for (void* p : {(void*)b->d_block, (void*)b->d_scratch})
    if (p) cudaFreeAsync(p, ss);
  delete b;
}

extern "C" moma_status moma_batch_submit(const moma_job* jobs, int njobs, void* stream) {
  moma_batch* b = nullptr;
  moma_status rc = moma_batch_create(jobs, njobs, &b);
  if (rc) return rc;
  rc = wait_ready(b, (cudaStream_t)stream);
  if (!rc) rc = batch_launch(b, (cudaStream_t)stream);
  if (!rc && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) rc = MOMA_ERR_CUDA;
  if (!rc) rc = moma_batch_sync_status(b);
  moma_batch_destroy(b);
  return rc;
}
