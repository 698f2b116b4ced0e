// moma_noalloc.cu -- forward NTT that allocates no device memory.
//
// The ordinary transform asks the CUDA stream-ordered allocator for its ping-pong
// buffers on every call.  Some callers cannot let a library allocate: a process whose
// device memory is owned by another allocator under a fixed budget (a framework's caching
// allocator, a server that reserved its memory up front), or a hot path that must not pick
// up allocator latency or synchronisation.  moma_ntt_fwd_noalloc runs the same kernels
// with its scratch in the fixed array below instead.
#include <mutex>

#include "moma_internal.hpp"

namespace moma {

// Two ping-pong buffers of kNoAllocWords 32-bit words each (8 MiB in total).  Every GPU
// that loads this library holds the array until the process exits.
constexpr size_t kNoAllocWords = (size_t)1 << 20;
static __device__ __align__(256) uint32_t g_noalloc_scratch[2 * kNoAllocWords];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_lock;
uint32_t* g_noalloc_addr[kMaxDevices] = {};
}  // namespace

// Device address of the array on device `dev`, which must be current (host code only sees a
// stand-in symbol).  Looked up once per device, when the first context on that device is
// created: with lazy module loading the driver loads this file's module, and places the array,
// at that first look-up, so it happens in a call that is allowed to allocate.
moma_status noalloc_prepare(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return MOMA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(g_noalloc_lock);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MOMA_ERR_CUDA;
    g_noalloc_addr[dev] = static_cast<uint32_t*>(p);
  }
  return MOMA_OK;
}

static uint32_t* noalloc_scratch(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> g(g_noalloc_lock);
  return g_noalloc_addr[dev];
}

}  // namespace moma

using namespace moma;

extern "C" moma_status moma_ntt_fwd_noalloc(moma_ctx* ctx, size_t n, const uint32_t* in, uint32_t* out,
                                            void* stream) {
  if (!ctx || !in || !out) return MOMA_ERR_INVALID_ARG;
  if (((uintptr_t)in & 3u) || ((uintptr_t)out & 3u)) return MOMA_ERR_ALIGN;
  if (n == 0 || (n & (n - 1))) return MOMA_ERR_SIZE;
  int lg = 0;
  while (((size_t)1 << lg) < n) ++lg;
  if (lg < 1 || lg > kMaxLogN) return MOMA_ERR_SIZE;
  if (ctx->L > 12) return MOMA_ERR_UNSUPPORTED;
  if ((size_t)ctx->L * n > kNoAllocWords) return MOMA_ERR_SIZE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return MOMA_ERR_CUDA;
  if (dev != ctx->device) return MOMA_ERR_INVALID_ARG;
  const moma_config cfg = ntt_config(ctx, MOMA_OP_NTT_FWD, lg, 1);  // the schedule moma_ntt_fwd uses
  Plan* pl = find_plan(ctx, lg, false, cfg.tile_log, cfg.max_logr);
  if (!pl) return MOMA_ERR_INVALID_ARG;  // twiddle tables not built yet: call moma_ntt_fwd once
  uint32_t* scratch = noalloc_scratch(dev);  // resolved when the context was created
  if (!scratch) return MOMA_ERR_CUDA;
  return run_plan_buffers(ctx, pl, 1, in, nullptr, out, cfg, scratch, scratch + kNoAllocWords, (cudaStream_t)stream);
}
