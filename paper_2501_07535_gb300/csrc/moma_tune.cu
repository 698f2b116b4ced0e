// moma_tune.cu -- per-context kernel schedules and the autotuner.
//
// A schedule (moma_config) picks the word-product form of the multi-word multiplication
// (carry chains or whole mad.wide products), the shared-memory tile of the transform and
// the largest radix of one Stockham pass, and the vector width of the BLAS kernels.  Every
// schedule computes bit-identical results; only speed differs.  The autotuner times each
// candidate with CUDA events on the caller's stream and keeps the fastest.
#include <set>
#include <tuple>
#include <vector>

#include "moma_internal.hpp"

using namespace moma;

static bool is_ntt_op(int op) { return op == MOMA_OP_NTT_FWD || op == MOMA_OP_NTT_INV || op == MOMA_OP_POLYMUL; }
static bool is_vec_op(int op) { return op >= MOMA_OP_ADD && op <= MOMA_OP_AXPY; }

static int log2_of(size_t n) {
  if (n == 0 || (n & (n - 1))) return -1;
  int k = 0;
  while (((size_t)1 << k) < n) ++k;
  return k;
}

extern "C" moma_status moma_ctx_set_config(moma_ctx* ctx, int op, size_t n, const moma_config* cfg) {
  if (!ctx || !cfg) return MOMA_ERR_INVALID_ARG;
  if (is_ntt_op(op)) {
    const int lg = log2_of(n);
    if (lg < 1 || lg > kMaxLogN) return MOMA_ERR_SIZE;
    if (!ntt_config_valid(ctx->L, lg, *cfg)) return MOMA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->lock);
    ctx->configs[std::make_pair(op, lg)] = *cfg;
    return MOMA_OK;
  }
  if (is_vec_op(op)) {
    if (cfg->engine < 0 || cfg->engine > 4) return MOMA_ERR_INVALID_ARG;
    if (cfg->engine == 4 && !(ctx->mont && op == MOMA_OP_MUL)) return MOMA_ERR_INVALID_ARG;
    if (cfg->vec_width != 0 && cfg->vec_width != 1 && cfg->vec_width != 2 && cfg->vec_width != 4)
      return MOMA_ERR_INVALID_ARG;
    if (cfg->tile_log != 0 && cfg->tile_log != vec_max_log_tile(ctx->L)) return MOMA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(ctx->lock);
    ctx->configs[std::make_pair(op, -1)] = *cfg;
    return MOMA_OK;
  }
  return MOMA_ERR_INVALID_ARG;
}

extern "C" moma_status moma_ctx_get_config(moma_ctx* ctx, int op, size_t n, moma_config* cfg) {
  if (!ctx || !cfg) return MOMA_ERR_INVALID_ARG;
  if (is_ntt_op(op)) {
    const int lg = log2_of(n);
    if (lg < 1 || lg > kMaxLogN) return MOMA_ERR_SIZE;
    *cfg = ntt_config(ctx, op, lg, 1);  // a single transform's; takes the context's lock for the lookup
    return MOMA_OK;
  }
  if (is_vec_op(op)) {
    *cfg = vec_config(ctx, op - MOMA_OP_ADD);
    return MOMA_OK;
  }
  return MOMA_ERR_INVALID_ARG;
}

namespace {

struct Scratch {
  std::vector<uint32_t*> bufs;
  ~Scratch() {
    for (auto* p : bufs) cudaFree(p);
  }
  uint32_t* get(size_t words, cudaStream_t st) {
    uint32_t* p = nullptr;
    if (cudaMalloc(&p, words * 4) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    // 0x01010101 in every limb: canonical for every supported modulus (top limb < q's)
    cudaMemsetAsync(p, 0x01, words * 4, st);
    return p;
  }
};

}  // namespace

extern "C" moma_status moma_autotune(moma_ctx* ctx, int op, size_t n, size_t count, void* stream, moma_config* best,
                                     double* best_us) {
  if (!ctx) return MOMA_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<moma_config> cands;
  int lg = -1;
  if (is_ntt_op(op)) {
    lg = log2_of(n);
    if (lg < 1 || lg > kMaxLogN) return MOMA_ERR_SIZE;
    if (count == 0) count = 1;
    if (op == MOMA_OP_POLYMUL) count = 1;
    // CTA size and tile go together: 2^1..2^4 elements per thread (2^1 and 2^2 for calls with
    // little work, where more CTAs and fewer butterflies per thread pay); radices leave 8 to 32
    // groups per tile.
    for (int engine = 1; engine <= 2; ++engine)
      for (int th = 32, lth = 5; th <= 256; th *= 2, ++lth)
        for (int t = -2; t <= 1; ++t) {
          const int tl = lth + 3 + t;
          if (tl > max_tile_log(ctx->L)) continue;
          if (lg <= tl) {
            cands.push_back({engine, tl, tl, 0, th, 0});
            if (th <= 128) cands.push_back({engine, tl, tl, 0, th, 1});
            continue;
          }
          for (int r = tl - 3; r >= tl - 5; --r)
            if (r >= 1) {
              cands.push_back({engine, tl, r, 0, th, 0});
              if (th <= 128) cands.push_back({engine, tl, r, 0, th, 1});
            }
        }
  } else if (is_vec_op(op)) {
    if (n == 0) return MOMA_ERR_SIZE;
    // full-width contexts: one element per thread, and mulmod's engine 4 (two Montgomery products)
    const int engines = op == MOMA_OP_MUL ? (ctx->mont ? 4 : 3) : (op == MOMA_OP_AXPY && !ctx->mont ? 2 : 1);
    const int vmax = ctx->mont ? 1 : vec_max_width(ctx->L);
    const int tmax = ctx->mont ? 0 : vec_max_log_tile(ctx->L);
    for (int engine = 1; engine <= engines; ++engine) {
      for (int v = 1; v <= vmax; v *= 2) cands.push_back({engine, 0, 0, v, 0, 0});
      // staged by bulk copies in the width's tile (the vector width does not apply)
      if (tmax) cands.push_back({engine, tmax, 0, 1, 0, 0});
    }
  } else {
    return MOMA_ERR_INVALID_ARG;
  }

  Scratch sc;
  const size_t words = (size_t)ctx->L * n * (count ? count : 1);
  uint32_t* a = sc.get(words, st);
  uint32_t* b = sc.get(words, st);
  uint32_t* c = sc.get(words, st);
  if (!a || !b || !c) return MOMA_ERR_OOM;
  std::vector<uint32_t> alpha(ctx->L, 0x01010101u);

  auto run = [&](const moma_config& cfg) -> moma_status {
    switch (op) {
      case MOMA_OP_NTT_FWD: return launch_ntt_cfg(ctx, lg, count, false, a, c, cfg, st);
      case MOMA_OP_NTT_INV: return launch_ntt_cfg(ctx, lg, count, true, a, c, cfg, st);
      case MOMA_OP_POLYMUL: return launch_polymul_cfg(ctx, lg, a, b, c, cfg, st);
      default: return launch_vec_cfg(ctx, op - MOMA_OP_ADD, n, a, b, c, alpha.data(), cfg, st);
    }
  };

  // plans that exist before tuning stay; those built only for losing candidates are freed after
  std::set<std::tuple<int, int, int, int, int>> plans_before;
  if (lg >= 0) {
    std::lock_guard<std::mutex> g(ctx->lock);
    for (const auto& kv : ctx->plans) plans_before.insert(kv.first);
  }

  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MOMA_ERR_CUDA;
  double best_t = 1e30;
  moma_config best_c = cands.empty() ? moma_config{0, 0, 0, 0, 0, 0} : cands[0];
  moma_status rc = MOMA_OK;
  for (const auto& cfg : cands) {
    rc = run(cfg);  // first use builds the plan (twiddle tables) outside the timing
    if (rc) break;
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = MOMA_ERR_CUDA; break; }
    double t_cfg = 1e30;
    for (int round = 0; round < 2 && rc == MOMA_OK; ++round) {
      const int reps = 3;
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && rc == MOMA_OK; ++r) rc = run(cfg);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = MOMA_ERR_CUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t_cfg = std::min(t_cfg, 1e3 * ms / reps);
    }
    if (rc) break;
    if (t_cfg < best_t) {
      best_t = t_cfg;
      best_c = cfg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (lg >= 0 && cudaStreamSynchronize(st) == cudaSuccess) {
    // every candidate's transforms have finished: free the twiddle tables built only for candidates
    // that lost (at 2^24 points and 384 bits each plan holds about 1.6 GB)
    const int keep_t = best_c.tile_log, keep_r = lg <= best_c.tile_log ? 0 : best_c.max_logr;
    std::lock_guard<std::mutex> g(ctx->lock);
    for (auto it = ctx->plans.begin(); it != ctx->plans.end();) {
      const auto& key = it->first;
      const bool kept = plans_before.count(key) || std::get<0>(key) != lg ||
                        (rc == MOMA_OK && std::get<2>(key) == keep_t && std::get<3>(key) == keep_r);
      if (kept) {
        ++it;
      } else {
        free_plan(it->second);
        it = ctx->plans.erase(it);
      }
    }
  }
  if (rc) return rc;
  rc = moma_ctx_set_config(ctx, op, n, &best_c);
  if (rc) return rc;
  if (best)  // the effective schedule, defaults filled in (as moma_ctx_get_config reports it)
    *best = lg >= 0 ? ntt_config(ctx, op, lg, 1) : vec_config(ctx, op - MOMA_OP_ADD);
  if (best_us) *best_us = best_t;
  return MOMA_OK;
}
