// moma_probe.cu -- integer multiply-add issue-rate microbenchmark.
//
// The compute roofline of every kernel here is its count of 32-bit word multiplies at
// the chip's integer multiply-add rate.  This kernel measures that rate for each PTX
// instruction form the arithmetic can use.
#include "moma_internal.hpp"
#include "moma_limbs.cuh"

namespace moma {

// Every variant issues 64 multiply instructions per thread per loop iteration on eight
// independent accumulators (except variant 1, one dependent chain):
//   0  rows of mad.lo.cc/madc.lo.cc and mad.hi.cc/madc.hi.cc carry chains (the arithmetic's mix)
//   1  the same rows as one dependent chain (latency bound)
//   2  mad.lo and mad.hi without carries, alternating
//   3  mad.lo only            4  mad.hi only
//   5  mad.wide.u32 (32x32 -> 64-bit product plus 64-bit addend: a whole word product)
//   6  mad.lo.cc/madc.lo.cc rows only      7  mad.hi.cc/madc.hi.cc rows only
//   8  add.cc/addc.cc chains (no multiply; the carry-propagation cost)
//   9  rows written as plain 64-bit C arithmetic: t = x*y[j] + acc[j] + (t >> 32)
template <int VARIANT>
__global__ void __launch_bounds__(256) probe_imad_kernel(uint32_t* sink, int iters, uint32_t seed) {
  uint32_t acc[8][4];
  uint32_t y[4];
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int c = 0; c < 8; ++c)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[c][k] = seed * (t + 1) + 0x9e3779b9u * (uint32_t)(c * 4 + k + 1);
#pragma unroll
  for (int k = 0; k < 4; ++k) y[k] = seed ^ (0x85ebca6bu * (uint32_t)(k + 3));
  uint64_t w[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) w[c] = ((uint64_t)acc[c][1] << 32) | acc[c][0];
  for (int it = 0; it < iters; ++it) {
    if constexpr (VARIANT == 0) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint32_t x = acc[c][3] | 1u;
        row_lo<4, false>(acc[c], x, y);
        row_hi<4, false>(acc[c], x, y);
      }
    } else if constexpr (VARIANT == 1) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint32_t x = acc[0][3] | 1u;
        row_lo<4, false>(acc[0], x, y);
        row_hi<4, false>(acc[0], x, y);
      }
    } else if constexpr (VARIANT == 6 || VARIANT == 7) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint32_t x = acc[c][3] | 1u;
        if constexpr (VARIANT == 6) {
          row_lo<4, false>(acc[c], x, y);
          row_lo<4, false>(acc[c], x ^ 0x5bd1e995u, y);
        } else {
          row_hi<4, false>(acc[c], x, y);
          row_hi<4, false>(acc[c], x ^ 0x5bd1e995u, y);
        }
      }
    } else if constexpr (VARIANT == 8) {
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 8; c += 2) {
          add_words<4, false>(acc[c], acc[c], acc[c + 1]);
          add_words<4, false>(acc[c + 1], acc[c + 1], acc[c]);
          add_words<4, false>(acc[c], acc[c], y);
          add_words<4, false>(acc[c + 1], acc[c + 1], y);
        }
    } else if constexpr (VARIANT == 9) {
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const uint32_t x = acc[c][3] | 1u;
          uint64_t t = 0;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            t = (uint64_t)x * y[k] + acc[c][k] + (t >> 32);
            acc[c][k] = (uint32_t)t;
          }
          acc[c][0] ^= (uint32_t)(t >> 32);
        }
    } else if constexpr (VARIANT == 5) {
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          uint64_t d;
          asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"((uint32_t)w[c]), "r"(y[r & 3]), "l"(w[c]));
          w[c] = d;
        }
    } else {
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            uint32_t v;
            if (VARIANT == 3 || (VARIANT == 2 && (k & 1) == 0))
              asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(v) : "r"(acc[c][k]), "r"(y[k]), "r"(acc[c][(k + 1) & 3]));
            else
              asm volatile("mad.hi.u32 %0, %1, %2, %3;" : "=r"(v) : "r"(acc[c][k]), "r"(y[k]), "r"(acc[c][(k + 1) & 3]));
            acc[c][k] = v;
          }
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    s ^= (uint32_t)w[c] ^ (uint32_t)(w[c] >> 32);
#pragma unroll
    for (int k = 0; k < 4; ++k) s ^= acc[c][k];
  }
  sink[t] = s;
}

}  // namespace moma

using namespace moma;

extern "C" moma_status moma_probe_imad(int variant, int blocks, int threads, int iters, double* ms_out,
                                       double* imad_out) {
  if (blocks <= 0 || threads <= 0 || threads > 256 || iters <= 0 || variant < 0 || variant > 9)
    return MOMA_ERR_INVALID_ARG;
  uint32_t* sink = nullptr;
  if (cudaMalloc(&sink, (size_t)blocks * threads * sizeof(uint32_t)) != cudaSuccess) return MOMA_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](int it) {
    switch (variant) {
      case 0: probe_imad_kernel<0><<<blocks, threads>>>(sink, it, 12345u); break;
      case 1: probe_imad_kernel<1><<<blocks, threads>>>(sink, it, 12345u); break;
      case 2: probe_imad_kernel<2><<<blocks, threads>>>(sink, it, 12345u); break;
      case 3: probe_imad_kernel<3><<<blocks, threads>>>(sink, it, 12345u); break;
      case 4: probe_imad_kernel<4><<<blocks, threads>>>(sink, it, 12345u); break;
      case 5: probe_imad_kernel<5><<<blocks, threads>>>(sink, it, 12345u); break;
      case 6: probe_imad_kernel<6><<<blocks, threads>>>(sink, it, 12345u); break;
      case 7: probe_imad_kernel<7><<<blocks, threads>>>(sink, it, 12345u); break;
      case 8: probe_imad_kernel<8><<<blocks, threads>>>(sink, it, 12345u); break;
      default: probe_imad_kernel<9><<<blocks, threads>>>(sink, it, 12345u); break;
    }
  };
  launch(iters / 8 + 1);  // warm-up
  cudaEventRecord(e0);
  launch(iters);
  cudaEventRecord(e1);
  moma_status st = cuda_status(cudaEventSynchronize(e1));
  float ms = 0.f;
  if (st == MOMA_OK) st = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
  if (ms_out) *ms_out = ms;
  if (imad_out) *imad_out = 64.0 * (double)iters * (double)blocks * (double)threads;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return st;
}
