// moma_probe.cu -- integer multiply-add issue-rate microbenchmark.
//
// The compute roofline of every kernel here is its count of 32-bit word multiplies at
// the chip's integer multiply-add rate.  This kernel measures that rate with the same
// instruction forms the arithmetic uses: rows of mad.lo.cc / madc.lo.cc and
// mad.hi.cc / madc.hi.cc carry chains on independent accumulators (variant 0), one
// dependent chain (variant 1, latency-bound), and plain mad.lo without carries
// (variant 2).  Each loop iteration issues 64 multiply-adds per thread.
#include "moma_internal.hpp"
#include "moma_limbs.cuh"

namespace moma {

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
  for (int it = 0; it < iters; ++it) {
    if constexpr (VARIANT == 0) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {  // 8 independent chains of 8
        const uint32_t x = acc[c][3] | 1u;
        row_lo<4, false>(acc[c], x, y);
        row_hi<4, false>(acc[c], x, y);
      }
    } else if constexpr (VARIANT == 1) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {  // one chain, each row depending on the previous
        const uint32_t x = acc[0][3] | 1u;
        row_lo<4, false>(acc[0], x, y);
        row_hi<4, false>(acc[0], x, y);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          uint32_t r;
          asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(acc[c][k]), "r"(y[k]), "r"(acc[c][(k + 1) & 3]));
          acc[c][k] = r;
          asm volatile("mad.hi.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(acc[c][k]), "r"(y[k]), "r"(acc[c][k]));
          acc[c][(k + 2) & 3] ^= r;
        }
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c)
#pragma unroll
    for (int k = 0; k < 4; ++k) s ^= acc[c][k];
  sink[t] = s;
}

}  // namespace moma

using namespace moma;

extern "C" moma_status moma_probe_imad(int variant, int blocks, int threads, int iters, double* ms_out,
                                       double* imad_out) {
  if (blocks <= 0 || threads <= 0 || threads > 256 || iters <= 0 || variant < 0 || variant > 2)
    return MOMA_ERR_INVALID_ARG;
  uint32_t* sink = nullptr;
  if (cudaMalloc(&sink, (size_t)blocks * threads * sizeof(uint32_t)) != cudaSuccess) return MOMA_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](int it) {
    if (variant == 0) probe_imad_kernel<0><<<blocks, threads>>>(sink, it, 12345u);
    else if (variant == 1) probe_imad_kernel<1><<<blocks, threads>>>(sink, it, 12345u);
    else probe_imad_kernel<2><<<blocks, threads>>>(sink, it, 12345u);
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
