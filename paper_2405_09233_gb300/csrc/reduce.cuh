// Deterministic block reductions shared by the kernels of libtstar.
#pragma once
#include <cuda_runtime.h>
#include "internal.cuh"

namespace ts {

// Sum over the block in a fixed tree (warp shuffles, then the first warp).  Every thread gets
// the result.  blockDim.x must be a multiple of 32 and <= 1024.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red_smem[32];
  __shared__ double red_out;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // protect red_smem against a previous use
  if (lane == 0) red_smem[warp] = v;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    double w = lane < nw ? red_smem[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (lane == 0) red_out = w;
  }
  __syncthreads();
  return red_out;
}

// Final sum of kRedBlocks partial sums, identical in every block that calls it.
__device__ __forceinline__ double finalize_partials(const double* __restrict__ P) {
  double v = 0.0;
  for (int b = threadIdx.x; b < kRedBlocks; b += blockDim.x) v += P[b];
  return block_sum(v);
}

}  // namespace ts
