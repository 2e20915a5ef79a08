// reduce.cuh -- deterministic block and grid reductions shared by the
// vector kernels.  A grid reduction writes one partial per block; the last
// block to finish (an atomic ticket, no waiting) adds the partials in block
// order, so the result does not depend on the order in which blocks ran.
#pragma once

#include <cuda_runtime.h>

namespace hofv {

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  }
  __syncthreads();
  return s;  // valid in thread 0
}

// Block sum in the precision of the values (FP32 stays on the FP32 pipe);
// the per-warp results are added by warp 0 in double.  Valid in thread 0.
// FP64 warp instructions cost 16 cycles of the SM's FP64 pipe on this GPU,
// so FP64 reductions are kept to one warp wherever possible.
template <typename T>
__device__ __forceinline__ double block_sum_t(T v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;
}

// Sum of partials red[0..nb) by warp 0 of the block (fixed order: lane l adds
// partials l, l+32, ..., then a fixed shuffle tree), accumulated in A.
// Valid in thread 0.
template <typename A = double>
__device__ __forceinline__ double warp0_sum(const double* red, unsigned int nb) {
  A s = (A)0;
  if (threadIdx.x < 32) {
#pragma unroll 8
    for (unsigned int b = threadIdx.x; b < nb; b += 32) s += (A)__ldcg(red + b);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return (double)s;
}

// Returns true in thread 0 of the block that finished last.
__device__ __forceinline__ bool last_block(unsigned int* count, unsigned int nblocks) {
  __shared__ bool is_last;
  __threadfence();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(count, 1u);
    is_last = (t == nblocks - 1);
  }
  __syncthreads();
  return is_last;
}

// Sum of partials red[0..nb) by the whole (last) block: thread t adds
// partials t, t + blockDim, ... in order, then a fixed-shape tree.  The
// result (valid in thread 0) does not depend on which block finished last.
__device__ __forceinline__ double final_sum(const double* red, unsigned int nb, double* sh) {
  double s = 0.0;
  for (unsigned int b = threadIdx.x; b < nb; b += blockDim.x) s += __ldcg(red + b);
  return block_sum(s, sh);
}

}  // namespace hofv
