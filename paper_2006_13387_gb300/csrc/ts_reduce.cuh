// Deterministic block reductions (fixed shuffle tree + fixed smem order).
#pragma once
#include <cuda_runtime.h>

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over a block of NT threads; result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red_s[NT / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red_s[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = (lane < NT / 32) ? red_s[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

// N sums over a block of NT threads at once: the values are staged in shared
// memory and one warp adds them (a fixed order), so the FP64 additions are
// those of one warp instead of every warp's shuffle tree.  Results valid in
// lane 0 of warp 0 (v[] of thread 0).
template <int NT, int N>
__device__ __forceinline__ void block_sum_n(double (&v)[N]) {
  __shared__ double sh_n[N][NT];
#pragma unroll
  for (int j = 0; j < N; ++j) sh_n[j][threadIdx.x] = v[j];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < NT / 32; ++k) s += sh_n[j][threadIdx.x + 32 * k];
      v[j] = warp_sum(s);
    }
  }
  __syncthreads();
}

// The same sum, valid in every thread of the block.
template <int NT>
__device__ __forceinline__ double block_sum_all(double v) {
  __shared__ double tot_s;
  v = block_sum<NT>(v);
  if (threadIdx.x == 0) tot_s = v;
  __syncthreads();
  v = tot_s;
  __syncthreads();
  return v;
}

// Dynamic-size variant (blockDim.x multiple of 32, <= 1024); result in thread 0.
__device__ __forceinline__ double block_sum_dyn(double v, double* scratch32) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) scratch32[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = (lane < nw) ? scratch32[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}
