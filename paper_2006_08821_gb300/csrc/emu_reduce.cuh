// Block-level FP64 reduction used by the per-tet kernels.
#pragma once
#include <cuda_runtime.h>

namespace emu {

// Sums v[0..NV) over the block (<= 256 threads) in a fixed order and writes
// the NV totals to out[0..NV). Deterministic for a fixed launch shape.
template <int NV>
__device__ __forceinline__ void block_reduce_write(double (&v)[NV], double* out) {
  __shared__ double sm[8 * NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sm[warp * NV + k] = x;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double x = 0.0;
    for (int w = 0; w < nw; ++w) x += sm[w * NV + k];
    out[k] = x;
  }
}

// Sum of partials[b * NV + k] over b < nblk for k < NV, by a whole block of
// 256 threads: each thread takes a strided subset of the blocks, then a fixed
// tree; every k total lands in out[k] (shared or global). Deterministic.
template <int NV>
__device__ __forceinline__ void block_sum_partials(const double* __restrict__ partials, int nblk, double* out) {
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  // eight strides of loads in flight at once, added in a fixed order
  constexpr int U = 8;
  const int step = blockDim.x;
  int b = threadIdx.x;
  for (; b + (U - 1) * step < nblk; b += U * step) {
    double t[U][NV];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < NV; ++k) t[u][k] = __ldcg(partials + (size_t)(b + u * step) * NV + k);
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < NV; ++k) v[k] += t[u][k];
  }
  for (; b < nblk; b += step) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += __ldcg(partials + (size_t)b * NV + k);
  }
  block_reduce_write<NV>(v, out);
  __syncthreads();
}

// True in the block that finishes last among the grid's blocks (the pattern
// of a threadfence reduction): each block makes its partial sums visible,
// then takes a ticket; the block with the last ticket may read every
// block's partials. The caller resets *ticket to 0 from that block.
__device__ __forceinline__ bool last_block(unsigned* ticket) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

}  // namespace emu
