// ACAP coupling solve of Eq. 4 on the device: q* = (G^T W G)^-1 G^T W F.
//
// With full-vertex pins the 3n x 3n matrix is L (x) I_3, so the three
// coordinates are three right-hand sides of one scalar Laplacian L. The
// solve is a Jacobi-preconditioned conjugate gradient in FP64, written as one
// persistent cooperative kernel. It uses the Chronopoulos-Gear form of CG:
// each iteration does one SpMV and one fused reduction, so it needs two
// grid-wide barriers. Every block reduces the per-block partial sums itself,
// in a fixed order, so all blocks take identical branch decisions and the
// result is deterministic. The paper prefactors this matrix with Pardiso
// (Sec. 3.3); on the GPU an iterative solve with warm starts replaces the
// sparse back-substitution.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "emu_internal.h"
#include "emu_pcg.h"

namespace emu {

// Bounded grid barrier. ``count`` grows by gridDim.x per barrier (reset by the
// host before each launch); the last block to arrive publishes the epoch.
// A block that spins longer than kSpinLimit polls sets ``err`` and leaves;
// the others see ``err`` and leave too, so no wait is unbounded.
static constexpr unsigned long long kSpinLimit = 1ull << 25;  // ~ seconds with nanosleep

__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned& epoch, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1u;
    __threadfence();
    unsigned prev = atomicAdd(&bar->count, 1u);
    if (prev + 1u == gridDim.x * epoch) {
      __threadfence();
      atomicExch(&bar->gen, epoch);
    } else {
      unsigned long long spins = 0;
      while (true) {
        unsigned g = *((volatile unsigned*)&bar->gen);
        if (g >= epoch) break;
        if (*((volatile int*)&bar->err)) break;
        if (++spins > kSpinLimit) {
          atomicExch(&bar->err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    *s_flag = *((volatile int*)&bar->err);
  }
  __syncthreads();
  return *s_flag == 0;
}

template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* out, double* sm) {
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
  __syncthreads();
}

// Every block sums the per-block partials with the same fixed tree, so all
// blocks hold bit-identical scalars. Loads bypass L1 (__ldcg): the partials
// were written by other SMs.
template <int NV>
__device__ __forceinline__ void sum_partials(const double* partials, double* s_out, double* sm) {
  // thread t sums blocks t, t + blockDim, ... for every value, then a
  // shared-memory tree over the 256 threads
  double loc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) loc[k] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < NV; ++k) loc[k] += __ldcg(partials + (size_t)b * NV + k);
  }
  block_partials<NV>(loc, s_out, sm);
}

template <int NR>
__device__ __forceinline__ void spmv_row(const Laplacian& L, const double* __restrict__ x, int64_t v, double* acc) {
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = 0.0;
  const int32_t e0 = L.rowptr[v], e1 = L.rowptr[v + 1];
  for (int32_t e = e0; e < e1; ++e) {
    const int64_t c = L.col[e];
    const double a = L.val[e];
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[j] += a * __ldcg(x + c * NR + j);
  }
}

template <int NR>
__global__ void __launch_bounds__(256) pcg_kernel(PcgArgs a) {
  constexpr int NV0 = 4 * NR;  // gamma, delta, rr, bb
  constexpr int NV = 3 * NR;   // gamma, delta, rr
  __shared__ double sm[8 * NV0];
  __shared__ double sc[NV0];
  __shared__ int s_flag;
  __shared__ double s_alpha[NR], s_beta[NR], s_gamma[NR], s_thr[NR];
  __shared__ int s_active[NR];
  unsigned epoch = 0;
  const Laplacian L = a.L;
  const int64_t n = L.n;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = r0 + per < n ? r0 + per : n;
  const double* __restrict__ b = a.b;
  double* __restrict__ x = a.x;
  double* __restrict__ r = a.r;
  double* __restrict__ u = a.u;
  double* __restrict__ w = a.w;
  double* __restrict__ p = a.p;
  double* __restrict__ s = a.s;

  // r = b - A x ; u = D^-1 r
  for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
    double acc[NR];
    spmv_row<NR>(L, x, v, acc);
    const double di = L.dinv[v];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const double rv = b[v * NR + j] - acc[j];
      r[v * NR + j] = rv;
      u[v * NR + j] = di * rv;
    }
  }
  if (!grid_sync(a.bar, epoch, &s_flag)) goto timeout;
  {
    double loc[NV0];
#pragma unroll
    for (int k = 0; k < NV0; ++k) loc[k] = 0.0;
    for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
      double acc[NR];
      spmv_row<NR>(L, u, v, acc);
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const double rv = r[v * NR + j], uv = u[v * NR + j], bv = b[v * NR + j];
        w[v * NR + j] = acc[j];
        loc[j] += rv * uv;
        loc[NR + j] += acc[j] * uv;
        loc[2 * NR + j] += rv * rv;
        loc[3 * NR + j] += bv * bv;
      }
    }
    block_partials<NV0>(loc, a.partials + (size_t)blockIdx.x * NV0, sm);
  }
  if (!grid_sync(a.bar, epoch, &s_flag)) goto timeout;
  sum_partials<NV0>(a.partials, sc, sm);
  if (threadIdx.x == 0) {
    for (int j = 0; j < NR; ++j) {
      const double bb = sc[3 * NR + j];
      s_thr[j] = a.tol * a.tol * bb;
      s_gamma[j] = sc[j];
      const bool done = (sc[2 * NR + j] <= s_thr[j]) || !(sc[NR + j] > 0.0);
      s_active[j] = done ? 0 : 1;
      s_alpha[j] = done ? 0.0 : sc[j] / sc[NR + j];
      s_beta[j] = 0.0;
    }
  }
  __syncthreads();
  for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      p[v * NR + j] = u[v * NR + j];
      s[v * NR + j] = w[v * NR + j];
      if (sc[3 * NR + j] == 0.0) x[v * NR + j] = 0.0;  // zero right-hand side: x = 0 exactly
    }
  }
  {
    int it = 0;
    bool all_done = true;
    for (int j = 0; j < NR; ++j) all_done = all_done && (s_active[j] == 0);
    while (!all_done && it < a.max_iter) {
      ++it;
      for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
        const double di = L.dinv[v];
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (!s_active[j]) continue;
          const double al = s_alpha[j];
          x[v * NR + j] += al * p[v * NR + j];
          const double rv = r[v * NR + j] - al * s[v * NR + j];
          r[v * NR + j] = rv;
          u[v * NR + j] = di * rv;
        }
      }
      if (!grid_sync(a.bar, epoch, &s_flag)) goto timeout;
      {
        double loc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) loc[k] = 0.0;
        for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
          double acc[NR];
          spmv_row<NR>(L, u, v, acc);
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            const double rv = r[v * NR + j], uv = u[v * NR + j];
            w[v * NR + j] = acc[j];
            loc[j] += rv * uv;
            loc[NR + j] += acc[j] * uv;
            loc[2 * NR + j] += rv * rv;
          }
        }
        block_partials<NV>(loc, a.partials + (size_t)blockIdx.x * NV, sm);
      }
      if (!grid_sync(a.bar, epoch, &s_flag)) goto timeout;
      sum_partials<NV>(a.partials, sc, sm);
      if (threadIdx.x == 0) {
        for (int j = 0; j < NR; ++j) {
          if (!s_active[j]) continue;
          const double g_new = sc[j], dl = sc[NR + j], rr = sc[2 * NR + j];
          if (rr <= s_thr[j]) {
            s_active[j] = 0;
            continue;
          }
          const double be = g_new / s_gamma[j];
          const double den = dl - be * g_new / s_alpha[j];
          if (!(den > 0.0)) {  // breakdown: stop this column
            s_active[j] = 0;
            continue;
          }
          s_beta[j] = be;
          s_alpha[j] = g_new / den;
          s_gamma[j] = g_new;
        }
      }
      __syncthreads();
      all_done = true;
      for (int j = 0; j < NR; ++j) all_done = all_done && (s_active[j] == 0);
      if (all_done) break;
      for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (!s_active[j]) continue;
          const double be = s_beta[j];
          p[v * NR + j] = u[v * NR + j] + be * p[v * NR + j];
          s[v * NR + j] = w[v * NR + j] + be * s[v * NR + j];
        }
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (a.iters_out) atomicAdd(a.iters_out, it);
      if (a.fail_out && !all_done) atomicExch(a.fail_out, 1);
      if (a.last_iters) *a.last_iters = it;
    }
  }
  return;
timeout:
  if (threadIdx.x == 0 && a.timeout_out) atomicExch(a.timeout_out, 1);
}

template <int NR> static cudaError_t launch_pcg_impl(const PcgArgs& args, int grid, cudaStream_t st) {
  PcgArgs a = args;
  void* params[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)pcg_kernel<NR>, dim3(grid), dim3(256), params, 0, st);
}

int pcg_max_grid(int nrhs, int64_t n) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (nrhs == 3)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg_kernel<3>, 256, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg_kernel<16>, 256, 0);
  if (occ < 1) occ = 1;
  // One block per SM at most: the barrier and the partial sums cost grow with
  // the block count, and 256 threads per SM already cover ~500 rows each.
  int64_t want = (n + 511) / 512;
  int64_t cap = (int64_t)sms;
  int64_t g = want < cap ? want : cap;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_pcg(int nrhs, const PcgArgs& args, int grid, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(args.bar, 0, sizeof(GridBarrier), st);
  if (e != cudaSuccess) return e;
  if (nrhs == 3) return launch_pcg_impl<3>(args, grid, st);
  if (nrhs == 16) return launch_pcg_impl<16>(args, grid, st);
  return cudaErrorInvalidValue;
}

}  // namespace emu
