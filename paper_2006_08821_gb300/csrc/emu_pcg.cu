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
// A block that waits longer than wait_ns (GPU clock) or kWaitSpinCap polls
// sets ``err`` and leaves; the others see ``err`` and leave too, so no wait
// is unbounded. ``arrive`` false leaves without arriving (the self-check of
// launch_wait_check only).
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned& epoch, int* s_flag,
                                          unsigned long long wait_ns, bool arrive = true) {
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1u;
    __threadfence();
    const unsigned prev = arrive ? atomicAdd(&bar->count, 1u) : 0u;
    if (arrive && prev + 1u == gridDim.x * epoch) {
      __threadfence();
      atomicExch(&bar->gen, epoch);
    } else {
      const unsigned long long t0 = global_ns();
      unsigned long long spins = 0;
      while (true) {
        unsigned g = *((volatile unsigned*)&bar->gen);
        if (g >= epoch) break;
        if (*((volatile int*)&bar->err)) break;
        ++spins;
        if (spins > kWaitSpinCap || ((spins & 63u) == 0u && global_ns() - t0 > wait_ns)) {
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

// Values carried per reduction, padded to a power of two (the butterfly below).
__host__ __device__ constexpr int red_pad(int nv) { return nv <= 1 ? 1 : 2 * red_pad((nv + 1) / 2); }

// Block sum of v[0..NV) in a fixed order, written to out[0..NV) (shared or
// global; sm holds 8 * red_pad(NV) doubles). Within a warp a halving
// butterfly: at each of the five steps a lane keeps half of the values it
// carries and adds its partner's copy of that half, so a lane does about
// P adds (P = red_pad(NV)) instead of 5 NV shuffle-adds of a plain tree per
// value. That matters in FP64, whose warp instructions occupy GB300's FP64
// pipe for many cycles each. Lane l ends with the sums of indices
// l * (P / 32) .. when P >= 32, else of index l / (32 / P). Warps from
// ``nw_data`` on hold only zeros (their threads own no rows) and are left
// out of the sum.
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* out, double* sm, int nw_data = 32) {
  constexpr int P = red_pad(NV);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = min(nw_data, (int)(blockDim.x >> 5));
  if (warp < nw) {
  double x[P];
#pragma unroll
  for (int k = 0; k < P; ++k) x[k] = k < NV ? v[k] : 0.0;
  int base = 0;  // index of x[0] after the halving steps
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    const int o = 16 >> t;
    constexpr int P0 = P;
    const int h = (P0 >> t) / 2;  // values kept at this step (0: one value left)
    if (h >= 1) {
      const bool hi = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < P0 / 2; ++i) {
        if (i < h) {
          const double keep = hi ? x[h + i] : x[i];
          const double send = hi ? x[i] : x[h + i];
          x[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      if (hi) base += h;
    } else {
      x[0] += __shfl_xor_sync(0xffffffffu, x[0], o);
    }
  }
  constexpr int C = P >= 32 ? P / 32 : 1;
  if (P >= 32 || (lane % (32 / P)) == 0) {
#pragma unroll
    for (int i = 0; i < C; ++i) sm[warp * P + base + i] = x[i];
  }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sm[w * P + k];
    out[k] = t;
  }
  __syncthreads();
}

// Every block sums the per-block partials in the same fixed order, so all
// blocks hold bit-identical scalars: the block's 256 threads form G groups
// of P = red_pad(NV) (thread g P + k takes value k of the blocks g, g + G,
// ..., eight loads in flight), then thread k adds the G group sums in
// order. Loads bypass L1 (__ldcg): the partials were written by other SMs.
// Needs blockDim.x == 256.
template <int NV>
__device__ __forceinline__ void sum_partials(const double* partials, double* s_out, double*) {
  constexpr int P = red_pad(NV);
  constexpr int G = P <= 256 ? 256 / P : 1;
  __shared__ double sg[256];
  const int g = threadIdx.x / P, k = threadIdx.x % P;
  if (g < G && k < NV) {
    const unsigned nb = gridDim.x;
    double t = 0.0;
    unsigned b = g;
    for (; b + 7 * G < nb; b += 8 * G) {
      double l[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) l[u] = __ldcg(partials + (size_t)(b + u * G) * NV + k);
#pragma unroll
      for (int u = 0; u < 8; ++u) t += l[u];
    }
    for (; b < nb; b += G) t += __ldcg(partials + (size_t)b * NV + k);
    sg[g * P + k] = t;
  }
  __syncthreads();
  for (int kk = threadIdx.x; kk < NV; kk += blockDim.x) {
    double t = 0.0;
    for (int gg = 0; gg < G; ++gg) t += sg[gg * P + kk];
    s_out[kk] = t;
  }
  __syncthreads();
}

template <int NR, typename T>
__device__ __forceinline__ void spmv_row(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                         const T* __restrict__ val, const T* __restrict__ x, int64_t v, T* acc) {
#pragma unroll
  for (int j = 0; j < NR; ++j) acc[j] = T(0);
  const int32_t e0 = rowptr[v], e1 = rowptr[v + 1];
  int32_t e = e0;
  // four entries per step keeps several independent L2 loads in flight
  for (; e + 4 <= e1; e += 4) {
    int64_t c[4];
    T a[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      c[k] = col[e + k];
      a[k] = val[e + k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int j = 0; j < NR; ++j) acc[j] += a[k] * __ldcg(x + c[k] * NR + j);
  }
  for (; e < e1; ++e) {
    const int64_t c = col[e];
    const T a = val[e];
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[j] += a * __ldcg(x + c * NR + j);
  }
}

// Preconditioner M = D^-1 + Phi E^-1 Phi^T (Jacobi plus an additive coarse
// correction on the low-rank basis Phi of Eq. 9, E = Phi^T L Phi), when
// COARSE. Phi^T r and Phi^T s are carried as recurrences
// (rho <- rho - alpha sigma, sigma <- Phi^T w + beta sigma), and Phi^T w is
// summed in the same reduction as the CG dot products, so the coarse term
// adds no grid barrier to the two per iteration.
template <int NR, typename T, bool COARSE>
__global__ void __launch_bounds__(256) pcg_kernel(PcgArgsT<T> a) {
  constexpr int NC = COARSE ? kModes * NR : 0;  // coarse values (mode j, column c) at j * NR + c
  constexpr int NV0 = 4 * NR + NC;              // gamma, delta, rr, bb, Phi^T w
  constexpr int NV = 3 * NR + NC;               // gamma, delta, rr, Phi^T w
  __shared__ double sm[8 * red_pad(NV0)];
  __shared__ double sc[NV0];
  __shared__ int s_flag;
  __shared__ double s_alpha[NR], s_beta[NR], s_gamma[NR], s_thr[NR], s_bb[NR], s_rr[NR];
  __shared__ int s_active[NR];
  __shared__ double s_rho[NC > 0 ? NC : 1], s_sig[NC > 0 ? NC : 1];
  __shared__ T s_cc[NC > 0 ? NC : 1];        // E^-1 rho: coarse coefficients of u
  __shared__ double s_Einv[COARSE ? kModes * kModes : 1];
  unsigned epoch = 0;
  const int64_t n = a.n;
  const int32_t* __restrict__ rowptr = a.rowptr;
  const int32_t* __restrict__ col = a.col;
  const T* __restrict__ val = a.val;
  const T* __restrict__ dinv = a.dinv;
  const T* __restrict__ phi = a.phi;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = r0 + per < n ? r0 + per : n;
  // warps whose threads own rows (the others' partial sums are zero)
  const int nwr = r1 > r0 ? (int)((r1 - r0 + 31) / 32 < 8 ? (r1 - r0 + 31) / 32 : 8) : 0;
  const T* __restrict__ b = a.b;
  T* __restrict__ x = a.x;
  T* __restrict__ r = a.r;
  T* __restrict__ u = a.u;
  T* __restrict__ w = a.w;
  T* __restrict__ p = a.p;
  T* __restrict__ s = a.s;
  if constexpr (COARSE) {
    for (int k = threadIdx.x; k < kModes * kModes; k += blockDim.x) s_Einv[k] = a.Einv[k];
  }

  // u_v = D^-1 r_v + sum_j phi_vj cc_j (coarse term when COARSE)
  auto precond_row = [&](int64_t v) {
    const T di = dinv[v];
    T acc[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[j] = di * r[v * NR + j];
    if constexpr (COARSE) {
#pragma unroll
      for (int k = 0; k < kModes; ++k) {
        const T ph = phi[v * kModes + k];
#pragma unroll
        for (int j = 0; j < NR; ++j) acc[j] += ph * s_cc[k * NR + j];
      }
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) u[v * NR + j] = acc[j];
  };
  auto coarse_coeffs = [&]() {  // s_cc = E^-1 rho (all blocks identically)
    if constexpr (COARSE) {
      for (int e = threadIdx.x; e < NC; e += blockDim.x) {
        const int k = e / NR, j = e % NR;
        double acc = 0.0;
        for (int l = 0; l < kModes; ++l) acc += s_Einv[k * kModes + l] * s_rho[l * NR + j];
        s_cc[e] = (T)acc;
      }
      __syncthreads();
    }
  };

  // r = b - A x
  for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
    T acc[NR];
    spmv_row<NR, T>(rowptr, col, val, x, v, acc);
#pragma unroll
    for (int j = 0; j < NR; ++j) r[v * NR + j] = b[v * NR + j] - acc[j];
  }
  if constexpr (COARSE) {  // rho = Phi^T r
    double loc[NC > 0 ? NC : 1];
#pragma unroll
    for (int k = 0; k < NC; ++k) loc[k] = 0.0;
    for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
#pragma unroll
      for (int k = 0; k < kModes; ++k) {
        const double ph = (double)phi[v * kModes + k];
#pragma unroll
        for (int j = 0; j < NR; ++j) loc[k * NR + j] += ph * (double)r[v * NR + j];
      }
    }
    block_partials<NC>(loc, a.partials + (size_t)blockIdx.x * NV0, sm, nwr);
    if (!grid_sync(a.bar, epoch, &s_flag, a.wait_ns)) goto timeout;
    {
      double tmp[NC > 0 ? NC : 1];
#pragma unroll
      for (int k = 0; k < NC; ++k) tmp[k] = 0.0;
      for (unsigned bb = threadIdx.x; bb < gridDim.x; bb += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NC; ++k) tmp[k] += __ldcg(a.partials + (size_t)bb * NV0 + k);
      }
      block_partials<NC>(tmp, s_rho, sm);
    }
    coarse_coeffs();
    if (!grid_sync(a.bar, epoch, &s_flag, a.wait_ns)) goto timeout;  // partials are rewritten below
  }
  for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) precond_row(v);
  if (!grid_sync(a.bar, epoch, &s_flag, a.wait_ns)) goto timeout;
  {
    double loc[NV0];
#pragma unroll
    for (int k = 0; k < NV0; ++k) loc[k] = 0.0;
    for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
      T acc[NR];
      spmv_row<NR, T>(rowptr, col, val, u, v, acc);
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const double rv = r[v * NR + j], uv = u[v * NR + j], bv = b[v * NR + j];
        w[v * NR + j] = acc[j];
        loc[j] += rv * uv;
        loc[NR + j] += (double)acc[j] * uv;
        loc[2 * NR + j] += rv * rv;
        loc[3 * NR + j] += bv * bv;
      }
      if constexpr (COARSE) {
#pragma unroll
        for (int k = 0; k < kModes; ++k) {
          const double ph = (double)phi[v * kModes + k];
#pragma unroll
          for (int j = 0; j < NR; ++j) loc[4 * NR + k * NR + j] += ph * (double)acc[j];
        }
      }
    }
    block_partials<NV0>(loc, a.partials + (size_t)blockIdx.x * NV0, sm, nwr);
  }
  if (!grid_sync(a.bar, epoch, &s_flag, a.wait_ns)) goto timeout;
  sum_partials<NV0>(a.partials, sc, sm);
  if (threadIdx.x == 0) {
    for (int j = 0; j < NR; ++j) {
      const double bb = sc[3 * NR + j];
      s_bb[j] = bb;
      s_rr[j] = sc[2 * NR + j];
      s_thr[j] = a.tol * a.tol * bb;
      s_gamma[j] = sc[j];
      const bool done = (sc[2 * NR + j] <= s_thr[j]) || !(sc[NR + j] > 0.0);
      s_active[j] = done ? 0 : 1;
      s_alpha[j] = done ? 0.0 : sc[j] / sc[NR + j];
      s_beta[j] = 0.0;
    }
  }
  if constexpr (COARSE) {
    for (int e = threadIdx.x; e < NC; e += blockDim.x) s_sig[e] = sc[4 * NR + e];
  }
  __syncthreads();
  for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      p[v * NR + j] = u[v * NR + j];
      s[v * NR + j] = w[v * NR + j];
      if (s_bb[j] == 0.0) x[v * NR + j] = T(0);  // zero right-hand side: x = 0 exactly
    }
  }
  {
    int it = 0;
    bool all_done = true;
    for (int j = 0; j < NR; ++j) all_done = all_done && (s_active[j] == 0);
    while (!all_done && it < a.max_iter) {
      ++it;
      if constexpr (COARSE) {  // rho <- rho - alpha sigma, then the coarse coefficients
        for (int e = threadIdx.x; e < NC; e += blockDim.x) {
          const int j = e % NR;
          if (s_active[j]) s_rho[e] -= s_alpha[j] * s_sig[e];
        }
        __syncthreads();
        coarse_coeffs();
      }
      for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (!s_active[j]) continue;
          const T al = (T)s_alpha[j];
          x[v * NR + j] += al * p[v * NR + j];
          r[v * NR + j] -= al * s[v * NR + j];
        }
        precond_row(v);
      }
      if (!grid_sync(a.bar, epoch, &s_flag, a.wait_ns)) goto timeout;
      {
        double loc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) loc[k] = 0.0;
        for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
          T acc[NR];
          spmv_row<NR, T>(rowptr, col, val, u, v, acc);
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            const double rv = r[v * NR + j], uv = u[v * NR + j];
            w[v * NR + j] = acc[j];
            loc[j] += rv * uv;
            loc[NR + j] += (double)acc[j] * uv;
            loc[2 * NR + j] += rv * rv;
          }
          if constexpr (COARSE) {
#pragma unroll
            for (int k = 0; k < kModes; ++k) {
              const double ph = (double)phi[v * kModes + k];
#pragma unroll
              for (int j = 0; j < NR; ++j) loc[3 * NR + k * NR + j] += ph * (double)acc[j];
            }
          }
        }
        block_partials<NV>(loc, a.partials + (size_t)blockIdx.x * NV, sm, nwr);
      }
      if (!grid_sync(a.bar, epoch, &s_flag, a.wait_ns)) goto timeout;
      sum_partials<NV>(a.partials, sc, sm);
      if (threadIdx.x == 0) {
        for (int j = 0; j < NR; ++j) {
          if (!s_active[j]) continue;
          const double g_new = sc[j], dl = sc[NR + j], rr = sc[2 * NR + j];
          s_rr[j] = rr;
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
      if constexpr (COARSE) {  // sigma <- Phi^T w + beta sigma
        for (int e = threadIdx.x; e < NC; e += blockDim.x) {
          const int j = e % NR;
          if (s_active[j]) s_sig[e] = sc[3 * NR + e] + s_beta[j] * s_sig[e];
        }
      }
      all_done = true;
      for (int j = 0; j < NR; ++j) all_done = all_done && (s_active[j] == 0);
      __syncthreads();
      if (all_done) break;
      for (int64_t v = r0 + threadIdx.x; v < r1; v += blockDim.x) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (!s_active[j]) continue;
          const T be = (T)s_beta[j];
          p[v * NR + j] = u[v * NR + j] + be * p[v * NR + j];
          s[v * NR + j] = w[v * NR + j] + be * s[v * NR + j];
        }
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (a.iters_out) atomicAdd(a.iters_out, it);
      if (a.fail_out && !all_done) atomicExch(a.fail_out, 1);
      if (a.last_iters) *a.last_iters = it;
      if (a.relres_out) {
        for (int j = 0; j < NR; ++j) a.relres_out[j] = s_bb[j] > 0.0 ? sqrt(s_rr[j] / s_bb[j]) : 0.0;
      }
    }
  }
  return;
timeout:
  if (threadIdx.x == 0 && a.timeout_out) atomicExch(a.timeout_out, 1);
}

template <int NR, typename T, bool COARSE>
static cudaError_t launch_pcg_impl(const PcgArgsT<T>& args, int grid, cudaStream_t st) {
  PcgArgsT<T> a = args;
  void* params[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)pcg_kernel<NR, T, COARSE>, dim3(grid), dim3(256), params, 0, st);
}

__global__ void __launch_bounds__(32) k_wait_check(GridBarrier* bar, unsigned long long wait_ns, int* timed_out) {
  __shared__ int s_flag;
  unsigned epoch = 0;
  // block 1 leaves without arriving: block 0's wait can only run out
  const bool ok = grid_sync(bar, epoch, &s_flag, wait_ns, blockIdx.x == 0);
  if (blockIdx.x == 0 && threadIdx.x == 0) *timed_out = ok ? 0 : 1;
}

cudaError_t launch_wait_check(GridBarrier* bar, unsigned long long wait_ns, int* timed_out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st);
  if (e != cudaSuccess) return e;
  void* params[] = {(void*)&bar, (void*)&wait_ns, (void*)&timed_out};
  return cudaLaunchCooperativeKernel((const void*)k_wait_check, dim3(2), dim3(32), params, 0, st);
}

int pcg_max_grid(int nrhs, int64_t n) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (nrhs == 3)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg_kernel<3, double, true>, 256, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg_kernel<16, double, false>, 256, 0);
  if (occ < 1) return 1;  // cooperative launch needs co-residency; one block always fits
  // One block per SM at most: the barrier and the partial sums cost grow with
  // the block count. At least ~128 rows per block otherwise: FP64 issues at a
  // small fraction of the FP32 rate on GB300, so a small system spread over
  // few SMs is bound by their FP64 pipes (measured: 8,640 rows on 17 blocks,
  // about 140 us per CG iteration).
  int64_t want = (n + 127) / 128;
  int64_t cap = (int64_t)sms;
  int64_t g = want < cap ? want : cap;
  return (int)(g < 1 ? 1 : g);
}

template <typename T> cudaError_t launch_pcg(int nrhs, const PcgArgsT<T>& args, int grid, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(args.bar, 0, sizeof(GridBarrier), st);
  if (e != cudaSuccess) return e;
  if (nrhs == 3) {
    if (args.phi && args.Einv) return launch_pcg_impl<3, T, true>(args, grid, st);
    return launch_pcg_impl<3, T, false>(args, grid, st);
  }
  if (nrhs == 16) return launch_pcg_impl<16, T, false>(args, grid, st);
  return cudaErrorInvalidValue;
}

template cudaError_t launch_pcg<double>(int, const PcgArgsT<double>&, int, cudaStream_t);
template cudaError_t launch_pcg<float>(int, const PcgArgsT<float>&, int, cudaStream_t);

// ----------------------------------------------------- FP64 refinement ----
// r = b - K x in FP64 for the first n rows, with a float copy for the inner
// solve and per-block partial sums of |r|^2 and |b|^2 (3 columns each).
__global__ void __launch_bounds__(256) k_residual64(int64_t n, const int32_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ col, const double* __restrict__ val,
                                                    const double* __restrict__ b, const double* __restrict__ x,
                                                    float* __restrict__ r32, double* __restrict__ r64,
                                                    double* __restrict__ partials, const uint8_t* __restrict__ skip) {
  __shared__ double sm[8 * red_pad(6)];
  double loc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    double acc[3];
    spmv_row<3, double>(rowptr, col, val, x, v, acc);
    const bool sum = !(skip && skip[v]);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double bv = b[3 * v + j];
      const double rv = bv - acc[j];
      if (r32) r32[3 * v + j] = (float)rv;
      if (r64) r64[3 * v + j] = rv;
      if (sum) {
        loc[j] += rv * rv;
        loc[3 + j] += bv * bv;
      }
    }
  }
  block_partials<6>(loc, partials + (size_t)blockIdx.x * 6, sm);
}

// out[k] = sum over the blocks of partials[b * 6 + k]: 32 groups of 8 threads
// (thread 8 g + k takes blocks g, g + 32, ..., eight loads in flight), then
// the group sums in a fixed order.
__global__ void __launch_bounds__(256) k_sum_partials6(const double* partials, int nblk, double* out) {
  __shared__ double sg[32][8];
  const int g = threadIdx.x >> 3, k = threadIdx.x & 7;
  double t = 0.0;
  if (k < 6) {
    int b = g;
    for (; b + 7 * 32 < nblk; b += 8 * 32) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = partials[(size_t)(b + 32 * u) * 6 + k];
#pragma unroll
      for (int u = 0; u < 8; ++u) t += v[u];
    }
    for (; b < nblk; b += 32) t += partials[(size_t)b * 6 + k];
  }
  sg[g][k] = t;
  __syncthreads();
  if (threadIdx.x < 6) {
    double x = 0.0;
    for (int gg = 0; gg < 32; ++gg) x += sg[gg][threadIdx.x];
    out[threadIdx.x] = x;
  }
}

__global__ void __launch_bounds__(256) k_axpy_f2d(int64_t n3, const float* __restrict__ e, double* __restrict__ x) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x)
    x[k] += (double)e[k];
}

cudaError_t launch_residual64(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* b,
                              const double* x, float* r32, double* r64, double* partials, int grid, double* out6,
                              cudaStream_t st, const uint8_t* skip) {
  k_residual64<<<grid, 256, 0, st>>>(n, rowptr, col, val, b, x, r32, r64, partials, skip);
  k_sum_partials6<<<1, 256, 0, st>>>(partials, grid, out6);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_axpy_d2d(int64_t n3, const double* __restrict__ e, double* __restrict__ x) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x)
    x[k] += e[k];
}

cudaError_t launch_axpy_d2d(int64_t n3, const double* e, double* x, cudaStream_t st) {
  int grid = (int)((n3 + 255) / 256);
  if (grid < 1) grid = 1;
  k_axpy_d2d<<<grid, 256, 0, st>>>(n3, e, x);
  return cudaGetLastError();
}

cudaError_t launch_axpy_f2d(int64_t n3, const float* e, double* x, cudaStream_t st) {
  int grid = (int)((n3 + 255) / 256);
  if (grid < 1) grid = 1;
  k_axpy_f2d<<<grid, 256, 0, st>>>(n3, e, x);
  return cudaGetLastError();
}

}  // namespace emu
