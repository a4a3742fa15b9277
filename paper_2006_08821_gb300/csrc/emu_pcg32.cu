// Register-resident FP32 conjugate gradient for the inner solves of the
// mixed path (the dq solve and the correction solves of the FP64-refined
// coupling solve, Eq. 4).
//
// Same iteration as the generic kernel (Chronopoulos-Gear CG, Jacobi plus
// the additive coarse space on the low-rank basis Phi), but GB300's FP64
// rate shapes it:
//   * every vector of the rows a thread owns lives in registers for the
//     whole solve; only u (needed by neighbouring rows) goes through global
//     memory, as one float4 per vertex;
//   * every reduction is FP32 with a fixed shuffle/shared-memory tree, so all
//     blocks hold bit-identical scalars and the result is deterministic;
//   * the matrix, D^-1 and Phi are read-only for the whole launch (__ldg).
// Two grid-wide barriers per iteration (after u, after the partial sums).
#include <cuda_runtime.h>
#include <stdint.h>

#include "emu_internal.h"
#include "emu_pcg.h"

namespace emu {

namespace {

constexpr int NT = 256;  // threads per block
constexpr int NR = 3;    // right-hand sides (x, y, z)
constexpr unsigned long long kSpinLimit32 = 1ull << 25;

__device__ __forceinline__ bool gsync(GridBarrier* bar, unsigned& epoch, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1u;
    __threadfence();
    const unsigned prev = atomicAdd(&bar->count, 1u);
    if (prev + 1u == gridDim.x * epoch) {
      __threadfence();
      atomicExch(&bar->gen, epoch);
    } else {
      unsigned long long spins = 0;
      while (true) {
        const unsigned g = *((volatile unsigned*)&bar->gen);
        if (g >= epoch) break;
        if (*((volatile int*)&bar->err)) break;
        if (++spins > kSpinLimit32) {
          atomicExch(&bar->err, 1);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    *s_flag = *((volatile int*)&bar->err);
  }
  __syncthreads();
  return *s_flag == 0;
}

// Block-wide FP32 sum of v[0..NV) into out[0..NV) (shared), fixed order.
template <int NV>
__device__ __forceinline__ void block_sum_f(float (&v)[NV], float* out, float* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sm[warp * NV + k] = x;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += NT) {
    float x = 0.f;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) x += sm[w * NV + k];
    out[k] = x;
  }
  __syncthreads();
}

}  // namespace

template <int RPT, bool COARSE>
__global__ void __launch_bounds__(NT) pcg32_kernel(PcgArgsT<float> a, float4* __restrict__ ug, float* __restrict__ part) {
  constexpr int NC = COARSE ? kModes * NR : 0;
  constexpr int NV0 = 4 * NR + NC;  // gamma, delta, rr, bb, Phi^T w
  constexpr int NV = 3 * NR + NC;   // gamma, delta, rr, Phi^T w
  __shared__ float sm[(NT / 32) * NV0];
  __shared__ float ssum[NV0];
  __shared__ float s_al[NR], s_be[NR], s_ga[NR], s_thr[NR], s_bb[NR], s_rr[NR];
  __shared__ int s_act[NR];
  __shared__ float s_rho[NC > 0 ? NC : 1], s_sig[NC > 0 ? NC : 1], s_cc[NC > 0 ? NC : 1];
  __shared__ float s_Einv[COARSE ? kModes * kModes : 1];
  __shared__ int s_flag;
  unsigned epoch = 0;
  const int64_t n = a.n;
  const int64_t stride = (int64_t)gridDim.x * NT;
  const int64_t g0 = (int64_t)blockIdx.x * NT + threadIdx.x;
  const int32_t* __restrict__ rowptr = a.rowptr;
  const int32_t* __restrict__ col = a.col;
  const float* __restrict__ val = a.val;
  if constexpr (COARSE) {
    for (int k = threadIdx.x; k < kModes * kModes; k += NT) s_Einv[k] = (float)a.Einv[k];
  }

  float x[RPT][NR], r[RPT][NR], p[RPT][NR], s[RPT][NR], u[RPT][NR], w[RPT][NR];
  float di[RPT];
  bool own[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int64_t v = g0 + k * stride;
    own[k] = v < n;
    di[k] = own[k] ? __ldg(a.dinv + v) : 0.f;
#pragma unroll
    for (int j = 0; j < NR; ++j) x[k][j] = own[k] ? a.x[v * NR + j] : 0.f;
  }

  // y = A z for the owned rows, z read as float4 per vertex (neighbours' values)
  auto spmv = [&](const float4* __restrict__ z, float (&y)[RPT][NR]) {
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      y[k][0] = y[k][1] = y[k][2] = 0.f;
      if (!own[k]) continue;
      const int64_t v = g0 + k * stride;
      const int32_t e0 = __ldg(rowptr + v), e1 = __ldg(rowptr + v + 1);
      int32_t e = e0;
      for (; e + 4 <= e1; e += 4) {
        int32_t c4[4];
        float a4[4];
        float4 z4[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          c4[t] = __ldg(col + e + t);
          a4[t] = __ldg(val + e + t);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) z4[t] = __ldcg(z + c4[t]);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          y[k][0] += a4[t] * z4[t].x;
          y[k][1] += a4[t] * z4[t].y;
          y[k][2] += a4[t] * z4[t].z;
        }
      }
      for (; e < e1; ++e) {
        const float av = __ldg(val + e);
        const float4 zz = __ldcg(z + __ldg(col + e));
        y[k][0] += av * zz.x;
        y[k][1] += av * zz.y;
        y[k][2] += av * zz.z;
      }
    }
  };
  // u = D^-1 r + Phi cc, stored for the neighbours
  auto precond = [&]() {
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      if (!own[k]) continue;
      const int64_t v = g0 + k * stride;
#pragma unroll
      for (int j = 0; j < NR; ++j) u[k][j] = di[k] * r[k][j];
      if constexpr (COARSE) {
#pragma unroll
        for (int m = 0; m < kModes; ++m) {
          const float ph = __ldg(a.phi + v * kModes + m);
#pragma unroll
          for (int j = 0; j < NR; ++j) u[k][j] += ph * s_cc[m * NR + j];
        }
      }
      ug[v] = make_float4(u[k][0], u[k][1], u[k][2], 0.f);
    }
  };
  auto coarse_cc = [&]() {  // s_cc = E^-1 rho
    if constexpr (COARSE) {
      for (int e = threadIdx.x; e < NC; e += NT) {
        const int m = e / NR, j = e % NR;
        float acc = 0.f;
#pragma unroll
        for (int l = 0; l < kModes; ++l) acc += s_Einv[m * kModes + l] * s_rho[l * NR + j];
        s_cc[e] = acc;
      }
      __syncthreads();
    }
  };
  // global sums: every block sums all block partials in the same fixed order
  auto global_sum = [&](int nv) {
    float v[NV0];
#pragma unroll
    for (int k = 0; k < NV0; ++k) v[k] = 0.f;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += NT) {
#pragma unroll
      for (int k = 0; k < NV0; ++k)
        if (k < nv) v[k] += __ldcg(part + (size_t)b * NV0 + k);
    }
    block_sum_f<NV0>(v, ssum, sm);
  };

  // ---- r = b - A x ------------------------------------------------------
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int64_t v = g0 + k * stride;
    if (own[k]) ug[v] = make_float4(x[k][0], x[k][1], x[k][2], 0.f);
  }
  if (!gsync(a.bar, epoch, &s_flag)) goto timeout;
  spmv(ug, w);
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int64_t v = g0 + k * stride;
#pragma unroll
    for (int j = 0; j < NR; ++j) r[k][j] = own[k] ? a.b[v * NR + j] - w[k][j] : 0.f;
  }
  if constexpr (COARSE) {  // rho = Phi^T r
    float loc[NV0];
#pragma unroll
    for (int k = 0; k < NV0; ++k) loc[k] = 0.f;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      if (!own[k]) continue;
      const int64_t v = g0 + k * stride;
#pragma unroll
      for (int m = 0; m < kModes; ++m) {
        const float ph = __ldg(a.phi + v * kModes + m);
#pragma unroll
        for (int j = 0; j < NR; ++j) loc[m * NR + j] += ph * r[k][j];
      }
    }
    block_sum_f<NV0>(loc, ssum, sm);
    for (int k = threadIdx.x; k < NC; k += NT) part[(size_t)blockIdx.x * NV0 + k] = ssum[k];
    if (!gsync(a.bar, epoch, &s_flag)) goto timeout;
    global_sum(NC);
    for (int k = threadIdx.x; k < NC; k += NT) s_rho[k] = ssum[k];
    __syncthreads();
    coarse_cc();
  }
  // ug still holds x; every block must have finished reading it
  if (!gsync(a.bar, epoch, &s_flag)) goto timeout;
  precond();
  if (!gsync(a.bar, epoch, &s_flag)) goto timeout;
  spmv(ug, w);
  {
    float loc[NV0];
#pragma unroll
    for (int k = 0; k < NV0; ++k) loc[k] = 0.f;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      if (!own[k]) continue;
      const int64_t v = g0 + k * stride;
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const float bv = a.b[v * NR + j];
        loc[j] += r[k][j] * u[k][j];
        loc[NR + j] += w[k][j] * u[k][j];
        loc[2 * NR + j] += r[k][j] * r[k][j];
        loc[3 * NR + j] += bv * bv;
      }
      if constexpr (COARSE) {
#pragma unroll
        for (int m = 0; m < kModes; ++m) {
          const float ph = __ldg(a.phi + v * kModes + m);
#pragma unroll
          for (int j = 0; j < NR; ++j) loc[4 * NR + m * NR + j] += ph * w[k][j];
        }
      }
    }
    block_sum_f<NV0>(loc, ssum, sm);
    for (int k = threadIdx.x; k < NV0; k += NT) part[(size_t)blockIdx.x * NV0 + k] = ssum[k];
  }
  if (!gsync(a.bar, epoch, &s_flag)) goto timeout;
  global_sum(NV0);
  if (threadIdx.x < NR) {
    const int j = threadIdx.x;
    const float bb = ssum[3 * NR + j];
    s_bb[j] = bb;
    s_rr[j] = ssum[2 * NR + j];
    s_thr[j] = (float)(a.tol * a.tol) * bb;
    s_ga[j] = ssum[j];
    const bool done = (ssum[2 * NR + j] <= s_thr[j]) || !(ssum[NR + j] > 0.f);
    s_act[j] = done ? 0 : 1;
    s_al[j] = done ? 0.f : ssum[j] / ssum[NR + j];
    s_be[j] = 0.f;
  }
  if constexpr (COARSE) {
    for (int k = threadIdx.x; k < NC; k += NT) s_sig[k] = ssum[4 * NR + k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < RPT; ++k)
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      p[k][j] = u[k][j];
      s[k][j] = w[k][j];
      if (s_bb[j] == 0.f) x[k][j] = 0.f;  // zero right-hand side: x = 0 exactly
    }
  {
    int it = 0;
    bool all_done = !(s_act[0] || s_act[1] || s_act[2]);
    while (!all_done && it < a.max_iter) {
      ++it;
      // x += alpha p, r -= alpha s, rho -= alpha sigma; u = M r
#pragma unroll
      for (int k = 0; k < RPT; ++k)
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (!s_act[j]) continue;
          x[k][j] += s_al[j] * p[k][j];
          r[k][j] -= s_al[j] * s[k][j];
        }
      if constexpr (COARSE) {
        for (int e = threadIdx.x; e < NC; e += NT) {
          const int j = e % NR;
          if (s_act[j]) s_rho[e] -= s_al[j] * s_sig[e];
        }
        __syncthreads();
        coarse_cc();
      }
      precond();
      if (!gsync(a.bar, epoch, &s_flag)) goto timeout;
      spmv(ug, w);
      {
        float loc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) loc[k] = 0.f;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          if (!own[k]) continue;
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            loc[j] += r[k][j] * u[k][j];
            loc[NR + j] += w[k][j] * u[k][j];
            loc[2 * NR + j] += r[k][j] * r[k][j];
          }
          if constexpr (COARSE) {
            const int64_t v = g0 + k * stride;
#pragma unroll
            for (int m = 0; m < kModes; ++m) {
              const float ph = __ldg(a.phi + v * kModes + m);
#pragma unroll
              for (int j = 0; j < NR; ++j) loc[3 * NR + m * NR + j] += ph * w[k][j];
            }
          }
        }
        float lfull[NV0];
#pragma unroll
        for (int k = 0; k < NV0; ++k) lfull[k] = k < NV ? loc[k] : 0.f;
        block_sum_f<NV0>(lfull, ssum, sm);
        for (int k = threadIdx.x; k < NV; k += NT) part[(size_t)blockIdx.x * NV0 + k] = ssum[k];
      }
      if (!gsync(a.bar, epoch, &s_flag)) goto timeout;
      global_sum(NV);
      if (threadIdx.x < NR) {
        const int j = threadIdx.x;
        if (s_act[j]) {
          const float g_new = ssum[j], dl = ssum[NR + j], rr = ssum[2 * NR + j];
          s_rr[j] = rr;
          if (rr <= s_thr[j]) {
            s_act[j] = 0;
          } else {
            const float be = g_new / s_ga[j];
            const float den = dl - be * g_new / s_al[j];
            if (!(den > 0.f)) {
              s_act[j] = 0;
            } else {
              s_be[j] = be;
              s_al[j] = g_new / den;
              s_ga[j] = g_new;
            }
          }
        }
      }
      __syncthreads();
      if constexpr (COARSE) {
        for (int e = threadIdx.x; e < NC; e += NT) {
          const int j = e % NR;
          if (s_act[j]) s_sig[e] = ssum[3 * NR + e] + s_be[j] * s_sig[e];
        }
      }
      all_done = !(s_act[0] || s_act[1] || s_act[2]);
      if (all_done) break;
#pragma unroll
      for (int k = 0; k < RPT; ++k)
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (!s_act[j]) continue;
          p[k][j] = u[k][j] + s_be[j] * p[k][j];
          s[k][j] = w[k][j] + s_be[j] * s[k][j];
        }
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int64_t v = g0 + k * stride;
      if (own[k])
#pragma unroll
        for (int j = 0; j < NR; ++j) a.x[v * NR + j] = x[k][j];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (a.iters_out) atomicAdd(a.iters_out, it);
      if (a.fail_out && !all_done) atomicExch(a.fail_out, 1);
      if (a.last_iters) *a.last_iters = it;
      if (a.relres_out)
        for (int j = 0; j < NR; ++j) a.relres_out[j] = s_bb[j] > 0.f ? sqrt((double)s_rr[j] / s_bb[j]) : 0.0;
    }
  }
  return;
timeout:
  if (threadIdx.x == 0 && a.timeout_out) atomicExch(a.timeout_out, 1);
}

namespace {
template <int RPT, bool C>
cudaError_t launch32(const PcgArgsT<float>& args, float4* ug, float* part, int grid, cudaStream_t st) {
  PcgArgsT<float> a = args;
  void* params[] = {(void*)&a, (void*)&ug, (void*)&part};
  return cudaLaunchCooperativeKernel((const void*)pcg32_kernel<RPT, C>, dim3(grid), dim3(NT), params, 0, st);
}
}  // namespace

// Launch shape: blocks <= one per SM, rows per thread a power of two <= 8.
bool pcg32_shape(int64_t n, int sms, int* grid, int* rpt) {
  int64_t nb = (n + 2 * NT - 1) / (2 * NT);
  if (nb > sms) nb = sms;
  if (nb < 1) nb = 1;
  int r = 1;
  while ((int64_t)nb * NT * r < n) r *= 2;
  if (r > 8) return false;
  *grid = (int)nb;
  *rpt = r;
  return true;
}

cudaError_t launch_pcg32(const PcgArgsT<float>& args, float4* ug, float* part, int grid, int rpt, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(args.bar, 0, sizeof(GridBarrier), st);
  if (e != cudaSuccess) return e;
  const bool c = args.phi && args.Einv;
  switch (rpt) {
    case 1: return c ? launch32<1, true>(args, ug, part, grid, st) : launch32<1, false>(args, ug, part, grid, st);
    case 2: return c ? launch32<2, true>(args, ug, part, grid, st) : launch32<2, false>(args, ug, part, grid, st);
    case 4: return c ? launch32<4, true>(args, ug, part, grid, st) : launch32<4, false>(args, ug, part, grid, st);
    case 8: return c ? launch32<8, true>(args, ug, part, grid, st) : launch32<8, false>(args, ug, part, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace emu
