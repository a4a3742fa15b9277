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
//   * every reduction is FP32 with a fixed shuffle/shared-memory tree
//     (transposed butterflies: a warp moves each value through the shuffle
//     unit about once), so all blocks hold bit-identical scalars and the
//     result is deterministic;
//   * the matrix, D^-1 and Phi are read-only for the whole launch (__ldg).
// Two grid-wide barriers per iteration (after u, after the partial sums);
// pcg32p_kernel below is the pipelined variant with one.
#include <cuda_runtime.h>

#include <mutex>

#include <algorithm>
#include <stdint.h>

#include "emu_internal.h"
#include "emu_pcg.h"

namespace emu {

namespace {

constexpr int NT = 256;  // threads per block
constexpr int NR = 3;    // right-hand sides (x, y, z)
constexpr int kGather = 16;  // entries of a matrix row gathered at once
constexpr int kMaxGridStrides = 8;  // grid_sum_f handles up to 256 blocks
// words of Pcg32Work::sync, one 128-byte line apart
constexpr int kSyncCount = 0, kSyncDone = 32, kSyncErr = 64;

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier: every block adds 1 to an arrival counter with a release
// reduction (its writes become visible first), and one thread per block
// polls the counter with acquire loads until all blocks of this barrier
// have arrived. The counter is never reset inside a launch (barrier e waits
// for e * gridDim.x arrivals); the last block to leave the kernel zeroes it
// for the next launch. The wait is bounded: on timeout the block raises the
// error word, every other waiter sees it, and all blocks leave.
__device__ __forceinline__ bool gbar(const Pcg32Work& wk, unsigned& epoch, int* s_flag, unsigned long long wait_ns) {
  __syncthreads();
  epoch += 1u;
  if (threadIdx.x == 0) {
    red_release_add(wk.sync + kSyncCount, 1u);
    const unsigned target = gridDim.x * epoch;
    int bad = 0;
    unsigned long long spins = 0;
    unsigned long long t0 = 0;
    while (ld_acquire_u32(wk.sync + kSyncCount) < target) {
      ++spins;
      if ((spins & 63u) == 0u) {
        if (*((volatile unsigned*)(wk.sync + kSyncErr))) {
          bad = 1;
          break;
        }
        // the clock is read only once a wait is long (the fast path polls)
        const unsigned long long now = global_ns();
        if (t0 == 0) t0 = now;
        if (now - t0 > wait_ns || spins > kWaitSpinCap) {
          bad = 1;
          atomicExch(wk.sync + kSyncErr, 1u);
          break;
        }
      }
    }
    *s_flag = bad;
  }
  __syncthreads();
  return *s_flag == 0;
}

// Kernel exit of every block: the last one out zeroes the barrier words.
__device__ __forceinline__ void gbar_exit(const Pcg32Work& wk) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(wk.sync + kSyncDone, 1u);
    if (prev + 1u == gridDim.x) {
      atomicExch(wk.sync + kSyncCount, 0u);
      atomicExch(wk.sync + kSyncErr, 0u);
      atomicExch(wk.sync + kSyncDone, 0u);
    }
  }
}

// Transposed (reduce-scatter) butterfly over one warp. On entry every lane
// holds C values; at each step with partner offset O a lane sends half of
// its values to the partner and adds the partner's half to the half it
// keeps, so after five steps the warp has moved about C values through the
// shuffle unit instead of 5 C. With C < 32 the last steps are plain
// butterflies on one value. The order of every addition is fixed.
template <int C, int O>
__device__ __forceinline__ void warp_rs(float* v, int lane) {
  if constexpr (C >= 2) {
    constexpr int H = C / 2;
    const bool hi = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const float send = hi ? v[i] : v[H + i];
      const float keep = hi ? v[H + i] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
    if constexpr (O > 1) warp_rs<H, O / 2>(v, lane);
  } else {
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
    if constexpr (O > 1) warp_rs<1, O / 2>(v, lane);
  }
}

// Index of the first of the max(C / 32, 1) sums lane holds after warp_rs<C, 16>.
template <int C>
__device__ __forceinline__ int warp_rs_first(int lane) {
  int idx = 0, c = C;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1)
    if (c >= 2) {
      c >>= 1;
      if (lane & o) idx += c;
    }
  return idx;
}

__host__ __device__ constexpr int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p *= 2;
  return p;
}

// Block-wide FP32 sum of v[0..NV) into out[0..NV) (shared), fixed order.
template <int NV>
__device__ __forceinline__ void block_sum_f(float (&v)[NV], float* out, float* sm) {
  constexpr int P = pow2_at_least(NV);
  constexpr int HOLD = P >= 32 ? P / 32 : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float t[P];
#pragma unroll
  for (int k = 0; k < P; ++k) t[k] = k < NV ? v[k] : 0.f;
  warp_rs<P, 16>(t, lane);
  const int first = warp_rs_first<P>(lane);
#pragma unroll
  for (int h = 0; h < HOLD; ++h)
    if (first + h < NV) sm[warp * NV + first + h] = t[h];  // equal copies when P < 32
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += NT) {
    float x = 0.f;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) x += sm[w * NV + k];
    out[k] = x;
  }
  __syncthreads();
}

// Grid-wide sums of the first nv of NV block partials, stored value-major
// (part[k * G + b]): warp w sums the values k = w, w + 8, ... with its lanes
// striding over the blocks, then one transposed butterfly per warp.
template <int NV>
__device__ __forceinline__ void grid_sum_f(const float* __restrict__ part, int nv, float* out) {
  constexpr int VPW = (NV + NT / 32 - 1) / (NT / 32);
  constexpr int P = pow2_at_least(VPW);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = gridDim.x;
  float t[P];
#pragma unroll
  for (int j = 0; j < P; ++j) t[j] = 0.f;
#pragma unroll
  for (int s = 0; s < kMaxGridStrides; ++s) {
    const int b = lane + 32 * s;
    if (b < G) {
#pragma unroll
      for (int j = 0; j < VPW; ++j) {
        const int k = warp + (NT / 32) * j;
        if (k < nv) t[j] += __ldcg(part + (size_t)k * G + b);
      }
    }
  }
  warp_rs<P, 16>(t, lane);
  const int first = warp_rs_first<P>(lane);  // P <= 8 here: one sum per lane
  {
    const int k = warp + (NT / 32) * first;
    if (first < VPW && k < nv) out[k] = t[0];
  }
  __syncthreads();
}

// y = A z for the rows a thread owns (g0 + k stride, k < RPT), z read as
// float4 per vertex (the neighbours' values). The first kGather entries of a
// row are gathered at once, so a row costs one L2 round trip (a vertex of a
// tetrahedral grid has at most 14 neighbours); longer rows finish in a plain
// loop.
template <int RPT>
__device__ __forceinline__ void spmv_rows(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                          const float* __restrict__ val, const bool (&own)[RPT], int64_t g0,
                                          int64_t stride, const float4* __restrict__ z, float (&y)[RPT][NR]) {
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    y[k][0] = y[k][1] = y[k][2] = 0.f;
    if (!own[k]) continue;
    const int64_t v = g0 + k * stride;
    const int32_t e0 = __ldg(rowptr + v), e1 = __ldg(rowptr + v + 1);
    const int cnt = e1 - e0;
    float4 z4[kGather];
    float a4[kGather];
#pragma unroll
    for (int t = 0; t < kGather; ++t) {
      a4[t] = 0.f;
      z4[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (t < cnt) {
        a4[t] = __ldg(val + e0 + t);
        z4[t] = __ldcg(z + __ldg(col + e0 + t));
      }
    }
#pragma unroll
    for (int t = 0; t < kGather; ++t) {
      y[k][0] += a4[t] * z4[t].x;
      y[k][1] += a4[t] * z4[t].y;
      y[k][2] += a4[t] * z4[t].z;
    }
    for (int32_t e = e0 + kGather; e < e1; ++e) {
      const float av = __ldg(val + e);
      const float4 zz = __ldcg(z + __ldg(col + e));
      y[k][0] += av * zz.x;
      y[k][1] += av * zz.y;
      y[k][2] += av * zz.z;
    }
  }
}

// loc[m NR + j] += Phi[v][m] y[k][j] over the owned rows; the coarse rows of
// a thread live in shared memory, float4 q of row k at sPhi[(q RPT + k) NT + tid]
template <int RPT>
__device__ __forceinline__ void phi_t_rows(const float4* sPhi, const bool (&own)[RPT], const float (&y)[RPT][NR],
                                           float* loc) {
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    if (!own[k]) continue;
#pragma unroll
    for (int q = 0; q < kModes / 4; ++q) {
      const float4 ph = sPhi[(q * RPT + k) * NT + threadIdx.x];
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        loc[(4 * q) * NR + j] += ph.x * y[k][j];
        loc[(4 * q + 1) * NR + j] += ph.y * y[k][j];
        loc[(4 * q + 2) * NR + j] += ph.z * y[k][j];
        loc[(4 * q + 3) * NR + j] += ph.w * y[k][j];
      }
    }
  }
}

// cc = E^-1 rho for the 16 x 3 coarse coefficients (block-wide, then a barrier)
__device__ __forceinline__ void coarse_solve(const float* s_Einv, const float* s_rho, float* s_cc) {
  for (int e = threadIdx.x; e < kModes * NR; e += NT) {
    const int m = e / NR, j = e % NR;
    float acc = 0.f;
#pragma unroll
    for (int l = 0; l < kModes; ++l) acc += s_Einv[m * kModes + l] * s_rho[l * NR + j];
    s_cc[e] = acc;
  }
  __syncthreads();
}
}  // namespace

template <int RPT, bool COARSE>
__global__ void __launch_bounds__(NT, 1) pcg32_kernel(PcgArgsT<float> a, Pcg32Work wk) {
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
  // the coarse basis rows of this thread, float4 q of row k at
  // sPhi[(q * RPT + k) * NT + tid] (consecutive threads, consecutive 16 bytes)
  extern __shared__ float4 sPhi[];
  unsigned epoch = 0;
  const int64_t n = a.n;
  float4* __restrict__ ugx = wk.ug;      // x of the first residual
  float4* __restrict__ ugu = wk.ug + n;  // preconditioned residual u
  float* __restrict__ part = wk.part;
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
    if constexpr (COARSE) {
      const float4* ph = reinterpret_cast<const float4*>(a.phi + v * kModes);
#pragma unroll
      for (int q = 0; q < kModes / 4; ++q)
        sPhi[(q * RPT + k) * NT + threadIdx.x] = own[k] ? __ldg(ph + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }

  auto spmv = [&](const float4* __restrict__ z, float (&y)[RPT][NR]) {
    spmv_rows<RPT>(rowptr, col, val, own, g0, stride, z, y);
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
        for (int q = 0; q < kModes / 4; ++q) {
          const float4 ph = sPhi[(q * RPT + k) * NT + threadIdx.x];
#pragma unroll
          for (int j = 0; j < NR; ++j)
            u[k][j] += ph.x * s_cc[(4 * q) * NR + j] + ph.y * s_cc[(4 * q + 1) * NR + j] +
                       ph.z * s_cc[(4 * q + 2) * NR + j] + ph.w * s_cc[(4 * q + 3) * NR + j];
        }
      }
      ugu[v] = make_float4(u[k][0], u[k][1], u[k][2], 0.f);
    }
  };
  auto coarse_cc = [&]() {  // s_cc = E^-1 rho
    if constexpr (COARSE) coarse_solve(s_Einv, s_rho, s_cc);
  };
  // global sums: every block sums all block partials in the same fixed order
  auto global_sum = [&](int nv) { grid_sum_f<NV0>(part, nv, ssum); };
  // loc[off + m NR + j] += Phi[v][m] y[k][j] over the owned rows
  auto phi_t = [&](const float (&y)[RPT][NR], float* loc) {
    if constexpr (COARSE) phi_t_rows<RPT>(sPhi, own, y, loc);
  };
  const int G = gridDim.x;

  // ---- r = b - A x ------------------------------------------------------
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int64_t v = g0 + k * stride;
    if (own[k]) ugx[v] = make_float4(x[k][0], x[k][1], x[k][2], 0.f);
  }
  if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
  spmv(ugx, w);
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
    phi_t(r, loc);
    block_sum_f<NV0>(loc, ssum, sm);
    for (int k = threadIdx.x; k < NC; k += NT) part[(size_t)k * G + blockIdx.x] = ssum[k];
    if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
    global_sum(NC);
    for (int k = threadIdx.x; k < NC; k += NT) s_rho[k] = ssum[k];
    __syncthreads();
    coarse_cc();
  }
  // u goes to its own buffer, so no block can overwrite x while it is read
  precond();
  if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
  spmv(ugu, w);
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
    }
    phi_t(w, loc + 4 * NR);
    block_sum_f<NV0>(loc, ssum, sm);
    for (int k = threadIdx.x; k < NV0; k += NT) part[(size_t)k * G + blockIdx.x] = ssum[k];
  }
  if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
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
      if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
      spmv(ugu, w);
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
        }
        phi_t(w, loc + 3 * NR);
        float lfull[NV0];
#pragma unroll
        for (int k = 0; k < NV0; ++k) lfull[k] = k < NV ? loc[k] : 0.f;
        block_sum_f<NV0>(lfull, ssum, sm);
        for (int k = threadIdx.x; k < NV; k += NT) part[(size_t)k * G + blockIdx.x] = ssum[k];
      }
      if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
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
  gbar_exit(wk);
  return;
timeout:
  if (threadIdx.x == 0 && a.timeout_out) atomicExch(a.timeout_out, 1);
  gbar_exit(wk);
}


// Pipelined form of the same Chronopoulos-Gear iteration (after Ghysels and
// Vanroose), with one grid barrier per iteration instead of two. The
// preconditioned residual u = M r and w = A u are carried by recurrences,
// together with q = M s and z = A q, so that the only vector a block needs
// from its neighbours, v = D^-1 w, is published with the partial sums of the
// same iteration. The coarse part of M w, Phi E^-1 Phi^T w, needs Phi^T w,
// a global sum; it is applied after the barrier through the precomputed
// rows of A Phi: n = A M w = A v + (A Phi) c with c = E^-1 Phi^T w.
// Exchange vectors and partial sums alternate between two buffers: a block
// may publish iteration i + 1 while a slower one still reads iteration i.
template <int RPT>
__global__ void __launch_bounds__(NT, 1) pcg32p_kernel(PcgArgsT<float> a, Pcg32Work wk) {
  constexpr int NC = kModes * NR;
  constexpr int NV0 = 4 * NR + NC;  // gamma, delta, rr, bb, Phi^T w
  constexpr int PSTRIDE = 64;       // values per partial-sum buffer (x grid)
  static_assert(NV0 <= PSTRIDE, "partial sums exceed their buffer");
  __shared__ float sm[(NT / 32) * NV0];
  __shared__ float ssum[NV0];
  __shared__ float s_al[NR], s_be[NR], s_ga[NR], s_thr[NR], s_bb[NR], s_rr[NR];
  __shared__ int s_act[NR];
  __shared__ float s_rho[NC], s_cc[NC];
  __shared__ float s_Einv[kModes * kModes];
  __shared__ int s_flag;
  // rows of Phi, then rows of A Phi: float4 q of row k at [(q * RPT + k) * NT + tid]
  extern __shared__ float4 sPhi[];
  float4* sAPhi = sPhi + (kModes / 4) * RPT * NT;
  unsigned epoch = 0;
  const int64_t n = a.n;
  const int G = gridDim.x;
  const int64_t stride = (int64_t)G * NT;
  const int64_t g0 = (int64_t)blockIdx.x * NT + threadIdx.x;
  const int32_t* __restrict__ rowptr = a.rowptr;
  const int32_t* __restrict__ col = a.col;
  const float* __restrict__ val = a.val;
  for (int k = threadIdx.x; k < kModes * kModes; k += NT) s_Einv[k] = (float)a.Einv[k];

  float x[RPT][NR], r[RPT][NR], u[RPT][NR], w[RPT][NR], p[RPT][NR], s[RPT][NR], qv[RPT][NR], z[RPT][NR];
  float di[RPT];
  bool own[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int64_t v = g0 + k * stride;
    own[k] = v < n;
    di[k] = own[k] ? __ldg(a.dinv + v) : 0.f;
    const float4* ph = reinterpret_cast<const float4*>(a.phi + v * kModes);
    const float4* aph = reinterpret_cast<const float4*>(wk.aphi + v * kModes);
#pragma unroll
    for (int q = 0; q < kModes / 4; ++q) {
      sPhi[(q * RPT + k) * NT + threadIdx.x] = own[k] ? __ldg(ph + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      sAPhi[(q * RPT + k) * NT + threadIdx.x] = own[k] ? __ldg(aph + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      x[k][j] = own[k] ? a.x[v * NR + j] : 0.f;
      p[k][j] = s[k][j] = qv[k][j] = z[k][j] = 0.f;
    }
  }

  auto spmv = [&](const float4* __restrict__ zsrc, float (&y)[RPT][NR]) {
    spmv_rows<RPT>(rowptr, col, val, own, g0, stride, zsrc, y);
  };
  auto phi_t = [&](const float (&y)[RPT][NR], float* loc) { phi_t_rows<RPT>(sPhi, own, y, loc); };
  auto coarse_cc = [&]() { coarse_solve(s_Einv, s_rho, s_cc); };  // s_cc = E^-1 s_rho
  // sum_m rows[v][m] s_cc[m NR + j] for row k (rows: sPhi or sAPhi)
  auto coarse_row = [&](const float4* rows, int k, int j) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < kModes / 4; ++q) {
      const float4 ph = rows[(q * RPT + k) * NT + threadIdx.x];
      acc += ph.x * s_cc[(4 * q) * NR + j] + ph.y * s_cc[(4 * q + 1) * NR + j] + ph.z * s_cc[(4 * q + 2) * NR + j] +
             ph.w * s_cc[(4 * q + 3) * NR + j];
    }
    return acc;
  };

  // ---- r = b - A x ------------------------------------------------------
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int64_t v = g0 + k * stride;
    if (own[k]) wk.ug[v] = make_float4(x[k][0], x[k][1], x[k][2], 0.f);
  }
  if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
  spmv(wk.ug, w);
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int64_t v = g0 + k * stride;
#pragma unroll
    for (int j = 0; j < NR; ++j) r[k][j] = own[k] ? a.b[v * NR + j] - w[k][j] : 0.f;
  }
  {  // u = D^-1 r + Phi E^-1 Phi^T r, published in the second exchange buffer
    float loc[NV0];
#pragma unroll
    for (int k = 0; k < NV0; ++k) loc[k] = 0.f;
    phi_t(r, loc);
    block_sum_f<NV0>(loc, ssum, sm);
    for (int k = threadIdx.x; k < NC; k += NT) wk.part[(size_t)k * G + blockIdx.x] = ssum[k];
    if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
    grid_sum_f<NV0>(wk.part, NC, ssum);
    for (int k = threadIdx.x; k < NC; k += NT) s_rho[k] = ssum[k];
    __syncthreads();
    coarse_cc();
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int64_t v = g0 + k * stride;
#pragma unroll
      for (int j = 0; j < NR; ++j) u[k][j] = own[k] ? di[k] * r[k][j] + coarse_row(sPhi, k, j) : 0.f;
      if (own[k]) wk.ug[n + v] = make_float4(u[k][0], u[k][1], u[k][2], 0.f);
    }
  }
  if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
  spmv(wk.ug + n, w);  // w = A u

  {
    int it = 0, buf = 0;
    bool first = true, all_done = false;
    for (;;) {
      float* __restrict__ pb = wk.part + (size_t)buf * PSTRIDE * G;
      float4* __restrict__ ub = wk.ug + (size_t)buf * n;
      {  // partial sums of this iteration and v = D^-1 w for the neighbours
        float loc[NV0];
#pragma unroll
        for (int k = 0; k < NV0; ++k) loc[k] = 0.f;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          if (!own[k]) continue;
          const int64_t v = g0 + k * stride;
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            loc[j] += r[k][j] * u[k][j];
            loc[NR + j] += w[k][j] * u[k][j];
            loc[2 * NR + j] += r[k][j] * r[k][j];
            if (first) {
              const float bv = a.b[v * NR + j];
              loc[3 * NR + j] += bv * bv;
            }
          }
          ub[v] = make_float4(di[k] * w[k][0], di[k] * w[k][1], di[k] * w[k][2], 0.f);
        }
        phi_t(w, loc + 4 * NR);
        block_sum_f<NV0>(loc, ssum, sm);
        for (int k = threadIdx.x; k < NV0; k += NT) pb[(size_t)k * G + blockIdx.x] = ssum[k];
      }
      if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
      grid_sum_f<NV0>(pb, NV0, ssum);
      if (threadIdx.x < NR) {
        const int j = threadIdx.x;
        if (first) {
          const float bb = ssum[3 * NR + j];
          s_bb[j] = bb;
          s_thr[j] = (float)(a.tol * a.tol) * bb;
          s_act[j] = 1;
        }
        const float rr = ssum[2 * NR + j];
        s_rr[j] = rr;
        if (s_act[j]) {
          const float g_new = ssum[j], dl = ssum[NR + j];
          if (rr <= s_thr[j]) {
            s_act[j] = 0;
          } else {
            const float be = first ? 0.f : g_new / s_ga[j];
            const float den = first ? dl : dl - be * g_new / s_al[j];
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
      for (int e = threadIdx.x; e < NC; e += NT) s_rho[e] = ssum[4 * NR + e];
      __syncthreads();
      if (first) {
#pragma unroll
        for (int k = 0; k < RPT; ++k)
#pragma unroll
          for (int j = 0; j < NR; ++j)
            if (s_bb[j] == 0.f) x[k][j] = 0.f;  // zero right-hand side: x = 0 exactly
      }
      all_done = !(s_act[0] || s_act[1] || s_act[2]);
      if (all_done || it >= a.max_iter) break;
      ++it;
      coarse_cc();  // c = E^-1 Phi^T w
      float nv[RPT][NR];
      spmv(ub, nv);  // A D^-1 w
#pragma unroll
      for (int k = 0; k < RPT; ++k)
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (!s_act[j]) continue;
          const float be = s_be[j], al = s_al[j];
          const float mv = di[k] * w[k][j] + coarse_row(sPhi, k, j);   // m = M w
          const float nn = nv[k][j] + coarse_row(sAPhi, k, j);         // n = A M w
          z[k][j] = nn + be * z[k][j];
          qv[k][j] = mv + be * qv[k][j];
          s[k][j] = w[k][j] + be * s[k][j];
          p[k][j] = u[k][j] + be * p[k][j];
          x[k][j] += al * p[k][j];
          r[k][j] -= al * s[k][j];
          u[k][j] -= al * qv[k][j];
          w[k][j] -= al * z[k][j];
        }
      first = false;
      buf ^= 1;
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
  gbar_exit(wk);
  return;
timeout:
  if (threadIdx.x == 0 && a.timeout_out) atomicExch(a.timeout_out, 1);
  gbar_exit(wk);
}

// aphi = A phi, one thread per (row, four modes)
__global__ void k_aphi32(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                         const float* __restrict__ val, const float4* __restrict__ phi, float4* __restrict__ aphi) {
  const int64_t tot = n * (kModes / 4);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / (kModes / 4);
    const int q = (int)(i % (kModes / 4));
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
      const float av = val[e];
      const float4 ph = phi[(int64_t)col[e] * (kModes / 4) + q];
      acc.x += av * ph.x;
      acc.y += av * ph.y;
      acc.z += av * ph.z;
      acc.w += av * ph.w;
    }
    aphi[i] = acc;
  }
}

namespace {
template <int RPT, bool C>
cudaError_t prepare32() {
  // the coarse rows live in dynamic shared memory (RPT x 16 KB); above the
  // default 48 KB the kernel needs the opt-in, a per-device attribute
  const size_t smem = C ? sizeof(float4) * (kModes / 4) * RPT * NT : 0;
  if (smem <= 48 * 1024) return cudaSuccess;
  static bool set[64] = {false};
  static std::mutex mu;  // handles may be built from several threads
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (set[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(pcg32_kernel<RPT, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) set[dev] = true;
  return e;
}

template <int RPT, bool C>
cudaError_t launch32(const PcgArgsT<float>& args, const Pcg32Work& work, int grid, cudaStream_t st) {
  const size_t smem = C ? sizeof(float4) * (kModes / 4) * RPT * NT : 0;
  PcgArgsT<float> a = args;
  Pcg32Work w = work;
  void* params[] = {(void*)&a, (void*)&w};
  return cudaLaunchCooperativeKernel((const void*)pcg32_kernel<RPT, C>, dim3(grid), dim3(NT), params, smem, st);
}
}  // namespace

// Launch shape: blocks <= one per SM, rows per thread a power of two <= 8.
bool pcg32_shape(int64_t n, int sms, int* grid, int* rpt) {
  int64_t nb = (n + 2 * NT - 1) / (2 * NT);
  if (nb > sms) nb = sms;
  if (nb > 32 * kMaxGridStrides) nb = 32 * kMaxGridStrides;
  if (nb < 1) nb = 1;
  int r = 1;
  while ((int64_t)nb * NT * r < n) r *= 2;
  if (r > 8) return false;
  *grid = (int)nb;
  *rpt = r;
  return true;
}


namespace {
template <int RPT>
constexpr size_t pipe_smem() {
  return 2 * sizeof(float4) * (kModes / 4) * RPT * NT;  // rows of Phi and of A Phi
}

template <int RPT>
cudaError_t prepare32p() {
  static bool set[64] = {false};
  static std::mutex mu;  // handles may be built from several threads
  std::lock_guard<std::mutex> lock(mu);
  if (pipe_smem<RPT>() <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (set[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(pcg32p_kernel<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pipe_smem<RPT>());
  if (e == cudaSuccess) set[dev] = true;
  return e;
}

template <int RPT>
cudaError_t launch32p(const PcgArgsT<float>& args, const Pcg32Work& work, int grid, cudaStream_t st) {
  PcgArgsT<float> a = args;
  Pcg32Work w = work;
  void* params[] = {(void*)&a, (void*)&w};
  return cudaLaunchCooperativeKernel((const void*)pcg32p_kernel<RPT>, dim3(grid), dim3(NT), params, pipe_smem<RPT>(),
                                     st);
}
}  // namespace

bool pcg32_pipe_ok(int rpt) { return rpt == 1 || rpt == 2 || rpt == 4; }

cudaError_t launch_pcg32_pipe(const PcgArgsT<float>& args, const Pcg32Work& work, int grid, int rpt, cudaStream_t st) {
  if (grid > 32 * kMaxGridStrides || !args.phi || !args.Einv || !work.aphi) return cudaErrorInvalidValue;
  switch (rpt) {
    case 1: return launch32p<1>(args, work, grid, st);
    case 2: return launch32p<2>(args, work, grid, st);
    case 4: return launch32p<4>(args, work, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_aphi32(int64_t n, const int32_t* rowptr, const int32_t* col, const float* val, const float* phi,
                          float* aphi, cudaStream_t st) {
  const int64_t tot = n * (kModes / 4);
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(1, (tot + 255) / 256), 4096);
  k_aphi32<<<grid, 256, 0, st>>>(n, rowptr, col, val, reinterpret_cast<const float4*>(phi),
                                 reinterpret_cast<float4*>(aphi));
  return cudaGetLastError();
}

cudaError_t prepare_pcg32() {
  cudaError_t e = prepare32<4, true>();
  if (e == cudaSuccess) e = prepare32<8, true>();
  if (e == cudaSuccess) e = prepare32p<2>();
  if (e == cudaSuccess) e = prepare32p<4>();
  return e;
}

cudaError_t launch_pcg32(const PcgArgsT<float>& args, const Pcg32Work& work, int grid, int rpt, cudaStream_t st) {
  if (grid > 32 * kMaxGridStrides) return cudaErrorInvalidValue;
  const bool c = args.phi && args.Einv;
  switch (rpt) {
    case 1: return c ? launch32<1, true>(args, work, grid, st) : launch32<1, false>(args, work, grid, st);
    case 2: return c ? launch32<2, true>(args, work, grid, st) : launch32<2, false>(args, work, grid, st);
    case 4: return c ? launch32<4, true>(args, work, grid, st) : launch32<4, false>(args, work, grid, st);
    case 8: return c ? launch32<8, true>(args, work, grid, st) : launch32<8, false>(args, work, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace emu
