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
// pcg32p_kernel below is the pipelined variant with one. Both run on the
// partitioned system of emu_cgpart.h when the handle has one, with the
// block-local Chebyshev polynomial (LocalPrec) in place of D^-1.
#include <cuda_runtime.h>

#include <mutex>

#include <algorithm>
#include <stdint.h>

#include "emu_internal.h"
#include "emu_pcg.h"

namespace emu {

namespace {

constexpr int NT = kPcg32Threads;  // threads per block
constexpr int NR = 3;    // right-hand sides (x, y, z)
constexpr int kGather = 16;  // entries of a matrix row gathered at once
constexpr int kGatherPart = 8;  // the same for the pruned, partitioned system
constexpr int kLocUnroll = 8;   // local-table entries of a row read at once
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

// The same product for the rows vr[k] of a partitioned system, GW entries
// gathered at once (the pruned rows of a tetrahedral grid hold about 7).
template <int RPT, int GW>
__device__ __forceinline__ void spmv_rows_v(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                            const float* __restrict__ val, const bool (&own)[RPT],
                                            const int64_t (&vr)[RPT], const float4* __restrict__ z,
                                            float (&y)[RPT][NR]) {
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    y[k][0] = y[k][1] = y[k][2] = 0.f;
    if (!own[k]) continue;
    const int64_t v = vr[k];
    const int32_t e0 = __ldg(rowptr + v), e1 = __ldg(rowptr + v + 1);
    const int cnt = e1 - e0;
    float4 z4[GW];
    float a4[GW];
#pragma unroll
    for (int t = 0; t < GW; ++t) {
      a4[t] = 0.f;
      z4[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (t < cnt) {
        a4[t] = __ldg(val + e0 + t);
        z4[t] = __ldcg(z + __ldg(col + e0 + t));
      }
    }
#pragma unroll
    for (int t = 0; t < GW; ++t) {
      y[k][0] += a4[t] * z4[t].x;
      y[k][1] += a4[t] * z4[t].y;
      y[k][2] += a4[t] * z4[t].z;
    }
    for (int32_t e = e0 + GW; e < e1; ++e) {
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

// The same, written as one float4 (3 columns and a zero) per mode.
__device__ __forceinline__ void coarse_solve4(const float* s_Einv, const float* s_rho, float4* s_cc4) {
  for (int e = threadIdx.x; e < kModes * NR; e += NT) {
    const int m = e / NR, j = e % NR;
    float acc = 0.f;
#pragma unroll
    for (int l = 0; l < kModes; ++l) acc += s_Einv[m * kModes + l] * s_rho[l * NR + j];
    reinterpret_cast<float*>(s_cc4)[4 * m + j] = acc;
  }
  if (threadIdx.x < kModes) reinterpret_cast<float*>(s_cc4)[4 * threadIdx.x + 3] = 0.f;
  __syncthreads();
}

// Block-local part P of the two-level preconditioner (emu_cgpart.h) on a
// partitioned system: P y = D^-1/2 x_k, x_k the Chebyshev iterate of degree
// k for A_b x = D^-1/2 y from x = 0, A_b the block's diagonal block of
// D^-1/2 A D^-1/2 held in shared memory as words of a 16-bit local column
// and a bfloat16 weight (D^-1 y when the degree is 1). Every thread of the
// block calls apply (it holds block barriers); the two product buffers
// alternate, so one barrier per product suffices.
template <int RPT>
struct LocalPrec {
  float4* buf;            // 2 RPT NT float4 of shared memory
  const uint32_t* table;  // RPT lw NT words of shared memory
  const float* c1;        // Chebyshev coefficients (shared)
  const float* c2;
  float c0;
  int lw;                 // 0: Jacobi only
  int degree;
  int pb;

  // t = O y on the block's rows, O the off-diagonal part of A_b
  __device__ __forceinline__ void off(const bool (&own)[RPT], const float (&y)[RPT][NR], float (&t)[RPT][NR]) {
    float4* b = buf + pb * (RPT * NT);
    pb ^= 1;
#pragma unroll
    for (int k = 0; k < RPT; ++k)
      b[k * NT + threadIdx.x] = own[k] ? make_float4(y[k][0], y[k][1], y[k][2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      float t0 = 0.f, t1 = 0.f, t2 = 0.f;
      const uint32_t* le = table + (size_t)k * lw * NT + threadIdx.x;
      // the first kLocUnroll entries at once (all loads in flight), the rest in a loop
      uint32_t wd[kLocUnroll];
#pragma unroll
      for (int e = 0; e < kLocUnroll; ++e) wd[e] = e < lw ? le[e * NT] : 0u;
      float4 yv[kLocUnroll];
#pragma unroll
      for (int e = 0; e < kLocUnroll; ++e) yv[e] = b[wd[e] & 0xFFFFu];
#pragma unroll
      for (int e = 0; e < kLocUnroll; ++e) {
        const float av = __uint_as_float(wd[e] & 0xFFFF0000u);
        t0 += av * yv[e].x;
        t1 += av * yv[e].y;
        t2 += av * yv[e].z;
      }
      for (int e = kLocUnroll; e < lw; ++e) {
        const uint32_t word = le[e * NT];
        const float av = __uint_as_float(word & 0xFFFF0000u);
        const float4 y4 = b[word & 0xFFFFu];
        t0 += av * y4.x;
        t1 += av * y4.y;
        t2 += av * y4.z;
      }
      t[k][0] = t0;
      t[k][1] = t1;
      t[k][2] = t2;
    }
  }

  // out = P y
  __device__ __forceinline__ void apply(const bool (&own)[RPT], const float (&di)[RPT], const float (&sd)[RPT],
                                        const float (&y)[RPT][NR], float (&out)[RPT][NR]) {
    if (lw == 0) {
#pragma unroll
      for (int k = 0; k < RPT; ++k)
#pragma unroll
        for (int j = 0; j < NR; ++j) out[k][j] = di[k] * y[k][j];
      return;
    }
    float xk[RPT][NR], dk[RPT][NR], res[RPT][NR], t[RPT][NR];
#pragma unroll
    for (int k = 0; k < RPT; ++k)
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        res[k][j] = sd[k] * y[k][j];
        xk[k][j] = dk[k][j] = c0 * res[k][j];
      }
    off(own, xk, t);
#pragma unroll
    for (int k = 0; k < RPT; ++k)
#pragma unroll
      for (int j = 0; j < NR; ++j) res[k][j] -= xk[k][j] + t[k][j];
    // one copy of the step in the code (a short kernel body stays in the instruction cache)
#pragma unroll 1
    for (int i = 1; i < degree; ++i) {
      const float a1 = c1[i], a2 = c2[i];
#pragma unroll
      for (int k = 0; k < RPT; ++k)
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          dk[k][j] = a1 * dk[k][j] + a2 * res[k][j];
          xk[k][j] += dk[k][j];
        }
      if (i + 1 < degree) {
        off(own, dk, t);
#pragma unroll
        for (int k = 0; k < RPT; ++k)
#pragma unroll
          for (int j = 0; j < NR; ++j) res[k][j] -= dk[k][j] + t[k][j];
      }
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k)
#pragma unroll
      for (int j = 0; j < NR; ++j) out[k][j] = sd[k] * xk[k][j];
  }
};

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
  __shared__ float s_c1[kChebMax], s_c2[kChebMax];  // Chebyshev coefficients
  // the coarse basis rows of this thread, float4 q of row k at
  // sPhi[(q * RPT + k) * NT + tid] (consecutive threads, consecutive 16 bytes);
  // then, on a partitioned system, two buffers of the local products and the local table
  extern __shared__ float4 sPhi[];
  float4* sBuf = sPhi + (COARSE ? (kModes / 4) * RPT * NT : 0);
  uint32_t* sLoc = reinterpret_cast<uint32_t*>(sBuf + 2 * RPT * NT);
  const bool parted = wk.off != nullptr;  // rows in the partition of emu_cgpart.h
  const int lw = (parted && wk.degree > 1) ? wk.lw : 0;
  const int32_t* __restrict__ perm = wk.perm;
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
  if (threadIdx.x < kChebMax) {
    s_c1[threadIdx.x] = wk.c1[threadIdx.x];
    s_c2[threadIdx.x] = wk.c2[threadIdx.x];
  }
  if (lw > 0) {
    const uint32_t* __restrict__ lsrc = wk.loc + (size_t)blockIdx.x * RPT * lw * NT;
    for (int e = threadIdx.x; e < RPT * lw * NT; e += NT) sLoc[e] = __ldg(lsrc + e);
  }

  float x[RPT][NR], r[RPT][NR], p[RPT][NR], s[RPT][NR], u[RPT][NR], w[RPT][NR];
  float di[RPT], sd[RPT];
  int64_t vr[RPT];
  bool own[RPT];
  const int64_t rbeg = parted ? wk.off[blockIdx.x] : 0, rend = parted ? wk.off[blockIdx.x + 1] : n;
  // row k of this thread and the vertex it stands for (b and x are in vertex order)
  auto vert = [&](int k) -> int64_t { return parted ? (int64_t)__ldg(perm + vr[k]) : vr[k]; };
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int64_t v = parted ? rbeg + k * NT + threadIdx.x : g0 + k * stride;
    vr[k] = v;
    own[k] = v < rend;
    di[k] = own[k] ? __ldg(a.dinv + v) : 0.f;
    sd[k] = sqrtf(di[k]);
    const int64_t o = own[k] ? vert(k) : 0;
#pragma unroll
    for (int j = 0; j < NR; ++j) x[k][j] = own[k] ? a.x[o * NR + j] : 0.f;
    if constexpr (COARSE) {
      const float4* ph = reinterpret_cast<const float4*>(a.phi + (own[k] ? v : 0) * kModes);
#pragma unroll
      for (int q = 0; q < kModes / 4; ++q)
        sPhi[(q * RPT + k) * NT + threadIdx.x] = own[k] ? __ldg(ph + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }

  auto spmv = [&](const float4* __restrict__ z, float (&y)[RPT][NR]) {
    spmv_rows_v<RPT, kGather>(rowptr, col, val, own, vr, z, y);
  };
  LocalPrec<RPT> lp{sBuf, sLoc, s_c1, s_c2, wk.c0, lw, wk.degree, 0};
  // u = P r + Phi cc (P: the block-local polynomial, D^-1 without one), stored
  // for the neighbours; every thread of the block calls it
  auto precond = [&]() {
    float ul[RPT][NR];
    if constexpr (RPT <= 4) {  // partitioned systems have at most 4 rows per thread
      lp.apply(own, di, sd, r, ul);
    } else {
#pragma unroll
      for (int k = 0; k < RPT; ++k)
#pragma unroll
        for (int j = 0; j < NR; ++j) ul[k][j] = di[k] * r[k][j];
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      if (!own[k]) continue;
      const int64_t v = vr[k];
#pragma unroll
      for (int j = 0; j < NR; ++j) u[k][j] = ul[k][j];
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
  for (int k = 0; k < RPT; ++k)
    if (own[k]) ugx[vr[k]] = make_float4(x[k][0], x[k][1], x[k][2], 0.f);
  if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
  spmv(ugx, w);
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int64_t o = own[k] ? vert(k) : 0;
#pragma unroll
    for (int j = 0; j < NR; ++j) r[k][j] = own[k] ? a.b[o * NR + j] - w[k][j] : 0.f;
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
      const int64_t o = vert(k);
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const float bv = a.b[o * NR + j];
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
      if (own[k]) {
        const int64_t o = vert(k);
#pragma unroll
        for (int j = 0; j < NR; ++j) a.x[o * NR + j] = x[k][j];
      }
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
// from its neighbours, v = P w (the local part of M w), is published with
// the partial sums of the same iteration. The coarse part of M w,
// Phi E^-1 Phi^T w, needs Phi^T w, a global sum; it is applied after the
// barrier through the precomputed rows of A Phi:
// n = A M w = A v + (A Phi) c with c = E^-1 Phi^T w.
// Exchange vectors and partial sums alternate between two buffers: a block
// may publish iteration i + 1 while a slower one still reads iteration i.
//
// The system is the partitioned one of emu_cgpart.h: block b owns the rows
// off[b] .. off[b + 1] - 1 (a spatially compact part of the mesh), thread t
// the rows off[b] + k NT + t. The local part of the preconditioner,
// P = D^-1/2 p(A_b) D^-1/2 with A_b the block's diagonal block of
// D^-1/2 A D^-1/2 and p the Chebyshev polynomial of the given degree, needs
// no exchange: its products run on the block's rows in shared memory.
// With the coarse space, M = P + Phi E^-1 Phi^T is a two-level additive
// Schwarz preconditioner (degree 1: P = D^-1, plain Jacobi).
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
  __shared__ float s_rho[NC];
  __shared__ float4 s_cc4[kModes];  // E^-1 rho, one float4 (3 columns) per mode
  __shared__ float s_Einv[kModes * kModes];
  __shared__ int s_flag;
  __shared__ float s_c1[kChebMax], s_c2[kChebMax];  // Chebyshev coefficients
  // rows of Phi, then rows of A Phi: float4 q of row k at [(q * RPT + k) * NT + tid];
  // then two buffers of the local products and the local table
  extern __shared__ float4 sPhi[];
  float4* sAPhi = sPhi + (kModes / 4) * RPT * NT;
  float4* sBuf = sAPhi + (kModes / 4) * RPT * NT;
  uint32_t* sLoc = reinterpret_cast<uint32_t*>(sBuf + 2 * RPT * NT);
  unsigned epoch = 0;
  const int G = gridDim.x;
  const int lw = wk.degree > 1 ? wk.lw : 0;
  const int64_t rbeg = wk.off[blockIdx.x], rend = wk.off[blockIdx.x + 1];
  const int32_t* __restrict__ rowptr = a.rowptr;
  const int32_t* __restrict__ col = a.col;
  const float* __restrict__ val = a.val;
  const int32_t* __restrict__ perm = wk.perm;
  for (int k = threadIdx.x; k < kModes * kModes; k += NT) s_Einv[k] = (float)a.Einv[k];
  if (threadIdx.x < kChebMax) {
    s_c1[threadIdx.x] = wk.c1[threadIdx.x];
    s_c2[threadIdx.x] = wk.c2[threadIdx.x];
  }
  {
    const uint32_t* __restrict__ lsrc = wk.loc + (size_t)blockIdx.x * RPT * lw * NT;
    for (int e = threadIdx.x; e < RPT * lw * NT; e += NT) sLoc[e] = __ldg(lsrc + e);
  }

  float x[RPT][NR], r[RPT][NR], u[RPT][NR], w[RPT][NR], p[RPT][NR], s[RPT][NR], qv[RPT][NR], z[RPT][NR];
  float di[RPT], sd[RPT];  // D^-1 and D^-1/2 of the rows
  int64_t vr[RPT];
  bool own[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int64_t v = rbeg + k * NT + threadIdx.x;
    vr[k] = v;
    own[k] = v < rend;
    di[k] = own[k] ? __ldg(a.dinv + v) : 0.f;
    sd[k] = sqrtf(di[k]);
    const float4* ph = reinterpret_cast<const float4*>(a.phi + (own[k] ? v : 0) * kModes);
    const float4* aph = reinterpret_cast<const float4*>(wk.aphi + (own[k] ? v : 0) * kModes);
#pragma unroll
    for (int q = 0; q < kModes / 4; ++q) {
      sPhi[(q * RPT + k) * NT + threadIdx.x] = own[k] ? __ldg(ph + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      sAPhi[(q * RPT + k) * NT + threadIdx.x] = own[k] ? __ldg(aph + q) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int64_t o = own[k] ? (int64_t)__ldg(perm + v) : 0;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      x[k][j] = own[k] ? a.x[o * NR + j] : 0.f;
      p[k][j] = s[k][j] = qv[k][j] = z[k][j] = 0.f;
    }
  }

  auto spmv = [&](const float4* __restrict__ zsrc, float (&y)[RPT][NR]) {
    spmv_rows_v<RPT, kGatherPart>(rowptr, col, val, own, vr, zsrc, y);
  };
  auto phi_t = [&](const float (&y)[RPT][NR], float* loc) { phi_t_rows<RPT>(sPhi, own, y, loc); };
  auto coarse_cc = [&]() { coarse_solve4(s_Einv, s_rho, s_cc4); };  // s_cc4 = E^-1 s_rho
  // o[j] = sum_m rows[v][m] cc[m][j] for row k (rows: sPhi or sAPhi)
  auto coarse3 = [&](const float4* rows, int k, float (&o)[NR]) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < kModes / 4; ++q) {
      const float4 ph = rows[(q * RPT + k) * NT + threadIdx.x];
      const float4 c0 = s_cc4[4 * q], c1 = s_cc4[4 * q + 1], c2 = s_cc4[4 * q + 2], c3 = s_cc4[4 * q + 3];
      acc.x += ph.x * c0.x + ph.y * c1.x + ph.z * c2.x + ph.w * c3.x;
      acc.y += ph.x * c0.y + ph.y * c1.y + ph.z * c2.y + ph.w * c3.y;
      acc.z += ph.x * c0.z + ph.y * c1.z + ph.z * c2.z + ph.w * c3.z;
    }
    o[0] = acc.x;
    o[1] = acc.y;
    o[2] = acc.z;
  };
  // out = P y, the block-local part of M (a Chebyshev polynomial of the block's diagonal block)
  LocalPrec<RPT> lp{sBuf, sLoc, s_c1, s_c2, wk.c0, lw, wk.degree, 0};
  auto local_apply = [&](const float (&y)[RPT][NR], float (&out)[RPT][NR]) { lp.apply(own, di, sd, y, out); };
  auto rhs = [&](int k, int j) {  // b of row k (vertex order on input)
    return a.b[(int64_t)__ldg(perm + vr[k]) * NR + j];
  };

  // ---- r = b - A x ------------------------------------------------------
#pragma unroll
  for (int k = 0; k < RPT; ++k)
    if (own[k]) wk.ug[vr[k]] = make_float4(x[k][0], x[k][1], x[k][2], 0.f);
  if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
  spmv(wk.ug, w);
#pragma unroll
  for (int k = 0; k < RPT; ++k)
#pragma unroll
    for (int j = 0; j < NR; ++j) r[k][j] = own[k] ? rhs(k, j) - w[k][j] : 0.f;
  {  // u = P r + Phi E^-1 Phi^T r, published in the second exchange buffer
    float loc[NV0];
#pragma unroll
    for (int k = 0; k < NV0; ++k) loc[k] = 0.f;
    phi_t(r, loc);
    block_sum_f<NV0>(loc, ssum, sm);
    for (int k = threadIdx.x; k < NC; k += NT) wk.part[(size_t)k * G + blockIdx.x] = ssum[k];
    float ul[RPT][NR];
    local_apply(r, ul);
    if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
    grid_sum_f<NV0>(wk.part, NC, ssum);
    for (int k = threadIdx.x; k < NC; k += NT) s_rho[k] = ssum[k];
    __syncthreads();
    coarse_cc();
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      float cm[NR];
      coarse3(sPhi, k, cm);
#pragma unroll
      for (int j = 0; j < NR; ++j) u[k][j] = own[k] ? ul[k][j] + cm[j] : 0.f;
      if (own[k]) wk.ug[a.n + vr[k]] = make_float4(u[k][0], u[k][1], u[k][2], 0.f);
    }
  }
  if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
  spmv(wk.ug + a.n, w);  // w = A u

  {
    int it = 0, buf = 0;
    bool first = true, all_done = false;
    for (;;) {
      float* __restrict__ pbuf = wk.part + (size_t)buf * PSTRIDE * G;
      float4* __restrict__ ub = wk.ug + (size_t)buf * a.n;
      float vl[RPT][NR];  // v = P w, published for the neighbours
      local_apply(w, vl);
      {  // partial sums of this iteration
        float loc[NV0];
#pragma unroll
        for (int k = 0; k < NV0; ++k) loc[k] = 0.f;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          if (!own[k]) continue;
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            loc[j] += r[k][j] * u[k][j];
            loc[NR + j] += w[k][j] * u[k][j];
            loc[2 * NR + j] += r[k][j] * r[k][j];
            if (first) {
              const float bv = rhs(k, j);
              loc[3 * NR + j] += bv * bv;
            }
          }
          ub[vr[k]] = make_float4(vl[k][0], vl[k][1], vl[k][2], 0.f);
        }
        phi_t(w, loc + 4 * NR);
        block_sum_f<NV0>(loc, ssum, sm);
        for (int k = threadIdx.x; k < NV0; k += NT) pbuf[(size_t)k * G + blockIdx.x] = ssum[k];
      }
      if (!gbar(wk, epoch, &s_flag, a.wait_ns)) goto timeout;
      grid_sum_f<NV0>(pbuf, NV0, ssum);
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
      spmv(ub, nv);  // A P w
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        float cm[NR], cn[NR];
        coarse3(sPhi, k, cm);
        coarse3(sAPhi, k, cn);
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          if (!s_act[j]) continue;
          const float be = s_be[j], al = s_al[j];
          const float mv = vl[k][j] + cm[j];  // m = M w
          const float nn = nv[k][j] + cn[j];  // n = A M w
          z[k][j] = nn + be * z[k][j];
          qv[k][j] = mv + be * qv[k][j];
          s[k][j] = w[k][j] + be * s[k][j];
          p[k][j] = u[k][j] + be * p[k][j];
          x[k][j] += al * p[k][j];
          r[k][j] -= al * s[k][j];
          u[k][j] -= al * qv[k][j];
          w[k][j] -= al * z[k][j];
        }
      }
      first = false;
      buf ^= 1;
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      if (own[k]) {
        const int64_t o = __ldg(perm + vr[k]);
#pragma unroll
        for (int j = 0; j < NR; ++j) a.x[o * NR + j] = x[k][j];
      }
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

// dst[r][:] = src[perm[r]][:], 16 floats per row (four float4)
__global__ void k_gather_rows16(int64_t n, const int32_t* __restrict__ perm, const float4* __restrict__ src,
                                float4* __restrict__ dst) {
  const int64_t tot = n * (kModes / 4);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / (kModes / 4);
    const int q = (int)(i % (kModes / 4));
    dst[i] = src[(int64_t)perm[r] * (kModes / 4) + q];
  }
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
// dynamic shared memory: the coarse rows (C), then on a partitioned system
// two buffers of the local products and a local table of lw words per row slot
template <int RPT, bool C>
constexpr size_t plain_smem(bool parted, int lw) {
  return (C ? sizeof(float4) * (kModes / 4) * RPT * NT : 0) +
         (parted ? 2 * sizeof(float4) * RPT * NT + sizeof(uint32_t) * (size_t)RPT * lw * NT : 0);
}

template <int RPT, bool C>
cudaError_t prepare32() {
  // above the default 48 KB the kernel needs the opt-in, a per-device attribute
  const size_t smem = plain_smem<RPT, C>(RPT <= 4, RPT <= 4 ? cg_local_width_max(RPT) : 0);
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
  const bool parted = work.off != nullptr;
  const int lw = (parted && work.degree > 1) ? work.lw : 0;
  if (parted && (RPT > 4 || !work.perm || lw > cg_local_width_max(RPT) || (lw > 0 && !work.loc) ||
                 work.degree < 1 || work.degree > kChebMax))
    return cudaErrorInvalidValue;
  const size_t smem = plain_smem<RPT, C>(parted, lw);
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
// rows of Phi and of A Phi, two buffers of the local products, the local table
template <int RPT>
constexpr size_t pipe_smem(int lw) {
  return 2 * sizeof(float4) * (kModes / 4) * RPT * NT + 2 * sizeof(float4) * RPT * NT +
         sizeof(uint32_t) * (size_t)RPT * lw * NT;
}

template <int RPT>
cudaError_t prepare32p() {
  static bool set[64] = {false};
  static std::mutex mu;  // handles may be built from several threads
  std::lock_guard<std::mutex> lock(mu);
  const size_t smem = pipe_smem<RPT>(cg_local_width_max(RPT));
  if (smem <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (set[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(pcg32p_kernel<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) set[dev] = true;
  return e;
}

template <int RPT>
cudaError_t launch32p(const PcgArgsT<float>& args, const Pcg32Work& work, int grid, cudaStream_t st) {
  PcgArgsT<float> a = args;
  Pcg32Work w = work;
  const int lw = w.degree > 1 ? w.lw : 0;
  if (lw > cg_local_width_max(RPT) || (w.degree > 1 && !w.loc)) return cudaErrorInvalidValue;
  void* params[] = {(void*)&a, (void*)&w};
  return cudaLaunchCooperativeKernel((const void*)pcg32p_kernel<RPT>, dim3(grid), dim3(NT), params, pipe_smem<RPT>(lw),
                                     st);
}
}  // namespace

bool pcg32_pipe_ok(int rpt) { return rpt == 1 || rpt == 2 || rpt == 4; }

cudaError_t launch_pcg32_pipe(const PcgArgsT<float>& args, const Pcg32Work& work, int grid, int rpt, cudaStream_t st) {
  if (grid > 32 * kMaxGridStrides || !args.phi || !args.Einv || !work.aphi || !work.perm || !work.off ||
      work.degree < 1 || work.degree > kChebMax)
    return cudaErrorInvalidValue;
  switch (rpt) {
    case 1: return launch32p<1>(args, work, grid, st);
    case 2: return launch32p<2>(args, work, grid, st);
    case 4: return launch32p<4>(args, work, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gather_rows16(int64_t n, const int32_t* perm, const float* src, float* dst, cudaStream_t st) {
  const int64_t tot = n * (kModes / 4);
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(1, (tot + 255) / 256), 4096);
  k_gather_rows16<<<grid, 256, 0, st>>>(n, perm, reinterpret_cast<const float4*>(src), reinterpret_cast<float4*>(dst));
  return cudaGetLastError();
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
  cudaError_t e = prepare32<1, true>();
  if (e == cudaSuccess) e = prepare32<1, false>();
  if (e == cudaSuccess) e = prepare32<2, true>();
  if (e == cudaSuccess) e = prepare32<2, false>();
  if (e == cudaSuccess) e = prepare32<4, true>();
  if (e == cudaSuccess) e = prepare32<4, false>();
  if (e == cudaSuccess) e = prepare32<8, true>();
  if (e == cudaSuccess) e = prepare32p<1>();
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
