// Mixed-precision kernels: per-tet work in FP32 on a (unit quaternion,
// E = S - I) state, every global sum and the positions in FP64.
//
// Precision rules (they decide which expressions are used):
//   * the residual terms V R Pr and alpha w (R S - G q) are formed from
//     difference-free expressions in E (S - S^-1 = (2E + E^2) S^-1,
//     ln J = log1p(tr E + e2(E) + det E)), so a stiff element with tiny strain
//     keeps the relative precision of its stress;
//   * the line-search energy change V [Psi(F + s d) - Psi(F)] is written
//     term by term without the O(|d|) cancellation of mu <F, d> - mu tr(F^-1 d);
//   * the polar update works on I + Y with the rotation kept as a quaternion
//     and R - I written without cancellation.
#include <cuda_runtime.h>

#include <mutex>
#include <math.h>
#include <stdint.h>

#include "emu_kernels.cuh"
#include "emu_math.cuh"
#include "emu_mixed.cuh"
#include "emu_reduce.cuh"

namespace emu {

__device__ __forceinline__ void load9f(const float* __restrict__ a, int64_t m, int64_t i, float* D) {
#pragma unroll
  for (int k = 0; k < 9; ++k) D[k] = a[k * m + i];
}

__device__ __forceinline__ ElemMat<float> load_mat_f(const MixArgs& a, int64_t i) {
  ElemMat<float> e;
  e.V = a.V[i];
  e.mu = a.mu[i];
  e.lam = a.lam[i];
  e.ka = a.ka[i];
  e.u[0] = a.u[i];
  e.u[1] = a.u[a.m + i];
  e.u[2] = a.u[2 * a.m + i];
  return e;
}

// A - I = G_i (q - Q) + (G_i Q - I). The displacement edges come from the
// float pair uh + ul = q - Q: (uh_k - uh_3) is rounded relative to the edge
// itself (not to the displacement), and (ul_k - ul_3) restores the part the
// FP32 rounding of the displacement dropped, so A - I keeps the relative
// precision the FP64 difference gave, with FP32 arithmetic only.
__device__ __forceinline__ void defgrad_disp(const float* __restrict__ uh, const float* __restrict__ ul, int4 t,
                                             const float* D, const float* __restrict__ E0, int64_t m, int64_t i,
                                             float* AmI) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float h3 = uh[3 * (int64_t)t.w + r], l3 = ul[3 * (int64_t)t.w + r];
    const float e0 = (uh[3 * (int64_t)t.x + r] - h3) + (ul[3 * (int64_t)t.x + r] - l3);
    const float e1 = (uh[3 * (int64_t)t.y + r] - h3) + (ul[3 * (int64_t)t.y + r] - l3);
    const float e2 = (uh[3 * (int64_t)t.z + r] - h3) + (ul[3 * (int64_t)t.z + r] - l3);
#pragma unroll
    for (int c = 0; c < 3; ++c) AmI[3 * r + c] = e0 * D[c] + e1 * D[3 + c] + e2 * D[6 + c] + E0[(3 * r + c) * m + i];
  }
}

// Mismatch D = G_i q - R S = (A - I) - (R - I) - R E, every term small.
__device__ __forceinline__ void mismatch(const MixArgs& a, int4 t, const float* Dm, int64_t i, const float4 qq,
                                         const float* RE, float* Dk) {
  float AmI[9], RmI[9];
  defgrad_disp(a.uh, a.ul, t, Dm, a.E0, a.m, i, AmI);
  quat_rot_minus_I(qq.x, qq.y, qq.z, qq.w, RmI);
#pragma unroll
  for (int k = 0; k < 9; ++k) Dk[k] = (AmI[k] - RmI[k]) - RE[k];
}

__device__ __forceinline__ void defgrad_ff(const float* __restrict__ q, int4 t, const float* D, float* A) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float q3 = q[3 * (int64_t)t.w + r];
    const float e0 = q[3 * (int64_t)t.x + r] - q3;
    const float e1 = q[3 * (int64_t)t.y + r] - q3;
    const float e2 = q[3 * (int64_t)t.z + r] - q3;
#pragma unroll
    for (int c = 0; c < 3; ++c) A[3 * r + c] = e0 * D[c] + e1 * D[3 + c] + e2 * D[6 + c];
  }
}

__device__ __forceinline__ void load_state(const MixArgs& a, int64_t i, float* R, float* e6) {
  const float4 qq = a.quat[i];
  quat_to_R(qq.x, qq.y, qq.z, qq.w, R);
#pragma unroll
  for (int k = 0; k < 6; ++k) e6[k] = a.E[k * a.m + i];
}

template <typename TO, typename TX>
__device__ __forceinline__ void corners_f(TO* __restrict__ contrib, int64_t i, float w, const TX* X, const float* D) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  TO* out = contrib + 12 * i;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float v[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) v[r] = w * (X[3 * r] * D[3 * k] + X[3 * r + 1] * D[3 * k + 1] + X[3 * r + 2] * D[3 * k + 2]);
    out[3 * k] = v[0];
    out[3 * k + 1] = v[1];
    out[3 * k + 2] = v[2];
    s0 += v[0];
    s1 += v[1];
    s2 += v[2];
  }
  out[9] = -s0;
  out[10] = -s1;
  out[11] = -s2;
}

// ------------------------------------------------------------ gradient ----
__global__ void __launch_bounds__(128, 4) k_grad_m(MixArgs a) {
  const int64_t m = a.m;
  // per-thread sums in FP32 (a few tets each), FP64 from the block sum on:
  // GB300's FP64 pipe issues far below its FP32 rate, and per-tet FP64
  // conversions and adds bound these kernels (measured on the line search)
  float accf = 0.f;
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    // tets of bones are no variables of their own (their g, y, U stay zero)
    if (a.tkind && a.tkind[i] != kTetDeformable) continue;
    const int4 t = a.tet[i];
    float D[9], R[9], e6[6];
    load9f(a.Dinv, m, i, D);
    load_state(a, i, R, e6);
    StretchE st;
    if (!stretch_from_E(e6, st)) bad = 1;
    const ElemMat<float> mat = load_mat_f(a, i);
    const float c = a.c[i];
    float Pr[9], RP[9], Em[9], RE[9], Dk[9];
    piola_rotated_E(st, mat, Pr);
    matmul3(R, Pr, RP);
    sym_from_s(e6, Em);
    matmul3(R, Em, RE);
    mismatch(a, t, D, i, a.quat[i], RE, Dk);
    float g[9];
    float gg = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      g[k] = mat.V * RP[k] - c * Dk[k];
      if (a.nu) g[k] -= a.nu[k * m + i];  // external force (Sec. 3.4)
      gg = fmaf(g[k], g[k], gg);
      a.g[k * m + i] = g[k];
    }
    if (!isfinite(gg)) bad = 1;
    accf += gg;
    float M6[36], U[54];
    stretch_hessian(st.Sinv, st.lnJ, mat, M6);
    bool ok = true;
    chart_factor(R, st.S, M6, c, U, ok);
    if (!ok) bad = 1;
    apply_I_minus_N(U, g);
    const float ic = 1.f / c;
#pragma unroll
    for (int k = 0; k < 9; ++k) a.y[k * m + i] = g[k] * ic;
#pragma unroll
    for (int k = 0; k < 54; ++k) a.Uw[k * m + i] = U[k];
  }
  double acc[1] = {(double)accf};
  block_reduce_write<1>(acc, a.partials + blockIdx.x);
  if (bad) atomicExch(&a.sc->nonfinite, 1);
  // the last block to finish sums the squared gradient norm
  if (last_block(&a.sc->ticket[kTicketGrad])) {
    __shared__ double tot[1];
    block_sum_partials<1>(a.partials, gridDim.x, tot);
    if (threadIdx.x == 0) {
      a.sc->gnorm2 = tot[0];
      a.sc->ticket[kTicketGrad] = 0u;
    }
  }
}

void launch_grad_mixed(const MixArgs& a, int grid, cudaStream_t st) { k_grad_m<<<grid, 128, 0, st>>>(a); }

// ------------------------------------------------------------ capacitance --
// C = sum_i Yh_i^T Yh_i with Yh_i = sqrt(w_i) U_i (G_i Phi^T) (6 x 48 per
// tet; the Gram form of Eq. 12's capacitance, see emu_math.cuh) and the
// Woodbury right-hand side B y = sum_i w_i (G_i Phi^T)^T y_i.
// The contraction C += Yh^T Yh runs on TF32 tensor
// cores (mma.sync m16n8k8, FP32 accumulate). Yh is rounded to TF32 once,
// before the product, so C is still the exact Gram matrix of the rounded
// rows and stays positive semi-definite.
//
// The kernel streams U, gamma, y and w (about 450 bytes per tet) and is
// meant to run at HBM speed, so the loads are decoupled from the math: the
// raw inputs of the next 32-tet chunk are copied into shared memory with
// cp.async while the current chunk is formed and multiplied (two buffers).
// Each warp owns a contiguous K-range of every chunk and the 12 output tiles
// (16 x 8) that touch the upper triangle; the warps' tiles are summed in
// shared memory and the lower triangle mirrored at the end.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async4(uint32_t saddr, const float* g, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(saddr), "l"(g), "r"(ok ? 4 : 0) : "memory");
}
// 16-byte copy of which the first ``bytes`` (0, 4, 8, 12 or 16) come from
// global memory and the rest is zero-filled
__device__ __forceinline__ void cp_async16(uint32_t saddr, const float* g, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(g), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

constexpr int kTcCH = 40;              // tets per chunk: 240 staging threads of 256
constexpr int kTcKR = 256;             // rows of Yh per chunk (240 + 16 zero rows): 32 k-steps of 8, 4 per warp
constexpr int kTcKS = kTcKR / 64;      // k-steps per warp
constexpr int kTcSegs = kTcCH / 4;     // 16-byte segments of a raw row
constexpr int kTcLD = kK + 4;          // padded row of Yh (TF32 bits)
constexpr int kTcRawRows = 54 + 48 + 9 + 1;  // U, gamma, y, w of a chunk
constexpr int kTcRL = kTcCH + 8;             // padded raw row (16-byte rows, conflict-free reads)
constexpr size_t kTcYBytes = sizeof(uint32_t) * kTcKR * kTcLD;
constexpr size_t kTcRawBytes = sizeof(float) * kTcRawRows * kTcRL;
constexpr size_t kTcSmem = kTcYBytes + 2 * kTcRawBytes;

template <bool VEC>
__global__ void __launch_bounds__(256, kTcBlocksPerSM) k_syrk_tc(MixArgs a, double* __restrict__ cpart) {
  constexpr int CH = kTcCH, LD = kTcLD, RL = kTcRL;
  __shared__ const float* s_src[kTcRawRows];  // first element of each raw row
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t* sY = reinterpret_cast<uint32_t*>(smem_raw);
  float* sRaw = reinterpret_cast<float*>(smem_raw + kTcYBytes);
  float* sC = reinterpret_cast<float*>(sY);  // reused for the final sum of the warps' tiles
  float* sBy = sC + kK * kK;                  // and for the final sum of B y
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int64_t m = a.m;
  const int64_t nch = (m + CH - 1) / CH;
  if (tid < kTcRawRows) {
    const int row = tid;
    s_src[row] = row < 54 ? a.Uw + (int64_t)row * m
                 : row < 102 ? a.gam + (int64_t)(row - 54) * m
                 : row < 111 ? a.y + (int64_t)(row - 102) * m
                             : a.w;
  }
  __syncthreads();

  // cp.async of one chunk's raw rows. VEC (rows 16-byte aligned, m % 4 == 0):
  // CH / 4 copies of 16 bytes per row; otherwise CH copies of 4 bytes.
  auto issue = [&](int64_t ch, int buf) {
    const int64_t base = ch * CH;
    float* dst = sRaw + buf * (kTcRawRows * RL);
    if constexpr (VEC) {
      for (int e = tid; e < kTcRawRows * kTcSegs; e += 256) {
        const int row = e / kTcSegs, seg = e % kTcSegs;
        const int64_t i = base + 4 * seg;
        const int64_t left = m - i;
        const int bytes = left >= 4 ? 16 : left > 0 ? 4 * (int)left : 0;
        const float* src = s_src[row] + (bytes > 0 ? i : 0);
        cp_async16((uint32_t)__cvta_generic_to_shared(dst + row * RL + 4 * seg), src, bytes);
      }
    } else {
      for (int e = tid; e < kTcRawRows * CH; e += 256) {
        const int row = e / CH, tt = e % CH;
        const int64_t i = base + tt;
        const bool ok = i < m;
        cp_async4((uint32_t)__cvta_generic_to_shared(dst + row * RL + tt), s_src[row] + (ok ? i : 0), ok);
      }
    }
  };

  // staging role: threads 0..6 CH - 1 own (tet slot stt = tid / 6, row k = tid % 6);
  // rows 6 CH .. kTcKR - 1 of Yh stay zero
  const int stt = tid / 6, sk = tid % 6;
  for (int e = 6 * CH * LD + tid; e < kTcKR * LD; e += 256) sY[e] = 0u;
  float acc[12][4];
#pragma unroll
  for (int t = 0; t < 12; ++t)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[t][c] = 0.f;
  // B y entries 8 sk .. 8 sk + 7 (r = sk / 2, j = 8 (sk % 2) + t) of the
  // staging thread's tet slot, summed over the block's chunks
  float by8[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) by8[t] = 0.f;
  const int br = sk >> 1, bh = sk & 1;

  if (blockIdx.x < nch) issue(blockIdx.x, 0);
  cp_async_commit();
  int it = 0;
  for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x, ++it) {
    const int64_t nxt = ch + gridDim.x;
    if (nxt < nch) issue(nxt, (it + 1) & 1);
    cp_async_commit();
    cp_async_wait1();  // this thread's copies of chunk ch have landed
    __syncthreads();   // and everyone else's
    if (tid < 6 * CH) {
      // Yh[tt*6 + k][16 r + j] = sqrt(w) sum_b U[k][3r+b] gam_j[b]
      const float* raw = sRaw + (it & 1) * (kTcRawRows * RL) + stt;
      const float wi = raw[111 * RL];
      const float sw = sqrtf(wi);
      float u9[9];  // sqrt(w) U[k][:]
#pragma unroll
      for (int c = 0; c < 9; ++c) u9[c] = sw * raw[(9 * sk + c) * RL];
      const float y0 = wi * raw[(102 + 3 * br) * RL];
      const float y1 = wi * raw[(102 + 3 * br + 1) * RL];
      const float y2 = wi * raw[(102 + 3 * br + 2) * RL];
      uint32_t* row = sY + (stt * 6 + sk) * LD;  // 16-byte aligned (LD = 52)
#pragma unroll
      for (int jq = 0; jq < 4; ++jq) {  // four j at a time: 16-byte stores
        uint32_t v[3][4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int j = 4 * jq + t;
          const float g0 = raw[(54 + 3 * j) * RL];
          const float g1 = raw[(54 + 3 * j + 1) * RL];
          const float g2 = raw[(54 + 3 * j + 2) * RL];
#pragma unroll
          for (int r = 0; r < 3; ++r) v[r][t] = to_tf32(u9[3 * r] * g0 + u9[3 * r + 1] * g1 + u9[3 * r + 2] * g2);
          const float byj = y0 * g0 + y1 * g1 + y2 * g2;
          by8[j & 7] += ((j >> 3) == bh) ? byj : 0.f;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
          *reinterpret_cast<uint4*>(row + 16 * r + 4 * jq) = make_uint4(v[r][0], v[r][1], v[r][2], v[r][3]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kTcKS; ++ks) {
      const int k0 = (warp * kTcKS + ks) * 8;
      uint32_t af[3][4], bf[6][2];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int m0 = 16 * i;
        af[i][0] = sY[(k0 + tig) * LD + m0 + gid];
        af[i][1] = sY[(k0 + tig) * LD + m0 + gid + 8];
        af[i][2] = sY[(k0 + tig + 4) * LD + m0 + gid];
        af[i][3] = sY[(k0 + tig + 4) * LD + m0 + gid + 8];
      }
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const int n0 = 8 * j;
        bf[j][0] = sY[(k0 + tig) * LD + n0 + gid];
        bf[j][1] = sY[(k0 + tig + 4) * LD + n0 + gid];
      }
      int t = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 2 * i; j < 6; ++j) mma_tf32(acc[t++], af[i], bf[j]);
    }
    __syncthreads();
  }
  // sum the warps' tiles in shared memory (warp order fixed)
  for (int e = tid; e < kK * kK; e += 256) sC[e] = 0.f;
  __syncthreads();
  for (int w = 0; w < 8; ++w) {
    if (warp == w) {
      int t = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 2 * i; j < 6; ++j, ++t) {
          const int r0 = 16 * i + gid, c0 = 8 * j + 2 * tig;
          sC[r0 * kK + c0] += acc[t][0];
          sC[r0 * kK + c0 + 1] += acc[t][1];
          sC[(r0 + 8) * kK + c0] += acc[t][2];
          sC[(r0 + 8) * kK + c0 + 1] += acc[t][3];
        }
    }
    __syncthreads();
  }
  if (tid < 6 * CH)
#pragma unroll
    for (int t = 0; t < 8; ++t) sBy[stt * kK + 8 * sk + t] = by8[t];
  __syncthreads();
  const size_t nb = gridDim.x;
  for (int e = tid; e < kK * kK; e += 256) {
    const int r = e / kK, c = e % kK;
    const bool computed = (c >> 3) >= 2 * (r >> 4);  // tile (r / 16, c / 8) was multiplied
    cpart[(size_t)e * nb + blockIdx.x] = (double)(computed ? sC[e] : sC[c * kK + r]);
  }
  if (tid < kK) {
    double by = 0.0;
    for (int tt = 0; tt < CH; ++tt) by += (double)sBy[tt * kK + tid];
    cpart[(size_t)(kCapEntries + tid) * nb + blockIdx.x] = by;
  }
}

// Opts the TC SYRK into its dynamic shared memory on the current device
// (once per device; call outside stream capture).
cudaError_t prepare_syrk_tc() {
  static bool attr_set[64] = {false};
  static std::mutex mu;  // handles may be built from several threads
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (attr_set[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(k_syrk_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_syrk_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e == cudaSuccess) attr_set[dev] = true;
  return e;
}

void launch_syrk_tc(const MixArgs& a, int grid, double* cpart, cudaStream_t st) {
  if (a.m % 4 == 0)
    k_syrk_tc<true><<<grid, 256, kTcSmem, st>>>(a, cpart);
  else
    k_syrk_tc<false><<<grid, 256, kTcSmem, st>>>(a, cpart);
}

// ------------------------------------------------------------ direction ---
// U is read twice (t = U v, then v - U^T t) instead of being held in 54
// registers, so more tets are in flight per SM; the second pass is served
// mostly by L1.
__global__ void __launch_bounds__(128, 8) k_dir_m(MixArgs a) {
  __shared__ float sz[kK];
  if (threadIdx.x < kK) sz[threadIdx.x] = (float)a.z[threadIdx.x];
  __syncthreads();
  const int64_t m = a.m;
  float accf = 0.f;  // per-thread g . d in FP32, FP64 from the block sum on
  const float* __restrict__ Uw = a.Uw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (a.tkind) {
      const int32_t kind = a.tkind[i];
      if (kind != kTetDeformable) {
        // a free bone's tet takes the bone's direction, a pinned bone's tet
        // none; their g . d is the bone's (summed by the bone kernel)
        float dv[9], D[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          dv[k] = kind >= 0 ? (float)a.bone_st[(size_t)kind * kBoneStride + kBoneD + k] : 0.f;
          a.d[k * m + i] = dv[k];
        }
        load9f(a.Dinv, m, i, D);
        corners_f(a.contrib32, i, a.w[i], dv, D);
        continue;
      }
    }
    float v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float g0 = __ldg(a.gam + (3 * j) * m + i), g1 = __ldg(a.gam + (3 * j + 1) * m + i),
                  g2 = __ldg(a.gam + (3 * j + 2) * m + i);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float zr = sz[16 * r + j];
        v[3 * r] += zr * g0;
        v[3 * r + 1] += zr * g1;
        v[3 * r + 2] += zr * g2;
      }
    }
    // (I - N) v with N = U^T U
    float t[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float acc_k = 0.f;
#pragma unroll
      for (int c = 0; c < 9; ++c) acc_k += __ldg(Uw + (9 * k + c) * m + i) * v[c];
      t[k] = acc_k;
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      float acc_c = 0.f;
#pragma unroll
      for (int k = 0; k < 6; ++k) acc_c += __ldg(Uw + (9 * k + c) * m + i) * t[k];
      v[c] -= acc_c;
    }
    float dv[9];
    float gtd = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      dv[k] = -(a.y[k * m + i] + v[k]);
      a.d[k * m + i] = dv[k];
      gtd = fmaf(a.g[k * m + i], dv[k], gtd);
    }
    accf += gtd;
    float D[9];
    load9f(a.Dinv, m, i, D);
    corners_f(a.contrib32, i, a.w[i], dv, D);
  }
  double acc[1] = {(double)accf};
  block_reduce_write<1>(acc, a.partials + blockIdx.x);
}

void launch_dir_mixed(const MixArgs& a, int grid, cudaStream_t st) { k_dir_m<<<grid, 128, 0, st>>>(a); }

// ------------------------------------------------------------ line search --
// V [Psi(F + s d) - Psi(F)] with M = F^-1 d = S^-1 R^T d and
// x = s tr M + s^2 e2(M) + s^3 det M (= det(I + sM) - 1):
//   mu [ s <F - F^-T, d> + s^2 |d|^2 / 2 - s^2 e2 - s^3 det M + (x - log1p x) ]
//   + lam/2 log1p(x) (2 ln J + log1p(x)) + ka (2 s (Fu).(du) + s^2 |du|^2),
// with F - F^-T = R (2E + E^2) S^-1; plus the ACAP coefficients.
__global__ void __launch_bounds__(128) k_ls_m(MixArgs a, LsSelect sel) {
  const float rho = (float)sel.rho;
  const int64_t m = a.m;
  const float s0 = (float)a.sc->sigma_start;
  // per-thread sums in FP32 (a few tets each), FP64 from the block sum on
  float accf[kLsNV];
#pragma unroll
  for (int k = 0; k < kLsNV; ++k) accf[k] = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    // free bones' tets: their terms come from the FP64 bone kernel (a stiff
    // bone's energy change is beyond FP32); pinned bones' tets contribute 0
    if (a.tkind && a.tkind[i] != kTetDeformable) continue;
    const int4 t = a.tet[i];
    float D[9], R[9], e6[6], dA[9], d[9];
    load9f(a.Dinv, m, i, D);
    load_state(a, i, R, e6);
    load9f(a.d, m, i, d);
    StretchE st;
    stretch_from_E(e6, st);
    defgrad_ff(a.dq, t, D, dA);
    const float c = a.c[i];
    float Em[9], RE[9], Dm[9];
    sym_from_s(e6, Em);
    matmul3(R, Em, RE);
    mismatch(a, t, D, i, a.quat[i], RE, Dm);  // G q - R S
    float cDd = 0.f, cdd = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float dDk = dA[k] - d[k];
      cDd += Dm[k] * dDk;
      cdd += dDk * dDk;
    }
    accf[kLsTrials] += c * cDd;
    accf[kLsTrials + 1] += c * cdd;
    const ElemMat<float> md = load_mat_f(a, i);
    float Rtd[9], M[9], F[9];
    matTmul3(R, d, Rtd);
    matmul3(st.Sinv, Rtd, M);
    matmul3(R, st.S, F);
    const float trM = M[0] + M[4] + M[8];
    const float e2 = inv2(M);
    const float detM = det3(M);
    float FFd = 0.f, dd = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      FFd += st.SmSi[k] * Rtd[k];  // <(S - S^-1), R^T d> = <F - F^-T, d>
      dd += d[k] * d[k];
    }
    float Fu[3], du[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      Fu[r] = F[3 * r] * md.u[0] + F[3 * r + 1] * md.u[1] + F[3 * r + 2] * md.u[2];
      du[r] = d[3 * r] * md.u[0] + d[3 * r + 1] * md.u[1] + d[3 * r + 2] * md.u[2];
    }
    const float Fudu = Fu[0] * du[0] + Fu[1] * du[1] + Fu[2] * du[2];
    const float dudu = du[0] * du[0] + du[1] * du[1] + du[2] * du[2];
    float dnu = 0.f;  // <d, nu>: the external work's change is -sigma <d, nu>
    if (a.nu)
#pragma unroll
      for (int k = 0; k < 9; ++k) dnu += d[k] * a.nu[k * m + i];
    float sig = s0;
#pragma unroll
    for (int j = 0; j < kLsTrials; ++j) {
      const float x = sig * trM + sig * sig * e2 + sig * sig * sig * detM;
      float dpsi;
      if (x > -1.f) {
        const float dl = log1pf(x);
        const float nh = md.mu * (sig * FFd + 0.5f * sig * sig * dd - sig * sig * e2 - sig * sig * sig * detM +
                                  x_minus_log1p(x));
        const float vol = 0.5f * md.lam * dl * (2.f * st.lnJ + dl);
        const float fib = md.ka * (2.f * sig * Fudu + sig * sig * dudu);
        dpsi = md.V * (nh + vol + fib) - sig * dnu;
      } else {
        dpsi = INFINITY;  // an inverted trial: never accepted
      }
      accf[j] += dpsi;
      sig *= rho;
    }
  }
  double acc[kLsNV];
#pragma unroll
  for (int k = 0; k < kLsNV; ++k) acc[k] = (double)accf[k];
  block_reduce_write<kLsNV>(acc, a.partials + (size_t)blockIdx.x * kLsNV);
  // the last block to finish sums every block's partials and selects the step
  if (last_block(&a.sc->ticket[kTicketLs])) {
    ls_select_block(sel.dir_partials, sel.nblk_dir, a.partials, gridDim.x + sel.nblk_extra, a.sc, sel.sigma0, sel.rho,
                    sel.c_armijo);
    if (threadIdx.x == 0) a.sc->ticket[kTicketLs] = 0u;
  }
}

void launch_ls_mixed(const MixArgs& a, int grid, const LsSelect& sel, cudaStream_t st) {
  k_ls_m<<<grid, 128, 0, st>>>(a, sel);
}

// ------------------------------------------------------------ update ------
// F' = R (S + s R^T d) = R (I + Y), Y = E + s R^T d; I + Y = Rx (I + E'):
// q' = q Rx, E' from the near-identity polar factor.
__global__ void __launch_bounds__(128) k_update_m(MixArgs a) {
  const double sigd = a.sc->sigma;
  if (sigd == 0.0) return;
  const float sig = (float)sigd;
  const int64_t m = a.m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (a.tkind && a.tkind[i] != kTetDeformable) continue;  // bones: FP64 state of their own
    float R[9], e6[6], d[9], Rtd[9], Y[9];
    load_state(a, i, R, e6);
    load9f(a.d, m, i, d);
    matTmul3(R, d, Rtd);
    sym_from_s(e6, Y);
#pragma unroll
    for (int k = 0; k < 9; ++k) Y[k] += sig * Rtd[k];
    Quat qx;
    float en[6];
    polar_near_identity(Y, qx, en, 12);
    const float4 q0 = a.quat[i];
    const Quat qn = qnormalize(qmul(Quat{q0.x, q0.y, q0.z, q0.w}, qx));
    a.quat[i] = make_float4(qn.x, qn.y, qn.z, qn.w);
#pragma unroll
    for (int k = 0; k < 6; ++k) a.E[k * m + i] = en[k];
  }
}

void launch_update_mixed(const MixArgs& a, int grid, cudaStream_t st) { k_update_m<<<grid, 128, 0, st>>>(a); }

__global__ void __launch_bounds__(256) k_update_verts_f(int64_t n3, const DevScalars* sc, const float* dq, double* q) {
  const double sig = sc->sigma;
  if (sig == 0.0) return;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x)
    q[k] += sig * (double)dq[k];
}

__global__ void __launch_bounds__(256) k_split_disp(int64_t n3, const double* __restrict__ q, const double* __restrict__ Q,
                                                    float* __restrict__ uh, float* __restrict__ ul) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x) {
    const double u = q[k] - Q[k];
    const float hi = (float)u;
    uh[k] = hi;
    ul[k] = (float)(u - (double)hi);
  }
}

void launch_split_disp(int64_t n, const double* q, const double* Q, float* uh, float* ul, cudaStream_t st) {
  const int64_t n3 = 3 * n;
  int grid = (int)((n3 + 255) / 256);
  if (grid < 1) grid = 1;
  k_split_disp<<<grid, 256, 0, st>>>(n3, q, Q, uh, ul);
}

void launch_update_verts_f(int64_t n, const DevScalars* sc, const float* dq, double* q, cudaStream_t st) {
  const int64_t n3 = 3 * n;
  int grid = (int)((n3 + 255) / 256);
  if (grid < 1) grid = 1;
  k_update_verts_f<<<grid, 256, 0, st>>>(n3, sc, dq, q);
}

// ------------------------------------------------------- coupling RHS ----
// FP64 corner terms of G^T W (R S) for the exact coupling solve: the FP32
// state values are exact in FP64, R is rebuilt from the normalised
// quaternion in FP64.
__global__ void __launch_bounds__(256) k_rhs_state_m(MixArgs a) {
  const int64_t m = a.m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t kind = a.tkind ? a.tkind[i] : kTetDeformable;
    double R[9], e6[6], S[9], F[9];
    if (kind >= 0) {  // a free bone's tet: the bone's FP64 state
      const double* o = a.bone_st + (size_t)kind * kBoneStride;
#pragma unroll
      for (int k = 0; k < 9; ++k) R[k] = o[kBoneR + k];
#pragma unroll
      for (int k = 0; k < 6; ++k) e6[k] = o[kBoneS + k];
      sym_from_s(e6, S);
    } else if (kind == kTetPinnedBone) {
#pragma unroll
      for (int k = 0; k < 9; ++k) R[k] = S[k] = (k % 4 == 0) ? 1.0 : 0.0;
    } else {
      const float4 qq = a.quat[i];
      double qx = qq.x, qy = qq.y, qz = qq.z, qw = qq.w;
      const double nn = 1.0 / sqrt(qx * qx + qy * qy + qz * qz + qw * qw);
      qx *= nn;
      qy *= nn;
      qz *= nn;
      qw *= nn;
      quat_to_R(qx, qy, qz, qw, R);
#pragma unroll
      for (int k = 0; k < 6; ++k) e6[k] = (double)a.E[k * m + i];
      sym_from_s(e6, S);
      S[0] += 1.0;
      S[4] += 1.0;
      S[8] += 1.0;
    }
    matmul3(R, S, F);
    double D[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) D[k] = (double)a.Dinv[k * m + i];
    const double w = (double)a.w[i];
    double s0 = 0, s1 = 0, s2 = 0;
    double* out = a.contrib + 12 * i;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double v[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) v[r] = w * (F[3 * r] * D[3 * k] + F[3 * r + 1] * D[3 * k + 1] + F[3 * r + 2] * D[3 * k + 2]);
      out[3 * k] = v[0];
      out[3 * k + 1] = v[1];
      out[3 * k + 2] = v[2];
      s0 += v[0];
      s1 += v[1];
      s2 += v[2];
    }
    out[9] = -s0;
    out[10] = -s1;
    out[11] = -s2;
  }
}

void launch_rhs_state_mixed(const MixArgs& a, int grid, cudaStream_t st) { k_rhs_state_m<<<grid, 256, 0, st>>>(a); }

__global__ void __launch_bounds__(256) k_assemble_f(int64_t n, const int32_t* __restrict__ slot_ptr,
                                                    const int32_t* __restrict__ slot_idx,
                                                    const float* __restrict__ contrib,
                                                    const uint8_t* __restrict__ is_fixed, float* __restrict__ b) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    if (!is_fixed[v]) {
      const int32_t e0 = slot_ptr[v], e1 = slot_ptr[v + 1];
      for (int32_t e = e0; e < e1; ++e) {
        const int64_t sl = slot_idx[e];
        s0 += contrib[3 * sl];
        s1 += contrib[3 * sl + 1];
        s2 += contrib[3 * sl + 2];
      }
    }
    b[3 * v] = s0;
    b[3 * v + 1] = s1;
    b[3 * v + 2] = s2;
  }
}

void launch_assemble_f(int64_t n, const int32_t* slot_ptr, const int32_t* slot_idx, const float* contrib,
                       const uint8_t* is_fixed, float* b, cudaStream_t st) {
  int grid = (int)((n + 255) / 256);
  if (grid < 1) grid = 1;
  k_assemble_f<<<grid, 256, 0, st>>>(n, slot_ptr, slot_idx, contrib, is_fixed, b);
}

// ------------------------------------------------------------ conversion --
__global__ void k_mixed_to_Rs(int64_t m, const float4* quat, const float* E, double* R, double* s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 qq = quat[i];
    double qx = qq.x, qy = qq.y, qz = qq.z, qw = qq.w;
    const double nn = 1.0 / sqrt(qx * qx + qy * qy + qz * qz + qw * qw);
    double Rr[9];
    quat_to_R(qx * nn, qy * nn, qz * nn, qw * nn, Rr);
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k * m + i] = Rr[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) s[k * m + i] = (double)E[k * m + i] + (k < 3 ? 1.0 : 0.0);
  }
}

__global__ void k_Rs_to_mixed(int64_t m, const double* R, const double* s, float4* quat, float* E) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double Rr[9], qd[4];
#pragma unroll
    for (int k = 0; k < 9; ++k) Rr[k] = R[k * m + i];
    R_to_quat(Rr, qd);
    quat[i] = make_float4((float)qd[0], (float)qd[1], (float)qd[2], (float)qd[3]);
#pragma unroll
    for (int k = 0; k < 6; ++k) E[k * m + i] = (float)(s[k * m + i] - (k < 3 ? 1.0 : 0.0));
  }
}

void launch_mixed_to_Rs(int64_t m, const float4* quat, const float* E, double* R, double* s, cudaStream_t st) {
  int grid = (int)((m + 255) / 256);
  if (grid < 1) grid = 1;
  k_mixed_to_Rs<<<grid, 256, 0, st>>>(m, quat, E, R, s);
}

void launch_Rs_to_mixed(int64_t m, const double* R, const double* s, float4* quat, float* E, cudaStream_t st) {
  int grid = (int)((m + 255) / 256);
  if (grid < 1) grid = 1;
  k_Rs_to_mixed<<<grid, 256, 0, st>>>(m, R, s, quat, E);
}

}  // namespace emu
