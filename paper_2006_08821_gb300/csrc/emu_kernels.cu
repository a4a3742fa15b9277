// Per-tet and per-vertex kernels of one Newton iteration of EMU's
// quasi-static solve in rotation/stretch form (arXiv 2006.08821, Sec. 3).
//
// One iteration (the host drives the order, everything stays on the device):
//   rhs_from_state -> assemble -> PCG          q = q*(R S)              (Eq. 4)
//   grad            g = V P(F) + alpha w (F - G q), |g|^2, Uw, y = H^-1 g  (Eqs. 6-7)
//   syrk + cap      C = sum w (G Phi)^T N (G Phi), B y, z = C^-1 B y    (Eqs. 9-12)
//   dir             d = -(y + (I - N) (G Phi) z), corner RHS of G^T W d
//   assemble -> PCG dq = q*(d) linear part
//   ls + select     Armijo backtracking on E(F + sigma d)              (Algorithm 1)
//   update          F <- F + sigma d, polar re-extraction of R, S; q += sigma dq
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "emu_kernels.cuh"
#include "emu_math.cuh"
#include "emu_reduce.cuh"
#include "emu_tetio.cuh"

namespace emu {

// ------------------------------------------------- coupling-solve RHS ----
__global__ void __launch_bounds__(256) k_rhs_from_state(TetArgs<double> a) {
  const int64_t m = a.m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double D[9], R[9], sv[6], S[9], F[9];
    load_dinv(a.Dinv, m, i, D);
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = a.R[k * m + i];
#pragma unroll
    for (int k = 0; k < 6; ++k) sv[k] = a.s[k * m + i];
    sym_from_s(sv, S);
    matmul3(R, S, F);
    write_corners(a.contrib, i, a.w[i], F, D);
  }
}

void launch_rhs_from_state(const TetArgs<double>& a, int grid, cudaStream_t st) {
  k_rhs_from_state<<<grid, 256, 0, st>>>(a);
}

__global__ void __launch_bounds__(256) k_assemble(int64_t n, const int32_t* __restrict__ slot_ptr,
                                                  const int32_t* __restrict__ slot_idx,
                                                  const double* __restrict__ contrib, const double* __restrict__ bfix,
                                                  const uint8_t* __restrict__ is_fixed,
                                                  const double* __restrict__ qfix, int mode, double* __restrict__ b) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    double s0 = 0, s1 = 0, s2 = 0;
    if (is_fixed[v]) {
      if (mode == 0) {
        s0 = qfix[3 * v];
        s1 = qfix[3 * v + 1];
        s2 = qfix[3 * v + 2];
      }
    } else {
      const int32_t e0 = slot_ptr[v], e1 = slot_ptr[v + 1];
      for (int32_t e = e0; e < e1; ++e) {
        const int64_t sl = slot_idx[e];
        s0 += contrib[3 * sl];
        s1 += contrib[3 * sl + 1];
        s2 += contrib[3 * sl + 2];
      }
      if (mode == 0) {
        s0 -= bfix[3 * v];
        s1 -= bfix[3 * v + 1];
        s2 -= bfix[3 * v + 2];
      }
    }
    b[3 * v] = s0;
    b[3 * v + 1] = s1;
    b[3 * v + 2] = s2;
  }
}

void launch_assemble(int64_t n, const int32_t* slot_ptr, const int32_t* slot_idx, const double* contrib,
                     const double* bfix, const uint8_t* is_fixed, const double* qfix, int mode, double* b,
                     cudaStream_t st) {
  int grid = (int)((n + 255) / 256);
  if (grid < 1) grid = 1;
  k_assemble<<<grid, 256, 0, st>>>(n, slot_ptr, slot_idx, contrib, bfix, is_fixed, qfix, mode, b);
}

// ------------------------------------------------------------ gradient ----
// g = V R Pr(S) + alpha w (R S - G_i q) in FP64 (Eqs. 6-7); the chart factor
// Uw and y = H_F^-1 g = (g - N g) / (alpha w) in TW.
template <typename TW>
__global__ void __launch_bounds__(128) k_grad(TetArgs<TW> a) {
  const int64_t m = a.m;
  double acc[1] = {0.0};
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    // tets of bones are no variables of their own (their g, y, U stay zero)
    if (a.tkind && a.tkind[i] != kTetDeformable) continue;
    const int4 t = a.tet[i];
    double D[9], R[9], sv[6], S[9], F[9], A[9];
    load_dinv(a.Dinv, m, i, D);
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = a.R[k * m + i];
#pragma unroll
    for (int k = 0; k < 6; ++k) sv[k] = a.s[k * m + i];
    sym_from_s(sv, S);
    matmul3(R, S, F);
    gather_defgrad(a.q, t, D, A);
    const ElemMat<double> md = load_mat<double>(a.V, a.mu, a.lam, a.ka, a.u, m, i);
    const double c = a.c[i];
    double Pr[9], Sinv[9], lnJ;
    piola_rotated(S, md, Pr, Sinv, lnJ);
    double RP[9];
    matmul3(R, Pr, RP);
    double g[9];
    double gg = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      g[k] = md.V * RP[k] + c * (F[k] - A[k]);
      if (a.nu) g[k] -= a.nu[k * m + i];  // external force (Sec. 3.4)
      gg += g[k] * g[k];
      a.g[k * m + i] = g[k];
    }
    if (!isfinite(gg)) bad = 1;
    acc[0] += gg;

    // Hessian / Woodbury quantities in TW
    TW Sw[9], Siw[9], Rw[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      Sw[k] = (TW)S[k];
      Siw[k] = (TW)Sinv[k];
      Rw[k] = (TW)R[k];
    }
    const ElemMat<TW> mw = load_mat<TW>(a.V, a.mu, a.lam, a.ka, a.u, m, i);
    TW M6[36];
    stretch_hessian(Siw, (TW)lnJ, mw, M6);
    TW U[54];
    bool ok = true;
    chart_factor(Rw, Sw, M6, (TW)c, U, ok);
    if (!ok) bad = 1;
    TW yv[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) yv[k] = (TW)g[k];
    apply_I_minus_N(U, yv);
    const TW ic = (TW)(1.0 / c);
#pragma unroll
    for (int k = 0; k < 9; ++k) a.y[k * m + i] = yv[k] * ic;
#pragma unroll
    for (int k = 0; k < 54; ++k) a.Uw[k * m + i] = U[k];
  }
  block_reduce_write<1>(acc, a.partials + blockIdx.x);
  if (bad) atomicExch(&a.sc->nonfinite, 1);
}

template <typename TW> void launch_grad(const TetArgs<TW>& a, int grid, cudaStream_t st) {
  k_grad<TW><<<grid, 128, 0, st>>>(a);
}

__global__ void __launch_bounds__(256) k_reduce_grad(const double* partials, int nblk, DevScalars* sc) {
  __shared__ double tot[1];
  block_sum_partials<1>(partials, nblk, tot);
  if (threadIdx.x == 0) sc->gnorm2 = tot[0];
}

void launch_reduce_grad(const double* partials, int nblk, DevScalars* sc, double*, double*, cudaStream_t st) {
  k_reduce_grad<<<1, 256, 0, st>>>(partials, nblk, sc);
}

// ------------------------------------------------------------ capacitance --
// C = sum_i w_i (G_i Phi^T)^T N_i (G_i Phi^T) = sum_i Yh_i^T Yh_i with
// Yh_i = sqrt(w_i) Uw_i (G_i Phi^T) (6 x 48): column 16 r + j of (G_i Phi^T) is
// the matrix e_r gam_j^T, so Yh[k][16r+j] = sqrt(w) sum_b Uw[k][3r+b] gam_j[b].
// Also B y = sum_i w_i (G_i Phi^T)^T y_i: By[16r+j] = sum_i w_i sum_b y[r][b] gam_j[b].
template <typename TW>
__global__ void __launch_bounds__(256) k_syrk(TetArgs<TW> a, double* __restrict__ cpart) {
  constexpr int CH = sizeof(TW) == 8 ? 8 : 16;  // tets per chunk
  constexpr int KR = CH * 6;
  __shared__ TW sY[KR][kK + 1];
  __shared__ TW sU[CH][54];
  __shared__ TW sg[CH][48];
  __shared__ TW sy[CH][9];
  __shared__ double sw[CH];
  const int tid = threadIdx.x;
  int tr = 0, tc = 0;
  const bool tile = lower_tile(tid, tr, tc);  // 5 of the 8 warps issue the product
  TW acc[3][3];  // per-block partial sums in TW; across blocks in FP64
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) acc[p][q] = TW(0);
  double by = 0.0;
  const int64_t m = a.m;
  const int64_t nch = (m + CH - 1) / CH;
  for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const int64_t base = ch * CH;
    for (int e = tid; e < CH * 54; e += 256) {
      const int tt = e / 54, k = e % 54;
      const int64_t i = base + tt;
      sU[tt][k] = i < m ? a.Uw[k * m + i] : TW(0);
    }
    for (int e = tid; e < CH * 48; e += 256) {
      const int tt = e / 48, k = e % 48;
      const int64_t i = base + tt;
      sg[tt][k] = i < m ? a.gam[k * m + i] : TW(0);
    }
    for (int e = tid; e < CH * 9; e += 256) {
      const int tt = e / 9, k = e % 9;
      const int64_t i = base + tt;
      sy[tt][k] = i < m ? a.y[k * m + i] : TW(0);
    }
    if (tid < CH) sw[tid] = (base + tid) < m ? a.w[base + tid] : 0.0;
    __syncthreads();
    for (int e = tid; e < CH * 6 * kK; e += 256) {
      const int tt = e / (6 * kK), rem = e % (6 * kK);
      const int k = rem / kK, col = rem % kK;
      const int r = col >> 4, j = col & 15;
      TW v = sU[tt][9 * k + 3 * r] * sg[tt][3 * j] + sU[tt][9 * k + 3 * r + 1] * sg[tt][3 * j + 1] +
             sU[tt][9 * k + 3 * r + 2] * sg[tt][3 * j + 2];
      sY[tt * 6 + k][col] = v * (TW)sqrt(sw[tt]);
    }
    __syncthreads();
#pragma unroll 4
    for (int kr = 0; kr < (tile ? KR : 0); ++kr) {
      const TW a0 = sY[kr][3 * tr], a1 = sY[kr][3 * tr + 1], a2 = sY[kr][3 * tr + 2];
      const TW b0 = sY[kr][3 * tc], b1 = sY[kr][3 * tc + 1], b2 = sY[kr][3 * tc + 2];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[0][2] += a0 * b2;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
      acc[1][2] += a1 * b2;
      acc[2][0] += a2 * b0;
      acc[2][1] += a2 * b1;
      acc[2][2] += a2 * b2;
    }
    if (tid < kK) {
      const int r = tid >> 4, j = tid & 15;
      for (int tt = 0; tt < CH; ++tt) {
        by += sw[tt] * ((double)sy[tt][3 * r] * (double)sg[tt][3 * j] + (double)sy[tt][3 * r + 1] * (double)sg[tt][3 * j + 1] +
                        (double)sy[tt][3 * r + 2] * (double)sg[tt][3 * j + 2]);
      }
    }
    __syncthreads();
  }
  // entry-major partials: cpart[e * gridDim.x + block]
  const size_t nb = gridDim.x;
  if (tile)
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const double v = (double)acc[p][q];
        cpart[(size_t)((3 * tr + p) * kK + 3 * tc + q) * nb + blockIdx.x] = v;
        if (tr != tc) cpart[(size_t)((3 * tc + q) * kK + 3 * tr + p) * nb + blockIdx.x] = v;
      }
  if (tid < kK) cpart[(size_t)(kCapEntries + tid) * nb + blockIdx.x] = by;
}

template <typename TW> void launch_syrk(const TetArgs<TW>& a, int grid, double* cpart, cudaStream_t st) {
  k_syrk<TW><<<grid, 256, 0, st>>>(a, cpart);
}

// One warp per entry of C and B y sums that entry's per-block partials
// (entry-major, coalesced) with a fixed shuffle tree.
__global__ void __launch_bounds__(256) k_reduce_cpart(const double* __restrict__ cpart, int nblk, double* __restrict__ cfull,
                                                      const double* __restrict__ cadd) {
  const int e = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= kCapEntries + kK) return;
  double x = 0.0;
  for (int b = lane; b < nblk; b += 32) x += cpart[(size_t)e * nblk + b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if (lane == 0) cfull[e] = cadd ? x + cadd[e] : x;
}

// Factor C = L L^T (C symmetrised) and solve z = C^-1 (B y), in T arithmetic
// (FP64; FP32 for the mixed path, whose C comes from TF32 products).
// Right-looking Cholesky with all 256 threads and one barrier per column:
// the column below the diagonal is left unscaled (L_ij = C_ij / sqrt(d_j),
// d_j the pivot), so each column is a single rank-1 update of the trailing
// lower triangle, C_ik -= C_ij C_kj / d_j, on a fixed 16 x 16 thread grid.
// The two triangular solves run in one warp with the right-hand side in
// registers. In FP64 the pivots' reciprocals and square roots on GB300's
// narrow FP64 path set its latency.
template <typename T>
__global__ void __launch_bounds__(256) k_cap_solve(const double* __restrict__ cfull, double* z, DevScalars* sc) {
  __shared__ T C[kK][kK + 1];
  __shared__ T rinv[kK];  // 1 / sqrt(d_j)
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  const int ti = tid >> 4, tk = tid & 15;
  for (int e = tid; e < kCapEntries; e += blockDim.x) C[e / kK][e % kK] = (T)cfull[e];
  if (tid == 0) s_ok = 1;
  __syncthreads();
  // unused modes (k_modes < 48) have zero rows: make them identity rows
  if (tid < kK && cfull[tid * kK + tid] == 0.0) C[tid][tid] = T(1);
  // symmetrise into the lower triangle
  for (int e = tid; e < kCapEntries; e += blockDim.x) {
    const int i = e / kK, j = e % kK;
    if (j < i) C[i][j] = T(0.5) * (C[i][j] + C[j][i]);
  }
  __syncthreads();
  for (int j = 0; j < kK; ++j) {
    T d = C[j][j];
    if (!(d > T(0))) d = T(1);  // failure is recorded below
    const T rho = T(1) / d;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int i = j + 1 + ti + 16 * a;
      if (i >= kK) break;
      const T cij = C[i][j] * rho;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int k = j + 1 + tk + 16 * b;
        if (k <= i) C[i][k] -= cij * C[k][j];
      }
    }
    __syncthreads();
  }
  if (tid < kK) {
    const T d = C[tid][tid];
    if (!(d > T(0))) atomicExch(&s_ok, 0);
    rinv[tid] = d > T(0) ? T(1) / sqrt(d) : T(1);
  }
  __syncthreads();
  if (tid < 32) {
    const int lane = tid;
    const bool has1 = lane + 32 < kK;
    T x0 = (T)cfull[kCapEntries + lane];
    T x1 = has1 ? (T)cfull[kCapEntries + lane + 32] : T(0);
    if (cfull[lane * kK + lane] == 0.0) x0 = T(0);  // unused mode: identity row, zero right-hand side
    if (has1 && cfull[(lane + 32) * kK + lane + 32] == 0.0) x1 = T(0);
    // L y = b: y_j = x_j / L_jj, then x_i -= L_ij y_j for i > j
    for (int j = 0; j < kK; ++j) {
      const T xj = __shfl_sync(0xffffffffu, j < 32 ? x0 : x1, j & 31);
      const T yj = xj * rinv[j];
      const T f = rinv[j] * yj;  // L_ij y_j = C_ij f
      if (lane == (j & 31)) {
        if (j < 32) x0 = yj; else x1 = yj;
      }
      if (lane > j) x0 -= C[lane][j] * f;
      if (has1 && lane + 32 > j) x1 -= C[lane + 32][j] * f;
    }
    // L^T z = y: z_j = x_j / L_jj, then x_i -= L_ji z_j for i < j
    for (int j = kK - 1; j >= 0; --j) {
      const T xj = __shfl_sync(0xffffffffu, j < 32 ? x0 : x1, j & 31);
      const T zj = xj * rinv[j];
      if (lane == (j & 31)) {
        if (j < 32) x0 = zj; else x1 = zj;
      }
      if (lane < j) x0 -= C[j][lane] * rinv[lane] * zj;
      if (has1 && lane + 32 < j) x1 -= C[j][lane + 32] * rinv[lane + 32] * zj;
    }
    const int ok = s_ok;
    z[lane] = ok ? (double)x0 : 0.0;
    if (has1) z[lane + 32] = ok ? (double)x1 : 0.0;
    if (lane == 0) sc->cap_ok = ok ? 1.0 : 0.0;
  }
}

__global__ void k_ls_reset(DevScalars* sc, double sigma0) {
  sc->ls_fail = 0;
  sc->sigma_start = sigma0;
}

void launch_ls_reset(DevScalars* sc, double sigma0, cudaStream_t st) { k_ls_reset<<<1, 1, 0, st>>>(sc, sigma0); }

void launch_cap_solve(const double* cpart, int nblk, const double* cfull_scratch, double* z, DevScalars* sc,
                      bool fp32_factor, cudaStream_t st, const double* cadd) {
  double* cfull = const_cast<double*>(cfull_scratch);
  k_reduce_cpart<<<(kCapEntries + kK + 7) / 8, 256, 0, st>>>(cpart, nblk, cfull, cadd);
  if (fp32_factor)
    k_cap_solve<float><<<1, 256, 0, st>>>(cfull, z, sc);
  else
    k_cap_solve<double><<<1, 256, 0, st>>>(cfull, z, sc);
}

// ------------------------------------------------------------ direction ---
// d = -(y + alpha H_F^-1 w (G Phi^T) z) = -(y + (I - N) v), v = (G_i Phi^T) z.
template <typename TW>
__global__ void __launch_bounds__(128) k_dir(TetArgs<TW> a) {
  __shared__ double sz[kK];
  if (threadIdx.x < kK) sz[threadIdx.x] = a.z[threadIdx.x];
  __syncthreads();
  const int64_t m = a.m;
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (a.tkind) {
      const int32_t kind = a.tkind[i];
      if (kind != kTetDeformable) {
        // a free bone's tet takes the bone's direction, a pinned bone's tet
        // none; their g . d is the bone's (summed by the bone kernel)
        double dv[9], D[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          dv[k] = kind >= 0 ? a.bone_st[(size_t)kind * kBoneStride + kBoneD + k] : 0.0;
          a.d[k * m + i] = (TW)dv[k];
        }
        load_dinv(a.Dinv, m, i, D);
        write_corners(a.contrib, i, a.w[i], dv, D);
        continue;
      }
    }
    TW gm[48];
#pragma unroll
    for (int k = 0; k < 48; ++k) gm[k] = a.gam[k * m + i];
    TW v[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        TW x = TW(0);
#pragma unroll
        for (int j = 0; j < 16; ++j) x += (TW)sz[16 * r + j] * gm[3 * j + cc];
        v[3 * r + cc] = x;
      }
    TW U[54];
#pragma unroll
    for (int k = 0; k < 54; ++k) U[k] = a.Uw[k * m + i];
    apply_I_minus_N(U, v);
    TW dv[9];
    double gtd = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      dv[k] = -(a.y[k * m + i] + v[k]);
      a.d[k * m + i] = dv[k];
      gtd += a.g[k * m + i] * (double)dv[k];
    }
    acc[0] += gtd;
    double D[9];
    load_dinv(a.Dinv, m, i, D);
    write_corners(a.contrib, i, a.w[i], dv, D);
  }
  block_reduce_write<1>(acc, a.partials + blockIdx.x);
}

template <typename TW> void launch_dir(const TetArgs<TW>& a, int grid, cudaStream_t st) {
  k_dir<TW><<<grid, 128, 0, st>>>(a);
}

// ------------------------------------------------------------ line search --
// Per trial sigma_j = sigma_start rho^j: V [Psi(F + sigma d) - Psi(F)] in FP64,
// written term by term (Algorithm 1's Armijo test needs the difference
// itself): with M = F^-1 d, ln det(I + sigma M) = log1p(sigma tr M
// + sigma^2 e2(M) + sigma^3 det M). The ACAP part is the exact quadratic
// alpha/2 sum w |D + sigma dD|^2 - |D|^2, D = G q - F, dD = G dq - d.
template <typename TW>
__global__ void __launch_bounds__(128) k_ls(TetArgs<TW> a, double rho) {
  const int64_t m = a.m;
  const double s0 = a.sc->sigma_start;
  double acc[kLsNV];
#pragma unroll
  for (int k = 0; k < kLsNV; ++k) acc[k] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    // free bones' tets: once per bone in the bone kernel; pinned bones' tets contribute 0
    if (a.tkind && a.tkind[i] != kTetDeformable) continue;
    const int4 t = a.tet[i];
    double D9[9], R[9], sv[6], S[9], F[9], A[9], dA[9], d[9];
    load_dinv(a.Dinv, m, i, D9);
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = a.R[k * m + i];
#pragma unroll
    for (int k = 0; k < 6; ++k) sv[k] = a.s[k * m + i];
#pragma unroll
    for (int k = 0; k < 9; ++k) d[k] = (double)a.d[k * m + i];
    sym_from_s(sv, S);
    matmul3(R, S, F);
    gather_defgrad(a.q, t, D9, A);
    gather_defgrad(a.dq, t, D9, dA);
    const double c = a.c[i];
    double cDd = 0.0, cdd = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double Dk = A[k] - F[k], dDk = dA[k] - d[k];
      cDd += Dk * dDk;
      cdd += dDk * dDk;
    }
    acc[kLsTrials] += c * cDd;
    acc[kLsTrials + 1] += c * cdd;
    const ElemMat<double> md = load_mat<double>(a.V, a.mu, a.lam, a.ka, a.u, m, i);
    double Sinv[9];
    const double J = inv3(S, Sinv);
    const double lnJ = log(J);
    double Rtd[9], M[9];
    matTmul3(R, d, Rtd);
    matmul3(Sinv, Rtd, M);
    const double trM = M[0] + M[4] + M[8];
    const double e2 = inv2(M);
    const double detM = det3(M);
    // <F - F^-T, d> = <S - S^-1, R^T d>: the O(|d|) parts of mu <F, d> and
    // mu tr(F^-1 d) cancel before they are formed (a stiff, barely strained
    // element, a bone, would otherwise keep only their rounding)
    double FFd = 0.0, dd = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      FFd += (S[k] - Sinv[k]) * Rtd[k];
      dd += d[k] * d[k];
    }
    double Fu[3], du[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      Fu[r] = F[3 * r] * md.u[0] + F[3 * r + 1] * md.u[1] + F[3 * r + 2] * md.u[2];
      du[r] = d[3 * r] * md.u[0] + d[3 * r + 1] * md.u[1] + d[3 * r + 2] * md.u[2];
    }
    const double Fudu = Fu[0] * du[0] + Fu[1] * du[1] + Fu[2] * du[2];
    const double dudu = du[0] * du[0] + du[1] * du[1] + du[2] * du[2];
    double dnu = 0.0;  // <d, nu>: the external work's change is -sigma <d, nu>
    if (a.nu)
#pragma unroll
      for (int k = 0; k < 9; ++k) dnu += d[k] * a.nu[k * m + i];
    double sig = s0;
#pragma unroll
    for (int j = 0; j < kLsTrials; ++j) {
      const double x = sig * trM + sig * sig * e2 + sig * sig * sig * detM;
      double dpsi;
      if (x > -1.0) {
        // mu [s <F, d> + s^2 |d|^2 / 2 - log1p(x)] with log1p(x) = x - (x - log1p x)
        const double dl = log1p(x);
        const double nh = sig * FFd + 0.5 * sig * sig * dd - sig * sig * e2 - sig * sig * sig * detM + x_minus_log1p(x);
        dpsi = md.mu * nh + 0.5 * md.lam * dl * (2.0 * lnJ + dl) + md.ka * (2.0 * sig * Fudu + sig * sig * dudu);
        dpsi = dpsi * md.V - sig * dnu;
      } else {
        dpsi = 1e300;
      }
      acc[j] += dpsi;
      sig *= rho;
    }
  }
  block_reduce_write<kLsNV>(acc, a.partials + (size_t)blockIdx.x * kLsNV);
}

template <typename TW> void launch_ls(const TetArgs<TW>& a, int grid, double rho, cudaStream_t st) {
  k_ls<TW><<<grid, 128, 0, st>>>(a, rho);
}

__global__ void __launch_bounds__(256) k_ls_select(const double* dir_partials, int nblk_dir, const double* ls_partials,
                                                    int nblk_ls, DevScalars* sc, double sigma0, double rho, double c_armijo) {
  ls_select_block(dir_partials, nblk_dir, ls_partials, nblk_ls, sc, sigma0, rho, c_armijo);
}

void launch_ls_select(const double* dir_partials, int nblk_dir, const double* ls_partials, int nblk_ls,
                      DevScalars* sc, double sigma0, double rho, double c_armijo, cudaStream_t st) {
  k_ls_select<<<1, 256, 0, st>>>(dir_partials, nblk_dir, ls_partials, nblk_ls, sc, sigma0, rho, c_armijo);
}

// ------------------------------------------------------------ update ------
// F' = R S + sigma d; X = R^T F' = S + sigma R^T d is nearly symmetric, so its
// polar factor Rx is close to I; R' = R Rx, S' = sym(Rx^T X).
template <typename TW>
__global__ void __launch_bounds__(128) k_update_tets(TetArgs<TW> a) {
  const double sig = a.sc->sigma;
  if (sig == 0.0) return;
  const int64_t m = a.m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double R[9], sv[6], S[9], d[9], Rtd[9], X[9], Rx[9], Rn[9], Sn[9], sn[6];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = a.R[k * m + i];
#pragma unroll
    for (int k = 0; k < 6; ++k) sv[k] = a.s[k * m + i];
#pragma unroll
    for (int k = 0; k < 9; ++k) d[k] = (double)a.d[k * m + i];
    sym_from_s(sv, S);
    matTmul3(R, d, Rtd);
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = S[k] + sig * Rtd[k];
    polar_rotation(X, Rx, 1e-15, 40);
    matTmul3(Rx, X, Sn);
    s_from_mat(Sn, sn);
    matmul3(R, Rx, Rn);
#pragma unroll
    for (int k = 0; k < 9; ++k) a.R[k * m + i] = Rn[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) a.s[k * m + i] = sn[k];
  }
}

template <typename TW> void launch_update_tets(const TetArgs<TW>& a, int grid, cudaStream_t st) {
  k_update_tets<TW><<<grid, 128, 0, st>>>(a);
}

__global__ void __launch_bounds__(256) k_update_verts(int64_t n3, const DevScalars* sc, const double* dq, double* q) {
  const double sig = sc->sigma;
  if (sig == 0.0) return;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x)
    q[k] += sig * dq[k];
}

void launch_update_verts(int64_t n, const DevScalars* sc, const double* dq, double* q, cudaStream_t st) {
  int64_t n3 = 3 * n;
  int grid = (int)((n3 + 255) / 256);
  if (grid < 1) grid = 1;
  k_update_verts<<<grid, 256, 0, st>>>(n3, sc, dq, q);
}

// ------------------------------------------------------------ normaliser --
// ||g(F = I, q0)||: g = V * 2 ka u u^T + alpha w (I - G q0) (the neo-Hookean
// stress vanishes at I).
__global__ void __launch_bounds__(128) k_gref(TetArgs<double> a, const double* q0, double* partials) {
  const int64_t m = a.m;
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (a.tkind && a.tkind[i] != kTetDeformable) continue;  // bones: summed per bone elsewhere
    double D[9], A[9];
    load_dinv(a.Dinv, m, i, D);
    gather_defgrad(q0, a.tet[i], D, A);
    const double V = a.V[i], c = a.c[i], ka = a.ka[i];
    const double u[3] = {a.u[i], a.u[m + i], a.u[2 * m + i]};
    double gg = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        double gv = V * 2.0 * ka * u[r] * u[cc] + c * ((r == cc ? 1.0 : 0.0) - A[3 * r + cc]);
        if (a.nu) gv -= a.nu[(3 * r + cc) * m + i];
        gg += gv * gv;
      }
    acc[0] += gg;
  }
  block_reduce_write<1>(acc, partials + blockIdx.x);
}

__global__ void __launch_bounds__(256) k_sum_scalar(const double* partials, int nblk, double* out) {
  __shared__ double tot[1];
  block_sum_partials<1>(partials, nblk, tot);
  if (threadIdx.x == 0) out[0] = tot[0];
}

void launch_gref(const TetArgs<double>& a, const double* q0, int grid, double* partials, double* out,
                 cudaStream_t st) {
  k_gref<<<grid, 128, 0, st>>>(a, q0, partials);
  k_sum_scalar<<<1, 256, 0, st>>>(partials, grid, out);
}

// ------------------------------------------------------------ modes -------
__global__ void __launch_bounds__(256) k_gram16(int64_t n, const double* __restrict__ X, double* partials) {
  const int a = threadIdx.x >> 4, b = threadIdx.x & 15;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t v0 = blockIdx.x * per;
  const int64_t v1 = v0 + per < n ? v0 + per : n;
  double acc = 0.0;
  for (int64_t v = v0; v < v1; ++v) acc += X[v * 16 + a] * X[v * 16 + b];
  partials[(size_t)blockIdx.x * 256 + threadIdx.x] = acc;
}

void launch_gram16(int64_t n, const double* X, int grid, double* partials, cudaStream_t st) {
  k_gram16<<<grid, 256, 0, st>>>(n, X, partials);
}

// Y = L X for 16 columns (L in CSR, X and Y vertex-major n x 16)
__global__ void __launch_bounds__(256) k_spmv16(int64_t n, const int32_t* __restrict__ rowptr,
                                                const int32_t* __restrict__ col, const double* __restrict__ val,
                                                const double* __restrict__ X, double* __restrict__ Y) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    double acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.0;
    for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
      const double a = val[e];
      const int64_t c = col[e];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] += a * X[c * 16 + j];
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) Y[v * 16 + j] = acc[j];
  }
}

// partials of X^T Y (16 x 16) over contiguous vertex ranges
__global__ void __launch_bounds__(256) k_cross16(int64_t n, const double* __restrict__ X, const double* __restrict__ Y,
                                                 double* partials) {
  const int a = threadIdx.x >> 4, b = threadIdx.x & 15;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t v0 = blockIdx.x * per;
  const int64_t v1 = v0 + per < n ? v0 + per : n;
  double acc = 0.0;
  for (int64_t v = v0; v < v1; ++v) acc += X[v * 16 + a] * Y[v * 16 + b];
  partials[(size_t)blockIdx.x * 256 + threadIdx.x] = acc;
}

void launch_galerkin16(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* X,
                       double* Y, int grid, double* partials, cudaStream_t st) {
  int g2 = (int)((n + 255) / 256);
  if (g2 < 1) g2 = 1;
  k_spmv16<<<g2, 256, 0, st>>>(n, rowptr, col, val, X, Y);
  k_cross16<<<grid, 256, 0, st>>>(n, X, Y, partials);
}

__global__ void k_d2f(int64_t k, const double* a, float* b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

void launch_d2f(int64_t k, const double* a, float* b, cudaStream_t st) {
  int grid = (int)((k + 255) / 256);
  if (grid < 1) grid = 1;
  k_d2f<<<grid, 256, 0, st>>>(k, a, b);
}

__global__ void k_reduce_cols(const double* partials, int nblk, int nv, double* out) {
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    double x = 0.0;
    for (int b = 0; b < nblk; ++b) x += partials[(size_t)b * nv + k];
    out[k] = x;
  }
}

void launch_reduce_cols(const double* partials, int nblk, int nv, double* out, cudaStream_t st) {
  k_reduce_cols<<<1, 256, 0, st>>>(partials, nblk, nv, out);
}

__global__ void __launch_bounds__(256) k_xform16(int64_t n, const double* __restrict__ T, double* X) {
  __shared__ double sT[256];
  sT[threadIdx.x] = T[threadIdx.x];
  __syncthreads();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    double x[16], y[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = X[v * 16 + k];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < 16; ++k) s += x[k] * sT[16 * k + j];
      y[j] = s;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) X[v * 16 + k] = y[k];
  }
}

void launch_xform16(int64_t n, const double* T, double* X, cudaStream_t st) {
  int grid = (int)((n + 255) / 256);
  if (grid < 1) grid = 1;
  k_xform16<<<grid, 256, 0, st>>>(n, T, X);
}

// gam_j = gradient of mode j on tet i: sum_k (phi_j(v_k) - phi_j(v_3)) Dinv[k][:]
template <typename TW>
__global__ void __launch_bounds__(256) k_gamma(int64_t m, const int4* __restrict__ tet, const double* __restrict__ Dinv,
                                               const double* __restrict__ X, TW* gam) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int4 t = tet[i];
    double D[9];
    load_dinv(Dinv, m, i, D);
    for (int j = 0; j < 16; ++j) {
      const double x3 = X[(int64_t)t.w * 16 + j];
      const double e0 = X[(int64_t)t.x * 16 + j] - x3;
      const double e1 = X[(int64_t)t.y * 16 + j] - x3;
      const double e2 = X[(int64_t)t.z * 16 + j] - x3;
#pragma unroll
      for (int c = 0; c < 3; ++c) gam[(3 * j + c) * m + i] = (TW)(e0 * D[c] + e1 * D[3 + c] + e2 * D[6 + c]);
    }
  }
}

template <typename TW>
void launch_gamma(int64_t m, const int4* tet, const double* Dinv, const double* X, TW* gam, cudaStream_t st) {
  int grid = (int)((m + 255) / 256);
  if (grid < 1) grid = 1;
  k_gamma<TW><<<grid, 256, 0, st>>>(m, tet, Dinv, X, gam);
}

// ------------------------------------------------------- external force ---
__global__ void __launch_bounds__(256) k_nu(int64_t m, const int4* __restrict__ tet, const double* __restrict__ Dinv,
                                            const double* __restrict__ w, const double* __restrict__ x,
                                            double* __restrict__ nu64, float* __restrict__ nu32) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double D[9], A[9];
    load_dinv(Dinv, m, i, D);
    gather_defgrad(x, tet[i], D, A);
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double v = wi * A[k];
      nu64[k * m + i] = v;
      if (nu32) nu32[k * m + i] = (float)v;
    }
  }
}

void launch_nu(int64_t m, const int4* tet, const double* Dinv, const double* w, const double* x, double* nu64,
               float* nu32, cudaStream_t st) {
  int grid = (int)((m + 255) / 256);
  if (grid < 1) grid = 1;
  k_nu<<<grid, 256, 0, st>>>(m, tet, Dinv, w, x, nu64, nu32);
}

// ------------------------------------------------------------ element API --
template <typename T>
__global__ void k_eval_stretch(const double* s, const double* prm, int64_t n, double* psi, double* grad, double* hess) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T sv[6], S[9], Sinv[9];
#pragma unroll
    for (int k = 0; k < 6; ++k) sv[k] = (T)s[6 * i + k];
    ElemMat<T> e;
    e.V = (T)prm[8 * i];
    e.mu = (T)prm[8 * i + 1];
    e.lam = (T)prm[8 * i + 2];
    e.ka = (T)prm[8 * i + 3];
    e.u[0] = (T)prm[8 * i + 4];
    e.u[1] = (T)prm[8 * i + 5];
    e.u[2] = (T)prm[8 * i + 6];
    sym_from_s(sv, S);
    const T J = inv3(S, Sinv);
    const T lnJ = log(J);
    if (psi) psi[i] = (double)(e.V * psi_stretch(S, e));
    if (grad) {
      T g[6];
      stretch_gradient(S, Sinv, lnJ, e, g);
#pragma unroll
      for (int k = 0; k < 6; ++k) grad[6 * i + k] = (double)g[k];
    }
    if (hess) {
      T H[36];
      stretch_hessian(Sinv, lnJ, e, H);
#pragma unroll
      for (int k = 0; k < 36; ++k) hess[36 * i + k] = (double)H[k];
    }
  }
}

void launch_eval_stretch(const double* s, const double* prm, int64_t n, int mixed, double* psi, double* grad,
                         double* hess, cudaStream_t st) {
  int grid = (int)((n + 127) / 128);
  if (grid < 1) grid = 1;
  if (mixed)
    k_eval_stretch<float><<<grid, 128, 0, st>>>(s, prm, n, psi, grad, hess);
  else
    k_eval_stretch<double><<<grid, 128, 0, st>>>(s, prm, n, psi, grad, hess);
}

__global__ void k_eval_polar(const double* F, int64_t n, double* R, double* s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double X[9], Rr[9], S[9], sv[6];
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = F[9 * i + k];
    polar_rotation(X, Rr, 1e-15, 60);
    matTmul3(Rr, X, S);
    s_from_mat(S, sv);
#pragma unroll
    for (int k = 0; k < 9; ++k) R[9 * i + k] = Rr[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) s[6 * i + k] = sv[k];
  }
}

void launch_eval_polar(const double* F, int64_t n, double* R, double* s, cudaStream_t st) {
  int grid = (int)((n + 127) / 128);
  if (grid < 1) grid = 1;
  k_eval_polar<<<grid, 128, 0, st>>>(F, n, R, s);
}

// F may alias R: each thread reads its tet's R before it writes F.
__global__ void k_compose_F(int64_t m, const double* R, const double* s, double* F) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double Rr[9], sv[6], S[9], Fi[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Rr[k] = R[k * m + i];
#pragma unroll
    for (int k = 0; k < 6; ++k) sv[k] = s[k * m + i];
    sym_from_s(sv, S);
    matmul3(Rr, S, Fi);
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k * m + i] = Fi[k];
  }
}

void launch_compose_F(int64_t m, const double* R, const double* s, double* F, cudaStream_t st) {
  int grid = (int)((m + 255) / 256);
  if (grid < 1) grid = 1;
  k_compose_F<<<grid, 256, 0, st>>>(m, R, s, F);
}

// explicit instantiations
template void launch_grad<double>(const TetArgs<double>&, int, cudaStream_t);
template void launch_grad<float>(const TetArgs<float>&, int, cudaStream_t);
template void launch_syrk<double>(const TetArgs<double>&, int, double*, cudaStream_t);
template void launch_syrk<float>(const TetArgs<float>&, int, double*, cudaStream_t);
template void launch_dir<double>(const TetArgs<double>&, int, cudaStream_t);
template void launch_dir<float>(const TetArgs<float>&, int, cudaStream_t);
template void launch_ls<double>(const TetArgs<double>&, int, double, cudaStream_t);
template void launch_ls<float>(const TetArgs<float>&, int, double, cudaStream_t);
template void launch_update_tets<double>(const TetArgs<double>&, int, cudaStream_t);
template void launch_update_tets<float>(const TetArgs<float>&, int, cudaStream_t);
template void launch_gamma<double>(int64_t, const int4*, const double*, const double*, double*, cudaStream_t);
template void launch_gamma<float>(int64_t, const int4*, const double*, const double*, float*, cudaStream_t);

}  // namespace emu
