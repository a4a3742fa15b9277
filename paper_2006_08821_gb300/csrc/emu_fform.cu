// Kernels of the F-form iteration (arXiv 2006.08821, Sec. 3.2.1, Eqs. 10-12;
// Algorithm 1), FP64 throughout. One iteration:
//   grad      g = V P(F) + alpha w (F - G q) - nu, |g|^2, H = L L^T, y = H^-1 g
//   syrk+cap  C = Lambda - alpha sum w^2 (G Phi)^T H^-1 (G Phi), B y, z = C^-1 B y
//   dir       d = -(y + alpha w H^-1 (G Phi) z), corner terms of G^T W d
//   assemble -> CG  dq (the linear part of q*(F + d) - q*(F), Eq. 4)
//   ls        Armijo trials on E(F + sigma d) with q + sigma dq
//   update    F += sigma d, q += sigma dq
// The definiteness fix of Sec. 3.2.1 is applied to the elastic (isotropic
// neo-Hookean) term through its analytic eigen-system; the fiber term and
// alpha w I are positive semi-definite as they stand.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "emu_fform.h"
#include "emu_kernels.cuh"
#include "emu_math.cuh"
#include "emu_reduce.cuh"
#include "emu_tetio.cuh"

namespace emu {
namespace {

__device__ __forceinline__ constexpr int pk(int r, int c) { return r * (r + 1) / 2 + c; }  // c <= r

// Eigen-decomposition of a symmetric 3 x 3 matrix by the cyclic Jacobi
// method (Golub and Van Loan, Matrix Computations, Sec. 8.5): each rotation
// in the (p, q) plane zeroes a_pq; A = W diag(lam) W^T with W's columns the
// eigenvectors (W[3 r + k] = component r of vector k). A is read as its
// symmetric part.
__device__ void sym3_eig(const double* A, double* lam, double* W) {
  double a[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) a[r][c] = 0.5 * (A[3 * r + c] + A[3 * c + r]);
#pragma unroll
  for (int k = 0; k < 9; ++k) W[k] = (k % 4 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 16; ++sweep) {
    const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (!(off > 1e-34 * dia)) break;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int p = e == 2 ? 1 : 0, q = e == 0 ? 1 : 2, o = 3 - p - q;
      const double apq = a[p][q];
      if (apq == 0.0) continue;
      const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
      const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
      const double aop = a[o][p], aoq = a[o][q];
      a[o][p] = a[p][o] = c * aop - s * aoq;
      a[o][q] = a[q][o] = s * aop + c * aoq;
      a[p][p] -= t * apq;
      a[q][q] += t * apq;
      a[p][q] = a[q][p] = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double wp = W[3 * k + p], wq = W[3 * k + q];
        W[3 * k + p] = c * wp - s * wq;
        W[3 * k + q] = s * wp + c * wq;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) lam[k] = a[k][k];
}

// H (packed lower) += lam z z^T
__device__ __forceinline__ void add_rank1(double* H, double lam, const double* z) {
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const double lz = lam * z[p];
#pragma unroll
    for (int q = 0; q <= p; ++q) H[pk(p, q)] += lz * z[q];
  }
}

// Psi(F) of Sec. 3.1: mu/2 (|F|^2 - 3) - mu ln J + lam/2 ln^2 J + ka |F u|^2
// (J <= 0 gives a huge value, the inverted-element energy).
__device__ double psi_F(const double* F, const ElemMat<double>& md) {
  const double J = det3(F);
  if (!(J > 0.0)) return 1e40;
  const double lnJ = log(J);
  double I1 = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) I1 += F[k] * F[k];
  double fu = 0.0;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double x = F[3 * r] * md.u[0] + F[3 * r + 1] * md.u[1] + F[3 * r + 2] * md.u[2];
    fu += x * x;
  }
  return 0.5 * md.mu * (I1 - 3.0) - md.mu * lnJ + 0.5 * md.lam * lnJ * lnJ + md.ka * fu;
}

// First Piola stress P = mu (F - F^-T) + lam ln J F^-T + 2 ka (F u) u^T.
__device__ __forceinline__ void piola_F(const double* F, const double* Finv, double lnJ, const ElemMat<double>& md,
                                        double* P) {
  double Fu[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) Fu[r] = F[3 * r] * md.u[0] + F[3 * r + 1] * md.u[1] + F[3 * r + 2] * md.u[2];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double FiT = Finv[3 * c + r];
      P[3 * r + c] = md.mu * (F[3 * r + c] - FiT) + md.lam * lnJ * FiT + 2.0 * md.ka * Fu[r] * md.u[c];
    }
}

// V times the Hessian of Psi in row-major vec(F) (index 3 r + c), packed
// lower, with the definiteness fix on the isotropic part: in the frame of
// the singular value decomposition F = U diag(sig) V^T (from the polar
// decomposition F = R S and the eigen-decomposition S = V diag(sig) V^T,
// U = R V) the neo-Hookean Hessian
//   mu I + (mu - lam ln J) F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T
// splits into a 3 x 3 block on the diagonal entries of U^T dF V,
//   A_ij = lam / (sig_i sig_j) + [i = j] (mu + (mu - lam ln J) / sig_i^2),
// and, for each pair i < j, the eigenvectors (u_i v_j^T +- u_j v_i^T) / sqrt2
// with eigenvalues mu +- (mu - lam ln J) / (sig_i sig_j). Their negative
// eigenvalues are clamped at zero (the eigen-system of an isotropic energy:
// Smith, de Goes and Kim, "Analytic eigensystems for isotropic distortion
// energies", ACM TOG 2019). The fiber term 2 ka I (x) u u^T is added as it
// stands. ok = false when the polar iteration meets a non-positive det F.
__device__ void hessian_F(const double* F, double lnJ, const ElemMat<double>& md, double* H, bool& ok) {
#pragma unroll
  for (int k = 0; k < kFformL; ++k) H[k] = 0.0;
  double R[9], S[9], sig[3], Vm[9], U[9];
  polar_rotation(F, R, 1e-15, 60);
  matTmul3(R, F, S);
  sym3_eig(S, sig, Vm);
  matmul3(R, Vm, U);
  ok = sig[0] > 0.0 && sig[1] > 0.0 && sig[2] > 0.0;
  const double cm = md.mu - md.lam * lnJ;
  // the 3 x 3 block on the diagonal entries
  double A3[9], eta[3], Wd[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      A3[3 * i + j] = md.lam / (sig[i] * sig[j]) + (i == j ? md.mu + cm / (sig[i] * sig[i]) : 0.0);
  sym3_eig(A3, eta, Wd);
  double z[9];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (!(eta[k] > 0.0)) continue;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        z[3 * r + c] = Wd[k] * U[3 * r] * Vm[3 * c] + Wd[3 + k] * U[3 * r + 1] * Vm[3 * c + 1] +
                       Wd[6 + k] * U[3 * r + 2] * Vm[3 * c + 2];
    add_rank1(H, eta[k], z);
  }
  // the three pairs
  const double h = rsqrt2<double>();
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int i = e == 2 ? 1 : 0, j = e == 0 ? 1 : 2;
    const double tw = cm / (sig[i] * sig[j]);
#pragma unroll
    for (int sgn = 0; sgn < 2; ++sgn) {
      const double lam = sgn == 0 ? md.mu + tw : md.mu - tw;
      if (!(lam > 0.0)) continue;
      const double sv = sgn == 0 ? h : -h;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) z[3 * r + c] = h * U[3 * r + i] * Vm[3 * c + j] + sv * U[3 * r + j] * Vm[3 * c + i];
      add_rank1(H, lam, z);
    }
  }
  // fiber: 2 ka delta_rr' u_c u_c'
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int c2 = 0; c2 <= c; ++c2) H[pk(3 * r + c, 3 * r + c2)] += 2.0 * md.ka * md.u[c] * md.u[c2];
#pragma unroll
  for (int k = 0; k < kFformL; ++k) H[k] *= md.V;
}

// In-place Cholesky of the packed 9 x 9 SPD matrix: H = L L^T with 1 / L_jj
// stored on the diagonal. False when a pivot is not positive.
__device__ __forceinline__ bool chol9(double* H) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    double d = H[pk(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= H[pk(j, k)] * H[pk(j, k)];
    ok = ok && d > 0.0;
    const double id = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
    H[pk(j, j)] = id;
#pragma unroll
    for (int i = j + 1; i < 9; ++i) {
      double v = H[pk(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= H[pk(i, k)] * H[pk(j, k)];
      H[pk(i, j)] = v * id;
    }
  }
  return ok;
}

// x <- L^-1 x
__device__ __forceinline__ void lsolve9(const double* L, double* x) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    double v = x[i];
#pragma unroll
    for (int k = 0; k < i; ++k) v -= L[pk(i, k)] * x[k];
    x[i] = v * L[pk(i, i)];
  }
}

// x <- L^-T x
__device__ __forceinline__ void ltsolve9(const double* L, double* x) {
#pragma unroll
  for (int i = 8; i >= 0; --i) {
    double v = x[i];
#pragma unroll
    for (int k = i + 1; k < 9; ++k) v -= L[pk(k, i)] * x[k];
    x[i] = v * L[pk(i, i)];
  }
}

__device__ __forceinline__ void load_F(const double* Fs, int64_t m, int64_t i, double* F) {
#pragma unroll
  for (int k = 0; k < 9; ++k) F[k] = Fs[k * m + i];
}

// ------------------------------------------------- coupling-solve RHS ----
__global__ void __launch_bounds__(256) k_rhs_fform(TetArgs<double> a) {
  const int64_t m = a.m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double D[9], F[9];
    load_dinv(a.Dinv, m, i, D);
    load_F(a.R, m, i, F);
    write_corners(a.contrib, i, a.w[i], F, D);
  }
}

// ------------------------------------------------------------ gradient ----
// g = V P(F) + alpha w (F - G_i q) - nu (Eqs. 6-7, Sec. 3.4), |g|^2; the
// factor of H = hessian_F + alpha w I and y = H^-1 g.
__global__ void __launch_bounds__(128) k_grad_fform(TetArgs<double> a) {
  const int64_t m = a.m;
  double acc[1] = {0.0};
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double D[9], F[9], A[9], Finv[9], P[9];
    load_dinv(a.Dinv, m, i, D);
    load_F(a.R, m, i, F);
    gather_defgrad(a.q, a.tet[i], D, A);
    const ElemMat<double> md = load_mat<double>(a.V, a.mu, a.lam, a.ka, a.u, m, i);
    const double c = a.c[i];
    const double J = inv3(F, Finv);
    const double lnJ = log(J);
    piola_F(F, Finv, lnJ, md, P);
    double g[9];
    double gg = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      g[k] = md.V * P[k] + c * (F[k] - A[k]);
      if (a.nu) g[k] -= a.nu[k * m + i];
      gg += g[k] * g[k];
      a.g[k * m + i] = g[k];
    }
    if (!isfinite(gg) || !(J > 0.0)) bad = 1;
    acc[0] += gg;
    double H[kFformL];
    bool ok = true;
    hessian_F(F, lnJ, md, H, ok);
#pragma unroll
    for (int k = 0; k < 9; ++k) H[pk(k, k)] += c;
    ok = chol9(H) && ok;
    if (!ok) bad = 1;
    lsolve9(H, g);
    ltsolve9(H, g);
#pragma unroll
    for (int k = 0; k < 9; ++k) a.y[k * m + i] = g[k];
#pragma unroll
    for (int k = 0; k < kFformL; ++k) a.Uw[k * m + i] = H[k];
  }
  block_reduce_write<1>(acc, a.partials + blockIdx.x);
  if (bad) atomicExch(&a.sc->nonfinite, 1);
}

// ------------------------------------------------------------ capacitance --
// Yh_i = sqrt(alpha w_i^2) L_i^-1 (G_i Phi) (9 x 48): column 16 r + j of
// G_i Phi is the matrix e_r gam_j^T, so its vec holds gam_j in rows
// 3r .. 3r+2. The block sums -Yh^T Yh (the Woodbury term of Eq. 12) and
// B y = sum_i w_i (G_i Phi)^T y_i: By[16r+j] = sum_i w_i sum_b y[r][b] gam_j[b].
__global__ void __launch_bounds__(256) k_syrk_fform(TetArgs<double> a, double* __restrict__ cpart) {
  constexpr int CH = 8;  // tets per chunk
  constexpr int KR = CH * 9;
  __shared__ double sY[KR][kK + 1];
  __shared__ double sL[CH][kFformL];
  __shared__ double sg[CH][48];
  __shared__ double sy[CH][9];
  __shared__ double sw[CH], scw[CH];
  const int tid = threadIdx.x;
  int tr = 0, tc = 0;
  const bool tile = lower_tile(tid, tr, tc);  // 5 of the 8 warps issue the product
  double acc[3][3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) acc[p][q] = 0.0;
  double by = 0.0;
  const int64_t m = a.m;
  const int64_t nch = (m + CH - 1) / CH;
  for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const int64_t base = ch * CH;
    for (int e = tid; e < CH * kFformL; e += 256) {
      const int tt = e / kFformL, k = e % kFformL;
      const int64_t i = base + tt;
      // a tail tet gets the identity factor and a zero weight
      sL[tt][k] = i < m ? a.Uw[k * m + i] : ((k == 0 || k == 2 || k == 5 || k == 9 || k == 14 || k == 20 ||
                                             k == 27 || k == 35 || k == 44) ? 1.0 : 0.0);
    }
    for (int e = tid; e < CH * 48; e += 256) {
      const int tt = e / 48, k = e % 48;
      const int64_t i = base + tt;
      sg[tt][k] = i < m ? a.gam[k * m + i] : 0.0;
    }
    for (int e = tid; e < CH * 9; e += 256) {
      const int tt = e / 9, k = e % 9;
      const int64_t i = base + tt;
      sy[tt][k] = i < m ? a.y[k * m + i] : 0.0;
    }
    if (tid < CH) {
      const int64_t i = base + tid;
      sw[tid] = i < m ? a.w[i] : 0.0;
      scw[tid] = i < m ? sqrt(a.c[i] * a.w[i]) : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < CH * kK; e += 256) {
      const int tt = e / kK, col = e % kK;
      const int r = col >> 4, j = col & 15;
      double x[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) x[k] = (k / 3 == r) ? sg[tt][3 * j + k % 3] : 0.0;
      lsolve9(sL[tt], x);
      const double sc = scw[tt];
#pragma unroll
      for (int k = 0; k < 9; ++k) sY[tt * 9 + k][col] = x[k] * sc;
    }
    __syncthreads();
#pragma unroll 4
    for (int kr = 0; kr < (tile ? KR : 0); ++kr) {
      const double a0 = sY[kr][3 * tr], a1 = sY[kr][3 * tr + 1], a2 = sY[kr][3 * tr + 2];
      const double b0 = sY[kr][3 * tc], b1 = sY[kr][3 * tc + 1], b2 = sY[kr][3 * tc + 2];
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
      for (int tt = 0; tt < CH; ++tt)
        by += sw[tt] * (sy[tt][3 * r] * sg[tt][3 * j] + sy[tt][3 * r + 1] * sg[tt][3 * j + 1] +
                        sy[tt][3 * r + 2] * sg[tt][3 * j + 2]);
    }
    __syncthreads();
  }
  const size_t nb = gridDim.x;
  if (tile)
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        cpart[(size_t)((3 * tr + p) * kK + 3 * tc + q) * nb + blockIdx.x] = -acc[p][q];
        if (tr != tc) cpart[(size_t)((3 * tc + q) * kK + 3 * tr + p) * nb + blockIdx.x] = -acc[p][q];
      }
  if (tid < kK) cpart[(size_t)(kCapEntries + tid) * nb + blockIdx.x] = by;
}

// ------------------------------------------------------------ direction ---
// d = -(y + alpha w H^-1 v), v = (G_i Phi) z; g . d; corners of w G^T d.
__global__ void __launch_bounds__(128) k_dir_fform(TetArgs<double> a) {
  __shared__ double sz[kK];
  if (threadIdx.x < kK) sz[threadIdx.x] = a.z[threadIdx.x];
  __syncthreads();
  const int64_t m = a.m;
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double gm[48];
#pragma unroll
    for (int k = 0; k < 48; ++k) gm[k] = a.gam[k * m + i];
    double v[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        double x = 0.0;
#pragma unroll
        for (int j = 0; j < 16; ++j) x += sz[16 * r + j] * gm[3 * j + cc];
        v[3 * r + cc] = x;
      }
    double L[kFformL];
#pragma unroll
    for (int k = 0; k < kFformL; ++k) L[k] = a.Uw[k * m + i];
    lsolve9(L, v);
    ltsolve9(L, v);
    const double c = a.c[i];
    double dv[9];
    double gtd = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      dv[k] = -(a.y[k * m + i] + c * v[k]);
      a.d[k * m + i] = dv[k];
      gtd += a.g[k * m + i] * dv[k];
    }
    acc[0] += gtd;
    double D[9];
    load_dinv(a.Dinv, m, i, D);
    write_corners(a.contrib, i, a.w[i], dv, D);
  }
  block_reduce_write<1>(acc, a.partials + blockIdx.x);
}

// ------------------------------------------------------------ line search --
// The trial energies of the rotation/stretch line search with F read
// directly: per trial sigma_j, V [Psi(F + sigma d) - Psi(F)] term by term
// (ln det(I + sigma M), M = F^-1 d, through log1p of its polynomial), and
// the ACAP part's two coefficients alpha w <D, dD>, alpha w |dD|^2 with
// D = G q - F, dD = G dq - d.
__global__ void __launch_bounds__(128) k_ls_fform(TetArgs<double> a, double rho) {
  const int64_t m = a.m;
  const double s0 = a.sc->sigma_start;
  double acc[kLsNV];
#pragma unroll
  for (int k = 0; k < kLsNV; ++k) acc[k] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int4 t = a.tet[i];
    double D9[9], F[9], A[9], dA[9], d[9];
    load_dinv(a.Dinv, m, i, D9);
    load_F(a.R, m, i, F);
#pragma unroll
    for (int k = 0; k < 9; ++k) d[k] = a.d[k * m + i];
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
    double Finv[9], M[9];
    const double J = inv3(F, Finv);
    const double lnJ = log(J);
    matmul3(Finv, d, M);
    const double trM = M[0] + M[4] + M[8];
    const double e2 = inv2(M);
    const double detM = det3(M);
    // <F - F^-T, d> and |d|^2
    double FFd = 0.0, dd = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        FFd += (F[3 * r + cc] - Finv[3 * cc + r]) * d[3 * r + cc];
        dd += d[3 * r + cc] * d[3 * r + cc];
      }
    double Fu[3], du[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      Fu[r] = F[3 * r] * md.u[0] + F[3 * r + 1] * md.u[1] + F[3 * r + 2] * md.u[2];
      du[r] = d[3 * r] * md.u[0] + d[3 * r + 1] * md.u[1] + d[3 * r + 2] * md.u[2];
    }
    const double Fudu = Fu[0] * du[0] + Fu[1] * du[1] + Fu[2] * du[2];
    const double dudu = du[0] * du[0] + du[1] * du[1] + du[2] * du[2];
    double dnu = 0.0;
    if (a.nu)
#pragma unroll
      for (int k = 0; k < 9; ++k) dnu += d[k] * a.nu[k * m + i];
    double sig = s0;
#pragma unroll
    for (int j = 0; j < kLsTrials; ++j) {
      const double x = sig * trM + sig * sig * e2 + sig * sig * sig * detM;
      double dpsi;
      if (x > -1.0 && J > 0.0) {
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

// ------------------------------------------------------------ update ------
__global__ void __launch_bounds__(256) k_update_fform(TetArgs<double> a) {
  const double sig = a.sc->sigma;
  if (sig == 0.0) return;
  const int64_t m = a.m;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int k = 0; k < 9; ++k) a.R[k * m + i] += sig * a.d[k * m + i];
}

__global__ void __launch_bounds__(128) k_fform_to_Rs(int64_t m, const double* F, double* R, double* s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double X[9], Rr[9], S[9], sv[6];
    load_F(F, m, i, X);
    polar_rotation(X, Rr, 1e-15, 60);
    matTmul3(Rr, X, S);
    s_from_mat(S, sv);
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k * m + i] = Rr[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) s[k * m + i] = sv[k];
  }
}

__global__ void __launch_bounds__(128) k_eval_fform(const double* F, const double* prm, int64_t n, double* psi,
                                                    double* grad, double* hess) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double Fi[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Fi[k] = F[9 * i + k];
    ElemMat<double> e;
    e.V = prm[8 * i];
    e.mu = prm[8 * i + 1];
    e.lam = prm[8 * i + 2];
    e.ka = prm[8 * i + 3];
    e.u[0] = prm[8 * i + 4];
    e.u[1] = prm[8 * i + 5];
    e.u[2] = prm[8 * i + 6];
    if (psi) psi[i] = e.V * psi_F(Fi, e);
    double Finv[9];
    const double lnJ = log(inv3(Fi, Finv));
    if (grad) {
      double P[9];
      piola_F(Fi, Finv, lnJ, e, P);
#pragma unroll
      for (int k = 0; k < 9; ++k) grad[9 * i + k] = e.V * P[k];
    }
    if (hess) {
      double H[kFformL];
      bool ok = true;
      hessian_F(Fi, lnJ, e, H, ok);
#pragma unroll
      for (int p = 0; p < 9; ++p)
#pragma unroll
        for (int q = 0; q <= p; ++q) {
          const double v = ok ? H[pk(p, q)] : NAN;
          hess[81 * i + 9 * p + q] = v;
          hess[81 * i + 9 * q + p] = v;
        }
    }
  }
}

}  // namespace

static int fform_grid(int64_t m, int threads) { return (int)(m > 0 ? (m + threads - 1) / threads : 1); }

void launch_rhs_fform(const TetArgs<double>& a, int grid, cudaStream_t st) { k_rhs_fform<<<grid, 256, 0, st>>>(a); }
void launch_grad_fform(const TetArgs<double>& a, int grid, cudaStream_t st) { k_grad_fform<<<grid, 128, 0, st>>>(a); }
void launch_syrk_fform(const TetArgs<double>& a, int grid, double* cpart, cudaStream_t st) {
  k_syrk_fform<<<grid, 256, 0, st>>>(a, cpart);
}
void launch_dir_fform(const TetArgs<double>& a, int grid, cudaStream_t st) { k_dir_fform<<<grid, 128, 0, st>>>(a); }
void launch_ls_fform(const TetArgs<double>& a, int grid, double rho, cudaStream_t st) {
  k_ls_fform<<<grid, 128, 0, st>>>(a, rho);
}
void launch_update_fform(const TetArgs<double>& a, int grid, cudaStream_t st) {
  k_update_fform<<<grid, 256, 0, st>>>(a);
}
void launch_fform_to_Rs(int64_t m, const double* F, double* R, double* s, cudaStream_t st) {
  k_fform_to_Rs<<<fform_grid(m, 128), 128, 0, st>>>(m, F, R, s);
}
void launch_eval_fform(const double* F, const double* prm, int64_t n, double* psi, double* grad, double* hess,
                       cudaStream_t st) {
  k_eval_fform<<<fform_grid(n, 128), 128, 0, st>>>(F, prm, n, psi, grad, hess);
}

}  // namespace emu
