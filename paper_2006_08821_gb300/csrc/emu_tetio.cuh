// Per-tet gathers and scatters shared by the rotation/stretch kernels and
// the F-form kernels: D_m^-1, the material of a tet, G_i q (Eq. 2) and the
// corner terms of w G_i^T X (the right-hand side of Eq. 4).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "emu_math.cuh"

namespace emu {

// ------------------------------------------------------------ gathers ----
__device__ __forceinline__ void load_dinv(const double* __restrict__ Dinv, int64_t m, int64_t i, double* D) {
#pragma unroll
  for (int k = 0; k < 9; ++k) D[k] = Dinv[k * m + i];
}

// A = G_i q = D_s(q) D_m^-1 (Eq. 2): A[r][c] = sum_k (q_k - q_3)[r] Dinv[k][c]
__device__ __forceinline__ void gather_defgrad(const double* __restrict__ q, int4 t, const double* D, double* A) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double q3 = q[3 * (int64_t)t.w + r];
    const double e0 = q[3 * (int64_t)t.x + r] - q3;
    const double e1 = q[3 * (int64_t)t.y + r] - q3;
    const double e2 = q[3 * (int64_t)t.z + r] - q3;
#pragma unroll
    for (int c = 0; c < 3; ++c) A[3 * r + c] = e0 * D[c] + e1 * D[3 + c] + e2 * D[6 + c];
  }
}

// Corner contributions of w G_i^T X: for corner k < 3 the shape gradient is
// row k of D_m^-1; corner 3 has minus their sum.
template <typename TX>
__device__ __forceinline__ void write_corners(double* __restrict__ contrib, int64_t i, double w, const TX* X,
                                              const double* D) {
  double s0 = 0, s1 = 0, s2 = 0;
  double* out = contrib + 12 * i;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double v[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      v[r] = w * ((double)X[3 * r] * D[3 * k] + (double)X[3 * r + 1] * D[3 * k + 1] + (double)X[3 * r + 2] * D[3 * k + 2]);
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

template <typename T>
__device__ __forceinline__ ElemMat<T> load_mat(const double* V, const double* mu, const double* lam,
                                               const double* ka, const double* u, int64_t m, int64_t i) {
  ElemMat<T> e;
  e.V = (T)V[i];
  e.mu = (T)mu[i];
  e.lam = (T)lam[i];
  e.ka = (T)ka[i];
  e.u[0] = (T)u[i];
  e.u[1] = (T)u[m + i];
  e.u[2] = (T)u[2 * m + i];
  return e;
}

}  // namespace emu
