// Per-element device math for the rotation/stretch form of EMU (arXiv 2006.08821).
//
// Conventions (shared with the host side and the C ABI):
//   * 3x3 matrices are row-major arrays of 9 values.
//   * A symmetric stretch S is stored as six coordinates s in the order
//     (xx, yy, zz, yz, xz, xy) with off-diagonals scaled by sqrt(2); the six
//     basis matrices E_k are then orthonormal in the Frobenius metric and
//     |s| = ||S||_F.
//   * F = R S, R a proper rotation, S symmetric positive definite.
//
// The energy is the Sec. 3.1 density (compressible neo-Hookean plus the
// fiber term a u^T F^T F u scaled by kappa). It is evaluated on S because
// Psi(R S) = Psi(S).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace emu {

#define EMU_HD __host__ __device__ __forceinline__

template <typename T> EMU_HD T rsqrt2() { return T(0.70710678118654752440); }

// ---------------------------------------------------------------- 3x3 ------
template <typename T> EMU_HD T det3(const T* A) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// B = A^-1 (returns det A)
template <typename T> EMU_HD T inv3(const T* A, T* B) {
  T c00 = A[4] * A[8] - A[5] * A[7];
  T c01 = A[5] * A[6] - A[3] * A[8];
  T c02 = A[3] * A[7] - A[4] * A[6];
  T det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  T id = T(1) / det;
  B[0] = c00 * id;
  B[1] = (A[2] * A[7] - A[1] * A[8]) * id;
  B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  B[3] = c01 * id;
  B[4] = (A[0] * A[8] - A[2] * A[6]) * id;
  B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  B[6] = c02 * id;
  B[7] = (A[1] * A[6] - A[0] * A[7]) * id;
  B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  return det;
}

template <typename T> EMU_HD void matmul3(const T* A, const T* B, T* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

// C = A^T B
template <typename T> EMU_HD void matTmul3(const T* A, const T* B, T* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) C[3 * r + c] = A[r] * B[c] + A[3 + r] * B[3 + c] + A[6 + r] * B[6 + c];
}

template <typename T> EMU_HD void sym_from_s(const T* s, T* S) {
  const T h = rsqrt2<T>();
  S[0] = s[0];
  S[4] = s[1];
  S[8] = s[2];
  S[5] = S[7] = h * s[3];
  S[2] = S[6] = h * s[4];
  S[1] = S[3] = h * s[5];
}

// s = symvec(sym(M)) for a general M
template <typename T> EMU_HD void s_from_mat(const T* M, T* s) {
  const T h = rsqrt2<T>();
  s[0] = M[0];
  s[1] = M[4];
  s[2] = M[8];
  s[3] = h * (M[5] + M[7]);
  s[4] = h * (M[2] + M[6]);
  s[5] = h * (M[1] + M[3]);
}

// Basis E_k as (row, col, coefficient) entry lists; off-diagonals carry 1/sqrt2
// on both entries. Used with compile-time k so everything folds.
struct SymEntry {
  int a, b;
};
EMU_HD int sym_nent(int k) { return k < 3 ? 1 : 2; }
EMU_HD SymEntry sym_ent(int k, int e) {
  // k: 0 xx, 1 yy, 2 zz, 3 yz, 4 xz, 5 xy
  switch (k) {
    case 0: return {0, 0};
    case 1: return {1, 1};
    case 2: return {2, 2};
    case 3: return e == 0 ? SymEntry{1, 2} : SymEntry{2, 1};
    case 4: return e == 0 ? SymEntry{0, 2} : SymEntry{2, 0};
    default: return e == 0 ? SymEntry{0, 1} : SymEntry{1, 0};
  }
}
template <typename T> EMU_HD T sym_coef(int k) { return k < 3 ? T(1) : rsqrt2<T>(); }

// --------------------------------------------------- material parameters --
template <typename T> struct ElemMat {
  T V;       // rest volume
  T mu, lam; // Lame parameters
  T ka;      // kappa * a_i
  T u[3];    // unit fiber direction
};

// --------------------------------------------------- stretch energy -------
// Psi(S) = mu/2 (tr S^2 - 3) - mu ln J + lam/2 ln^2 J + ka |S u|^2, J = det S.
// Returns +inf (as a huge value) when J <= 0.
template <typename T> EMU_HD T psi_stretch(const T* S, const ElemMat<T>& m) {
  T J = det3(S);
  if (!(J > T(0))) return T(1e30);
  T lnJ = log(J);
  T trS2 = S[0] * S[0] + S[4] * S[4] + S[8] * S[8] + T(2) * (S[1] * S[1] + S[2] * S[2] + S[5] * S[5]);
  T Su0 = S[0] * m.u[0] + S[1] * m.u[1] + S[2] * m.u[2];
  T Su1 = S[3] * m.u[0] + S[4] * m.u[1] + S[5] * m.u[2];
  T Su2 = S[6] * m.u[0] + S[7] * m.u[1] + S[8] * m.u[2];
  return T(0.5) * m.mu * (trS2 - T(3)) - m.mu * lnJ + T(0.5) * m.lam * lnJ * lnJ +
         m.ka * (Su0 * Su0 + Su1 * Su1 + Su2 * Su2);
}

// Rotated-frame first Piola stress Pr = R^T P(R S):
//   Pr = mu S - (mu - lam ln J) S^-1 + 2 ka S u u^T.
// Also returns S^-1 and ln J.
template <typename T> EMU_HD void piola_rotated(const T* S, const ElemMat<T>& m, T* Pr, T* Sinv, T& lnJ) {
  T J = inv3(S, Sinv);
  lnJ = log(J);
  T cf = m.mu - m.lam * lnJ;
  T Su[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) Su[r] = S[3 * r] * m.u[0] + S[3 * r + 1] * m.u[1] + S[3 * r + 2] * m.u[2];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) Pr[3 * r + c] = m.mu * S[3 * r + c] - cf * Sinv[3 * r + c] + T(2) * m.ka * Su[r] * m.u[c];
}

// V * d2Psi/ds2 (6x6, symmetric, stored full row-major) with the definiteness
// fix: the coefficient (mu - lam ln J) of the S^-1 dS S^-1 term is clamped at
// zero; every other term is positive semi-definite by construction, so the
// result is >= V mu I.
//   H_kl = mu d_kl + c tr(T E_k T E_l) + lam tr(T E_k) tr(T E_l)
//          + ka (u^T E_k E_l u + u^T E_l E_k u),  T = S^-1.
template <typename T> EMU_HD void stretch_hessian(const T* Sinv, T lnJ, const ElemMat<T>& m, T* H) {
  T cf = m.mu - m.lam * lnJ;
  cf = cf > T(0) ? cf : T(0);
  T trTE[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    T acc = T(0);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      if (e < sym_nent(k)) {
        SymEntry q = sym_ent(k, e);
        acc += Sinv[3 * q.b + q.a];
      }
    }
    trTE[k] = sym_coef<T>(k) * acc;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
#pragma unroll
    for (int l = k; l < 6; ++l) {
      T tt = T(0), uu = T(0);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (e < sym_nent(k)) {
          SymEntry p = sym_ent(k, e);
#pragma unroll
          for (int f = 0; f < 2; ++f) {
            if (f < sym_nent(l)) {
              SymEntry q = sym_ent(l, f);
              // tr(T e_a e_b^T T e_c e_d^T) = T_bc T_da
              tt += Sinv[3 * p.b + q.a] * Sinv[3 * q.b + p.a];
              // u^T e_a e_b^T e_c e_d^T u = d_bc u_a u_d (+ symmetric partner)
              if (p.b == q.a) uu += m.u[p.a] * m.u[q.b];
              if (q.b == p.a) uu += m.u[q.a] * m.u[p.b];
            }
          }
        }
      }
      T ck = sym_coef<T>(k) * sym_coef<T>(l);
      T h = cf * ck * tt + m.lam * trTE[k] * trTE[l] + m.ka * ck * uu;
      if (k == l) h += m.mu;
      H[6 * k + l] = m.V * h;
      H[6 * l + k] = m.V * h;
    }
  }
}

// V * dPsi/ds: symvec of P_S = mu S - (mu - lam lnJ) S^-1 + ka (S u u^T + u u^T S).
template <typename T> EMU_HD void stretch_gradient(const T* S, const T* Sinv, T lnJ, const ElemMat<T>& m, T* g) {
  T cf = m.mu - m.lam * lnJ;
  T Su[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) Su[r] = S[3 * r] * m.u[0] + S[3 * r + 1] * m.u[1] + S[3 * r + 2] * m.u[2];
  T P[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      P[3 * r + c] = m.mu * S[3 * r + c] - cf * Sinv[3 * r + c] + m.ka * (Su[r] * m.u[c] + m.u[r] * Su[c]);
  T s[6];
  s_from_mat(P, s);
  // s_from_mat symmetrises with 1/sqrt2 (M_ab + M_ba); P is symmetric so the
  // off-diagonals come out as sqrt2 P_ab, the gradient in the s metric.
#pragma unroll
  for (int k = 0; k < 6; ++k) g[k] = m.V * s[k];
}

// ------------------------------------------------------ dense Cholesky ----
// In-place lower Cholesky of an N x N SPD matrix (row-major full storage).
// Returns false if a pivot is not positive.
template <typename T, int N> EMU_HD bool chol(T* A, T* idiag = nullptr) {
  // every loop has a fixed trip count (bounds as conditions), so full
  // unrolling folds all indices and A stays in registers. idiag (optional)
  // receives 1 / L_jj.
  bool ok = true;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T d = A[N * j + j];
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (k < j) d -= A[N * j + k] * A[N * j + k];
    ok = ok & (d > T(0));
    d = d > T(0) ? sqrt(d) : T(1);
    A[N * j + j] = d;
    T id = T(1) / d;
    if (idiag) idiag[j] = id;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (i > j) {
        T v = A[N * i + j];
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (k < j) v -= A[N * i + k] * A[N * j + k];
        A[N * i + j] = v * id;
      }
    }
  }
  return ok;
}

// Solve L x = b in place (L lower, row-major N x N, idiag = 1 / diag(L)).
template <typename T, int N> EMU_HD void fwd_sub_inv(const T* L, const T* idiag, T* x) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T v = x[i];
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (k < i) v -= L[N * i + k] * x[k];
    x[i] = v * idiag[i];
  }
}

// Solve L x = b in place (L lower, row-major N x N).
template <typename T, int N> EMU_HD void fwd_sub(const T* L, T* x) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T v = x[i];
#pragma unroll
    for (int k = 0; k < i; ++k) v -= L[N * i + k] * x[k];
    x[i] = v / L[N * i + i];
  }
}

// ------------------------------------------------------ chart factor -----
// For the elastic Hessian written in rotation/stretch coordinates
// (F = R exp([w]x) S(s)): rotation invariance makes its rotation block zero,
// so in F-space it is  H_el = Z M Z^T,  where M = V d2Psi/ds2 (6x6) and
// Z^T maps an F-space direction dF to its stretch coordinates in the
// (oblique) split R^T dF = [w]x S + dS.  With c = alpha w_i the per-tet
// quasi-Newton block is H_F = c I + Z M Z^T and
//     N := I - c H_F^-1 = Z (Z^T Z + c M^-1)^-1 Z^T = U^T U,
//     U  = L2^-1 L_M^T Z^T,   L_M L_M^T = M,   L2 L2^T = L_M^T Z^T Z L_M + c I,
// a positive semi-definite form without cancellation. This returns the
// world-frame factor Uw (6 x 9, row-major, column index 3r+b) with
// N dF = Uw^T (Uw dF) for world-frame dF.
//
// Stretch coordinates of a rotated-frame Y: k = 2 axial(skew Y),
// ((tr S) I - S) w = k, dS = sym(Y) - sym([w]x S).
template <typename T> EMU_HD void chart_factor(const T* R, const T* S, const T* M6, T c, T* Uw, bool& ok) {
  // Zr: 6 x 9, column (a,b) = stretch coords of e_a e_b^T (rotated frame)
  T Kinv[9];
  {
    T tr = S[0] + S[4] + S[8];
    T Km[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Km[i] = -S[i];
    Km[0] += tr;
    Km[4] += tr;
    Km[8] += tr;
    inv3(Km, Kinv);
  }
  // Y = e_a e_b^T has k = 0 when a = b and k = +-e_c otherwise, so w is
  // +-column c of Kinv; the three [w]x S are formed once (their stretch
  // coordinates ws[c]) and each column of Zr is s(sym Y) -+ ws[c].
  T ws[3][6];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T w0 = Kinv[c], w1 = Kinv[3 + c], w2 = Kinv[6 + c];
    // [w]x S ; [w]x = [[0,-w2,w1],[w2,0,-w0],[-w1,w0,0]]
    T Wm[9];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      Wm[cc] = -w2 * S[3 + cc] + w1 * S[6 + cc];
      Wm[3 + cc] = w2 * S[cc] - w0 * S[6 + cc];
      Wm[6 + cc] = -w1 * S[cc] + w0 * S[3 + cc];
    }
    s_from_mat(Wm, ws[c]);
  }
  const T h = rsqrt2<T>();
  T Zr[6 * 9];  // column 3a + b
#pragma unroll
  for (int kk = 0; kk < 6; ++kk) {
    const T z0 = ws[0][kk], z1 = ws[1][kk], z2 = ws[2][kk];
    Zr[9 * kk + 0] = kk == 0 ? T(1) : T(0);  // (0,0)
    Zr[9 * kk + 4] = kk == 1 ? T(1) : T(0);  // (1,1)
    Zr[9 * kk + 8] = kk == 2 ? T(1) : T(0);  // (2,2)
    Zr[9 * kk + 1] = (kk == 5 ? h : T(0)) + z2;  // (0,1): k = -e_2
    Zr[9 * kk + 3] = (kk == 5 ? h : T(0)) - z2;  // (1,0): k = +e_2
    Zr[9 * kk + 2] = (kk == 4 ? h : T(0)) - z1;  // (0,2): k = +e_1
    Zr[9 * kk + 6] = (kk == 4 ? h : T(0)) + z1;  // (2,0): k = -e_1
    Zr[9 * kk + 5] = (kk == 3 ? h : T(0)) + z0;  // (1,2): k = -e_0
    Zr[9 * kk + 7] = (kk == 3 ? h : T(0)) - z0;  // (2,1): k = +e_0
  }
  // L_M = chol(M)
  T LM[36];
#pragma unroll
  for (int i = 0; i < 36; ++i) LM[i] = M6[i];
  ok = chol<T, 6>(LM);
  // W = L_M^T Zr  (6 x 9)
  T Wf[54];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      T acc = T(0);
#pragma unroll
      for (int k = i; k < 6; ++k) acc += LM[6 * k + i] * Zr[9 * k + j];
      Wf[9 * i + j] = acc;
    }
  // K2 = W W^T + c I, L2 = chol(K2)
  T L2[36];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < 9; ++k) acc += Wf[9 * i + k] * Wf[9 * j + k];
      if (i == j) acc += c;
      L2[6 * i + j] = acc;
      L2[6 * j + i] = acc;
    }
  T id2[6];
  ok = chol<T, 6>(L2, id2) && ok;
  // U = L2^-1 W (column by column forward substitution)
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    T col[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) col[i] = Wf[9 * i + j];
    fwd_sub_inv<T, 6>(L2, id2, col);
#pragma unroll
    for (int i = 0; i < 6; ++i) Wf[9 * i + j] = col[i];
  }
  // world frame: Uw[:, (r,b)] = sum_a U[:, (a,b)] R[r][a]
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        Uw[9 * i + 3 * r + b] = Wf[9 * i + b] * R[3 * r] + Wf[9 * i + 3 + b] * R[3 * r + 1] + Wf[9 * i + 6 + b] * R[3 * r + 2];
}

// x <- x - Uw^T (Uw x)   (applies I - N to a world-frame 9-vector)
template <typename T> EMU_HD void apply_I_minus_N(const T* Uw, T* x) {
  T t[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < 9; ++j) acc += Uw[9 * i + j] * x[j];
    t[i] = acc;
  }
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) acc += Uw[9 * i + j] * t[i];
    x[j] -= acc;
  }
}

// ------------------------------------------------------ polar ------------
// Polar factor of X (det X > 0) by Higham's scaled Newton iteration
// X <- (g X + X^-T / g) / 2 with determinant scaling g = |det X|^(-1/3)
// (N. J. Higham, "Computing the polar decomposition, with applications",
// SIAM J. Sci. Stat. Comput. 7, 1986). Returns the rotation in R and the
// iteration count; ``tol`` bounds the Frobenius change of the last step.
template <typename T> EMU_HD int polar_rotation(const T* X0, T* R, T tol, int max_iter) {
  T X[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) X[i] = X0[i];
  int it = 0;
  for (; it < max_iter; ++it) {
    T Xi[9];
    T det = inv3(X, Xi);
    T g = T(1);
    if (it < 4) {
      T ad = det > T(0) ? det : -det;
      g = T(1) / cbrt(ad);
    }
    T ig = T(1) / g;
    T diff = T(0);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T nx = T(0.5) * (g * X[3 * r + c] + ig * Xi[3 * c + r]);
        T dd = nx - X[3 * r + c];
        diff += dd * dd;
        X[3 * r + c] = nx;
      }
    if (diff <= tol * tol && it >= 1) {
      ++it;
      break;
    }
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = X[i];
  return it;
}

// ================================================================ mixed ===
// FP32 helpers of the mixed path. The state is a unit quaternion q (rotation)
// and E = S - I; every quantity that enters the residual is written as a
// difference-free expression in E so that stiff materials (tiny strains) keep
// their relative precision.

// Quaternion (x, y, z, w), w the scalar part.
struct Quat {
  float x, y, z, w;
};

EMU_HD Quat qmul(Quat a, Quat b) {  // R(a b) = R(a) R(b)
  Quat r;
  r.w = a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z;
  r.x = a.w * b.x + b.w * a.x + a.y * b.z - a.z * b.y;
  r.y = a.w * b.y + b.w * a.y + a.z * b.x - a.x * b.z;
  r.z = a.w * b.z + b.w * a.z + a.x * b.y - a.y * b.x;
  return r;
}

EMU_HD Quat qnormalize(Quat a) {
  float n = rsqrtf(a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w);
  return Quat{a.x * n, a.y * n, a.z * n, a.w * n};
}

// R(q) - I = 2 w [v]x + 2 [v]x^2 for a unit quaternion; accurate for small
// rotations (no 1 - ... cancellation).
template <typename T> EMU_HD void quat_rot_minus_I(T x, T y, T z, T w, T* D) {
  const T xx = x * x, yy = y * y, zz = z * z;
  const T xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
  D[0] = -T(2) * (yy + zz);
  D[1] = T(2) * (xy - wz);
  D[2] = T(2) * (xz + wy);
  D[3] = T(2) * (xy + wz);
  D[4] = -T(2) * (xx + zz);
  D[5] = T(2) * (yz - wx);
  D[6] = T(2) * (xz - wy);
  D[7] = T(2) * (yz + wx);
  D[8] = -T(2) * (xx + yy);
}

template <typename T> EMU_HD void quat_to_R(T x, T y, T z, T w, T* R) {
  quat_rot_minus_I(x, y, z, w, R);
  R[0] += T(1);
  R[4] += T(1);
  R[8] += T(1);
}

// Rotation matrix -> unit quaternion (Shepperd's branch on the largest pivot).
template <typename T> EMU_HD void R_to_quat(const T* R, T* q) {
  const T tr = R[0] + R[4] + R[8];
  if (tr > R[0] && tr > R[4] && tr > R[8]) {
    T s = sqrt(T(1) + tr) * T(2);
    q[3] = T(0.25) * s;
    q[0] = (R[7] - R[5]) / s;
    q[1] = (R[2] - R[6]) / s;
    q[2] = (R[3] - R[1]) / s;
  } else if (R[0] > R[4] && R[0] > R[8]) {
    T s = sqrt(T(1) + R[0] - R[4] - R[8]) * T(2);
    q[3] = (R[7] - R[5]) / s;
    q[0] = T(0.25) * s;
    q[1] = (R[1] + R[3]) / s;
    q[2] = (R[2] + R[6]) / s;
  } else if (R[4] > R[8]) {
    T s = sqrt(T(1) + R[4] - R[0] - R[8]) * T(2);
    q[3] = (R[2] - R[6]) / s;
    q[0] = (R[1] + R[3]) / s;
    q[1] = T(0.25) * s;
    q[2] = (R[5] + R[7]) / s;
  } else {
    T s = sqrt(T(1) + R[8] - R[0] - R[4]) * T(2);
    q[3] = (R[3] - R[1]) / s;
    q[0] = (R[2] + R[6]) / s;
    q[1] = (R[5] + R[7]) / s;
    q[2] = T(0.25) * s;
  }
  if (q[3] < T(0)) {
    q[0] = -q[0];
    q[1] = -q[1];
    q[2] = -q[2];
    q[3] = -q[3];
  }
  T n = T(1) / sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  q[0] *= n;
  q[1] *= n;
  q[2] *= n;
  q[3] *= n;
}

// e2(M) = ((tr M)^2 - tr(M M)) / 2 (second invariant; det(I + M) =
// 1 + tr M + e2(M) + det M).
template <typename T> EMU_HD T inv2(const T* M) {
  const T tr = M[0] + M[4] + M[8];
  const T trMM = M[0] * M[0] + M[4] * M[4] + M[8] * M[8] + T(2) * (M[1] * M[3] + M[2] * M[6] + M[5] * M[7]);
  return T(0.5) * (tr * tr - trMM);
}

// x - log1p(x) without cancellation: series for small |x|.
EMU_HD float x_minus_log1p(float x) {
  if (fabsf(x) < 0.1f) {
    // x^2/2 - x^3/3 + x^4/4 - ... (error < 0.1^10 relative)
    float t = x * x;
    float s = 1.f / 2 - x * (1.f / 3 - x * (1.f / 4 - x * (1.f / 5 - x * (1.f / 6 - x * (1.f / 7 - x * (1.f / 8 - x * (1.f / 9)))))));
    return t * s;
  }
  return x - log1pf(x);
}

// FP64: the series up to x^20 for |x| < 0.05 (next term below 0.05^19 relative).
EMU_HD double x_minus_log1p(double x) {
  if (fabs(x) < 0.05) {
    double s = 1.0 / 20;
    for (int k = 19; k >= 2; --k) s = 1.0 / k - x * s;
    return x * x * s;
  }
  return x - log1p(x);
}

// Stretch quantities from E = S - I (FP32, difference-free):
//   S, S^-1, ln J = log1p(tr E + e2(E) + det E), and S - S^-1 = (2E + E^2) S^-1.
struct StretchE {
  float S[9], Sinv[9], SmSi[9], lnJ;
};

EMU_HD bool stretch_from_E(const float* e6, StretchE& st) {
  float E[9];
  sym_from_s(e6, E);
#pragma unroll
  for (int k = 0; k < 9; ++k) st.S[k] = E[k];
  st.S[0] += 1.f;
  st.S[4] += 1.f;
  st.S[8] += 1.f;
  const float x = (E[0] + E[4] + E[8]) + inv2(E) + det3(E);
  if (!(x > -1.f)) return false;
  st.lnJ = log1pf(x);
  inv3(st.S, st.Sinv);
  float T2[9], EE[9];
  matmul3(E, E, EE);
#pragma unroll
  for (int k = 0; k < 9; ++k) T2[k] = 2.f * E[k] + EE[k];
  matmul3(T2, st.Sinv, st.SmSi);
  return true;
}

// Rotated-frame Piola from E: Pr = mu (S - S^-1) + lam ln J S^-1 + 2 ka S u u^T.
EMU_HD void piola_rotated_E(const StretchE& st, const ElemMat<float>& m, float* Pr) {
  float Su[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) Su[r] = st.S[3 * r] * m.u[0] + st.S[3 * r + 1] * m.u[1] + st.S[3 * r + 2] * m.u[2];
  const float ll = m.lam * st.lnJ;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) Pr[3 * r + c] = m.mu * st.SmSi[3 * r + c] + ll * st.Sinv[3 * r + c] + 2.f * m.ka * Su[r] * m.u[c];
}

// Polar factor of I + Y close to the identity, in FP32 with relative
// precision in Y: I + Y = Rx (I + Ex), Rx returned as a unit quaternion, Ex
// (symmetric) as six stretch coordinates. Newton iteration on the rotation:
// with M = Rx^T (I + Y) = I + Z, the step w solves
// ((2 + tr Z) I - sym Z) w = 2 axial(skew Z) and Rx <- Rx exp([w]x).
// Z = (Rx^T - I) + Y + (Rx^T - I) Y uses the cancellation-free R - I.
EMU_HD int polar_near_identity(const float* Y, Quat& qx, float* e6, int max_iter) {
  qx = Quat{0.f, 0.f, 0.f, 1.f};
  float Z[9];
  int it = 0;
  for (;; ++it) {
    float D[9];
    quat_rot_minus_I(qx.x, qx.y, qx.z, qx.w, D);
    float DT[9] = {D[0], D[3], D[6], D[1], D[4], D[7], D[2], D[5], D[8]};
    float DY[9];
    matmul3(DT, Y, DY);
#pragma unroll
    for (int k = 0; k < 9; ++k) Z[k] = DT[k] + Y[k] + DY[k];
    if (it >= max_iter) break;
    const float k0 = Z[7] - Z[5], k1 = Z[2] - Z[6], k2 = Z[3] - Z[1];
    const float trz = Z[0] + Z[4] + Z[8];
    float Ms[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) Ms[3 * r + c] = -0.5f * (Z[3 * r + c] + Z[3 * c + r]);
    Ms[0] += 2.f + trz;
    Ms[4] += 2.f + trz;
    Ms[8] += 2.f + trz;
    float Mi[9];
    inv3(Ms, Mi);
    const float w0 = Mi[0] * k0 + Mi[1] * k1 + Mi[2] * k2;
    const float w1 = Mi[3] * k0 + Mi[4] * k1 + Mi[5] * k2;
    const float w2 = Mi[6] * k0 + Mi[7] * k1 + Mi[8] * k2;
    const float ang2 = w0 * w0 + w1 * w1 + w2 * w2;
    if (!(ang2 > 1e-16f)) break;  // |w| < 1e-8: converged (also stops on NaN)
    const float ang = sqrtf(ang2);
    float sh, ch;
    sincosf(0.5f * ang, &sh, &ch);
    const float f = sh / ang;
    qx = qnormalize(qmul(qx, Quat{w0 * f, w1 * f, w2 * f, ch}));
  }
  s_from_mat(Z, e6);
  return it;
}

}  // namespace emu
