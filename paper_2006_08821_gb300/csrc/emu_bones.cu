// Device kernels of affine bones and joints (Sec. 3.3 of arXiv 2006.08821).
// The reading and the data layout are described in emu_bones.h.
//
// Every kernel here is small: the per-bone work (one virtual element per
// free bone) runs in one block in FP64 on both precision paths, and the
// joint corrections touch the few vertices of the joint rows plus one pass
// over the vertices. The per-tet work of bone tets stays in the ordinary
// per-tet kernels (their copies of the bone's state).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "emu_bones.h"
#include "emu_kernels.cuh"
#include "emu_math.cuh"
#include "emu_reduce.cuh"

namespace emu {

namespace {

inline int grid_for(int64_t items, int threads, int cap = 4096) {
  int64_t g = (items + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// State of free bone b (its representative tet) in FP64: R, R - I, S, E = S - I.
// ``ident``: the rest state.
__device__ void bone_state(const BoneArgs& a, int b, bool ident, double* R, double* RmI, double* S, double* E) {
  if (ident) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      R[k] = (k % 4 == 0) ? 1.0 : 0.0;
      S[k] = R[k];
      RmI[k] = 0.0;
      E[k] = 0.0;
    }
    return;
  }
  const int64_t i = a.rep[b], m = a.m;
  double sv[6];
  if (a.mixed) {
    const double* o = a.bst + (size_t)b * kBoneStride;
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = o[kBoneR + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) sv[k] = o[kBoneS + k];
  } else {
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = a.R[k * m + i];
#pragma unroll
    for (int k = 0; k < 6; ++k) sv[k] = a.s[k * m + i];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) RmI[k] = R[k] - ((k % 4 == 0) ? 1.0 : 0.0);
#pragma unroll
  for (int k = 0; k < 3; ++k) sv[k] -= 1.0;
  sym_from_s(sv, E);
#pragma unroll
  for (int k = 0; k < 9; ++k) S[k] = E[k] + ((k % 4 == 0) ? 1.0 : 0.0);
}

// ------------------------------------------------------------ bone mean ---
// Partial sums over the tets of free bone b of c_i (G_i q - I), with
// G_i q - I = G_i (q - Q) + (G_i Q - I) (displacement form).
__global__ void __launch_bounds__(256) k_bone_mean(BoneArgs a, const double* __restrict__ q) {
  const int b = blockIdx.x / kBoneMeanBlocks, part = blockIdx.x % kBoneMeanBlocks;
  const int64_t i0 = a.bptr[b], i1 = a.bptr[b + 1], m = a.m;
  double acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.0;
  for (int64_t idx = i0 + (int64_t)part * blockDim.x + threadIdx.x; idx < i1;
       idx += (int64_t)kBoneMeanBlocks * blockDim.x) {
    const int64_t i = a.btets[idx];
    const int4 t = a.tet[i];
    const int64_t v[4] = {t.x, t.y, t.z, t.w};
    double D[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) D[k] = a.Dinv[k * m + i];
    const double ci = a.c[i];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double u3 = q[3 * v[3] + r] - a.Q[3 * v[3] + r];
      double du[3], dQ[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        du[k] = (q[3 * v[k] + r] - a.Q[3 * v[k] + r]) - u3;
        dQ[k] = a.Q[3 * v[k] + r] - a.Q[3 * v[3] + r];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double g0 = dQ[0] * D[c] + dQ[1] * D[3 + c] + dQ[2] * D[6 + c] - (r == c ? 1.0 : 0.0);
        acc[3 * r + c] += ci * (du[0] * D[c] + du[1] * D[3 + c] + du[2] * D[6 + c] + g0);
      }
    }
  }
  block_reduce_write<9>(acc, a.part + (size_t)blockIdx.x * 9);
}

// ------------------------------------------------------------ bone eval ---
__global__ void __launch_bounds__(128) k_bone_eval(BoneArgs a, double* gref_out) {
  __shared__ double sU[kMaxFreeBones][54];   // sqrt(w_b) U_b
  __shared__ double sy[kMaxFreeBones][9];    // w_b y_b
  __shared__ double sg2[kMaxFreeBones];
  __shared__ double sYh[kMaxFreeBones][6][kK];
  __shared__ int sbad;
  const int tid = threadIdx.x;
  if (tid == 0) sbad = 0;
  __syncthreads();
  const bool gref = gref_out != nullptr;
  if (tid < a.nfb) {
    const int b = tid;
    const double ct = a.alpha * a.wb[b];
    double AmI[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) AmI[e] = 0.0;
    for (int k = 0; k < kBoneMeanBlocks; ++k)
#pragma unroll
      for (int e = 0; e < 9; ++e) AmI[e] += a.part[((size_t)b * kBoneMeanBlocks + k) * 9 + e];
#pragma unroll
    for (int e = 0; e < 9; ++e) AmI[e] /= ct;
    double R[9], RmI[9], S[9], E[9], RE[9], Dm[9];
    bone_state(a, b, gref, R, RmI, S, E);
    matmul3(R, E, RE);
#pragma unroll
    for (int k = 0; k < 9; ++k) Dm[k] = AmI[k] - (RmI[k] + RE[k]);  // Abar - F
    ElemMat<double> md;
    md.V = a.Vb[b];
    md.mu = a.mu[b];
    md.lam = a.lam[b];
    md.ka = 0.0;
    md.u[0] = 0.0;
    md.u[1] = 0.0;
    md.u[2] = 1.0;
    double Pr[9], Sinv[9], lnJ, RP[9];
    piola_rotated(S, md, Pr, Sinv, lnJ);
    matmul3(R, Pr, RP);
    double g[9], gg = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      g[k] = md.V * RP[k] - ct * Dm[k];
      gg += g[k] * g[k];
    }
    sg2[b] = gg;
    if (!isfinite(gg)) atomicExch(&sbad, 1);
    if (!gref) {
      double M6[36], U[54];
      stretch_hessian(Sinv, lnJ, md, M6);
      bool ok = true;
      chart_factor(R, S, M6, ct, U, ok);
      if (!ok) atomicExch(&sbad, 1);
      double y[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) y[k] = g[k];
      apply_I_minus_N(U, y);
      double* o = a.bst + (size_t)b * kBoneStride;
      const double sw = sqrt(a.wb[b]);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        y[k] /= ct;
        o[kBoneG + k] = g[k];
        o[kBoneY + k] = y[k];
        sy[b][k] = a.wb[b] * y[k];
      }
#pragma unroll
      for (int k = 0; k < 54; ++k) {
        o[kBoneU + k] = U[k];
        sU[b][k] = sw * U[k];
      }
    }
  }
  __syncthreads();
  if (gref) {
    if (tid == 0) {
      double t = 0.0;
      for (int b = 0; b < a.nfb; ++b) t += sg2[b];
      *gref_out += t;
    }
    return;
  }
  if (tid == 0) {
    double t = 0.0;
    for (int b = 0; b < a.nfb; ++b) t += sg2[b];
    a.sc->gnorm2 += t;
    if (sbad) a.sc->nonfinite = 1;
  }
  // Yh_b[k][16 r + j] = sum_c sqrt(w_b) U_b[k][3 r + c] Gbar_b[3 j + c]
  for (int e = tid; e < a.nfb * 6 * kK; e += blockDim.x) {
    const int b = e / (6 * kK), rem = e % (6 * kK), k = rem / kK, col = rem % kK;
    const int r = col >> 4, j = col & 15;
    const double* gb = a.gbar + (size_t)b * kK;
    sYh[b][k][col] = sU[b][9 * k + 3 * r] * gb[3 * j] + sU[b][9 * k + 3 * r + 1] * gb[3 * j + 1] +
                     sU[b][9 * k + 3 * r + 2] * gb[3 * j + 2];
  }
  __syncthreads();
  for (int e = tid; e < kK * kK; e += blockDim.x) {
    const int row = e / kK, col = e % kK;
    double acc = a.cconst[e];
    for (int b = 0; b < a.nfb; ++b)
#pragma unroll
      for (int k = 0; k < 6; ++k) acc += sYh[b][k][row] * sYh[b][k][col];
    a.cadd[e] = acc;
  }
  for (int e = tid; e < kK; e += blockDim.x) {
    const int r = e >> 4, j = e & 15;
    double acc = 0.0;
    for (int b = 0; b < a.nfb; ++b) {
      const double* gb = a.gbar + (size_t)b * kK;
      acc += sy[b][3 * r] * gb[3 * j] + sy[b][3 * r + 1] * gb[3 * j + 1] + sy[b][3 * r + 2] * gb[3 * j + 2];
    }
    a.cadd[kK * kK + e] = acc;
  }
}

// ------------------------------------------------------------ bone dir ----
__global__ void k_bone_dir(BoneArgs a, const double* __restrict__ z, double* gtd_out) {
  __shared__ double sgtd[kMaxFreeBones];
  const int b = threadIdx.x;
  if (b < a.nfb) {
    double* o = a.bst + (size_t)b * kBoneStride;
    const double* gb = a.gbar + (size_t)b * kK;
    double v[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double x = 0.0;
        for (int j = 0; j < 16; ++j) x += z[16 * r + j] * gb[3 * j + c];
        v[3 * r + c] = x;
      }
    apply_I_minus_N(o + kBoneU, v);
    double gtd = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double d = -(o[kBoneY + k] + v[k]);
      o[kBoneD + k] = d;
      gtd += o[kBoneG + k] * d;
    }
    sgtd[b] = gtd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < a.nfb; ++k) t += sgtd[k];
    *gtd_out = t;
  }
}

// ------------------------------------------------------------ line search --
template <typename TQ>
__global__ void __launch_bounds__(256) k_bone_ls(BoneArgs a, const TQ* __restrict__ dq32, double rho,
                                                 double* __restrict__ out) {
  __shared__ double sFmI[kMaxFreeBones][9], sd[kMaxFreeBones][9];
  double acc[kLsNV];
#pragma unroll
  for (int k = 0; k < kLsNV; ++k) acc[k] = 0.0;
  const double s0 = a.sc->sigma_start;
  if (threadIdx.x < a.nfb) {
    const int b = threadIdx.x;
    double R[9], RmI[9], S[9], E[9], RE[9];
    bone_state(a, b, false, R, RmI, S, E);
    matmul3(R, E, RE);
    const double* d = a.bst + (size_t)b * kBoneStride + kBoneD;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      sFmI[b][k] = RmI[k] + RE[k];  // F_b - I
      sd[b][k] = d[k];
    }
    if (blockIdx.x == 0) {
      // the bone's elastic energy change, term by term (one evaluation for all its tets)
      double Sinv[9], Rtd[9], M[9];
      const double lnJ = log(inv3(S, Sinv));
      matTmul3(R, d, Rtd);
      matmul3(Sinv, Rtd, M);
      const double trM = M[0] + M[4] + M[8], e2 = inv2(M), detM = det3(M);
      double FFd = 0.0, dd = 0.0;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        FFd += (S[k] - Sinv[k]) * Rtd[k];
        dd += d[k] * d[k];
      }
      double sig = s0;
      for (int j = 0; j < kLsTrials; ++j) {
        const double x = sig * trM + sig * sig * e2 + sig * sig * sig * detM;
        if (x > -1.0) {
          const double dl = log1p(x);
          const double nh = sig * FFd + 0.5 * sig * sig * dd - sig * sig * e2 - sig * sig * sig * detM + x_minus_log1p(x);
          acc[j] += a.Vb[b] * (a.mu[b] * nh + 0.5 * a.lam[b] * dl * (2.0 * lnJ + dl));
        } else {
          acc[j] += 1e300;
        }
        sig *= rho;
      }
    }
  }
  __syncthreads();
  // ACAP coefficients of the bones' tets: D = (G q - I) - (F_b - I), dD = G dq - d_b
  const int64_t m = a.m, nbt = a.bptr[a.nfb];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nbt; idx += (int64_t)gridDim.x * blockDim.x) {
    int b = 0;
    while (b + 1 < a.nfb && idx >= a.bptr[b + 1]) ++b;
    const int64_t i = a.btets[idx];
    const int4 t = a.tet[i];
    const int64_t v[4] = {t.x, t.y, t.z, t.w};
    double D[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) D[k] = a.Dinv[k * m + i];
    double cDd = 0.0, cdd = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double u3 = a.q[3 * v[3] + r] - a.Q[3 * v[3] + r];
      const double w3 = (double)dq32[3 * v[3] + r];
      double du[3], dQ[3], dw[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        du[k] = (a.q[3 * v[k] + r] - a.Q[3 * v[k] + r]) - u3;
        dQ[k] = a.Q[3 * v[k] + r] - a.Q[3 * v[3] + r];
        dw[k] = (double)dq32[3 * v[k] + r] - w3;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double AmI = du[0] * D[c] + du[1] * D[3 + c] + du[2] * D[6 + c] +
                           (dQ[0] * D[c] + dQ[1] * D[3 + c] + dQ[2] * D[6 + c] - (r == c ? 1.0 : 0.0));
        const double dA = dw[0] * D[c] + dw[1] * D[3 + c] + dw[2] * D[6 + c];
        const double Dm = AmI - sFmI[b][3 * r + c], dD = dA - sd[b][3 * r + c];
        cDd += Dm * dD;
        cdd += dD * dD;
      }
    }
    const double ci = a.c[i];
    acc[kLsTrials] += ci * cDd;
    acc[kLsTrials + 1] += ci * cdd;
  }
  block_reduce_write<kLsNV>(acc, out + (size_t)blockIdx.x * kLsNV);
}

// ------------------------------------------------------------ bone state --
__global__ void k_bone_update(BoneArgs a) {
  const int b = threadIdx.x;
  const double sig = a.sc->sigma;
  if (b >= a.nfb || sig == 0.0) return;
  double* o = a.bst + (size_t)b * kBoneStride;
  double R[9], sv[6], S[9], Rtd[9], X[9], Rx[9], Rn[9], Sn[9], sn[6];
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = o[kBoneR + k];
#pragma unroll
  for (int k = 0; k < 6; ++k) sv[k] = o[kBoneS + k];
  sym_from_s(sv, S);
  matTmul3(R, o + kBoneD, Rtd);
#pragma unroll
  for (int k = 0; k < 9; ++k) X[k] = S[k] + sig * Rtd[k];
  polar_rotation(X, Rx, 1e-15, 40);
  matTmul3(Rx, X, Sn);
  s_from_mat(Sn, sn);
  matmul3(R, Rx, Rn);
#pragma unroll
  for (int k = 0; k < 9; ++k) o[kBoneR + k] = Rn[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) o[kBoneS + k] = sn[k];
}

__global__ void k_bone_state_from_tets(BoneArgs a) {
  const int b = threadIdx.x;
  if (b >= a.nfb) return;
  const int64_t i = a.rep[b], m = a.m;
  double* o = a.bst + (size_t)b * kBoneStride;
#pragma unroll
  for (int k = 0; k < 9; ++k) o[kBoneR + k] = a.R[k * m + i];
#pragma unroll
  for (int k = 0; k < 6; ++k) o[kBoneS + k] = a.s[k * m + i];
}

__global__ void __launch_bounds__(256) k_bone_state_to_tets(BoneArgs a, const int32_t* __restrict__ tkind) {
  const int64_t m = a.m;
  double* R = const_cast<double*>(a.R);
  double* s = const_cast<double*>(a.s);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t kind = tkind[i];
    if (kind == kTetDeformable) continue;
    if (kind >= 0) {
      const double* o = a.bst + (size_t)kind * kBoneStride;
#pragma unroll
      for (int k = 0; k < 9; ++k) R[k * m + i] = o[kBoneR + k];
#pragma unroll
      for (int k = 0; k < 6; ++k) s[k * m + i] = o[kBoneS + k];
    } else {  // tet of a pinned bone: F = I
#pragma unroll
      for (int k = 0; k < 9; ++k) R[k * m + i] = (k % 4 == 0) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) s[k * m + i] = k < 3 ? 1.0 : 0.0;
    }
  }
}

// ------------------------------------------------------------ joints ------
// J x (npts x 3) for an n x 3 field, summed over all J vertices by one
// block; then lam = Sinv (J x).
template <typename T>
__global__ void __launch_bounds__(256) k_joint_lambda(JointArgs j, const T* __restrict__ x) {
  __shared__ double sJx[kMaxJointPts * 3];
  double acc[kMaxJointPts * 3];
#pragma unroll
  for (int k = 0; k < kMaxJointPts * 3; ++k) acc[k] = 0.0;
  const int np = j.npts;
  for (int vi = threadIdx.x; vi < j.njv; vi += blockDim.x) {
    const int64_t v = j.jv[vi];
    const double x0 = (double)x[3 * v], x1 = (double)x[3 * v + 1], x2 = (double)x[3 * v + 2];
#pragma unroll
    for (int r = 0; r < kMaxJointPts; ++r) {
      if (r < np) {
        const double wv = j.jw[(size_t)vi * np + r];
        acc[3 * r] += wv * x0;
        acc[3 * r + 1] += wv * x1;
        acc[3 * r + 2] += wv * x2;
      }
    }
  }
  block_reduce_write<kMaxJointPts * 3>(acc, sJx);
  __syncthreads();
  for (int e = threadIdx.x; e < np * 3; e += blockDim.x) {
    const int r = e / 3, c = e % 3;
    double l = 0.0;
    for (int k = 0; k < np; ++k) l += j.Sinv[r * np + k] * sJx[3 * k + c];
    j.lam[e] = l;
  }
}

// x -= Y lam (n x 3)
template <typename T>
__global__ void __launch_bounds__(256) k_joint_apply(JointArgs j, int64_t n, T* __restrict__ x) {
  __shared__ double sl[kMaxJointPts * 3];
  const int np = j.npts;
  if (threadIdx.x < np * 3) sl[threadIdx.x] = j.lam[threadIdx.x];
  __syncthreads();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    double d0 = 0.0, d1 = 0.0, d2 = 0.0;
    for (int r = 0; r < np; ++r) {
      const double y = sizeof(T) == 8 ? j.Y64[v * 16 + r] : (double)j.Y32[v * 16 + r];
      d0 += y * sl[3 * r];
      d1 += y * sl[3 * r + 1];
      d2 += y * sl[3 * r + 2];
    }
    x[3 * v] -= (T)d0;
    x[3 * v + 1] -= (T)d1;
    x[3 * v + 2] -= (T)d2;
  }
}

// r <- r - J_f^T (J_f J_f^T)^-1 J_f r on the free J vertices; their |r_p|^2 into out3
__global__ void __launch_bounds__(256) k_joint_rproj(JointArgs j, double* __restrict__ r64, float* __restrict__ r32,
                                                     double* __restrict__ out3) {
  __shared__ double sJr[kMaxJointPts * 3];
  __shared__ double smu[kMaxJointPts * 3];
  __shared__ double sn[3];
  const int np = j.npts;
  double acc[kMaxJointPts * 3];
#pragma unroll
  for (int k = 0; k < kMaxJointPts * 3; ++k) acc[k] = 0.0;
  for (int vi = threadIdx.x; vi < j.njv; vi += blockDim.x) {
    if (!j.jfree[vi]) continue;
    const int64_t v = j.jv[vi];
    const double x0 = r64[3 * v], x1 = r64[3 * v + 1], x2 = r64[3 * v + 2];
#pragma unroll
    for (int r = 0; r < kMaxJointPts; ++r) {
      if (r < np) {
        const double wv = j.jw[(size_t)vi * np + r];
        acc[3 * r] += wv * x0;
        acc[3 * r + 1] += wv * x1;
        acc[3 * r + 2] += wv * x2;
      }
    }
  }
  block_reduce_write<kMaxJointPts * 3>(acc, sJr);
  __syncthreads();
  for (int e = threadIdx.x; e < np * 3; e += blockDim.x) {
    const int r = e / 3, c = e % 3;
    double l = 0.0;
    for (int k = 0; k < np; ++k) l += j.JJinv[r * np + k] * sJr[3 * k + c];
    smu[e] = l;
  }
  __syncthreads();
  double nrm[3] = {0.0, 0.0, 0.0};
  for (int vi = threadIdx.x; vi < j.njv; vi += blockDim.x) {
    if (!j.jfree[vi]) continue;
    const int64_t v = j.jv[vi];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double x = r64[3 * v + c];
      for (int r = 0; r < np; ++r) x -= j.jw[(size_t)vi * np + r] * smu[3 * r + c];
      r64[3 * v + c] = x;
      if (r32) r32[3 * v + c] = (float)x;
      nrm[c] += x * x;
    }
  }
  block_reduce_write<3>(nrm, sn);
  __syncthreads();
  if (threadIdx.x < 3) out3[threadIdx.x] += sn[threadIdx.x];
}

// out[r * 16 + k] = sum over J vertices of jw[vi][r] X[v][k]
__global__ void __launch_bounds__(256) k_joint_dot16(JointArgs j, const double* __restrict__ X, double* out) {
  const int np = j.npts;
  const int r = threadIdx.x >> 4, k = threadIdx.x & 15;
  if (r >= np) return;
  double acc = 0.0;
  for (int vi = 0; vi < j.njv; ++vi) acc += j.jw[(size_t)vi * np + r] * X[(int64_t)j.jv[vi] * 16 + k];
  out[r * 16 + k] = acc;
}

__global__ void __launch_bounds__(256) k_joint_sub16_Y(JointArgs j, int64_t n, const double* __restrict__ M,
                                                       double* __restrict__ X) {
  const int np = j.npts;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * 16; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = e >> 4;
    const int k = (int)(e & 15);
    double d = 0.0;
    for (int r = 0; r < np; ++r) d += j.Y64[v * 16 + r] * M[r * 16 + k];
    X[e] -= d;
  }
}

__global__ void __launch_bounds__(256) k_joint_sub16_J(JointArgs j, const double* __restrict__ M, double* __restrict__ X) {
  const int np = j.npts;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)j.njv * 16;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int vi = (int)(e >> 4), k = (int)(e & 15);
    if (!j.jfree[vi]) continue;
    double d = 0.0;
    for (int r = 0; r < np; ++r) d += j.jw[(size_t)vi * np + r] * M[r * 16 + k];
    X[(int64_t)j.jv[vi] * 16 + k] -= d;
  }
}

// ------------------------------------------------------------ final solve --
__global__ void __launch_bounds__(256) k_final_set_bones(BoneArgs a, FinalArgs f, double* __restrict__ q) {
  __shared__ double sF[9], st[3];
  const int b = blockIdx.x;
  if (threadIdx.x == 0) {
    double R[9], RmI[9], S[9], E[9];
    bone_state(a, b, false, R, RmI, S, E);
    matmul3(R, S, sF);
  }
  __syncthreads();
  const int64_t i0 = f.bvptr[b], i1 = f.bvptr[b + 1];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t k = i0 + threadIdx.x; k < i1; k += blockDim.x) {
    const int64_t v = f.bvert[k];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      acc[r] += q[3 * v + r] - (sF[3 * r] * a.Q[3 * v] + sF[3 * r + 1] * a.Q[3 * v + 1] + sF[3 * r + 2] * a.Q[3 * v + 2]);
  }
  block_reduce_write<3>(acc, st);
  __syncthreads();
  const double inv = 1.0 / (double)(i1 - i0);
  for (int64_t k = i0 + threadIdx.x; k < i1; k += blockDim.x) {
    const int64_t v = f.bvert[k];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      q[3 * v + r] = sF[3 * r] * a.Q[3 * v] + sF[3 * r + 1] * a.Q[3 * v + 1] + sF[3 * r + 2] * a.Q[3 * v + 2] + st[r] * inv;
  }
}

__global__ void __launch_bounds__(256) k_final_mask(const uint8_t* __restrict__ fin_fixed, int64_t n, double* __restrict__ r) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (fin_fixed[v]) r[3 * v] = r[3 * v + 1] = r[3 * v + 2] = 0.0;
}

__global__ void __launch_bounds__(256) k_final_tstep(FinalArgs f, JointArgs j, const double* __restrict__ r,
                                                     const double* __restrict__ q) {
  __shared__ double sR[kMaxFreeBones * 3];
  __shared__ double sJq[kMaxJointPts * 3];
  for (int b = 0; b < f.nfb; ++b) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t k = f.bvptr[b] + threadIdx.x; k < f.bvptr[b + 1]; k += blockDim.x) {
      const int64_t v = f.bvert[k];
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] += r[3 * v + c];
    }
    block_reduce_write<3>(acc, sR + 3 * b);
    __syncthreads();
  }
  {
    const int np = j.npts;
    double acc[kMaxJointPts * 3];
#pragma unroll
    for (int k = 0; k < kMaxJointPts * 3; ++k) acc[k] = 0.0;
    for (int vi = threadIdx.x; vi < j.njv; vi += blockDim.x) {
      const int64_t v = j.jv[vi];
#pragma unroll
      for (int rr = 0; rr < kMaxJointPts; ++rr) {
        if (rr < np) {
          const double wv = j.jw[(size_t)vi * np + rr];
#pragma unroll
          for (int c = 0; c < 3; ++c) acc[3 * rr + c] += wv * q[3 * v + c];
        }
      }
    }
    block_reduce_write<kMaxJointPts * 3>(acc, sJq);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // gradient of E in t_b: -(sum of the residual b - K q over bone b's rows)
    // + kj sum_r (J zeta_b)_r (J q)_r; the step is -A^-1 gradient
    double grad[kMaxFreeBones * 3];
    for (int b = 0; b < f.nfb; ++b)
      for (int c = 0; c < 3; ++c) {
        double gj = 0.0;
        for (int rr = 0; rr < j.npts; ++rr) gj += f.sgn[rr * kMaxFreeBones + b] * sJq[3 * rr + c];
        grad[3 * b + c] = -sR[3 * b + c] + f.kj * gj;
      }
    for (int b = 0; b < f.nfb; ++b)
      for (int c = 0; c < 3; ++c) {
        double d = 0.0;
        for (int b2 = 0; b2 < f.nfb; ++b2) d += f.Ainv[b * kMaxFreeBones + b2] * grad[3 * b2 + c];
        f.dt[3 * b + c] = -d;
      }
  }
}

__global__ void __launch_bounds__(256) k_final_apply(FinalArgs f, int64_t n, double* __restrict__ q) {
  __shared__ double sdt[kMaxFreeBones * 3];
  if (threadIdx.x < 3 * f.nfb) sdt[threadIdx.x] = f.dt[threadIdx.x];
  __syncthreads();
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    double d0 = 0.0, d1 = 0.0, d2 = 0.0;
    for (int b = 0; b < f.nfb; ++b) {
      const double z = f.zeta[v * 16 + b];
      d0 += z * sdt[3 * b];
      d1 += z * sdt[3 * b + 1];
      d2 += z * sdt[3 * b + 2];
    }
    q[3 * v] += d0;
    q[3 * v + 1] += d1;
    q[3 * v + 2] += d2;
  }
}

}  // namespace

// ------------------------------------------------------------ launchers ---
void launch_bone_mean(const BoneArgs& a, const double* q, cudaStream_t st) {
  if (a.nfb <= 0) return;
  k_bone_mean<<<a.nfb * kBoneMeanBlocks, 256, 0, st>>>(a, q);
}

void launch_bone_eval(const BoneArgs& a, double* gref_out, cudaStream_t st) {
  k_bone_eval<<<1, 128, 0, st>>>(a, gref_out);
}

void launch_bone_dir(const BoneArgs& a, const double* z, double* gtd_out, cudaStream_t st) {
  k_bone_dir<<<1, 32, 0, st>>>(a, z, gtd_out);
}

void launch_bone_ls(const BoneArgs& a, const float* dq32, double rho, double* partials_out, cudaStream_t st) {
  k_bone_ls<float><<<kBoneLsBlocks, 256, 0, st>>>(a, dq32, rho, partials_out);
}

void launch_bone_ls(const BoneArgs& a, const double* dq64, double rho, double* partials_out, cudaStream_t st) {
  k_bone_ls<double><<<kBoneLsBlocks, 256, 0, st>>>(a, dq64, rho, partials_out);
}

void launch_bone_update(const BoneArgs& a, cudaStream_t st) {
  if (a.nfb <= 0) return;
  k_bone_update<<<1, 32, 0, st>>>(a);
}

void launch_bone_state_from_tets(const BoneArgs& a, cudaStream_t st) {
  if (a.nfb <= 0) return;
  k_bone_state_from_tets<<<1, 32, 0, st>>>(a);
}

void launch_bone_state_to_tets(const BoneArgs& a, const int32_t* tkind, cudaStream_t st) {
  k_bone_state_to_tets<<<grid_for(a.m, 256), 256, 0, st>>>(a, tkind);
}

void launch_joint_project(const JointArgs& j, int64_t n, double* x64, float* x32, cudaStream_t st) {
  if (j.npts <= 0) return;
  if (x64) {
    k_joint_lambda<double><<<1, 256, 0, st>>>(j, x64);
    k_joint_apply<double><<<grid_for(n, 256), 256, 0, st>>>(j, n, x64);
  } else {
    k_joint_lambda<float><<<1, 256, 0, st>>>(j, x32);
    k_joint_apply<float><<<grid_for(n, 256), 256, 0, st>>>(j, n, x32);
  }
}

void launch_joint_rproj(const JointArgs& j, double* r64, float* r32, double* out3, cudaStream_t st) {
  if (j.npts <= 0) return;
  k_joint_rproj<<<1, 256, 0, st>>>(j, r64, r32, out3);
}

void launch_joint_dot16(const JointArgs& j, const double* X, double* out, cudaStream_t st) {
  k_joint_dot16<<<1, 256, 0, st>>>(j, X, out);
}

void launch_joint_sub16(const JointArgs& j, int64_t n, const double* M, int use_jw, double* X, cudaStream_t st) {
  if (use_jw)
    k_joint_sub16_J<<<grid_for((int64_t)j.njv * 16, 256), 256, 0, st>>>(j, M, X);
  else
    k_joint_sub16_Y<<<grid_for(n * 16, 256), 256, 0, st>>>(j, n, M, X);
}

void launch_final_set_bones(const BoneArgs& b, const FinalArgs& f, double* q, cudaStream_t st) {
  if (f.nfb <= 0) return;
  k_final_set_bones<<<f.nfb, 256, 0, st>>>(b, f, q);
}

void launch_final_mask(const FinalArgs& f, int64_t n, double* r, cudaStream_t st) {
  k_final_mask<<<grid_for(n, 256), 256, 0, st>>>(f.fin_fixed, n, r);
}

void launch_final_tstep(const FinalArgs& f, const JointArgs& j, const double* r, const double* q, cudaStream_t st) {
  if (f.nfb <= 0) return;
  k_final_tstep<<<1, 256, 0, st>>>(f, j, r, q);
}

void launch_final_apply(const FinalArgs& f, int64_t n, double* q, cudaStream_t st) {
  if (f.nfb <= 0) return;
  k_final_apply<<<grid_for(n, 256), 256, 0, st>>>(f, n, q);
}

}  // namespace emu
