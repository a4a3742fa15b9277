// Affine bones and joints of Sec. 3.3 (arXiv 2006.08821) on the device.
//
// Reading of the section (shared with the FP64 oracle of the test suite):
//   * every tet of bone b uses the bone's single deformation gradient F_b;
//     a bone whose vertices are all pinned keeps F_b = I and is no variable;
//   * during Newton the bone rows G_i q = F_b are a penalty (slack eps_bone
//     < 0): each bone tet's ACAP weight grows by Vbar / |eps_bone| (Vbar the
//     mean rest volume), in the coupling matrix and in E_C alike;
//   * joint rows: at each joint point p the least-squares affine fits of the
//     two bones' vertex positions, evaluated at p, coincide (a hinge has two
//     points on its axis, a ball joint one); during Newton they are hard;
//   * after convergence one final coupling solve makes every bone's vertices
//     affine, q_v = F_b Q_v + t_b, and turns the joints into a penalty
//     Vbar^(1/3) / |eps_joint| on |J q|^2.
//
// GPU layout. The tets of a free bone keep identical copies of the bone's
// (R, S) state, so the line search, the update and the right-hand sides treat
// them as ordinary tets. The Newton variable of the bone is one virtual
// element: volume V_b = sum V_i, weight w_b = sum w_i, mode gradients
// Gbar_b = sum w_i Gamma_i / w_b, and the weighted mean Abar_b of the bone's
// G_i q in place of its own gather. The capacitance keeps its Gram form:
//   C = sum_deformable w_i Gamma_i^T N_i Gamma_i + sum_pinned-bone-tets
//       w_i Gamma_i^T Gamma_i + sum_b [ sum_{i in b} w_i (Gamma_i - Gbar_b)^T
//       (Gamma_i - Gbar_b) + w_b Gbar_b^T N_b Gbar_b ],
// whose two bone sums over tets are constant (formed at setup).
//
// Joint rows J (one scalar row per joint point, the same for the three
// coordinates) are imposed after every coupling solve by the exact
// correction x <- x - Y S^-1 (J x - j), Y = L^-1 J_f^T, S = J_f Y, formed at
// setup by CG solves.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "emu_internal.h"

namespace emu {

constexpr int kMaxFreeBones = 4;      // 3 scalar basis columns per free bone of the 16
constexpr int kMaxJointPts = 16;      // joint points (a hinge has 2, a ball joint 1)
constexpr int kBoneMeanBlocks = 32;   // blocks per free bone of the Abar reduction
constexpr int kBoneStride = 96;       // per free bone: g 9, y 9, U 54, d 9, R 9, s 6 (FP64)
constexpr int kBoneG = 0, kBoneY = 9, kBoneU = 18, kBoneD = 72, kBoneR = 81, kBoneS = 90;

// tkind[i]: kind of tet i
constexpr int32_t kTetDeformable = -1;  // an ordinary tet (its own Newton variable)
constexpr int32_t kTetPinnedBone = -2;  // a tet of a bone whose vertices are all pinned
                                        // b >= 0: a tet of free bone b

// Where a free bone's state (R_b, S_b) lives: on the FP64 path in the FP64
// (R, s) of its tets (identical copies); on the mixed path in FP64 in the
// bone's own iteration state (kBoneR, kBoneS), updated by launch_bone_update,
// because an FP32 rotation of a bone, whose ACAP weight carries the
// 1/|eps_bone| penalty, leaves a gradient error far above 1e-6.
struct BoneArgs {
  int nfb;                             // free bones
  int mixed;                           // 1: state in bst (mixed path), 0: in R, s of the rep tets
  int64_t m, n;
  const int4* tet;
  const double* Dinv;                  // 9 m FP64 structure of arrays
  const double* c;                     // m: alpha w_i (bone tets: with the penalty)
  const double* q;                     // 3 n
  const double* Q;                     // 3 n rest positions
  const double* R;                     // FP64 state (mixed == 0)
  const double* s;
  const float4* quat;                  // mixed state (mixed == 1)
  const float* E;
  const int32_t* btets;                // tets of the free bones, bone after bone
  int32_t bptr[kMaxFreeBones + 1];     // offsets into btets
  int32_t rep[kMaxFreeBones];          // a tet of each free bone (its state is the bone's)
  double Vb[kMaxFreeBones], wb[kMaxFreeBones], mu[kMaxFreeBones], lam[kMaxFreeBones];
  double alpha;
  const double* gbar;                  // nfb x 48: Gbar_b[(3 j + c)] = d phi_j / dx_c
  const double* cconst;                // 48 x 48 constant part of C (By part none)
  double* part;                        // nfb x kBoneMeanBlocks x 9 partial sums
  double* cadd;                        // 48 x 48 + 48 added to the capacitance and B y
  double* bst;                         // nfb x kBoneStride iteration state
  DevScalars* sc;
};

// sum over each free bone's tets of c_i (G_i q - I), per-block partials
void launch_bone_mean(const BoneArgs& a, const double* q, cudaStream_t st);
// The virtual elements: gradient, chart factor, y, their |g|^2 added to
// sc->gnorm2 and their terms of C and B y (plus the constant) in cadd. With
// gref_out non-null, only |g(F = I)|^2 of the bones is added to *gref_out.
void launch_bone_eval(const BoneArgs& a, double* gref_out, cudaStream_t st);
// d_b = -(y_b + (I - N_b) Gbar_b z) per free bone; sum_b g_b . d_b into *gtd_out.
void launch_bone_dir(const BoneArgs& a, const double* z, double* gtd_out, cudaStream_t st);
// Line-search terms of the free bones in FP64 (both paths): each
// bone's V_b [Psi(F_b + s_j d_b) - Psi(F_b)] for the kLsTrials trial steps
// s_j = sigma_start rho^j, and over the bones' tets the ACAP coefficients
// sum c_i D_i . dD_i and sum c_i |dD_i|^2 (D_i = G_i q - F_b, dD_i = G_i dq
// - d_b). Written as kBoneLsBlocks block partials of kLsNV values.
constexpr int kBoneLsBlocks = 32;
void launch_bone_ls(const BoneArgs& a, const float* dq32, double rho, double* partials_out, cudaStream_t st);
void launch_bone_ls(const BoneArgs& a, const double* dq64, double rho, double* partials_out, cudaStream_t st);
// F' = R (S + sigma R^T d_b) per free bone, polar re-extraction in FP64, into
// the bone state (mixed path; sigma from sc, nothing when it is 0).
void launch_bone_update(const BoneArgs& a, cudaStream_t st);
// Bone state <- the FP64 (R, s) of each free bone's representative tet.
void launch_bone_state_from_tets(const BoneArgs& a, cudaStream_t st);
// FP64 (R, s) of every free bone's tet <- the bone state (a.R, a.s written);
// tets of pinned bones <- R = I, S = I.
void launch_bone_state_to_tets(const BoneArgs& a, const int32_t* tkind, cudaStream_t st);

struct JointArgs {
  int npts;                            // joint points (rows of J)
  int njv;                             // vertices with a non-zero J entry
  const int32_t* jv;                   // njv vertex ids
  const double* jw;                    // njv x npts weights (vertex-major)
  const uint8_t* jfree;                // njv: 1 if the vertex is not pinned
  const double* Sinv;                  // npts x npts: (J_f Y)^-1
  const double* JJinv;                 // npts x npts: (J_f J_f^T)^-1
  const double* Y64;                   // n x 16: column r = L^-1 J_f^T e_r (zero on pins)
  const float* Y32;                    // the same in FP32
  double* lam;                         // 16 x 3 multipliers of the last projection
};

// x <- x - Y S^-1 (J x) for an n x 3 field x (FP64 or FP32): after it J x = 0,
// the joint rows of the Newton-phase coupling solve (positions: J q = 0;
// changes dq, corrections: homogeneous).
void launch_joint_project(const JointArgs& j, int64_t n, double* x64, float* x32, cudaStream_t st);
// Residual r of the joint-constrained coupling problem, projected onto the
// null space of J_f: r <- r - J_f^T (J_f J_f^T)^-1 J_f r at the J vertices
// (r64 and, when non-null, its FP32 copy r32), and sum_{free J vertices}
// |r_p|^2 per coordinate added to out3 (the residual kernel leaves those
// vertices out of its sums).
void launch_joint_rproj(const JointArgs& j, double* r64, float* r32, double* out3, cudaStream_t st);
// (J X) for an n x 16 field X into out (npts x 16, row-major), one block.
void launch_joint_dot16(const JointArgs& j, const double* X, double* out, cudaStream_t st);
// X[v][k] -= sum_r W[v][r] M[r][k] for n x 16 fields: W = Y64 (Sinv-weighted
// multipliers, constrained projection) or, with use_jw, the J vertices'
// weights (Euclidean projection onto the null space of J_f).
void launch_joint_sub16(const JointArgs& j, int64_t n, const double* M, int use_jw, double* X, cudaStream_t st);

// Final coupling solve of Sec. 3.3 (bone rows hard, joints as a penalty).
struct FinalArgs {
  int nfb, npts;
  const int32_t* bvert;                // vertices of the free bones, bone after bone
  int32_t bvptr[kMaxFreeBones + 1];
  const double* zeta;                  // n x 16: column b = response to translating bone b
  double Ainv[kMaxFreeBones * kMaxFreeBones];  // (zeta^T L zeta + kj s^T s)^-1
  double sgn[kMaxJointPts * kMaxFreeBones];    // (J zeta_b)_r
  double kj;                           // joint penalty Vbar^(1/3) / |eps_joint|
  double* dt;                          // nfb x 3 translation steps
  const uint8_t* fin_fixed;            // n: pinned in the final solve (pins and bone vertices)
};
// Every free bone's vertices to F_b Q_v + t_b, t_b their mean offset from F_b Q_v.
void launch_final_set_bones(const BoneArgs& b, const FinalArgs& f, double* q, cudaStream_t st);
// r = 0 on the rows pinned in the final solve.
void launch_final_mask(const FinalArgs& f, int64_t n, double* r, cudaStream_t st);
// Translation step from the residual r = b - K q (all rows) and J q.
void launch_final_tstep(const FinalArgs& f, const JointArgs& j, const double* r, const double* q, cudaStream_t st);
// q += sum_b zeta_b dt_b.
void launch_final_apply(const FinalArgs& f, int64_t n, double* q, cudaStream_t st);

}  // namespace emu
