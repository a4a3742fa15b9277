// Mixed-precision (FP32 per tet, FP64 global) kernels of the Newton iteration.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "emu_bones.h"
#include "emu_internal.h"

namespace emu {

// Device arrays of the mixed path. Per-tet constants and the stretch state
// are FP32; positions q and every global sum are FP64. The discrete operator
// G is defined by the FP32 D_m^-1 values, and the host builds the FP64 ACAP
// Laplacian from the same rounded values, so both precisions see one mesh.
struct MixArgs {
  int64_t m, n;
  const int4* tet;
  const float* Dinv;   // 9m
  const float* V;      // m
  const float* c;      // m  alpha w
  const float* w;      // m
  const float* sw = nullptr;  // m: sqrt(w), for the tcgen05 capacitance kernel
  const float* mu;     // m
  const float* lam;    // m
  const float* ka;     // m  kappa a
  const float* u;      // 3m
  const float* gam;    // 48m
  float4* quat;        // m  rotation (x, y, z, w)
  float* E;            // 6m stretch coordinates of S - I
  const double* q;     // 3n
  const double* Q;     // 3n rest positions
  // displacement q - Q as an unevaluated float pair (hi + lo, 3n each),
  // refreshed from q before every gradient: the per-tet kernels form the
  // edges of G_i (q - Q) in FP32 from it without losing the FP64 difference
  const float* uh;
  const float* ul;
  const float* E0;     // 9m: G_i Q - I (rounding of the FP32 D_m^-1, static)
  const float* dq;     // 3n
  float* g;            // 9m
  float* y;            // 9m
  float* d;            // 9m
  float* Uw;           // 54m
  double* contrib;     // 12m corner terms (FP64: exact re-solves of q)
  float* contrib32;    // 12m corner terms of the direction (FP32: dq solve)
  float* b32;          // 3n float RHS (unused by the tet kernels)
  const double* z;     // 48
  DevScalars* sc;
  double* partials;
  // bones (Sec. 3.3; null without bones): kind of each tet (kTetDeformable,
  // kTetPinnedBone or the free bone's index) and the free bones' iteration
  // state (their directions at kBoneD)
  const int32_t* tkind = nullptr;
  const double* bone_st = nullptr;
  const float* nu = nullptr;  // 9m generalized external force (Sec. 3.4), null without one
};

void launch_grad_mixed(const MixArgs& a, int grid, cudaStream_t st);
void launch_dir_mixed(const MixArgs& a, int grid, cudaStream_t st);
// Line-search constants and the direction kernel's g.d partials, for the
// Armijo selection the last block of the line-search kernel performs.
struct LsSelect {
  const double* dir_partials;
  int nblk_dir;
  double sigma0, rho, c_armijo;
  // blocks of line-search partials written after the kernel's own (the free
  // bones' FP64 terms, Sec. 3.3), summed by the selection too
  int nblk_extra = 0;
};
// Trial energies of one pass and, in its last block, the selected step
// (k_ls_select's work); the gradient kernel likewise leaves ||g||^2 in sc.
void launch_ls_mixed(const MixArgs& a, int grid, const LsSelect& sel, cudaStream_t st);
void launch_update_mixed(const MixArgs& a, int grid, cudaStream_t st);
void launch_rhs_state_mixed(const MixArgs& a, int grid, cudaStream_t st);
// Capacitance partials C and B y on TF32 tensor cores (mma.sync), grid
// blocks striding over 32-tet chunks; cpart is entry-major (entry * grid + block).
void launch_syrk_tc(const MixArgs& a, int grid, double* cpart, cudaStream_t st);
// Blocks of the TC SYRK resident per SM (its launch bounds; grid = this x SMs).
constexpr int kTcBlocksPerSM = 2;
// Per-device kernel attributes of the TC SYRK (before its first launch).
cudaError_t prepare_syrk_tc();
void launch_update_verts_f(int64_t n, const DevScalars* sc, const float* dq, double* q, cudaStream_t st);
// uh + ul = q - Q: hi = the FP32 rounding of the FP64 difference, lo = the
// FP32 rounding of what hi leaves over.
void launch_split_disp(int64_t n, const double* q, const double* Q, float* uh, float* ul, cudaStream_t st);
void launch_assemble_f(int64_t n, const int32_t* slot_ptr, const int32_t* slot_idx, const float* contrib32,
                       const uint8_t* is_fixed, float* b, cudaStream_t st);
// state conversion: (quat, E) <-> (R 9m, s 6m) FP64 structure of arrays
void launch_mixed_to_Rs(int64_t m, const float4* quat, const float* E, double* R, double* s, cudaStream_t st);
void launch_Rs_to_mixed(int64_t m, const double* R, const double* s, float4* quat, float* E, cudaStream_t st);

}  // namespace emu
