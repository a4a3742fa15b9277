// Declarations of the per-tet and per-vertex kernels of one Newton iteration.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "emu_bones.h"
#include "emu_internal.h"
#include "emu_reduce.cuh"

namespace emu {

// Arrays the per-tet kernels read and write. FP64 path: TW = double.
// Mixed path: TW = float for the Hessian / Woodbury quantities (Uw, y, d, gam).
template <typename TW> struct TetArgs {
  int64_t m, n;
  const int4* tet;
  const double* Dinv;   // 9m  (k*m + i)
  const double* V;      // m
  const double* c;      // m  alpha * w
  const double* w;      // m
  const double* mu;     // m
  const double* lam;    // m
  const double* u;      // 3m
  const double* ka;     // m  kappa * a
  const TW* gam;        // 48m (3j + c)*m + i
  double* R;            // 9m
  double* s;            // 6m
  const double* q;      // 3n
  const double* dq;     // 3n
  double* g;            // 9m  F-space gradient
  TW* y;                // 9m  H_F^-1 g
  TW* d;                // 9m  search direction
  TW* Uw;               // 54m chart factor
  double* contrib;      // 12m corner contributions (slot 4i+k, 3 values)
  const double* z;      // 48 Woodbury coefficients
  DevScalars* sc;
  double* partials;     // per-block partial sums
  const int32_t* tkind = nullptr;    // bones: kind of each tet (null without bones)
  const double* bone_st = nullptr;   // bones: free bones' iteration state
  const double* nu = nullptr;        // 9m generalized external force (Sec. 3.4), null without one
};

void launch_rhs_from_state(const TetArgs<double>& a, int grid, cudaStream_t st);
template <typename TW> void launch_grad(const TetArgs<TW>& a, int grid, cudaStream_t st);
template <typename TW> void launch_syrk(const TetArgs<TW>& a, int grid, double* cpart, cudaStream_t st);
template <typename TW> void launch_dir(const TetArgs<TW>& a, int grid, cudaStream_t st);
template <typename TW> void launch_ls(const TetArgs<TW>& a, int grid, double rho, cudaStream_t st);
template <typename TW> void launch_update_tets(const TetArgs<TW>& a, int grid, cudaStream_t st);

// Per-vertex RHS gather: b_v = sum over incident corner slots, minus the
// pinned-column term (mode 0, coupling solve for q) or not (mode 1, dq).
void launch_assemble(int64_t n, const int32_t* slot_ptr, const int32_t* slot_idx, const double* contrib,
                     const double* bfix, const uint8_t* is_fixed, const double* qfix, int mode, double* b,
                     cudaStream_t st);
void launch_update_verts(int64_t n, const DevScalars* sc, const double* dq, double* q, cudaStream_t st);
// Generalized external force of Sec. 3.4: nu_i = w_i G_i x (x = K^-1 f, 3n),
// written component-major to nu64 (9m) and, when non-null, nu32.
void launch_nu(int64_t m, const int4* tet, const double* Dinv, const double* w, const double* x, double* nu64,
               float* nu32, cudaStream_t st);

// Single-block reducers.
void launch_reduce_grad(const double* partials, int nblk, DevScalars* sc, double* By, double* gsum,
                        cudaStream_t st);
// cpart: entry-major partials (kCapEntries + kK entries x nblk blocks);
// cfull_scratch receives their sums. fp32_factor: factor and solve in FP32.
// cadd (null, or kCapEntries + kK values) is added to the summed entries
// (the bones' terms of Sec. 3.3).
void launch_cap_solve(const double* cpart, int nblk, const double* cfull_scratch, double* z, DevScalars* sc,
                      bool fp32_factor, cudaStream_t st, const double* cadd = nullptr);
// Restart the line search: ls_fail = 0, sigma_start = sigma0.
void launch_ls_reset(DevScalars* sc, double sigma0, cudaStream_t st);
void launch_ls_select(const double* dir_partials, int nblk_dir, const double* ls_partials, int nblk_ls,
                      DevScalars* sc, double sigma0, double rho, double c_armijo, cudaStream_t st);

// Normaliser of the residual: ||g(F = I, q0)||^2 into out[0].
void launch_gref(const TetArgs<double>& a, const double* q0, int grid, double* partials, double* out,
                 cudaStream_t st);

// Setup kernels for the low-rank basis.
void launch_gram16(int64_t n, const double* X, int grid, double* partials, cudaStream_t st);
void launch_reduce_cols(const double* partials, int nblk, int nv, double* out, cudaStream_t st);
void launch_xform16(int64_t n, const double* T, double* X, cudaStream_t st);
// partials of X^T (L X) for the 16-column basis X (Y receives L X)
void launch_galerkin16(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* X,
                       double* Y, int grid, double* partials, cudaStream_t st);
void launch_d2f(int64_t k, const double* a, float* b, cudaStream_t st);
template <typename TW>
void launch_gamma(int64_t m, const int4* tet, const double* Dinv, const double* X, TW* gam, cudaStream_t st);

// Element-level evaluation entry points.
void launch_eval_stretch(const double* s, const double* prm, int64_t n, int mixed, double* psi, double* grad,
                         double* hess, cudaStream_t st);
void launch_eval_polar(const double* F, int64_t n, double* R, double* s, cudaStream_t st);
void launch_compose_F(int64_t m, const double* R, const double* s, double* F, cudaStream_t st);

constexpr int kGradNV = 1 + kK;        // gnorm2 + By
constexpr int kLsNV = kLsTrials + 2;   // dPsi per trial + c<D,dD> + c|dD|^2

// Armijo selection among the trial steps of one line-search pass, from the
// block partials of g.d (direction kernel) and of the trial energies. All
// kLsTrials steps sigma_start * rho^j are evaluated in the same pass anyway,
// so of those that satisfy the Armijo condition the one with the largest
// energy decrease is taken (not merely the first).
__device__ __forceinline__ void ls_select_block(const double* dir_partials, int nblk_dir, const double* ls_partials, int nblk_ls,
                                DevScalars* sc, double sigma0, double rho, double c_armijo) {
  __shared__ double s_gtd[1], s_v[kLsNV];
  block_sum_partials<1>(dir_partials, nblk_dir, s_gtd);
  block_sum_partials<kLsNV>(ls_partials, nblk_ls, s_v);
  if (threadIdx.x != 0) return;
  const double gtd = s_gtd[0];
  double v[kLsNV];
  for (int k = 0; k < kLsNV; ++k) v[k] = s_v[k];
  sc->gtd = gtd;
  double sig = sc->sigma_start;
  int accepted = -1;
  double dE = 0.0;
  if (gtd < 0.0) {
    double s_j = sig, best_sig = sig;
    for (int j = 0; j < kLsTrials; ++j) {
      const double dEj = v[j] + s_j * v[kLsTrials] + 0.5 * s_j * s_j * v[kLsTrials + 1];
      if (dEj <= c_armijo * s_j * gtd && (accepted < 0 || dEj < dE)) {
        accepted = j;
        dE = dEj;
        best_sig = s_j;
      }
      s_j *= rho;
    }
    sig = best_sig;
  }
  if (accepted >= 0) {
    sc->sigma = sig;
    sc->sigma_start = sigma0;
    sc->dE += dE;
    sc->ls_trials += accepted + 1;
    sc->ls_fail = 0;
  } else {
    sc->sigma = 0.0;
    double st = sc->sigma_start;
    for (int j = 0; j < kLsTrials; ++j) st *= rho;
    sc->sigma_start = st;
    sc->ls_trials += kLsTrials;
    sc->ls_fail += 1;
  }
}

constexpr int kCapEntries = kK * kK;   // 48 x 48 partial capacitance

// The 3 x 3 tiles of the lower triangle of the 48 x 48 symmetric product
// (tile row >= tile column), 136 of them: thread t < 136 of a block takes
// tile t in row order; the others have none. The upper triangle is the
// mirror image (a_p b_q and b_q a_p are the same product, so each entry's
// sum is the one a full tiling would form).
constexpr int kLowerTiles = (kK / 3) * (kK / 3 + 1) / 2;
__device__ __forceinline__ bool lower_tile(int t, int& tr, int& tc) {
  if (t >= kLowerTiles) return false;
  int r = 0;
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  tr = r;
  tc = t - r * (r + 1) / 2;
  return true;
}

}  // namespace emu
