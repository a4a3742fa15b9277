// The F-form of EMU's quasi-Newton iteration on the device (arXiv 2006.08821,
// Sec. 3.2.1, Eqs. 10-12): one free deformation gradient F_i per tet, the
// 9 x 9 block Hessian H_i = PSD(V Psi_iso''(F_i)) + V Psi_fiber''(F_i)
// + alpha w_i I, and the low-rank Woodbury direction with the constant
// B = Phi^T G^T W. F <- F + sigma d and q <- q + sigma dq (Eq. 4 is affine
// in F), so one coupling solve (for dq) per iteration.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "emu_kernels.cuh"

namespace emu {

// Entries of a tet's packed 9 x 9 lower Cholesky factor of H_i (row r,
// column c <= r at r (r + 1) / 2 + c; the diagonal holds 1 / L_rr).
constexpr int kFformL = 45;

// The kernels take the rotation/stretch path's TetArgs<double> with a.R
// holding F (9m, component-major k * m + i), a.Uw the factors (45m), and
// a.g, a.y, a.d, a.gam, a.contrib, a.z, a.partials as there. No bones.
void launch_rhs_fform(const TetArgs<double>& a, int grid, cudaStream_t st);
void launch_grad_fform(const TetArgs<double>& a, int grid, cudaStream_t st);
// cpart as for launch_syrk, holding the partials of -alpha sum w^2
// (G Phi)^T H^-1 (G Phi): C = Lambda + that sum takes Lambda = Phi^T K Phi
// as the addend of launch_cap_solve.
void launch_syrk_fform(const TetArgs<double>& a, int grid, double* cpart, cudaStream_t st);
void launch_dir_fform(const TetArgs<double>& a, int grid, cudaStream_t st);
void launch_ls_fform(const TetArgs<double>& a, int grid, double rho, cudaStream_t st);
void launch_update_fform(const TetArgs<double>& a, int grid, cudaStream_t st);
// R and s (component-major, like the rotation/stretch state) of the polar
// decomposition F = R S of each tet's F.
void launch_fform_to_Rs(int64_t m, const double* F, double* R, double* s, cudaStream_t st);
// Element terms: psi = V Psi(F), grad = V P(F) (9), hess = the 9 x 9 block
// above without the alpha w I term (81, row-major); AoS device arrays, F
// n x 9 row-major, prm n x 8 (V, mu, lambda, kappa a, u).
void launch_eval_fform(const double* F, const double* prm, int64_t n, double* psi, double* grad, double* hess,
                       cudaStream_t st);

}  // namespace emu
