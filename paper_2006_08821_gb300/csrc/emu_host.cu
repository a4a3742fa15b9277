// Host side of the C ABI declared in include/emu.h: mesh setup, the Newton
// loop of Algorithm 1 (arXiv 2006.08821) and the entry points.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <thread>
#include <vector>

#include "emu_internal.h"
#include "emu_kernels.cuh"
#include "emu_fform.h"
#include "emu_mixed.cuh"
#include "emu_pcg.h"

namespace emu {
namespace {
int enqueue_grad(emu_handle* h);
int enqueue_direction(emu_handle* h);
}  // namespace
}  // namespace emu

using namespace emu;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define EMU_CK(call)                                                                           \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(EMU_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)


}  // namespace

#include "emu_handle.h"
#include "emu_syrk05.h"

// Cyclic Jacobi eigen-decomposition of a symmetric N x N matrix (row-major):
// A is overwritten (its diagonal holds the eigenvalues), V receives the
// eigenvectors as columns.
void emu::host_jacobi_eig(std::vector<double>& A, std::vector<double>& V, int N) {
  V.assign(N * N, 0.0);
  for (int i = 0; i < N; ++i) V[N * i + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        tot += A[N * i + j] * A[N * i + j];
        if (i != j) off += A[N * i + j] * A[N * i + j];
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < N; ++p)
      for (int q = p + 1; q < N; ++q) {
        const double apq = A[N * p + q];
        if (apq == 0.0) continue;
        const double theta = (A[N * q + q] - A[N * p + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s_ = t * c;
        for (int k = 0; k < N; ++k) {  // A <- J^T A J
          const double akp = A[N * k + p], akq = A[N * k + q];
          A[N * k + p] = c * akp - s_ * akq;
          A[N * k + q] = s_ * akp + c * akq;
        }
        for (int k = 0; k < N; ++k) {
          const double apk = A[N * p + k], aqk = A[N * q + k];
          A[N * p + k] = c * apk - s_ * aqk;
          A[N * q + k] = s_ * apk + c * aqk;
        }
        for (int k = 0; k < N; ++k) {
          const double vkp = V[N * k + p], vkq = V[N * k + q];
          V[N * k + p] = c * vkp - s_ * vkq;
          V[N * k + q] = s_ * vkp + c * vkq;
        }
      }
  }
}


namespace {

uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}


int validate_mesh(const emu_mesh_desc* d) {
  if (!d) return fail(EMU_ERR_INVALID_ARG, "mesh is NULL");
  if (d->n_verts < 4 || d->n_tets < 1) return fail(EMU_ERR_INVALID_ARG, "need n_verts >= 4 and n_tets >= 1");
  if (d->n_verts > (int64_t)1 << 30 || d->n_tets > (int64_t)1 << 28)
    return fail(EMU_ERR_INVALID_ARG, "mesh too large for 32-bit indexing");
  if (!d->rest_pos || !d->tets || !d->youngs || !d->poisson || !d->material_id)
    return fail(EMU_ERR_INVALID_ARG, "missing mesh array");
  if (d->n_materials < 1) return fail(EMU_ERR_INVALID_ARG, "n_materials < 1");
  for (int32_t k = 0; k < d->n_materials; ++k) {
    if (!(d->youngs[k] > 0.0) || !std::isfinite(d->youngs[k])) return fail(EMU_ERR_INVALID_ARG, "youngs must be > 0");
    if (!(d->poisson[k] >= 0.0 && d->poisson[k] < 0.5)) return fail(EMU_ERR_INVALID_ARG, "poisson must be in [0, 0.5)");
  }
  for (int64_t i = 0; i < 4 * d->n_tets; ++i)
    if (d->tets[i] < 0 || d->tets[i] >= d->n_verts) return fail(EMU_ERR_INVALID_ARG, "tet index out of range");
  for (int64_t i = 0; i < d->n_tets; ++i)
    if (d->material_id[i] >= d->n_materials) return fail(EMU_ERR_INVALID_ARG, "material_id out of range");
  if (d->n_fixed < 1 || !d->fixed_verts) return fail(EMU_ERR_INVALID_ARG, "at least one pinned vertex is required");
  for (int64_t i = 0; i < d->n_fixed; ++i)
    if (d->fixed_verts[i] < 0 || d->fixed_verts[i] >= d->n_verts) return fail(EMU_ERR_INVALID_ARG, "fixed vertex out of range");
  for (int64_t i = 0; i < 3 * d->n_verts; ++i)
    if (!std::isfinite(d->rest_pos[i])) return fail(EMU_ERR_INVALID_ARG, "non-finite rest position");
  if (d->n_joints < 0) return fail(EMU_ERR_INVALID_ARG, "n_joints must be >= 0");
  if (d->n_joints > 0 && (!d->joint_type || !d->joint_bones || !d->joint_point || !d->joint_axis ||
                          !d->joint_half_length))
    return fail(EMU_ERR_INVALID_ARG, "missing joint array");
  if (d->bone_id)
    for (int64_t i = 0; i < d->n_tets; ++i)
      if (d->bone_id[i] < -1) return fail(EMU_ERR_INVALID_ARG, "bone_id must be -1 or a bone index");
  return EMU_OK;
}

int validate_params(const emu_params* p) {
  if (!(p->alpha_rel > 0.0) || !std::isfinite(p->alpha_rel)) return fail(EMU_ERR_INVALID_ARG, "alpha_rel must be > 0");
  if (p->weight_mode != 0 && p->weight_mode != 1) return fail(EMU_ERR_INVALID_ARG, "weight_mode must be 0 or 1");
  if (p->k_modes < 3 || p->k_modes > 48 || p->k_modes % 3) return fail(EMU_ERR_INVALID_ARG, "k_modes must be 3..48, multiple of 3");
  if (!(p->fiber_scale >= 0.0)) return fail(EMU_ERR_INVALID_ARG, "fiber_scale must be >= 0");
  if (!(p->tol_rel_residual >= 0.0)) return fail(EMU_ERR_INVALID_ARG, "tol_rel_residual must be >= 0");
  if (p->max_newton < 0) return fail(EMU_ERR_INVALID_ARG, "max_newton must be >= 0");
  if (!(p->ls_sigma0 > 0.0) || !(p->ls_rho > 0.0 && p->ls_rho < 1.0) || !(p->ls_c > 0.0 && p->ls_c < 1.0))
    return fail(EMU_ERR_INVALID_ARG, "bad line-search constants");
  if (p->ls_max_trials < 1) return fail(EMU_ERR_INVALID_ARG, "ls_max_trials must be >= 1");
  if (!(p->pcg_tol > 0.0 && p->pcg_tol < 1.0) || p->pcg_max < 1) return fail(EMU_ERR_INVALID_ARG, "bad pcg settings");
  if (p->precision != EMU_PRECISION_FP64 && p->precision != EMU_PRECISION_MIXED)
    return fail(EMU_ERR_INVALID_ARG, "precision must be FP64 or MIXED");
  if (p->mode_iters < 1 || p->mode_iters > 50) return fail(EMU_ERR_INVALID_ARG, "mode_iters must be 1..50");
  if (!(p->dq_tol > 0.0 && p->dq_tol < 1.0)) return fail(EMU_ERR_INVALID_ARG, "dq_tol must be in (0, 1)");
  if (p->q_refresh < 1) return fail(EMU_ERR_INVALID_ARG, "q_refresh must be >= 1");
  if (!(p->eps_bone < 0.0) || !(p->eps_joint < 0.0) || !std::isfinite(p->eps_bone) || !std::isfinite(p->eps_joint))
    return fail(EMU_ERR_INVALID_ARG, "eps_bone and eps_joint must be negative");
  if (p->cg_local_degree < 1 || p->cg_local_degree > kChebMax)
    return fail(EMU_ERR_INVALID_ARG, "cg_local_degree must be in [1, 8]");
  if (p->form != EMU_FORM_RS && p->form != EMU_FORM_F) return fail(EMU_ERR_INVALID_ARG, "form must be RS or F");
  if (p->autotune != 0 && p->autotune != 1) return fail(EMU_ERR_INVALID_ARG, "autotune must be 0 or 1");
  return EMU_OK;
}

int read_scalars(emu_handle* h);

// FP32 CG of the mixed path: the register-resident kernel when the mesh fits
// its launch shape, the generic kernel otherwise. Solves to kPipeMinTol or
// looser take the pipelined register-resident kernel (one grid barrier per
// iteration); its recurrences drift from the true residual near FP32
// precision, so tighter solves keep the plain one. (The correction rounds of
// the exact re-solve, at 1e-5 to 1e-3, measured slower on it: 260 instead of
// 243 us of CG per Newton iteration on the 401,920-tet unit.)
constexpr double kPipeMinTol = 1e-3;
cudaError_t run_pcg32(emu_handle* h, const float* rhs, float* x, double tol) {
  PcgArgsT<float> a = h->pcg32(rhs, x, tol);
  if (h->rpt32 > 0) {
    Pcg32Work w;
    w.ug = h->ug32;
    w.part = h->part32;
    w.sync = h->sync32;
    if (h->cg_part) {
      // the partitioned system with the block-local preconditioner (b and x
      // stay in vertex order)
      a.rowptr = h->cg_rowptr;
      a.col = h->cg_col;
      a.val = h->cg_val;
      a.dinv = h->cg_dinv;
      a.phi = a.phi ? h->cg_phi : nullptr;
      w.perm = h->cg_perm;
      w.off = h->cg_off;
      w.loc = h->cg_loc;
      w.lw = h->cg_lw;
      w.degree = h->cg_degree;
      w.c0 = h->cg_c0;
      for (int i = 0; i < kChebMax; ++i) {
        w.c1[i] = h->cg_c1[i];
        w.c2[i] = h->cg_c2[i];
      }
      if (tol >= kPipeMinTol && h->aphi_ready && a.phi && pcg32_pipe_ok(h->rpt32)) {
        w.aphi = h->cg_aphi;
        return launch_pcg32_pipe(a, w, h->grid32, h->rpt32, h->st);
      }
    }
    return launch_pcg32(a, w, h->grid32, h->rpt32, h->st);
  }
  return launch_pcg<float>(3, a, h->grid_pcg3, h->st);
}

// Exact coupling solve q = q*(F) of Eq. 4 from the current F, warm-started
// from the current q: iterative refinement, the residual b - K q in FP64 and
// a correction solve (FP32 CG on the mixed path, FP64 CG on the FP64 path),
// until every column's residual is below ``tol`` times the residual of the
// undeformed solution q*(I) for this F, |b(F) - K q*(I)| = |G^T W (F - I)|.
// That normaliser scales with the deformation: measured against |b|, which
// is dominated by the rest shape, a small deformation (a weak activation)
// would leave q with an error of 1e-8 of the mesh size, far above the
// displacement's own precision. Pure rounding (|r| <= 1e-14 |b|) also ends it.
//
// The steps are enqueued separately so that a solve can wait for the
// residual without blocking the host: refresh_begin (right-hand side and the
// normaliser), then rounds of refresh_residual (sums into o6_host),
// refresh_converged and refresh_correction.
constexpr int kRefreshRounds = 8;
// a solve whose best residual is within kStallBand of the tolerance and has
// not improved by 0.1 % for kEscalateIters iterations shortens its first
// trial step to 1, or else switches from the mixed to the FP64 kernels, or
// else tightens dq; after kStallIters with none left it ends as not converged
constexpr double kStallBand = 10.0;
constexpr int kEscalateIters = 50;
constexpr int kStallIters = 200;

// Coupling solves in FP64 CG: on the FP64 path, and on the mixed path when
// the mesh has bones. A bone tet's ACAP weight carries the 1/|eps_bone|
// penalty, which multiplies the Laplacian's condition number by about
// 1000: beyond what an FP32 CG resolves (measured on the 40,152-tet arm:
// mixed with FP32 dq solves took 2,765 Newton iterations over three
// frames where the FP64 path took 608).
bool cg64(const emu_handle* h) { return !h->mixed || h->has_bones; }

int refresh_begin(emu_handle* h, double /*tol*/) {
  h->ph_begin();
  if (h->mixed)
    launch_rhs_state_mixed(h->margs(), h->grid_tet, h->st);
  else if (h->fform)
    launch_rhs_fform(h->args<double>(), h->grid_tet, h->st);
  else
    launch_rhs_from_state(h->args<double>(), h->grid_tet, h->st);
  h->ph_end(EMU_PHASE_RHS, 1);
  h->ph_begin();
  launch_assemble(h->n, h->slot_ptr, h->slot_idx, h->contrib, h->bfix, h->is_fixed, h->qfix, 0, h->b, h->st);
  h->ph_end(EMU_PHASE_ASSEMBLE, 1);
  EMU_CK(cudaGetLastError());
  const int rgrid = (int)std::min<int64_t>(std::max<int64_t>(1, (h->n + 255) / 256), 2 * (int64_t)h->sms);
  h->ph_begin();
  if (h->npts > 0) {
    // with joints the residual of the constrained problem is the projected one
    double* rs = h->b + 9 * h->n;
    EMU_CK(launch_residual64(h->n, h->rowptr, h->col, h->val, h->b, h->q0, nullptr, rs, h->part_pcg, rgrid,
                             h->small + 8, h->st, h->jmask));
    launch_joint_rproj(h->jargs(), rs, nullptr, h->small + 8, h->st);
    h->ph_end(EMU_PHASE_PCG, 3);
  } else {
    EMU_CK(launch_residual64(h->n, h->rowptr, h->col, h->val, h->b, h->q0, nullptr, nullptr, h->part_pcg, rgrid,
                             h->small + 8, h->st));
    h->ph_end(EMU_PHASE_PCG, 2);
  }
  return EMU_OK;
}

int refresh_residual(emu_handle* h) {
  const int rgrid = (int)std::min<int64_t>(std::max<int64_t>(1, (h->n + 255) / 256), 2 * (int64_t)h->sms);
  const bool c64 = cg64(h);
  float* r32 = c64 ? nullptr : h->r32;
  h->ph_begin();
  if (h->npts > 0) {
    EMU_CK(launch_residual64(h->n, h->rowptr, h->col, h->val, h->b, h->q, r32, h->b + 3 * h->n, h->part_pcg, rgrid,
                             h->small, h->st, h->jmask));
    launch_joint_rproj(h->jargs(), h->b + 3 * h->n, r32, h->small, h->st);
    h->ph_end(EMU_PHASE_PCG, 3);
  } else {
    EMU_CK(launch_residual64(h->n, h->rowptr, h->col, h->val, h->b, h->q, r32, c64 ? h->b + 3 * h->n : nullptr,
                             h->part_pcg, rgrid, h->small, h->st));
    h->ph_end(EMU_PHASE_PCG, 2);
  }
  EMU_CK(cudaMemcpyAsync(h->o6_host, h->small, 14 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  return EMU_OK;
}

// valid once the copy of refresh_residual has completed
bool refresh_converged(const emu_handle* h, double tol) {
  const double* o = h->o6_host;
  bool done = true;
  for (int j = 0; j < 3; ++j) done = done && (o[j] <= tol * tol * o[8 + j] || o[j] <= 1e-28 * o[3 + j]);
  return done;
}

// Relative tolerance of the next correction solve: just enough to bring
// every column's residual to ``tol`` of its normaliser (with a 5x margin),
// within what the correction's arithmetic can reach. Valid after the copy
// of refresh_residual has completed.
double refresh_round_tol(const emu_handle* h, double tol) {
  const double* o = h->o6_host;
  double need = 0.5;
  for (int j = 0; j < 3; ++j)
    if (o[j] > 0.0) need = std::min(need, 0.2 * tol * std::sqrt(o[8 + j] / o[j]));
  return std::max(need, cg64(h) ? 1e-12 : 1e-6);
}

int refresh_correction(emu_handle* h, double round_tol) {
  if (!cg64(h)) {
    EMU_CK(cudaMemsetAsync(h->e32, 0, 12 * h->n, h->st));
    h->ph_begin();
    EMU_CK(run_pcg32(h, h->r32, h->e32, round_tol));
    EMU_CK(launch_axpy_f2d(3 * h->n, h->e32, h->q, h->st));
    joints_project(h, h->q, nullptr);  // J q = 0 again (the joint rows of Sec. 3.3)
    h->ph_end(EMU_PHASE_PCG, 2);
    return EMU_OK;
  }
  double* r64 = h->b + 3 * h->n;  // written by refresh_residual
  double* e64 = h->b + 6 * h->n;
  EMU_CK(cudaMemsetAsync(e64, 0, 24 * h->n, h->st));
  h->ph_begin();
  EMU_CK(launch_pcg<double>(3, h->pcg64(r64, e64, round_tol), h->grid_pcg3, h->st));
  EMU_CK(launch_axpy_d2d(3 * h->n, e64, h->q, h->st));
  joints_project(h, h->q, nullptr);
  h->ph_end(EMU_PHASE_PCG, 2);
  return EMU_OK;
}

int refresh_q(emu_handle* h, double tol) {
  int rc = refresh_begin(h, tol);
  if (rc) return rc;
  for (int round = 0; round < kRefreshRounds; ++round) {
    rc = refresh_residual(h);
    if (rc) return rc;
    EMU_CK(cudaStreamSynchronize(h->st));
    h->prof_flush();
    if (refresh_converged(h, tol)) break;
    rc = refresh_correction(h, refresh_round_tol(h, tol));
    if (rc) return rc;
  }
  return EMU_OK;
}

// dq: the linear change of q* along the direction d, to dq_tol (loose), or
// to the exact-solve tolerance once a line search has failed in this call.
int solve_dq(emu_handle* h) {
  const double tol = h->dq_tol_now;
  if (!h->mixed) {
    h->ph_begin();
    launch_assemble(h->n, h->slot_ptr, h->slot_idx, h->contrib, h->bfix, h->is_fixed, h->qfix, 1, h->b, h->st);
    h->ph_end(EMU_PHASE_ASSEMBLE, 1);
    EMU_CK(cudaGetLastError());
    h->ph_begin();
    EMU_CK(launch_pcg<double>(3, h->pcg64(h->b, h->dq, tol), h->grid_pcg3, h->st));
    joints_project(h, h->dq, nullptr);
    h->ph_end(EMU_PHASE_PCG, 1);
    return EMU_OK;
  }
  h->ph_begin();
  launch_assemble_f(h->n, h->slot_ptr, h->slot_idx, h->contrib32, h->is_fixed, h->b32, h->st);
  h->ph_end(EMU_PHASE_ASSEMBLE, 1);
  EMU_CK(cudaGetLastError());
  h->ph_begin();
  if (cg64(h)) {
    // mixed path with bones: the FP32 right-hand side, the solve in FP64
    // (dq in FP64 for the position update, an FP32 copy for the per-tet kernels)
    EMU_CK(cudaMemsetAsync(h->b, 0, 24 * h->n, h->st));
    EMU_CK(launch_axpy_f2d(3 * h->n, h->b32, h->b, h->st));
    EMU_CK(launch_pcg<double>(3, h->pcg64(h->b, h->dq, tol), h->grid_pcg3, h->st));
    joints_project(h, h->dq, nullptr);
    launch_d2f(3 * h->n, h->dq, h->dq32, h->st);
    h->ph_end(EMU_PHASE_PCG, 4);
    return EMU_OK;
  }
  EMU_CK(run_pcg32(h, h->b32, h->dq32, tol));
  joints_project(h, nullptr, h->dq32);
  h->ph_end(EMU_PHASE_PCG, 1);
  return EMU_OK;
}

// ---- autotuner (emu_params.autotune) ----
// Candidate launch settings of the coupling solves are timed at set-up on
// the handle's own matrix, and the fastest is kept:
//  * the degree of the block-local Chebyshev polynomial in the mixed path's
//    pipelined FP32 CG (its dq solves): one solve to dq_tol from zero per
//    degree on the right-hand side of a real first Newton direction, the
//    better of two runs each;
//  * the rows per block of the FP64 CG (the FP64 path, meshes with bones):
//    a fixed count of iterations per candidate on a seeded right-hand side
//    (the count to a tolerance does not depend on the launch shape).
// Each candidate runs the same method; only rounding differs between them.
// A choice is kept for the process per (device, mesh size, kind), so every
// handle of one mesh in a process runs the same settings (a batch stays
// bit-identical to its meshes solved alone).
constexpr int kTuneDegrees[] = {2, 3, 4, 6, 8};
constexpr int kTuneRows[] = {64, 128, 256};
constexpr int kTuneIters64 = 40;
std::mutex g_tune_mu;
std::map<std::tuple<int, int64_t, int64_t, int, double>, int> g_tune;

// Right-hand side of a real dq solve: the first Newton direction from rest
// at activation 0.5 on every tet (the handle's activation is zero again
// afterwards). The coupling solves see the spectrum of real directions;
// a random right-hand side would favour low local degrees.
int tune_dq_rhs(emu_handle* h) {
  std::vector<double> act(h->m, 0.5);
  int rc = emu_set_activation(h, act.data(), h->m);
  if (rc) return rc;
  DevScalars init;
  memset(&init, 0, sizeof(init));
  init.sigma_start = h->sigma0_now;
  EMU_CK(cudaMemcpyAsync(h->sc, &init, sizeof(init), cudaMemcpyHostToDevice, h->st));
  rc = enqueue_grad(h);
  if (!rc) rc = enqueue_direction(h);
  if (rc) return rc;
  launch_assemble_f(h->n, h->slot_ptr, h->slot_idx, h->contrib32, h->is_fixed, h->b32, h->st);
  EMU_CK(cudaGetLastError());
  EMU_CK(cudaStreamSynchronize(h->st));
  std::fill(act.begin(), act.end(), 0.0);
  return emu_set_activation(h, act.data(), h->m);
}

int tune_rhs(emu_handle* h) {
  const int64_t n = h->n;
  std::vector<uint8_t> fixed(n);
  EMU_CK(cudaMemcpyAsync(fixed.data(), h->is_fixed, n, cudaMemcpyDeviceToHost, h->st));
  EMU_CK(cudaStreamSynchronize(h->st));
  uint64_t seed = h->prm.seed ^ 0x7E57AB1Eull;
  std::vector<double> b(3 * n, 0.0);
  for (int64_t k = 0; k < 3 * n; ++k) {
    const double r = (double)(splitmix64(seed) >> 11) * (1.0 / 9007199254740992.0);
    b[k] = fixed[k / 3] ? 0.0 : 2.0 * r - 1.0;
  }
  EMU_CK(cudaMemcpyAsync(h->b, b.data(), 24 * n, cudaMemcpyHostToDevice, h->st));
  EMU_CK(cudaStreamSynchronize(h->st));
  return EMU_OK;
}

// device time of ``run`` on the handle's stream (ms); -1 on a CUDA error
template <typename F> float tune_time(emu_handle* h, F&& run) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = -1.f;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
      cudaEventRecord(e0, h->st) == cudaSuccess && run() == cudaSuccess && cudaEventRecord(e1, h->st) == cudaSuccess &&
      cudaEventSynchronize(e1) == cudaSuccess)
    cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return ms;
}

void set_cg_degree(emu_handle* h, int d) {
  h->cg_degree = d;
  cg_cheb_coeffs(h->cg_lmax, d, &h->cg_c0, h->cg_c1, h->cg_c2);
}

void set_cg64_rows(emu_handle* h, int rows) {
  h->cg64_rows = rows;
  h->grid_pcg3 = (int)std::max<int64_t>(1, std::min<int64_t>((h->n + rows - 1) / rows, h->sms));
}

int autotune(emu_handle* h) {
  h->tuned = true;
  const auto key = [&](int kind, double tol) { return std::make_tuple(h->device, h->n, h->m, kind, tol); };
  // the local polynomial's degree (pipelined FP32 CG of the dq solves)
  if (h->mixed && !cg64(h) && h->cg_part && h->cg_lw > 0 && h->aphi_ready && pcg32_pipe_ok(h->rpt32)) {
    const double tol = h->prm.dq_tol;
    int best = -1;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune.find(key(0, tol));
      if (it != g_tune.end()) best = it->second;
    }
    if (best < 0) {
      int rc = tune_dq_rhs(h);
      if (rc) return rc;
      float tbest = 0.f;
      for (int d : kTuneDegrees) {
        set_cg_degree(h, d);
        float t = -1.f;
        for (int rep = 0; rep < 2; ++rep) {
          const float ms = tune_time(h, [&]() {
            cudaError_t e = cudaMemsetAsync(h->dq32, 0, 12 * h->n, h->st);
            return e == cudaSuccess ? run_pcg32(h, h->b32, h->dq32, tol) : e;
          });
          if (ms < 0.f) return fail(EMU_ERR_CUDA, "autotune: CG launch failed");
          t = (t < 0.f || ms < t) ? ms : t;
        }
        if (best < 0 || t < tbest) {
          best = d;
          tbest = t;
        }
      }
      std::lock_guard<std::mutex> lock(g_tune_mu);
      best = g_tune.emplace(key(0, tol), best).first->second;  // a concurrent set-up may have stored one first
    }
    set_cg_degree(h, best);
  }
  // rows per block of the FP64 CG
  if (cg64(h)) {
    int best = -1;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune.find(key(1, 0.0));
      if (it != g_tune.end()) best = it->second;
    }
    if (best < 0) {
      int rc = tune_rhs(h);
      if (rc) return rc;
      float tbest = 0.f;
      for (int rows : kTuneRows) {
        set_cg64_rows(h, rows);
        const float ms = tune_time(h, [&]() {
          cudaError_t e = cudaMemsetAsync(h->dq, 0, 24 * h->n, h->st);
          if (e != cudaSuccess) return e;
          PcgArgsT<double> a = h->pcg64(h->b, h->dq, 0.0);
          a.max_iter = kTuneIters64;
          a.iters_out = nullptr;
          a.fail_out = nullptr;
          return launch_pcg<double>(3, a, h->grid_pcg3, h->st);
        });
        if (ms < 0.f) return fail(EMU_ERR_CUDA, "autotune: CG launch failed");
        if (best < 0 || ms < tbest) {
          best = rows;
          tbest = ms;
        }
      }
      std::lock_guard<std::mutex> lock(g_tune_mu);
      best = g_tune.emplace(key(1, 0.0), best).first->second;
    }
    set_cg64_rows(h, best);
  }
  EMU_CK(cudaMemsetAsync(h->dq, 0, 24 * h->n, h->st));
  if (h->dq32) EMU_CK(cudaMemsetAsync(h->dq32, 0, 12 * h->n, h->st));
  EMU_CK(cudaStreamSynchronize(h->st));
  return EMU_OK;
}

int set_rest_state(emu_handle* h) {
  std::vector<double> Rh(9 * h->m, 0.0), sh(6 * h->m, 0.0);
  for (int64_t i = 0; i < h->m; ++i) {
    Rh[0 * h->m + i] = Rh[4 * h->m + i] = Rh[8 * h->m + i] = 1.0;
    sh[0 * h->m + i] = sh[1 * h->m + i] = sh[2 * h->m + i] = 1.0;
  }
  EMU_CK(cudaMemcpyAsync(h->R, Rh.data(), Rh.size() * 8, cudaMemcpyHostToDevice, h->st));
  EMU_CK(cudaMemcpyAsync(h->s, sh.data(), sh.size() * 8, cudaMemcpyHostToDevice, h->st));
  EMU_CK(cudaMemsetAsync(h->dq, 0, 3 * h->n * 8, h->st));
  if (h->mixed) {
    launch_Rs_to_mixed(h->m, h->R, h->s, h->quat, h->E32, h->st);
    EMU_CK(cudaGetLastError());
    EMU_CK(cudaMemsetAsync(h->dq32, 0, 3 * h->n * 4, h->st));
  }
  EMU_CK(cudaStreamSynchronize(h->st));
  return bones_state_rest(h);
}

int read_scalars(emu_handle* h) {
  EMU_CK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->st));
  EMU_CK(cudaStreamSynchronize(h->st));
  h->prof_flush();
  return EMU_OK;
}

// Low-rank basis of Eq. 9: block inverse (subspace) iteration on the scalar
// ACAP Laplacian, X <- orth(L^-1 X), from a seeded random start. Any
// full-rank basis keeps the quasi-Newton matrix positive definite; better
// approximations of the lowest eigenvectors only speed up convergence.
int build_modes(emu_handle* h) {
  const int64_t n = h->n;
  std::vector<double> X(n * 16, 0.0);
  std::vector<uint8_t> fixed(n);
  EMU_CK(cudaMemcpyAsync(fixed.data(), h->is_fixed, n, cudaMemcpyDeviceToHost, h->st));
  EMU_CK(cudaStreamSynchronize(h->st));
  uint64_t seed = h->prm.seed ^ 0x5EEDF00Dull;
  for (int64_t v = 0; v < n; ++v)
    for (int j = 0; j < 16; ++j) {
      double r = (double)(splitmix64(seed) >> 11) * (1.0 / 9007199254740992.0);
      X[v * 16 + j] = fixed[v] ? 0.0 : 2.0 * r - 1.0;
    }
  double* Xd = h->scratch16;
  double* Yd = h->scratch16 + n * 16;
  EMU_CK(cudaMemcpyAsync(Xd, X.data(), X.size() * 8, cudaMemcpyHostToDevice, h->st));
  const int ggrid = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 511) / 512), 2 * h->sms);
  // X = Y T with Y^T Y = V diag(lambda) V^T, T = V diag(lambda^-1/2):
  // orthonormal columns; directions with a negligible Gram eigenvalue (fewer
  // free vertices than modes) are dropped as zero columns
  auto orthonormalise = [&](const double* Ysrc, bool last) -> int {
    launch_gram16(n, Ysrc, ggrid, h->part_pcg, h->st);
    launch_reduce_cols(h->part_pcg, ggrid, 256, h->small, h->st);
    std::vector<double> Gm(256);
    EMU_CK(cudaMemcpyAsync(Gm.data(), h->small, 256 * 8, cudaMemcpyDeviceToHost, h->st));
    EMU_CK(cudaStreamSynchronize(h->st));
    for (int i = 0; i < 16; ++i)
      for (int j = 0; j < 16; ++j) Gm[16 * i + j] = 0.5 * (Gm[16 * i + j] + Gm[16 * j + i]);
    std::vector<double> Ev;
    host_jacobi_eig(Gm, Ev, 16);
    double lmax = 0.0;
    for (int i = 0; i < 16; ++i) lmax = std::max(lmax, Gm[17 * i]);
    if (!(lmax > 0.0)) return fail(EMU_ERR_CUDA, "mode basis is empty");
    std::vector<double> T(256, 0.0);
    for (int j = 0; j < 16; ++j) {
      const double lj = Gm[17 * j];
      if (!(lj > 1e-12 * lmax)) continue;
      const double sc_ = 1.0 / std::sqrt(lj);
      for (int i = 0; i < 16; ++i) T[16 * i + j] = Ev[16 * i + j] * sc_;
    }
    // drop unused modes (k_modes < 48) after the last iteration
    if (last)
      for (int i = 0; i < 16; ++i)
        for (int j = h->kmodes; j < 16; ++j) T[16 * i + j] = 0.0;
    EMU_CK(cudaMemcpyAsync(h->small, T.data(), 256 * 8, cudaMemcpyHostToDevice, h->st));
    if (Ysrc != Xd) EMU_CK(cudaMemcpyAsync(Xd, Ysrc, n * 16 * 8, cudaMemcpyDeviceToDevice, h->st));
    launch_xform16(n, h->small, Xd, h->st);
    EMU_CK(cudaGetLastError());
    EMU_CK(cudaStreamSynchronize(h->st));
    return EMU_OK;
  };
  for (int it = 0; it < h->prm.mode_iters; ++it) {
    // Y = L^-1 X (pinned rows: right-hand side 0)
    EMU_CK(cudaMemsetAsync(Yd, 0, n * 16 * 8, h->st));
    PcgArgsT<double> a = h->pcg64(Xd, Yd, 1e-6);
    a.max_iter = std::max(h->prm.pcg_max, 1000);
    a.iters_out = nullptr;
    a.fail_out = nullptr;
    EMU_CK(launch_pcg<double>(16, a, h->grid_pcg16, h->st));
    // with joints, the basis lives in the null space of the joint rows (a
    // Galerkin basis of the constrained coupling problem keeps the
    // quasi-Newton matrix positive definite)
    int rc = joints_project_basis(h, Yd);
    if (rc) return rc;
    rc = orthonormalise(Yd, it + 1 == h->prm.mode_iters && h->nfb == 0);
    if (rc) return rc;
  }
  if (h->nfb > 0) {
    // the last 3 columns per free bone become the constrained responses of q
    // to the bone's F_b: without them the bone's block of the approximate
    // Hessian misses how q follows F_b (bone tets weigh ~1000x)
    int rc = bones_basis_responses(h, Xd);
    if (rc) return rc;
    rc = orthonormalise(Xd, true);
    if (rc) return rc;
  }
  if (h->mixed)
    launch_gamma<float>(h->m, h->tet, h->Dinv, Xd, h->gam32, h->st);
  else
    launch_gamma<double>(h->m, h->tet, h->Dinv, Xd, h->gam64, h->st);
  EMU_CK(cudaGetLastError());
  {
    int rc = bones_after_gamma(h);  // the bones' mean mode gradients and constant capacitance terms
    if (rc) return rc;
  }
  // coarse space of the ACAP preconditioner: Phi and (Phi^T L Phi)^+
  EMU_CK(cudaMemcpyAsync(h->phi64, Xd, n * 16 * 8, cudaMemcpyDeviceToDevice, h->st));
  if (h->mixed) launch_d2f(n * 16, h->phi64, h->phi32, h->st);
  launch_galerkin16(n, h->rowptr, h->col, h->val, h->phi64, Yd, ggrid, h->part_pcg, h->st);
  launch_reduce_cols(h->part_pcg, ggrid, 256, h->small, h->st);
  EMU_CK(cudaGetLastError());
  std::vector<double> Eg(256);
  EMU_CK(cudaMemcpyAsync(Eg.data(), h->small, 256 * 8, cudaMemcpyDeviceToHost, h->st));
  EMU_CK(cudaStreamSynchronize(h->st));
  for (int i = 0; i < 16; ++i)
    for (int j = 0; j < 16; ++j) Eg[16 * i + j] = 0.5 * (Eg[16 * i + j] + Eg[16 * j + i]);
  if (h->fform) {
    // Lambda = Phi^T K Phi of Eqs. 9-12 for the 48 columns (coordinate r,
    // scalar mode j) at 16 r + j: K = L (x) I_3, so three copies of E
    std::vector<double> lam(kCapEntries + kK, 0.0);
    for (int r = 0; r < 3; ++r)
      for (int i = 0; i < 16; ++i)
        for (int j = 0; j < 16; ++j) lam[(16 * r + i) * kK + 16 * r + j] = Eg[16 * i + j];
    EMU_CK(cudaMemcpyAsync(h->lam_add, lam.data(), lam.size() * 8, cudaMemcpyHostToDevice, h->st));
    EMU_CK(cudaStreamSynchronize(h->st));
  }
  std::vector<double> Ev;
  host_jacobi_eig(Eg, Ev, 16);
  double emax = 0.0;
  for (int i = 0; i < 16; ++i) emax = std::max(emax, Eg[17 * i]);
  std::vector<double> Ei(256, 0.0);
  for (int k = 0; k < 16; ++k) {
    const double lk = Eg[17 * k];
    if (!(lk > 1e-12 * emax)) continue;
    for (int i = 0; i < 16; ++i)
      for (int j = 0; j < 16; ++j) Ei[16 * i + j] += Ev[16 * i + k] * Ev[16 * j + k] / lk;
  }
  EMU_CK(cudaMemcpyAsync(h->Einv, Ei.data(), 256 * 8, cudaMemcpyHostToDevice, h->st));
  if (h->mixed && h->rpt32 > 0)
    EMU_CK(launch_aphi32(n, h->rowptr, h->col, h->val32, h->phi32, h->aphi32, h->st));
  if (h->cg_part) {  // the coarse rows in the partition order of the pipelined CG
    EMU_CK(launch_gather_rows16(n, h->cg_perm, h->phi32, h->cg_phi, h->st));
    EMU_CK(launch_gather_rows16(n, h->cg_perm, h->aphi32, h->cg_aphi, h->st));
  }
  EMU_CK(cudaStreamSynchronize(h->st));
  h->coarse_ready = emax > 0.0;
  h->aphi_ready = h->mixed && h->rpt32 > 0;
  return EMU_OK;
}

// Zeroes the per-tet iteration arrays of the kernels in use (bone tets keep
// zero gradient, y and chart factor throughout).
bool zero_tet_work(emu_handle* h) {
  const int64_t m = h->m;
  bool ok = cudaMemsetAsync(h->g, 0, 72 * m, h->st) == cudaSuccess;
  if (h->y64) ok = ok && cudaMemsetAsync(h->y64, 0, 72 * m, h->st) == cudaSuccess &&
                   cudaMemsetAsync(h->Uw64, 0, 432 * m, h->st) == cudaSuccess &&
                   cudaMemsetAsync(h->d64, 0, 72 * m, h->st) == cudaSuccess;
  if (h->y32) ok = ok && cudaMemsetAsync(h->y32, 0, 36 * m, h->st) == cudaSuccess &&
                   cudaMemsetAsync(h->Uw32, 0, 216 * m, h->st) == cudaSuccess &&
                   cudaMemsetAsync(h->d32, 0, 36 * m, h->st) == cudaSuccess &&
                   cudaMemsetAsync(h->g32, 0, 36 * m, h->st) == cudaSuccess;
  return ok && cudaStreamSynchronize(h->st) == cudaSuccess;
}

// Every device buffer of a handle (n, m, mixed and sms set). In dry mode
// (h->dry) nothing is allocated and h->dry_bytes receives the total.
bool alloc_device(emu_handle* h, int64_t nnz) {
  const int64_t n = h->n, m = h->m;
  bool ok = true;
  ok = ok && h->get(h->tet, m) && h->get(h->Dinv, 9 * m) && h->get(h->V, m) && h->get(h->c, m) && h->get(h->w, m) &&
       h->get(h->mu, m) && h->get(h->lam, m) && h->get(h->u, 3 * m) && h->get(h->ka, m);
  ok = ok && h->get(h->R, 9 * m) && h->get(h->s, 6 * m) && h->get(h->q, 3 * n) && h->get(h->dq, 3 * n) &&
       h->get(h->q0, 3 * n) && h->get(h->g, 9 * m) && h->get(h->contrib, 12 * m) && h->get(h->b, 16 * n);
  if (h->mixed) {
    ok = ok && h->get(h->gam32, 48 * m) && h->get(h->y32, 9 * m) && h->get(h->d32, 9 * m) && h->get(h->Uw32, 54 * m);
    ok = ok && h->get(h->Dinv32, 9 * m) && h->get(h->V32, m) && h->get(h->c32, m) && h->get(h->w32, m) &&
         h->get(h->sw32, m) &&
         h->get(h->mu32, m) && h->get(h->lam32, m) && h->get(h->u32, 3 * m) && h->get(h->ka32, m) &&
         h->get(h->E32, 6 * m) && h->get(h->g32, 9 * m) && h->get(h->quat, m) && h->get(h->dq32, 3 * n) &&
         h->get(h->b32, 3 * n) && h->get(h->r32, 3 * n) && h->get(h->e32, 3 * n) && h->get(h->fr, 3 * n) &&
         h->get(h->fu, 3 * n) && h->get(h->fw, 3 * n) && h->get(h->fp, 3 * n) && h->get(h->fs, 3 * n) &&
         h->get(h->E0, 9 * m) && h->get(h->Qrest, 3 * n) && h->get(h->contrib32, 12 * m) &&
         h->get(h->uh32, 3 * n) && h->get(h->ul32, 3 * n);
  } else
    ok = ok && h->get(h->gam64, 48 * m) && h->get(h->y64, 9 * m) && h->get(h->d64, 9 * m) && h->get(h->Uw64, 54 * m);
  ok = ok && h->get(h->pr, 16 * n) && h->get(h->pu, 16 * n) && h->get(h->pw, 16 * n) && h->get(h->pp, 16 * n) &&
       h->get(h->ps, 16 * n) && h->get(h->scratch16, 32 * n) && h->get(h->phi64, 16 * n) && h->get(h->Einv, 256);
  if (h->mixed) {
    ok = ok && h->get(h->phi32, 16 * n) && h->get(h->ug32, 2 * n) && h->get(h->part32, 128 * (int64_t)h->sms) &&
         h->get(h->sync32, 96) && h->get(h->aphi32, 16 * n);
    if (!pcg32_shape(n, h->sms, &h->grid32, &h->rpt32)) h->rpt32 = 0;
    // partitioned system of the pipelined CG (a dry run counts the widest table)
    if (h->dry ? (h->rpt32 > 0 && pcg32_pipe_ok(h->rpt32)) : h->cg_part) {
      const int lw = h->dry ? cg_local_width_max(h->rpt32) : h->cg_lw;
      ok = ok && h->get(h->cg_perm, n) && h->get(h->cg_off, h->grid32 + 1) && h->get(h->cg_rowptr, n + 1) &&
           h->get(h->cg_col, nnz) && h->get(h->cg_val, nnz) && h->get(h->cg_dinv, n) && h->get(h->cg_phi, 16 * n) &&
           h->get(h->cg_aphi, 16 * n) &&
           h->get(h->cg_loc, std::max<int64_t>(1, (int64_t)h->grid32 * h->rpt32 * lw * kPcg32Threads));
    }
  }
  h->grid_tet = (int)std::min<int64_t>(std::max<int64_t>(1, (m + 127) / 128), 8 * (int64_t)h->sms);
  h->grid_syrk = (int)std::min<int64_t>(std::max<int64_t>(1, (m + 23) / 24), 2 * (int64_t)h->sms);
  h->grid_tet4 = (int)std::min<int64_t>(std::max<int64_t>(1, (m + 127) / 128), 4 * (int64_t)h->sms);
  h->grid_pcg3 = pcg_max_grid(3, n);
  h->grid_pcg16 = pcg_max_grid(16, n);
  // the autotuner may take up to one block per 64 rows for the FP64 CG
  const int g3max = h->prm.autotune ? std::max<int>(h->grid_pcg3, (int)std::min<int64_t>((n + 63) / 64, h->sms))
                                    : h->grid_pcg3;
  const int pcg_part = std::max(g3max * (4 * 3 + 3 * kModes), h->grid_pcg16 * 64);  // per-block partials
  const int64_t gpart = std::max<int64_t>(h->grid_tet * (int64_t)kLsNV, 256 * (int64_t)(2 * h->sms + 1));
  ok = ok && h->get(h->part_grad, gpart) && h->get(h->part_dir, h->grid_tet + 1) && h->get(h->part_ls, (h->grid_tet + kBoneLsBlocks) * kLsNV) &&
       h->get(h->part_pcg, std::max<int64_t>(pcg_part, 256 * (int64_t)(2 * h->sms + 1))) &&
       h->get(h->cpart, std::max<int64_t>(h->grid_syrk, std::max(kTcBlocksPerSM, kSyrk05BlocksPerSM) * (int64_t)h->sms) *
                            (kCapEntries + kK)) && h->get(h->z, kK) && h->get(h->cfull, kCapEntries + kK) && h->get(h->small, 256) &&
       h->get(h->sc, 1) && h->get(h->bar, 1);
  if (h->mixed) ok = ok && h->get(h->val32, nnz) && h->get(h->ldinv32, n);
  ok = ok && h->get(h->rowptr, n + 1) && h->get(h->col, nnz) && h->get(h->val, nnz) && h->get(h->ldinv, n) &&
       h->get(h->bfix, 3 * n) && h->get(h->qfix, 3 * n) && h->get(h->is_fixed, n) && h->get(h->slot_ptr, n + 1) &&
       h->get(h->slot_idx, 4 * m);
  if (h->fform) ok = ok && h->get(h->lam_add, kCapEntries + kK);
  ok = ok && bones_alloc(h);
  return ok;
}

int compute_gref(emu_handle* h) {
  TetArgs<double> a = h->args<double>();
  launch_gref(a, h->q0, h->grid_tet, h->part_grad, h->small, h->st);
  bones_gref(h, h->small);  // the free bones' |g(I)|^2 (their tets are skipped above)
  double g2 = 0.0;
  EMU_CK(cudaMemcpyAsync(&g2, h->small, 8, cudaMemcpyDeviceToHost, h->st));
  EMU_CK(cudaStreamSynchronize(h->st));
  h->gref = std::sqrt(g2);
  h->gref_valid = true;
  return EMU_OK;
}

}  // namespace

namespace emu {
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

bool acap_view(const emu_handle* h, AcapView* v) {
  if (!h || !v) return false;
  v->device = h->device;
  v->npts = h->npts;
  v->n = h->n;
  v->m = h->m;
  v->tet = h->tet;
  v->Dinv = h->Dinv;
  v->w = h->w;
  v->slot_ptr = h->slot_ptr;
  v->slot_idx = h->slot_idx;
  v->bfix = h->bfix;
  v->is_fixed = h->is_fixed;
  v->qfix = h->qfix;
  v->rowptr = h->rowptr;
  v->col = h->col;
  v->val = h->val;
  v->ldinv = h->ldinv;
  v->phi = h->coarse_ready ? h->phi64 : nullptr;
  v->Einv = h->coarse_ready ? h->Einv : nullptr;
  v->q0 = h->q0;
  v->grid_pcg = h->grid_pcg3;
  v->pcg_max = h->prm.pcg_max;
  v->pcg_tol = h->q_tol;
  v->sms = h->sms;
  return true;
}
}  // namespace emu

// ============================================================== C ABI =====
extern "C" {

void emu_default_params(emu_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->alpha_rel = 1.0;
  p->weight_mode = 0;
  p->k_modes = 48;
  p->fiber_scale = 1.0;
  p->tol_rel_residual = 1e-6;
  p->max_newton = 2000;
  p->ls_sigma0 = 4.0;
  p->ls_c = 1e-4;
  p->ls_rho = 0.5;
  p->ls_max_trials = 40;
  p->pcg_tol = 1e-8;
  p->pcg_max = 5000;
  p->precision = EMU_PRECISION_FP64;
  p->mode_iters = 8;
  p->dq_tol = 8e-2;
  p->q_refresh = 32;
  p->seed = 12345;
  p->eps_bone = -1e-3;
  p->eps_joint = -1e-4;
  p->cg_local_degree = 4;
  p->form = EMU_FORM_RS;
  p->autotune = 0;
}

const char* emu_status_string(int status) {
  switch (status) {
    case EMU_OK: return "ok";
    case EMU_ERR_INVALID_ARG: return "invalid argument";
    case EMU_ERR_DEGENERATE_TET: return "degenerate tet";
    case EMU_ERR_OOM: return "out of device memory";
    case EMU_ERR_NOT_CONVERGED: return "not converged";
    case EMU_ERR_LINESEARCH: return "line search failed";
    case EMU_ERR_PCG: return "ACAP solve did not converge";
    case EMU_ERR_INVERTED: return "non-finite gradient or inverted element";
    case EMU_ERR_TIMEOUT: return "device wait timed out";
    case EMU_ERR_CUDA: return "CUDA error";
    case EMU_ERR_NOT_IMPLEMENTED: return "not implemented";
    default: return "unknown status";
  }
}

const char* emu_last_error(void) { return g_last_error.c_str(); }

int emu_destroy(emu_handle* h) {
  if (!h) return EMU_OK;
  h->release();
  delete h;
  return EMU_OK;
}

int emu_create(const emu_mesh_desc* desc, const emu_params* params, const emu_allocator* alloc, void* stream,
               emu_handle** out) {
  if (!out) return fail(EMU_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int rc = validate_mesh(desc);
  if (rc) return rc;
  emu_params prm;
  if (params)
    prm = *params;
  else
    emu_default_params(&prm);
  rc = validate_params(&prm);
  if (rc) return rc;
  if (prm.form == EMU_FORM_F) {
    // the F-form runs the FP64 kernels on meshes without bones or joints
    if (prm.precision != EMU_PRECISION_FP64)
      return fail(EMU_ERR_NOT_IMPLEMENTED, "the F-form runs in FP64 only");
    bool bones = desc->n_joints > 0;
    for (int64_t i = 0; i < desc->n_tets && !bones && desc->bone_id; ++i) bones = desc->bone_id[i] >= 0;
    if (bones) return fail(EMU_ERR_NOT_IMPLEMENTED, "the F-form is not combined with bones");
  }

  emu_handle* h = new (std::nothrow) emu_handle();
  if (!h) return fail(EMU_ERR_OOM, "host allocation failed");
  h->prm = prm;
  h->sigma0_now = prm.ls_sigma0;
  h->st = (cudaStream_t)stream;
  if (alloc && alloc->alloc && alloc->free) {
    h->alloc = *alloc;
    h->has_alloc = true;
  }
  h->mixed = prm.precision == EMU_PRECISION_MIXED;
  h->fform = prm.form == EMU_FORM_F;
  h->kmodes = prm.k_modes / 3;
  const int64_t n = desc->n_verts, m = desc->n_tets;
  h->n = n;
  h->m = m;
  // ---- geometry (Eq. 2), volumes, orientation ----
  const double* Q = desc->rest_pos;
  std::vector<int32_t> tet(4 * m);
  std::vector<double> Dinv(9 * m), V(m);
  for (int64_t i = 0; i < m; ++i) {
    int32_t t[4] = {desc->tets[4 * i], desc->tets[4 * i + 1], desc->tets[4 * i + 2], desc->tets[4 * i + 3]};
    auto build = [&](double* Dm) {
      for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) Dm[3 * r + k] = Q[3 * t[k] + r] - Q[3 * t[3] + r];
    };
    double Dm[9];
    build(Dm);
    double det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
                 Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
    if (det < 0.0) {
      std::swap(t[1], t[2]);
      build(Dm);
      det = -det;
    }
    double hmax = 0.0;
    for (int a_ = 0; a_ < 4; ++a_)
      for (int b_ = a_ + 1; b_ < 4; ++b_) {
        double dx = Q[3 * t[a_]] - Q[3 * t[b_]], dy = Q[3 * t[a_] + 1] - Q[3 * t[b_] + 1],
               dz = Q[3 * t[a_] + 2] - Q[3 * t[b_] + 2];
        hmax = std::max(hmax, std::sqrt(dx * dx + dy * dy + dz * dz));
      }
    if (!(det > 1e-14 * hmax * hmax * hmax)) {
      delete h;
      return fail(EMU_ERR_DEGENERATE_TET, "degenerate tet " + std::to_string(i));
    }
    double Di[9];
    Di[0] = (Dm[4] * Dm[8] - Dm[5] * Dm[7]) / det;
    Di[1] = (Dm[2] * Dm[7] - Dm[1] * Dm[8]) / det;
    Di[2] = (Dm[1] * Dm[5] - Dm[2] * Dm[4]) / det;
    Di[3] = (Dm[5] * Dm[6] - Dm[3] * Dm[8]) / det;
    Di[4] = (Dm[0] * Dm[8] - Dm[2] * Dm[6]) / det;
    Di[5] = (Dm[2] * Dm[3] - Dm[0] * Dm[5]) / det;
    Di[6] = (Dm[3] * Dm[7] - Dm[4] * Dm[6]) / det;
    Di[7] = (Dm[1] * Dm[6] - Dm[0] * Dm[7]) / det;
    Di[8] = (Dm[0] * Dm[4] - Dm[1] * Dm[3]) / det;
    for (int k = 0; k < 9; ++k) Dinv[k * m + i] = Di[k];
    V[i] = det / 6.0;
    for (int k = 0; k < 4; ++k) tet[4 * i + k] = t[k];
  }

  if (h->mixed) {
    // The FP32 kernels see D_m^-1 and V rounded to FP32; the FP64 Laplacian
    // and right-hand sides are built from the same rounded values.
    for (int64_t k = 0; k < 9 * m; ++k) Dinv[k] = (double)(float)Dinv[k];
    for (int64_t i = 0; i < m; ++i) V[i] = (double)(float)V[i];
  }

  // ---- pins ----
  std::vector<uint8_t> is_fixed(n, 0);
  std::vector<double> qfix(Q, Q + 3 * n);
  for (int64_t k = 0; k < desc->n_fixed; ++k) {
    const int32_t v = desc->fixed_verts[k];
    is_fixed[v] = 1;
    if (desc->fixed_pos)
      for (int r = 0; r < 3; ++r) qfix[3 * v + r] = desc->fixed_pos[3 * k + r];
  }

  // ---- bones and joints (Sec. 3.3) ----
  rc = bones_prepare(h, desc, tet, V, is_fixed);
  if (rc) {
    delete h;
    return rc;
  }

  // ---- materials, weights (Eq. 3 with the Sec. 3.3 weights option) ----
  std::vector<double> mu(m), lam(m), wv(m), cv(m), uv(3 * m, 0.0);
  double mu_ref = 1e300, mu_ref_all = 1e300;
  for (int64_t i = 0; i < m; ++i) {
    const int k = desc->material_id[i];
    const double E = desc->youngs[k], nu = desc->poisson[k];
    mu[i] = E / (2.0 * (1.0 + nu));
    lam[i] = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    mu_ref_all = std::min(mu_ref_all, mu[i]);
    // mu_ref: the softest material that is not bone
    if (!h->has_bones || h->tkind_h[i] == kTetDeformable) mu_ref = std::min(mu_ref, mu[i]);
  }
  if (mu_ref > 1e299) mu_ref = mu_ref_all;
  h->mu_ref = mu_ref;
  h->alpha = prm.alpha_rel * mu_ref;
  h->kappa = prm.fiber_scale * mu_ref;
  double fl = 0.0;
  for (int64_t i = 0; i < m; ++i) wv[i] = prm.weight_mode == 1 ? V[i] * std::max(1.0, mu[i] / mu_ref) : V[i];
  bones_weights(h, V, wv);  // bone tets: V_i + Vbar / |eps_bone|
  for (int64_t i = 0; i < m; ++i) {
    if (h->mixed) wv[i] = (double)(float)wv[i];
    cv[i] = h->alpha * wv[i];
    fl += (V[i] * mu[i]) * (V[i] * mu[i]);
    if (desc->fiber_dir) {
      double x = desc->fiber_dir[3 * i], y = desc->fiber_dir[3 * i + 1], z = desc->fiber_dir[3 * i + 2];
      double nrm = std::sqrt(x * x + y * y + z * z);
      if (!(nrm > 0.0) || !std::isfinite(nrm)) {
        delete h;
        return fail(EMU_ERR_INVALID_ARG, "fiber direction must be non-zero and finite");
      }
      uv[i] = x / nrm;
      uv[m + i] = y / nrm;
      uv[2 * m + i] = z / nrm;
    }
  }
  h->floor = 1e-12 * std::sqrt(fl);
  h->V_h = V;
  bones_weight_sums(h, wv);
  h->q_tol = std::max(1e-13, std::min(prm.pcg_tol, 1e-2 * prm.tol_rel_residual));

  // ---- scalar ACAP Laplacian L_ab = sum_i w_i gradN_a . gradN_b (Eq. 4) ----
  std::vector<std::pair<int64_t, double>> trip;
  trip.reserve(16 * m);
  std::vector<double> bfix(3 * n, 0.0);
  for (int64_t i = 0; i < m; ++i) {
    double gN[4][3];
    for (int k = 0; k < 3; ++k)
      for (int c2 = 0; c2 < 3; ++c2) gN[k][c2] = Dinv[(3 * k + c2) * m + i];
    for (int c2 = 0; c2 < 3; ++c2) gN[3][c2] = -(gN[0][c2] + gN[1][c2] + gN[2][c2]);
    for (int a_ = 0; a_ < 4; ++a_) {
      const int32_t va = tet[4 * i + a_];
      if (is_fixed[va]) continue;
      for (int b_ = 0; b_ < 4; ++b_) {
        const int32_t vb = tet[4 * i + b_];
        const double lv = wv[i] * (gN[a_][0] * gN[b_][0] + gN[a_][1] * gN[b_][1] + gN[a_][2] * gN[b_][2]);
        if (is_fixed[vb]) {
          for (int r = 0; r < 3; ++r) bfix[3 * va + r] += lv * qfix[3 * vb + r];
        } else {
          trip.push_back({(int64_t)va * n + vb, lv});
        }
      }
    }
  }
  for (int64_t v = 0; v < n; ++v)
    if (is_fixed[v]) trip.push_back({v * n + v, 1.0});
  std::sort(trip.begin(), trip.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  std::vector<int32_t> rowptr(n + 1, 0), colv;
  std::vector<double> valv, ldinv(n, 1.0);
  colv.reserve(trip.size());
  valv.reserve(trip.size());
  for (size_t k = 0; k < trip.size();) {
    const int64_t key = trip[k].first;
    double s_ = 0.0;
    while (k < trip.size() && trip[k].first == key) s_ += trip[k++].second;
    const int64_t r = key / n, cc = key % n;
    colv.push_back((int32_t)cc);
    valv.push_back(s_);
    rowptr[r + 1]++;
    if (r == cc) ldinv[r] = 1.0 / s_;
  }
  for (int64_t v = 0; v < n; ++v) rowptr[v + 1] += rowptr[v];
  for (int64_t v = 0; v < n; ++v)
    if (!is_fixed[v] && rowptr[v + 1] == rowptr[v]) {
      delete h;
      return fail(EMU_ERR_INVALID_ARG, "vertex " + std::to_string(v) + " is in no tet and not pinned");
    }

  // ---- corner slots per vertex (atomic-free gather of G^T W X) ----
  std::vector<int32_t> slot_ptr(n + 1, 0), slot_idx(4 * m);
  for (int64_t k = 0; k < 4 * m; ++k) slot_ptr[tet[k] + 1]++;
  for (int64_t v = 0; v < n; ++v) slot_ptr[v + 1] += slot_ptr[v];
  {
    std::vector<int32_t> fillp(slot_ptr.begin(), slot_ptr.end() - 1);
    for (int64_t k = 0; k < 4 * m; ++k) slot_idx[fillp[tet[k]]++] = (int32_t)k;
  }

  // final-solve operator of the bones (Sec. 3.3)
  rc = bones_final_host(h, tet, Dinv, wv, is_fixed);
  if (rc) {
    delete h;
    return rc;
  }

  // ---- device allocation (every host-side check has passed) ----
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    delete h;
    return fail(EMU_ERR_CUDA, "no CUDA device");
  }
  h->device = dev;
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nnz = (int64_t)colv.size();
  // row partition and local preconditioner of the pipelined FP32 CG
  CgPartHost cgp;
  if (h->mixed) {
    int g32 = 0, r32 = 0;
    if (pcg32_shape(n, h->sms, &g32, &r32) && pcg32_pipe_ok(r32))
      h->cg_part = build_cg_partition(n, Q, rowptr, colv, valv, g32, r32, kPcg32Threads, prm.cg_local_degree, &cgp);
    if (h->cg_part) {
      h->cg_lw = cgp.lw;
      h->cg_degree = cgp.degree;
      h->cg_lmax = cgp.lmax;
      h->cg_c0 = cgp.c0;
      for (int i = 0; i < kChebMax; ++i) {
        h->cg_c1[i] = cgp.c1[i];
        h->cg_c2[i] = cgp.c2[i];
      }
    }
  }
  bool ok = alloc_device(h, nnz);
  if (!ok) {
    h->release();
    delete h;
    return fail(EMU_ERR_OOM, "device allocation failed");
  }
  if (cudaMallocHost(&h->sc_host, sizeof(DevScalars)) != cudaSuccess ||
      cudaMallocHost(&h->o6_host, 16 * sizeof(double)) != cudaSuccess) {
    h->release();
    delete h;
    return fail(EMU_ERR_OOM, "pinned host allocation failed");
  }
  if (cudaEventCreateWithFlags(&h->wait_ev, cudaEventDisableTiming) != cudaSuccess) {
    h->release();
    delete h;
    return fail(EMU_ERR_CUDA, "cudaEventCreate failed");
  }
  // kernel attributes are set here, outside any stream capture
  if (h->mixed && (prepare_syrk_tc() != cudaSuccess || prepare_pcg32() != cudaSuccess)) {
    h->release();
    delete h;
    return fail(EMU_ERR_CUDA, "cudaFuncSetAttribute failed");
  }
  // the tcgen05 capacitance kernel where its bulk copies can run (else mma.sync)
  h->syrk05 = h->mixed && make_syrk05_maps(h->margs(), &h->syrk05_maps) && prepare_syrk05() == cudaSuccess;
  // barrier words of the FP32 CG start at zero (every launch leaves them so)
  if (h->sync32 && cudaMemsetAsync(h->sync32, 0, 96 * sizeof(unsigned), h->st) != cudaSuccess) {
    h->release();
    delete h;
    return fail(EMU_ERR_CUDA, "cudaMemsetAsync failed");
  }

  auto up = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->st) == cudaSuccess;
  };
  std::vector<double> zeros(m, 0.0);
  ok = up(h->tet, tet.data(), 16 * m) && up(h->Dinv, Dinv.data(), 72 * m) && up(h->V, V.data(), 8 * m) &&
       up(h->c, cv.data(), 8 * m) && up(h->w, wv.data(), 8 * m) && up(h->mu, mu.data(), 8 * m) &&
       up(h->lam, lam.data(), 8 * m) && up(h->u, uv.data(), 24 * m) && up(h->ka, zeros.data(), 8 * m) &&
       up(h->rowptr, rowptr.data(), 4 * (n + 1)) && up(h->col, colv.data(), 4 * nnz) && up(h->val, valv.data(), 8 * nnz) &&
       up(h->ldinv, ldinv.data(), 8 * n) && up(h->bfix, bfix.data(), 24 * n) && up(h->qfix, qfix.data(), 24 * n) &&
       up(h->is_fixed, is_fixed.data(), n) && up(h->slot_ptr, slot_ptr.data(), 4 * (n + 1)) &&
       up(h->slot_idx, slot_idx.data(), 16 * m) && up(h->q, qfix.data(), 24 * n);
  if (ok && h->mixed) {
    auto f32 = [](const std::vector<double>& v) {
      std::vector<float> f(v.size());
      for (size_t k = 0; k < v.size(); ++k) f[k] = (float)v[k];
      return f;
    };
    std::vector<float> Df = f32(Dinv), Vf = f32(V), cf = f32(cv), wf = f32(wv), muf = f32(mu), lf = f32(lam),
                       uf = f32(uv), valf = f32(valv), ldf = f32(ldinv);
    std::vector<float> zf(m, 0.f), swf(m);
    for (int64_t i = 0; i < m; ++i) swf[i] = (float)std::sqrt(wv[i]);
    // E0_i = D_m D_m^-1 - I with the rounded D_m^-1 (FP64 arithmetic)
    std::vector<float> e0f(9 * m);
    for (int64_t i = 0; i < m; ++i) {
      const int32_t* t = &tet[4 * i];
      for (int r = 0; r < 3; ++r)
        for (int c2 = 0; c2 < 3; ++c2) {
          double acc = (r == c2) ? -1.0 : 0.0;
          for (int k = 0; k < 3; ++k) acc += (Q[3 * t[k] + r] - Q[3 * t[3] + r]) * Dinv[(3 * k + c2) * m + i];
          e0f[(3 * r + c2) * m + i] = (float)acc;
        }
    }
    ok = up(h->E0, e0f.data(), 36 * m) && up(h->Qrest, Q, 24 * n) && up(h->Dinv32, Df.data(), 36 * m) && up(h->V32, Vf.data(), 4 * m) && up(h->c32, cf.data(), 4 * m) &&
         up(h->w32, wf.data(), 4 * m) && up(h->sw32, swf.data(), 4 * m) && up(h->mu32, muf.data(), 4 * m) &&
         up(h->lam32, lf.data(), 4 * m) &&
         up(h->u32, uf.data(), 12 * m) && up(h->ka32, zf.data(), 4 * m) && up(h->val32, valf.data(), 4 * nnz) &&
         up(h->ldinv32, ldf.data(), 4 * n) && cudaStreamSynchronize(h->st) == cudaSuccess;
    if (ok && h->cg_part) {
      ok = up(h->cg_perm, cgp.perm.data(), 4 * n) && up(h->cg_off, cgp.off.data(), 4 * (h->grid32 + 1)) &&
           up(h->cg_rowptr, cgp.rowptr.data(), 4 * (n + 1)) && up(h->cg_col, cgp.col.data(), 4 * cgp.col.size()) &&
           up(h->cg_val, cgp.val.data(), 4 * cgp.val.size()) && up(h->cg_dinv, cgp.dinv.data(), 4 * n) &&
           (cgp.loc.empty() || up(h->cg_loc, cgp.loc.data(), 4 * cgp.loc.size())) &&
           cudaStreamSynchronize(h->st) == cudaSuccess;
    }
  }
  if (!ok || cudaMemsetAsync(h->sc, 0, sizeof(DevScalars), h->st) != cudaSuccess) {
    h->release();
    delete h;
    return fail(EMU_ERR_CUDA, "upload failed");
  }
  // tets of bones are never written by the gradient kernels: their
  // per-iteration g, y, U stay zero (the capacitance and B y skip them)
  if (h->has_bones) {
    ok = zero_tet_work(h) && bones_upload(h, Q) == EMU_OK;
    if (!ok) {
      h->release();
      delete h;
      return fail(EMU_ERR_CUDA, "bone set-up upload failed");
    }
  }

  // ---- rest state: R = I, S = I, q = q*(I) ----
  rc = set_rest_state(h);
  // the normaliser of the exact solve is the residual at q0: here q0 = Q
  if (!rc && cudaMemcpyAsync(h->q0, h->q, 24 * n, cudaMemcpyDeviceToDevice, h->st) != cudaSuccess)
    rc = fail(EMU_ERR_CUDA, "copy q0");
  if (!rc) rc = joints_setup_device(h);  // joint corrections for the coupling solves
  if (!rc) rc = refresh_q(h, h->q_tol);
  if (!rc && cudaMemcpyAsync(h->q0, h->q, 24 * n, cudaMemcpyDeviceToDevice, h->st) != cudaSuccess)
    rc = fail(EMU_ERR_CUDA, "copy q0");
  if (!rc) rc = build_modes(h);
  if (!rc) rc = final_setup_device(h);
  if (!rc && h->prm.autotune) rc = autotune(h);
  if (!rc) rc = read_scalars(h);
  if (!rc && h->sc_host->barrier_timeout) rc = fail(EMU_ERR_TIMEOUT, "grid barrier timed out during setup");
  if (rc) {
    h->release();
    delete h;
    return rc;
  }
  *out = h;
  return EMU_OK;
}

int emu_set_activation(emu_handle* h, const double* a, int64_t count) {
  if (!h || !a) return fail(EMU_ERR_INVALID_ARG, "NULL argument");
  if (count != h->m) return fail(EMU_ERR_INVALID_ARG, "activation count must equal n_tets");
  std::vector<double> ka(h->m);
  for (int64_t i = 0; i < h->m; ++i) {
    if (!(a[i] >= 0.0) || !std::isfinite(a[i])) return fail(EMU_ERR_INVALID_ARG, "activation must be finite and >= 0");
    if (h->has_bones && a[i] != 0.0 && h->tkind_h[i] != kTetDeformable)
      return fail(EMU_ERR_INVALID_ARG, "activation must be 0 on bone tets");
    ka[i] = h->kappa * a[i];
  }
  EMU_CK(cudaMemcpyAsync(h->ka, ka.data(), 8 * h->m, cudaMemcpyHostToDevice, h->st));
  std::vector<float> kaf;
  if (h->mixed) {
    kaf.resize(h->m);
    for (int64_t i = 0; i < h->m; ++i) kaf[i] = (float)ka[i];
    EMU_CK(cudaMemcpyAsync(h->ka32, kaf.data(), 4 * h->m, cudaMemcpyHostToDevice, h->st));
  }
  EMU_CK(cudaStreamSynchronize(h->st));
  h->gref_valid = false;
  return EMU_OK;
}

int emu_set_external_forces(emu_handle* h, const double* f, int64_t n_verts) {
  if (!h) return fail(EMU_ERR_INVALID_ARG, "NULL handle");
  if (!f) {
    h->has_force = false;
  } else {
    if (n_verts != h->n) return fail(EMU_ERR_INVALID_ARG, "n_verts must equal the mesh's vertex count");
    if (h->has_bones) return fail(EMU_ERR_NOT_IMPLEMENTED, "external forces are not combined with bones");
    const int64_t n = h->n, m = h->m;
    for (int64_t k = 0; k < 3 * n; ++k)
      if (!std::isfinite(f[k])) return fail(EMU_ERR_INVALID_ARG, "forces must be finite");
    if (!h->nu64 && !h->get(h->nu64, 9 * m)) return fail(EMU_ERR_OOM, "device allocation failed");
    if (h->mixed && !h->nu32 && !h->get(h->nu32, 9 * m)) return fail(EMU_ERR_OOM, "device allocation failed");
    // right-hand side: f on the free rows; the pinned rows are identity rows with 0
    std::vector<uint8_t> fixed(n);
    EMU_CK(cudaMemcpyAsync(fixed.data(), h->is_fixed, n, cudaMemcpyDeviceToHost, h->st));
    EMU_CK(cudaStreamSynchronize(h->st));
    std::vector<double> fb(f, f + 3 * n);
    for (int64_t v = 0; v < n; ++v)
      if (fixed[v]) fb[3 * v] = fb[3 * v + 1] = fb[3 * v + 2] = 0.0;
    double* rhs = h->b;
    double* x = h->b + 3 * n;
    DevScalars init;
    memset(&init, 0, sizeof(init));
    EMU_CK(cudaMemcpyAsync(h->sc, &init, sizeof(init), cudaMemcpyHostToDevice, h->st));
    EMU_CK(cudaMemcpyAsync(rhs, fb.data(), 24 * n, cudaMemcpyHostToDevice, h->st));
    EMU_CK(cudaMemsetAsync(x, 0, 24 * n, h->st));
    EMU_CK(launch_pcg<double>(3, h->pcg64(rhs, x, 1e-13), h->grid_pcg3, h->st));
    launch_nu(m, h->tet, h->Dinv, h->w, x, h->nu64, h->mixed ? h->nu32 : nullptr, h->st);
    EMU_CK(cudaGetLastError());
    DevScalars out;
    EMU_CK(cudaMemcpyAsync(&out, h->sc, sizeof(out), cudaMemcpyDeviceToHost, h->st));
    EMU_CK(cudaStreamSynchronize(h->st));
    if (out.barrier_timeout) return fail(EMU_ERR_TIMEOUT, "grid barrier timed out in the force solve");
    if (out.pcg_fail) return fail(EMU_ERR_PCG, "the solve for the generalized force did not converge");
    h->has_force = true;
  }
  // g(I) changes; the captured iteration graph holds the old kernel arguments
  h->gref_valid = false;
  if (h->iter_exec) cudaGraphExecDestroy(h->iter_exec);
  h->iter_exec = nullptr;
  return EMU_OK;
}

int emu_set_activation_device(emu_handle* h, const double* a_device, int64_t count) {
  if (!h || !a_device) return fail(EMU_ERR_INVALID_ARG, "NULL argument");
  if (count != h->m) return fail(EMU_ERR_INVALID_ARG, "activation count must equal n_tets");
  std::vector<double> a(h->m);
  EMU_CK(cudaMemcpyAsync(a.data(), a_device, 8 * h->m, cudaMemcpyDeviceToHost, h->st));
  EMU_CK(cudaStreamSynchronize(h->st));
  return emu_set_activation(h, a.data(), count);
}

}  // extern "C"

namespace emu {

// One quasi-static solve (Algorithm 1) as a resumable task. step() enqueues
// work on the handle's stream up to the next point where the host must read
// a device result (the residual of an exact coupling solve, the gradient
// norm and line-search state of an iteration), records wait_ev there and
// returns 1; once that work has finished, the next step() takes the decision
// and enqueues the following stretch. A single solve steps it with blocking
// waits; a batch or the server interleaves many handles' tasks on their own
// streams so their work overlaps on the device.
struct SolveTask {
  enum Phase { START, TOP, REF_RES, REF_CHECK, GRAD, DECIDE, FINISH, DONE };
  emu_handle* h = nullptr;
  emu_solve_stats* stats = nullptr;
  Phase phase = START;
  int it = 0, since = 0, round = 0;
  int status = EMU_OK;
  double res = 0.0, gnorm_ref = 0.0;
  bool first_eval = true;
  bool ls_refreshed = false;  // q re-solved during the current run of rejected passes
  bool ref_short = false;     // the last exact re-solve stopped above its tolerance
  bool ls_retried = false;    // and dq tightened after it, too
  double best_res = 1e300;    // smallest residual so far and the iteration it was seen
  int best_it = 0;
  std::chrono::steady_clock::time_point t0;
};

SolveTask* task_new(emu_handle* h, emu_solve_stats* stats) {
  SolveTask* t = new (std::nothrow) SolveTask;
  if (!t) return nullptr;
  t->h = h;
  t->stats = stats;
  return t;
}
void task_delete(SolveTask* t) { delete t; }
int task_status(const SolveTask* t) { return t->status; }
bool task_done(const SolveTask* t) { return t->phase == SolveTask::DONE; }
bool task_ready(const SolveTask* t) {
  // a failed query (not "not ready") is surfaced by the next step's calls
  return cudaEventQuery(t->h->wait_ev) != cudaErrorNotReady;
}

namespace {
// enqueue the gradient and its reduction, then wait for the scalars
int enqueue_grad(emu_handle* h) {
  h->ph_begin();
  if (h->mixed) {
    // the displacement's float pair for this iteration's per-tet kernels
    launch_split_disp(h->n, h->q, h->Qrest, h->uh32, h->ul32, h->st);
    launch_grad_mixed(h->margs(), h->grid_tet4, h->st);
  } else if (h->fform) {
    launch_grad_fform(h->args<double>(), h->grid_tet, h->st);
  } else {
    launch_grad<double>(h->args<double>(), h->grid_tet, h->st);
  }
  h->ph_end(EMU_PHASE_GRAD, h->mixed ? 2 : 1);
  if (!h->mixed) {  // the mixed gradient kernel reduces ||g||^2 in its last block
    h->ph_begin();
    launch_reduce_grad(h->part_grad, h->grid_tet, h->sc, nullptr, nullptr, h->st);
    h->ph_end(EMU_PHASE_SMALL, 1);
  }
  if (h->nfb > 0) {  // the free bones' virtual elements (Sec. 3.3)
    h->ph_begin();
    bones_after_grad(h);
    h->ph_end(EMU_PHASE_SMALL, 0);
  }
  EMU_CK(cudaGetLastError());
  EMU_CK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->st));
  return EMU_OK;
}

// the Woodbury direction (Eqs. 9-12) and its corner terms
int enqueue_direction(emu_handle* h) {
  TetArgs<double> a64 = h->args<double>();
  MixArgs am = h->margs();
  h->ph_begin();
  int syrk_blocks = h->grid_syrk;
  if (h->mixed && h->syrk05) {
    syrk_blocks = syrk05_grid(h->m, h->sms);
    launch_syrk05(am, h->syrk05_maps, syrk_blocks, h->cpart, h->st);
  } else if (h->mixed) {
    syrk_blocks = (int)std::min<int64_t>(std::max<int64_t>(1, (h->m + 31) / 32), kTcBlocksPerSM * (int64_t)h->sms);
    launch_syrk_tc(am, syrk_blocks, h->cpart, h->st);
  } else if (h->fform) {
    launch_syrk_fform(a64, h->grid_syrk, h->cpart, h->st);
  } else {
    launch_syrk<double>(a64, h->grid_syrk, h->cpart, h->st);
  }
  h->ph_end(EMU_PHASE_SYRK, 1);
  h->ph_begin();
  // the 48 x 48 factor in FP32 on the mixed path, in FP64 with bones (their
  // 1/|eps_bone|-weighted terms widen the capacitance's spectrum)
  launch_cap_solve(h->cpart, syrk_blocks, h->cfull, h->z, h->sc, h->mixed && !h->has_bones, h->st,
                   h->fform ? h->lam_add : bones_cap_addend(h));
  bones_before_dir(h);
  h->ph_end(EMU_PHASE_SMALL, 2);
  h->ph_begin();
  if (h->mixed) {
    MixArgs ad = am;
    ad.partials = h->part_dir;
    launch_dir_mixed(ad, h->grid_tet, h->st);
  } else {
    TetArgs<double> ad = a64;
    ad.partials = h->part_dir;
    if (h->fform)
      launch_dir_fform(ad, h->grid_tet, h->st);
    else
      launch_dir<double>(ad, h->grid_tet, h->st);
  }
  h->ph_end(EMU_PHASE_DIR, 1);
  EMU_CK(cudaGetLastError());
  return EMU_OK;
}

// enqueue the rest of one Newton iteration: direction, dq, line search, update
int enqueue_step(emu_handle* h) {
  TetArgs<double> a64 = h->args<double>();
  MixArgs am = h->margs();
  int rc = enqueue_direction(h);
  if (rc) return rc;
  rc = solve_dq(h);
  if (rc) return rc;
  // Armijo line search (Algorithm 1)
  h->ph_begin();
  if (h->mixed) {
    MixArgs al = am;
    al.partials = h->part_ls;
    LsSelect sel;  // the line-search kernel's last block selects the step
    sel.dir_partials = h->part_dir;
    sel.nblk_dir = dir_partial_count(h);
    sel.sigma0 = h->sigma0_now;
    sel.rho = h->prm.ls_rho;
    sel.c_armijo = h->prm.ls_c;
    if (h->nfb > 0) {  // the free bones' terms in FP64, after the kernel's own partials
      launch_bone_ls(h->bargs(), h->dq32, h->prm.ls_rho, h->part_ls + (size_t)h->grid_tet4 * kLsNV, h->st);
      sel.nblk_extra = kBoneLsBlocks;
    }
    launch_ls_mixed(al, h->grid_tet4, sel, h->st);
    h->ph_end(EMU_PHASE_LS, 1);
  } else {
    TetArgs<double> al = a64;
    al.partials = h->part_ls;
    int nls = h->grid_tet;
    if (h->nfb > 0) {  // the free bones' terms, after the per-tet partials
      launch_bone_ls(h->bargs(), h->dq, h->prm.ls_rho, h->part_ls + (size_t)h->grid_tet * kLsNV, h->st);
      nls += kBoneLsBlocks;
    }
    if (h->fform)
      launch_ls_fform(al, h->grid_tet, h->prm.ls_rho, h->st);
    else
      launch_ls<double>(al, h->grid_tet, h->prm.ls_rho, h->st);
    h->ph_end(EMU_PHASE_LS, 1);
    h->ph_begin();
    launch_ls_select(h->part_dir, dir_partial_count(h), h->part_ls, nls, h->sc, h->sigma0_now, h->prm.ls_rho,
                     h->prm.ls_c, h->st);
    h->ph_end(EMU_PHASE_SMALL, 1);
  }
  h->ph_begin();
  if (h->mixed) {
    launch_update_mixed(am, h->grid_tet, h->st);
    bones_update_mixed(h);
    if (cg64(h))
      launch_update_verts(h->n, h->sc, h->dq, h->q, h->st);
    else
      launch_update_verts_f(h->n, h->sc, h->dq32, h->q, h->st);
  } else {
    if (h->fform)
      launch_update_fform(a64, h->grid_tet, h->st);
    else
      launch_update_tets<double>(a64, h->grid_tet, h->st);
    launch_update_verts(h->n, h->sc, h->dq, h->q, h->st);
  }
  h->ph_end(EMU_PHASE_UPDATE, 2);
  EMU_CK(cudaGetLastError());
  return EMU_OK;
}
// Enqueues enqueue_step + enqueue_grad as one CUDA graph launch (captured
// on first use and again when the dq tolerance or first trial step changes). Returns 1 when the
// graph was launched, 0 when the caller must enqueue directly (profiling
// on, the legacy default stream, or a capture that failed).
int launch_iteration_graph(emu_handle* h) {
  if (!h->graphs_ok || h->prof_on || h->st == nullptr) return 0;
  if (!h->iter_exec || h->iter_exec_dq != h->dq_tol_now || h->iter_exec_sigma0 != h->sigma0_now) {
    if (h->iter_exec) cudaGraphExecDestroy(h->iter_exec);
    h->iter_exec = nullptr;
    if (cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      h->graphs_ok = false;
      return 0;
    }
    const int64_t launches0 = h->launches;
    int rc = enqueue_step(h);
    if (!rc) rc = enqueue_grad(h);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->st, &g);
    h->iter_graph_kernels = h->launches - launches0;  // kernels of one launch
    h->launches = launches0;                          // nothing ran yet
    cudaGraphExec_t ex = nullptr;
    if (rc || e != cudaSuccess || !g || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      h->graphs_ok = false;
      return 0;
    }
    cudaGraphDestroy(g);
    h->iter_exec = ex;
    h->iter_exec_dq = h->dq_tol_now;
    h->iter_exec_sigma0 = h->sigma0_now;
  }
  if (cudaGraphLaunch(h->iter_exec, h->st) != cudaSuccess) {
    cudaGetLastError();
    h->graphs_ok = false;
    return 0;
  }
  h->launches += h->iter_graph_kernels;
  return 1;
}
void drop_iteration_graph(emu_handle* h) {
  if (h->iter_exec) cudaGraphExecDestroy(h->iter_exec);
  h->iter_exec = nullptr;
  h->iter_exec_dq = -1.0;
}

// dq tolerance a solve starts with: params.dq_tol, or the tighter one a
// stalled earlier solve settled on (with_base). With free bones (Sec. 3.3)
// at most kBoneDqTol: a bone tet's ACAP weight carries the 1/|eps_bone|
// penalty, and a loosely solved dq misses how the soft tissue follows the
// bone, so the line search rejects steps (measured on the arm assemblies:
// 576 tets FP64, 452 Newton iterations and a line-search failure near
// 1.6e-10 at 5e-2 against 74 iterations to 1e-10 at 1e-6; 40,152 tets FP64,
// 2,856 iterations over three frames at 5e-2 against 608 at 1e-4).
constexpr double kBoneDqTol = 1e-4;
double start_dq_tol(const emu_handle* h, bool with_base = true) {
  double t = (with_base && h->dq_tol_base > 0.0) ? h->dq_tol_base : h->prm.dq_tol;
  if (h->nfb > 0) t = std::min(t, kBoneDqTol);
  return t;
}

// Precision escalation of a mixed handle whose residual has stalled at the
// rounding floor of its FP32 per-tet arithmetic: the state (quaternion, E)
// is converted to (R, s) and the FP64 kernels take over for the rest of the
// solve (their per-tet buffers are allocated on first use). Positions q are
// FP64 on both paths. Returns false when it cannot (allocation failed).
bool escalate(emu_handle* h) {
  if (!h->mixed || h->escalated) return false;
  if (!h->gam64) {
    const int64_t m = h->m;
    if (!(h->get(h->gam64, 48 * m) && h->get(h->y64, 9 * m) && h->get(h->d64, 9 * m) && h->get(h->Uw64, 54 * m)))
      return false;
    if (h->has_bones && !zero_tet_work(h)) return false;
    launch_gamma<double>(m, h->tet, h->Dinv, h->phi64, h->gam64, h->st);
  }
  launch_mixed_to_Rs(h->m, h->quat, h->E32, h->R, h->s, h->st);
  bones_state_to_element_arrays(h);  // the FP64 kernels keep a bone's state in its tets
  if (cudaMemsetAsync(h->dq, 0, 24 * h->n, h->st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return false;
  drop_iteration_graph(h);
  h->mixed = false;
  h->escalated = true;
  return true;
}

// Back to the mixed kernels at the end of an escalated solve.
void deescalate(emu_handle* h) {
  if (!h->escalated) return;
  bones_state_from_rep(h);
  launch_Rs_to_mixed(h->m, h->R, h->s, h->quat, h->E32, h->st);
  cudaMemsetAsync(h->dq32, 0, 12 * h->n, h->st);
  drop_iteration_graph(h);
  h->mixed = true;
  h->escalated = false;
}
}  // namespace

int task_step(SolveTask* t) {
  emu_handle* h = t->h;
  auto wait = [&]() {
    if (cudaEventRecord(h->wait_ev, h->st) != cudaSuccess) {
      t->status = fail(EMU_ERR_CUDA, "cudaEventRecord failed");
      t->phase = SolveTask::DONE;
      return 0;
    }
    return 1;
  };
  auto abort = [&](int rc) {
    deescalate(h);
    t->status = rc;
    t->phase = SolveTask::DONE;
    return 0;
  };
  const double tol = h->prm.tol_rel_residual;
  for (;;) {
    int rc = EMU_OK;
    switch (t->phase) {
      case SolveTask::START: {
        t->t0 = std::chrono::steady_clock::now();
        if (!h->gref_valid) {
          rc = compute_gref(h);
          if (rc) return abort(rc);
        }
        DevScalars init;
        memset(&init, 0, sizeof(init));
        init.sigma_start = h->sigma0_now;
        if (cudaMemcpyAsync(h->sc, &init, sizeof(init), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
          return abort(fail(EMU_ERR_CUDA, "cudaMemcpyAsync failed"));
        t->gnorm_ref = h->gref > h->floor ? h->gref : 0.0;
        t->since = h->prm.q_refresh;  // iterations since q was last solved exactly
        // dq starts from zero in every solve: the result depends only on the
        // element state, q and the activation (resume from
        // emu_set_element_state is bit-for-bit an uninterrupted run)
        if (cudaMemsetAsync(h->dq, 0, 24 * h->n, h->st) != cudaSuccess ||
            (h->dq32 && cudaMemsetAsync(h->dq32, 0, 12 * h->n, h->st) != cudaSuccess))
          return abort(fail(EMU_ERR_CUDA, "cudaMemsetAsync failed"));
        h->dq_tol_now = start_dq_tol(h);
        t->phase = SolveTask::TOP;
        break;
      }
      case SolveTask::TOP:
        // q = q*(F) exactly every q_refresh iterations; in between q follows
        // q*(F + s d) = q + s dq (Eq. 4 is affine in F).
        if (t->since >= h->prm.q_refresh) {
          rc = refresh_begin(h, h->q_tol);
          if (rc) return abort(rc);
          t->round = 0;
          t->phase = SolveTask::REF_RES;
          break;
        }
        t->phase = SolveTask::GRAD;
        break;
      case SolveTask::REF_RES:
        rc = refresh_residual(h);
        if (rc) return abort(rc);
        t->phase = SolveTask::REF_CHECK;
        return wait();
      case SolveTask::REF_CHECK: {
        h->prof_flush();
        const bool conv = refresh_converged(h, h->q_tol);
        if (conv || t->round + 1 >= kRefreshRounds) {
          t->ref_short = !conv;
          t->since = 0;
          t->phase = SolveTask::GRAD;
          break;
        }
        rc = refresh_correction(h, refresh_round_tol(h, h->q_tol));
        if (rc) return abort(rc);
        ++t->round;
        t->phase = SolveTask::REF_RES;
        break;
      }
      case SolveTask::GRAD:
        rc = enqueue_grad(h);
        if (rc) return abort(rc);
        t->phase = SolveTask::DECIDE;
        return wait();
      case SolveTask::DECIDE: {
        h->prof_flush();
        const DevScalars& hs = *h->sc_host;
        if (hs.barrier_timeout) {
          t->status = fail(EMU_ERR_TIMEOUT, "grid barrier timed out");
          t->phase = SolveTask::FINISH;
          break;
        }
        if (hs.nonfinite || !std::isfinite(hs.gnorm2)) {
          t->status = fail(EMU_ERR_INVERTED, "non-finite gradient");
          t->phase = SolveTask::FINISH;
          break;
        }
        if (t->ref_short && hs.pcg_fail) {
          // the exact coupling solve (Eq. 4) stopped above its tolerance
          // because its CG solves ran into pcg_max
          t->status = fail(EMU_ERR_PCG, "the coupling solve reached pcg_max before its tolerance");
          t->phase = SolveTask::FINISH;
          break;
        }
        const double gn = std::sqrt(hs.gnorm2);
        if (t->first_eval && t->gnorm_ref == 0.0) t->gnorm_ref = gn > h->floor ? gn : 0.0;
        t->first_eval = false;
        t->res = t->gnorm_ref > 0.0 ? gn / t->gnorm_ref : 0.0;
        if (t->res < t->best_res * (1.0 - 1e-3)) {
          t->best_res = t->res;
          t->best_it = t->it;
        }
        // Stalled just above the tolerance: the residual has stopped falling.
        // Three causes are known, each with a remedy tried in turn before the
        // solve gives up with the state kept: trial steps longer than the
        // quasi-Newton step, which the energy test accepts while the gradient
        // zig-zags (first trial 1 from then on), the rounding floor of the
        // FP32 per-tet arithmetic relative to a normaliser that vanishes with
        // the activation (finish on the FP64 kernels), and q drifting from
        // q*(F) between exact re-solves when dq is solved loosely and the
        // steps are long (solve dq 100x tighter). The first and last persist
        // into later solves on the handle.
        if (t->res > tol && t->best_res <= kStallBand * tol) {
          if (t->it - t->best_it >= kEscalateIters) {
            const double dq_tight = std::max(h->q_tol, 1e-2 * start_dq_tol(h, false));
            bool restart = false;
            if (h->sigma0_now > 1.0) {
              h->sigma0_now = 1.0;
              restart = true;
            } else if (h->mixed && escalate(h)) {
              h->dq_tol_now = start_dq_tol(h);
              restart = true;
            } else if (h->dq_tol_now > dq_tight) {
              // later solves on this handle (the next frames) start tight
              h->dq_tol_now = h->dq_tol_base = dq_tight;
              restart = true;
            }
            if (restart) {  // from an exact q, with a fresh line search
              launch_ls_reset(h->sc, h->sigma0_now, h->st);
              t->best_it = t->it;
              t->since = h->prm.q_refresh;
              t->ls_refreshed = t->ls_retried = false;
              t->phase = SolveTask::TOP;
              break;
            }
          }
          if (t->it - t->best_it >= kStallIters) {
            t->status = fail(EMU_ERR_NOT_CONVERGED, "residual stalled above the tolerance");
            t->phase = SolveTask::FINISH;
            break;
          }
        }
        if (t->res <= tol) {
          if (t->since > 0) {  // confirm with an exact q before declaring convergence
            t->since = h->prm.q_refresh;
            t->phase = SolveTask::TOP;
          } else {
            t->phase = SolveTask::FINISH;
          }
          break;
        }
        if (hs.sigma > 0.0) t->ls_retried = t->ls_refreshed = false;  // the last pass accepted a step
        // Rejected passes while q follows F only through the loose dq solves
        // mean that q has drifted from q*(F): the slope the Armijo test uses
        // then no longer matches the energy (a loose residual can leave a
        // large error in the K-norm). Re-solve q exactly after two rejected
        // passes, and restart the line search.
        if (hs.ls_fail >= 2 && t->since > 0 && !t->ls_refreshed) {
          launch_ls_reset(h->sc, h->sigma0_now, h->st);
          t->since = h->prm.q_refresh;
          t->ls_refreshed = true;
          t->phase = SolveTask::TOP;
          break;
        }
        if (hs.ls_fail * kLsTrials >= h->prm.ls_max_trials) {
          if (!t->ls_retried) {
            // still no step with an exact q: solve dq tightly from now on
            // (q then stays exact along the steps) and give it one more run
            launch_ls_reset(h->sc, h->sigma0_now, h->st);
            if (t->since > 0) t->since = h->prm.q_refresh;
            h->dq_tol_now = h->q_tol;
            t->ls_retried = true;
            t->phase = SolveTask::TOP;
            break;
          }
          t->status = fail(EMU_ERR_LINESEARCH, "no Armijo step");
          t->phase = SolveTask::FINISH;
          break;
        }
        if (t->it >= h->prm.max_newton) {
          t->status = fail(EMU_ERR_NOT_CONVERGED, "max_newton reached");
          t->phase = SolveTask::FINISH;
          break;
        }
        ++t->it;
        ++t->since;
        // an iteration with no exact re-solve of q after it runs as one graph
        if (t->since < h->prm.q_refresh && launch_iteration_graph(h)) {
          t->phase = SolveTask::DECIDE;
          return wait();
        }
        rc = enqueue_step(h);
        if (rc) return abort(rc);
        t->phase = SolveTask::TOP;
        break;
      }
      case SolveTask::FINISH: {
        deescalate(h);
        if (cudaStreamSynchronize(h->st) != cudaSuccess) return abort(fail(EMU_ERR_CUDA, "cudaStreamSynchronize failed"));
        // with free bones, the final coupling solve of Sec. 3.3 gives the positions
        if (h->nfb > 0 && (t->status == EMU_OK || t->status == EMU_ERR_NOT_CONVERGED)) {
          const int frc = bones_final_solve(h);
          if (frc) return abort(frc);
        }
        h->prof_flush();
        auto t1 = std::chrono::steady_clock::now();
        if (t->stats) {
          t->stats->newton_iters = t->it;
          t->stats->ls_trials = h->sc_host->ls_trials;
          t->stats->pcg_iters = h->sc_host->pcg_iters;
          t->stats->status = t->status;
          t->stats->rel_residual = t->res;
          t->stats->energy_change = h->sc_host->dE;
          t->stats->ms = std::chrono::duration<double, std::milli>(t1 - t->t0).count();
        }
        t->phase = SolveTask::DONE;
        return 0;
      }
      case SolveTask::DONE:
        return 0;
    }
  }
}

}  // namespace emu

extern "C" {

int emu_solve_quasistatic(emu_handle* h, emu_solve_stats* stats) {
  if (!h) return fail(EMU_ERR_INVALID_ARG, "NULL handle");
  SolveTask t;
  t.h = h;
  t.stats = stats;
  while (task_step(&t)) {
    if (cudaEventSynchronize(h->wait_ev) != cudaSuccess) return fail(EMU_ERR_CUDA, "cudaEventSynchronize failed");
  }
  return t.status;
}

int emu_required_bytes(const emu_mesh_desc* desc, const emu_params* params, size_t* bytes) {
  if (!bytes) return fail(EMU_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = 0;
  int rc = validate_mesh(desc);
  if (rc) return rc;
  emu_params prm;
  if (params)
    prm = *params;
  else
    emu_default_params(&prm);
  rc = validate_params(&prm);
  if (rc) return rc;
  emu_handle h;
  h.dry = true;
  h.prm = prm;
  h.n = desc->n_verts;
  h.m = desc->n_tets;
  h.mixed = prm.precision == EMU_PRECISION_MIXED;
  h.fform = prm.form == EMU_FORM_F;
  if (desc->bone_id)
    for (int64_t i = 0; i < h.m && !h.has_bones; ++i) h.has_bones = desc->bone_id[i] >= 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(EMU_ERR_CUDA, "no CUDA device");
  if (cudaDeviceGetAttribute(&h.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(EMU_ERR_CUDA, "cudaDeviceGetAttribute failed");
  // the Laplacian has at most 16 entries per tet plus one per pinned row
  alloc_device(&h, 16 * h.m + h.n);
  *bytes = h.dry_bytes;
  return EMU_OK;
}

int emu_batch_solve(emu_handle* const* hs, int32_t count, emu_solve_stats* stats) {
  if (count < 0 || (count > 0 && !hs)) return fail(EMU_ERR_INVALID_ARG, "emu_batch_solve: bad handle array");
  for (int32_t i = 0; i < count; ++i) {
    if (!hs[i]) return fail(EMU_ERR_INVALID_ARG, "emu_batch_solve: NULL handle");
    for (int32_t j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(EMU_ERR_INVALID_ARG, "emu_batch_solve: a handle appears twice");
  }
  std::vector<SolveTask> ts(count);
  std::vector<char> waiting(count, 0);
  int32_t live = 0;
  for (int32_t i = 0; i < count; ++i) {
    ts[i].h = hs[i];
    ts[i].stats = stats ? stats + i : nullptr;
    waiting[i] = (char)task_step(&ts[i]);
    live += waiting[i];
  }
  while (live > 0) {
    bool progressed = false;
    for (int32_t i = 0; i < count; ++i) {
      if (!waiting[i] || !task_ready(&ts[i])) continue;
      waiting[i] = (char)task_step(&ts[i]);
      if (!waiting[i]) --live;
      progressed = true;
    }
    if (!progressed) std::this_thread::yield();
  }
  std::string first_err;
  int status = EMU_OK;
  for (int32_t i = 0; i < count; ++i)
    if (ts[i].status != EMU_OK && status == EMU_OK) status = ts[i].status;
  if (status != EMU_OK) set_last_error("emu_batch_solve: at least one solve failed (see the per-handle stats)");
  return status;
}

int emu_get_positions(emu_handle* h, double* out, int32_t out_is_device) {
  if (!h || !out) return fail(EMU_ERR_INVALID_ARG, "NULL argument");
  EMU_CK(cudaMemcpyAsync(out, h->q, 24 * h->n, out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
  EMU_CK(cudaStreamSynchronize(h->st));
  return EMU_OK;
}

int emu_get_element_state(emu_handle* h, double* R, double* s, double* F) {
  if (!h) return fail(EMU_ERR_INVALID_ARG, "NULL handle");
  const int64_t m = h->m;
  std::vector<double> tmp(9 * m);
  auto soa_to_aos = [&](const double* dsrc, int k, double* dst) -> int {
    EMU_CK(cudaMemcpyAsync(tmp.data(), dsrc, 8 * k * m, cudaMemcpyDeviceToHost, h->st));
    EMU_CK(cudaStreamSynchronize(h->st));
    for (int64_t i = 0; i < m; ++i)
      for (int j = 0; j < k; ++j) dst[k * i + j] = tmp[j * m + i];
    return EMU_OK;
  };
  int rc;
  if (h->mixed) {
    launch_mixed_to_Rs(m, h->quat, h->E32, h->R, h->s, h->st);
    bones_state_to_element_arrays(h);  // the bones' FP64 states
    EMU_CK(cudaGetLastError());
  }
  if (h->fform) {
    // the state is F itself; R and s from its polar decomposition (in the
    // corner and direction buffers, which each iteration rewrites)
    if (R || s) {
      launch_fform_to_Rs(m, h->R, h->contrib, h->d64, h->st);
      EMU_CK(cudaGetLastError());
    }
    if (R && (rc = soa_to_aos(h->contrib, 9, R))) return rc;
    if (s && (rc = soa_to_aos(h->d64, 6, s))) return rc;
    if (F && (rc = soa_to_aos(h->R, 9, F))) return rc;
    return EMU_OK;
  }
  if (R && (rc = soa_to_aos(h->R, 9, R))) return rc;
  if (s && (rc = soa_to_aos(h->s, 6, s))) return rc;
  if (F) {
    launch_compose_F(m, h->R, h->s, h->contrib, h->st);
    EMU_CK(cudaGetLastError());
    if ((rc = soa_to_aos(h->contrib, 9, F))) return rc;
  }
  return EMU_OK;
}

int emu_set_element_state(emu_handle* h, const double* R, const double* s, const double* q) {
  if (!h) return fail(EMU_ERR_INVALID_ARG, "NULL handle");
  const int64_t m = h->m;
  if (h->fform && (R || s) && (!R || !s)) {
    // F-form: the untouched factor comes from the current F = R S
    std::vector<double> Rc(9 * m), sc_(6 * m);
    int rc = emu_get_element_state(h, R ? nullptr : Rc.data(), s ? nullptr : sc_.data(), nullptr);
    if (rc) return rc;
    return emu_set_element_state(h, R ? R : Rc.data(), s ? s : sc_.data(), q);
  }
  std::vector<double> tmp(9 * m);
  if (R) {
    for (int64_t i = 0; i < m; ++i)
      for (int j = 0; j < 9; ++j) tmp[j * m + i] = R[9 * i + j];
    EMU_CK(cudaMemcpyAsync(h->R, tmp.data(), 72 * m, cudaMemcpyHostToDevice, h->st));
    EMU_CK(cudaStreamSynchronize(h->st));
  }
  if (s) {
    for (int64_t i = 0; i < m; ++i)
      for (int j = 0; j < 6; ++j) tmp[j * m + i] = s[6 * i + j];
    EMU_CK(cudaMemcpyAsync(h->s, tmp.data(), 48 * m, cudaMemcpyHostToDevice, h->st));
    EMU_CK(cudaStreamSynchronize(h->st));
  }
  if (h->mixed && (R || s) && (!R || !s)) {
    // keep the untouched part: bring the current state to (R, s) first
    std::vector<double> Rc(9 * m), sc_(6 * m);
    int rc = emu_get_element_state(h, R ? nullptr : Rc.data(), s ? nullptr : sc_.data(), nullptr);
    if (rc) return rc;
    return emu_set_element_state(h, R ? R : Rc.data(), s ? s : sc_.data(), q);
  }
  if (h->has_bones && (R || s)) {
    // a free bone's tets share one state: every copy takes its first tet's
    bones_state_from_element_arrays(h);
    EMU_CK(cudaGetLastError());
  }
  if (h->fform && (R || s)) {  // F = R S in place of R
    launch_compose_F(m, h->R, h->s, h->R, h->st);
    EMU_CK(cudaGetLastError());
    EMU_CK(cudaStreamSynchronize(h->st));
  }
  if (h->mixed && (R || s)) {
    launch_Rs_to_mixed(m, h->R, h->s, h->quat, h->E32, h->st);
    EMU_CK(cudaGetLastError());
    EMU_CK(cudaStreamSynchronize(h->st));
  }
  if (q) {
    EMU_CK(cudaMemcpyAsync(h->q, q, 24 * h->n, cudaMemcpyHostToDevice, h->st));
    EMU_CK(cudaStreamSynchronize(h->st));
  }
  return EMU_OK;
}

int emu_reset(emu_handle* h) {
  if (!h) return fail(EMU_ERR_INVALID_ARG, "NULL handle");
  int rc = set_rest_state(h);
  if (rc) return rc;
  h->dq_tol_base = 0.0;
  h->sigma0_now = h->prm.ls_sigma0;
  EMU_CK(cudaMemcpyAsync(h->q, h->q0, 24 * h->n, cudaMemcpyDeviceToDevice, h->st));
  EMU_CK(cudaStreamSynchronize(h->st));
  return EMU_OK;
}

int emu_get_sizes(emu_handle* h, int64_t* n_verts, int64_t* n_tets, int32_t* k_modes) {
  if (!h) return fail(EMU_ERR_INVALID_ARG, "NULL handle");
  if (n_verts) *n_verts = h->n;
  if (n_tets) *n_tets = h->m;
  if (k_modes) *k_modes = 3 * h->kmodes;
  return EMU_OK;
}

int emu_set_profiling(emu_handle* h, int32_t enable) {
  if (!h) return fail(EMU_ERR_INVALID_ARG, "NULL handle");
  EMU_CK(cudaStreamSynchronize(h->st));
  h->prof_flush();
  h->prof_on = enable != 0;
  for (int k = 0; k < EMU_N_PHASES; ++k) {
    h->prof_ms[k] = 0.0;
    h->prof_cnt[k] = 0;
  }
  h->launches = 0;
  return EMU_OK;
}

int emu_get_profile(emu_handle* h, double* phase_ms, int32_t* phase_launches, int32_t n_phases,
                    int64_t* total_launches) {
  if (!h || n_phases < 0 || n_phases > EMU_N_PHASES) return fail(EMU_ERR_INVALID_ARG, "bad arguments");
  EMU_CK(cudaStreamSynchronize(h->st));
  h->prof_flush();
  for (int k = 0; k < n_phases; ++k) {
    if (phase_ms) phase_ms[k] = h->prof_ms[k];
    if (phase_launches) phase_launches[k] = h->prof_cnt[k];
  }
  if (total_launches) *total_launches = h->launches;
  return EMU_OK;
}

int emu_eval_stretch_terms(const double* s, const double* params, int64_t n, int32_t mixed, double* psi,
                           double* grad, double* hess, void* stream) {
  if (!s || !params || n < 0) return fail(EMU_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return EMU_OK;
  launch_eval_stretch(s, params, n, mixed, psi, grad, hess, (cudaStream_t)stream);
  EMU_CK(cudaGetLastError());
  EMU_CK(cudaStreamSynchronize((cudaStream_t)stream));
  return EMU_OK;
}

int emu_eval_fform_terms(const double* F, const double* params, int64_t n, double* psi, double* grad, double* hess,
                         void* stream) {
  if (!F || !params || n < 0) return fail(EMU_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return EMU_OK;
  launch_eval_fform(F, params, n, psi, grad, hess, (cudaStream_t)stream);
  EMU_CK(cudaGetLastError());
  EMU_CK(cudaStreamSynchronize((cudaStream_t)stream));
  return EMU_OK;
}

int emu_get_tuning(emu_handle* h, int32_t* cg_local_degree, int32_t* cg64_rows_per_block, int32_t* tuned) {
  if (!h) return fail(EMU_ERR_INVALID_ARG, "NULL handle");
  if (cg_local_degree) *cg_local_degree = h->cg_part ? h->cg_degree : 0;
  if (cg64_rows_per_block) *cg64_rows_per_block = h->cg64_rows;
  if (tuned) *tuned = h->tuned ? 1 : 0;
  return EMU_OK;
}

int emu_check_bounded_wait(int64_t wait_ns, void* stream) {
  if (wait_ns < 1000 || wait_ns > 10000000000ll) return fail(EMU_ERR_INVALID_ARG, "wait_ns must be in [1e3, 1e10]");
  cudaStream_t st = (cudaStream_t)stream;
  void* buf = nullptr;
  EMU_CK(cudaMalloc(&buf, 256));
  int timed_out = 0;
  cudaError_t e = launch_wait_check(static_cast<GridBarrier*>(buf), (unsigned long long)wait_ns,
                                    reinterpret_cast<int*>(static_cast<char*>(buf) + 128), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&timed_out, static_cast<char*>(buf) + 128, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return fail(EMU_ERR_CUDA, std::string("emu_check_bounded_wait: ") + cudaGetErrorString(e));
  if (timed_out) return fail(EMU_ERR_TIMEOUT, "the check's grid-barrier wait ran out after its limit (as designed)");
  return EMU_OK;
}

int emu_eval_capacitance(int64_t m, const float* U, const float* gamma, const float* y, const float* w,
                         int32_t kernel, double* C, double* By, void* stream) {
  if (m <= 0 || m > (int64_t)1 << 28 || !U || !gamma || !y || !w || !C || !By || kernel < 0 || kernel > 2)
    return fail(EMU_ERR_INVALID_ARG, "bad arguments");
  if (kernel == 1 && m % 4 != 0) return fail(EMU_ERR_INVALID_ARG, "the tcgen05 kernel needs m % 4 == 0");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  EMU_CK(cudaGetDevice(&dev));
  EMU_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  EMU_CK(prepare_syrk_tc());
  EMU_CK(prepare_syrk05());
  const int64_t rows = 54 + 48 + 9 + 2;  // U, gamma, y, w, sqrt(w)
  float* dbuf = nullptr;
  double* cpart = nullptr;
  const int grid_max = std::max(kTcBlocksPerSM, kSyrk05BlocksPerSM) * sms;
  EMU_CK(cudaMalloc(&dbuf, sizeof(float) * rows * m));
  cudaError_t e = cudaMalloc(&cpart, sizeof(double) * (size_t)grid_max * (kCapEntries + kK));
  MixArgs a{};
  a.m = m;
  a.Uw = dbuf;
  a.gam = dbuf + 54 * m;
  a.y = dbuf + 102 * m;
  a.w = dbuf + 111 * m;
  a.sw = dbuf + 112 * m;
  std::vector<float> swh(m);
  for (int64_t i = 0; i < m; ++i) swh[i] = (float)std::sqrt((double)std::max(w[i], 0.f));
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbuf + 112 * m, swh.data(), sizeof(float) * m, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbuf, U, sizeof(float) * 54 * m, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbuf + 54 * m, gamma, sizeof(float) * 48 * m, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbuf + 102 * m, y, sizeof(float) * 9 * m, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbuf + 111 * m, w, sizeof(float) * m, cudaMemcpyHostToDevice, st);
  Syrk05Maps maps;
  const bool use05 = (kernel == 1 || kernel == 0) && make_syrk05_maps(a, &maps);
  if (kernel == 1 && !use05 && e == cudaSuccess) e = cudaErrorNotSupported;
  int grid = 0;
  if (use05) {
    grid = syrk05_grid(m, sms);
    if (e == cudaSuccess) launch_syrk05(a, maps, grid, cpart, st);
  } else {
    grid = (int)std::min<int64_t>(std::max<int64_t>(1, (m + 31) / 32), kTcBlocksPerSM * (int64_t)sms);
    if (e == cudaSuccess) launch_syrk_tc(a, grid, cpart, st);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  std::vector<double> part((size_t)grid * (kCapEntries + kK));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part.data(), cpart, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dbuf);
  cudaFree(cpart);
  if (e != cudaSuccess) return fail(EMU_ERR_CUDA, std::string("emu_eval_capacitance: ") + cudaGetErrorString(e));
  for (int k = 0; k < kCapEntries + kK; ++k) {
    double acc = 0.0;
    for (int b = 0; b < grid; ++b) acc += part[(size_t)k * grid + b];
    if (k < kCapEntries)
      C[k] = acc;
    else
      By[k - kCapEntries] = acc;
  }
  return EMU_OK;
}

int emu_eval_polar(const double* F, int64_t n, double* R, double* s, void* stream) {
  if (!F || !R || !s || n < 0) return fail(EMU_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return EMU_OK;
  launch_eval_polar(F, n, R, s, (cudaStream_t)stream);
  EMU_CK(cudaGetLastError());
  EMU_CK(cudaStreamSynchronize((cudaStream_t)stream));
  return EMU_OK;
}

}  // extern "C"
