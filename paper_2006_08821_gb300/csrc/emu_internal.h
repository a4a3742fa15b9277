// Internal declarations shared by the host code and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/emu.h"

namespace emu {

constexpr int kModes = 16;          // scalar low-rank modes (k = 3 * kModes = 48)
constexpr int kK = 3 * kModes;      // Woodbury size k of Eq. 9
constexpr int kLsTrials = 4;        // line-search trials evaluated per pass
constexpr int kRedBlock = 256;      // threads of the single-block reducers

// Device-side scalars of one Newton iteration (one struct per handle).
struct DevScalars {
  double gnorm2;        // ||dE/dF||^2 (FP64)
  double gtd;           // g . d
  double sigma;         // accepted step (0 = rejected)
  double sigma_start;   // first trial of the next line search
  double dE;            // accumulated energy change of accepted steps
  double cap_ok;        // 1 if the capacitance Cholesky succeeded
  int32_t ls_trials;    // total trials evaluated
  int32_t ls_fail;      // consecutive rejected passes
  int32_t pcg_iters;    // CG iterations, summed
  int32_t pcg_fail;     // a CG solve hit pcg_max
  int32_t barrier_timeout;
  int32_t nonfinite;    // a non-finite value was produced
  uint32_t ticket[2];   // blocks done in the current gradient / line-search launch
};
constexpr int kTicketGrad = 0, kTicketLs = 1;

// Mesh constants on the device (structure of arrays, index i = tet).
template <typename T> struct MeshArrays {
  int64_t m, n;
  const int4* tet;      // m
  const T* Dinv;        // 9 m: Dinv[k * m + i], row-major 3x3 per tet
  const T* V;           // m
  const T* c;           // m: alpha * w_i
  const T* w;           // m
  const T* mu;          // m
  const T* lam;         // m
  const T* u;           // 3 m
  const T* ka;          // m: kappa * a_i
  const T* gam;         // 48 m: gam[(3 j + c) * m + i] = d phi_j / dx_c on tet i
};

// CSR of the scalar ACAP Laplacian (Eq. 4 with full-vertex pins: the
// 3n x 3n matrix is L (x) I_3). Pinned rows are identity.
struct Laplacian {
  int64_t n;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  const double* dinv;   // 1 / L_vv
};

// Read-only view of a handle's mesh operator, for entry points that live
// outside the handle's translation unit.
struct AcapView {
  int device;            // CUDA device the handle was created on
  int npts;              // joint rows (Sec. 3.3) of the handle's coupling problem
  int64_t n, m;
  const int4* tet;
  const double* Dinv;    // 9m structure of arrays
  const double* w;       // m
  const int32_t* slot_ptr;
  const int32_t* slot_idx;
  const double* bfix;
  const uint8_t* is_fixed;
  const double* qfix;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  const double* ldinv;
  const double* phi;     // null when the coarse space is not built
  const double* Einv;
  const double* q0;      // rest-state solution q*(I)
  int grid_pcg;
  int pcg_max;
  double pcg_tol;
  int sms;
};
bool acap_view(const emu_handle* h, AcapView* v);

// Bounded waits. Every spin-wait of the library's kernels (the grid barriers
// of the persistent CG kernels) gives up after kWaitLimitNs of GPU time (the
// %globaltimer clock), raises an error word that the other blocks see, and
// the kernel returns with a timeout flag the host reads (EMU_ERR_TIMEOUT).
// A spin-count cap backs the clock up.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s
constexpr unsigned long long kWaitSpinCap = 1ull << 28;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
void set_last_error(const char* msg);

// Resumable quasi-static solve of one handle (the same steps as
// emu_solve_quasistatic). task_step enqueues work on the handle's stream up
// to the next host decision and returns 1 while that work is in flight (poll
// task_ready), 0 once the solve has finished (task_status is its result).
struct SolveTask;
SolveTask* task_new(emu_handle* h, emu_solve_stats* stats);
int task_step(SolveTask* t);
bool task_ready(const SolveTask* t);
bool task_done(const SolveTask* t);
int task_status(const SolveTask* t);
void task_delete(SolveTask* t);

}  // namespace emu
