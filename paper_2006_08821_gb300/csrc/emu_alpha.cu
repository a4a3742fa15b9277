// The alpha heuristic of Sec. 3.7 on the device solver: alpha_rel =
// alpha0 * factor^k, one solve from the rest state per value at the given
// activation, stopping at the first Newton count above jump times the
// previous one (a solve that does not converge counts as such an increase)
// and returning the value before it, or the last value tried.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "emu.h"
#include "emu_internal.h"

using namespace emu;

namespace {
int sweep_fail(int code, const std::string& msg) {
  set_last_error(msg.c_str());
  return code;
}
}  // namespace

extern "C" int emu_alpha_sweep(const emu_mesh_desc* desc, const emu_params* params, const double* activation,
                               double alpha0, double factor, int32_t max_steps, double jump, double* alpha_out,
                               int32_t* newton_iters, int32_t* n_tried, void* stream) {
  if (!desc || !activation || !alpha_out || !n_tried || max_steps < 1 || max_steps > 64 || !(alpha0 > 0.0) ||
      !(factor > 1.0) || !(jump > 1.0) || !std::isfinite(alpha0) || !std::isfinite(factor) || !std::isfinite(jump))
    return sweep_fail(EMU_ERR_INVALID_ARG, "bad arguments");
  emu_params base;
  if (params)
    base = *params;
  else
    emu_default_params(&base);
  int32_t prev = -1;  // -1: no previous count
  double alpha = alpha0;
  for (int32_t k = 0; k < max_steps; ++k, alpha *= factor) {
    emu_params p = base;
    p.alpha_rel = alpha;
    emu_handle* h = nullptr;
    int rc = emu_create(desc, &p, nullptr, stream, &h);
    if (rc != EMU_OK) return rc;
    rc = emu_set_activation(h, activation, desc->n_tets);
    emu_solve_stats st;
    int solve_rc = rc == EMU_OK ? emu_solve_quasistatic(h, &st) : rc;
    emu_destroy(h);
    if (solve_rc != EMU_OK && solve_rc != EMU_ERR_NOT_CONVERGED && solve_rc != EMU_ERR_LINESEARCH) return solve_rc;
    const bool converged = solve_rc == EMU_OK;
    const int32_t it = converged ? st.newton_iters : -1;
    if (newton_iters) newton_iters[k] = it;
    *n_tried = k + 1;
    const bool sharp = k > 0 && (!converged || (prev >= 0 && (double)it > jump * (double)prev));
    if (sharp) {
      *alpha_out = alpha / factor;
      return EMU_OK;
    }
    if (!converged && k == 0) {  // not even the first value converged
      *alpha_out = alpha;
      return sweep_fail(EMU_ERR_NOT_CONVERGED, "the solve at the first alpha did not converge");
    }
    prev = it;
    *alpha_out = alpha;
  }
  return EMU_OK;
}
