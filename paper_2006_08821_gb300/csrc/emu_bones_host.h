// Host side of affine bones and joints (Sec. 3.3): set-up steps called by
// emu_create and the launches the Newton loop adds for bones and joints.
#pragma once
#include <stdint.h>

#include <vector>

#include "../../include/emu.h"

struct emu_handle;

namespace emu {

// Classifies the bone tets (free / pinned bones, one material per bone, no
// shared vertices, pins all-or-none) and builds the joint rows. Needs
// h->prm, h->kmodes. EMU_ERR_INVALID_ARG with a message on a bad assembly.
int bones_prepare(emu_handle* h, const emu_mesh_desc* d, const std::vector<int32_t>& tet,
                  const std::vector<double>& V, const std::vector<uint8_t>& is_fixed);
// Bone tets' ACAP weights: V_i + Vbar / |eps_bone| (the Newton-phase penalty).
void bones_weights(emu_handle* h, const std::vector<double>& V, std::vector<double>& w);
// Keeps the final weights and sums them per free bone.
void bones_weight_sums(emu_handle* h, const std::vector<double>& w);
// Final-solve Laplacian (pins plus every bone vertex) and the right-hand
// sides of the bones' translation responses.
int bones_final_host(emu_handle* h, const std::vector<int32_t>& tet, const std::vector<double>& Dinv,
                     const std::vector<double>& w, const std::vector<uint8_t>& is_fixed);
// Device arrays (respects the dry-run memory estimate).
bool bones_alloc(emu_handle* h);
int bones_upload(emu_handle* h, const double* Q);
// Y = L^-1 J_f^T and S^-1 (needs the Laplacian on the device).
int joints_setup_device(emu_handle* h);
// Euclidean projection of an n x 16 device field onto the joint rows' null space.
int joints_project_basis(emu_handle* h, double* X);
// Columns 16 - 3 nfb .. 15 of X <- the free bones' constrained responses.
int bones_basis_responses(emu_handle* h, double* X);
// Gbar and the constant capacitance terms (after the mode gradients exist).
int bones_after_gamma(emu_handle* h);
// Translation responses and their quadratic form for the final solve.
int final_setup_device(emu_handle* h);

// ---- launches of the Newton loop (stream-ordered, graph-capturable) ----
void bones_after_grad(emu_handle* h);
void bones_gref(emu_handle* h, double* out);
const double* bones_cap_addend(const emu_handle* h);
void bones_before_dir(emu_handle* h);
int dir_partial_count(const emu_handle* h);
void joints_project(emu_handle* h, double* x64, float* x32);
// Bone states and the element arrays (R, s of the bones' tets):
// from_element_arrays takes each free bone's state from its first tet and
// copies it to every tet of the bone (pinned bones' tets to I);
// to_element_arrays writes the bone states into the bones' tets; from_rep
// takes the bone states from the first tets only; rest sets R = I, S = I.
void bones_state_from_element_arrays(emu_handle* h);
void bones_state_to_element_arrays(emu_handle* h);
void bones_state_from_rep(emu_handle* h);
int bones_state_rest(emu_handle* h);
// FP64 update of the bones' states on the mixed path (after the step).
void bones_update_mixed(emu_handle* h);
// Final coupling solve after a solve (blocking).
int bones_final_solve(emu_handle* h);

}  // namespace emu
