// Row partition and block-local preconditioner of the pipelined FP32 CG.
//
// The rows (vertices) of the scalar ACAP Laplacian of Eq. 4 are split into
// one spatially compact part per CUDA block by recursive coordinate
// bisection of the rest positions; the CG runs on the permuted system, so a
// block's rows are contiguous. Each block then applies, without any
// grid-wide exchange, a fixed polynomial in its own diagonal block of the
// Jacobi-scaled matrix (Chebyshev, degree k): with the additive coarse space
// on the low-rank basis this is a two-level additive Schwarz preconditioner,
// symmetric positive definite by construction (the polynomial is positive
// on [0, lmax] and lmax bounds the block's spectrum by Gershgorin).
#pragma once
#include <stdint.h>

#include <vector>

namespace emu {

constexpr int kChebMax = 8;  // largest polynomial degree of the local part

struct CgPartHost {
  int G = 0, rpt = 0, nt = 0;
  int lw = 0;                      // local off-diagonal entries per row slot
  int degree = 1;                  // polynomial degree (1: Jacobi only)
  std::vector<int32_t> perm;       // partition row -> vertex
  std::vector<int32_t> off;        // G + 1 row offsets of the parts
  std::vector<int32_t> rowptr, col;  // the permuted Laplacian
  std::vector<float> val, dinv;
  // entry (part b, slot k, entry e, thread t) at ((b rpt + k) lw + e) nt + t:
  // local column (the row's offset in its part) in the low 16 bits, the
  // entry of D^-1/2 A D^-1/2 as bfloat16 in the high 16 bits
  std::vector<uint32_t> loc;
  double lmax = 0.0;               // Gershgorin bound of the local blocks
  float c0 = 1.f;                  // 1 / theta
  float c1[kChebMax] = {0}, c2[kChebMax] = {0};  // step i: d = c1 d + c2 res
};

// Largest number of local entries per row slot the pipelined kernel holds in
// shared memory for ``rpt`` rows per thread.
int cg_local_width_max(int rpt);

// Builds the partition of n rows (rest positions Q, 3 n) into G parts of at
// most rpt * nt rows, the permuted Laplacian (rowptr/col/val, FP64 on input)
// and the local table for a polynomial of ``degree`` (1: no local table).
// Rows with more local entries than cg_local_width_max(rpt) keep their
// largest ones, symmetrically. Returns false if the sizes do not fit.
// Coefficients of the local Chebyshev polynomial of ``degree`` (>= 2) on
// [lmax / kChebRatio, lmax] (c0 and the steps c1[i], c2[i] for i < degree).
void cg_cheb_coeffs(double lmax, int degree, float* c0, float* c1, float* c2);

bool build_cg_partition(int64_t n, const double* Q, const std::vector<int32_t>& rowptr,
                        const std::vector<int32_t>& col, const std::vector<double>& val, int G, int rpt, int nt,
                        int degree, CgPartHost* out);

}  // namespace emu
