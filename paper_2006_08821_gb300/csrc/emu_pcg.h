// Cooperative conjugate-gradient solve of the scalar ACAP Laplacian.
#pragma once
#include <cuda_runtime.h>

#include "emu_internal.h"

namespace emu {

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

// Vectors are vertex-major with nrhs values per vertex (x[v * nrhs + j]).
struct PcgArgs {
  Laplacian L;
  const double* b;
  double* x;  // in: warm start, out: solution
  double* r;
  double* u;
  double* w;
  double* p;
  double* s;
  double* partials;  // grid * 4 * nrhs
  GridBarrier* bar;
  double tol;        // stop when ||r_j|| <= tol ||b_j|| for every column j
  int max_iter;
  int* iters_out;    // accumulated CG iterations (may be null)
  int* fail_out;     // set to 1 when max_iter is reached (may be null)
  int* timeout_out;  // set to 1 when a grid barrier gave up (may be null)
  int* last_iters;   // iterations of this solve (may be null)
};

int pcg_max_grid(int nrhs, int64_t n);
cudaError_t launch_pcg(int nrhs, const PcgArgs& args, int grid, cudaStream_t st);

}  // namespace emu
