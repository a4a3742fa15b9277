// Cooperative conjugate-gradient solve of the scalar ACAP Laplacian.
#pragma once
#include <cuda_runtime.h>

#include "emu_cgpart.h"
#include "emu_internal.h"

namespace emu {

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

// Vectors are vertex-major with nrhs values per vertex (x[v * nrhs + j]).
// T is the arithmetic of the iteration (double, or float for the inner
// solves of the mixed path); reductions are always accumulated in FP64.
template <typename T> struct PcgArgsT {
  int64_t n;
  const int32_t* rowptr;
  const int32_t* col;
  const T* val;
  const T* dinv;
  const T* b;
  T* x;  // in: warm start, out: solution
  T* r;
  T* u;
  T* w;
  T* p;
  T* s;
  double* partials;  // grid * 4 * nrhs
  GridBarrier* bar;
  double tol;        // stop when ||r_j|| <= tol ||b_j|| for every column j
  int max_iter;
  int* iters_out;    // accumulated CG iterations (may be null)
  int* fail_out;     // set to 1 when max_iter is reached (may be null)
  int* timeout_out;  // set to 1 when a grid barrier gave up (may be null)
  int* last_iters;   // iterations of this solve (may be null)
  double* relres_out;  // final ||r_j|| / ||b_j|| per column (may be null)
  const T* phi;        // n x 16 coarse basis (null: Jacobi only; 3 columns only)
  const double* Einv;  // 16 x 16 (pseudo-)inverse of Phi^T L Phi
  unsigned long long wait_ns = kWaitLimitNs;  // limit of each grid-barrier wait
};

int pcg_max_grid(int nrhs, int64_t n);
template <typename T> cudaError_t launch_pcg(int nrhs, const PcgArgsT<T>& args, int grid, cudaStream_t st);

constexpr int kPcg32Threads = 256;  // threads per block of the FP32 CG kernels

// Work space of the register-resident FP32 CG.
struct Pcg32Work {
  float4* ug;      // 2 n exchange entries (x, then u, per vertex)
  float* part;     // 128 * grid block partial sums, value-major (two buffers
                   // of 64 * grid; the plain kernel uses the first)
  unsigned* sync;  // 96 words of barrier state, zero before the first launch
                   // (each launch leaves them zero)
  const float* aphi = nullptr;  // n x 16 rows of A Phi (pipelined kernel only)
  // the system in the row partition of emu_cgpart.h (required by the
  // pipelined kernel, optional for the plain one): args.rowptr/col/val/dinv/
  // phi and aphi permuted; b and x in vertex order
  const int32_t* perm = nullptr;  // partition row -> vertex (n)
  const int32_t* off = nullptr;   // grid + 1 row offsets of the blocks' parts
  const uint32_t* loc = nullptr;  // local table: (grid x rpt x lw x 256) words
  int lw = 0;                     // local entries per row slot
  int degree = 1;                 // degree of the local polynomial (1: Jacobi)
  float c0 = 1.f;                 // Chebyshev coefficients (emu_cgpart.h)
  float c1[kChebMax] = {0}, c2[kChebMax] = {0};
};

// Register-resident FP32 CG (3 columns): shape for n rows on ``sms`` SMs
// (false when n needs more than 8 rows per thread), and its launch (at most
// 256 blocks). args.bar, args.r .. args.s and args.partials are unused. With
// work.off set (rpt <= 4) it runs on the partitioned system of emu_cgpart.h
// with the block-local polynomial in its preconditioner, like the pipelined
// kernel; otherwise thread t of block b owns the rows (b + k grid) 256 + t.
bool pcg32_shape(int64_t n, int sms, int* grid, int* rpt);
cudaError_t launch_pcg32(const PcgArgsT<float>& args, const Pcg32Work& work, int grid, int rpt, cudaStream_t st);
// Per-device kernel attributes of the FP32 CG (before its first launch).
cudaError_t prepare_pcg32();
// Pipelined form of the same iteration with one grid barrier per iteration
// instead of two, on the partitioned system with the block-local polynomial
// preconditioner. It needs the coarse space (args.phi, args.Einv),
// work.aphi, work.perm and work.off, and supports rpt <= 4;
// launch_pcg32_pipe returns cudaErrorInvalidValue otherwise. Its
// recurrences drift from the true residual near FP32 precision, so it serves
// the loose inner solves.
bool pcg32_pipe_ok(int rpt);
cudaError_t launch_pcg32_pipe(const PcgArgsT<float>& args, const Pcg32Work& work, int grid, int rpt, cudaStream_t st);
// dst[r][:] = src[perm[r]][:] for n rows of 16 floats (the coarse rows in
// the partition order).
cudaError_t launch_gather_rows16(int64_t n, const int32_t* perm, const float* src, float* dst, cudaStream_t st);
// aphi = A phi for the n x 16 row-major coarse basis (FP32 CSR matrix).
cudaError_t launch_aphi32(int64_t n, const int32_t* rowptr, const int32_t* col, const float* val, const float* phi,
                          float* aphi, cudaStream_t st);

// FP64 residual r = b - K x (3 columns), written as float (r32) and/or double
// (r64) when those are non-null; out6 receives sum |r_j|^2 (j < 3) and
// sum |b_j|^2 (3 + j), over the rows v with skip[v] == 0 (all rows when skip
// is null).
cudaError_t launch_residual64(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* b,
                              const double* x, float* r32, double* r64, double* partials, int grid, double* out6,
                              cudaStream_t st, const uint8_t* skip = nullptr);
// x += e (float correction into the FP64 iterate), 3n values.
cudaError_t launch_axpy_f2d(int64_t n3, const float* e, double* x, cudaStream_t st);
// x += e, 3n values (FP64).
cudaError_t launch_axpy_d2d(int64_t n3, const double* e, double* x, cudaStream_t st);

// Self-check of the bounded grid-barrier wait: a cooperative launch of two
// blocks in which block 1 leaves without arriving, so block 0's wait must run
// out after wait_ns and report it. *timed_out (device int) receives 1 when
// the wait gave up as designed.
cudaError_t launch_wait_check(GridBarrier* bar, unsigned long long wait_ns, int* timed_out, cudaStream_t st);

}  // namespace emu
