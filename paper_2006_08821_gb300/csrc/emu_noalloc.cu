// emu_acap_solve_noalloc: the coupling solve q = q*(F) without any device
// allocation, for callers that cannot allocate device memory (see emu.h).
//
// Its scratch memory is one file-scope device array of kNoAllocScratchBytes.
// Every GPU that loads this library reserves that array for the lifetime of
// the process. Host code must not use the array's name as a device address:
// on the host the symbol is only a stand-in. The device address comes from
// cudaGetSymbolAddress with the handle's device current (set up by the first
// call on a device, refreshed by every call outside stream capture) and is
// passed to the kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "emu_internal.h"
#include "emu_kernels.cuh"
#include "emu_pcg.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device. Outside stream
// capture it is looked up again on every call (a host-side query, no device
// work), so a primary context torn down and re-created since the last call
// (cudaDeviceReset) cannot leave a stale address behind. During capture the
// address recorded by the last call outside capture is used, so the first
// call on a device must come before any capture.
cudaError_t scratch_address(cudaStream_t st, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  } else if (!g_scratch_ptr[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Records the failing step and returns ``code``.
int noalloc_fail(int code, const char* step, cudaError_t e = cudaSuccess) {
  std::string msg = std::string("emu_acap_solve_noalloc: ") + step;
  if (e != cudaSuccess) msg += std::string(": ") + cudaGetErrorString(e);
  emu::set_last_error(msg.c_str());
  return code;
}

// Corner terms of w_i G_i^T F_i for a caller-given F (n_tets x 9, row-major
// per tet): the right-hand side of Eq. 4 per tet corner, as the solver's own
// right-hand-side kernel forms them from R S.
__global__ void __launch_bounds__(256) k_rhs_from_F(int64_t m, const double* __restrict__ F,
                                                    const double* __restrict__ Dinv, const double* __restrict__ w,
                                                    double* __restrict__ contrib) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double D[9], X[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      D[k] = Dinv[k * m + i];
      X[k] = F[9 * i + k];
    }
    const double wi = w[i];
    double s0 = 0, s1 = 0, s2 = 0;
    double* out = contrib + 12 * i;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double v[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) v[r] = wi * (X[3 * r] * D[3 * k] + X[3 * r + 1] * D[3 * k + 1] + X[3 * r + 2] * D[3 * k + 2]);
      out[3 * k] = v[0];
      out[3 * k + 1] = v[1];
      out[3 * k + 2] = v[2];
      s0 += v[0];
      s1 += v[1];
      s2 += v[2];
    }
    out[9] = -s0;
    out[10] = -s1;
    out[11] = -s2;
  }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" int emu_acap_solve_noalloc(emu_handle* h, const double* F_device, double* q_device, void* stream) {
  using namespace emu;
  AcapView v;
  if (!h || !F_device || !q_device || !acap_view(h, &v))
    return noalloc_fail(EMU_ERR_INVALID_ARG, "NULL handle or pointer");
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return noalloc_fail(EMU_ERR_CUDA, "cudaGetDevice", e);
  if (cur != v.device)
    return noalloc_fail(EMU_ERR_INVALID_ARG, "the current device is not the one the handle was created on");
  if (v.npts > 0)
    return noalloc_fail(EMU_ERR_NOT_IMPLEMENTED, "a handle with joints (their rows need the solver's own buffers)");
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = v.grid_pcg;
  // scratch layout: corner terms, right-hand side, five CG vectors, partial
  // sums, barrier and counters
  const size_t b_contrib = align256(96 * (size_t)v.m);
  const size_t b_vec = align256(24 * (size_t)v.n);
  const size_t b_part = align256(8 * (size_t)grid * (4 * 3 + 3 * kModes));
  const size_t b_bar = align256(sizeof(GridBarrier));
  const size_t b_cnt = align256(4 * sizeof(int));
  const size_t need = b_contrib + 6 * b_vec + b_part + b_bar + b_cnt;
  if (need > kNoAllocScratchBytes)
    return noalloc_fail(EMU_ERR_INVALID_ARG,
                        "the mesh needs more scratch than the fixed 32 MiB array (96 bytes per tet + 144 per vertex)");
  void* base = nullptr;
  e = scratch_address(st, &base);
  if (e != cudaSuccess) return noalloc_fail(EMU_ERR_CUDA, "looking up the scratch array's device address", e);
  unsigned char* p = static_cast<unsigned char*>(base);
  double* contrib = reinterpret_cast<double*>(p);
  p += b_contrib;
  double* b = reinterpret_cast<double*>(p);
  p += b_vec;
  double* vr = reinterpret_cast<double*>(p);
  p += b_vec;
  double* vu = reinterpret_cast<double*>(p);
  p += b_vec;
  double* vw = reinterpret_cast<double*>(p);
  p += b_vec;
  double* vp = reinterpret_cast<double*>(p);
  p += b_vec;
  double* vs = reinterpret_cast<double*>(p);
  p += b_vec;
  double* part = reinterpret_cast<double*>(p);
  p += b_part;
  GridBarrier* bar = reinterpret_cast<GridBarrier*>(p);
  p += b_bar;
  int* cnt = reinterpret_cast<int*>(p);

  // counters start at zero on every call (the array keeps the last call's)
  e = cudaMemsetAsync(cnt, 0, 4 * sizeof(int), st);
  if (e != cudaSuccess) return noalloc_fail(EMU_ERR_CUDA, "clearing the counters", e);
  // start from the rest-state solution, then Eq. 4 for the given F
  e = cudaMemcpyAsync(q_device, v.q0, 24 * (size_t)v.n, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return noalloc_fail(EMU_ERR_CUDA, "copying the start vector", e);
  int tgrid = (int)((v.m + 255) / 256);
  if (tgrid > 8 * v.sms) tgrid = 8 * v.sms;
  if (tgrid < 1) tgrid = 1;
  k_rhs_from_F<<<tgrid, 256, 0, st>>>(v.m, F_device, v.Dinv, v.w, contrib);
  launch_assemble(v.n, v.slot_ptr, v.slot_idx, contrib, v.bfix, v.is_fixed, v.qfix, 0, b, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(EMU_ERR_CUDA, "launching the right-hand-side kernels", e);
  PcgArgsT<double> a;
  a.n = v.n;
  a.rowptr = v.rowptr;
  a.col = v.col;
  a.val = v.val;
  a.dinv = v.ldinv;
  a.b = b;
  a.x = q_device;
  a.r = vr;
  a.u = vu;
  a.w = vw;
  a.p = vp;
  a.s = vs;
  a.partials = part;
  a.bar = bar;  // launch_pcg clears it before the launch
  a.tol = v.pcg_tol;
  a.max_iter = v.pcg_max;
  a.iters_out = cnt;
  a.fail_out = cnt + 1;
  a.timeout_out = cnt + 2;
  a.last_iters = cnt + 3;
  a.relres_out = nullptr;
  a.phi = v.phi;
  a.Einv = v.Einv;
  e = launch_pcg<double>(3, a, grid, st);
  if (e != cudaSuccess) return noalloc_fail(EMU_ERR_CUDA, "launching the CG kernel", e);
  int hc[4] = {0, 0, 0, 0};
  e = cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return noalloc_fail(EMU_ERR_CUDA, "reading the counters", e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return noalloc_fail(EMU_ERR_CUDA, "cudaStreamSynchronize", e);
  if (hc[2]) return noalloc_fail(EMU_ERR_TIMEOUT, "a grid barrier of the CG kernel ran out of its wait limit");
  if (hc[1]) return noalloc_fail(EMU_ERR_PCG, "the CG iteration cap was reached before the tolerance");
  return EMU_OK;
}
