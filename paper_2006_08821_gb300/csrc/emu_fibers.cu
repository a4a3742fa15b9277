// Fiber directions from the heat equation (Sec. 3.6, "Modeling"): the P1
// harmonic field with Dirichlet values -1 on the origin vertices and +1 on
// the insertion vertices, solved on the device with the FP64 CG, and per tet
// the normalised gradient of that field.
//
// The discrete Laplacian is L_ab = sum_i V_i gradN_a . gradN_b over the tets
// (the scalar ACAP Laplacian of Eq. 4 with w = V). Dirichlet rows become
// identity rows and their known values move to the right-hand side of the
// free rows, which keeps the system symmetric positive definite; vertices in
// no tet get identity rows with 0.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "emu.h"
#include "emu_internal.h"
#include "emu_pcg.h"

namespace emu {
namespace {

int fiber_fail(int code, const std::string& msg) {
  set_last_error(msg.c_str());
  return code;
}

// u_i = grad f_i / |grad f_i| (0 where the gradient vanishes); f is column 0
// of the vertex-major 3-column solution x
__global__ void __launch_bounds__(256) k_fiber_grad(int64_t m, const int4* __restrict__ tet,
                                                    const double* __restrict__ Dinv, const double* __restrict__ x,
                                                    double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int4 t = tet[i];
    const double f3 = x[3 * (int64_t)t.w];
    const double e0 = x[3 * (int64_t)t.x] - f3, e1 = x[3 * (int64_t)t.y] - f3, e2 = x[3 * (int64_t)t.z] - f3;
    double g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c] = e0 * Dinv[(0 + c) * m + i] + e1 * Dinv[(3 + c) * m + i] + e2 * Dinv[(6 + c) * m + i];
    const double nn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    const double s = nn > 0.0 ? 1.0 / nn : 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3 * i + c] = g[c] * s;
  }
}

struct DevMem {
  std::vector<void*> ptrs;
  template <typename T> T* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 256)) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~DevMem() {
    for (void* p : ptrs) cudaFree(p);
  }
};

}  // namespace
}  // namespace emu

using namespace emu;

extern "C" int emu_fiber_field(int64_t n_verts, const double* rest_pos, int64_t n_tets, const int32_t* tets,
                               const int32_t* origin, int64_t n_origin, const int32_t* insertion,
                               int64_t n_insertion, double* fibers, void* stream) {
  if (n_verts < 4 || n_tets < 1 || !rest_pos || !tets || !origin || !insertion || !fibers || n_origin < 1 ||
      n_insertion < 1 || n_verts > ((int64_t)1 << 30) || n_tets > ((int64_t)1 << 30))
    return fiber_fail(EMU_ERR_INVALID_ARG, "bad arguments");
  const int64_t n = n_verts, m = n_tets;
  // Dirichlet values: -1 origin, +1 insertion (0: free)
  std::vector<int8_t> dir(n, 0);
  for (int64_t k = 0; k < n_origin; ++k) {
    if (origin[k] < 0 || origin[k] >= n) return fiber_fail(EMU_ERR_INVALID_ARG, "origin vertex out of range");
    dir[origin[k]] = -1;
  }
  for (int64_t k = 0; k < n_insertion; ++k) {
    if (insertion[k] < 0 || insertion[k] >= n) return fiber_fail(EMU_ERR_INVALID_ARG, "insertion vertex out of range");
    if (dir[insertion[k]] == -1) return fiber_fail(EMU_ERR_INVALID_ARG, "a vertex is both origin and insertion");
    dir[insertion[k]] = 1;
  }
  // rest geometry (D_m^-1 component-major, V) and the Laplacian's triplets
  std::vector<double> Dinv(9 * m), V(m);
  std::vector<uint8_t> in_tet(n, 0);
  for (int64_t i = 0; i < m; ++i) {
    const int32_t* t = tets + 4 * i;
    for (int k = 0; k < 4; ++k)
      if (t[k] < 0 || t[k] >= n) return fiber_fail(EMU_ERR_INVALID_ARG, "tet vertex out of range");
    double D[9];  // columns Q_j - Q_3
    for (int r = 0; r < 3; ++r)
      for (int j = 0; j < 3; ++j) D[3 * r + j] = rest_pos[3 * t[j] + r] - rest_pos[3 * t[3] + r];
    const double det = D[0] * (D[4] * D[8] - D[5] * D[7]) - D[1] * (D[3] * D[8] - D[5] * D[6]) +
                       D[2] * (D[3] * D[7] - D[4] * D[6]);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det))
      return fiber_fail(EMU_ERR_INVALID_ARG, "degenerate tet " + std::to_string(i));
    const double id = 1.0 / det;
    const double inv[9] = {(D[4] * D[8] - D[5] * D[7]) * id, (D[2] * D[7] - D[1] * D[8]) * id,
                           (D[1] * D[5] - D[2] * D[4]) * id, (D[5] * D[6] - D[3] * D[8]) * id,
                           (D[0] * D[8] - D[2] * D[6]) * id, (D[2] * D[3] - D[0] * D[5]) * id,
                           (D[3] * D[7] - D[4] * D[6]) * id, (D[1] * D[6] - D[0] * D[7]) * id,
                           (D[0] * D[4] - D[1] * D[3]) * id};
    for (int k = 0; k < 9; ++k) Dinv[k * m + i] = inv[k];
    V[i] = std::fabs(det) / 6.0;
    for (int k = 0; k < 4; ++k) in_tet[t[k]] = 1;
  }
  std::vector<std::pair<int64_t, double>> trip;
  trip.reserve(16 * m + n);
  std::vector<double> rhs(3 * n, 0.0);
  for (int64_t i = 0; i < m; ++i) {
    const int32_t* t = tets + 4 * i;
    double gN[4][3];
    for (int k = 0; k < 3; ++k)
      for (int c = 0; c < 3; ++c) gN[k][c] = Dinv[(3 * k + c) * m + i];
    for (int c = 0; c < 3; ++c) gN[3][c] = -(gN[0][c] + gN[1][c] + gN[2][c]);
    for (int a = 0; a < 4; ++a) {
      if (dir[t[a]] != 0) continue;
      for (int b = 0; b < 4; ++b) {
        const double lv = V[i] * (gN[a][0] * gN[b][0] + gN[a][1] * gN[b][1] + gN[a][2] * gN[b][2]);
        if (dir[t[b]] != 0)
          rhs[3 * t[a]] -= lv * (double)dir[t[b]];
        else
          trip.push_back({(int64_t)t[a] * n + t[b], lv});
      }
    }
  }
  for (int64_t v = 0; v < n; ++v)
    if (dir[v] != 0 || !in_tet[v]) {
      trip.push_back({v * n + v, 1.0});
      rhs[3 * v] = (double)dir[v];
    }
  std::sort(trip.begin(), trip.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  std::vector<int32_t> rowptr(n + 1, 0), col;
  std::vector<double> val, dinv(n, 1.0);
  col.reserve(trip.size());
  val.reserve(trip.size());
  for (size_t k = 0; k < trip.size();) {
    const int64_t key = trip[k].first;
    double s = 0.0;
    while (k < trip.size() && trip[k].first == key) s += trip[k++].second;
    const int64_t r = key / n, c = key % n;
    col.push_back((int32_t)c);
    val.push_back(s);
    rowptr[r + 1]++;
    if (r == c) dinv[r] = s > 0.0 ? 1.0 / s : 1.0;
  }
  for (int64_t v = 0; v < n; ++v) rowptr[v + 1] += rowptr[v];
  const int64_t nnz = (int64_t)col.size();

  // device solve (3 columns of the CG kernel; columns 1 and 2 are zero)
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = pcg_max_grid(3, n);
  DevMem dm;
  int32_t *d_rowptr = dm.get<int32_t>(n + 1), *d_col = dm.get<int32_t>(nnz);
  double *d_val = dm.get<double>(nnz), *d_dinv = dm.get<double>(n), *d_b = dm.get<double>(3 * n),
         *d_x = dm.get<double>(3 * n), *d_r = dm.get<double>(3 * n), *d_u = dm.get<double>(3 * n),
         *d_w = dm.get<double>(3 * n), *d_p = dm.get<double>(3 * n), *d_s = dm.get<double>(3 * n),
         *d_part = dm.get<double>((size_t)grid * (4 * 3 + 3 * kModes)), *d_D = dm.get<double>(9 * m),
         *d_out = dm.get<double>(3 * m);
  int4* d_tet = dm.get<int4>(m);
  GridBarrier* d_bar = dm.get<GridBarrier>(1);
  int* d_cnt = dm.get<int>(4);
  if (!d_rowptr || !d_col || !d_val || !d_dinv || !d_b || !d_x || !d_r || !d_u || !d_w || !d_p || !d_s || !d_part ||
      !d_D || !d_out || !d_tet || !d_bar || !d_cnt)
    return fiber_fail(EMU_ERR_OOM, "device allocation failed");
  cudaError_t e = cudaSuccess;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  up(d_rowptr, rowptr.data(), 4 * (n + 1));
  up(d_col, col.data(), 4 * nnz);
  up(d_val, val.data(), 8 * nnz);
  up(d_dinv, dinv.data(), 8 * n);
  up(d_b, rhs.data(), 24 * n);
  up(d_D, Dinv.data(), 72 * m);
  up(d_tet, tets, 16 * m);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_x, 0, 24 * n, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, 4 * sizeof(int), st);
  PcgArgsT<double> a;
  a.n = n;
  a.rowptr = d_rowptr;
  a.col = d_col;
  a.val = d_val;
  a.dinv = d_dinv;
  a.b = d_b;
  a.x = d_x;
  a.r = d_r;
  a.u = d_u;
  a.w = d_w;
  a.p = d_p;
  a.s = d_s;
  a.partials = d_part;
  a.bar = d_bar;
  a.tol = 1e-13;
  a.max_iter = (int)std::min<int64_t>(std::max<int64_t>(20000, 4 * n), 1 << 30);
  a.iters_out = d_cnt;
  a.fail_out = d_cnt + 1;
  a.timeout_out = d_cnt + 2;
  a.last_iters = d_cnt + 3;
  a.relres_out = nullptr;
  a.phi = nullptr;
  a.Einv = nullptr;
  if (e == cudaSuccess) e = launch_pcg<double>(3, a, grid, st);
  if (e == cudaSuccess) {
    const int tgrid = (int)std::min<int64_t>(std::max<int64_t>(1, (m + 255) / 256), 4096);
    k_fiber_grad<<<tgrid, 256, 0, st>>>(m, d_tet, d_D, d_x, d_out);
    e = cudaGetLastError();
  }
  int hc[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hc, d_cnt, sizeof(hc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(fibers, d_out, 24 * m, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fiber_fail(EMU_ERR_CUDA, std::string("emu_fiber_field: ") + cudaGetErrorString(e));
  if (hc[2]) return fiber_fail(EMU_ERR_TIMEOUT, "a grid barrier of the CG kernel ran out of its wait limit");
  if (hc[1]) return fiber_fail(EMU_ERR_PCG, "the heat-equation solve did not converge");
  return EMU_OK;
}
