// Host side of affine bones and joints (Sec. 3.3 of arXiv 2006.08821):
// classification of the bone tets, the joint rows, the final-solve operator,
// the device set-up (joint responses Y = L^-1 J_f^T, the bones' constant
// capacitance terms, the final solve's translation responses) and the
// per-iteration and final-solve launches. The reading of the section and
// the data layout are described in emu_bones.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <utility>
#include <vector>

#include "emu_bones_host.h"
#include "emu_handle.h"

namespace emu {

namespace {

int bfail(int code, const std::string& msg) {
  set_last_error(msg.c_str());
  return code;
}

#define BONE_CK(call)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return bfail(EMU_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// In-place inverse of a symmetric positive definite N x N matrix (row-major)
// by Gauss-Jordan elimination with partial pivoting. False if singular.
bool invert_small(std::vector<double>& A, int N) {
  std::vector<double> I(N * N, 0.0);
  for (int i = 0; i < N; ++i) I[N * i + i] = 1.0;
  double scale = 0.0;
  for (int i = 0; i < N; ++i) scale = std::max(scale, std::fabs(A[N * i + i]));
  for (int c = 0; c < N; ++c) {
    int p = c;
    for (int r = c + 1; r < N; ++r)
      if (std::fabs(A[N * r + c]) > std::fabs(A[N * p + c])) p = r;
    if (!(std::fabs(A[N * p + c]) > 1e-14 * scale)) return false;
    if (p != c)
      for (int k = 0; k < N; ++k) {
        std::swap(A[N * p + k], A[N * c + k]);
        std::swap(I[N * p + k], I[N * c + k]);
      }
    const double d = 1.0 / A[N * c + c];
    for (int k = 0; k < N; ++k) {
      A[N * c + k] *= d;
      I[N * c + k] *= d;
    }
    for (int r = 0; r < N; ++r) {
      if (r == c) continue;
      const double f = A[N * r + c];
      if (f == 0.0) continue;
      for (int k = 0; k < N; ++k) {
        A[N * r + k] -= f * A[N * c + k];
        I[N * r + k] -= f * I[N * c + k];
      }
    }
  }
  A.swap(I);
  return true;
}

// Least-squares affine fit weights: c_v with sum_v c_v x_v = A p + t for the
// fit x_v ~ A Q_v + t over the vertices vs (exact for affine x). Computed in
// coordinates centred on the vertices' mean for conditioning.
bool affine_fit(const double* Q, const std::vector<int32_t>& vs, const double* p, std::vector<double>& c) {
  const size_t k = vs.size();
  double mean[3] = {0, 0, 0};
  for (int32_t v : vs)
    for (int r = 0; r < 3; ++r) mean[r] += Q[3 * (int64_t)v + r];
  for (int r = 0; r < 3; ++r) mean[r] /= (double)k;
  std::vector<double> M(16, 0.0);  // A^T A with rows [Q_v - mean, 1]
  for (int32_t v : vs) {
    const double a[4] = {Q[3 * (int64_t)v] - mean[0], Q[3 * (int64_t)v + 1] - mean[1], Q[3 * (int64_t)v + 2] - mean[2],
                         1.0};
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) M[4 * i + j] += a[i] * a[j];
  }
  if (!invert_small(M, 4)) return false;
  const double pp[4] = {p[0] - mean[0], p[1] - mean[1], p[2] - mean[2], 1.0};
  double y[4];
  for (int i = 0; i < 4; ++i) y[i] = M[4 * i] * pp[0] + M[4 * i + 1] * pp[1] + M[4 * i + 2] * pp[2] + M[4 * i + 3] * pp[3];
  c.resize(k);
  for (size_t t = 0; t < k; ++t) {
    const int64_t v = vs[t];
    c[t] = (Q[3 * v] - mean[0]) * y[0] + (Q[3 * v + 1] - mean[1]) * y[1] + (Q[3 * v + 2] - mean[2]) * y[2] + y[3];
  }
  return true;
}

}  // namespace

// ------------------------------------------------------------ set-up ------
int bones_prepare(emu_handle* h, const emu_mesh_desc* d, const std::vector<int32_t>& tet,
                  const std::vector<double>& V, const std::vector<uint8_t>& is_fixed) {
  const int64_t m = d->n_tets, n = d->n_verts;
  h->eps_bone = h->prm.eps_bone;
  h->eps_joint = h->prm.eps_joint;
  int nb = 0;
  if (d->bone_id)
    for (int64_t i = 0; i < m; ++i) nb = std::max(nb, d->bone_id[i] + 1);
  if (nb == 0) {
    if (d->n_joints > 0) return bfail(EMU_ERR_INVALID_ARG, "joints need bones (bone_id)");
    return EMU_OK;
  }
  if (h->kmodes != 16) return bfail(EMU_ERR_INVALID_ARG, "a mesh with bones needs k_modes = 48");
  h->has_bones = true;
  h->nb = nb;
  double vsum = 0.0;
  for (int64_t i = 0; i < m; ++i) vsum += V[i];
  h->Vbar = vsum / (double)m;
  // vertices and material of every bone
  h->bverts_h.assign(nb, {});
  std::vector<int> bmat(nb, -1);
  for (int64_t i = 0; i < m; ++i) {
    const int b = d->bone_id[i];
    if (b < 0) continue;
    if (bmat[b] < 0) bmat[b] = d->material_id[i];
    if (bmat[b] != d->material_id[i]) return bfail(EMU_ERR_INVALID_ARG, "every tet of a bone must have the bone's material");
    for (int k = 0; k < 4; ++k) h->bverts_h[b].push_back(tet[4 * i + k]);
  }
  std::vector<int> owner(n, -1);
  h->free_index_h.assign(nb, -1);
  h->nfb = 0;
  for (int b = 0; b < nb; ++b) {
    auto& vs = h->bverts_h[b];
    if (vs.empty()) return bfail(EMU_ERR_INVALID_ARG, "bone ids must be contiguous from 0 (bone " + std::to_string(b) + " has no tet)");
    std::sort(vs.begin(), vs.end());
    vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
    int64_t pinned = 0;
    for (int32_t v : vs) {
      if (owner[v] >= 0) return bfail(EMU_ERR_INVALID_ARG, "two bones share a vertex");
      owner[v] = b;
      pinned += is_fixed[v] ? 1 : 0;
    }
    if (pinned > 0 && pinned < (int64_t)vs.size())
      return bfail(EMU_ERR_INVALID_ARG, "bone " + std::to_string(b) + " is partly pinned (pin all of its vertices or none)");
    if (pinned == 0) {
      if (h->nfb >= kMaxFreeBones) return bfail(EMU_ERR_INVALID_ARG, "at most 4 free (unpinned) bones are supported");
      h->free_index_h[b] = h->nfb++;
    }
  }
  const int nfb = h->nfb;
  h->tkind_h.assign(m, kTetDeformable);
  for (int64_t i = 0; i < m; ++i) {
    const int b = d->bone_id[i];
    if (b >= 0) h->tkind_h[i] = h->free_index_h[b] >= 0 ? h->free_index_h[b] : kTetPinnedBone;
  }
  h->btets_h.clear();
  h->bptr_h.assign(nfb + 1, 0);
  h->rep_h.assign(nfb, 0);
  h->Vb_h.assign(nfb, 0.0);
  h->wb_h.assign(nfb, 0.0);
  h->mub_h.assign(nfb, 0.0);
  h->lamb_h.assign(nfb, 0.0);
  h->bvert_h.clear();
  h->bvptr_h.assign(nfb + 1, 0);
  for (int b = 0; b < nb; ++b) {
    const int fi = h->free_index_h[b];
    if (fi < 0) continue;
    h->bptr_h[fi] = (int32_t)h->btets_h.size();
    for (int64_t i = 0; i < m; ++i)
      if (h->tkind_h[i] == fi) {
        h->btets_h.push_back((int32_t)i);
        h->Vb_h[fi] += V[i];
      }
    h->rep_h[fi] = h->btets_h[h->bptr_h[fi]];
    const double E = d->youngs[bmat[b]], nu = d->poisson[bmat[b]];
    h->mub_h[fi] = E / (2.0 * (1.0 + nu));
    h->lamb_h[fi] = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    h->bvptr_h[fi] = (int32_t)h->bvert_h.size();
    h->bvert_h.insert(h->bvert_h.end(), h->bverts_h[b].begin(), h->bverts_h[b].end());
  }
  h->bptr_h[nfb] = (int32_t)h->btets_h.size();
  h->bvptr_h[nfb] = (int32_t)h->bvert_h.size();

  // ---- joint rows: per point, fit of bone 1 minus fit of bone 2 ----
  struct Pt {
    int b1, b2;
    double p[3];
  };
  std::vector<Pt> pts;
  for (int32_t jn = 0; jn < d->n_joints; ++jn) {
    const int type = d->joint_type[jn];
    const int b1 = d->joint_bones[2 * jn], b2 = d->joint_bones[2 * jn + 1];
    if (b1 < 0 || b1 >= nb || b2 < 0 || b2 >= nb || b1 == b2)
      return bfail(EMU_ERR_INVALID_ARG, "a joint must name two distinct bones");
    if (h->free_index_h[b1] < 0 && h->free_index_h[b2] < 0)
      return bfail(EMU_ERR_INVALID_ARG, "a joint between two pinned bones has nothing to constrain");
    const double* p0 = d->joint_point + 3 * jn;
    for (int r = 0; r < 3; ++r)
      if (!std::isfinite(p0[r])) return bfail(EMU_ERR_INVALID_ARG, "non-finite joint point");
    if (type == 1) {
      const double* ax = d->joint_axis + 3 * jn;
      const double hl = d->joint_half_length[jn];
      const double nrm = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
      if (!(nrm > 0.0) || !std::isfinite(nrm) || !(hl > 0.0) || !std::isfinite(hl))
        return bfail(EMU_ERR_INVALID_ARG, "a hinge needs a non-zero axis and a positive half-length");
      for (int sgn = 1; sgn >= -1; sgn -= 2) {
        Pt q;
        q.b1 = b1;
        q.b2 = b2;
        for (int r = 0; r < 3; ++r) q.p[r] = p0[r] + sgn * hl * ax[r] / nrm;
        pts.push_back(q);
      }
    } else if (type == 0) {
      Pt q;
      q.b1 = b1;
      q.b2 = b2;
      for (int r = 0; r < 3; ++r) q.p[r] = p0[r];
      pts.push_back(q);
    } else {
      return bfail(EMU_ERR_INVALID_ARG, "joint type must be 0 (ball) or 1 (hinge)");
    }
  }
  const int np = (int)pts.size();
  if (np > kMaxJointPts) return bfail(EMU_ERR_INVALID_ARG, "at most 16 joint points (8 hinges) are supported");
  h->npts = np;
  h->kj = std::cbrt(h->Vbar) / std::fabs(h->eps_joint);
  h->jv_h.clear();
  h->jw_h.clear();
  h->jfree_h.clear();
  h->sgn_h.assign(kMaxJointPts * kMaxFreeBones, 0.0);
  if (np > 0) {
    std::vector<int> slot(n, -1);
    std::vector<double> wrow;  // njv x np, grown as vertices appear
    for (int r = 0; r < np; ++r) {
      for (int side = 0; side < 2; ++side) {
        const int b = side == 0 ? pts[r].b1 : pts[r].b2;
        const double sg = side == 0 ? 1.0 : -1.0;
        std::vector<double> c;
        if (!affine_fit(d->rest_pos, h->bverts_h[b], pts[r].p, c))
          return bfail(EMU_ERR_INVALID_ARG, "a bone's vertices do not span 3-D space (affine fit)");
        const int fi = h->free_index_h[b];
        for (size_t t = 0; t < c.size(); ++t) {
          const int32_t v = h->bverts_h[b][t];
          if (slot[v] < 0) {
            slot[v] = (int)h->jv_h.size();
            h->jv_h.push_back(v);
            h->jfree_h.push_back(is_fixed[v] ? 0 : 1);
            wrow.resize(wrow.size() + np, 0.0);
          }
          wrow[(size_t)slot[v] * np + r] += sg * c[t];
          if (fi >= 0) h->sgn_h[r * kMaxFreeBones + fi] += sg * c[t];
        }
      }
    }
    h->jw_h = wrow;
    h->njv = (int)h->jv_h.size();
    std::vector<double> JJ(np * np, 0.0);
    for (int vi = 0; vi < h->njv; ++vi) {
      if (!h->jfree_h[vi]) continue;
      for (int r = 0; r < np; ++r)
        for (int r2 = 0; r2 < np; ++r2) JJ[r * np + r2] += h->jw_h[(size_t)vi * np + r] * h->jw_h[(size_t)vi * np + r2];
    }
    if (!invert_small(JJ, np)) return bfail(EMU_ERR_INVALID_ARG, "the joint rows are linearly dependent");
    h->JJinv_h = JJ;
  }
  return EMU_OK;
}

void bones_weights(emu_handle* h, const std::vector<double>& V, std::vector<double>& w) {
  if (!h->has_bones) return;
  const double add = h->Vbar / std::fabs(h->eps_bone);
  for (size_t i = 0; i < w.size(); ++i)
    if (h->tkind_h[i] != kTetDeformable) w[i] = V[i] + add;
}

void bones_weight_sums(emu_handle* h, const std::vector<double>& w) {
  if (!h->has_bones) return;
  h->w_h = w;
  for (int fi = 0; fi < h->nfb; ++fi) {
    double s = 0.0;
    for (int32_t k = h->bptr_h[fi]; k < h->bptr_h[fi + 1]; ++k) s += w[h->btets_h[k]];
    h->wb_h[fi] = s;
  }
}

int bones_final_host(emu_handle* h, const std::vector<int32_t>& tet, const std::vector<double>& Dinv,
                     const std::vector<double>& w, const std::vector<uint8_t>& is_fixed) {
  if (!h->has_bones || h->nfb == 0) return EMU_OK;
  const int64_t n = h->n, m = h->m;
  h->fin_fixed_h.assign(is_fixed.begin(), is_fixed.end());
  std::vector<int> vfree_bone(n, -1);
  for (int b = 0; b < h->nb; ++b)
    for (int32_t v : h->bverts_h[b]) {
      h->fin_fixed_h[v] = 1;
      vfree_bone[v] = h->free_index_h[b];
    }
  h->zrhs_h.assign((size_t)n * 16, 0.0);
  std::vector<std::pair<int64_t, double>> trip;
  trip.reserve(16 * m);
  for (int64_t i = 0; i < m; ++i) {
    if (h->tkind_h[i] != kTetDeformable) continue;  // bone tets touch only bone vertices
    double gN[4][3];
    for (int k = 0; k < 3; ++k)
      for (int c = 0; c < 3; ++c) gN[k][c] = Dinv[(3 * k + c) * m + i];
    for (int c = 0; c < 3; ++c) gN[3][c] = -(gN[0][c] + gN[1][c] + gN[2][c]);
    for (int a = 0; a < 4; ++a) {
      const int32_t va = tet[4 * i + a];
      if (h->fin_fixed_h[va]) continue;
      for (int b = 0; b < 4; ++b) {
        const int32_t vb = tet[4 * i + b];
        const double lv = w[i] * (gN[a][0] * gN[b][0] + gN[a][1] * gN[b][1] + gN[a][2] * gN[b][2]);
        if (h->fin_fixed_h[vb]) {
          if (vfree_bone[vb] >= 0) h->zrhs_h[(size_t)va * 16 + vfree_bone[vb]] -= lv;
        } else {
          trip.push_back({(int64_t)va * n + vb, lv});
        }
      }
    }
  }
  for (int64_t v = 0; v < n; ++v)
    if (h->fin_fixed_h[v]) trip.push_back({v * n + v, 1.0});
  std::sort(trip.begin(), trip.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  h->frowptr_h.assign(n + 1, 0);
  h->fcol_h.clear();
  h->fval_h.clear();
  h->fldinv_h.assign(n, 1.0);
  for (size_t k = 0; k < trip.size();) {
    const int64_t key = trip[k].first;
    double s = 0.0;
    while (k < trip.size() && trip[k].first == key) s += trip[k++].second;
    const int64_t r = key / n, c = key % n;
    h->fcol_h.push_back((int32_t)c);
    h->fval_h.push_back(s);
    h->frowptr_h[r + 1]++;
    if (r == c) h->fldinv_h[r] = 1.0 / s;
  }
  for (int64_t v = 0; v < n; ++v) h->frowptr_h[v + 1] += h->frowptr_h[v];
  h->fnnz = (int64_t)h->fcol_h.size();
  return EMU_OK;
}

bool bones_alloc(emu_handle* h) {
  if (!h->has_bones) return true;
  const int64_t n = h->n, m = h->m;
  const bool dry = h->dry;
  // in a dry run (memory estimate) the host arrays are not built: bounds
  const int64_t nbt = dry ? m : (int64_t)std::max<size_t>(1, h->btets_h.size());
  const int64_t nbv = dry ? n : (int64_t)std::max<size_t>(1, h->bvert_h.size());
  const int64_t njv = dry ? n : std::max(1, h->njv);
  const int64_t fnnz = dry ? 16 * m + n : std::max<int64_t>(1, h->fnnz);
  const int np = dry ? kMaxJointPts : std::max(1, h->npts);
  bool ok = h->get(h->tkind, m) && h->get(h->btets, nbt) && h->get(h->bvert, nbv) &&
            h->get(h->gbar, kMaxFreeBones * kK) && h->get(h->cconst, kCapEntries + kK) &&
            h->get(h->bpart, kMaxFreeBones * kBoneMeanBlocks * 9) && h->get(h->cadd, kCapEntries + kK) &&
            h->get(h->bst, kMaxFreeBones * kBoneStride) && h->get(h->Qd, 3 * n);
  if (dry || h->npts > 0)
    ok = ok && h->get(h->jv, njv) && h->get(h->jw, njv * np) && h->get(h->jfree, njv) && h->get(h->jmask, n) &&
         h->get(h->Sinv, 256) && h->get(h->JJinv, 256) && h->get(h->Y64, 16 * n) && h->get(h->Y32, 16 * n) &&
         h->get(h->jlam, 3 * kMaxJointPts);
  if (dry || h->nfb > 0)
    ok = ok && h->get(h->frowptr, n + 1) && h->get(h->fcol, fnnz) && h->get(h->fval, fnnz) && h->get(h->fldinv, n) &&
         h->get(h->fin_fixed, n) && h->get(h->zeta, 16 * n) && h->get(h->fdt, 3 * kMaxFreeBones) &&
         h->get(h->phi_fin, 16 * n) && h->get(h->Einv_fin, 256);
  return ok;
}

int bones_upload(emu_handle* h, const double* Q) {
  if (!h->has_bones) return EMU_OK;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return bytes == 0 || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->st) == cudaSuccess;
  };
  const int64_t n = h->n, m = h->m;
  bool ok = up(h->tkind, h->tkind_h.data(), 4 * m) && up(h->btets, h->btets_h.data(), 4 * h->btets_h.size()) &&
            up(h->bvert, h->bvert_h.data(), 4 * h->bvert_h.size()) && up(h->Qd, Q, 24 * n);
  ok = ok && cudaMemsetAsync(h->cconst, 0, 8 * (kCapEntries + kK), h->st) == cudaSuccess &&
       cudaMemsetAsync(h->gbar, 0, 8 * kMaxFreeBones * kK, h->st) == cudaSuccess &&
       cudaMemsetAsync(h->bst, 0, 8 * kMaxFreeBones * kBoneStride, h->st) == cudaSuccess;
  if (h->npts > 0) {
    std::vector<uint8_t> mask(n, 0);
    for (int vi = 0; vi < h->njv; ++vi)
      if (h->jfree_h[vi]) mask[h->jv_h[vi]] = 1;
    std::vector<double> JJ(256, 0.0);
    for (size_t k = 0; k < h->JJinv_h.size(); ++k) JJ[k] = h->JJinv_h[k];
    ok = ok && up(h->jv, h->jv_h.data(), 4 * h->jv_h.size()) && up(h->jw, h->jw_h.data(), 8 * h->jw_h.size()) &&
         up(h->jfree, h->jfree_h.data(), h->jfree_h.size()) && up(h->jmask, mask.data(), n) &&
         up(h->JJinv, JJ.data(), 8 * 256) && cudaStreamSynchronize(h->st) == cudaSuccess;
  }
  if (h->nfb > 0)
    ok = ok && up(h->frowptr, h->frowptr_h.data(), 4 * (n + 1)) && up(h->fcol, h->fcol_h.data(), 4 * h->fnnz) &&
         up(h->fval, h->fval_h.data(), 8 * h->fnnz) && up(h->fldinv, h->fldinv_h.data(), 8 * n) &&
         up(h->fin_fixed, h->fin_fixed_h.data(), n);
  ok = ok && cudaStreamSynchronize(h->st) == cudaSuccess;
  return ok ? EMU_OK : bfail(EMU_ERR_CUDA, "upload of the bone and joint arrays failed");
}

// 16-column FP64 CG on a CSR matrix (Jacobi only): X_out = A^-1 X_in.
static int cg16(emu_handle* h, const int32_t* rowptr, const int32_t* col, const double* val, const double* dinv,
                const double* rhs, double* x, double tol) {
  PcgArgsT<double> a = h->pcg64(rhs, x, tol);
  a.rowptr = rowptr;
  a.col = col;
  a.val = val;
  a.dinv = dinv;
  a.max_iter = std::max(20000, 4 * h->prm.pcg_max);
  a.iters_out = nullptr;
  a.fail_out = nullptr;
  a.phi = nullptr;
  a.Einv = nullptr;
  BONE_CK(cudaMemsetAsync(x, 0, 16 * 8 * h->n, h->st));
  BONE_CK(launch_pcg<double>(16, a, h->grid_pcg16, h->st));
  return EMU_OK;
}

int joints_setup_device(emu_handle* h) {
  if (h->npts == 0) return EMU_OK;
  const int64_t n = h->n;
  const int np = h->npts;
  std::vector<double> rhs((size_t)n * 16, 0.0);
  for (int vi = 0; vi < h->njv; ++vi)
    if (h->jfree_h[vi])
      for (int r = 0; r < np; ++r) rhs[(size_t)h->jv_h[vi] * 16 + r] = h->jw_h[(size_t)vi * np + r];
  double* X = h->scratch16;
  BONE_CK(cudaMemcpyAsync(X, rhs.data(), rhs.size() * 8, cudaMemcpyHostToDevice, h->st));
  int rc = cg16(h, h->rowptr, h->col, h->val, h->ldinv, X, h->Y64, 1e-12);
  if (rc) return rc;
  launch_d2f(16 * n, h->Y64, h->Y32, h->st);
  JointArgs j = h->jargs();
  launch_joint_dot16(j, h->Y64, h->small, h->st);
  BONE_CK(cudaGetLastError());
  std::vector<double> S16(256);
  BONE_CK(cudaMemcpyAsync(S16.data(), h->small, 256 * 8, cudaMemcpyDeviceToHost, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  std::vector<double> S(np * np);
  for (int r = 0; r < np; ++r)
    for (int r2 = 0; r2 < np; ++r2) S[r * np + r2] = 0.5 * (S16[r * 16 + r2] + S16[r2 * 16 + r]);
  if (!invert_small(S, np)) return bfail(EMU_ERR_INVALID_ARG, "the joint rows' Schur complement is singular");
  std::vector<double> Sp(256, 0.0);
  for (size_t k = 0; k < S.size(); ++k) Sp[k] = S[k];
  BONE_CK(cudaMemcpyAsync(h->Sinv, Sp.data(), 256 * 8, cudaMemcpyHostToDevice, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  return EMU_OK;
}

// X (n x 16, device) <- X - J_f^T (J_f J_f^T)^-1 J_f X (Euclidean projection
// onto the null space of the joint rows).
int joints_project_basis(emu_handle* h, double* X) {
  if (h->npts == 0) return EMU_OK;
  const int np = h->npts;
  JointArgs j = h->jargs();
  launch_joint_dot16(j, X, h->small, h->st);
  std::vector<double> JX(256), M(256, 0.0);
  BONE_CK(cudaMemcpyAsync(JX.data(), h->small, 256 * 8, cudaMemcpyDeviceToHost, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  for (int r = 0; r < np; ++r)
    for (int k = 0; k < 16; ++k) {
      double s = 0.0;
      for (int r2 = 0; r2 < np; ++r2) s += h->JJinv_h[r * np + r2] * JX[r2 * 16 + k];
      M[r * 16 + k] = s;
    }
  BONE_CK(cudaMemcpyAsync(h->small, M.data(), 256 * 8, cudaMemcpyHostToDevice, h->st));
  launch_joint_sub16(j, h->n, h->small, 1, X, h->st);
  BONE_CK(cudaGetLastError());
  BONE_CK(cudaStreamSynchronize(h->st));
  return EMU_OK;
}

// Responses of q to each column of each free bone's F_b (the same scalar
// field for the three coordinates), solved with the joint rows: columns
// 16 - 3 nfb .. 15 of the device field X (n x 16) receive them.
int bones_basis_responses(emu_handle* h, double* X) {
  if (h->nfb == 0) return EMU_OK;
  const int64_t n = h->n, m = h->m;
  const int c0 = 16 - 3 * h->nfb;
  std::vector<double> Dinv(9 * m);
  BONE_CK(cudaMemcpyAsync(Dinv.data(), h->Dinv, 72 * m, cudaMemcpyDeviceToHost, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  std::vector<int32_t> tet(4 * m);
  BONE_CK(cudaMemcpyAsync(tet.data(), h->tet, 16 * m, cudaMemcpyDeviceToHost, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  std::vector<uint8_t> fixed(n);
  BONE_CK(cudaMemcpyAsync(fixed.data(), h->is_fixed, n, cudaMemcpyDeviceToHost, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  std::vector<double> rhs((size_t)n * 16, 0.0);
  for (int fi = 0; fi < h->nfb; ++fi)
    for (int32_t k = h->bptr_h[fi]; k < h->bptr_h[fi + 1]; ++k) {
      const int64_t i = h->btets_h[k];
      double gN[4][3];
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) gN[a][c] = Dinv[(3 * a + c) * m + i];
      for (int c = 0; c < 3; ++c) gN[3][c] = -(gN[0][c] + gN[1][c] + gN[2][c]);
      for (int a = 0; a < 4; ++a) {
        const int32_t v = tet[4 * i + a];
        if (fixed[v]) continue;
        for (int c = 0; c < 3; ++c) rhs[(size_t)v * 16 + 3 * fi + c] += h->w_h[i] * gN[a][c];
      }
    }
  double* R = h->scratch16 + n * 16;  // the caller's second n x 16 field is free here
  double* P = h->phi64;               // filled from the basis only after this step
  BONE_CK(cudaMemcpyAsync(R, rhs.data(), rhs.size() * 8, cudaMemcpyHostToDevice, h->st));
  int rc = cg16(h, h->rowptr, h->col, h->val, h->ldinv, R, P, 1e-12);
  if (rc) return rc;
  if (h->npts > 0) {  // constrained responses: psi - Y S^-1 J psi
    const int np = h->npts;
    JointArgs j = h->jargs();
    launch_joint_dot16(j, P, h->small, h->st);
    std::vector<double> JX(256), Sinv(256), M(256, 0.0);
    BONE_CK(cudaMemcpyAsync(JX.data(), h->small, 256 * 8, cudaMemcpyDeviceToHost, h->st));
    BONE_CK(cudaMemcpyAsync(Sinv.data(), h->Sinv, 256 * 8, cudaMemcpyDeviceToHost, h->st));
    BONE_CK(cudaStreamSynchronize(h->st));
    for (int r = 0; r < np; ++r)
      for (int k = 0; k < 16; ++k) {
        double s = 0.0;
        for (int r2 = 0; r2 < np; ++r2) s += Sinv[r * np + r2] * JX[r2 * 16 + k];
        M[r * 16 + k] = s;
      }
    BONE_CK(cudaMemcpyAsync(h->small, M.data(), 256 * 8, cudaMemcpyHostToDevice, h->st));
    launch_joint_sub16(j, n, h->small, 0, P, h->st);
    BONE_CK(cudaGetLastError());
  }
  std::vector<double> Xh((size_t)n * 16), Ph((size_t)n * 16);
  BONE_CK(cudaMemcpyAsync(Xh.data(), X, Xh.size() * 8, cudaMemcpyDeviceToHost, h->st));
  BONE_CK(cudaMemcpyAsync(Ph.data(), P, Ph.size() * 8, cudaMemcpyDeviceToHost, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  for (int64_t v = 0; v < n; ++v)
    for (int k = 0; k < 3 * h->nfb; ++k) Xh[(size_t)v * 16 + c0 + k] = Ph[(size_t)v * 16 + k];
  BONE_CK(cudaMemcpyAsync(X, Xh.data(), Xh.size() * 8, cudaMemcpyHostToDevice, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  return EMU_OK;
}

// The bones' constant capacitance terms and each free bone's Gbar, from the
// mode gradients Gamma of the bone tets (as the per-tet kernels use them).
int bones_after_gamma(emu_handle* h) {
  if (!h->has_bones) return EMU_OK;
  const int64_t m = h->m;
  std::vector<double> gam((size_t)kK * m);
  if (h->mixed) {
    std::vector<float> g32((size_t)kK * m);
    BONE_CK(cudaMemcpyAsync(g32.data(), h->gam32, g32.size() * 4, cudaMemcpyDeviceToHost, h->st));
    BONE_CK(cudaStreamSynchronize(h->st));
    for (size_t k = 0; k < gam.size(); ++k) gam[k] = g32[k];
  } else {
    BONE_CK(cudaMemcpyAsync(gam.data(), h->gam64, gam.size() * 8, cudaMemcpyDeviceToHost, h->st));
    BONE_CK(cudaStreamSynchronize(h->st));
  }
  auto G = [&](int64_t i, int j, int c) { return gam[(size_t)(3 * j + c) * m + i]; };
  std::vector<double> S16(256, 0.0), gbar(kMaxFreeBones * kK, 0.0);
  for (int64_t i = 0; i < m; ++i) {
    if (h->tkind_h[i] != kTetPinnedBone) continue;
    for (int j = 0; j < 16; ++j)
      for (int j2 = 0; j2 < 16; ++j2)
        S16[16 * j + j2] += h->w_h[i] * (G(i, j, 0) * G(i, j2, 0) + G(i, j, 1) * G(i, j2, 1) + G(i, j, 2) * G(i, j2, 2));
  }
  for (int fi = 0; fi < h->nfb; ++fi) {
    double* gb = gbar.data() + fi * kK;
    for (int32_t k = h->bptr_h[fi]; k < h->bptr_h[fi + 1]; ++k) {
      const int64_t i = h->btets_h[k];
      for (int e = 0; e < kK; ++e) gb[e] += h->w_h[i] * gam[(size_t)e * m + i];
    }
    for (int e = 0; e < kK; ++e) gb[e] /= h->wb_h[fi];
    for (int32_t k = h->bptr_h[fi]; k < h->bptr_h[fi + 1]; ++k) {
      const int64_t i = h->btets_h[k];
      double dg[kK];
      for (int e = 0; e < kK; ++e) dg[e] = gam[(size_t)e * m + i] - gb[e];
      for (int j = 0; j < 16; ++j)
        for (int j2 = 0; j2 < 16; ++j2)
          S16[16 * j + j2] += h->w_h[i] * (dg[3 * j] * dg[3 * j2] + dg[3 * j + 1] * dg[3 * j2 + 1] + dg[3 * j + 2] * dg[3 * j2 + 2]);
    }
  }
  std::vector<double> cc(kCapEntries + kK, 0.0);
  for (int r = 0; r < 3; ++r)
    for (int j = 0; j < 16; ++j)
      for (int j2 = 0; j2 < 16; ++j2) cc[(16 * r + j) * kK + 16 * r + j2] = S16[16 * j + j2];
  BONE_CK(cudaMemcpyAsync(h->cconst, cc.data(), cc.size() * 8, cudaMemcpyHostToDevice, h->st));
  BONE_CK(cudaMemcpyAsync(h->gbar, gbar.data(), gbar.size() * 8, cudaMemcpyHostToDevice, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  return EMU_OK;
}

int final_setup_device(emu_handle* h) {
  if (h->nfb == 0) return EMU_OK;
  const int64_t n = h->n;
  double* R = h->scratch16;
  double* Z = h->scratch16 + n * 16;
  BONE_CK(cudaMemcpyAsync(R, h->zrhs_h.data(), (size_t)n * 16 * 8, cudaMemcpyHostToDevice, h->st));
  int rc = cg16(h, h->frowptr, h->fcol, h->fval, h->fldinv, R, Z, 1e-12);
  if (rc) return rc;
  std::vector<double> Zh((size_t)n * 16);
  BONE_CK(cudaMemcpyAsync(Zh.data(), Z, Zh.size() * 8, cudaMemcpyDeviceToHost, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  for (int fi = 0; fi < h->nfb; ++fi)
    for (int32_t k = h->bvptr_h[fi]; k < h->bvptr_h[fi + 1]; ++k) Zh[(size_t)h->bvert_h[k] * 16 + fi] = 1.0;
  BONE_CK(cudaMemcpyAsync(h->zeta, Zh.data(), Zh.size() * 8, cudaMemcpyHostToDevice, h->st));
  // A = zeta^T L zeta (Newton-phase operator: the bone tets see zeta constant)
  const int ggrid = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 511) / 512), 2 * h->sms);
  launch_galerkin16(n, h->rowptr, h->col, h->val, h->zeta, Z, ggrid, h->part_pcg, h->st);
  launch_reduce_cols(h->part_pcg, ggrid, 256, h->small, h->st);
  BONE_CK(cudaGetLastError());
  std::vector<double> A16(256);
  BONE_CK(cudaMemcpyAsync(A16.data(), h->small, 256 * 8, cudaMemcpyDeviceToHost, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  const int nf = h->nfb;
  std::vector<double> A(nf * nf);
  for (int b = 0; b < nf; ++b)
    for (int b2 = 0; b2 < nf; ++b2) {
      double s = 0.5 * (A16[16 * b + b2] + A16[16 * b2 + b]);
      for (int r = 0; r < h->npts; ++r) s += h->kj * h->sgn_h[r * kMaxFreeBones + b] * h->sgn_h[r * kMaxFreeBones + b2];
      A[b * nf + b2] = s;
    }
  if (!invert_small(A, nf)) return bfail(EMU_ERR_INVALID_ARG, "the final solve's bone translations are singular");
  for (int b = 0; b < nf; ++b)
    for (int b2 = 0; b2 < nf; ++b2) h->Ainv_h[b * kMaxFreeBones + b2] = A[b * nf + b2];
  // coarse space of the final solve's CG: the basis with the rows the final
  // solve pins set to zero, and the pseudo-inverse of its Galerkin matrix
  std::vector<double> Ph((size_t)n * 16);
  BONE_CK(cudaMemcpyAsync(Ph.data(), h->phi64, Ph.size() * 8, cudaMemcpyDeviceToHost, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  for (int64_t v = 0; v < n; ++v)
    if (h->fin_fixed_h[v])
      for (int k = 0; k < 16; ++k) Ph[(size_t)v * 16 + k] = 0.0;
  BONE_CK(cudaMemcpyAsync(h->phi_fin, Ph.data(), Ph.size() * 8, cudaMemcpyHostToDevice, h->st));
  launch_galerkin16(n, h->frowptr, h->fcol, h->fval, h->phi_fin, Z, ggrid, h->part_pcg, h->st);
  launch_reduce_cols(h->part_pcg, ggrid, 256, h->small, h->st);
  BONE_CK(cudaGetLastError());
  std::vector<double> Eg(256), Ev;
  BONE_CK(cudaMemcpyAsync(Eg.data(), h->small, 256 * 8, cudaMemcpyDeviceToHost, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  for (int i = 0; i < 16; ++i)
    for (int j = 0; j < 16; ++j) Eg[16 * i + j] = 0.5 * (Eg[16 * i + j] + Eg[16 * j + i]);
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
  BONE_CK(cudaMemcpyAsync(h->Einv_fin, Ei.data(), 256 * 8, cudaMemcpyHostToDevice, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  return EMU_OK;
}

// ------------------------------------------------------------ iteration ---
void bones_after_grad(emu_handle* h) {
  if (h->nfb == 0) return;
  const BoneArgs a = h->bargs();
  launch_bone_mean(a, h->q, h->st);
  launch_bone_eval(a, nullptr, h->st);
  h->launches += 2;
}

void bones_gref(emu_handle* h, double* out) {
  if (h->nfb == 0) return;
  const BoneArgs a = h->bargs();
  launch_bone_mean(a, h->q0, h->st);
  launch_bone_eval(a, out, h->st);
}

const double* bones_cap_addend(const emu_handle* h) {
  if (!h->has_bones) return nullptr;
  return h->nfb > 0 ? h->cadd : h->cconst;
}

void bones_before_dir(emu_handle* h) {
  if (h->nfb == 0) return;
  launch_bone_dir(h->bargs(), h->z, h->part_dir + h->grid_tet, h->st);
  h->launches += 1;
}

int dir_partial_count(const emu_handle* h) { return h->grid_tet + (h->nfb > 0 ? 1 : 0); }

void joints_project(emu_handle* h, double* x64, float* x32) {
  if (h->npts == 0) return;
  launch_joint_project(h->jargs(), h->n, x64, x32, h->st);
  h->launches += 2;
}

void bones_state_from_element_arrays(emu_handle* h) {
  if (!h->has_bones) return;
  const BoneArgs a = h->bargs();
  launch_bone_state_from_tets(a, h->st);
  launch_bone_state_to_tets(a, h->tkind, h->st);
}

void bones_state_to_element_arrays(emu_handle* h) {
  if (!h->has_bones) return;
  launch_bone_state_to_tets(h->bargs(), h->tkind, h->st);
}

void bones_state_from_rep(emu_handle* h) {
  if (h->nfb == 0) return;
  launch_bone_state_from_tets(h->bargs(), h->st);
}

int bones_state_rest(emu_handle* h) {
  if (h->nfb == 0) return EMU_OK;
  std::vector<double> st((size_t)kMaxFreeBones * kBoneStride, 0.0);
  for (int b = 0; b < kMaxFreeBones; ++b) {
    double* o = st.data() + (size_t)b * kBoneStride;
    o[kBoneR] = o[kBoneR + 4] = o[kBoneR + 8] = 1.0;
    o[kBoneS] = o[kBoneS + 1] = o[kBoneS + 2] = 1.0;
  }
  BONE_CK(cudaMemcpyAsync(h->bst, st.data(), st.size() * 8, cudaMemcpyHostToDevice, h->st));
  BONE_CK(cudaStreamSynchronize(h->st));
  return EMU_OK;
}

void bones_update_mixed(emu_handle* h) {
  if (h->nfb == 0 || !h->mixed) return;
  launch_bone_update(h->bargs(), h->st);
  h->launches += 1;
}

// Final coupling solve (bone rows hard, joints as a penalty), blocking.
int bones_final_solve(emu_handle* h) {
  if (h->nfb == 0) return EMU_OK;
  const int64_t n = h->n;
  const BoneArgs ba = h->bargs();
  const FinalArgs fa = h->fargs();
  const JointArgs ja = h->jargs();
  double* b = h->b;
  double* r64 = h->b + 3 * n;
  double* e64 = h->b + 6 * n;
  // b = G^T W F of the current state (Eq. 4's right-hand side)
  if (h->mixed)
    launch_rhs_state_mixed(h->margs(), h->grid_tet, h->st);
  else
    launch_rhs_from_state(h->args<double>(), h->grid_tet, h->st);
  launch_assemble(n, h->slot_ptr, h->slot_idx, h->contrib, h->bfix, h->is_fixed, h->qfix, 0, b, h->st);
  launch_final_set_bones(ba, fa, h->q, h->st);
  BONE_CK(cudaGetLastError());
  const int rgrid = (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 2 * (int64_t)h->sms);
  double nrm[3] = {0, 0, 0};
  for (int j = 0; j < 3; ++j) nrm[j] = h->o6_host[8 + j];  // |G^T W (F - I)|^2 of the last exact solve
  const double tol = h->q_tol;
  for (int round = 0; round < 4; ++round) {
    BONE_CK(launch_residual64(n, h->rowptr, h->col, h->val, b, h->q, nullptr, r64, h->part_pcg, rgrid, h->small, h->st,
                              h->fin_fixed));
    launch_final_mask(fa, n, r64, h->st);
    double o[6];
    BONE_CK(cudaMemcpyAsync(o, h->small, 6 * 8, cudaMemcpyDeviceToHost, h->st));
    BONE_CK(cudaStreamSynchronize(h->st));
    bool done = true;
    double need = 0.5;
    for (int j = 0; j < 3; ++j) {
      done = done && (o[j] <= 1e-2 * tol * tol * nrm[j] || o[j] <= 1e-30 * o[3 + j]);
      if (o[j] > 0.0 && nrm[j] > 0.0) need = std::min(need, 0.02 * tol * std::sqrt(nrm[j] / o[j]));
    }
    if (done) break;
    PcgArgsT<double> a = h->pcg64(r64, e64, std::max(need, 1e-13));
    a.rowptr = h->frowptr;
    a.col = h->fcol;
    a.val = h->fval;
    a.dinv = h->fldinv;
    a.phi = h->phi_fin;
    a.Einv = h->Einv_fin;
    a.max_iter = std::max(20000, 4 * h->prm.pcg_max);
    BONE_CK(cudaMemsetAsync(e64, 0, 24 * n, h->st));
    BONE_CK(launch_pcg<double>(3, a, h->grid_pcg3, h->st));
    BONE_CK(launch_axpy_d2d(3 * n, e64, h->q, h->st));
  }
  // the bones' translations: one exact step of the quadratic in t
  BONE_CK(launch_residual64(n, h->rowptr, h->col, h->val, b, h->q, nullptr, r64, h->part_pcg, rgrid, h->small, h->st,
                            nullptr));
  launch_final_tstep(fa, ja, r64, h->q, h->st);
  launch_final_apply(fa, n, h->q, h->st);
  BONE_CK(cudaGetLastError());
  BONE_CK(cudaStreamSynchronize(h->st));
  return EMU_OK;
}

}  // namespace emu

// ------------------------------------------------------------ arg builders --
BoneArgs emu_handle::bargs() const {
  BoneArgs a;
  memset(&a, 0, sizeof(a));
  a.nfb = nfb;
  a.mixed = mixed ? 1 : 0;
  a.m = m;
  a.n = n;
  a.tet = tet;
  a.Dinv = Dinv;
  a.c = c;
  a.q = q;
  a.Q = Qd;
  a.R = R;
  a.s = s;
  a.quat = quat;
  a.E = E32;
  a.btets = btets;
  for (int k = 0; k <= nfb && k <= kMaxFreeBones; ++k) a.bptr[k] = k < (int)bptr_h.size() ? bptr_h[k] : 0;
  for (int k = 0; k < nfb; ++k) {
    a.rep[k] = rep_h[k];
    a.Vb[k] = Vb_h[k];
    a.wb[k] = wb_h[k];
    a.mu[k] = mub_h[k];
    a.lam[k] = lamb_h[k];
  }
  a.alpha = alpha;
  a.gbar = gbar;
  a.cconst = cconst;
  a.part = bpart;
  a.cadd = cadd;
  a.bst = bst;
  a.sc = sc;
  return a;
}

JointArgs emu_handle::jargs() const {
  JointArgs j;
  memset(&j, 0, sizeof(j));
  j.npts = npts;
  j.njv = njv;
  j.jv = jv;
  j.jw = jw;
  j.jfree = jfree;
  j.Sinv = Sinv;
  j.JJinv = JJinv;
  j.Y64 = Y64;
  j.Y32 = Y32;
  j.lam = jlam;
  return j;
}

FinalArgs emu_handle::fargs() const {
  FinalArgs f;
  memset(&f, 0, sizeof(f));
  f.nfb = nfb;
  f.npts = npts;
  f.bvert = bvert;
  for (int k = 0; k <= nfb && k <= kMaxFreeBones; ++k) f.bvptr[k] = k < (int)bvptr_h.size() ? bvptr_h[k] : 0;
  f.zeta = zeta;
  for (int k = 0; k < kMaxFreeBones * kMaxFreeBones; ++k) f.Ainv[k] = Ainv_h[k];
  for (int k = 0; k < kMaxJointPts * kMaxFreeBones && k < (int)sgn_h.size(); ++k) f.sgn[k] = sgn_h[k];
  f.kj = kj;
  f.dt = fdt;
  f.fin_fixed = fin_fixed;
  return f;
}
