// Host construction of the CG row partition and its block-local
// preconditioner table (see emu_cgpart.h).
#include "emu_cgpart.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace emu {

namespace {

// the local polynomial approximates the inverse on [lmax / kChebRatio, lmax]
constexpr double kChebRatio = 30.0;
// Off-diagonal entries below kPrune sqrt(A_ii A_jj) are left out of the
// permuted FP32 system: on a tetrahedral grid most of them are the rounding
// residue of sums that cancel exactly (on a Kuhn grid the stiffness of the
// diagonal edges is zero, about half of each row), and at that size they are
// below FP32's resolution of the row anyway.
constexpr double kPrune = 1e-8;

uint32_t bf16_bits(float f) {  // round to nearest even (finite input)
  uint32_t b;
  std::memcpy(&b, &f, 4);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return b & 0xFFFF0000u;
}

float from_bits(uint32_t b) {
  float f;
  std::memcpy(&f, &b, 4);
  return f;
}

// Recursive coordinate bisection: idx[0, cnt) goes to parts p0 .. p0 + p - 1
// whose sizes are pre[p0 + i + 1] - pre[p0 + i]. Each split is along the
// longest extent of the set, at the exact row count of the first half of
// the parts; ties in the coordinate go by vertex index (a total order, so
// the split is unique).
void rcb(const double* Q, int32_t* idx, int64_t cnt, int p0, int p, const std::vector<int64_t>& pre,
         std::vector<int32_t>& part) {
  if (p == 1) {
    for (int64_t k = 0; k < cnt; ++k) part[idx[k]] = p0;
    return;
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t k = 0; k < cnt; ++k)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], Q[3 * (int64_t)idx[k] + a]);
      hi[a] = std::max(hi[a], Q[3 * (int64_t)idx[k] + a]);
    }
  int ax = 0;
  for (int a = 1; a < 3; ++a)
    if (hi[a] - lo[a] > hi[ax] - lo[ax]) ax = a;
  const int p1 = p / 2;
  const int64_t c1 = pre[p0 + p1] - pre[p0];
  auto less = [&](int32_t x, int32_t y) {
    const double qx = Q[3 * (int64_t)x + ax], qy = Q[3 * (int64_t)y + ax];
    return qx < qy || (qx == qy && x < y);
  };
  if (c1 > 0 && c1 < cnt) std::nth_element(idx, idx + c1, idx + cnt, less);
  rcb(Q, idx, c1, p0, p1, pre, part);
  rcb(Q, idx + c1, cnt - c1, p0 + p1, p - p1, pre, part);
}

}  // namespace

int cg_local_width_max(int rpt) { return rpt <= 2 ? 24 : 15; }

bool build_cg_partition(int64_t n, const double* Q, const std::vector<int32_t>& rowptr,
                        const std::vector<int32_t>& col, const std::vector<double>& val, int G, int rpt, int nt,
                        int degree, CgPartHost* out) {
  if (G < 1 || rpt < 1 || nt < 1 || n < 1 || (int64_t)G * rpt * nt < n || degree < 1 || degree > kChebMax)
    return false;
  const int64_t cap = (int64_t)rpt * nt;
  if (cap > 65536) return false;  // local columns are 16-bit
  CgPartHost& P = *out;
  P = CgPartHost();
  P.G = G;
  P.rpt = rpt;
  P.nt = nt;
  P.degree = degree;

  // ---- balanced parts: n / G rows, the first n % G parts one more ----
  std::vector<int64_t> pre(G + 1, 0);
  for (int b = 0; b < G; ++b) pre[b + 1] = pre[b] + n / G + (b < n % G ? 1 : 0);
  if (pre[1] > cap) return false;
  std::vector<int32_t> idx(n), part(n, 0);
  for (int64_t v = 0; v < n; ++v) idx[v] = (int32_t)v;
  rcb(Q, idx.data(), n, 0, G, pre, part);
  // rows of a part in vertex order (the mesh's own locality)
  P.perm.resize(n);
  P.off.assign(pre.begin(), pre.end());
  {
    std::vector<int64_t> fill(pre.begin(), pre.end() - 1);
    for (int64_t v = 0; v < n; ++v) P.perm[fill[part[v]]++] = (int32_t)v;
  }
  std::vector<int32_t> iperm(n);
  for (int64_t r = 0; r < n; ++r) iperm[P.perm[r]] = (int32_t)r;

  // ---- the permuted Laplacian (columns ascending per row) ----
  const int64_t nnz = rowptr[n];
  P.rowptr.assign(n + 1, 0);
  P.col.reserve(nnz);
  P.val.reserve(nnz);
  P.dinv.resize(n);
  std::vector<double> diag(n, 1.0), pval;
  pval.reserve(nnz);
  for (int64_t v = 0; v < n; ++v)
    for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e)
      if (col[e] == v) diag[v] = val[e];
  {
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t r = 0; r < n; ++r) {
      const int32_t v = P.perm[r];
      row.clear();
      for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
        const int32_t c = col[e];
        if (c != v && std::fabs(val[e]) <= kPrune * std::sqrt(std::fabs(diag[v] * diag[c]))) continue;
        row.push_back({iperm[c], val[e]});
      }
      std::sort(row.begin(), row.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
      P.rowptr[r + 1] = P.rowptr[r] + (int32_t)row.size();
      for (size_t k = 0; k < row.size(); ++k) {
        P.col.push_back(row[k].first);
        P.val.push_back((float)row[k].second);
        pval.push_back(row[k].second);
      }
      P.dinv[r] = (float)(1.0 / diag[v]);
    }
  }
  if (degree == 1) {
    P.lw = 0;
    P.c0 = 1.f;
    P.lmax = 1.0;
    return true;
  }

  // ---- local entries of D^-1/2 A D^-1/2 (symmetrised), largest kept ----
  const int W = cg_local_width_max(rpt);
  auto part_of = [&](int64_t r) { return (int)(std::upper_bound(pre.begin(), pre.end(), r) - pre.begin()) - 1; };
  auto entry_val = [&](int64_t r, int32_t c) -> double {  // A_rc in the permuted numbering, 0 if absent
    const int32_t* b0 = P.col.data() + P.rowptr[r];
    const int32_t* b1 = P.col.data() + P.rowptr[r + 1];
    const int32_t* it = std::lower_bound(b0, b1, c);
    return (it != b1 && *it == c) ? pval[it - P.col.data()] : 0.0;
  };
  std::vector<std::vector<std::pair<int32_t, double>>> keep(n);
  for (int64_t r = 0; r < n; ++r) {
    const int b = part_of(r);
    const double dr = diag[P.perm[r]];
    auto& kr = keep[r];
    for (int32_t e = P.rowptr[r]; e < P.rowptr[r + 1]; ++e) {
      const int32_t c = P.col[e];
      if (c == r || c < pre[b] || c >= pre[b + 1]) continue;
      const double sym = 0.5 * (pval[e] + entry_val(c, (int32_t)r));
      kr.push_back({c, sym / std::sqrt(dr * diag[P.perm[c]])});
    }
    if ((int)kr.size() > W) {
      std::sort(kr.begin(), kr.end(), [](const auto& x, const auto& y) {
        const double ax = std::fabs(x.second), ay = std::fabs(y.second);
        return ax > ay || (ax == ay && x.first < y.first);
      });
      kr.resize(W);
      std::sort(kr.begin(), kr.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    }
  }
  // an entry stays only if both of its rows kept it
  auto kept = [&](int64_t r, int32_t c) {
    const auto& kr = keep[r];
    auto it = std::lower_bound(kr.begin(), kr.end(), c, [](const auto& x, int32_t cc) { return x.first < cc; });
    return it != kr.end() && it->first == c;
  };
  std::vector<std::vector<std::pair<int32_t, double>>> fin(n);
  int lw = 0;
  for (int64_t r = 0; r < n; ++r) {
    for (const auto& e : keep[r])
      if (kept(e.first, (int32_t)r)) fin[r].push_back(e);
    lw = std::max(lw, (int)fin[r].size());
  }
  if (lw == 0) {  // no coupling inside any part: Jacobi
    P.degree = 1;
    P.lw = 0;
    P.c0 = 1.f;
    P.lmax = 1.0;
    return true;
  }
  P.lw = lw;
  P.loc.assign((size_t)G * rpt * lw * nt, 0u);
  double lmax = 1.0;
  for (int b = 0; b < G; ++b)
    for (int64_t r = pre[b]; r < pre[b + 1]; ++r) {
      const int64_t li = r - pre[b];
      const int k = (int)(li / nt), t = (int)(li % nt);
      double rs = 1.0;
      for (int e = 0; e < lw; ++e) {
        uint32_t word = (uint32_t)li;  // padding: the row's own slot, weight 0
        if (e < (int)fin[r].size()) {
          const uint32_t vb = bf16_bits((float)fin[r][e].second);
          rs += std::fabs((double)from_bits(vb));
          word = (uint32_t)(fin[r][e].first - pre[b]) | vb;
        }
        P.loc[(((size_t)b * rpt + k) * lw + e) * nt + t] = word;
      }
      lmax = std::max(lmax, rs);
    }
  P.lmax = lmax;
  cg_cheb_coeffs(lmax, degree, &P.c0, P.c1, P.c2);
  return true;
}

// Chebyshev acceleration on [lmin, lmax] from a zero start (Saad,
// Iterative Methods for Sparse Linear Systems, Alg. 12.1): d_0 = r / theta,
// then d_i = rho_i rho_{i-1} d_{i-1} + (2 rho_i / delta) res_i
void cg_cheb_coeffs(double lmax, int degree, float* c0, float* c1, float* c2) {
  const double lmin = lmax / kChebRatio;
  const double th = 0.5 * (lmax + lmin), de = 0.5 * (lmax - lmin), sg = th / de;
  double rho = 1.0 / sg;
  *c0 = (float)(1.0 / th);
  for (int i = 0; i < kChebMax; ++i) c1[i] = c2[i] = 0.f;
  for (int i = 1; i < degree; ++i) {
    const double rn = 1.0 / (2.0 * sg - rho);
    c1[i] = (float)(rn * rho);
    c2[i] = (float)(2.0 * rn / de);
    rho = rn;
  }
}

}  // namespace emu
