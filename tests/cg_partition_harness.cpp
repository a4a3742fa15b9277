// Host-only driver of build_cg_partition for the CPU tests: reads the
// Laplacian and the rest positions from a binary file, writes the partition,
// the permuted system and the local table to another.
//
// input  (little-endian): int64 n, nnz; int32 G, rpt, nt, degree;
//                         double Q[3n]; int32 rowptr[n+1], col[nnz]; double val[nnz]
// output: int32 ok, G, rpt, nt, lw, degree; double lmax; float c0, c1[8], c2[8];
//         int32 perm[n], off[G+1]; int64 nnz_p; int32 rowptr[n+1], col[nnz_p];
//         float val[nnz_p], dinv[n]; int64 nloc; uint32 loc[nloc]
#include <cstdio>
#include <vector>

#include "emu_cgpart.h"

template <typename T> static bool rd(FILE* f, T* p, size_t cnt) { return fread(p, sizeof(T), cnt, f) == cnt; }
template <typename T> static void wr(FILE* f, const T* p, size_t cnt) { fwrite(p, sizeof(T), cnt, f); }

int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* fi = fopen(argv[1], "rb");
  if (!fi) return 3;
  int64_t n = 0, nnz = 0;
  int32_t G = 0, rpt = 0, nt = 0, degree = 0;
  if (!rd(fi, &n, 1) || !rd(fi, &nnz, 1) || !rd(fi, &G, 1) || !rd(fi, &rpt, 1) || !rd(fi, &nt, 1) ||
      !rd(fi, &degree, 1))
    return 4;
  std::vector<double> Q(3 * n), val(nnz);
  std::vector<int32_t> rowptr(n + 1), col(nnz);
  if (!rd(fi, Q.data(), Q.size()) || !rd(fi, rowptr.data(), rowptr.size()) || !rd(fi, col.data(), col.size()) ||
      !rd(fi, val.data(), val.size()))
    return 5;
  fclose(fi);
  emu::CgPartHost P;
  const int32_t ok = emu::build_cg_partition(n, Q.data(), rowptr, col, val, G, rpt, nt, degree, &P) ? 1 : 0;
  FILE* fo = fopen(argv[2], "wb");
  if (!fo) return 6;
  const int32_t hdr[6] = {ok, P.G, P.rpt, P.nt, P.lw, P.degree};
  wr(fo, hdr, 6);
  wr(fo, &P.lmax, 1);
  wr(fo, &P.c0, 1);
  wr(fo, P.c1, emu::kChebMax);
  wr(fo, P.c2, emu::kChebMax);
  if (ok) {
    wr(fo, P.perm.data(), P.perm.size());
    wr(fo, P.off.data(), P.off.size());
    const int64_t nnz_p = (int64_t)P.col.size();
    wr(fo, &nnz_p, 1);
    wr(fo, P.rowptr.data(), P.rowptr.size());
    wr(fo, P.col.data(), P.col.size());
    wr(fo, P.val.data(), P.val.size());
    wr(fo, P.dinv.data(), P.dinv.size());
    const int64_t nloc = (int64_t)P.loc.size();
    wr(fo, &nloc, 1);
    wr(fo, P.loc.data(), P.loc.size());
  }
  fclose(fo);
  return 0;
}
