// Test harness for the host set-up (setup.cpp) on the CPU: builds the model
// and the impressed-field projection structures of a mesh and writes the
// assembled matrices, so the CPU tests can compare them with the oracle
// without a GPU.
//
//   host_dump <mesh.bin> <out.bin> <order>
//   mesh.bin: int32 n_nodes, n_tets; double xyz[3 n_nodes]; int32 tets[4 n_tets];
//             int32 tags[4 n_tets]
//   out.bin:  CSRs M, K, C, D, M2, Ival (on M's pattern), DA, LA, LAI (on LA's
//             pattern), Dv; then uint8 pec1[n1], bnd0[n0]; the load's rule
//             (int32 nq, double lam[nq][4], w[nq]); the injection faces (int32
//             F, double xyz[F][9], int32 tet[F], double cum[F])
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../paper_2111_12411_gb300/csrc/internal.h"

using namespace fempic;

static void dump(FILE* o, const HostCSR& A) {
  const int32_t h[2] = {A.n_rows, A.n_cols};
  const int64_t nnz = A.nnz();
  fwrite(h, 4, 2, o);
  fwrite(&nnz, 8, 1, o);
  if (A.rowptr.empty()) {  // an operator that was not built: zero rows
    const int32_t zero = 0;
    fwrite(&zero, 4, 1, o);
  } else {
    fwrite(A.rowptr.data(), 4, A.rowptr.size(), o);
  }
  fwrite(A.col.data(), 4, (size_t)nnz, o);
  fwrite(A.val.data(), 8, (size_t)nnz, o);
}

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  const int order = atoi(argv[3]);
  int32_t nn = 0, nt = 0;
  if (fread(&nn, 4, 1, f) != 1 || fread(&nt, 4, 1, f) != 1) return 2;
  std::vector<double> xyz(3 * (size_t)nn);
  std::vector<int32_t> tets(4 * (size_t)nt), tags(4 * (size_t)nt);
  if (fread(xyz.data(), 8, xyz.size(), f) != xyz.size() || fread(tets.data(), 4, tets.size(), f) != tets.size() ||
      fread(tags.data(), 4, tags.size(), f) != tags.size())
    return 2;
  fclose(f);
  HostModel m;
  std::string err;
  if (build_model(xyz.data(), nn, tets.data(), nt, order, &m, &err, tags.data())) {
    fprintf(stderr, "%s\n", err.c_str());
    return 1;
  }
  ProjModel P;
  err = build_projection(order, m.n_tets, m.n_faces, m.n2, xyz.data(), m.tets.data(), m.dof2.data(), m.M2, &P);
  if (!err.empty()) {
    fprintf(stderr, "%s\n", err.c_str());
    return 1;
  }
  FILE* o = fopen(argv[2], "wb");
  if (!o) return 2;
  HostCSR I = m.M;
  I.val = m.Ival.empty() ? std::vector<double>(m.M.val.size(), 0.0) : m.Ival;
  HostCSR LI = m.LA;
  LI.val = m.LAI;
  for (const HostCSR* A : {&m.M, &m.K, &m.C, &m.D, &m.M2, &I, &m.DA, &m.LA, &LI, &P.Dv}) dump(o, *A);
  fwrite(m.pec1.data(), 1, m.pec1.size(), o);
  fwrite(m.bnd0.data(), 1, m.bnd0.size(), o);
  // the load's quadrature rule and the injection faces
  const int32_t nq = P.nq, nf = (int32_t)m.inj_tet.size();
  fwrite(&nq, 4, 1, o);
  fwrite(P.qlam.data(), 8, P.qlam.size(), o);
  fwrite(P.qw.data(), 8, P.qw.size(), o);
  fwrite(&nf, 4, 1, o);
  fwrite(m.inj_xyz.data(), 8, m.inj_xyz.size(), o);
  fwrite(m.inj_tet.data(), 4, m.inj_tet.size(), o);
  fwrite(m.inj_cum.data(), 8, m.inj_cum.size(), o);
  fclose(o);
  return 0;
}
