// Internal structures shared by the host set-up (setup.cpp) and the device
// code (fempic.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace fempic {

// Local DOF counts per tet (Appendix): W0 (k+1)(k+2)(k+3)/6, W1 k(k+2)(k+3)/2,
// W2 k(k+1)(k+3)/2.
inline int nloc0(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
inline int nloc1(int p) { return p * (p + 2) * (p + 3) / 2; }
inline int nloc2(int p) { return p * (p + 1) * (p + 3) / 2; }

constexpr int kLocalEdges[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
constexpr int kLocalFaces[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};  // face i opposite vertex i

struct HostCSR {
  int32_t n_rows = 0, n_cols = 0;
  std::vector<int32_t> rowptr, col;
  std::vector<double> val;
  int64_t nnz() const { return (int64_t)col.size(); }
};

// Everything the device needs, built on the host at create time.
struct HostModel {
  int order = 1, nl0 = 4, nl1 = 6, nl2 = 4;
  int32_t n_nodes = 0, n_tets = 0, n_edges = 0, n_faces = 0;
  int32_t n0 = 0, n1 = 0, n2 = 0, n_bfaces = 0;
  std::vector<int32_t> tets;     // [nt][4] sorted vertex ids
  std::vector<double> geom;      // [nt][16]: g (4x3 row-major), c[4]
  std::vector<double> vol;       // [nt]
  std::vector<int32_t> nbr;      // [nt][4]: (neighbour << 2) | neighbour's local face, -1 = wall,
                                 // -2 = wall that absorbs particles
  std::vector<int32_t> dof0, dof1, dof2;  // [nt][nl*]
  std::vector<uint8_t> pec1;     // [n1] 1 on boundary W1 DOFs
  std::vector<uint8_t> bnd0;     // [n0] 1 on boundary W0 DOFs
  HostCSR M, K;                  // [*eps], curl-curl (free rows/cols), same pattern
  HostCSR Q;                     // C^T [*mu^-1] (free rows), N1 x N2
  HostCSR C;                     // N2 x N1 (free cols)
  HostCSR M2;                    // [*mu^-1]
  HostCSR D;                     // N1 x N0 (interior cols)
  HostCSR DT;                    // N0 x N1
  HostCSR L;                     // nodal Laplacian D^T [*eps] D, interior rows/cols
  std::vector<double> load0;     // <W0_k, 1>
  HostCSR Pi, PiT;               // vector nodal interpolation: W1 coefficients of hat_v e_c
  std::vector<double> dvM, dvK;  // diag(Pi^T M Pi), diag(Pi^T K Pi)
  int32_t n_imp_faces = 0;       // boundary faces with the impedance (absorbing) condition
  int32_t n_absorb_faces = 0;    // boundary faces that absorb particles (nbr = -2 there)
  std::vector<double> inj_xyz;   // [F][3][3] injection faces (global order), sorted vertices
  std::vector<int32_t> inj_tet;  // [F] owning tet
  std::vector<double> inj_cum;   // [F] running sum of the faces' areas
  std::vector<double> Ival;      // Y0 <n x W1_i, n x W1_j> over impedance faces, on M's pattern
  HostCSR DA, DAT, LA;           // with impedance faces only: the gradient map on the W0 DOFs
                                 // off PEC faces (free W1 rows), its transpose, and
                                 // D_a^T [*eps] D_a on those DOFs (preconditioner space)
  std::vector<double> LAI;       // D_a^T [*_I] D_a on LA's pattern
  HostCSR VM;                    // Pi^T M Pi (values) and its pattern
  std::vector<double> VK;        // Pi^T K Pi on VM's pattern
};

// Local tables of the order-p bases, computed exactly on the reference tet.
struct LocalTables {
  int order = 1, nl0 = 4, nl1 = 6, nl2 = 4;
  std::vector<double> Dloc;  // [nl1][nl0]: grad W0_k = sum_i Dloc[i][k] W1_i
  std::vector<double> Cloc;  // [nl2][nl1]: curl W1_j = sum_f Cloc[f][j] W2_f
  std::vector<double> T1;    // [nl1][nl1][4][4]: int_ref P1_ia P1_jb
  std::vector<double> T2;    // [nl2][nl2][6][6]: int_ref P2_{f,ab} P2_{h,cd}
  std::vector<double> I0;    // [nl0]: int_ref W0_k
  std::vector<double> Rv;    // order 2: [4][4][nl1]: W1 coefficients of l_v grad l_a
  std::vector<double> TF;    // [4][nl1][nl1][4][4]: int over the face opposite vertex i of the
                             // reference tet of P1_ia P1_jb, per unit of twice the face area
};

// Returns "" on success, else an error message.
std::string build_local_tables(int order, LocalTables* out);
// code: 0 ok, 2 mesh error, 1 argument error.
// bface_tag (nullable): [4*n_tets], tag of the face opposite the i-th vertex
// of each tet as given: 0 PEC, 1 impedance (read for boundary faces only).
int build_model(const double* xyz, int32_t n_nodes, const int32_t* tets, int32_t n_tets,
                int order, HostModel* m, std::string* err, const int32_t* bface_tag = nullptr);

// Host structures of the impressed-field projection (Section III-C, eq. conB).
struct ProjModel {
  int n3 = 0, nq = 0;            // W3 per tet; quadrature points per tet
  std::vector<double> qlam, qw;  // [nq][4] barycentric points, [nq] weights (sum 1/6)
  std::vector<double> vol6;      // [nt] 6 |V_t|
  HostCSR Dv, DvT;               // [~div]_ij = <W3_i, div W2_j>, N3 x N2, and its transpose
  HostCSR Bm;                    // block-Jacobi inverse of [*mu^-1] (face and interior DOF groups)
  HostCSR Bs;                    // per-tet block inverse of Dv Bm Dv^T
  HostCSR Asm;                   // N2 x (nt nl2): sums per-tet load vectors into global DOFs
};

// Exact table Dref [n3][nl2] = int_ref W3_i div W2_j of the order-p volume
// functions against the W2 divergences on the reference tet (a physical tet's
// [~div] block is sign(det J) Dref).
void div_table(int order, std::vector<double>* Dref, int* n3);
// The load's quadrature on the reference tet: conical product of (p + 3)-point
// Gauss-Legendre rules, x = u, y = (1-u) v, z = (1-u)(1-v) w, Jacobian
// (1-u)^2 (1-v); exact for total degree 2p + 3.  Fills nq, qlam, qw.
void projection_rule(int order, ProjModel* out);
// tets: [nt][4] sorted vertex ids (as in HostModel); M2 the assembled [*mu^-1].
// Returns "" on success, else an error message.
std::string build_projection(int order, int32_t n_tets, int32_t n_faces, int32_t n2, const double* xyz,
                             const int32_t* tets, const int32_t* dof2, const HostCSR& M2, ProjModel* out);

// Physical constants (CODATA 2018).
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.25663706212e-6;
// free-space admittance sqrt(eps0 / mu0) of the first-order absorbing condition

}  // namespace fempic
