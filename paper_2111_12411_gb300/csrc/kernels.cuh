// Device code of the EM-FEMPIC step: the fused particle kernel (gather E and B,
// Lorentz push, ray-face walk, charge-conserving path-integral deposit, charge
// measurement), counting sort by tet, CSR kernels and the device-resident
// preconditioned conjugate-gradient solve.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fempic {
namespace dev {

constexpr double kGL2X = 0.5773502691896257645;  // 1/sqrt(3)
constexpr uint64_t kFnvOffset = 14695981039346656037ull;
constexpr uint64_t kFnvPrime = 1099511628211ull;

// Device status bits (latched; the host maps them to FEMPIC_ERR_*).
constexpr int kStatusWalk = 1;
constexpr int kStatusCG = 2;
constexpr int kStatusBarrier = 4;
constexpr int kStatusBounds = 8;

// Checked builds (-DFEMPIC_CHECKS=1): a tet id outside [0, n) sets the status
// word (reported as FEMPIC_ERR_BOUNDS) and the particle is skipped instead of
// reading out of bounds; without the flag the test folds away.
#ifndef FEMPIC_CHECKS
#define FEMPIC_CHECKS 0
#endif
__device__ __forceinline__ bool index_ok(int64_t i, int64_t n, int32_t* status) {
  if (!FEMPIC_CHECKS) return true;
  if (i >= 0 && i < n) return true;
  atomicOr(status, kStatusBounds);
  return false;
}

// Checked builds: tet ids that arrive from a caller's device buffer.
__global__ void k_check_ids(int64_t n, const int32_t* ids, int32_t n_tets, int32_t* status) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    index_ok(ids[i], n_tets, status);
}

// Checked builds, once at create: every entry of the per-tet DOF tables within
// its space and every neighbour record (tet << 2 | face) naming a tet.
__global__ void k_check_tables(int32_t n_tets, int nl0, int nl1, int nl2, const int32_t* dof0, const int32_t* dof1,
                               const int32_t* dof2, const int32_t* nbr, int32_t n0, int32_t n1, int32_t n2,
                               int32_t* status) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tets; t += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < nl0; ++k) index_ok(dof0[t * nl0 + k], n0, status);
    for (int k = 0; k < nl1; ++k) index_ok(dof1[t * nl1 + k], n1, status);
    for (int k = 0; k < nl2; ++k) index_ok(dof2[t * nl2 + k], n2, status);
    for (int k = 0; k < 4; ++k) {
      const int32_t nb = nbr[t * 4 + k];
      if (nb >= 0)
        index_ok(nb >> 2, n_tets, status);
      else if (nb < -2)
        index_ok(-1, 1, status);
    }
  }
}

// ---- arithmetic policies ----------------------------------------------------
// Strict: one rounding per operation, in the written order (no contraction).
struct Strict {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
  // a*b + c with two roundings
  static __device__ __forceinline__ double mad(double a, double b, double c) { return __dadd_rn(__dmul_rn(a, b), c); }
};
// Fast: the compiler may fuse multiply-adds.
struct Fast {
  static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
};

// ---- compile-time tables (constexpr functions fold to immediates after unrolling)
// local edge j = (edge_s(j), edge_t(j)); local face f = (face_v(f,0..2)), opposite vertex f
__host__ __device__ constexpr int edge_s(int j) { constexpr int t[6] = {0, 0, 0, 1, 1, 2}; return t[j]; }
__host__ __device__ constexpr int edge_t(int j) { constexpr int t[6] = {1, 2, 3, 2, 3, 3}; return t[j]; }
__host__ __device__ constexpr int face_v(int f, int k) {
  constexpr int t[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  return t[f][k];
}
// index of the local edge (a,b), a < b
__host__ __device__ constexpr int pair_of(int a, int b) {
  return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}
// W1 of order 2: function j = m(l) (l_a grad l_b - l_b grad l_a), {a, b, x, kind}
// kind 1: m = 3 l_x - 1 (edge functions), kind 2: m = 3 l_x (face functions)
__host__ __device__ constexpr int w1q(int j, int c) {
  constexpr int t[20][4] = {{0, 1, 0, 1}, {0, 1, 1, 1}, {0, 2, 0, 1}, {0, 2, 2, 1}, {0, 3, 0, 1},
                            {0, 3, 3, 1}, {1, 2, 1, 1}, {1, 2, 2, 1}, {1, 3, 1, 1}, {1, 3, 3, 1},
                            {2, 3, 2, 1}, {2, 3, 3, 1}, {1, 2, 3, 2}, {1, 3, 2, 2}, {0, 2, 3, 2},
                            {0, 3, 2, 2}, {0, 1, 3, 2}, {0, 3, 1, 2}, {0, 1, 2, 2}, {0, 2, 1, 2}};
  return t[j][c];
}
// W2 of order 2: function j = m(l) w_face, {face, x, kind}; kind 1: 4 l_x - 1, 2: 4 l_x
__host__ __device__ constexpr int w2q(int j, int c) {
  constexpr int t[15][3] = {{0, 1, 1}, {0, 2, 1}, {0, 3, 1}, {1, 0, 1}, {1, 2, 1}, {1, 3, 1}, {2, 0, 1}, {2, 1, 1},
                            {2, 3, 1}, {3, 0, 1}, {3, 1, 1}, {3, 2, 1}, {0, 0, 2}, {1, 1, 2}, {2, 2, 2}};
  return t[j][c];
}

template <class Ar>
__device__ __forceinline__ void cross3(const double* a, const double* b, double* o) {
  o[0] = Ar::sub(Ar::mul(a[1], b[2]), Ar::mul(a[2], b[1]));
  o[1] = Ar::sub(Ar::mul(a[2], b[0]), Ar::mul(a[0], b[2]));
  o[2] = Ar::sub(Ar::mul(a[0], b[1]), Ar::mul(a[1], b[0]));
}

template <class Ar>
__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return Ar::add(Ar::add(Ar::mul(a[0], b[0]), Ar::mul(a[1], b[1])), Ar::mul(a[2], b[2]));
}

// geom layout per tet: g[4][3] row-major then c[4]
struct TetGeom {
  double g[4][3];
  double c[4];
};

__device__ __forceinline__ void load_geom(const double* __restrict__ geom, int t, TetGeom& G) {
  const double2* p = reinterpret_cast<const double2*>(geom + (size_t)t * 16);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    double2 v = __ldg(p + k);
    double* dst = &G.g[0][0];
    dst[2 * k] = v.x;
    dst[2 * k + 1] = v.y;
  }
}

// lambda_i(x) = ((g_i0 x0 + g_i1 x1) + g_i2 x2) + c_i
template <class Ar>
__device__ __forceinline__ void bary(const TetGeom& G, const double* x, double* l) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
    l[i] = Ar::add(Ar::add(Ar::add(Ar::mul(G.g[i][0], x[0]), Ar::mul(G.g[i][1], x[1])), Ar::mul(G.g[i][2], x[2])),
                   G.c[i]);
}

// ---- order 3 (Appendix): multipliers as products of Silvester polynomials,
// P_i(l) = prod_{m<i} (n l - m) / i!, P^_i(l) = prod_{1<=m<i} (n l - m) / (i-1)!,
// evaluated factor by factor from 1.0, one rounding per operation.
template <class Ar>
__device__ __forceinline__ double silv(int i, double n, double l, bool hat) {
  double val = 1.0;
  for (int m = hat ? 1 : 0; m < i; ++m) val = Ar::mul(val, Ar::sub(Ar::mul(n, l), (double)m));
  const int k = hat ? i - 1 : i;
  const double fac = k <= 1 ? 1.0 : (k == 2 ? 2.0 : 6.0);
  return Ar::div(val, fac);
}

// W1 of order 3, function j: m(l) (l_a grad l_b - l_b grad l_a), scale 4.
// j < 18: edge j/3 with (P^_a(l_s), P^_b(l_t)), (a, b) = (3,1), (2,2), (1,3);
// j < 42: face (j-18)/6, pairs (s,t) then (s,u) of the face s<t<u, each with
// (P^_a, P^_b, P_c) on (pair first, pair second, third vertex), (a,b,c) =
// (2,1,1), (1,2,1), (1,1,2); j < 45: pairs (0,1), (0,2), (0,3) with
// P^_1 P^_1 P_1 P_1 (the other two vertices ascending).
template <class Ar>
__device__ __forceinline__ double w1_p3(int j, const double* l, int& a, int& b) {
  if (j < 18) {
    const int e = j / 3, q = j % 3;
    a = edge_s(e);
    b = edge_t(e);
    double m = 1.0;
    m = Ar::mul(m, silv<Ar>(3 - q, 4.0, l[a], true));
    m = Ar::mul(m, silv<Ar>(1 + q, 4.0, l[b], true));
    return m;
  }
  if (j < 42) {
    const int f = (j - 18) / 6, r = (j - 18) % 6, pr = r / 3, q = r % 3;
    const int s = face_v(f, 0), t = face_v(f, 1), u = face_v(f, 2);
    a = s;
    b = pr == 0 ? t : u;
    const int c = pr == 0 ? u : t;
    const int ia = q == 0 ? 2 : 1, ib = q == 1 ? 2 : 1, ic = q == 2 ? 2 : 1;
    double m = 1.0;
    m = Ar::mul(m, silv<Ar>(ia, 4.0, l[a], true));
    m = Ar::mul(m, silv<Ar>(ib, 4.0, l[b], true));
    m = Ar::mul(m, silv<Ar>(ic, 4.0, l[c], false));
    return m;
  }
  a = 0;
  b = j - 41;
  int o0 = -1, o1 = -1;
#pragma unroll
  for (int v = 1; v < 4; ++v)
    if (v != b) {
      if (o0 < 0)
        o0 = v;
      else
        o1 = v;
    }
  double m = 1.0;
  m = Ar::mul(m, silv<Ar>(1, 4.0, l[a], true));
  m = Ar::mul(m, silv<Ar>(1, 4.0, l[b], true));
  m = Ar::mul(m, silv<Ar>(1, 4.0, l[o0], false));
  m = Ar::mul(m, silv<Ar>(1, 4.0, l[o1], false));
  return m;
}

// W2 of order 3, function j: m(l) w_face, scale 5.  j < 24: face j/6 with
// (P^_a, P^_b, P^_c) on its vertices, (a,b,c) = (3,1,1), (1,3,1), (1,1,3),
// (2,2,1), (2,1,2), (1,2,2); j < 36: the faces opposite vertices 0, 1, 2,
// (j-24)/4, with (a,b,c,d) = (2,1,1,1), (1,2,1,1), (1,1,2,1), (1,1,1,2), d on
// the opposite vertex (P_d).
template <class Ar>
__device__ __forceinline__ double w2_p3(int j, const double* l, int& f) {
  if (j < 24) {
    f = j / 6;
    const int q = j % 6;
    constexpr int T[6][3] = {{3, 1, 1}, {1, 3, 1}, {1, 1, 3}, {2, 2, 1}, {2, 1, 2}, {1, 2, 2}};
    double m = 1.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) m = Ar::mul(m, silv<Ar>(T[q][k], 5.0, l[face_v(f, k)], true));
    return m;
  }
  f = (j - 24) / 4;
  const int q = (j - 24) % 4;
  double m = 1.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) m = Ar::mul(m, silv<Ar>(q == k ? 2 : 1, 5.0, l[face_v(f, k)], true));
  m = Ar::mul(m, silv<Ar>(q == 3 ? 2 : 1, 5.0, l[f], false));
  return m;
}

// W0 of order 3 (Lagrange on the scale-3 lattice), function k: nodes, then two
// per edge ((2,1) then (1,2) on (s,t)), then one per face; factors in vertex order
template <class Ar>
__device__ __forceinline__ double w0_p3(int k, const double* l) {
  if (k < 4) return Ar::mul(1.0, silv<Ar>(3, 3.0, l[k], false));
  if (k < 16) {
    const int e = (k - 4) / 2, q = (k - 4) % 2;
    double m = 1.0;
    m = Ar::mul(m, silv<Ar>(q == 0 ? 2 : 1, 3.0, l[edge_s(e)], false));
    m = Ar::mul(m, silv<Ar>(q == 0 ? 1 : 2, 3.0, l[edge_t(e)], false));
    return m;
  }
  const int f = k - 16;
  double m = 1.0;
#pragma unroll
  for (int v = 0; v < 3; ++v) m = Ar::mul(m, silv<Ar>(1, 3.0, l[face_v(f, v)], false));
  return m;
}

template <int P>
struct Nloc {
  static constexpr int n1 = P == 1 ? 6 : (P == 2 ? 20 : 45);
  static constexpr int n2 = P == 1 ? 4 : (P == 2 ? 15 : 36);
  static constexpr int n0 = P == 1 ? 4 : (P == 2 ? 10 : 20);
};

// E = sum_j e_j W1_j(x), accumulated in j order
template <int P, class Ar>
__device__ __forceinline__ void gather_E(const TetGeom& G, const double* l, const double* ev, double* E) {
  E[0] = E[1] = E[2] = 0.0;
  if (P == 3) {
    #pragma unroll
    for (int j = 0; j < 45; ++j) {
      int a, b;
      const double m = w1_p3<Ar>(j, l, a, b);
      double w[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) w[k] = Ar::mul(m, Ar::sub(Ar::mul(l[a], G.g[b][k]), Ar::mul(l[b], G.g[a][k])));
#pragma unroll
      for (int k = 0; k < 3; ++k) E[k] = Ar::add(E[k], Ar::mul(ev[j], w[k]));
    }
    return;
  }
  constexpr int N = P == 1 ? 6 : 20;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    int a, b, x = 0, kind = 0;
    if (P == 1) {
      a = edge_s(j);
      b = edge_t(j);
    } else {
      a = w1q(j, 0);
      b = w1q(j, 1);
      x = w1q(j, 2);
      kind = w1q(j, 3);
    }
    double w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = Ar::sub(Ar::mul(l[a], G.g[b][k]), Ar::mul(l[b], G.g[a][k]));
    if (P == 2) {
      double m = kind == 1 ? Ar::sub(Ar::mul(3.0, l[x]), 1.0) : Ar::mul(3.0, l[x]);
#pragma unroll
      for (int k = 0; k < 3; ++k) w[k] = Ar::mul(m, w[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) E[k] = Ar::add(E[k], Ar::mul(ev[j], w[k]));
  }
}

// Whitney face function of local face f: 2 ((l_s X_tu + l_t X_us) + l_u X_st)
template <class Ar>
__device__ __forceinline__ void whitney_face(const TetGeom& G, const double* l, int f, double* w) {
  const int s = face_v(f, 0), t = face_v(f, 1), u = face_v(f, 2);
  double xtu[3], xus[3], xst[3];
  cross3<Ar>(G.g[t], G.g[u], xtu);
  cross3<Ar>(G.g[u], G.g[s], xus);
  cross3<Ar>(G.g[s], G.g[t], xst);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    w[k] = Ar::mul(Ar::add(Ar::add(Ar::mul(l[s], xtu[k]), Ar::mul(l[t], xus[k])), Ar::mul(l[u], xst[k])), 2.0);
}

template <int P, class Ar>
__device__ __forceinline__ void gather_B(const TetGeom& G, const double* l, const double* bv, const double* B0,
                                         double* B) {
  double acc[3] = {0.0, 0.0, 0.0};
  if (P == 1) {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      double w[3];
      whitney_face<Ar>(G, l, f, w);
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[k] = Ar::add(acc[k], Ar::mul(bv[f], w[k]));
    }
  } else if (P == 3) {
    double wf[4][3];
#pragma unroll
    for (int f = 0; f < 4; ++f) whitney_face<Ar>(G, l, f, wf[f]);
    #pragma unroll
    for (int j = 0; j < 36; ++j) {
      int f;
      const double m = w2_p3<Ar>(j, l, f);
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[k] = Ar::add(acc[k], Ar::mul(bv[j], Ar::mul(m, wf[f][k])));
    }
  } else {
    double wf[4][3];
#pragma unroll
    for (int f = 0; f < 4; ++f) whitney_face<Ar>(G, l, f, wf[f]);
#pragma unroll
    for (int j = 0; j < 15; ++j) {
      const int f = w2q(j, 0), x = w2q(j, 1), kind = w2q(j, 2);
      double m = kind == 1 ? Ar::sub(Ar::mul(4.0, l[x]), 1.0) : Ar::mul(4.0, l[x]);
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[k] = Ar::add(acc[k], Ar::mul(bv[j], Ar::mul(m, wf[f][k])));
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) B[k] = Ar::add(acc[k], B0[k]);
}

// Boris rotation (h = q dt / 2m precomputed on the host as ((q/m) dt) 0.5)
template <class Ar>
__device__ __forceinline__ void boris(double* v, const double* E, const double* B, double h) {
  double eh[3], vm[3], t[3], s[3], vp[3], cr[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    eh[k] = Ar::mul(E[k], h);
    vm[k] = Ar::add(v[k], eh[k]);
    t[k] = Ar::mul(B[k], h);
  }
  double t2 = Ar::add(Ar::add(Ar::mul(t[0], t[0]), Ar::mul(t[1], t[1])), Ar::mul(t[2], t[2]));
  double sf = Ar::div(2.0, Ar::add(1.0, t2));
#pragma unroll
  for (int k = 0; k < 3; ++k) s[k] = Ar::mul(t[k], sf);
  cross3<Ar>(vm, t, cr);
#pragma unroll
  for (int k = 0; k < 3; ++k) vp[k] = Ar::add(vm[k], cr[k]);
  cross3<Ar>(vp, s, cr);
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = Ar::add(Ar::add(vm[k], cr[k]), eh[k]);
}

// q w int_{s0}^{s1} W1_j(r(s)) . (b - a) ds for all local j, added into dg
template <int P, class Ar>
__device__ __forceinline__ void deposit_segment(const double* la, const double* lb, double s0, double s1, double qw,
                                                const int32_t* __restrict__ dofs, double* __restrict__ dg) {
  double d[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) d[i] = Ar::sub(lb[i], la[i]);
  if (P == 1) {
    double Pv[4], Qv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      Pv[i] = Ar::add(la[i], Ar::mul(s0, d[i]));
      Qv[i] = Ar::add(la[i], Ar::mul(s1, d[i]));
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int s = edge_s(j), t = edge_t(j);
      double val = Ar::sub(Ar::mul(Pv[s], Qv[t]), Ar::mul(Pv[t], Qv[s]));
      atomicAdd(dg + __ldg(dofs + j), Ar::mul(qw, val));
    }
  } else if (P == 3) {
    double half = Ar::mul(Ar::sub(s1, s0), 0.5);
    double mid = Ar::mul(Ar::add(s0, s1), 0.5);
    double r = Ar::mul(half, kGL2X);
    double sg[2] = {Ar::sub(mid, r), Ar::add(mid, r)};
    double L[2][4];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int i = 0; i < 4; ++i) L[q][i] = Ar::add(la[i], Ar::mul(sg[q], d[i]));
    #pragma unroll
    for (int j = 0; j < 45; ++j) {
      double f[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        int a, b;
        const double m = w1_p3<Ar>(j, L[q], a, b);
        f[q] = Ar::mul(m, Ar::sub(Ar::mul(L[q][a], d[b]), Ar::mul(L[q][b], d[a])));
      }
      atomicAdd(dg + __ldg(dofs + j), Ar::mul(qw, Ar::mul(half, Ar::add(f[0], f[1]))));
    }
  } else {
    double half = Ar::mul(Ar::sub(s1, s0), 0.5);
    double mid = Ar::mul(Ar::add(s0, s1), 0.5);
    double r = Ar::mul(half, kGL2X);
    double sg[2] = {Ar::sub(mid, r), Ar::add(mid, r)};
    double L[2][4];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int i = 0; i < 4; ++i) L[q][i] = Ar::add(la[i], Ar::mul(sg[q], d[i]));
#pragma unroll
    for (int j = 0; j < 20; ++j) {
      const int a = w1q(j, 0), b = w1q(j, 1), x = w1q(j, 2), kind = w1q(j, 3);
      double f[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        double m = kind == 1 ? Ar::sub(Ar::mul(3.0, L[q][x]), 1.0) : Ar::mul(3.0, L[q][x]);
        f[q] = Ar::mul(m, Ar::sub(Ar::mul(L[q][a], d[b]), Ar::mul(L[q][b], d[a])));
      }
      atomicAdd(dg + __ldg(dofs + j), Ar::mul(qw, Ar::mul(half, Ar::add(f[0], f[1]))));
    }
  }
}

template <int P, class Ar>
__device__ __forceinline__ void deposit_rho(const double* l, double qw, const int32_t* __restrict__ dofs,
                                            double* __restrict__ rho) {
  if (P == 1) {
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(rho + __ldg(dofs + k), Ar::mul(qw, l[k]));
  } else if (P == 3) {
    #pragma unroll
    for (int k = 0; k < 20; ++k) atomicAdd(rho + __ldg(dofs + k), Ar::mul(qw, w0_p3<Ar>(k, l)));
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      atomicAdd(rho + __ldg(dofs + k), Ar::mul(qw, Ar::mul(l[k], Ar::sub(Ar::mul(2.0, l[k]), 1.0))));
#pragma unroll
    for (int j = 0; j < 6; ++j)
      atomicAdd(rho + __ldg(dofs + 4 + j), Ar::mul(qw, Ar::mul(Ar::mul(4.0, l[edge_s(j)]), l[edge_t(j)])));
  }
}

// Several species: particle ids are given out in species order, so species k
// owns the ids [off[k], off[k+1]); its charge weight q w and push factor
// q dt / 2m come from the table (n == 1: the scalar qw, h of the launch).
constexpr int kMaxSpecies = 8;
struct SpeciesTable {
  int n;
  int32_t off[kMaxSpecies + 1];
  double qw[kMaxSpecies];
  double h[kMaxSpecies];
};

__device__ __forceinline__ int species_of(const SpeciesTable& s, int32_t id) {
  int k = 0;
  while (k + 1 < s.n && id >= s.off[k + 1]) ++k;
  return k;
}

struct ParticleArgs {
  int64_t n;
  double* x[3];
  double* v[3];
  int32_t* tet;
  int32_t* ncross;
  unsigned long long* hash;
  const double* geom;
  const int32_t* nbr;
  const int32_t* dof0;
  const int32_t* dof1;
  const int32_t* dof2;
  const double* e;
  const double* b;
  double* dg;
  double* rho;
  double B0[3];
  double h;    // q dt / 2m
  double dt;
  double qw;
  int max_cross;
  int32_t* status;
  unsigned long long* crossings;
  const int32_t* pid;  // particle ids in device order (read only with several species)
  SpeciesTable sp;
  uint8_t* absorbed = nullptr;  // [n] 1 where the path ended on an absorbing wall (null: none)
  int32_t n_tets = 0;           // bound of the tet ids (checked builds)
  // FP32 copies read by the mixed-precision gather (null: convert on use):
  // e and b rounded to FP32, and the gradients of each tet's barycentrics
  // ([nt][12]); the same values the conversions would give
  const float* e32 = nullptr;
  const float* b32 = nullptr;
  const float* geom32 = nullptr;
};

// q w and q dt / 2m of the particle in device slot i
__device__ __forceinline__ void particle_consts(const ParticleArgs& a, int64_t i, double& qw, double& h) {
  qw = a.qw;
  h = a.h;
  if (a.sp.n > 1) {
    const int k = species_of(a.sp, __ldg(a.pid + i));
    qw = a.sp.qw[k];
    h = a.sp.h[k];
  }
}

// One thread per particle: gather, push, walk, deposit, charge.
template <int P, class Ar>
__global__ void __launch_bounds__(256) k_particle(ParticleArgs a) {
  constexpr int N1 = Nloc<P>::n1;
  constexpr int N2 = Nloc<P>::n2;
  constexpr int N0 = Nloc<P>::n0;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long my_cross = 0;
  if (i < a.n && index_ok(a.tet[i], a.n_tets, a.status)) {
    int T = a.tet[i];
    double x[3] = {a.x[0][i], a.x[1][i], a.x[2][i]};
    double v[3] = {a.v[0][i], a.v[1][i], a.v[2][i]};
    double qw, hq;
    particle_consts(a, i, qw, hq);
    TetGeom G;
    load_geom(a.geom, T, G);
    double l[4];
    bary<Ar>(G, x, l);
    double ev[N1], bv[N2];
    const int32_t* d1 = a.dof1 + (size_t)T * N1;
    const int32_t* d2 = a.dof2 + (size_t)T * N2;
#pragma unroll
    for (int j = 0; j < N1; ++j) ev[j] = __ldg(a.e + __ldg(d1 + j));
#pragma unroll
    for (int j = 0; j < N2; ++j) bv[j] = __ldg(a.b + __ldg(d2 + j));
    double E[3], B[3];
    gather_E<P, Ar>(G, l, ev, E);
    gather_B<P, Ar>(G, l, bv, a.B0, B);
    boris<Ar>(v, E, B, hq);
    double pa[3] = {x[0], x[1], x[2]};
    double pb[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) pb[k] = Ar::add(x[k], Ar::mul(a.dt, v[k]));
    int entry = -1;
    double s0 = 0.0;
    int nc = 0;
    uint8_t absorbed = 0;
    unsigned long long hsh = kFnvOffset;
    for (;;) {
      double la[4], lb[4];
      bary<Ar>(G, pa, la);
      bary<Ar>(G, pb, lb);
      int best = -1;
      double sbest = __longlong_as_double(0x7ff0000000000000ll);  // +inf
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        if (f != entry && lb[f] < 0.0) {
          double si = Ar::div(la[f], Ar::sub(la[f], lb[f]));
          if (si < sbest) {
            sbest = si;
            best = f;
          }
        }
      }
      double s1 = best < 0 ? 1.0 : fmin(fmax(sbest, s0), 1.0);
      deposit_segment<P, Ar>(la, lb, s0, s1, qw, a.dof1 + (size_t)T * N1, a.dg);
      if (best < 0) {
        deposit_rho<P, Ar>(lb, qw, a.dof0 + (size_t)T * N0, a.rho);
        break;
      }
      ++nc;
      int nb = __ldg(a.nbr + (size_t)T * 4 + best);
      unsigned long long code = nb == -2  ? (0xC0000000ull | (unsigned)best)
                                : nb < 0 ? (0x80000000ull | (unsigned)best)
                                         : (unsigned long long)(nb >> 2);
      hsh = (hsh ^ code) * kFnvPrime;
      if (nb >= 0) {
        entry = nb & 3;
        T = nb >> 2;
        if (!index_ok(T, a.n_tets, a.status)) break;
        s0 = s1;
        load_geom(a.geom, T, G);
      } else if (nb == -2) {  // absorbing wall: the path ends at the hit point, no charge left
#pragma unroll
        for (int k = 0; k < 3; ++k) pb[k] = Ar::add(pa[k], Ar::mul(s1, Ar::sub(pb[k], pa[k])));
        absorbed = 1;
        break;
      } else {
        double gw[3];
#pragma unroll
        for (int f = 0; f < 4; ++f)
          if (f == best) {
            gw[0] = G.g[f][0];
            gw[1] = G.g[f][1];
            gw[2] = G.g[f][2];
          }
        double d[3], hit[3], dr[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = Ar::sub(pb[k], pa[k]);
#pragma unroll
        for (int k = 0; k < 3; ++k) hit[k] = Ar::add(pa[k], Ar::mul(s1, d[k]));
        double gg = dot3<Ar>(gw, gw);
        double fd = Ar::div(Ar::mul(2.0, dot3<Ar>(d, gw)), gg);
        double fv = Ar::div(Ar::mul(2.0, dot3<Ar>(v, gw)), gg);
        double rem = Ar::sub(1.0, s1);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          dr[k] = Ar::sub(d[k], Ar::mul(fd, gw[k]));
          v[k] = Ar::sub(v[k], Ar::mul(fv, gw[k]));
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          pb[k] = Ar::add(hit[k], Ar::mul(rem, dr[k]));
          pa[k] = hit[k];
        }
        s0 = 0.0;
        entry = best;
      }
      if (nc >= a.max_cross) {
        double lf[4];
        bary<Ar>(G, pb, lf);
        deposit_rho<P, Ar>(lf, qw, a.dof0 + (size_t)T * N0, a.rho);
        atomicOr(a.status, kStatusWalk);
        break;
      }
    }
    a.x[0][i] = pb[0];
    a.x[1][i] = pb[1];
    a.x[2][i] = pb[2];
    a.v[0][i] = v[0];
    a.v[1][i] = v[1];
    a.v[2][i] = v[2];
    a.tet[i] = T;
    if (a.ncross) a.ncross[i] = nc;
    if (a.hash) a.hash[i] = hsh;
    if (a.absorbed) a.absorbed[i] = absorbed;
    my_cross = nc;
  }
  // block-aggregated crossing count
  for (int o = 16; o > 0; o >>= 1) my_cross += __shfl_xor_sync(0xffffffffu, my_cross, o);
  if ((threadIdx.x & 31) == 0 && my_cross) atomicAdd(a.crossings, my_cross);
}

// rho from positions (used at start and after the state is set)
template <int P>
__global__ void k_rho(int64_t n, const double* x0, const double* x1, const double* x2, const int32_t* tet,
                      const double* geom, const int32_t* dof0, double qw, double* rho, const int32_t* pid,
                      SpeciesTable sp) {
  constexpr int N0 = Nloc<P>::n0;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (sp.n > 1) qw = sp.qw[species_of(sp, __ldg(pid + i))];
  int T = tet[i];
  TetGeom G;
  load_geom(geom, T, G);
  double x[3] = {x0[i], x1[i], x2[i]};
  double l[4];
  bary<Strict>(G, x, l);
  deposit_rho<P, Strict>(l, qw, dof0 + (size_t)T * N0, rho);
}

// E and B at given points (owning tets known)
template <int P, class Ar>
__global__ void k_eval_fields(int64_t n, const double* xs, const int32_t* tets, const double* geom,
                              const int32_t* dof1, const int32_t* dof2, const double* e, const double* b,
                              double B00, double B01, double B02, double* Eo, double* Bo) {
  constexpr int N1 = Nloc<P>::n1;
  constexpr int N2 = Nloc<P>::n2;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int T = tets[i];
  TetGeom G;
  load_geom(geom, T, G);
  double x[3] = {xs[3 * i], xs[3 * i + 1], xs[3 * i + 2]};
  double l[4];
  bary<Ar>(G, x, l);
  double ev[N1], bv[N2];
  for (int j = 0; j < N1; ++j) ev[j] = e[dof1[(size_t)T * N1 + j]];
  for (int j = 0; j < N2; ++j) bv[j] = b[dof2[(size_t)T * N2 + j]];
  double B0[3] = {B00, B01, B02};
  double E[3], B[3];
  gather_E<P, Ar>(G, l, ev, E);
  gather_B<P, Ar>(G, l, bv, B0, B);
  for (int k = 0; k < 3; ++k) {
    Eo[3 * i + k] = E[k];
    Bo[3 * i + k] = B[k];
  }
}

}  // namespace dev
}  // namespace fempic
