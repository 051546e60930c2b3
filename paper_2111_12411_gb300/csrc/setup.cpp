// Host set-up of the EM-FEMPIC model: exact local tables of the order-p
// interpolatory Whitney bases (Appendix), mesh complex and DOF numbering
// (Section III-A), barycentric maps, and CSR assembly of the Hodge matrices,
// the curl-curl matrix and the exact-sequence maps.
//
// This file must be compiled without floating-point contraction
// (-ffp-contract=off): the barycentric maps are evaluated in a fixed order with
// one rounding per operation so that the device walk is reproducible.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <thread>

#include "internal.h"

namespace fempic {
namespace {

// ------------------------------------------------------------------------
// Exact rational arithmetic and polynomials (local tables only).
// ------------------------------------------------------------------------
using i128 = __int128;

i128 gcd128(i128 a, i128 b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b != 0) {
    i128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}

struct Rat {
  i128 n = 0, d = 1;
};

Rat mk(i128 n, i128 d) {
  if (d < 0) {
    n = -n;
    d = -d;
  }
  i128 g = gcd128(n, d);
  if (g > 1) {
    n /= g;
    d /= g;
  }
  if (n == 0) d = 1;
  return Rat{n, d};
}
Rat operator+(Rat a, Rat b) { return mk(a.n * b.d + b.n * a.d, a.d * b.d); }
Rat operator-(Rat a, Rat b) { return mk(a.n * b.d - b.n * a.d, a.d * b.d); }
Rat operator*(Rat a, Rat b) { return mk(a.n * b.n, a.d * b.d); }
Rat operator/(Rat a, Rat b) { return mk(a.n * b.d, a.d * b.n); }
bool is_zero(Rat a) { return a.n == 0; }
double to_double(Rat a) { return (double)a.n / (double)a.d; }
Rat R(long long n, long long d = 1) { return mk(n, d); }

// Polynomial: exponent key -> coefficient.  Four 4-bit exponent fields, used
// either for barycentric (l0,l1,l2,l3) or Cartesian reference (x,y,z) terms.
struct Poly {
  std::map<uint32_t, Rat> c;
};

int ex(uint32_t key, int v) { return (key >> (4 * v)) & 15; }

Poly padd(const Poly& a, const Poly& b, Rat sb = R(1)) {
  Poly r = a;
  for (auto& kv : b.c) {
    Rat v = r.c.count(kv.first) ? r.c[kv.first] + sb * kv.second : sb * kv.second;
    if (is_zero(v))
      r.c.erase(kv.first);
    else
      r.c[kv.first] = v;
  }
  return r;
}
Poly pscale(const Poly& a, Rat s) {
  Poly r;
  if (is_zero(s)) return r;
  for (auto& kv : a.c) r.c[kv.first] = kv.second * s;
  return r;
}
Poly pmul(const Poly& a, const Poly& b) {
  Poly r;
  for (auto& x : a.c)
    for (auto& y : b.c) {
      uint32_t k = x.first + y.first;  // fields never exceed 15 here
      Rat v = r.c.count(k) ? r.c[k] + x.second * y.second : x.second * y.second;
      if (is_zero(v))
        r.c.erase(k);
      else
        r.c[k] = v;
    }
  return r;
}
Poly pconst(Rat v) {
  Poly r;
  if (!is_zero(v)) r.c[0] = v;
  return r;
}
Poly lam(int i) {  // barycentric l_i
  Poly r;
  r.c[1u << (4 * i)] = R(1);
  return r;
}
// a*l_i + b
Poly lin(int i, long long a, long long b) { return padd(pscale(lam(i), R(a)), pconst(R(b))); }

long long fact(int n) {
  long long f = 1;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// int over the reference tet of l0^a l1^b l2^c l3^d = a! b! c! d! / (a+b+c+d+3)!
Rat integrate_bary(const Poly& p) {
  Rat s = R(0);
  for (auto& kv : p.c) {
    int a = ex(kv.first, 0), b = ex(kv.first, 1), c = ex(kv.first, 2), d = ex(kv.first, 3);
    s = s + kv.second * mk((i128)fact(a) * fact(b) * fact(c) * fact(d), (i128)fact(a + b + c + d + 3));
  }
  return s;
}

// int over the face l_i = 0 of l_a^. l_b^. l_c^. (the other three), per unit
// of twice the face area: a! b! c! / (a+b+c+2)!; monomials with l_i vanish
Rat integrate_face(const Poly& p, int face) {
  Rat s = R(0);
  for (auto& kv : p.c) {
    if (ex(kv.first, face) != 0) continue;
    long long num = 1;
    int tot = 0;
    for (int v = 0; v < 4; ++v)
      if (v != face) {
        num *= fact(ex(kv.first, v));
        tot += ex(kv.first, v);
      }
    s = s + kv.second * mk((i128)num, (i128)fact(tot + 2));
  }
  return s;
}

// Barycentric -> Cartesian on the reference tet: l0 = 1-x-y-z, l1 = x, l2 = y, l3 = z.
Poly to_xyz(const Poly& p) {
  Poly X, Y, Z;
  X.c[1u] = R(1);
  Y.c[1u << 4] = R(1);
  Z.c[1u << 8] = R(1);
  Poly L0 = padd(padd(padd(pconst(R(1)), X, R(-1)), Y, R(-1)), Z, R(-1));
  Poly out;
  for (auto& kv : p.c) {
    Poly t = pconst(kv.second);
    for (int k = 0; k < ex(kv.first, 0); ++k) t = pmul(t, L0);
    for (int k = 0; k < ex(kv.first, 1); ++k) t = pmul(t, X);
    for (int k = 0; k < ex(kv.first, 2); ++k) t = pmul(t, Y);
    for (int k = 0; k < ex(kv.first, 3); ++k) t = pmul(t, Z);
    out = padd(out, t);
  }
  return out;
}

Poly deriv(const Poly& p, int v) {  // d/dx_v of a Cartesian polynomial
  Poly r;
  for (auto& kv : p.c) {
    int e = ex(kv.first, v);
    if (e == 0) continue;
    r.c[kv.first - (1u << (4 * v))] = kv.second * R(e);
  }
  return r;
}

using Vec = std::array<Poly, 3>;
const int kG[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};  // grad l on the reference tet

std::array<int, 3> gcross(int a, int b) {
  return {kG[a][1] * kG[b][2] - kG[a][2] * kG[b][1], kG[a][2] * kG[b][0] - kG[a][0] * kG[b][2],
          kG[a][0] * kG[b][1] - kG[a][1] * kG[b][0]};
}

int pair_index(int a, int b) {
  for (int k = 0; k < 6; ++k)
    if (kLocalEdges[k][0] == a && kLocalEdges[k][1] == b) return k;
  return -1;
}

// Silvester polynomials at scale n in l_v (Appendix): P_i = prod_{m<i} (n l - m) / i!,
// P^_i = prod_{1<=m<i} (n l - m) / (i-1)!
Poly silvester(int i, int n, int v, bool hat) {
  Poly r = pconst(R(1));
  for (int m = hat ? 1 : 0; m < i; ++m) r = pmul(r, lin(v, n, -m));
  return pscale(r, R(1, fact(hat ? i - 1 : i)));
}

// Order-3 multipliers (the same families as the reference evaluation): W1
// m w_st with m = P^_a(l_s) P^_b(l_t) P_c(l_u) P_d(l_v) at scale 4; W2
// m w_stu with P^_a P^_b P^_c P_d at scale 5; W0 the scale-3 lattice.
struct Factor {
  int v, i;
  bool hat;
};
Poly multiplier(const std::vector<Factor>& fs, int n) {
  Poly r = pconst(R(1));
  for (const Factor& f : fs) r = pmul(r, silvester(f.i, n, f.v, f.hat));
  return r;
}

// Redundant forms: W1 = sum_a P[a] grad l_a; W2 = sum_{a<b} P[pair] grad l_a x grad l_b.
std::vector<std::array<Poly, 4>> w1_forms(int p) {
  std::vector<std::array<Poly, 4>> out;
  auto add = [&](int a, int b, const Poly& m) {
    std::array<Poly, 4> f;
    f[b] = pmul(m, lam(a));
    f[a] = pscale(pmul(m, lam(b)), R(-1));
    out.push_back(f);
  };
  if (p == 1) {
    for (auto& e : kLocalEdges) add(e[0], e[1], pconst(R(1)));
    return out;
  }
  if (p == 3) {
    for (auto& e : kLocalEdges) {
      const int ab[3][2] = {{3, 1}, {2, 2}, {1, 3}};
      for (auto& q : ab) add(e[0], e[1], multiplier({{e[0], q[0], true}, {e[1], q[1], true}}, 4));
    }
    for (auto& f : kLocalFaces) {
      const int pr[2][3] = {{f[0], f[1], f[2]}, {f[0], f[2], f[1]}};
      const int abc[3][3] = {{2, 1, 1}, {1, 2, 1}, {1, 1, 2}};
      for (auto& P : pr)
        for (auto& q : abc)
          add(P[0], P[1], multiplier({{P[0], q[0], true}, {P[1], q[1], true}, {P[2], q[2], false}}, 4));
    }
    const int inner[3][2] = {{0, 1}, {0, 2}, {0, 3}};
    for (auto& P : inner) {
      int o[2], k = 0;
      for (int v = 0; v < 4; ++v)
        if (v != P[0] && v != P[1]) o[k++] = v;
      add(P[0], P[1], multiplier({{P[0], 1, true}, {P[1], 1, true}, {o[0], 1, false}, {o[1], 1, false}}, 4));
    }
    return out;
  }
  for (auto& e : kLocalEdges) {
    add(e[0], e[1], lin(e[0], 3, -1));  // (3 l_s - 1) w_st
    add(e[0], e[1], lin(e[1], 3, -1));  // (3 l_t - 1) w_st
  }
  for (auto& f : kLocalFaces) {
    add(f[0], f[1], lin(f[2], 3, 0));   // 3 l_u w_st
    add(f[0], f[2], lin(f[1], 3, 0));   // 3 l_t w_su
  }
  return out;
}

std::vector<std::array<Poly, 6>> w2_forms(int p) {
  std::vector<std::array<Poly, 6>> out;
  auto add = [&](int face, const Poly& m) {
    int s = kLocalFaces[face][0], t = kLocalFaces[face][1], u = kLocalFaces[face][2];
    std::array<Poly, 6> f;
    // 2 (l_s X_tu + l_t X_us + l_u X_st), X_us = -X_su
    f[pair_index(t, u)] = pscale(pmul(m, lam(s)), R(2));
    f[pair_index(s, u)] = pscale(pmul(m, lam(t)), R(-2));
    f[pair_index(s, t)] = pscale(pmul(m, lam(u)), R(2));
    out.push_back(f);
  };
  if (p == 1) {
    for (int f = 0; f < 4; ++f) add(f, pconst(R(1)));
    return out;
  }
  if (p == 3) {
    const int abc[6][3] = {{3, 1, 1}, {1, 3, 1}, {1, 1, 3}, {2, 2, 1}, {2, 1, 2}, {1, 2, 2}};
    for (int f = 0; f < 4; ++f) {
      const int* F = kLocalFaces[f];
      for (auto& q : abc) add(f, multiplier({{F[0], q[0], true}, {F[1], q[1], true}, {F[2], q[2], true}}, 5));
    }
    const int abcd[4][4] = {{2, 1, 1, 1}, {1, 2, 1, 1}, {1, 1, 2, 1}, {1, 1, 1, 2}};
    for (int f = 0; f < 3; ++f) {
      const int* F = kLocalFaces[f];
      for (auto& q : abcd)
        add(f, multiplier({{F[0], q[0], true}, {F[1], q[1], true}, {F[2], q[2], true}, {f, q[3], false}}, 5));
    }
    return out;
  }
  for (int f = 0; f < 4; ++f)
    for (int v = 0; v < 3; ++v) add(f, lin(kLocalFaces[f][v], 4, -1));  // (4 l_v - 1) w_stu
  for (int i = 0; i < 3; ++i) add(i, lin(i, 4, 0));                       // 4 l_i w_(face i)
  return out;
}

std::vector<Poly> w0_forms(int p) {
  std::vector<Poly> out;
  if (p == 1) {
    for (int i = 0; i < 4; ++i) out.push_back(lam(i));
    return out;
  }
  if (p == 3) {
    for (int v = 0; v < 4; ++v) out.push_back(multiplier({{v, 3, false}}, 3));
    for (auto& e : kLocalEdges) {
      out.push_back(multiplier({{e[0], 2, false}, {e[1], 1, false}}, 3));
      out.push_back(multiplier({{e[0], 1, false}, {e[1], 2, false}}, 3));
    }
    for (auto& f : kLocalFaces) out.push_back(multiplier({{f[0], 1, false}, {f[1], 1, false}, {f[2], 1, false}}, 3));
    return out;
  }
  for (int s = 0; s < 4; ++s) out.push_back(pmul(lam(s), lin(s, 2, -1)));
  for (auto& e : kLocalEdges) out.push_back(pscale(pmul(lam(e[0]), lam(e[1])), R(4)));
  return out;
}

Vec w1_xyz(const std::array<Poly, 4>& f) {
  Vec v;
  for (int k = 0; k < 3; ++k) {
    Poly s;
    for (int a = 0; a < 4; ++a)
      if (kG[a][k] != 0) s = padd(s, f[a], R(kG[a][k]));
    v[k] = to_xyz(s);
  }
  return v;
}

Vec w2_xyz(const std::array<Poly, 6>& f) {
  Vec v;
  for (int k = 0; k < 3; ++k) {
    Poly s;
    for (int q = 0; q < 6; ++q) {
      int c = gcross(kLocalEdges[q][0], kLocalEdges[q][1])[k];
      if (c != 0) s = padd(s, f[q], R(c));
    }
    v[k] = to_xyz(s);
  }
  return v;
}

Vec grad_xyz(const Poly& p) {
  Poly x = to_xyz(p);
  return {deriv(x, 0), deriv(x, 1), deriv(x, 2)};
}

Vec curl_xyz(const Vec& v) {
  return {padd(deriv(v[2], 1), deriv(v[1], 2), R(-1)), padd(deriv(v[0], 2), deriv(v[2], 0), R(-1)),
          padd(deriv(v[1], 0), deriv(v[0], 1), R(-1))};
}

// Solve sum_j X[j][k] basis_j = target_k exactly for every k (least squares is
// unnecessary: the targets lie in the span).  Returns "" or an error.
std::string solve_in_span(const std::vector<Vec>& basis, const std::vector<Vec>& target,
                          std::vector<double>* X) {
  std::map<std::pair<int, uint32_t>, int> rowid;
  auto collect = [&](const std::vector<Vec>& vs) {
    for (auto& v : vs)
      for (int k = 0; k < 3; ++k)
        for (auto& kv : v[k].c) rowid.emplace(std::make_pair(k, kv.first), 0);
  };
  collect(basis);
  collect(target);
  int nr = 0;
  for (auto& kv : rowid) kv.second = nr++;
  int nb = (int)basis.size(), nt = (int)target.size(), nc = nb + nt;
  std::vector<Rat> A((size_t)nr * nc);
  auto put = [&](const Vec& v, int col) {
    for (int k = 0; k < 3; ++k)
      for (auto& kv : v[k].c) A[(size_t)rowid[std::make_pair(k, kv.first)] * nc + col] = kv.second;
  };
  for (int j = 0; j < nb; ++j) put(basis[j], j);
  for (int j = 0; j < nt; ++j) put(target[j], nb + j);
  // Gauss-Jordan on the basis columns
  std::vector<int> pivcol;
  int r = 0;
  for (int c = 0; c < nb && r < nr; ++c) {
    int piv = -1;
    for (int i = r; i < nr; ++i)
      if (!is_zero(A[(size_t)i * nc + c])) {
        piv = i;
        break;
      }
    if (piv < 0) return "basis is rank deficient";
    for (int j = 0; j < nc; ++j) std::swap(A[(size_t)r * nc + j], A[(size_t)piv * nc + j]);
    Rat inv = R(1) / A[(size_t)r * nc + c];
    for (int j = 0; j < nc; ++j) A[(size_t)r * nc + j] = A[(size_t)r * nc + j] * inv;
    for (int i = 0; i < nr; ++i) {
      if (i == r || is_zero(A[(size_t)i * nc + c])) continue;
      Rat f = A[(size_t)i * nc + c];
      for (int j = 0; j < nc; ++j) A[(size_t)i * nc + j] = A[(size_t)i * nc + j] - f * A[(size_t)r * nc + j];
    }
    pivcol.push_back(c);
    ++r;
  }
  if ((int)pivcol.size() != nb) return "basis is rank deficient";
  for (int i = nb; i < nr; ++i)
    for (int j = nb; j < nc; ++j)
      if (!is_zero(A[(size_t)i * nc + j])) return "target not in the span of the basis";
  X->assign((size_t)nb * nt, 0.0);
  for (int i = 0; i < nb; ++i)
    for (int k = 0; k < nt; ++k) (*X)[(size_t)i * nt + k] = to_double(A[(size_t)i * nc + nb + k]);
  return "";
}

// ------------------------------------------------------------------------
// Helpers
// ------------------------------------------------------------------------
template <class F>
void parallel_for(int64_t n, F fn) {
  unsigned hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if (n < 256 || hw == 1) {
    fn(int64_t(0), n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + hw - 1) / hw;
  for (unsigned k = 0; k < hw; ++k) {
    int64_t a = k * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    th.emplace_back([=] { fn(a, b); });
  }
  for (auto& t : th) t.join();
}

// CSR pattern of sum_t P_r(t)^T (local) P_c(t): rows R[t][i], cols Cm[t][j],
// entries where localmask[i*lc+j] and both row and column are kept.
void build_pattern(int32_t nr, int32_t nc, int32_t nt, int lr, int lc, const int32_t* Rm,
                   const int32_t* Cm, const std::vector<uint8_t>& rowkeep,
                   const std::vector<uint8_t>& colkeep, const std::vector<uint8_t>& localmask,
                   HostCSR* out) {
  std::vector<int32_t> start((size_t)nr + 1, 0);
  for (int32_t t = 0; t < nt; ++t)
    for (int i = 0; i < lr; ++i) {
      int32_t r = Rm[(size_t)t * lr + i];
      if (rowkeep[r]) start[r + 1]++;
    }
  for (int32_t r = 0; r < nr; ++r) start[r + 1] += start[r];
  std::vector<int32_t> inc((size_t)start[nr]), ploc((size_t)start[nr]);
  std::vector<int32_t> fill(start.begin(), start.end() - 1);
  for (int32_t t = 0; t < nt; ++t)
    for (int i = 0; i < lr; ++i) {
      int32_t r = Rm[(size_t)t * lr + i];
      if (!rowkeep[r]) continue;
      inc[fill[r]] = t;
      ploc[fill[r]] = i;
      fill[r]++;
    }
  std::vector<std::vector<int32_t>> rows((size_t)nr);
  parallel_for(nr, [&](int64_t a, int64_t b) {
    for (int64_t r = a; r < b; ++r) {
      auto& v = rows[r];
      for (int32_t k = start[r]; k < start[r + 1]; ++k) {
        int32_t t = inc[k], i = ploc[k];
        for (int j = 0; j < lc; ++j) {
          if (!localmask[(size_t)i * lc + j]) continue;
          int32_t c = Cm[(size_t)t * lc + j];
          if (colkeep[c]) v.push_back(c);
        }
      }
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
    }
  });
  out->n_rows = nr;
  out->n_cols = nc;
  out->rowptr.assign((size_t)nr + 1, 0);
  for (int32_t r = 0; r < nr; ++r) out->rowptr[r + 1] = out->rowptr[r] + (int32_t)rows[r].size();
  out->col.resize((size_t)out->rowptr[nr]);
  for (int32_t r = 0; r < nr; ++r) std::copy(rows[r].begin(), rows[r].end(), out->col.begin() + out->rowptr[r]);
  out->val.assign(out->col.size(), 0.0);
}

// add (or set) a local matrix into the pattern
inline void scatter(HostCSR* A, const int32_t* Rm, const int32_t* Cm, int lr, int lc, const double* Ae,
                    const std::vector<uint8_t>& rowkeep, const std::vector<uint8_t>& colkeep, bool set) {
  for (int i = 0; i < lr; ++i) {
    int32_t r = Rm[i];
    if (!rowkeep[r]) continue;
    const int32_t* b = A->col.data() + A->rowptr[r];
    const int32_t* e = A->col.data() + A->rowptr[r + 1];
    for (int j = 0; j < lc; ++j) {
      double v = Ae[(size_t)i * lc + j];
      if (v == 0.0) continue;
      int32_t c = Cm[j];
      if (!colkeep[c]) continue;
      const int32_t* p = std::lower_bound(b, e, c);
      if (p == e || *p != c) continue;  // structurally zero
      double& dst = A->val[(size_t)(p - A->col.data())];
      if (set)
        dst = v;
      else
        dst += v;
    }
  }
}

// local W0 DOF j (numbering of the order-p forms) lies on local face k (the
// face opposite vertex k): its lattice multi-index has a zero at vertex k
bool w0_on_face(int p, int j, int k) {
  if (j < 4) return j != k;
  if (p == 2) return kLocalEdges[j - 4][0] != k && kLocalEdges[j - 4][1] != k;
  if (p == 3) {
    if (j < 16) return kLocalEdges[(j - 4) / 2][0] != k && kLocalEdges[(j - 4) / 2][1] != k;
    return j - 16 == k;
  }
  return false;
}

}  // namespace

// --------------------------------------------------------------------------
std::string build_local_tables(int p, LocalTables* T) {
  T->order = p;
  T->nl0 = nloc0(p);
  T->nl1 = nloc1(p);
  T->nl2 = nloc2(p);
  auto f1 = w1_forms(p);
  auto f2 = w2_forms(p);
  auto f0 = w0_forms(p);
  if ((int)f1.size() != T->nl1 || (int)f2.size() != T->nl2 || (int)f0.size() != T->nl0)
    return "local DOF count mismatch";
  std::vector<Vec> w1v, w2v, g0v, c1v;
  for (auto& f : f1) w1v.push_back(w1_xyz(f));
  for (auto& f : f2) w2v.push_back(w2_xyz(f));
  for (auto& f : f0) g0v.push_back(grad_xyz(f));
  for (auto& v : w1v) c1v.push_back(curl_xyz(v));
  std::string err = solve_in_span(w1v, g0v, &T->Dloc);
  if (!err.empty()) return "grad map: " + err;
  err = solve_in_span(w2v, c1v, &T->Cloc);
  if (!err.empty()) return "curl map: " + err;
  int n1 = T->nl1, n2 = T->nl2;
  T->T1.assign((size_t)n1 * n1 * 16, 0.0);
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n1; ++j)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          if (f1[i][a].c.empty() || f1[j][b].c.empty()) continue;
          T->T1[(((size_t)i * n1 + j) * 4 + a) * 4 + b] = to_double(integrate_bary(pmul(f1[i][a], f1[j][b])));
        }
  T->T2.assign((size_t)n2 * n2 * 36, 0.0);
  for (int i = 0; i < n2; ++i)
    for (int j = 0; j < n2; ++j)
      for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b) {
          if (f2[i][a].c.empty() || f2[j][b].c.empty()) continue;
          T->T2[(((size_t)i * n2 + j) * 6 + a) * 6 + b] = to_double(integrate_bary(pmul(f2[i][a], f2[j][b])));
        }
  T->TF.assign((size_t)4 * n1 * n1 * 16, 0.0);
  for (int fc = 0; fc < 4; ++fc)
    for (int i = 0; i < n1; ++i)
      for (int j = 0; j < n1; ++j)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            if (f1[i][a].c.empty() || f1[j][b].c.empty()) continue;
            T->TF[((((size_t)fc * n1 + i) * n1 + j) * 4 + a) * 4 + b] =
                to_double(integrate_face(pmul(f1[i][a], f1[j][b]), fc));
          }
  T->I0.resize(T->nl0);
  for (int k = 0; k < T->nl0; ++k) T->I0[k] = to_double(integrate_bary(f0[k]));
  if (p >= 2) {
    // l_v grad l_a lies in the order-p space (p >= 2): its exact W1 coefficients
    std::vector<Vec> tg;
    for (int v = 0; v < 4; ++v)
      for (int a = 0; a < 4; ++a) {
        std::array<Poly, 4> f;
        f[a] = lam(v);
        tg.push_back(w1_xyz(f));
      }
    std::vector<double> X;
    err = solve_in_span(w1v, tg, &X);  // [nl1][16]
    if (!err.empty()) return "vector interpolation: " + err;
    T->Rv.assign(16 * (size_t)n1, 0.0);
    for (int j = 0; j < n1; ++j)
      for (int q = 0; q < 16; ++q) T->Rv[(size_t)q * n1 + j] = X[(size_t)j * 16 + q];
  }
  return "";
}

int build_model(const double* xyz, int32_t n_nodes, const int32_t* tets_in, int32_t n_tets, int p,
                HostModel* m, std::string* err, const int32_t* bface_tag) {
  if (p < 1 || p > 3) {
    *err = "order must be 1, 2 or 3";
    return 1;
  }
  if (n_nodes < 4 || n_tets < 1 || !xyz || !tets_in) {
    *err = "empty mesh";
    return 1;
  }
  LocalTables T;
  std::string e = build_local_tables(p, &T);
  if (!e.empty()) {
    *err = "local tables: " + e;
    return 1;
  }
  m->order = p;
  m->nl0 = T.nl0;
  m->nl1 = T.nl1;
  m->nl2 = T.nl2;
  m->n_nodes = n_nodes;
  m->n_tets = n_tets;
  const int32_t nt = n_tets;
  m->tets.resize((size_t)nt * 4);
  for (int32_t t = 0; t < nt; ++t) {
    int32_t v[4];
    for (int k = 0; k < 4; ++k) {
      v[k] = tets_in[(size_t)t * 4 + k];
      if (v[k] < 0 || v[k] >= n_nodes) {
        *err = "tet " + std::to_string(t) + " references a node out of range";
        return 2;
      }
    }
    std::sort(v, v + 4);
    for (int k = 0; k < 3; ++k)
      if (v[k] == v[k + 1]) {
        *err = "tet " + std::to_string(t) + " has a repeated vertex";
        return 2;
      }
    std::copy(v, v + 4, m->tets.begin() + (size_t)t * 4);
  }
  // ---- edges (sorted pairs, lexicographic) --------------------------------
  std::vector<uint64_t> ek((size_t)nt * 6);
  for (int32_t t = 0; t < nt; ++t)
    for (int k = 0; k < 6; ++k) {
      uint64_t a = (uint32_t)m->tets[(size_t)t * 4 + kLocalEdges[k][0]];
      uint64_t b = (uint32_t)m->tets[(size_t)t * 4 + kLocalEdges[k][1]];
      ek[(size_t)t * 6 + k] = (a << 32) | b;
    }
  std::vector<uint64_t> edges(ek);
  std::sort(edges.begin(), edges.end());
  edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
  m->n_edges = (int32_t)edges.size();
  std::vector<int32_t> tet_edge((size_t)nt * 6);
  for (size_t i = 0; i < ek.size(); ++i)
    tet_edge[i] = (int32_t)(std::lower_bound(edges.begin(), edges.end(), ek[i]) - edges.begin());
  // ---- faces (sorted triples, lexicographic) -------------------------------
  struct F3 {
    int32_t a, b, c;
    bool operator<(const F3& o) const {
      return a != o.a ? a < o.a : (b != o.b ? b < o.b : c < o.c);
    }
    bool operator==(const F3& o) const { return a == o.a && b == o.b && c == o.c; }
  };
  std::vector<F3> fk((size_t)nt * 4);
  for (int32_t t = 0; t < nt; ++t)
    for (int k = 0; k < 4; ++k)
      fk[(size_t)t * 4 + k] = F3{m->tets[(size_t)t * 4 + kLocalFaces[k][0]],
                                 m->tets[(size_t)t * 4 + kLocalFaces[k][1]],
                                 m->tets[(size_t)t * 4 + kLocalFaces[k][2]]};
  std::vector<F3> faces(fk);
  std::sort(faces.begin(), faces.end());
  faces.erase(std::unique(faces.begin(), faces.end()), faces.end());
  m->n_faces = (int32_t)faces.size();
  std::vector<int32_t> tet_face((size_t)nt * 4);
  for (size_t i = 0; i < fk.size(); ++i)
    tet_face[i] = (int32_t)(std::lower_bound(faces.begin(), faces.end(), fk[i]) - faces.begin());
  // ---- face owners, neighbours, boundary ----------------------------------
  std::vector<int32_t> own((size_t)m->n_faces * 2, -1), cnt(m->n_faces, 0);
  for (int32_t t = 0; t < nt; ++t)
    for (int k = 0; k < 4; ++k) {
      int32_t f = tet_face[(size_t)t * 4 + k];
      if (cnt[f] >= 2) {
        *err = "face shared by more than two tets (non-manifold mesh)";
        return 2;
      }
      own[(size_t)f * 2 + cnt[f]] = t * 4 + k;
      cnt[f]++;
    }
  m->nbr.assign((size_t)nt * 4, -1);
  std::vector<uint8_t> bface(m->n_faces, 0), bedge(m->n_edges, 0), bnode(n_nodes, 0);
  m->n_bfaces = 0;
  for (int32_t f = 0; f < m->n_faces; ++f) {
    if (cnt[f] == 2) {
      int32_t a = own[(size_t)f * 2], b = own[(size_t)f * 2 + 1];
      m->nbr[a] = ((b >> 2) << 2) | (b & 3);
      m->nbr[b] = ((a >> 2) << 2) | (a & 3);
    } else {
      bface[f] = 1;
      m->n_bfaces++;
      bnode[faces[f].a] = bnode[faces[f].b] = bnode[faces[f].c] = 1;
    }
  }
  // boundary face tags (face opposite the i-th given vertex -> sorted local
  // face): bit 1 impedance, bit 2 absorbs particles, bit 4 injects them
  std::vector<uint8_t> fimp(m->n_faces, 0), fabs_(m->n_faces, 0), finj(m->n_faces, 0);
  if (bface_tag) {
    for (int32_t t = 0; t < nt; ++t)
      for (int i = 0; i < 4; ++i) {
        const int32_t tag = bface_tag[(size_t)t * 4 + i];
        if (tag < 0 || tag > 7) {
          *err = "face tags are 0..7 (1 impedance | 2 absorb | 4 inject)";
          return 1;
        }
        if (tag == 0) continue;
        const int32_t vid = tets_in[(size_t)t * 4 + i];
        int k = 0;
        while (k < 4 && m->tets[(size_t)t * 4 + k] != vid) ++k;
        const int32_t f = tet_face[(size_t)t * 4 + k];
        if (!bface[f]) continue;
        if (tag & 1) fimp[f] = 1;
        if (tag & 2) {
          fabs_[f] = 1;
          m->nbr[(size_t)t * 4 + k] = -2;  // the walk ends on this wall
        }
        if (tag & 4) finj[f] = 1;
      }
  }
  m->n_imp_faces = 0;
  m->n_absorb_faces = 0;
  for (int32_t f = 0; f < m->n_faces; ++f) {
    m->n_imp_faces += fimp[f];
    m->n_absorb_faces += fabs_[f];
  }
  // injection faces in global order: sorted vertices, owning tet, running area
  // (0.5 |(b - a) x (c - a)|, summed one face after the other)
  m->inj_xyz.clear();
  m->inj_tet.clear();
  m->inj_cum.clear();
  {
    double run = 0.0;
    for (int32_t f = 0; f < m->n_faces; ++f) {
      if (!finj[f]) continue;
      const double* A = xyz + 3 * (size_t)faces[f].a;
      const double* B = xyz + 3 * (size_t)faces[f].b;
      const double* C = xyz + 3 * (size_t)faces[f].c;
      const double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
      const double e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
      const double cx = e1[1] * e2[2] - e1[2] * e2[1];
      const double cy = e1[2] * e2[0] - e1[0] * e2[2];
      const double cz = e1[0] * e2[1] - e1[1] * e2[0];
      run = run + 0.5 * std::sqrt((cx * cx + cy * cy) + cz * cz);
      for (const double* P : {A, B, C}) m->inj_xyz.insert(m->inj_xyz.end(), P, P + 3);
      m->inj_tet.push_back(own[(size_t)f * 2] >> 2);
      m->inj_cum.push_back(run);
    }
  }
  // boundary edges: edges of boundary faces; PEC edges: edges of PEC faces
  std::vector<uint8_t> pedge(m->n_edges, 0);
  for (int32_t t = 0; t < nt; ++t)
    for (int k = 0; k < 4; ++k) {
      const int32_t f = tet_face[(size_t)t * 4 + k];
      if (!bface[f]) continue;
      for (int j = 0; j < 6; ++j) {
        int s = kLocalEdges[j][0], u = kLocalEdges[j][1];
        if (s != k && u != k) {
          bedge[tet_edge[(size_t)t * 6 + j]] = 1;
          if (!fimp[f]) pedge[tet_edge[(size_t)t * 6 + j]] = 1;
        }
      }
    }
  // ---- DOF numbering --------------------------------------------------------
  const int32_t ne = m->n_edges, nf = m->n_faces, nn = n_nodes;
  const int l0 = m->nl0, l1 = m->nl1, l2 = m->nl2;
  m->dof0.resize((size_t)nt * l0);
  m->dof1.resize((size_t)nt * l1);
  m->dof2.resize((size_t)nt * l2);
  if (p == 1) {
    m->n1 = ne;
    m->n2 = nf;
    m->n0 = nn;
    for (int32_t t = 0; t < nt; ++t) {
      for (int k = 0; k < 6; ++k) m->dof1[(size_t)t * 6 + k] = tet_edge[(size_t)t * 6 + k];
      for (int k = 0; k < 4; ++k) m->dof2[(size_t)t * 4 + k] = tet_face[(size_t)t * 4 + k];
      for (int k = 0; k < 4; ++k) m->dof0[(size_t)t * 4 + k] = m->tets[(size_t)t * 4 + k];
    }
    m->pec1.assign(pedge.begin(), pedge.end());
    m->bnd0.assign(bnode.begin(), bnode.end());
  } else if (p == 3) {
    // W1: 3 per edge, 6 per face, 3 per tet; W2: 6 per face, 12 per tet;
    // W0: nodes, 2 per edge, 1 per face (the local order of the forms above)
    if ((int64_t)3 * ne + 6 * (int64_t)nf + 3 * (int64_t)nt > INT32_MAX ||
        (int64_t)6 * nf + 12 * (int64_t)nt > INT32_MAX) {
      *err = "mesh too large for 32-bit DOF ids";
      return 1;
    }
    m->n1 = 3 * ne + 6 * nf + 3 * nt;
    m->n2 = 6 * nf + 12 * nt;
    m->n0 = nn + 2 * ne + nf;
    for (int32_t t = 0; t < nt; ++t) {
      int32_t* d1t = &m->dof1[(size_t)t * 45];
      for (int k = 0; k < 6; ++k)
        for (int v = 0; v < 3; ++v) d1t[3 * k + v] = 3 * tet_edge[(size_t)t * 6 + k] + v;
      for (int k = 0; k < 4; ++k)
        for (int v = 0; v < 6; ++v) d1t[18 + 6 * k + v] = 3 * ne + 6 * tet_face[(size_t)t * 4 + k] + v;
      for (int v = 0; v < 3; ++v) d1t[42 + v] = 3 * ne + 6 * nf + 3 * t + v;
      int32_t* d2t = &m->dof2[(size_t)t * 36];
      for (int k = 0; k < 4; ++k)
        for (int v = 0; v < 6; ++v) d2t[6 * k + v] = 6 * tet_face[(size_t)t * 4 + k] + v;
      for (int v = 0; v < 12; ++v) d2t[24 + v] = 6 * nf + 12 * t + v;
      int32_t* d0t = &m->dof0[(size_t)t * 20];
      for (int k = 0; k < 4; ++k) d0t[k] = m->tets[(size_t)t * 4 + k];
      for (int k = 0; k < 6; ++k)
        for (int v = 0; v < 2; ++v) d0t[4 + 2 * k + v] = nn + 2 * tet_edge[(size_t)t * 6 + k] + v;
      for (int k = 0; k < 4; ++k) d0t[16 + k] = nn + 2 * ne + tet_face[(size_t)t * 4 + k];
    }
    m->pec1.assign(m->n1, 0);
    for (int32_t e2 = 0; e2 < ne; ++e2)
      if (pedge[e2])
        for (int v = 0; v < 3; ++v) m->pec1[3 * e2 + v] = 1;
    for (int32_t f = 0; f < nf; ++f)
      if (bface[f] && !fimp[f])
        for (int v = 0; v < 6; ++v) m->pec1[3 * ne + 6 * f + v] = 1;
    m->bnd0.assign(m->n0, 0);
    for (int32_t v = 0; v < nn; ++v) m->bnd0[v] = bnode[v];
    for (int32_t e2 = 0; e2 < ne; ++e2) m->bnd0[nn + 2 * e2] = m->bnd0[nn + 2 * e2 + 1] = bedge[e2];
    for (int32_t f = 0; f < nf; ++f) m->bnd0[nn + 2 * ne + f] = bface[f];
  } else {
    if ((int64_t)2 * ne + 2 * (int64_t)nf > INT32_MAX || (int64_t)3 * nf + 3 * (int64_t)nt > INT32_MAX) {
      *err = "mesh too large for 32-bit DOF ids";
      return 1;
    }
    m->n1 = 2 * ne + 2 * nf;
    m->n2 = 3 * nf + 3 * nt;
    m->n0 = nn + ne;
    for (int32_t t = 0; t < nt; ++t) {
      for (int k = 0; k < 6; ++k) {
        m->dof1[(size_t)t * 20 + 2 * k] = 2 * tet_edge[(size_t)t * 6 + k];
        m->dof1[(size_t)t * 20 + 2 * k + 1] = 2 * tet_edge[(size_t)t * 6 + k] + 1;
      }
      for (int k = 0; k < 4; ++k) {
        m->dof1[(size_t)t * 20 + 12 + 2 * k] = 2 * ne + 2 * tet_face[(size_t)t * 4 + k];
        m->dof1[(size_t)t * 20 + 13 + 2 * k] = 2 * ne + 2 * tet_face[(size_t)t * 4 + k] + 1;
      }
      for (int k = 0; k < 4; ++k)
        for (int v = 0; v < 3; ++v) m->dof2[(size_t)t * 15 + 3 * k + v] = 3 * tet_face[(size_t)t * 4 + k] + v;
      for (int i = 0; i < 3; ++i) m->dof2[(size_t)t * 15 + 12 + i] = 3 * nf + 3 * t + i;
      for (int k = 0; k < 4; ++k) m->dof0[(size_t)t * 10 + k] = m->tets[(size_t)t * 4 + k];
      for (int k = 0; k < 6; ++k) m->dof0[(size_t)t * 10 + 4 + k] = nn + tet_edge[(size_t)t * 6 + k];
    }
    m->pec1.assign(m->n1, 0);
    for (int32_t e2 = 0; e2 < ne; ++e2)
      if (pedge[e2]) m->pec1[2 * e2] = m->pec1[2 * e2 + 1] = 1;
    for (int32_t f = 0; f < nf; ++f)
      if (bface[f] && !fimp[f]) m->pec1[2 * ne + 2 * f] = m->pec1[2 * ne + 2 * f + 1] = 1;
    m->bnd0.assign(m->n0, 0);
    for (int32_t v = 0; v < nn; ++v) m->bnd0[v] = bnode[v];
    for (int32_t e2 = 0; e2 < ne; ++e2) m->bnd0[nn + e2] = bedge[e2];
  }
  // ---- barycentric maps (fixed operation order, no contraction) -----------
  m->geom.resize((size_t)nt * 16);
  m->vol.resize(nt);
  double hmax = 0.0;
  for (int32_t t = 0; t < nt; ++t) {
    const double* P0 = xyz + 3 * (size_t)m->tets[(size_t)t * 4 + 0];
    double e1[3], e2v[3], e3[3];
    for (int k = 0; k < 3; ++k) {
      e1[k] = xyz[3 * (size_t)m->tets[(size_t)t * 4 + 1] + k] - P0[k];
      e2v[k] = xyz[3 * (size_t)m->tets[(size_t)t * 4 + 2] + k] - P0[k];
      e3[k] = xyz[3 * (size_t)m->tets[(size_t)t * 4 + 3] + k] - P0[k];
      hmax = std::max(hmax, std::max(std::fabs(e1[k]), std::max(std::fabs(e2v[k]), std::fabs(e3[k]))));
    }
    auto cross = [](const double* a, const double* b, double* o) {
      o[0] = a[1] * b[2] - a[2] * b[1];
      o[1] = a[2] * b[0] - a[0] * b[2];
      o[2] = a[0] * b[1] - a[1] * b[0];
    };
    double n1v[3], n2v[3], n3v[3];
    cross(e2v, e3, n1v);
    cross(e3, e1, n2v);
    cross(e1, e2v, n3v);
    double det = (e1[0] * n1v[0] + e1[1] * n1v[1]) + e1[2] * n1v[2];
    double len = std::max(std::fabs(e1[0]) + std::fabs(e1[1]) + std::fabs(e1[2]),
                          std::max(std::fabs(e2v[0]) + std::fabs(e2v[1]) + std::fabs(e2v[2]),
                                   std::fabs(e3[0]) + std::fabs(e3[1]) + std::fabs(e3[2])));
    if (!(std::fabs(det) > 1e-12 * len * len * len)) {
      *err = "tet " + std::to_string(t) + " is degenerate (zero volume)";
      return 2;
    }
    double* G = &m->geom[(size_t)t * 16];
    for (int k = 0; k < 3; ++k) {
      G[3 + k] = n1v[k] / det;
      G[6 + k] = n2v[k] / det;
      G[9 + k] = n3v[k] / det;
    }
    for (int k = 0; k < 3; ++k) G[k] = -((G[3 + k] + G[6 + k]) + G[9 + k]);
    double* c = G + 12;
    for (int i = 1; i < 4; ++i)
      c[i] = -((G[3 * i] * P0[0] + G[3 * i + 1] * P0[1]) + G[3 * i + 2] * P0[2]);
    c[0] = 1.0 - ((c[1] + c[2]) + c[3]);
    m->vol[t] = std::fabs(det) / 6.0;
  }
  (void)hmax;
  // ---- matrices --------------------------------------------------------------
  std::vector<uint8_t> free1(m->n1), all1(m->n1, 1), all2(m->n2, 1), int0(m->n0), all0(m->n0, 1);
  for (int32_t i = 0; i < m->n1; ++i) free1[i] = !m->pec1[i];
  for (int32_t i = 0; i < m->n0; ++i) int0[i] = !m->bnd0[i];
  std::vector<uint8_t> full11((size_t)l1 * l1, 1), full12((size_t)l1 * l2, 1), full22((size_t)l2 * l2, 1),
      full00((size_t)l0 * l0, 1), maskC((size_t)l2 * l1), maskD((size_t)l1 * l0), maskDT((size_t)l0 * l1);
  for (int f = 0; f < l2; ++f)
    for (int j = 0; j < l1; ++j) maskC[(size_t)f * l1 + j] = T.Cloc[(size_t)f * l1 + j] != 0.0;
  for (int i = 0; i < l1; ++i)
    for (int k = 0; k < l0; ++k) {
      maskD[(size_t)i * l0 + k] = T.Dloc[(size_t)i * l0 + k] != 0.0;
      maskDT[(size_t)k * l1 + i] = maskD[(size_t)i * l0 + k];
    }
  const int32_t* d1 = m->dof1.data();
  const int32_t* d2 = m->dof2.data();
  const int32_t* d0 = m->dof0.data();
  build_pattern(m->n1, m->n1, nt, l1, l1, d1, d1, free1, free1, full11, &m->M);
  m->K = m->M;
  build_pattern(m->n1, m->n2, nt, l1, l2, d1, d2, free1, all2, full12, &m->Q);
  build_pattern(m->n2, m->n2, nt, l2, l2, d2, d2, all2, all2, full22, &m->M2);
  build_pattern(m->n2, m->n1, nt, l2, l1, d2, d1, all2, free1, maskC, &m->C);
  build_pattern(m->n1, m->n0, nt, l1, l0, d1, d0, all1, int0, maskD, &m->D);
  build_pattern(m->n0, m->n1, nt, l0, l1, d0, d1, all0, all1, maskDT, &m->DT);
  build_pattern(m->n0, m->n0, nt, l0, l0, d0, d0, int0, int0, full00, &m->L);
  // With impedance faces the W1 DOFs on them are free, so the gradients of the
  // W0 functions that live there are in the near-kernel of K too: the
  // preconditioner's gradient space is every W0 DOF off the PEC faces
  // (aux0), its Laplacian D_a^T (M + c_I I) D_a (the I part depends on dt).
  std::vector<uint8_t> aux0;
  if (m->n_imp_faces > 0) {
    aux0.assign(m->n0, 1);
    for (int32_t t = 0; t < nt; ++t)
      for (int k = 0; k < 4; ++k) {
        const int32_t f = tet_face[(size_t)t * 4 + k];
        if (!bface[f] || fimp[f]) continue;
        for (int j = 0; j < l0; ++j)
          if (w0_on_face(p, j, k)) aux0[d0[(size_t)t * l0 + j]] = 0;
      }
    build_pattern(m->n1, m->n0, nt, l1, l0, d1, d0, free1, aux0, maskD, &m->DA);
    build_pattern(m->n0, m->n1, nt, l0, l1, d0, d1, aux0, free1, maskDT, &m->DAT);
    build_pattern(m->n0, m->n0, nt, l0, l0, d0, d0, aux0, aux0, full00, &m->LA);
  }
  m->load0.assign(m->n0, 0.0);

  std::vector<double> DT_loc((size_t)l0 * l1);
  for (int i = 0; i < l1; ++i)
    for (int k = 0; k < l0; ++k) DT_loc[(size_t)k * l1 + i] = T.Dloc[(size_t)i * l0 + k];

  const int CH = 4096;
  const size_t sM = (size_t)l1 * l1, sQ = (size_t)l1 * l2, sM2 = (size_t)l2 * l2, sL = (size_t)l0 * l0;
  std::vector<double> bM(CH * sM), bK(CH * sM), bQ(CH * sQ), bM2(CH * sM2), bL(CH * sL), bW(CH * l0);
  for (int32_t t0 = 0; t0 < nt; t0 += CH) {
    int32_t nc = std::min(CH, nt - t0);
    parallel_for(nc, [&](int64_t a, int64_t b) {
      std::vector<double> M2e(sM2), tmp((size_t)l1 * l2), tmp2((size_t)l0 * l1);
      for (int64_t q = a; q < b; ++q) {
        int32_t t = t0 + (int32_t)q;
        const double* g = &m->geom[(size_t)t * 16];
        double G[4][4];
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) G[i][j] = g[3 * i] * g[3 * j] + g[3 * i + 1] * g[3 * j + 1] + g[3 * i + 2] * g[3 * j + 2];
        double H[6][6];
        for (int P = 0; P < 6; ++P)
          for (int Qi = 0; Qi < 6; ++Qi) {
            int a1 = kLocalEdges[P][0], b1 = kLocalEdges[P][1], c1 = kLocalEdges[Qi][0], e1 = kLocalEdges[Qi][1];
            H[P][Qi] = G[a1][c1] * G[b1][e1] - G[a1][e1] * G[b1][c1];
          }
        double v6 = 6.0 * m->vol[t];
        double* Me = &bM[q * sM];
        for (int i = 0; i < l1; ++i)
          for (int j = 0; j < l1; ++j) {
            const double* tt = &T.T1[((size_t)i * l1 + j) * 16];
            double s = 0.0;
            for (int x = 0; x < 4; ++x)
              for (int y = 0; y < 4; ++y) s += G[x][y] * tt[x * 4 + y];
            Me[(size_t)i * l1 + j] = kEps0 * v6 * s;
          }
        for (int i = 0; i < l2; ++i)
          for (int j = 0; j < l2; ++j) {
            const double* tt = &T.T2[((size_t)i * l2 + j) * 36];
            double s = 0.0;
            for (int x = 0; x < 6; ++x)
              for (int y = 0; y < 6; ++y) s += H[x][y] * tt[x * 6 + y];
            M2e[(size_t)i * l2 + j] = v6 * s / kMu0;
          }
        std::copy(M2e.begin(), M2e.end(), &bM2[q * sM2]);
        // Q_e = Cloc^T M2e  (l1 x l2);  K_e = Q_e Cloc (l1 x l1)
        double* Qe = &bQ[q * sQ];
        for (int i = 0; i < l1; ++i)
          for (int h = 0; h < l2; ++h) {
            double s = 0.0;
            for (int f = 0; f < l2; ++f) s += T.Cloc[(size_t)f * l1 + i] * M2e[(size_t)f * l2 + h];
            Qe[(size_t)i * l2 + h] = s;
          }
        double* Ke = &bK[q * sM];
        for (int i = 0; i < l1; ++i)
          for (int j = 0; j < l1; ++j) {
            double s = 0.0;
            for (int h = 0; h < l2; ++h) s += Qe[(size_t)i * l2 + h] * T.Cloc[(size_t)h * l1 + j];
            Ke[(size_t)i * l1 + j] = s;
          }
        // L_e = Dloc^T M_e Dloc
        for (int k = 0; k < l0; ++k)
          for (int j = 0; j < l1; ++j) {
            double s = 0.0;
            for (int i = 0; i < l1; ++i) s += DT_loc[(size_t)k * l1 + i] * Me[(size_t)i * l1 + j];
            tmp2[(size_t)k * l1 + j] = s;
          }
        double* Le = &bL[q * sL];
        for (int k = 0; k < l0; ++k)
          for (int n = 0; n < l0; ++n) {
            double s = 0.0;
            for (int j = 0; j < l1; ++j) s += tmp2[(size_t)k * l1 + j] * T.Dloc[(size_t)j * l0 + n];
            Le[(size_t)k * l0 + n] = s;
          }
        for (int k = 0; k < l0; ++k) bW[q * l0 + k] = v6 * T.I0[k];
      }
    });
    for (int32_t q = 0; q < nc; ++q) {
      int32_t t = t0 + q;
      const int32_t* r1 = d1 + (size_t)t * l1;
      const int32_t* r2 = d2 + (size_t)t * l2;
      const int32_t* r0 = d0 + (size_t)t * l0;
      scatter(&m->M, r1, r1, l1, l1, &bM[q * sM], free1, free1, false);
      scatter(&m->K, r1, r1, l1, l1, &bK[q * sM], free1, free1, false);
      scatter(&m->Q, r1, r2, l1, l2, &bQ[q * sQ], free1, all2, false);
      scatter(&m->M2, r2, r2, l2, l2, &bM2[q * sM2], all2, all2, false);
      scatter(&m->L, r0, r0, l0, l0, &bL[q * sL], int0, int0, false);
      scatter(&m->C, r2, r1, l2, l1, T.Cloc.data(), all2, free1, true);
      scatter(&m->D, r1, r0, l1, l0, T.Dloc.data(), all1, int0, true);
      scatter(&m->DT, r0, r1, l0, l1, DT_loc.data(), all0, all1, true);
      if (!aux0.empty()) {
        scatter(&m->LA, r0, r0, l0, l0, &bL[q * sL], aux0, aux0, false);
        scatter(&m->DA, r1, r0, l1, l0, T.Dloc.data(), free1, aux0, true);
        scatter(&m->DAT, r0, r1, l0, l1, DT_loc.data(), aux0, free1, true);
      }
      for (int k = 0; k < l0; ++k) m->load0[r0[k]] += bW[q * l0 + k];
    }
  }
  // ---- surface impedance matrix Y0 <n x W1_i, n x W1_j> over the impedance
  // faces, on M's pattern: the tangential part of grad l_x on the face opposite
  // local vertex i is grad l_x - (grad l_x . n) n with n = grad l_i / |grad l_i|
  m->Ival.clear();
  m->LAI.clear();
  if (m->n_imp_faces > 0) {
    HostCSR Ih = m->M;
    std::fill(Ih.val.begin(), Ih.val.end(), 0.0);
    HostCSR LIh = m->LA;  // D_a^T I D_a on the pattern of L_a
    std::fill(LIh.val.begin(), LIh.val.end(), 0.0);
    std::vector<double> tmpI((size_t)l0 * l1), LIe((size_t)l0 * l0);
    const double Y0 = std::sqrt(kEps0 / kMu0);
    std::vector<double> Ie((size_t)l1 * l1);
    for (int32_t t = 0; t < nt; ++t)
      for (int i = 0; i < 4; ++i) {
        if (!fimp[tet_face[(size_t)t * 4 + i]]) continue;
        const double* g = &m->geom[(size_t)t * 16];
        const double gn = std::sqrt(g[3 * i] * g[3 * i] + g[3 * i + 1] * g[3 * i + 1] + g[3 * i + 2] * g[3 * i + 2]);
        const double nv[3] = {g[3 * i] / gn, g[3 * i + 1] / gn, g[3 * i + 2] / gn};
        double Gt[4][4];
        for (int x = 0; x < 4; ++x)
          for (int y = 0; y < 4; ++y) {
            const double* gx = g + 3 * x;
            const double* gy = g + 3 * y;
            const double dxy = gx[0] * gy[0] + gx[1] * gy[1] + gx[2] * gy[2];
            const double dxn = gx[0] * nv[0] + gx[1] * nv[1] + gx[2] * nv[2];
            const double dyn = gy[0] * nv[0] + gy[1] * nv[1] + gy[2] * nv[2];
            Gt[x][y] = dxy - dxn * dyn;
          }
        int fv[3], q = 0;
        for (int k = 0; k < 4; ++k)
          if (k != i) fv[q++] = m->tets[(size_t)t * 4 + k];
        double u[3], w[3];
        for (int k = 0; k < 3; ++k) {
          u[k] = xyz[3 * (size_t)fv[1] + k] - xyz[3 * (size_t)fv[0] + k];
          w[k] = xyz[3 * (size_t)fv[2] + k] - xyz[3 * (size_t)fv[0] + k];
        }
        const double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2], cz = u[0] * w[1] - u[1] * w[0];
        const double area2 = std::sqrt(cx * cx + cy * cy + cz * cz);
        for (int a = 0; a < l1; ++a)
          for (int b = 0; b < l1; ++b) {
            const double* tf = &T.TF[((((size_t)i * l1 + a) * l1 + b) * 4) * 4];
            double sum = 0.0;
            for (int x = 0; x < 4; ++x)
              for (int y = 0; y < 4; ++y) sum += Gt[x][y] * tf[x * 4 + y];
            Ie[(size_t)a * l1 + b] = Y0 * area2 * sum;
          }
        scatter(&Ih, d1 + (size_t)t * l1, d1 + (size_t)t * l1, l1, l1, Ie.data(), free1, free1, false);
        for (int k = 0; k < l0; ++k)
          for (int b = 0; b < l1; ++b) {
            double sacc = 0.0;
            for (int a = 0; a < l1; ++a) sacc += DT_loc[(size_t)k * l1 + a] * Ie[(size_t)a * l1 + b];
            tmpI[(size_t)k * l1 + b] = sacc;
          }
        for (int k = 0; k < l0; ++k)
          for (int n = 0; n < l0; ++n) {
            double sacc = 0.0;
            for (int b = 0; b < l1; ++b) sacc += tmpI[(size_t)k * l1 + b] * T.Dloc[(size_t)b * l0 + n];
            LIe[(size_t)k * l0 + n] = sacc;
          }
        scatter(&LIh, d0 + (size_t)t * l0, d0 + (size_t)t * l0, l0, l0, LIe.data(), aux0, aux0, false);
      }
    m->Ival = Ih.val;
    m->LAI = LIh.val;
  }
  // ---- vector nodal interpolation Pi (auxiliary space of the preconditioner)
  {
    const int lc = 12;  // (local vertex, component)
    std::vector<int32_t> colmap((size_t)nt * lc);
    for (int32_t t = 0; t < nt; ++t)
      for (int v = 0; v < 4; ++v)
        for (int c = 0; c < 3; ++c) colmap[(size_t)t * lc + 3 * v + c] = 3 * m->tets[(size_t)t * 4 + v] + c;
    std::vector<uint8_t> maskP((size_t)l1 * lc, 0), allv(3 * (size_t)nn, 1);
    for (int j = 0; j < l1; ++j)
      for (int v = 0; v < 4; ++v)
        for (int c = 0; c < 3; ++c) {
          bool nz = false;
          if (p == 1) {
            nz = kLocalEdges[j][0] == v || kLocalEdges[j][1] == v;
          } else {
            for (int a = 0; a < 4; ++a) nz = nz || T.Rv[(size_t)(4 * v + a) * l1 + j] != 0.0;
          }
          maskP[(size_t)j * lc + 3 * v + c] = nz;
        }
    build_pattern(m->n1, 3 * nn, nt, l1, lc, d1, colmap.data(), free1, allv, maskP, &m->Pi);
    std::vector<double> loc((size_t)l1 * lc);
    for (int32_t t = 0; t < nt; ++t) {
      const int32_t* tv = &m->tets[(size_t)t * 4];
      std::fill(loc.begin(), loc.end(), 0.0);
      for (int j = 0; j < l1; ++j)
        for (int v = 0; v < 4; ++v)
          for (int c = 0; c < 3; ++c) {
            double val = 0.0;
            if (p == 1) {
              int s0 = kLocalEdges[j][0], s1 = kLocalEdges[j][1];
              if (s0 == v || s1 == v) val = 0.5 * (xyz[3 * (size_t)tv[s1] + c] - xyz[3 * (size_t)tv[s0] + c]);
            } else {
              for (int a = 0; a < 4; ++a) val += xyz[3 * (size_t)tv[a] + c] * T.Rv[(size_t)(4 * v + a) * l1 + j];
            }
            loc[(size_t)j * lc + 3 * v + c] = val;
          }
      scatter(&m->Pi, d1 + (size_t)t * l1, colmap.data() + (size_t)t * lc, l1, lc, loc.data(), free1, allv, true);
    }
    // transpose
    HostCSR& P = m->Pi;
    HostCSR& PT = m->PiT;
    PT.n_rows = P.n_cols;
    PT.n_cols = P.n_rows;
    PT.rowptr.assign((size_t)PT.n_rows + 1, 0);
    for (int32_t c : P.col) PT.rowptr[c + 1]++;
    for (int32_t r = 0; r < PT.n_rows; ++r) PT.rowptr[r + 1] += PT.rowptr[r];
    PT.col.resize(P.col.size());
    PT.val.resize(P.col.size());
    std::vector<int32_t> fillp(PT.rowptr.begin(), PT.rowptr.end() - 1);
    for (int32_t r = 0; r < P.n_rows; ++r)
      for (int32_t k = P.rowptr[r]; k < P.rowptr[r + 1]; ++k) {
        int32_t c = P.col[k];
        PT.col[fillp[c]] = r;
        PT.val[fillp[c]] = P.val[k];
        fillp[c]++;
      }
    // Galerkin products V_M = Pi^T M Pi and V_K = Pi^T K Pi (one pattern), one
    // row of Pi^T at a time with a dense accumulator; their diagonals too
    const int32_t nv = PT.n_rows;
    std::vector<std::vector<int32_t>> vcol((size_t)nv);
    std::vector<std::vector<double>> vm((size_t)nv), vk((size_t)nv);
    parallel_for(nv, [&](int64_t a, int64_t b) {
      std::vector<double> am((size_t)nv, 0.0), ak((size_t)nv, 0.0);
      std::vector<uint8_t> seen((size_t)nv, 0);
      std::vector<int32_t> cols;
      for (int64_t c = a; c < b; ++c) {
        cols.clear();
        for (int32_t k = PT.rowptr[c]; k < PT.rowptr[c + 1]; ++k) {
          const int32_t i = PT.col[k];
          const double pi = PT.val[k];
          for (int32_t q = m->M.rowptr[i]; q < m->M.rowptr[i + 1]; ++q) {
            const int32_t j = m->M.col[q];
            const double wm = pi * m->M.val[q], wk = pi * m->K.val[q];
            for (int32_t r = P.rowptr[j]; r < P.rowptr[j + 1]; ++r) {
              const int32_t d = P.col[r];
              if (!seen[d]) {
                seen[d] = 1;
                cols.push_back(d);
              }
              am[d] += wm * P.val[r];
              ak[d] += wk * P.val[r];
            }
          }
        }
        std::sort(cols.begin(), cols.end());
        vcol[c] = cols;
        vm[c].resize(cols.size());
        vk[c].resize(cols.size());
        for (size_t e = 0; e < cols.size(); ++e) {
          const int32_t d = cols[e];
          vm[c][e] = am[d];
          vk[c][e] = ak[d];
          am[d] = ak[d] = 0.0;
          seen[d] = 0;
        }
      }
    });
    m->VM.n_rows = m->VM.n_cols = nv;
    m->VM.rowptr.assign((size_t)nv + 1, 0);
    for (int32_t c = 0; c < nv; ++c) m->VM.rowptr[c + 1] = m->VM.rowptr[c] + (int32_t)vcol[c].size();
    m->VM.col.reserve((size_t)m->VM.rowptr[nv]);
    m->VM.val.reserve((size_t)m->VM.rowptr[nv]);
    m->VK.reserve((size_t)m->VM.rowptr[nv]);
    m->dvM.assign(nv, 0.0);
    m->dvK.assign(nv, 0.0);
    for (int32_t c = 0; c < nv; ++c) {
      for (size_t e = 0; e < vcol[c].size(); ++e) {
        if (vcol[c][e] == c) {
          m->dvM[c] = vm[c][e];
          m->dvK[c] = vk[c][e];
        }
        m->VM.col.push_back(vcol[c][e]);
        m->VM.val.push_back(vm[c][e]);
        m->VK.push_back(vk[c][e]);
      }
    }
  }
  return 0;
}


// --------------------------------------------------------------------------
// Impressed-field projection (Section III-C, eq. conB)
// --------------------------------------------------------------------------
namespace {

// n-point Gauss-Legendre rule mapped to [0, 1]: Newton's iteration on P_n
// (three-term recurrence k P_k = (2k-1) x P_{k-1} - (k-1) P_{k-2}) from the
// guesses cos(pi (i + 3/4) / (n + 1/2)); weights 2 / ((1 - x^2) P_n'(x)^2)
void gauss_legendre01(int n, std::vector<double>* x, std::vector<double>* w) {
  x->assign(n, 0.0);
  w->assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) <= 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    (*x)[n - 1 - i] = 0.5 * (z + 1.0);
    (*w)[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Cholesky inverse of a dense SPD matrix (row-major, in place); false if not SPD
bool spd_inverse(int n, std::vector<double>& A) {
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > 0.0)) return false;
    L[(size_t)j * n + j] = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double s = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
    }
  }
  // columns of L^-T L^-1
  std::vector<double> col(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {  // forward: L y = e_c
      double s = i == c ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * col[k];
      col[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {  // backward: L^T x = y
      double s = col[i];
      for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * col[k];
      col[i] = s / L[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) A[(size_t)i * n + c] = col[i];
  }
  return true;
}

// W3 of order p: P^_a(l0) P^_b(l1) P^_c(l2) P^_d(l3), a, b, c, d >= 1,
// a + b + c + d = p + 3, scale p + 3 (the volume form's constant factor left out)
std::vector<Poly> w3_forms(int p) {
  const int n = p + 3;
  std::vector<Poly> out;
  for (int a = 1; a < n; ++a)
    for (int b = 1; b < n - a; ++b)
      for (int c = 1; c < n - a - b; ++c) {
        const int d = n - a - b - c;
        if (d < 1) continue;
        out.push_back(multiplier({{0, a, true}, {1, b, true}, {2, c, true}, {3, d, true}}, n));
      }
  return out;
}

// dense rows -> CSR (entries exactly zero dropped)
void rows_to_csr(int32_t n_rows, int32_t n_cols, std::vector<std::vector<std::pair<int32_t, double>>>& rows,
                 HostCSR* A) {
  A->n_rows = n_rows;
  A->n_cols = n_cols;
  A->rowptr.assign((size_t)n_rows + 1, 0);
  A->col.clear();
  A->val.clear();
  for (int32_t r = 0; r < n_rows; ++r) {
    auto& v = rows[r];
    std::sort(v.begin(), v.end());
    for (auto& e : v)
      if (e.second != 0.0) {
        A->col.push_back(e.first);
        A->val.push_back(e.second);
      }
    A->rowptr[r + 1] = (int32_t)A->col.size();
  }
}

}  // namespace

void projection_rule(int p, ProjModel* out) {
  std::vector<double> x, w;
  const int nq1 = p + 3;
  gauss_legendre01(nq1, &x, &w);
  out->nq = nq1 * nq1 * nq1;
  out->qlam.clear();
  out->qw.clear();
  for (int a = 0; a < nq1; ++a)
    for (int b = 0; b < nq1; ++b)
      for (int c = 0; c < nq1; ++c) {
        const double u = x[a], v = x[b], s = x[c];
        const double px = u, py = (1.0 - u) * v, pz = (1.0 - u) * (1.0 - v) * s;
        out->qlam.insert(out->qlam.end(), {1.0 - px - py - pz, px, py, pz});
        out->qw.push_back(w[a] * w[b] * w[c] * ((1.0 - u) * (1.0 - u) * (1.0 - v)));
      }
}

void div_table(int p, std::vector<double>* Dref, int* n3_out) {
  const int nl2 = nloc2(p);
  auto f3 = w3_forms(p);
  auto f2 = w2_forms(p);
  const int n3 = (int)f3.size();
  Dref->assign((size_t)n3 * nl2, 0.0);
  std::vector<Poly> div2;
  for (auto& f : f2) {
    Vec v = w2_xyz(f);
    div2.push_back(padd(padd(deriv(v[0], 0), deriv(v[1], 1)), deriv(v[2], 2)));
  }
  for (int i = 0; i < n3; ++i) {
    // int over the reference tet of x^a y^b z^c = a! b! c! / (a+b+c+3)!: the
    // barycentric formula with the fourth exponent 0
    Poly w = to_xyz(f3[i]);
    for (int j = 0; j < nl2; ++j) (*Dref)[(size_t)i * nl2 + j] = to_double(integrate_bary(pmul(w, div2[j])));
  }
  *n3_out = n3;
}

std::string build_projection(int p, int32_t nt, int32_t nf, int32_t n2, const double* xyz,
                             const int32_t* tets, const int32_t* dof2, const HostCSR& M2, ProjModel* out) {
  const int nl2 = nloc2(p);
  int n3 = 0;
  std::vector<double> Dref;
  div_table(p, &Dref, &n3);
  out->n3 = n3;
  projection_rule(p, out);
  // per-tet orientation and volume: sign(det J) and 6|V|, J = [x1-x0, x2-x0, x3-x0]
  std::vector<double> sgn(nt);
  out->vol6.assign(nt, 0.0);
  for (int32_t t = 0; t < nt; ++t) {
    const double* x0 = xyz + 3 * (size_t)tets[4 * (size_t)t];
    double e[3][3];
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) e[k][d] = xyz[3 * (size_t)tets[4 * (size_t)t + k + 1] + d] - x0[d];
    const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                       e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                       e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
    if (det == 0.0) return "degenerate tet " + std::to_string(t);
    sgn[t] = det > 0.0 ? 1.0 : -1.0;
    out->vol6[t] = std::fabs(det);
  }
  // [~div]: the physical divergence of W2 (contravariant Piola map) is the
  // reference one over det J, so int_T W3 div W2 = sign(det J) Dref
  const int32_t N3 = n3 * nt;
  {
    std::vector<std::vector<std::pair<int32_t, double>>> rows(N3), rowsT(n2);
    for (int32_t t = 0; t < nt; ++t)
      for (int i = 0; i < n3; ++i)
        for (int j = 0; j < nl2; ++j) {
          const double v = sgn[t] * Dref[(size_t)i * nl2 + j];
          if (v == 0.0) continue;
          const int32_t r = t * n3 + i, c = dof2[(size_t)t * nl2 + j];
          rows[r].push_back({c, v});
          rowsT[c].push_back({r, v});
        }
    rows_to_csr(N3, n2, rows, &out->Dv);
    rows_to_csr(n2, N3, rowsT, &out->DvT);
  }
  // block-Jacobi inverse of M2: the W2 DOFs of one face, and the interior DOFs of one tet
  const int nfg = p * (p + 1) / 2, nint = nl2 - 4 * nfg;
  const int32_t ngroups = nf + (nint > 0 ? nt : 0);
  std::vector<std::vector<double>> ginv(ngroups);
  auto group_base = [&](int32_t g) { return g < nf ? nfg * g : nfg * nf + nint * (g - nf); };
  auto group_size = [&](int32_t g) { return g < nf ? nfg : nint; };
  {
    std::vector<std::vector<std::pair<int32_t, double>>> rows(n2);
    for (int32_t g = 0; g < ngroups; ++g) {
      const int32_t b0 = group_base(g);
      const int gs = group_size(g);
      std::vector<double> B((size_t)gs * gs, 0.0);
      for (int a = 0; a < gs; ++a) {
        const int32_t r = b0 + a;
        for (int32_t k = M2.rowptr[r]; k < M2.rowptr[r + 1]; ++k) {
          const int32_t c = M2.col[k];
          if (c >= b0 && c < b0 + gs) B[(size_t)a * gs + (c - b0)] = M2.val[k];
        }
      }
      if (!spd_inverse(gs, B)) return "a diagonal block of the W2 mass matrix is not positive definite";
      for (int a = 0; a < gs; ++a)
        for (int c = 0; c < gs; ++c) rows[b0 + a].push_back({b0 + c, B[(size_t)a * gs + c]});
      ginv[g] = std::move(B);
    }
    rows_to_csr(n2, n2, rows, &out->Bm);
  }
  // per-tet block inverse of Dv Bm Dv^T (the tet's W2 DOFs cover whole groups)
  {
    std::vector<std::vector<std::pair<int32_t, double>>> rows(N3);
    std::vector<double> S((size_t)n3 * n3), DB((size_t)n3 * nl2);
    for (int32_t t = 0; t < nt; ++t) {
      std::fill(DB.begin(), DB.end(), 0.0);
      // DB = Dv_t Bm_t, block by block (local blocks: faces k, then the interior)
      for (int blk = 0; blk < 4 + (nint > 0); ++blk) {
        const int l0 = blk < 4 ? nfg * blk : 4 * nfg;
        const int gs = blk < 4 ? nfg : nint;
        const int32_t g = blk < 4 ? dof2[(size_t)t * nl2 + l0] / nfg : nf + t;
        const std::vector<double>& Bi = ginv[g];
        for (int i = 0; i < n3; ++i)
          for (int c = 0; c < gs; ++c) {
            double s = 0.0;
            for (int a = 0; a < gs; ++a) s += sgn[t] * Dref[(size_t)i * nl2 + l0 + a] * Bi[(size_t)a * gs + c];
            DB[(size_t)i * nl2 + l0 + c] = s;
          }
      }
      for (int i = 0; i < n3; ++i)
        for (int k = 0; k < n3; ++k) {
          double s = 0.0;
          for (int j = 0; j < nl2; ++j) s += DB[(size_t)i * nl2 + j] * sgn[t] * Dref[(size_t)k * nl2 + j];
          S[(size_t)i * n3 + k] = s;
        }
      if (!spd_inverse(n3, S)) return "the divergence Schur block of tet " + std::to_string(t) + " is singular";
      for (int i = 0; i < n3; ++i)
        for (int k = 0; k < n3; ++k) rows[t * n3 + i].push_back({t * n3 + k, S[(size_t)i * n3 + k]});
    }
    rows_to_csr(N3, N3, rows, &out->Bs);
  }
  // assembly of the per-tet local load vectors: f_r = sum over (t, j) with dof2[t][j] = r
  {
    std::vector<std::vector<std::pair<int32_t, double>>> rows(n2);
    for (int64_t k = 0; k < (int64_t)nt * nl2; ++k) rows[dof2[k]].push_back({(int32_t)k, 1.0});
    rows_to_csr(n2, (int32_t)std::min<int64_t>((int64_t)nt * nl2, INT32_MAX), rows, &out->Asm);
  }
  return "";
}

}  // namespace fempic
