// Adams-Bashforth push on the polynomial path (Section III-B, last paragraph:
// a fourth-order Adams-Bashforth push makes the particle path a fourth-order
// Lagrange polynomial, and the current integrates the edge basis along it).
//
// Per particle: x^n, v^n (integer times), the history v^{n-j}, a^{n-j}
// (j = 1..3), a = (q/m)(E + v x B) gathered at x^n.  With k the Adams-Bashforth
// order of the step (1..4 while the history fills):
//   v^{n+1} = v^n + dt sum_j beta_j a^{n-j},
//   x(s) = sum_m C_m s^m, C_0 = x^n, C_m = dt sum_j gam_jm v^{n-j}, s in [0, 1]
// (the integral of the Lagrange polynomial through the last k velocities,
// so x(1) is the Adams-Bashforth position update).  In each tet lambda(x(s))
// is a polynomial in s: each face's first sign change to negative after the
// entry parameter is isolated by Bernstein subdivision (Descartes' rule of
// signs on the Bernstein coefficients) and polished by safeguarded Newton
// steps; the smallest crossing wins (ties to the lowest face).  Walls mirror the rest of the path
// and the velocity history.  The current of each sub-path is
// q w int W1_i(x(s)) . x'(s) ds by the (2p + 2)-point Gauss-Legendre rule,
// exact for the degree pk + k - 1 integrand.  Every operation is rounded
// separately in a fixed order (Strict), so positions and walk decisions are
// reproducible.
#pragma once

#include "kernels.cuh"

namespace fempic {
namespace dev {

// A sign pattern that is still ambiguous on a parameter interval shorter than
// this (in s) is a graze: the path stays in the tet unless it ends negative.
constexpr double kAbGraze = 9.313225746154785e-10;  // 2^-30
constexpr int kAbMaxChecks = 256;                   // interval checks per face and sub-path
constexpr int kAbNewton = 48;                       // safeguarded Newton steps at most

// beta_j of order k (exact fractions, rounded once)
__host__ __device__ constexpr double ab_beta(int k, int j) {
  return k == 1   ? 1.0
         : k == 2 ? (j == 0 ? 3.0 / 2.0 : -1.0 / 2.0)
         : k == 3 ? (j == 0 ? 23.0 / 12.0 : (j == 1 ? -4.0 / 3.0 : 5.0 / 12.0))
                  : (j == 0 ? 55.0 / 24.0 : (j == 1 ? -59.0 / 24.0 : (j == 2 ? 37.0 / 24.0 : -3.0 / 8.0)));
}

// gam_jm of order k: int_0^s l_j = sum_m gam_jm s^m, l_j the Lagrange basis
// on the nodes 0, -1, ..., -(k-1)
__host__ __device__ constexpr double ab_gam(int k, int j, int m) {
  if (m == 0 || m > k || j >= k) return 0.0;
  if (k == 1) return m == 1 ? 1.0 : 0.0;
  if (k == 2) {
    constexpr double t[2][3] = {{0.0, 1.0, 1.0 / 2.0}, {0.0, 0.0, -1.0 / 2.0}};
    return t[j][m];
  }
  if (k == 3) {
    constexpr double t[3][4] = {{0.0, 1.0, 3.0 / 4.0, 1.0 / 6.0},
                                {0.0, 0.0, -1.0, -1.0 / 3.0},
                                {0.0, 0.0, 1.0 / 4.0, 1.0 / 6.0}};
    return t[j][m];
  }
  constexpr double t[4][5] = {{0.0, 1.0, 11.0 / 12.0, 1.0 / 3.0, 1.0 / 24.0},
                              {0.0, 0.0, -3.0 / 2.0, -5.0 / 6.0, -1.0 / 8.0},
                              {0.0, 0.0, 3.0 / 4.0, 2.0 / 3.0, 1.0 / 8.0},
                              {0.0, 0.0, -1.0 / 6.0, -1.0 / 6.0, -1.0 / 24.0}};
  return t[j][m];
}

// Gauss-Legendre on [0, 1]: 4 points (order 1) and 6 points (order 2), from
// the standard abscissae and weights on [-1, 1]
template <int P>
__device__ __forceinline__ void gl_rule(int q, double& x, double& w) {
  if (P == 1) {
    constexpr double xs[4] = {-0.86113631159405257522, -0.33998104358485626480, 0.33998104358485626480,
                              0.86113631159405257522};
    constexpr double ws[4] = {0.34785484513745385737, 0.65214515486254614263, 0.65214515486254614263,
                              0.34785484513745385737};
    x = 0.5 * (xs[q] + 1.0);
    w = 0.5 * ws[q];
  } else {
    constexpr double xs[6] = {-0.93246951420315202781, -0.66120938646626451366, -0.23861918608319690863,
                              0.23861918608319690863, 0.66120938646626451366, 0.93246951420315202781};
    constexpr double ws[6] = {0.17132449237917034504, 0.36076157304813860757, 0.46791393457269104739,
                              0.46791393457269104739, 0.36076157304813860757, 0.17132449237917034504};
    x = 0.5 * (xs[q] + 1.0);
    w = 0.5 * ws[q];
  }
}

struct Ab4Args {
  ParticleArgs p;
  double* vh[3][3];  // [j][component]: v^{n-1-j}
  double* ah[3][3];  // a^{n-1-j}
  int k;             // Adams-Bashforth order of this step (1..4)
  double qm;         // q / m (one species)
  double qm_s[kMaxSpecies];
};

// Horner over the K+1 ascending coefficients c[m][i], and its derivative
template <int K>
__device__ __forceinline__ double ab_horner(const double (&c)[5][4], int i, double s) {
  double p = c[K][i];
#pragma unroll
  for (int m = K - 1; m >= 0; --m) p = __dadd_rn(__dmul_rn(p, s), c[m][i]);
  return p;
}
template <int K>
__device__ __forceinline__ double ab_horner_d(const double (&c)[5][4], int i, double s) {
  double p = __dmul_rn((double)K, c[K][i]);
#pragma unroll
  for (int m = K - 1; m >= 1; --m) p = __dadd_rn(__dmul_rn(p, s), __dmul_rn((double)m, c[m][i]));
  return p;
}

__device__ __forceinline__ void ab_mirror(double* vec, const double* gw, double gg) {
  const double f = __ddiv_rn(__dmul_rn(2.0, dot3<Strict>(vec, gw)), gg);
#pragma unroll
  for (int c = 0; c < 3; ++c) vec[c] = __dsub_rn(vec[c], __dmul_rn(f, gw[c]));
}

// First s in [s0, 1] after which the polynomial c[0..n] (ascending powers of
// s, n a compile-time degree) is negative: the crossing of a face whose lambda is c along the path.
// Returns 2.0 when it stays non-negative (a graze included).  The interval
// [s0, 1] is mapped to u in [0, 1]; a window [ua, ua + w] is examined through
// the Bernstein coefficients of the polynomial on it: no sign change means no
// root there (the window moves on and widens), one sign change with a positive
// start means exactly one crossing (refined by Newton steps kept inside the
// window), more sign changes halve the window.
template <int n>
__device__ __forceinline__ double ab_first_negative(const double (&c)[5], double s0) {
  constexpr double binom[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0},
                                  {1, 4, 6, 4, 1}};
  const double span = 1.0 - s0;
  // P(u) = c(s0 + span u): Taylor shift to s0, then scale u^k by span^k
  double P[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) P[k] = k <= n ? c[k] : 0.0;
#pragma unroll
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int k = n - 1; k >= i; --k) P[k] = fma(s0, P[k + 1], P[k]);
  {
    double sc = span;
#pragma unroll
    for (int k = 1; k <= n; ++k) {
      P[k] *= sc;
      sc *= span;
    }
  }
  if (n == 0) return P[0] < 0.0 ? s0 : 2.0;  // constant
  const double wmin = kAbGraze / span;
  double ua = 0.0, w = 1.0;
  for (int it = 0; it < kAbMaxChecks; ++it) {
    // q(t) = P(ua + w t), monomial then Bernstein coefficients
    double q[5], b[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) q[k] = P[k];
#pragma unroll
    for (int i = 0; i < n; ++i)
#pragma unroll
      for (int k = n - 1; k >= i; --k) q[k] = fma(ua, q[k + 1], q[k]);
    {
      double sc = w;
#pragma unroll
      for (int k = 1; k <= n; ++k) {
        q[k] *= sc;
        sc *= w;
      }
    }
#pragma unroll
    for (int k = 0; k <= n; ++k) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j <= k; ++j) acc = fma(binom[k][j] / binom[n][j], q[j], acc);
      b[k] = acc;
    }
    // sign changes (zeros skipped) and the first nonzero sign
    int changes = 0, first = 0, last = 0;
#pragma unroll
    for (int k = 0; k <= n; ++k) {
      const int sg = b[k] > 0.0 ? 1 : (b[k] < 0.0 ? -1 : 0);
      if (sg == 0) continue;
      if (first == 0) first = sg;
      if (last != 0 && sg != last) ++changes;
      last = sg;
    }
    if (first < 0) return s0 + span * ua;  // negative from the window's start
    const bool ends_negative = last < 0;
    if (changes == 0 || (changes >= 2 && w <= wmin && !ends_negative)) {
      ua += w;  // no root, or a graze
      if (ua >= 1.0) return 2.0;
      w = fmin(2.0 * w, 1.0 - ua);
      continue;
    }
    if (changes >= 2 && w > wmin) {
      w *= 0.5;
      continue;
    }
    // one crossing to negative in (0, 1] of t (or a cluster narrower than the
    // graze width that ends negative): q(0) > 0, q(1) <= 0
    double lo = 0.0, hi = 1.0;
    double t = b[0] / (b[0] - b[n]);
    if (!(t > 0.0 && t < 1.0)) t = 0.5;
    for (int k = 0; k < kAbNewton; ++k) {
      double f = q[n], d = 0.0;
#pragma unroll
      for (int m = n - 1; m >= 0; --m) {
        d = fma(d, t, f);
        f = fma(f, t, q[m]);
      }
      if (f < 0.0)
        hi = t;
      else
        lo = t;
      double tn = d != 0.0 ? t - f / d : 0.5 * (lo + hi);
      if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
      if (tn == t || hi - lo <= 2.220446049250313e-16) {
        t = tn;
        break;
      }
      t = tn;
    }
    return s0 + span * (ua + w * t);
  }
  return 2.0;
}

// K: the Adams-Bashforth order of the step (a template parameter, so the path
// and lambda coefficients stay in registers)
template <int P, int K>
__global__ void __launch_bounds__(128) k_particle_ab4(Ab4Args A) {
  constexpr int N1 = P == 1 ? 6 : 20;
  constexpr int N2 = P == 1 ? 4 : 15;
  constexpr int N0 = P == 1 ? 4 : 10;
  constexpr int NQ = 2 * P + 2;
  const ParticleArgs& a = A.p;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long my_cross = 0;
  if (i < a.n) {
    double qw = a.qw, qm = A.qm;
    if (a.sp.n > 1) {
      const int s = species_of(a.sp, __ldg(a.pid + i));
      qw = a.sp.qw[s];
      qm = A.qm_s[s];
    }
    int T = a.tet[i];
    double x[3], v[3], vh[3][3], ah[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x[c] = a.x[c][i];
      v[c] = a.v[c][i];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        vh[j][c] = A.vh[j][c][i];
        ah[j][c] = A.ah[j][c][i];
      }
    }
    TetGeom G;
    load_geom(a.geom, T, G);
    double l[4];
    bary<Strict>(G, x, l);
    double ev[N1], bv[N2];
    const int32_t* d1 = a.dof1 + (size_t)T * N1;
    const int32_t* d2 = a.dof2 + (size_t)T * N2;
#pragma unroll
    for (int j = 0; j < N1; ++j) ev[j] = __ldg(a.e + __ldg(d1 + j));
#pragma unroll
    for (int j = 0; j < N2; ++j) bv[j] = __ldg(a.b + __ldg(d2 + j));
    double E[3], B[3], vxb[3], an[3];
    gather_E<P, Strict>(G, l, ev, E);
    gather_B<P, Strict>(G, l, bv, a.B0, B);
    cross3<Strict>(v, B, vxb);
#pragma unroll
    for (int c = 0; c < 3; ++c) an[c] = __dmul_rn(qm, __dadd_rn(E[c], vxb[c]));
    // velocity update and path coefficients
    double vnew[3], C[5][4];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double acc = __dmul_rn(ab_beta(K, 0), an[c]);
#pragma unroll
      for (int j = 1; j < K; ++j) acc = __dadd_rn(acc, __dmul_rn(ab_beta(K, j), ah[j - 1][c]));
      vnew[c] = __dadd_rn(v[c], __dmul_rn(a.dt, acc));
      C[0][c] = x[c];
#pragma unroll
      for (int m = 1; m <= K; ++m) {
        double s = __dmul_rn(ab_gam(K, 0, m), v[c]);
#pragma unroll
        for (int j = 1; j < K; ++j) s = __dadd_rn(s, __dmul_rn(ab_gam(K, j, m), vh[j - 1][c]));
        C[m][c] = __dmul_rn(a.dt, s);
      }
    }
    int entry = -1;
    double s0 = 0.0;
    int nc = 0;
    unsigned long long hsh = kFnvOffset;
    for (;;) {
      // lambda coefficients in this tet
      double L[5][4];
#pragma unroll
      for (int m = 0; m <= K; ++m)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const double t = __dadd_rn(__dadd_rn(__dmul_rn(G.g[f][0], C[m][0]), __dmul_rn(G.g[f][1], C[m][1])),
                                     __dmul_rn(G.g[f][2], C[m][2]));
          L[m][f] = m == 0 ? __dadd_rn(t, G.c[f]) : t;
        }
      int best = -1;
      double s1 = 1.0;
      {
        double sbest = 2.0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          double cf[5];
#pragma unroll
          for (int m = 0; m < 5; ++m) cf[m] = m <= K ? L[m][f] : 0.0;
          double sf;
          if (f == entry) {
            // lambda of the entry face vanishes at s0: divide out (s - s0)
            double acc = cf[K];
#pragma unroll
            for (int m = K - 1; m >= 0; --m) {
              const double nx = fma(acc, s0, cf[m]);
              cf[m] = acc;
              acc = nx;
            }
            cf[K] = 0.0;
            sf = ab_first_negative<K - 1>(cf, s0);
          } else {
            sf = ab_first_negative<K>(cf, s0);
          }
          if (sf < sbest) {
            sbest = sf;
            best = f;
          }
        }
        if (best >= 0) s1 = fmin(fmax(sbest, s0), 1.0);
      }
      // current of the sub-path [s0, s1]
      {
        const double ln = __dsub_rn(s1, s0);
        double acc[N1];
#pragma unroll
        for (int j = 0; j < N1; ++j) acc[j] = 0.0;
#pragma unroll 1
        for (int q = 0; q < NQ; ++q) {
          double xq, wq;
          gl_rule<P>(q, xq, wq);
          const double sq = __dadd_rn(s0, __dmul_rn(ln, xq));
          double lv[4], dl[4];
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            lv[f] = ab_horner<K>(L, f, sq);
            dl[f] = ab_horner_d<K>(L, f, sq);
          }
#pragma unroll
          for (int j = 0; j < N1; ++j) {
            int aa, bb, xx, kind;
            if (P == 1) {
              aa = edge_s(j);
              bb = edge_t(j);
              xx = 0;
              kind = 0;
            } else {
              aa = w1q(j, 0);
              bb = w1q(j, 1);
              xx = w1q(j, 2);
              kind = w1q(j, 3);
            }
            double wv = __dsub_rn(__dmul_rn(lv[aa], dl[bb]), __dmul_rn(lv[bb], dl[aa]));
            if (kind == 1)
              wv = __dmul_rn(__dsub_rn(__dmul_rn(3.0, lv[xx]), 1.0), wv);
            else if (kind == 2)
              wv = __dmul_rn(__dmul_rn(3.0, lv[xx]), wv);
            acc[j] = __dadd_rn(acc[j], __dmul_rn(wq, wv));
          }
        }
        const int32_t* dofs = a.dof1 + (size_t)T * N1;
#pragma unroll
        for (int j = 0; j < N1; ++j) atomicAdd(a.dg + __ldg(dofs + j), __dmul_rn(qw, __dmul_rn(ln, acc[j])));
      }
      if (best < 0) break;
      ++nc;
      const int nb = __ldg(a.nbr + (size_t)T * 4 + best);
      const unsigned long long code = nb < 0 ? (0x80000000ull | (unsigned)best) : (unsigned long long)(nb >> 2);
      hsh = (hsh ^ code) * kFnvPrime;
      if (nb >= 0) {
        entry = nb & 3;
        T = nb >> 2;
        s0 = s1;
        load_geom(a.geom, T, G);
      } else {
        double gw[3];
#pragma unroll
        for (int f = 0; f < 4; ++f)
          if (f == best) {
            gw[0] = G.g[f][0];
            gw[1] = G.g[f][1];
            gw[2] = G.g[f][2];
          }
        const double gg = dot3<Strict>(gw, gw);
        double hit[3], d0[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double p = C[K][c];
#pragma unroll
          for (int m = K - 1; m >= 0; --m) p = __dadd_rn(__dmul_rn(p, s1), C[m][c]);
          hit[c] = p;
          d0[c] = __dsub_rn(C[0][c], p);
        }
        ab_mirror(d0, gw, gg);
#pragma unroll
        for (int c = 0; c < 3; ++c) C[0][c] = __dadd_rn(hit[c], d0[c]);
#pragma unroll
        for (int m = 1; m <= K; ++m) {
          double cm[3] = {C[m][0], C[m][1], C[m][2]};
          ab_mirror(cm, gw, gg);
          C[m][0] = cm[0];
          C[m][1] = cm[1];
          C[m][2] = cm[2];
        }
        ab_mirror(vnew, gw, gg);
        ab_mirror(v, gw, gg);
        ab_mirror(an, gw, gg);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          ab_mirror(vh[j], gw, gg);
          ab_mirror(ah[j], gw, gg);
        }
        s0 = s1;
        entry = best;
      }
      if (nc >= a.max_cross) {
        atomicOr(a.status, kStatusWalk);
        break;
      }
    }
    // end point x(1), charge there, state and history
    double xe[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double p = C[K][c];
#pragma unroll
      for (int m = K - 1; m >= 0; --m) p = __dadd_rn(__dmul_rn(p, 1.0), C[m][c]);
      xe[c] = p;
    }
    double le[4];
    bary<Strict>(G, xe, le);
    deposit_rho<P, Strict>(le, qw, a.dof0 + (size_t)T * N0, a.rho);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a.x[c][i] = xe[c];
      a.v[c][i] = vnew[c];
      A.vh[2][c][i] = vh[1][c];
      A.vh[1][c][i] = vh[0][c];
      A.vh[0][c][i] = v[c];
      A.ah[2][c][i] = ah[1][c];
      A.ah[1][c][i] = ah[0][c];
      A.ah[0][c][i] = an[c];
    }
    a.tet[i] = T;
    if (a.ncross) a.ncross[i] = nc;
    if (a.hash) a.hash[i] = hsh;
    my_cross = nc;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_cross += __shfl_xor_sync(0xffffffffu, my_cross, o);
  if ((threadIdx.x & 31) == 0 && my_cross) atomicAdd(a.crossings, my_cross);
}

}  // namespace dev
}  // namespace fempic
