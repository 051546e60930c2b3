// FP64 particle kernel with fused multiply-adds and factored basis sums.
//
// Same method as k_particle (gather, Boris push, ray-face walk, path-integral
// deposit, charge), rearranged to cut work:
//   * E = sum_j e_j m_j(l) w_ab = sum_k alpha_k grad l_k, where the DOF sums
//     are first collected per local edge pair (c_ab), then
//     alpha_b += c_ab l_a, alpha_a -= c_ab l_b;
//   * B = B0 + sum_f beta_f w_f = B0 + sum_{a<b} gamma_ab grad l_a x grad l_b,
//     with the six cross products reduced to three (the gradients sum to 0);
//   * the deposit evaluates w_ab . (b - a) = l_a d_b - l_b d_a once per pair
//     (constant along the chord) and scales it by each DOF's multiplier at the
//     sub-segment's midpoint (exact: the integrand is affine in s);
//   * optionally (AGG), the first sub-segment's current and the end-point
//     charge are summed across the warp's lanes that share a tet (particles
//     are sorted by tet) before the atomic adds.
#pragma once

#include "kernels.cuh"

// Sum the first sub-segment's current and the end-point charge over the lanes
// of a warp that share a tet before the FP64 atomics (segmented warp scans).
// Off by default: on GB300 the scans' FP64 adds occupy the narrow FP64 pipe
// that bounds the particle kernel, while the atomics execute in L2; direct
// atomics measured 12-14 % faster (drift tube and 37^3 box, FP64 and mixed).
#ifndef FEMPIC_PARTICLE_AGG
#define FEMPIC_PARTICLE_AGG 0
#endif
#ifndef FEMPIC_DEPOSIT_SCALED
#define FEMPIC_DEPOSIT_SCALED 1
#endif

namespace fempic {
namespace dev {

struct WarpRuns {
  int lo, hi;   // first/last lane of this lane's run of equal keys
  bool ok;      // every run in the warp is contiguous
};

__device__ __forceinline__ WarpRuns warp_runs(int key) {
  unsigned m = __match_any_sync(0xffffffffu, key);
  int lo = __ffs(m) - 1;
  int hi = 31 - __clz(m);
  unsigned want = (hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u)) & ~((1u << lo) - 1u);
  bool ok = __all_sync(0xffffffffu, m == want);
  return WarpRuns{lo, hi, ok};
}

// inclusive segmented sum; the run total ends in lane hi
__device__ __forceinline__ double run_sum(double v, const WarpRuns& r, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    double t = __shfl_up_sync(0xffffffffu, v, off);
    if (lane - off >= r.lo) v += t;
  }
  return v;
}

// add v into dst: summed over the run first when `agg` (all lanes participate)
__device__ __forceinline__ void run_add(double* dst, double v, bool agg, const WarpRuns& r, int lane, bool valid) {
  if (agg) {
    v = run_sum(v, r, lane);
    if (valid && lane == r.hi) atomicAdd(dst, v);
  } else if (valid) {
    atomicAdd(dst, v);
  }
}

template <int P>
__device__ __forceinline__ void gather_E_fact(const TetGeom& G, const double* l, const double* __restrict__ e,
                                              const int32_t* __restrict__ d1, double* E) {
  double c[6];
  if (P == 1) {
#pragma unroll
    for (int j = 0; j < 6; ++j) c[j] = __ldg(e + __ldg(d1 + j));
  } else {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int s = edge_s(j), t = edge_t(j);
      double e0 = __ldg(e + __ldg(d1 + 2 * j)), e1 = __ldg(e + __ldg(d1 + 2 * j + 1));
      c[j] = fma(e0, fma(3.0, l[s], -1.0), e1 * fma(3.0, l[t], -1.0));
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int s = face_v(f, 0), t = face_v(f, 1), u = face_v(f, 2);
      double e0 = __ldg(e + __ldg(d1 + 12 + 2 * f)), e1 = __ldg(e + __ldg(d1 + 13 + 2 * f));
      c[pair_of(s, t)] = fma(e0, 3.0 * l[u], c[pair_of(s, t)]);
      c[pair_of(s, u)] = fma(e1, 3.0 * l[t], c[pair_of(s, u)]);
    }
  }
  double al[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int s = edge_s(j), t = edge_t(j);
    al[t] = fma(c[j], l[s], al[t]);
    al[s] = fma(-c[j], l[t], al[s]);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
    E[k] = fma(al[0], G.g[0][k], fma(al[1], G.g[1][k], fma(al[2], G.g[2][k], al[3] * G.g[3][k])));
}

template <int P>
__device__ __forceinline__ void gather_B_fact(const TetGeom& G, const double* l, const double* __restrict__ b,
                                              const int32_t* __restrict__ d2, const double* B0, double* B) {
  double beta[4];
  if (P == 1) {
#pragma unroll
    for (int f = 0; f < 4; ++f) beta[f] = __ldg(b + __ldg(d2 + f));
  } else {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      double s = 0.0;
#pragma unroll
      for (int v = 0; v < 3; ++v) s = fma(__ldg(b + __ldg(d2 + 3 * f + v)), fma(4.0, l[face_v(f, v)], -1.0), s);
      if (f < 3) s = fma(__ldg(b + __ldg(d2 + 12 + f)), 4.0 * l[f], s);
      beta[f] = s;
    }
  }
  // w_f = 2 (l_s X_tu - l_t X_su + l_u X_st)
  double gam[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int s = face_v(f, 0), t = face_v(f, 1), u = face_v(f, 2);
    double b2 = 2.0 * beta[f];
    gam[pair_of(t, u)] = fma(b2, l[s], gam[pair_of(t, u)]);
    gam[pair_of(s, u)] = fma(-b2, l[t], gam[pair_of(s, u)]);
    gam[pair_of(s, t)] = fma(b2, l[u], gam[pair_of(s, t)]);
  }
  // grad l_3 = -(grad l_0 + grad l_1 + grad l_2): the six products
  // grad l_a x grad l_b reduce to X01, X02, X12 with combined coefficients
  const double k01 = gam[pair_of(0, 1)] - gam[pair_of(0, 3)] + gam[pair_of(1, 3)];
  const double k02 = gam[pair_of(0, 2)] - gam[pair_of(0, 3)] + gam[pair_of(2, 3)];
  const double k12 = gam[pair_of(1, 2)] - gam[pair_of(1, 3)] + gam[pair_of(2, 3)];
  const double* g0 = G.g[0];
  const double* g1 = G.g[1];
  const double* g2 = G.g[2];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
    const double x01 = fma(g0[c1], g1[c2], -g0[c2] * g1[c1]);
    const double x02 = fma(g0[c1], g2[c2], -g0[c2] * g2[c1]);
    const double x12 = fma(g1[c1], g2[c2], -g1[c2] * g2[c1]);
    B[c] = fma(k01, x01, fma(k02, x02, fma(k12, x12, B0[c])));
  }
}

// current of the sub-segment [s0, s1] of the chord in one tet.  Along the
// straight chord l(s) = la + s d, w_ab . (b - a) = l_a d_b - l_b d_a does not
// depend on s, and the order-2 multipliers (3 l_x - 1, 3 l_x) are affine in s,
// so the path integral of every basis function is the sub-segment length times
// its value at the midpoint: the midpoint rule is exact here (the oracle's
// two-point Gauss-Legendre rule gives the same value up to rounding).
template <int P>
__device__ __forceinline__ void deposit_fact(const double* la, const double* lb, double s0, double s1, double qw,
                                             const int32_t* __restrict__ dofs, double* __restrict__ dg, bool agg,
                                             const WarpRuns& runs, int lane, bool valid) {
  double d[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) d[i] = lb[i] - la[i];
  const double sc = qw * (s1 - s0);
  double w[6];
#if FEMPIC_DEPOSIT_SCALED
  // the sub-segment's weight folded into the direction once (4 products
  // instead of one per edge pair)
  double ds[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) ds[i] = sc * d[i];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int s = edge_s(j), t = edge_t(j);
    w[j] = fma(la[s], ds[t], -la[t] * ds[s]);
  }
#else
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int s = edge_s(j), t = edge_t(j);
    w[j] = sc * fma(la[s], d[t], -la[t] * d[s]);
  }
#endif
  if (P == 1) {
#pragma unroll
    for (int j = 0; j < 6; ++j) run_add(dg + __ldg(dofs + j), w[j], agg, runs, lane, valid);
  } else {
    const double mid = (s0 + s1) * 0.5;
    double t3[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) t3[i] = 3.0 * fma(mid, d[i], la[i]);
#pragma unroll
    for (int j = 0; j < 20; ++j) {
      const int a = w1q(j, 0), b = w1q(j, 1), x = w1q(j, 2), kind = w1q(j, 3);
      const double wp = w[pair_of(a, b)];
      const double val = kind == 1 ? fma(t3[x], wp, -wp) : t3[x] * wp;
      run_add(dg + __ldg(dofs + j), val, agg, runs, lane, valid);
    }
  }
}

template <int P>
__device__ __forceinline__ void deposit_rho_fact(const double* l, double qw, const int32_t* __restrict__ dofs,
                                                 double* __restrict__ rho, bool agg, const WarpRuns& runs, int lane,
                                                 bool valid) {
  if (P == 1) {
#pragma unroll
    for (int k = 0; k < 4; ++k) run_add(rho + __ldg(dofs + k), qw * l[k], agg, runs, lane, valid);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) run_add(rho + __ldg(dofs + k), qw * l[k] * fma(2.0, l[k], -1.0), agg, runs, lane, valid);
#pragma unroll
    for (int j = 0; j < 6; ++j)
      run_add(rho + __ldg(dofs + 4 + j), qw * 4.0 * l[edge_s(j)] * l[edge_t(j)], agg, runs, lane, valid);
  }
}


// ---- FP32 gather and push (mixed precision): lambda and geometry rounded to
// float, DOF values read as FP64 and rounded, E, B and the Boris rotation in
// FP32.  Positions, the walk, the deposit and the charge stay FP64.
template <int P, class VT>
__device__ __forceinline__ void gather_EB_f32(const TetGeom& Gd, const double* lad, const VT* __restrict__ e,
                                              const int32_t* __restrict__ d1, const VT* __restrict__ b,
                                              const int32_t* __restrict__ d2, const double* B0d, float* E, float* B,
                                              const float* __restrict__ g32 = nullptr) {
  float l[4], g[4][3];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    l[i] = (float)lad[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) g[i][k] = g32 ? __ldg(g32 + 3 * i + k) : (float)Gd.g[i][k];
  }
  float c[6];
  if (P == 1) {
#pragma unroll
    for (int j = 0; j < 6; ++j) c[j] = (float)__ldg(e + __ldg(d1 + j));
  } else {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int s = edge_s(j), t = edge_t(j);
      float e0 = (float)__ldg(e + __ldg(d1 + 2 * j)), e1 = (float)__ldg(e + __ldg(d1 + 2 * j + 1));
      c[j] = fmaf(e0, fmaf(3.f, l[s], -1.f), e1 * fmaf(3.f, l[t], -1.f));
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int s = face_v(f, 0), t = face_v(f, 1), u = face_v(f, 2);
      float e0 = (float)__ldg(e + __ldg(d1 + 12 + 2 * f)), e1 = (float)__ldg(e + __ldg(d1 + 13 + 2 * f));
      c[pair_of(s, t)] = fmaf(e0, 3.f * l[u], c[pair_of(s, t)]);
      c[pair_of(s, u)] = fmaf(e1, 3.f * l[t], c[pair_of(s, u)]);
    }
  }
  float al[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int s = edge_s(j), t = edge_t(j);
    al[t] = fmaf(c[j], l[s], al[t]);
    al[s] = fmaf(-c[j], l[t], al[s]);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) E[k] = fmaf(al[0], g[0][k], fmaf(al[1], g[1][k], fmaf(al[2], g[2][k], al[3] * g[3][k])));
  float beta[4];
  if (P == 1) {
#pragma unroll
    for (int f = 0; f < 4; ++f) beta[f] = (float)__ldg(b + __ldg(d2 + f));
  } else {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      float sacc = 0.f;
#pragma unroll
      for (int v = 0; v < 3; ++v)
        sacc = fmaf((float)__ldg(b + __ldg(d2 + 3 * f + v)), fmaf(4.f, l[face_v(f, v)], -1.f), sacc);
      if (f < 3) sacc = fmaf((float)__ldg(b + __ldg(d2 + 12 + f)), 4.f * l[f], sacc);
      beta[f] = sacc;
    }
  }
  float gam[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int s = face_v(f, 0), t = face_v(f, 1), u = face_v(f, 2);
    float b2 = 2.f * beta[f];
    gam[pair_of(t, u)] = fmaf(b2, l[s], gam[pair_of(t, u)]);
    gam[pair_of(s, u)] = fmaf(-b2, l[t], gam[pair_of(s, u)]);
    gam[pair_of(s, t)] = fmaf(b2, l[u], gam[pair_of(s, t)]);
  }
  B[0] = (float)B0d[0];
  B[1] = (float)B0d[1];
  B[2] = (float)B0d[2];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float* ga = g[edge_s(j)];
    const float* gb = g[edge_t(j)];
    B[0] = fmaf(gam[j], ga[1] * gb[2] - ga[2] * gb[1], B[0]);
    B[1] = fmaf(gam[j], ga[2] * gb[0] - ga[0] * gb[2], B[1]);
    B[2] = fmaf(gam[j], ga[0] * gb[1] - ga[1] * gb[0], B[2]);
  }
}

__device__ __forceinline__ void boris_f32(float* v, const float* E, const float* B, float h) {
  float eh[3], vm[3], t[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    eh[k] = E[k] * h;
    vm[k] = v[k] + eh[k];
    t[k] = B[k] * h;
  }
  float sf = 2.f / (1.f + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  float vp[3] = {vm[0] + (vm[1] * t[2] - vm[2] * t[1]), vm[1] + (vm[2] * t[0] - vm[0] * t[2]),
                 vm[2] + (vm[0] * t[1] - vm[1] * t[0])};
  float sv[3] = {t[0] * sf, t[1] * sf, t[2] * sf};
  v[0] = vm[0] + (vp[1] * sv[2] - vp[2] * sv[1]) + eh[0];
  v[1] = vm[1] + (vp[2] * sv[0] - vp[0] * sv[2]) + eh[1];
  v[2] = vm[2] + (vp[0] * sv[1] - vp[1] * sv[0]) + eh[2];
}

// exit face of the chord in the current tet (entry face excluded); -1 if it ends here.
// The candidates' parameters s_f = la_f / (la_f - lb_f) are compared as
// cross products (one division, for the winner): with lb_f < 0 the
// denominator is positive unless the start lies outside face f by more than
// the end does, where s_f >= 1 and the candidate counts as s = 1.
#ifndef FEMPIC_EXIT_NODIV
#define FEMPIC_EXIT_NODIV 1
#endif
__device__ __forceinline__ int exit_face(const double* la, const double* lb, int entry, double s0, double& s1) {
  int best = -1;
#if FEMPIC_EXIT_NODIV
  double num = 1.0, den = 1.0;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    if (f != entry && lb[f] < 0.0) {
      double nf = la[f], df = la[f] - lb[f];
      if (!(df > 0.0)) nf = df = 1.0;
      if (best < 0 || nf * den < num * df) {
        num = nf;
        den = df;
        best = f;
      }
    }
  }
  s1 = best < 0 ? 1.0 : fmin(fmax(num / den, s0), 1.0);
#else
  double sbest = __longlong_as_double(0x7ff0000000000000ll);
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    if (f != entry && lb[f] < 0.0) {
      double si = la[f] / (la[f] - lb[f]);
      if (si < sbest) {
        sbest = si;
        best = f;
      }
    }
  }
  s1 = best < 0 ? 1.0 : fmin(fmax(sbest, s0), 1.0);
#endif
  return best;
}

__device__ __forceinline__ void bary_fma(const TetGeom& G, const double* x, double* l) {
#pragma unroll
  for (int i = 0; i < 4; ++i) l[i] = fma(G.g[i][0], x[0], fma(G.g[i][1], x[1], fma(G.g[i][2], x[2], G.c[i])));
}

// One particle per thread; every lane of the warp must call it (lanes past the
// end pass valid = false) because the first sub-segment and the charge are
// summed across lanes.
template <int P, bool AGG, bool MIXED>
__device__ __forceinline__ void particle_step(const ParticleArgs& a, int64_t i) {
  constexpr int N1 = P == 1 ? 6 : 20;
  constexpr int N2 = P == 1 ? 4 : 15;
  constexpr int N0 = P == 1 ? 4 : 10;
  const int lane = threadIdx.x & 31;
  const bool valid = i < a.n && index_ok(a.tet[i], a.n_tets, a.status);
  int T = valid ? a.tet[i] : 0;
  double qw = a.qw, hq = a.h;
  if (valid) particle_consts(a, i, qw, hq);
  double x[3], v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    x[k] = valid ? a.x[k][i] : 0.0;
    v[k] = valid ? a.v[k][i] : 0.0;
  }
  TetGeom G;
  load_geom(a.geom, T, G);
  double la[4];
  bary_fma(G, x, la);
  if (MIXED) {
    float Ef[3], Bf[3], vf[3] = {(float)v[0], (float)v[1], (float)v[2]};
    if (a.e32)
      gather_EB_f32<P>(G, la, a.e32, a.dof1 + (size_t)T * N1, a.b32, a.dof2 + (size_t)T * N2, a.B0, Ef, Bf,
                       a.geom32 + (size_t)T * 12);
    else
      gather_EB_f32<P>(G, la, a.e, a.dof1 + (size_t)T * N1, a.b, a.dof2 + (size_t)T * N2, a.B0, Ef, Bf);
    boris_f32(vf, Ef, Bf, (float)hq);
    v[0] = vf[0];
    v[1] = vf[1];
    v[2] = vf[2];
  } else {
    double E[3], B[3];
    gather_E_fact<P>(G, la, a.e, a.dof1 + (size_t)T * N1, E);
    gather_B_fact<P>(G, la, a.b, a.dof2 + (size_t)T * N2, a.B0, B);
    boris<Fast>(v, E, B, hq);
  }
  double pa[3] = {x[0], x[1], x[2]};
  double pb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) pb[k] = fma(a.dt, v[k], x[k]);
  // ---- first visit: every lane, current summed over lanes sharing the tet
  double lb[4];
  bary_fma(G, pb, lb);
  double s1;
  int best = exit_face(la, lb, -1, 0.0, s1);
  {
    const WarpRuns runs = AGG ? warp_runs(valid ? T : -1 - lane) : WarpRuns{0, 0, false};
    deposit_fact<P>(la, lb, 0.0, s1, qw, a.dof1 + (size_t)T * N1, a.dg, AGG && runs.ok, runs, lane, valid);
  }
  int nc = 0;
  unsigned long long hsh = kFnvOffset;
  int entry = -1;
  double s0 = 0.0;
  bool absorbed = false;
  bool walking = valid && best >= 0;
  while (walking) {
    ++nc;
    int nb = __ldg(a.nbr + (size_t)T * 4 + best);
    unsigned long long code = nb == -2  ? (0xC0000000ull | (unsigned)best)
                              : nb < 0 ? (0x80000000ull | (unsigned)best)
                                       : (unsigned long long)(nb >> 2);
    hsh = (hsh ^ code) * kFnvPrime;
    if (nb >= 0) {
      entry = nb & 3;
      T = nb >> 2;
      if (!index_ok(T, a.n_tets, a.status)) {
        T = 0;
        break;
      }
      s0 = s1;
      load_geom(a.geom, T, G);
    } else if (nb == -2) {  // absorbing wall: the path ends at the hit point, no charge left
#pragma unroll
      for (int k = 0; k < 3; ++k) pb[k] = fma(s1, pb[k] - pa[k], pa[k]);
      absorbed = true;
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
      double d[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) d[k] = pb[k] - pa[k];
      double gg = gw[0] * gw[0] + gw[1] * gw[1] + gw[2] * gw[2];
      double fd = 2.0 * (d[0] * gw[0] + d[1] * gw[1] + d[2] * gw[2]) / gg;
      double fv = 2.0 * (v[0] * gw[0] + v[1] * gw[1] + v[2] * gw[2]) / gg;
      double rem = 1.0 - s1;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double hit = fma(s1, d[k], pa[k]);
        pb[k] = fma(rem, d[k] - fd * gw[k], hit);
        pa[k] = hit;
        v[k] -= fv * gw[k];
      }
      s0 = 0.0;
      entry = best;
    }
    if (nc >= a.max_cross) {
      bary_fma(G, pb, lb);
      atomicOr(a.status, kStatusWalk);
      break;
    }
    bary_fma(G, pa, la);
    bary_fma(G, pb, lb);
    best = exit_face(la, lb, entry, s0, s1);
    WarpRuns none{0, 0, false};
    deposit_fact<P>(la, lb, s0, s1, qw, a.dof1 + (size_t)T * N1, a.dg, false, none, lane, true);
    walking = best >= 0;
  }
  // ---- charge at the end point, summed over lanes ending in the same tet
  {
    const bool keep = valid && !absorbed;
    const WarpRuns runs = AGG ? warp_runs(keep ? T : -1 - lane) : WarpRuns{0, 0, false};
    deposit_rho_fact<P>(lb, qw, a.dof0 + (size_t)T * N0, a.rho, AGG && runs.ok, runs, lane, keep);
  }
  if (valid) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      a.x[k][i] = pb[k];
      a.v[k][i] = v[k];
    }
    a.tet[i] = T;
    if (a.ncross) a.ncross[i] = nc;
    if (a.hash) a.hash[i] = hsh;
    if (a.absorbed) a.absorbed[i] = absorbed ? 1 : 0;
  }
  unsigned long long my_cross = nc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_cross += __shfl_xor_sync(0xffffffffu, my_cross, o);
  if (lane == 0 && my_cross) atomicAdd(a.crossings, my_cross);
}

template <int P, bool AGG, bool MIXED = false>
__global__ void __launch_bounds__(256, 2) k_particle_fast(ParticleArgs a) {
  particle_step<P, AGG, MIXED>(a, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

}  // namespace dev
}  // namespace fempic
