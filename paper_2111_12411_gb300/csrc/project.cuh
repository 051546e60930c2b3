// Divergence-free representation of an impressed magnetic flux density
// (Section III-C, eq. conB) on the device.
//
// The load f_i = <W2_i, B> / mu0 is integrated per tet with a conical-product
// Gauss rule (no atomics: per-tet vectors summed by a 0/1 assembly matrix),
// then the saddle-point system
//   [ [*mu^-1]  [~div]^T ] [ b ]   [ f ]
//   [ [~div]    0        ] [ l ] = [ 0 ]
// is solved by conjugate gradients on its Schur complement S = Dv M2^-1 Dv^T
// (outer, preconditioned by per-tet inverses of Dv Bm Dv^T) with inner CG
// solves of M2 (preconditioned by the block-Jacobi inverse Bm).  The outer
// iterate is kept as b itself: b = b_G - sum_k alpha_k M2^-1 Dv^T p_k, whose
// constraint residual Dv b is the outer CG residual.
//
// Every CG scalar lives on the device: the host launches chunks of iterations
// and reads a convergence flag between chunks.  Dot products are per-block
// partial sums over a fixed grid, summed in a fixed order (run-to-run
// deterministic).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "linalg.cuh"

namespace fempic {
namespace dev {

constexpr int kRedGrid = 1024;    // blocks of the reduction kernels (fixed: a deterministic sum order)
constexpr int kRedThreads = 256;  // threads per block
// device scalars of one CG
enum { kCgRZ = 0, kCgAlpha, kCgBeta, kCgRR, kCgBB, kCgTol2, kCgDone, kCgIt, kCgN };

// W2_j . B accumulated for every local j: acc[j] += wgt (W2_j(l) . B)
template <int P>
__device__ __forceinline__ void w2_load_point(const TetGeom& G, const double* l, const double* B, double wgt,
                                              double* acc) {
  double wf[4][3];
#pragma unroll
  for (int f = 0; f < 4; ++f) whitney_face<Fast>(G, l, f, wf[f]);
  double wb[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) wb[f] = wgt * (wf[f][0] * B[0] + wf[f][1] * B[1] + wf[f][2] * B[2]);
  if constexpr (P == 1) {
#pragma unroll
    for (int f = 0; f < 4; ++f) acc[f] += wb[f];
  } else if constexpr (P == 2) {
#pragma unroll
    for (int j = 0; j < 15; ++j) {
      const int f = w2q(j, 0), x = w2q(j, 1), kind = w2q(j, 2);
      const double m = kind == 1 ? 4.0 * l[x] - 1.0 : 4.0 * l[x];
      acc[j] += m * wb[f];
    }
  } else {
#pragma unroll
    for (int j = 0; j < 36; ++j) {
      int f;
      const double m = w2_p3<Fast>(j, l, f);
      acc[j] += m * wb[f];
    }
  }
}

// fl[t][j] = scale_t sum_q w_q W2_j(l_q) . B(x_tq); Bq [nt][nq][3]
template <int P>
__global__ void __launch_bounds__(128) k_w2_load(int32_t nt, int32_t nq, const double* __restrict__ qlam,
                                                 const double* __restrict__ qw, const double* __restrict__ scale,
                                                 double inv_mu0, const double* __restrict__ geom,
                                                 const double* __restrict__ Bq, double* __restrict__ fl) {
  constexpr int N2 = Nloc<P>::n2;
  for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    TetGeom G;
    load_geom(geom, t, G);
    double acc[N2];
#pragma unroll
    for (int j = 0; j < N2; ++j) acc[j] = 0.0;
    for (int32_t q = 0; q < nq; ++q) {
      double l[4], B[3];
#pragma unroll
      for (int k = 0; k < 4; ++k) l[k] = __ldg(qlam + 4 * q + k);
#pragma unroll
      for (int k = 0; k < 3; ++k) B[k] = __ldg(Bq + ((size_t)t * nq + q) * 3 + k);
      w2_load_point<P>(G, l, B, __ldg(qw + q), acc);
    }
    const double s = __ldg(scale + t) * inv_mu0;
#pragma unroll
    for (int j = 0; j < N2; ++j) fl[(size_t)t * N2 + j] = s * acc[j];
  }
}

// Divergence diagnostic of a W2 field b: per tet the moments of div b against
// the order-p volume functions, m_i = s_t sum_j Dref[i][j] b_j (s_t the sign
// of det J; the W3 span every degree p-1 polynomial, so m = 0 iff div b = 0 on
// the tet), and the size of their terms a_i = sum_j |Dref[i][j] b_j|:
// out[0] += sum m_i^2, out[1] += sum a_i^2 (the norms the caller compares).
template <int P>
__global__ void __launch_bounds__(256) k_divb(int32_t nt, const double* __restrict__ geom,
                                              const int32_t* __restrict__ dof2, const double* __restrict__ b,
                                              const double* __restrict__ dref, int32_t n3, double* out) {
  constexpr int N2 = Nloc<P>::n2;
  double s0 = 0.0, s1 = 0.0;
  for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    const double* g = geom + (size_t)t * 16;
    const double det = g[3] * (g[7] * g[11] - g[8] * g[10]) - g[4] * (g[6] * g[11] - g[8] * g[9]) +
                       g[5] * (g[6] * g[10] - g[7] * g[9]);
    const double sg = det > 0.0 ? 1.0 : -1.0;
    double bv[N2];
#pragma unroll
    for (int j = 0; j < N2; ++j) bv[j] = __ldg(b + __ldg(dof2 + (size_t)t * N2 + j));
    for (int32_t i = 0; i < n3; ++i) {
      double m = 0.0, a = 0.0;
#pragma unroll
      for (int j = 0; j < N2; ++j) {
        const double v = __ldg(dref + (size_t)i * N2 + j) * bv[j];
        m += v;
        a += fabs(v);
      }
      s0 += (sg * m) * (sg * m);
      s1 += a * a;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, s0);
    atomicAdd(out + 1, s1);
  }
}

// sum over the block (fixed shuffle tree, then warps in order); valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
  __syncthreads();
  return s;
}

// y = A x with per-block partials part[2b] = sum_r d_r y_r and, when SQ,
// part[2b+1] = sum_r x_r^2 (x square: A n x n).  Skipped once sc[kCgDone] is set.
template <int LPR, bool SQ>
__global__ void __launch_bounds__(kRedThreads) k_spmv_dot(CsrView A, const double* __restrict__ x,
                                                          double* __restrict__ y, const double* __restrict__ d,
                                                          double* __restrict__ part, const double* __restrict__ sc) {
  __shared__ double sh[kRedThreads / 32];
  if (sc && sc[kCgDone] != 0.0) return;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = gid % LPR;
  const int groups = gridDim.x * blockDim.x / LPR;
  double a1 = 0.0, a2 = 0.0;
  for (int r = gid / LPR;; r += groups) {
    const bool act = r < A.n_rows;
    if (!__any_sync(0xffffffffu, act)) break;
    double s = 0.0;
    if (act) {
      const int beg = __ldg(A.rp + r), end = __ldg(A.rp + r + 1);
      for (int k = beg + lane; k < end; k += LPR) s = fma(__ldg(A.v + k), __ldg(x + __ldg(A.ci + k)), s);
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LPR);
    if (act && lane == 0) {
      y[r] = s;
      a1 = fma(d[r], s, a1);
      if (SQ) a2 = fma(x[r], x[r], a2);
    }
  }
  const double s1 = block_sum(a1, sh);
  const double s2 = SQ ? block_sum(a2, sh) : 0.0;
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s1;
    part[2 * blockIdx.x + 1] = s2;
  }
}

// the kRedGrid partials (pairs), summed in a fixed order by one block
__device__ __forceinline__ void sum_partials(const double* part, double* sh, double* o1, double* o2) {
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < kRedGrid; k += blockDim.x) {
    a += part[2 * k];
    b += part[2 * k + 1];
  }
  const double s1 = block_sum(a, sh);
  const double s2 = block_sum(b, sh);
  if (threadIdx.x == 0) {
    *o1 = s1;
    *o2 = s2;
  }
}

// start of a solve from x = 0: the partials hold r.z and r.r of r = rhs
__global__ void __launch_bounds__(kRedThreads) k_cg_start(double* sc, const double* part, double tol2) {
  __shared__ double sh[kRedThreads / 32];
  double rz, rr;
  sum_partials(part, sh, &rz, &rr);
  if (threadIdx.x == 0) {
    sc[kCgRZ] = rz;
    sc[kCgRR] = rr;
    sc[kCgBB] = rr;
    sc[kCgTol2] = tol2;
    sc[kCgIt] = 0.0;
    sc[kCgAlpha] = sc[kCgBeta] = 0.0;
    sc[kCgDone] = rr == 0.0 ? 1.0 : 0.0;
  }
}

// alpha = r.z / p.q (the partials hold p.q); a non-positive p.q ends the solve (flag 2)
__global__ void __launch_bounds__(kRedThreads) k_cg_alpha(double* sc, const double* part) {
  __shared__ double sh[kRedThreads / 32];
  if (sc[kCgDone] != 0.0) return;
  double pq, unused;
  sum_partials(part, sh, &pq, &unused);
  if (threadIdx.x == 0) {
    if (pq > 0.0)
      sc[kCgAlpha] = sc[kCgRZ] / pq;
    else
      sc[kCgDone] = 2.0;
  }
}

// beta = r.z_new / r.z (the partials hold the new r.z and r.r); converged
// (flag 1) once r.r <= tol^2 rhs.rhs, iteration cap reached (flag 3)
__global__ void __launch_bounds__(kRedThreads) k_cg_beta(double* sc, const double* part, int32_t max_it) {
  __shared__ double sh[kRedThreads / 32];
  if (sc[kCgDone] != 0.0) return;
  double rz, rr;
  sum_partials(part, sh, &rz, &rr);
  if (threadIdx.x == 0) {
    const double it = sc[kCgIt] + 1.0;
    sc[kCgIt] = it;
    sc[kCgRR] = rr;
    sc[kCgBeta] = rz / sc[kCgRZ];
    sc[kCgRZ] = rz;
    if (rr <= sc[kCgTol2] * sc[kCgBB])
      sc[kCgDone] = 1.0;
    else if (it >= (double)max_it)
      sc[kCgDone] = 3.0;
  }
}

// x += alpha p; r -= alpha q
__global__ void k_cg_xr(int32_t n, const double* __restrict__ sc, const double* __restrict__ p,
                        const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r) {
  if (sc[kCgDone] != 0.0) return;
  const double a = sc[kCgAlpha];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] = fma(a, p[i], x[i]);
    r[i] = fma(-a, q[i], r[i]);
  }
}

// x -= alpha u
__global__ void k_cg_sub(int32_t n, const double* __restrict__ sc, const double* __restrict__ u,
                         double* __restrict__ x) {
  if (sc[kCgDone] != 0.0) return;
  const double a = sc[kCgAlpha];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] = fma(-a, u[i], x[i]);
}

// p = z + beta p
__global__ void k_cg_p(int32_t n, const double* __restrict__ sc, const double* __restrict__ z, double* __restrict__ p) {
  if (sc[kCgDone] != 0.0) return;
  const double be = sc[kCgBeta];
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = fma(be, p[i], z[i]);
}

}  // namespace dev
}  // namespace fempic
