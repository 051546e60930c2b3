// Sparse linear algebra on the device: CSR products, the Newmark right-hand
// side, the magnetic update and a persistent preconditioned conjugate-gradient
// solve whose blocks synchronise through a bounded grid barrier (one
// cooperative launch per solve; the host never sees the iterations).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace fempic {
namespace dev {

struct CsrView {
  int32_t n_rows;
  const int32_t* rp;
  const int32_t* ci;
  const double* v;
};

// 2x2-block CSR: block row k holds DOF rows 2k, 2k+1; each block is stored
// row-major (a00 a01 a10 a11) and multiplies DOFs 2c, 2c+1 of block column c
struct BsrView {
  int32_t nb;
  const int32_t* rp;
  const int32_t* ci;
  const double* v;
};

// 2x2-block CSR with FP32 values (the CG's direction products)
struct BsrView32 {
  int32_t nb;
  const int32_t* rp;
  const int32_t* ci;
  const float* v;
};

// 2x2-block matrix with bfloat16 values (the upper 16 bits of the FP32
// value, rounded to nearest even), four per block: the smoother's products
struct BsrView16 {
  int32_t nb;
  const int32_t* rp;
  const int32_t* ci;
  const uint16_t* v;
};

// FP32 -> bfloat16 bits, rounded to nearest even (finite values)
__global__ void k_to_bf16(int64_t n, const float* __restrict__ in, uint16_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t u = __float_as_uint(in[i]);
    out[i] = (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
  }
}

// largest Chebyshev degree of the preconditioner's polynomial parts
constexpr int kMaxCheb = 8;

// FP32 values: used for the preconditioner's auxiliary-space operators
struct CsrView32 {
  int32_t n_rows;
  const int32_t* rp;
  const int32_t* ci;
  const float* v;
};

// Power iteration for the largest eigenvalue of B^-1 A (B: the 2x2 diagonal
// blocks of A, inverted in binv): a start vector from an integer hash
// (SplitMix64 finaliser), x <- B^-1 y block by block, and the two dot
// products of the Rayleigh quotient x.(A x) / x.(B x).
__global__ void k_hash_vector(int32_t n, double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = (double)(z >> 11) * 0x1.0p-52 - 1.0;
  }
}
// Chebyshev coefficients of the smoother from the Rayleigh quotient rq[0] /
// rq[1] (one thread): the interval [l / ratio, l] with l = margin * lambda, as
// for the auxiliary problems; a quotient that is not positive and finite
// leaves 1/theta = 1 and no further steps, i.e. the block Jacobi B^-1 r.
__global__ void k_smooth_coeffs(const double* rq, int k, double margin, double ratio, float* c) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int i = 0; i < 3 * kMaxCheb; ++i) c[i] = 0.f;
  const double lam = rq[1] > 0.0 ? rq[0] / rq[1] : 0.0;
  if (!(lam > 0.0) || !isfinite(lam) || k <= 1) {
    c[0] = 1.f;
    return;
  }
  const double lmax = margin * lam, lmin = lmax / ratio, th = 0.5 * (lmax + lmin), de = 0.5 * (lmax - lmin);
  const double sig = th / de;
  double rho = 1.0 / sig;
  c[0] = (float)(1.0 / th);
  for (int i = 1; i < k && i < kMaxCheb; ++i) {
    const double rn = 1.0 / (2.0 * sig - rho);
    c[kMaxCheb + i] = (float)(rn * rho);
    c[2 * kMaxCheb + i] = (float)(2.0 * rn / de);
    rho = rn;
  }
}
__global__ void k_block_apply(int32_t nb, const double* __restrict__ binv, const double* __restrict__ y,
                              double* __restrict__ x) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += (int64_t)gridDim.x * blockDim.x) {
    const double y0 = y[2 * k], y1 = y[2 * k + 1];
    x[2 * k] = fma(binv[4 * k], y0, binv[4 * k + 1] * y1);
    x[2 * k + 1] = fma(binv[4 * k + 2], y0, binv[4 * k + 3] * y1);
  }
}
__global__ void k_dot2(int32_t n, const double* __restrict__ x, const double* __restrict__ y0,
                       const double* __restrict__ y1, double* out) {
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    s0 = fma(x[i], y0[i], s0);
    s1 = fma(x[i], y1[i], s1);
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

__global__ void k_to_f32(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// y = alpha * A x (+ beta * y)
template <int LPR>
__global__ void k_spmv(CsrView A, const double* __restrict__ x, double* __restrict__ y, double alpha, double beta) {
  int gid = blockIdx.x * blockDim.x + threadIdx.x;
  int lane = gid % LPR;
  int groups = gridDim.x * blockDim.x / LPR;
  for (int r = gid / LPR; ; r += groups) {
    bool act = r < A.n_rows;
    if (!__any_sync(0xffffffffu, act)) break;
    double s = 0.0;
    if (act) {
      int beg = __ldg(A.rp + r), end = __ldg(A.rp + r + 1);
      for (int k = beg + lane; k < end; k += LPR) s = fma(__ldg(A.v + k), __ldg(x + __ldg(A.ci + k)), s);
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LPR);
    if (act && lane == 0) y[r] = beta == 0.0 ? alpha * s : fma(beta, y[r], alpha * s);
  }
}

// Newmark right-hand side, one row per LPR lanes:
//   rhs = R1 e - R2 e_prev + qfac (Q b) - (dg - dgp_fac dg_prev), PEC rows 0.
// R1, R2 share M's pattern (R2 may be null).
template <int LPR>
__global__ void k_rhs(CsrView R1, const double* __restrict__ r2v, CsrView Q, const double* __restrict__ e,
                      const double* __restrict__ e_prev, const double* __restrict__ b, double qfac,
                      const double* __restrict__ dg, const double* __restrict__ dg_prev, double dgp_fac,
                      const uint8_t* __restrict__ pec, double* __restrict__ rhs) {
  int gid = blockIdx.x * blockDim.x + threadIdx.x;
  int lane = gid % LPR;
  int groups = gridDim.x * blockDim.x / LPR;
  int n = R1.n_rows;
  for (int r = gid / LPR; ; r += groups) {
    bool act = r < n;
    if (!__any_sync(0xffffffffu, act)) break;
    double s = 0.0;
    if (act) {
      int beg = __ldg(R1.rp + r), end = __ldg(R1.rp + r + 1);
      for (int k = beg + lane; k < end; k += LPR) {
        int c = __ldg(R1.ci + k);
        s = fma(__ldg(R1.v + k), __ldg(e + c), s);
        if (r2v) s = fma(-__ldg(r2v + k), __ldg(e_prev + c), s);
      }
      if (qfac != 0.0) {
        double t = 0.0;
        int qb = __ldg(Q.rp + r), qe = __ldg(Q.rp + r + 1);
        for (int k = qb + lane; k < qe; k += LPR) t = fma(__ldg(Q.v + k), __ldg(b + __ldg(Q.ci + k)), t);
        s = fma(qfac, t, s);
      }
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LPR);
    if (act && lane == 0) {
      double src = dg[r];
      if (dgp_fac != 0.0) src -= dgp_fac * dg_prev[r];
      rhs[r] = pec[r] ? 0.0 : s - src;
    }
  }
}

// b -= hdt * C (e_new + e)
template <int LPR>
__global__ void k_bupdate(CsrView C, const double* __restrict__ e_new, const double* __restrict__ e, double hdt,
                          double* __restrict__ b) {
  int gid = blockIdx.x * blockDim.x + threadIdx.x;
  int lane = gid % LPR;
  int groups = gridDim.x * blockDim.x / LPR;
  int n = C.n_rows;
  for (int r = gid / LPR; ; r += groups) {
    bool act = r < n;
    if (!__any_sync(0xffffffffu, act)) break;
    double s = 0.0;
    if (act) {
      int beg = __ldg(C.rp + r), end = __ldg(C.rp + r + 1);
      for (int k = beg + lane; k < end; k += LPR) {
        int c = __ldg(C.ci + k);
        s = fma(__ldg(C.v + k), __ldg(e_new + c) + __ldg(e + c), s);
      }
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LPR);
    if (act && lane == 0) b[r] = fma(-hdt, s, b[r]);
  }
}

// out = a x + b y
__global__ void k_lincomb(int32_t n, const double* __restrict__ x, const double* __restrict__ y, double a, double b,
                          double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = a * x[i] + b * y[i];
}

// dinvV = 1 / (dvM + c dvK), 0 where the sum vanishes (FP32 for the preconditioner)
__global__ void k_form_dv(int32_t n, const double* dvm, const double* dvk, double c, float* dinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = dvm[i] + c * dvk[i];
  dinv[i] = d > 0.0 ? (float)(1.0 / d) : 0.f;
}

// out = (float)(a + c b), elementwise
__global__ void k_axpy_to_f32(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double c,
                              float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)(a[i] + c * b[i]);
}

// A = M + ca K + ia I, R = M + cr K + ir I (one pattern; I, the surface
// impedance matrix, may be null), inverse diagonal of A (0 on empty rows)
__global__ void k_form_system(int32_t n, const int32_t* rp, const int32_t* ci, const double* m, const double* k,
                              double ca, double cr, double* a, double* r, double* dinv, const double* iv = nullptr,
                              double ia = 0.0, double ir = 0.0) {
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  double diag = 0.0;
  for (int j = rp[row]; j < rp[row + 1]; ++j) {
    double av = m[j] + ca * k[j];
    double rv = m[j] + cr * k[j];
    if (iv) {
      av += ia * iv[j];
      rv += ir * iv[j];
    }
    a[j] = av;
    if (r) r[j] = rv;
    if (ci[j] == row) diag = av;
  }
  dinv[row] = diag != 0.0 ? 1.0 / diag : 0.0;
}

// 2x2 blocks: Ab = bM + c bK and the inverse of each diagonal block (0 if absent)
__global__ void k_form_blocks(int32_t nb, const int32_t* rp, const int32_t* ci, const double* bm, const double* bk,
                              double c, double* ab, double* binv, const double* bi = nullptr, double ci_ = 0.0) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  double d[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = rp[k]; j < rp[k + 1]; ++j) {
    for (int q = 0; q < 4; ++q)
      ab[4 * j + q] = bi ? bm[4 * j + q] + c * bk[4 * j + q] + ci_ * bi[4 * j + q] : bm[4 * j + q] + c * bk[4 * j + q];
    if (ci[j] == k)
      for (int q = 0; q < 4; ++q) d[q] = ab[4 * j + q];
  }
  double det = d[0] * d[3] - d[1] * d[2];
  if (det != 0.0) {
    binv[4 * k + 0] = d[3] / det;
    binv[4 * k + 1] = -d[1] / det;
    binv[4 * k + 2] = -d[2] / det;
    binv[4 * k + 3] = d[0] / det;
  } else {
    binv[4 * k + 0] = binv[4 * k + 1] = binv[4 * k + 2] = binv[4 * k + 3] = 0.0;
  }
}

__global__ void k_inv_diag(int32_t n, const int32_t* rp, const int32_t* ci, const double* v, double* dinv) {
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  double diag = 0.0;
  for (int j = rp[row]; j < rp[row + 1]; ++j)
    if (ci[j] == row) diag = v[j];
  dinv[row] = diag != 0.0 ? 1.0 / diag : 0.0;
}

// Inverse of each diagonal block of A over a contiguous DOF group (at most 6
// DOFs: the W1 DOFs of one edge, face or tet interior at order 3) by Cholesky,
// written to the rows of Bg (each row holds its group's columns in order);
// a group without a diagonal (PEC rows) gets zeros, a block that is not
// numerically positive definite its diagonal inverse.
constexpr int kMaxGroup = 6;
__global__ void k_group_inverse(int32_t ng, const int32_t* __restrict__ gstart, const uint8_t* __restrict__ gsize,
                                CsrView A, const int32_t* __restrict__ brp, double* __restrict__ bval) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ng) return;
  const int s0 = gstart[g], n = gsize[g];
  double B[kMaxGroup][kMaxGroup], L[kMaxGroup][kMaxGroup], X[kMaxGroup][kMaxGroup];
  for (int r = 0; r < kMaxGroup; ++r)
    for (int c = 0; c < kMaxGroup; ++c) B[r][c] = L[r][c] = X[r][c] = 0.0;
  for (int r = 0; r < n; ++r)
    for (int k = A.rp[s0 + r]; k < A.rp[s0 + r + 1]; ++k) {
      const int c = A.ci[k] - s0;
      if (c >= 0 && c < n) B[r][c] = A.v[k];
    }
  bool spd = B[0][0] > 0.0;
  for (int j = 0; j < n && spd; ++j) {
    double d = B[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0)) {
      spd = false;
      break;
    }
    L[j][j] = sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      double t = B[i][j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / L[j][j];
    }
  }
  if (spd) {
    for (int c = 0; c < n; ++c) {  // column c of B^-1 = L^-T L^-1 e_c
      double y[kMaxGroup];
      for (int i = 0; i < n; ++i) {
        double t = i == c ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
        y[i] = t / L[i][i];
      }
      for (int i = n - 1; i >= 0; --i) {
        double t = y[i];
        for (int k = i + 1; k < n; ++k) t -= L[k][i] * X[k][c];
        X[i][c] = t / L[i][i];
      }
    }
  } else {
    for (int r = 0; r < n; ++r) X[r][r] = B[r][r] != 0.0 ? 1.0 / B[r][r] : 0.0;
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) bval[brp[s0 + r] + c] = X[r][c];
}

// ---- persistent PCG ---------------------------------------------------------
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};

#ifndef FEMPIC_BARRIER_SPIN_LIMIT
#define FEMPIC_BARRIER_SPIN_LIMIT 20000000  // ~1-2 s with the backoff below
#endif
constexpr long long kBarrierSpinLimit = FEMPIC_BARRIER_SPIN_LIMIT;

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) { return *(volatile const unsigned*)p; }

// Returns false (and latches kStatusBarrier) if the barrier timed out.
// Test builds with FEMPIC_TEST_ABSENT_CTA = b: CTA b never arrives (it leaves
// the kernel at its first barrier), so every other CTA's wait runs into the
// spin limit; nothing else changes.
__device__ bool grid_sync(GridBarrier* bar, int32_t* status) {
  __shared__ int ok;
  __syncthreads();
#ifdef FEMPIC_TEST_ABSENT_CTA
  if (blockIdx.x == FEMPIC_TEST_ABSENT_CTA) return false;
#endif
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned gen = ld_volatile(&bar->gen);
    __threadfence();
    unsigned arrived = atomicAdd(&bar->count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long spins = 0;
      while (ld_volatile(&bar->gen) == gen) {
        if (++spins > kBarrierSpinLimit) {
          atomicOr(status, kStatusBarrier);
          ok = 0;
          break;
        }
        if (spins > 64) __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}


struct PcgArgs {
  CsrView A;
  const double* dinv;
  // optional auxiliary-space corrections of the preconditioner, applied in
  // FP32: z = dinv r + D (dinvL (D^T r)) + Pi (dinvV (Pi^T r));
  // DT.n_rows == 0 disables both
  CsrView32 D;
  CsrView32 DT;
  const float* dinvL;
  float* t;    // [DT.n_rows] scratch
  CsrView32 Pi;
  CsrView32 PiT;
  const float* dinvV;
  float* u;    // [PiT.n_rows] scratch
  // Chebyshev smoothing of the two auxiliary problems L y = D^T r and
  // V y = Pi^T r (L = D^T M D, V = Pi^T A Pi, FP32, Jacobi-scaled): cheb_k
  // steps of the Chebyshev iteration from y = 0; cheb_k = 1 is the diagonal
  // scaling alone.  t/u hold the iterate, t2/u2 its second buffer, tf/uf the
  // right-hand sides, td/ud the last Chebyshev step.
  CsrView32 L;
  CsrView32 V;
  float *tf, *td, *t2;
  float *uf, *ud, *u2;
  int cheb_k;
  float chebL[3][kMaxCheb];  // [0][0] = 1/theta; [1][i], [2][i]: step i coefficients
  float chebV[3][kMaxCheb];
  float* q32;  // unused by k_pcg (its q shadow lives in r32)
  float* r32;  // [2][n] pairs (r_i, q_i): FP32 shadows of r and q, the inputs of the auxiliary products
  double* red; // [3][4] reduction slots, zeroed before the launch
  // order 2: the system matrix in 2x2 blocks and the inverses of its
  // diagonal blocks (block Jacobi); Ab.nb == 0 uses A and dinv
  BsrView Ab;
  const double* binv;
  // FP32 direction products (order 2): q = A p with A and p rounded to FP32
  // and summed in FP32; every `repl` iterations, and before convergence is
  // accepted, the residual is recomputed in FP64 as rhs - A x.  Ab32.nb == 0
  // keeps the FP64 products.
  BsrView32 Ab32;
  float* p32;
  int repl;
  // Chebyshev smoother of degree smooth_k on B^-1 A in place of the block
  // Jacobi term B^-1 r (order 2 with an FP32 copy of A; smooth_k = 1 keeps
  // B^-1 r): y_1 = B^-1 r / theta, y_{i+1} = y_i + d_{i+1} with
  // d_{i+1} = c1_i d_i + c2_i B^-1 (r - A y_i), the FP32 product A y_i run in
  // the i-th further phase of the auxiliary Chebyshev steps (no barrier of its
  // own) with A's values rounded to bfloat16 (host study: the same iteration
  // count as with FP64 values); a fixed polynomial in B^-1 A times B^-1, so the preconditioner stays
  // symmetric.  sy: [2][n] iterate (double-buffered), sd: [n] last step.
  int smooth_k;
  BsrView16 As16;      // A with bfloat16 values for the smoother's products
  const float* binv32; // FP32 copy of binv (the smoother runs in FP32 throughout)
  const float* chebS;  // [3 * kMaxCheb] on the device: [0] = 1/theta; [kMaxCheb + i], [2 kMaxCheb + i]: step i
  float* sy;
  float* sd;
  // order 3: inverses of A's diagonal blocks over the W1 DOFs of one edge, one
  // face and one tet interior, as a CSR (rows of a group hold its columns);
  // n_rows == 0 keeps the point Jacobi dinv
  CsrView Bg;
  const int32_t* Apart;  // [gridDim.x + 1] per-CTA row ranges of A (block rows at order 2), or null
  const double* rhs;
  double* x;   // in: initial guess, out: solution
  double* r[2];  // residual, double-buffered
  double* z;
  double* p[2];  // search direction, double-buffered
  double* q;
  double* partials[2];  // [gridDim.x * 4] each, used alternately
  GridBarrier* bar;
  int32_t* status;
  int32_t* iters_out;
  double* res_out;
  double rtol;
  int max_it;
};

// reduce up to 4 values over the block into partials[blockIdx.x*4 + k]
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* partials) {
  __shared__ double red[32][4];
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[w][k] = v[k];
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = l < nw ? red[l][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (l == 0) partials[blockIdx.x * 4 + k] = s;
    }
  }
  __syncthreads();
}

// Grid-wide sums through a ring of three accumulator slots: every CTA adds its
// block total with one atomic; after the next grid barrier every CTA reads the
// same value.  Slot k+1 is cleared by CTA 0 while slot k is being filled: its
// last readers finished before the previous barrier.
template <int NV>
__device__ __forceinline__ void grid_sum_add(double (&v)[NV], double* red, int k) {
  __shared__ double tot_sh[4];
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  __shared__ double wsum[64][4];
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) wsum[w][q] = v[q];
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = (l < nw ? wsum[l][q] : 0.0) + (l + 32 < nw ? wsum[l + 32][q] : 0.0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (l == 0) tot_sh[q] = s;
    }
    if (l == 0) {
      if (blockIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[((k + 1) % 3) * 4 + q] = 0.0;
#pragma unroll
      for (int q = 0; q < NV; ++q) atomicAdd(red + (k % 3) * 4 + q, tot_sh[q]);
    }
  }
  __syncthreads();
}

template <int NV>
__device__ __forceinline__ void grid_sum_read(const double* red, int k, double (&tot)[NV]) {
#pragma unroll
  for (int q = 0; q < NV; ++q) tot[q] = __ldcg(red + (k % 3) * 4 + q);
}

// every block sums the partials in the same order -> identical totals everywhere
template <int NV>
__device__ __forceinline__ void grid_totals(const double* partials, double (&tot)[NV]) {
  __shared__ double res[4];
  if (threadIdx.x < 32) {
    int l = threadIdx.x;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int b = l; b < (int)gridDim.x; b += 32) s += __ldcg(partials + b * 4 + k);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (l == 0) res[k] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = res[k];
  __syncthreads();
}

// ---- row products ------------------------------------------------------------
// Each "row body" computes one row with a group of LPR lanes (lane = index in
// the group; all 32 lanes of the warp call it together, act = this group has a
// row) and emits the result from lane 0 of the group.  Two drivers hand out
// the rows: a static grid stride (rows_*), and a dynamic one (for_rows) in
// which each CTA owns a contiguous range and its warps take the next pass of
// 32 / LPR rows from a shared-memory counter.

// y_r = sum_k A_rk f(k), FP64 CSR
template <int LPR, class X, class F>
__device__ __forceinline__ void spmv_row(const CsrView& A, int r0, bool act, int lane, X x_of, F emit) {
  double s = 0.0;
  if (act) {
    int beg = __ldg(A.rp + r0), end = __ldg(A.rp + r0 + 1);
    for (int k = beg + lane; k < end; k += LPR) s = fma(__ldg(A.v + k), x_of(__ldg(A.ci + k)), s);
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LPR);
  if (act && lane == 0) emit(r0, s);
}

// block row k0 of a 2x2-block matrix times a vector (two blocks per lane and
// pass with FEMPIC_BSPMV_UNROLL2)
#ifndef FEMPIC_BSPMV_UNROLL2
#define FEMPIC_BSPMV_UNROLL2 1
#endif
template <int LPR, class F>
__device__ __forceinline__ void bspmv_row(const BsrView& A, const double* x, int k0, bool act, int lane, F emit) {
  const double2* x2 = reinterpret_cast<const double2*>(x);
  const double2* v2 = reinterpret_cast<const double2*>(A.v);
  double s0 = 0.0, s1 = 0.0;
  if (act) {
    int beg = __ldg(A.rp + k0), end = __ldg(A.rp + k0 + 1);
#if FEMPIC_BSPMV_UNROLL2
    int j = beg + lane;
    for (; j + LPR < end; j += 2 * LPR) {
      const int c0 = __ldg(A.ci + j), c1 = __ldg(A.ci + j + LPR);
      const double2 x0 = __ldcg(x2 + c0), x1 = __ldcg(x2 + c1);
      const double2 a01 = __ldg(v2 + 2 * j), a23 = __ldg(v2 + 2 * j + 1);
      const double2 b01 = __ldg(v2 + 2 * (j + LPR)), b23 = __ldg(v2 + 2 * (j + LPR) + 1);
      s0 = fma(a01.x, x0.x, fma(a01.y, x0.y, s0));
      s1 = fma(a23.x, x0.x, fma(a23.y, x0.y, s1));
      s0 = fma(b01.x, x1.x, fma(b01.y, x1.y, s0));
      s1 = fma(b23.x, x1.x, fma(b23.y, x1.y, s1));
    }
    if (j < end) {
      const int c = __ldg(A.ci + j);
      const double2 xv = __ldcg(x2 + c);
      const double2 a01 = __ldg(v2 + 2 * j), a23 = __ldg(v2 + 2 * j + 1);
      s0 = fma(a01.x, xv.x, fma(a01.y, xv.y, s0));
      s1 = fma(a23.x, xv.x, fma(a23.y, xv.y, s1));
    }
#else
    for (int j = beg + lane; j < end; j += LPR) {
      int c = __ldg(A.ci + j);
      double2 xv = __ldcg(x2 + c);
      double2 a01 = __ldg(v2 + 2 * j), a23 = __ldg(v2 + 2 * j + 1);
      s0 = fma(a01.x, xv.x, fma(a01.y, xv.y, s0));
      s1 = fma(a23.x, xv.x, fma(a23.y, xv.y, s1));
    }
#endif
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o, LPR);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o, LPR);
  }
  if (act && lane == 0) emit(k0, s0, s1);
}

// block row k0 of the FP32 2x2-block matrix times an FP32 vector, summed in
// FP32 (two blocks per lane and pass, as bspmv_row)
template <int LPR, class F>
__device__ __forceinline__ void bspmv32_row(const BsrView32& A, const float* x, int k0, bool act, int lane, F emit) {
  const float2* x2 = reinterpret_cast<const float2*>(x);
  const float4* v4 = reinterpret_cast<const float4*>(A.v);
  float s0 = 0.f, s1 = 0.f;
  if (act) {
    const int beg = __ldg(A.rp + k0), end = __ldg(A.rp + k0 + 1);
    int j = beg + lane;
    for (; j + LPR < end; j += 2 * LPR) {
      const int c0 = __ldg(A.ci + j), c1 = __ldg(A.ci + j + LPR);
      const float2 x0 = __ldcg(x2 + c0), x1 = __ldcg(x2 + c1);
      const float4 a = __ldg(v4 + j), b = __ldg(v4 + j + LPR);
      s0 = fmaf(a.x, x0.x, fmaf(a.y, x0.y, s0));
      s1 = fmaf(a.z, x0.x, fmaf(a.w, x0.y, s1));
      s0 = fmaf(b.x, x1.x, fmaf(b.y, x1.y, s0));
      s1 = fmaf(b.z, x1.x, fmaf(b.w, x1.y, s1));
    }
    if (j < end) {
      const int c = __ldg(A.ci + j);
      const float2 xv = __ldcg(x2 + c);
      const float4 a = __ldg(v4 + j);
      s0 = fmaf(a.x, xv.x, fmaf(a.y, xv.y, s0));
      s1 = fmaf(a.z, xv.x, fmaf(a.w, xv.y, s1));
    }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o, LPR);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o, LPR);
  }
  if (act && lane == 0) emit(k0, s0, s1);
}

// block row k0 of the bfloat16 2x2-block matrix times an FP32 vector, summed
// in FP32 (as bspmv32_row; the four values of a block are one 8-byte load)
template <int LPR, class F>
__device__ __forceinline__ void bspmv16_row(const BsrView16& A, const float* x, int k0, bool act, int lane, F emit) {
  const float2* x2 = reinterpret_cast<const float2*>(x);
  const uint2* v2 = reinterpret_cast<const uint2*>(A.v);
  float s0 = 0.f, s1 = 0.f;
  auto acc = [&](const uint2 w, const float2 xv) {
    s0 = fmaf(__uint_as_float(w.x << 16), xv.x, fmaf(__uint_as_float(w.x & 0xFFFF0000u), xv.y, s0));
    s1 = fmaf(__uint_as_float(w.y << 16), xv.x, fmaf(__uint_as_float(w.y & 0xFFFF0000u), xv.y, s1));
  };
  if (act) {
    const int beg = __ldg(A.rp + k0), end = __ldg(A.rp + k0 + 1);
    int j = beg + lane;
    for (; j + LPR < end; j += 2 * LPR) {
      const int c0 = __ldg(A.ci + j), c1 = __ldg(A.ci + j + LPR);
      const float2 x0 = __ldcg(x2 + c0), x1 = __ldcg(x2 + c1);
      const uint2 a = __ldg(v2 + j), b = __ldg(v2 + j + LPR);
      acc(a, x0);
      acc(b, x1);
    }
    if (j < end) acc(__ldg(v2 + j), __ldcg(x2 + __ldg(A.ci + j)));
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o, LPR);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o, LPR);
  }
  if (act && lane == 0) emit(k0, s0, s1);
}

// FP32 row: each lane loads FEMPIC_SPMV32_UNROLL entries (column, value)
// before it gathers them, so that the dependent index -> vector loads of
// several entries overlap
#ifndef FEMPIC_SPMV32_UNROLL
#define FEMPIC_SPMV32_UNROLL 4
#endif
template <int LPR, class X, class F>
__device__ __forceinline__ void spmv32_row(const CsrView32& A, int r0, bool act, int lane, X x_of, F emit) {
  constexpr int U = FEMPIC_SPMV32_UNROLL;
  float s = 0.f;
  if (act) {
    int beg = __ldg(A.rp + r0), end = __ldg(A.rp + r0 + 1);
    if (U == 1) {
      for (int k = beg + lane; k < end; k += LPR) s = fmaf(__ldg(A.v + k), x_of(__ldg(A.ci + k)), s);
    } else {
      for (int k0 = beg + lane; k0 < end; k0 += U * LPR) {
        int c[U];
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int k = k0 + u * LPR;
          c[u] = k < end ? __ldg(A.ci + k) : -1;
          v[u] = k < end ? __ldg(A.v + k) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (c[u] >= 0) s = fmaf(v[u], x_of(c[u]), s);
      }
    }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LPR);
  if (act && lane == 0) emit(r0, s);
}

// As spmv32_row, with the row's epilogue operands loaded before its entries:
// pre(r0) (lane 0 of the row's group) returns them and emit(r0, sum, pre
// values) uses them, so their loads overlap the row's index -> vector loads
// instead of following the reduction.
#ifndef FEMPIC_CHEB_PREFETCH
#define FEMPIC_CHEB_PREFETCH 1
#endif
#ifndef FEMPIC_RESTRICT_PREFETCH
#define FEMPIC_RESTRICT_PREFETCH 1
#endif
#ifndef FEMPIC_APROD_PREFETCH
#define FEMPIC_APROD_PREFETCH 1
#endif
template <int LPR, class X, class P, class F>
__device__ __forceinline__ void spmv32_row_pre(const CsrView32& A, int r0, bool act, int lane, X x_of, P pre,
                                               F emit) {
  decltype(pre(0)) pv{};
  if (act && lane == 0) pv = pre(r0);
  spmv32_row<LPR>(A, r0, act, lane, x_of, [&](int r, float s) { emit(r, s, pv); });
}

// static driver: the groups of the grid stride through rows [0, n)
template <int LPR, class Body>
__device__ __forceinline__ void rows_static(int n, int gid, int groups, Body body) {
  const int lane = gid % LPR;
  for (int r0 = gid / LPR; ; r0 += groups) {
    bool act = r0 < n;
    if (!__any_sync(0xffffffffu, act)) break;
    body(r0, act, lane);
  }
}

template <int LPR, class X, class F>
__device__ __forceinline__ void rows_spmv(const CsrView& A, int gid, int groups, X x_of, F emit) {
  rows_static<LPR>(A.n_rows, gid, groups,
                   [&](int r, bool act, int lane) { spmv_row<LPR>(A, r, act, lane, x_of, emit); });
}

template <int LPR, class F>
__device__ __forceinline__ void rows_bspmv(const BsrView& A, const double* x, int gid, int groups, F emit) {
  rows_static<LPR>(A.nb, gid, groups, [&](int k, bool act, int lane) { bspmv_row<LPR>(A, x, k, act, lane, emit); });
}

template <int LPR, class X, class F>
__device__ __forceinline__ void rows_spmv32(const CsrView32& A, int gid, int groups, X x_of, F emit) {
  rows_static<LPR>(A.n_rows, gid, groups,
                   [&](int r, bool act, int lane) { spmv32_row<LPR>(A, r, act, lane, x_of, emit); });
}

// dynamic driver: this CTA's range of rows [0, n) (part[b]..part[b+1], or an
// equal share), handed to its warps in passes of 32 / LPR rows through the
// shared counter ring[id & 7].  The loop resets ring[(id + 4) & 7] for a later
// loop; a counter is reused only four loops later, and at most two loops run
// between grid barriers, so no warp still reads a counter being reset.
template <int LPR, class Body>
__device__ __forceinline__ void for_rows(int n, const int32_t* part, int* ring, int& id, Body body) {
  const int slot = id & 7;
  if (threadIdx.x == 0) ring[(id + 4) & 7] = 0;
  ++id;
  const int rb = part ? __ldg(part + blockIdx.x) : (int)((int64_t)n * blockIdx.x / gridDim.x);
  const int re = part ? __ldg(part + blockIdx.x + 1) : (int)((int64_t)n * (blockIdx.x + 1) / gridDim.x);
  constexpr int RPW = 32 / LPR;
  const int l32 = threadIdx.x & 31;
  for (;;) {
    int c = 0;
    if (l32 == 0) c = atomicAdd(ring + slot, 1);
    c = __shfl_sync(0xffffffffu, c, 0);
    const int r0 = rb + c * RPW;
    if (r0 >= re) break;
    const int r = r0 + l32 / LPR;
    body(r, r < re, l32 % LPR);
  }
}

// Row scheduling of the persistent CG: the static grid stride (default) or,
// with FEMPIC_PCG_DYN, one CTA per SM over an entry-balanced contiguous range
// whose warps take passes from a shared counter.  With the static stride the
// CTAs of each phase finish unevenly (drift tube, A product per CTA 63 / 88 /
// 131 us min / mean / max, later CTAs of an SM slowest); the dynamic form
// evens out the warps of an SM but not the SMs (96 / 105 / 150 us) and runs
// fewer warps per SM, and measured slower (451 vs 385 us per iteration).
#ifndef FEMPIC_PCG_DYN
#define FEMPIC_PCG_DYN 0
#endif
struct PcgSched {
  int gid, tpg;
  int* ring;
  int id;
  template <int LPR, class Body>
  __device__ __forceinline__ void run(int n, const int32_t* part, Body body) {
#if FEMPIC_PCG_DYN
    for_rows<LPR>(n, part, ring, id, body);
#else
    rows_static<LPR>(n, gid, tpg / LPR, body);
#endif
  }
};

// z_i = dinv_i r_i + (D t)_i + (Pi u)_i over the rows (returns this thread's r.z part).
// The row bounds of D and Pi, the residual and the Jacobi block are loaded
// together, and each lane takes two entries of each product per pass, so the
// index -> vector loads of both products overlap.
#ifndef FEMPIC_AUXZ_FUSED
#define FEMPIC_AUXZ_FUSED 1
#endif
#ifndef FEMPIC_AUXZ_PREFETCH
#define FEMPIC_AUXZ_PREFETCH 1
#endif
template <int LPR>
__device__ __forceinline__ double aux_z(const PcgArgs& a, const double* rvec, const float* tv, const float* uv,
                                        PcgSched& sc) {
  const bool vec = a.Pi.n_rows > 0;
  double rz = 0.0;
  sc.run<LPR>(a.D.n_rows, nullptr, [&](int i, bool act, int lane) {
    float s = 0.f;
    // the row's residual and smoother value, loaded ahead of its products
    double rr_pre = 0.0;
    float sy_pre = 0.f;
    if (FEMPIC_AUXZ_PREFETCH && act && lane == 0) {
      rr_pre = __ldcg(rvec + i);
      if (a.smooth_k > 1) sy_pre = __ldcg(a.sy + (size_t)((a.smooth_k - 1) & 1) * a.D.n_rows + i);
    }
    if (act) {
      if (FEMPIC_AUXZ_FUSED) {
        const int db = __ldg(a.D.rp + i), de = __ldg(a.D.rp + i + 1);
        const int pb = vec ? __ldg(a.Pi.rp + i) : 0, pe = vec ? __ldg(a.Pi.rp + i + 1) : 0;
        for (int k0 = lane; db + k0 < de || pb + k0 < pe; k0 += 2 * LPR) {
          const int kd0 = db + k0, kd1 = kd0 + LPR, kp0 = pb + k0, kp1 = kp0 + LPR;
          const int cd0 = kd0 < de ? __ldg(a.D.ci + kd0) : -1, cd1 = kd1 < de ? __ldg(a.D.ci + kd1) : -1;
          const int cp0 = kp0 < pe ? __ldg(a.Pi.ci + kp0) : -1, cp1 = kp1 < pe ? __ldg(a.Pi.ci + kp1) : -1;
          const float vd0 = cd0 >= 0 ? __ldg(a.D.v + kd0) : 0.f, vd1 = cd1 >= 0 ? __ldg(a.D.v + kd1) : 0.f;
          const float vp0 = cp0 >= 0 ? __ldg(a.Pi.v + kp0) : 0.f, vp1 = cp1 >= 0 ? __ldg(a.Pi.v + kp1) : 0.f;
          if (cd0 >= 0) s = fmaf(vd0, __ldcg(tv + cd0), s);
          if (cd1 >= 0) s = fmaf(vd1, __ldcg(tv + cd1), s);
          if (cp0 >= 0) s = fmaf(vp0, __ldcg(uv + cp0), s);
          if (cp1 >= 0) s = fmaf(vp1, __ldcg(uv + cp1), s);
        }
      } else {
        for (int k = __ldg(a.D.rp + i) + lane; k < __ldg(a.D.rp + i + 1); k += LPR)
          s = fmaf(__ldg(a.D.v + k), __ldcg(tv + __ldg(a.D.ci + k)), s);
        if (vec)
          for (int k = __ldg(a.Pi.rp + i) + lane; k < __ldg(a.Pi.rp + i + 1); k += LPR)
            s = fmaf(__ldg(a.Pi.v + k), __ldcg(uv + __ldg(a.Pi.ci + k)), s);
      }
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LPR);
    if (act && lane == 0) {
      double rr = FEMPIC_AUXZ_PREFETCH ? rr_pre : __ldcg(rvec + i);
      double zz;
      if (a.smooth_k > 1) {
        zz = (double)((FEMPIC_AUXZ_PREFETCH ? sy_pre : __ldcg(a.sy + (size_t)((a.smooth_k - 1) & 1) * a.D.n_rows + i)) + s);
      } else if (a.Ab.nb > 0) {
        const int k = i >> 1, par = i & 1;
        double r0 = __ldcg(rvec + 2 * k), r1 = __ldcg(rvec + 2 * k + 1);
        zz = fma(__ldg(a.binv + 4 * k + 2 * par), r0, fma(__ldg(a.binv + 4 * k + 2 * par + 1), r1, (double)s));
      } else if (a.Bg.n_rows > 0) {
        double t = (double)s;
        for (int k = __ldg(a.Bg.rp + i); k < __ldg(a.Bg.rp + i + 1); ++k)
          t = fma(__ldg(a.Bg.v + k), __ldcg(rvec + __ldg(a.Bg.ci + k)), t);
        zz = t;
      } else {
        zz = fma(__ldg(a.dinv + i), rr, (double)s);
      }
      a.z[i] = zz;
      rz += rr * zz;
    }
  });
  return rz;
}

// First iterate of the smoother for block k from the FP32 residual (r0, r1)
// of its two rows: y_1 = d_1 = B_k^-1 r / theta.
__device__ __forceinline__ void smooth_first(const PcgArgs& a, int k, float r0, float r1) {
  const float4 bi = __ldg(reinterpret_cast<const float4*>(a.binv32) + k);
  const float th = __ldg(a.chebS);
  const float y0 = th * fmaf(bi.x, r0, bi.y * r1);
  const float y1 = th * fmaf(bi.z, r0, bi.w * r1);
  a.sy[2 * k] = y0;
  a.sy[2 * k + 1] = y1;
  a.sd[2 * k] = y0;
  a.sd[2 * k + 1] = y1;
}

// Store the first Chebyshev iterate of the auxiliary problems from their
// right-hand sides f = (D^T r)_k or (Pi^T r)_k (the _d forms take the row's
// Jacobi scaling already loaded).
__device__ __forceinline__ void aux_first_t_d(const PcgArgs& a, int k, float f, float dl) {
  const float y = a.chebL[0][0] * dl * f;
  a.t[k] = y;
  if (a.cheb_k > 1) {
    a.tf[k] = f;
    a.td[k] = y;
  }
}
__device__ __forceinline__ void aux_first_u_d(const PcgArgs& a, int k, float f, float dv) {
  const float y = a.chebV[0][0] * dv * f;
  a.u[k] = y;
  if (a.cheb_k > 1) {
    a.uf[k] = f;
    a.ud[k] = y;
  }
}
__device__ __forceinline__ void aux_first_t(const PcgArgs& a, int k, float f) {
  const float y = a.chebL[0][0] * __ldg(a.dinvL + k) * f;
  a.t[k] = y;
  if (a.cheb_k > 1) {
    a.tf[k] = f;
    a.td[k] = y;
  }
}
__device__ __forceinline__ void aux_first_u(const PcgArgs& a, int k, float f) {
  const float y = a.chebV[0][0] * __ldg(a.dinvV + k) * f;
  a.u[k] = y;
  if (a.cheb_k > 1) {
    a.uf[k] = f;
    a.ud[k] = y;
  }
}

// lanes per row of L (rows of ~20-70 entries at order 2) and of V
// lanes per row of the residual's auxiliary products D^T r and Pi^T r
#ifndef FEMPIC_LPR_DT
#define FEMPIC_LPR_DT 8
#endif
// lanes per W1 row of the preconditioner's z phase (D t + Pi u)
#ifndef FEMPIC_LPR_Z
#define FEMPIC_LPR_Z 4
#endif
#ifndef FEMPIC_LPR_PIT
#define FEMPIC_LPR_PIT 16
#endif
#ifndef FEMPIC_LPR_L
#define FEMPIC_LPR_L 8
#endif
#ifndef FEMPIC_LPR_V
#define FEMPIC_LPR_V 16
#endif

// Remaining cheb_k - 1 Chebyshev steps of both auxiliary problems, one grid
// barrier before each (the step gathers the whole previous iterate):
//   d <- c1 d + c2 dinv (f - A y),  y <- y + d  (y double-buffered).
// Returns the buffers holding the final iterates; false if a barrier timed out.
__device__ bool aux_cheb(const PcgArgs& a, PcgSched& sc, const float2* rqs, const float*& tfin, const float*& ufin) {
  float* ty[2] = {a.t, a.t2};
  float* uy[2] = {a.u, a.u2};
  int cur = 0;
  const bool vec = a.V.n_rows > 0;
  for (int i = 1; i < a.cheb_k; ++i) {
    if (!grid_sync(a.bar, a.status)) return false;
    const float* yc = ty[cur];
    float* yn = ty[cur ^ 1];
    const float c1 = a.chebL[1][i], c2 = a.chebL[2][i];
    auto xl = [&](int c) { return __ldcg(yc + c); };
#if FEMPIC_CHEB_PREFETCH
    auto pl = [&](int k) { return make_float4(__ldcg(a.td + k), __ldcg(a.tf + k), __ldg(a.dinvL + k), __ldcg(yc + k)); };
    auto elp = [&](int k, float s, float4 p) {
      const float d = fmaf(c1, p.x, c2 * p.z * (p.y - s));
      a.td[k] = d;
      yn[k] = p.w + d;
    };
    sc.run<FEMPIC_LPR_L>(a.L.n_rows, nullptr, [&](int r, bool act, int lane) {
      spmv32_row_pre<FEMPIC_LPR_L>(a.L, r, act, lane, xl, pl, elp);
    });
#else
    auto el = [&](int k, float s) {
      const float d = fmaf(c1, __ldcg(a.td + k), c2 * __ldg(a.dinvL + k) * (__ldcg(a.tf + k) - s));
      a.td[k] = d;
      yn[k] = __ldcg(yc + k) + d;
    };
    sc.run<FEMPIC_LPR_L>(a.L.n_rows, nullptr,
                         [&](int r, bool act, int lane) { spmv32_row<FEMPIC_LPR_L>(a.L, r, act, lane, xl, el); });
#endif
    if (vec) {
      const float* vc = uy[cur];
      float* vn = uy[cur ^ 1];
      const float e1 = a.chebV[1][i], e2 = a.chebV[2][i];
      auto xv = [&](int c) { return __ldcg(vc + c); };
#if FEMPIC_CHEB_PREFETCH
      auto pv = [&](int k) { return make_float4(__ldcg(a.ud + k), __ldcg(a.uf + k), __ldg(a.dinvV + k), __ldcg(vc + k)); };
      auto evp = [&](int k, float s, float4 p) {
        const float d = fmaf(e1, p.x, e2 * p.z * (p.y - s));
        a.ud[k] = d;
        vn[k] = p.w + d;
      };
      sc.run<FEMPIC_LPR_V>(a.V.n_rows, nullptr, [&](int r, bool act, int lane) {
        spmv32_row_pre<FEMPIC_LPR_V>(a.V, r, act, lane, xv, pv, evp);
      });
#else
      auto ev = [&](int k, float s) {
        const float d = fmaf(e1, __ldcg(a.ud + k), e2 * __ldg(a.dinvV + k) * (__ldcg(a.uf + k) - s));
        a.ud[k] = d;
        vn[k] = __ldcg(vc + k) + d;
      };
      sc.run<FEMPIC_LPR_V>(a.V.n_rows, nullptr,
                           [&](int r, bool act, int lane) { spmv32_row<FEMPIC_LPR_V>(a.V, r, act, lane, xv, ev); });
#endif
    }
    if (i < a.smooth_k) {  // smoother step i + 1 on the same phase
      const int n = a.As16.nb * 2;
      const float* syc = a.sy + (size_t)((i - 1) & 1) * n;
      float* syn = a.sy + (size_t)(i & 1) * n;
      const float s1 = __ldg(a.chebS + kMaxCheb + i), s2 = __ldg(a.chebS + 2 * kMaxCheb + i);
      auto es = [&](int k, float w0, float w1) {
        const float g0 = __ldcg(&rqs[2 * k].x) - w0, g1 = __ldcg(&rqs[2 * k + 1].x) - w1;
        const float4 bi = __ldg(reinterpret_cast<const float4*>(a.binv32) + k);
        const float d0 = fmaf(s1, __ldcg(a.sd + 2 * k), s2 * fmaf(bi.x, g0, bi.y * g1));
        const float d1 = fmaf(s1, __ldcg(a.sd + 2 * k + 1), s2 * fmaf(bi.z, g0, bi.w * g1));
        a.sd[2 * k] = d0;
        a.sd[2 * k + 1] = d1;
        syn[2 * k] = __ldcg(syc + 2 * k) + d0;
        syn[2 * k + 1] = __ldcg(syc + 2 * k + 1) + d1;
      };
      sc.run<4>(a.As16.nb, nullptr, [&](int k, bool act, int lane) { bspmv16_row<4>(a.As16, syc, k, act, lane, es); });
    }
    cur ^= 1;
  }
  tfin = ty[cur];
  ufin = uy[cur];
  return true;
}

#ifdef FEMPIC_PCG_PROFILE
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// per-CTA time stamps of one iteration (FEMPIC_PCG_PROFILE builds only):
// [0] start of the A product, [1] its end, [2] after the reduction add,
// [3] after the barrier
__device__ unsigned long long g_pcg_stamp[4096][4];
#define PCG_STAMP(k, it)                                        \
  do {                                                          \
    if ((it) == 10 && threadIdx.x == 0 && blockIdx.x < 4096)    \
      g_pcg_stamp[blockIdx.x][k] = gtime();                     \
  } while (0)
#define PCG_MARK(k)                                                   \
  do {                                                                \
    if (blockIdx.x == 0 && threadIdx.x == 0) {                        \
      unsigned long long now_ = gtime();                              \
      prof_acc[k] += now_ - prof_last;                                \
      prof_last = now_;                                               \
    }                                                                 \
  } while (0)
#else
#define PCG_MARK(k) \
  do {              \
  } while (0)
#define PCG_STAMP(k, it) \
  do {                   \
  } while (0)
#endif

// Preconditioned CG; with the auxiliary-space preconditioner, 3 + cheb_k grid
// barriers per iteration (three without it; two more on the iterations that
// replace the residual when the direction products are FP32):
//   phase 0: p_k = z + beta p_{k-1}; barrier
//   phase 1: q = A p_k; barrier; alpha = rz / (p.q)
//   phase 2: x += alpha p, r' = r - alpha q; right-hand sides D^T r' and
//            Pi^T r' of the auxiliary problems with r' formed on the fly, and
//            their first Chebyshev iterate; cheb_k - 1 further steps, each
//            after a barrier; barrier
//   phase 3: z = B r' + D t + Pi u (B: block or point Jacobi); barrier;
//            rz', r'.r' -> convergence, beta
// Direction products in FP32 (FEMPIC_PCG_FP32A, order 2): the product q = A p
// is the heaviest phase and, in FP64, bound by the FP64 pipe (one DFMA per
// stored value at GB300's FP64 rate); in FP32 it reads half the bytes and runs
// on the FP32 pipe.  Its rounding (~1e-7 of |A||p|) enters the recursive
// residual, so every kPcgReplacePeriod iterations the residual is replaced by
// rhs - A x computed in FP64 (two more barriers and one FP64 product), and a
// solve ends only on a replaced residual below the tolerance: the stopping
// test is on the true residual, as with FP64 products.
#ifndef FEMPIC_PCG_FP32A
#define FEMPIC_PCG_FP32A 1
#endif
constexpr int kPcgReplacePeriod = 16;
// largest median ratio of the curl-curl to the mass diagonal, (dt^2/4) K_ii /
// M_ii, at which the FP32 products are used (drift tube at 33.3 ps: 880;
// 37^3 box at its dt: 600; the 6^3-20^3 boxes at theirs: 2.4e5, where they
// fail to converge)
constexpr double kPcgFp32MaxRatio = 1.0e4;

// Launch shape of the persistent CG kernel: with dynamic row scheduling one
// CTA of 1024 threads (the most a CTA can have) per SM; with the static
// stride, 6 co-resident 256-thread CTAs per SM measured fastest (5 and 8 were
// slower).
#ifndef FEMPIC_PCG_THREADS
#define FEMPIC_PCG_THREADS (FEMPIC_PCG_DYN ? 1024 : 256)
#endif
#ifndef FEMPIC_PCG_MIN_BLOCKS
#define FEMPIC_PCG_MIN_BLOCKS (FEMPIC_PCG_DYN ? 1 : 6)
#endif
template <int LPR>
__global__ void __launch_bounds__(FEMPIC_PCG_THREADS, FEMPIC_PCG_MIN_BLOCKS) k_pcg(PcgArgs a) {
  const int n = a.A.n_rows;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int tpg = gridDim.x * blockDim.x;
  const bool nodal = a.DT.n_rows > 0;
  __shared__ int ring[8];
  if (threadIdx.x < 8) ring[threadIdx.x] = 0;
  __syncthreads();
  PcgSched sc{gid, tpg, ring, 0};
  const int32_t* apart = a.Apart;
  double* r_cur = a.r[0];
  // FP32 shadows of r and q for the auxiliary products, the pair (r_i, q_i)
  // of one buffer side by side so that r - alpha q, formed on the fly in the
  // restriction products, takes one 8-byte gather; double-buffered like r
  float2* rq_cur = reinterpret_cast<float2*>(a.r32);
  float2* rq_alt = rq_cur + n;
  int kred = 0;  // reductions so far (slot of the ring)
#ifdef FEMPIC_PCG_PROFILE
  unsigned long long prof_acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  unsigned long long prof_last = (blockIdx.x == 0 && threadIdx.x == 0) ? gtime() : 0;
#endif
  // ---- start: r = rhs - A x; z = M^-1 r
  double acc[3] = {0.0, 0.0, 0.0};  // r.z, r.r, rhs.rhs
  auto start_row = [&](int r0, double s) -> float {
    double b = a.rhs[r0];
    double rr = b - s;
    r_cur[r0] = rr;
    const float rf = (float)rr;
    if (nodal) rq_cur[r0].x = rf;
    acc[1] += rr * rr;
    acc[2] += b * b;
    if (!nodal) {
      double zz = a.dinv[r0] * rr;
      a.z[r0] = zz;
      acc[0] += rr * zz;
    }
    return rf;
  };
  if (a.Ab.nb > 0) {
    auto em = [&](int k, double s0, double s1) {
      const float r0 = start_row(2 * k, s0);
      const float r1 = start_row(2 * k + 1, s1);
      if (a.smooth_k > 1) smooth_first(a, k, r0, r1);
    };
    sc.run<LPR>(a.Ab.nb, apart, [&](int k, bool act, int lane) { bspmv_row<LPR>(a.Ab, a.x, k, act, lane, em); });
  } else {
    auto xo = [&](int c) { return __ldcg(a.x + c); };
    sc.run<LPR>(n, apart, [&](int r, bool act, int lane) { spmv_row<LPR>(a.A, r, act, lane, xo, start_row); });
  }
  if (nodal) {
    if (!grid_sync(a.bar, a.status)) return;
    auto x0 = [&](int c) { return __ldcg(&rq_cur[c].x); };
    auto et = [&](int k, float s) { aux_first_t(a, k, s); };
    auto eu = [&](int k, float s) { aux_first_u(a, k, s); };
    sc.run<FEMPIC_LPR_DT>(a.DT.n_rows, nullptr, [&](int r, bool act, int lane) { spmv32_row<FEMPIC_LPR_DT>(a.DT, r, act, lane, x0, et); });
    if (a.PiT.n_rows > 0)
      sc.run<FEMPIC_LPR_PIT>(a.PiT.n_rows, nullptr,
                 [&](int r, bool act, int lane) { spmv32_row<FEMPIC_LPR_PIT>(a.PiT, r, act, lane, x0, eu); });
    const float *tv, *uv;
    if (!aux_cheb(a, sc, rq_cur, tv, uv)) return;
    if (!grid_sync(a.bar, a.status)) return;
    acc[0] += aux_z<FEMPIC_LPR_Z>(a, r_cur, tv, uv, sc);
  }
  grid_sum_add<3>(acc, a.red, kred);
  if (!grid_sync(a.bar, a.status)) return;
  double tot[3];
  grid_sum_read<3>(a.red, kred++, tot);
  double rz = tot[0];
  const double bnorm = sqrt(tot[2]);
  double rnorm = sqrt(tot[1]);
  const double thresh = a.rtol * bnorm;
  int it = 0;
  bool conv = rnorm <= thresh || bnorm == 0.0;
  double beta = 0.0;
  int pb = 0;  // p_{k-1} lives in p[pb], p_k is written to p[pb ^ 1]
  bool f32a = a.Ab32.nb > 0;
  bool verify = false;  // FP32 products: the recursive residual reached the tolerance
  double last_true = rnorm;  // FP32 products: the last FP64 (true) residual norm
  while (!conv && it < a.max_it) {
    const double* p_old = a.p[pb];
    double* p_new = a.p[pb ^ 1];
    const bool first = it == 0;
    // phase 0: p_k = z + beta p_{k-1} (elementwise), then q = A p_k
    PCG_MARK(0);
    if (!first || f32a) {
      if (f32a) {
        for (int i = gid; i < n; i += tpg) {
          const double pv = first ? __ldcg(a.z + i) : fma(beta, __ldcg(p_old + i), __ldcg(a.z + i));
          p_new[i] = pv;
          a.p32[i] = (float)pv;
        }
      } else {
        for (int i = gid; i < n; i += tpg) p_new[i] = fma(beta, __ldcg(p_old + i), __ldcg(a.z + i));
      }
      PCG_MARK(1);
      if (!grid_sync(a.bar, a.status)) return;
      PCG_MARK(2);
    } else {
      // p_0 = z_0: kept for the next iteration (z is overwritten below); this
      // iteration's product reads z itself, so no barrier is needed here
      for (int i = gid; i < n; i += tpg) p_new[i] = __ldcg(a.z + i);
    }
    const double* pk_vec = (first && !f32a) ? a.z : p_new;
    double acc1[1] = {0.0};
    PCG_STAMP(0, it);
    if (f32a) {
#if FEMPIC_APROD_PREFETCH
      // the block row's direction values (for p.q) loaded ahead of the product
      auto pp = [&](int k) { return __ldcg(reinterpret_cast<const double2*>(pk_vec) + k); };
      auto emp = [&](int k, float s0, float s1, double2 pv) {
        rq_cur[2 * k].y = s0;
        rq_cur[2 * k + 1].y = s1;
        acc1[0] += pv.x * (double)s0 + pv.y * (double)s1;
      };
      sc.run<LPR>(a.Ab32.nb, apart, [&](int k, bool act, int lane) {
        double2 pv{0.0, 0.0};
        if (act && lane == 0) pv = pp(k);
        bspmv32_row<LPR>(a.Ab32, a.p32, k, act, lane, [&](int kk, float s0, float s1) { emp(kk, s0, s1, pv); });
      });
#else
      auto em = [&](int k, float s0, float s1) {
        rq_cur[2 * k].y = s0;
        rq_cur[2 * k + 1].y = s1;
        acc1[0] += __ldcg(pk_vec + 2 * k) * (double)s0 + __ldcg(pk_vec + 2 * k + 1) * (double)s1;
      };
      sc.run<LPR>(a.Ab32.nb, apart,
                  [&](int k, bool act, int lane) { bspmv32_row<LPR>(a.Ab32, a.p32, k, act, lane, em); });
#endif
    } else if (a.Ab.nb > 0) {
      auto em = [&](int k, double s0, double s1) {
        a.q[2 * k] = s0;
        a.q[2 * k + 1] = s1;
        if (nodal) {
          rq_cur[2 * k].y = (float)s0;
          rq_cur[2 * k + 1].y = (float)s1;
        }
        acc1[0] += __ldcg(pk_vec + 2 * k) * s0 + __ldcg(pk_vec + 2 * k + 1) * s1;
      };
      sc.run<LPR>(a.Ab.nb, apart,
                  [&](int k, bool act, int lane) { bspmv_row<LPR>(a.Ab, pk_vec, k, act, lane, em); });
    } else {
      auto xo = [&](int c) { return __ldcg(pk_vec + c); };
      auto em = [&](int r0, double s) {
        a.q[r0] = s;
        if (nodal) rq_cur[r0].y = (float)s;
        acc1[0] += __ldcg(pk_vec + r0) * s;
      };
      sc.run<LPR>(n, apart, [&](int r, bool act, int lane) { spmv_row<LPR>(a.A, r, act, lane, xo, em); });
    }
    PCG_MARK(3);
    PCG_STAMP(1, it);
    grid_sum_add<1>(acc1, a.red, kred);
    PCG_STAMP(2, it);
    if (!grid_sync(a.bar, a.status)) return;
    PCG_STAMP(3, it);
    PCG_MARK(4);
    double t1[1];
    grid_sum_read<1>(a.red, kred++, t1);
    const double alpha = t1[0] != 0.0 ? rz / t1[0] : 0.0;
    // phase 2: x += alpha p, r' = r - alpha q; the auxiliary products form
    // r' on the fly from the FP32 shadows (r' itself is being written)
    double* r_new = a.r[(it + 1) & 1];
    const double* r_old = r_cur;
    double acc2[2] = {0.0, 0.0};  // r'.z', r'.r'
    // FP32 products: every repl-th iteration, and once the recursive residual
    // has reached the tolerance, r' = rhs - A x' in FP64
    const bool replace = f32a && (verify || (it + 1) % a.repl == 0);
    if (replace) {
      for (int i = gid; i < n; i += tpg) a.x[i] = fma(alpha, __ldcg(pk_vec + i), __ldcg(a.x + i));
      if (!grid_sync(a.bar, a.status)) return;
      auto em = [&](int k, double s0, double s1) {
        const double r0 = a.rhs[2 * k] - s0, r1 = a.rhs[2 * k + 1] - s1;
        r_new[2 * k] = r0;
        r_new[2 * k + 1] = r1;
        const float r0f = (float)r0, r1f = (float)r1;
        rq_alt[2 * k].x = r0f;
        rq_alt[2 * k + 1].x = r1f;
        acc2[1] += r0 * r0 + r1 * r1;
        if (a.smooth_k > 1) smooth_first(a, k, r0f, r1f);
      };
      sc.run<LPR>(a.Ab.nb, apart, [&](int k, bool act, int lane) { bspmv_row<LPR>(a.Ab, a.x, k, act, lane, em); });
      if (!grid_sync(a.bar, a.status)) return;
    } else {
      auto upd = [&](int i) -> float {
        a.x[i] = fma(alpha, __ldcg(pk_vec + i), __ldcg(a.x + i));
        const double qi = f32a ? (double)__ldcg(&rq_cur[i].y) : __ldcg(a.q + i);
        double rr = fma(-alpha, qi, __ldcg(r_old + i));
        r_new[i] = rr;
        const float rf = (float)rr;
        if (nodal) rq_alt[i].x = rf;
        acc2[1] += rr * rr;
        if (!nodal) {
          double zz = a.dinv[i] * rr;
          a.z[i] = zz;
          acc2[0] += rr * zz;
        }
        return rf;
      };
      if (a.smooth_k > 1) {  // by blocks: the smoother's first iterate needs both rows
        for (int k = gid; k < (n >> 1); k += tpg) {
          const float r0 = upd(2 * k);
          const float r1 = upd(2 * k + 1);
          smooth_first(a, k, r0, r1);
        }
      } else {
        for (int i = gid; i < n; i += tpg) upd(i);
      }
    }
    if (nodal) {
      const float alpha32 = (float)alpha;
      const float2* rqo = rq_cur;
      const float2* rqn = rq_alt;
      auto xr = [&](int c) {
        if (replace) return __ldcg(&rqn[c].x);
        const float2 v = __ldcg(rqo + c);
        return fmaf(-alpha32, v.y, v.x);
      };
#if FEMPIC_RESTRICT_PREFETCH
      // the rows' Jacobi scalings loaded ahead of their products
      auto pt = [&](int k) { return __ldg(a.dinvL + k); };
      auto pu = [&](int k) { return __ldg(a.dinvV + k); };
      auto et = [&](int k, float s, float dl) { aux_first_t_d(a, k, s, dl); };
      auto eu = [&](int k, float s, float dv) { aux_first_u_d(a, k, s, dv); };
      sc.run<FEMPIC_LPR_DT>(a.DT.n_rows, nullptr, [&](int r, bool act, int lane) {
        spmv32_row_pre<FEMPIC_LPR_DT>(a.DT, r, act, lane, xr, pt, et);
      });
      if (a.PiT.n_rows > 0)
        sc.run<FEMPIC_LPR_PIT>(a.PiT.n_rows, nullptr, [&](int r, bool act, int lane) {
          spmv32_row_pre<FEMPIC_LPR_PIT>(a.PiT, r, act, lane, xr, pu, eu);
        });
#else
      auto et = [&](int k, float s) { aux_first_t(a, k, s); };
      auto eu = [&](int k, float s) { aux_first_u(a, k, s); };
      sc.run<FEMPIC_LPR_DT>(a.DT.n_rows, nullptr, [&](int r, bool act, int lane) { spmv32_row<FEMPIC_LPR_DT>(a.DT, r, act, lane, xr, et); });
      if (a.PiT.n_rows > 0)
        sc.run<FEMPIC_LPR_PIT>(a.PiT.n_rows, nullptr,
                   [&](int r, bool act, int lane) { spmv32_row<FEMPIC_LPR_PIT>(a.PiT, r, act, lane, xr, eu); });
#endif
      PCG_MARK(5);
      const float *tv, *uv;
      if (!aux_cheb(a, sc, rq_alt, tv, uv)) return;
      PCG_MARK(8);
      if (!grid_sync(a.bar, a.status)) return;
      PCG_MARK(6);
      // phase 3: z = dinv r' + D t + Pi u
      acc2[0] += aux_z<FEMPIC_LPR_Z>(a, r_new, tv, uv, sc);
    }
    grid_sum_add<2>(acc2, a.red, kred);
    PCG_MARK(7);
    if (!grid_sync(a.bar, a.status)) return;
    double t2[2];
    grid_sum_read<2>(a.red, kred++, t2);
    ++it;
    r_cur = r_new;
    float2* tmp32 = rq_cur;
    rq_cur = rq_alt;
    rq_alt = tmp32;
    pb ^= 1;
    rnorm = sqrt(t2[1]);
    if (f32a) {  // accept only a replaced (true) residual; otherwise check it next iteration
      conv = replace && rnorm <= thresh;
      verify = !conv && rnorm <= thresh;
      if (replace && !conv) {
        // safeguard: a true residual that has not halved since the last one
        // means the FP32 products no longer lead; go on in FP64
        if (rnorm > 0.5 * last_true) {
          f32a = false;
          verify = false;
        }
        last_true = rnorm;
      }
    } else {
      conv = rnorm <= thresh;
    }
    beta = rz != 0.0 ? t2[0] / rz : 0.0;
    // A replaced residual can carry far more in the preconditioner's norm than
    // the recursive one did (the FP32 products' rounding in the near-kernel
    // directions the auxiliary spaces amplify), and beta > 1 formed from it no
    // longer continues the conjugate directions: restart from z (on a
    // 3 x 3 x 3 cavity box at p = 2 the CG otherwise stalled near 1e-6; on the
    // drift tube the iteration count is unchanged, host emulation)
    if (replace && beta > 1.0) beta = 0.0;
    rz = t2[0];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.iters_out = it;
    *a.res_out = bnorm > 0.0 ? rnorm / bnorm : 0.0;
    if (!conv) atomicOr(a.status, kStatusCG);
#ifdef FEMPIC_PCG_PROFILE
    if (it > 10) {
      const int nb = min((int)gridDim.x, 4096);
      double mn = 1e30, mx = 0, sum = 0, amx = 0, asum = 0;
      for (int b = 0; b < nb; ++b) {
        const double d = 1e-3 * (double)(g_pcg_stamp[b][1] - g_pcg_stamp[b][0]);
        const double ad = 1e-3 * (double)(g_pcg_stamp[b][2] - g_pcg_stamp[b][1]);
        mn = fmin(mn, d);
        mx = fmax(mx, d);
        sum += d;
        amx = fmax(amx, ad);
        asum += ad;
      }
      printf("PCGSTAMP it=10 A product per CTA min/mean/max %.1f/%.1f/%.1f us; reduction add mean/max %.1f/%.1f us; "
             "barrier exit CTA0 %.1f us\n",
             mn, sum / nb, mx, asum / nb, amx, 1e-3 * (double)(g_pcg_stamp[0][3] - g_pcg_stamp[0][0]));
    }
    printf("PCGPROF it=%d loop_top+totals=%.1f p_update=%.1f bar0=%.1f spmv=%.1f bar1=%.1f xr_aux_t=%.1f cheb=%.1f "
           "bar2=%.1f aux_z=%.1f (us)\n",
           it, prof_acc[0] * 1e-3, prof_acc[1] * 1e-3, prof_acc[2] * 1e-3, prof_acc[3] * 1e-3, prof_acc[4] * 1e-3,
           prof_acc[5] * 1e-3, prof_acc[8] * 1e-3, prof_acc[6] * 1e-3, prof_acc[7] * 1e-3);
#endif
  }
}

__global__ void k_accumulate_iters(const int32_t* it, int32_t* acc) { *acc += *it; }

// ---- counting sort by tet -----------------------------------------------------
__global__ void k_hist(int64_t n, const int32_t* __restrict__ tet, int32_t* __restrict__ cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(cnt + tet[i], 1);
}

// exclusive scan of one tile of 1024 values per block; tile totals to sums
// in and out may be the same array (the recursive level scans in place):
// each thread reads its element before the block's barriers and writes it after
__global__ void k_scan_tiles(int32_t n, const int32_t* in, int32_t* out, int32_t* __restrict__ sums) {
  __shared__ int32_t warp_tot[32];
  int i = blockIdx.x * 1024 + threadIdx.x;
  int v = i < n ? in[i] : 0;
  int l = threadIdx.x & 31, w = threadIdx.x >> 5;
  int s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, s, o);
    if (l >= o) s += t;
  }
  if (l == 31) warp_tot[w] = s;
  __syncthreads();
  if (w == 0) {
    int t = warp_tot[l];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, t, o);
      if (l >= o) t += u;
    }
    warp_tot[l] = t;
  }
  __syncthreads();
  int excl = s - v + (w > 0 ? warp_tot[w - 1] : 0);
  if (i < n) out[i] = excl;
  if (threadIdx.x == 1023 && sums) sums[blockIdx.x] = excl + v;
}

__global__ void k_scan_add(int32_t n, int32_t* __restrict__ out, const int32_t* __restrict__ tile_off) {
  int i = blockIdx.x * 1024 + threadIdx.x;
  if (i < n) out[i] += tile_off[blockIdx.x];
}

struct SortArgs {
  int64_t n;
  const int32_t* tet_in;
  int32_t* cursor;  // exclusive offsets, consumed
  const double* src[6];
  double* dst[6];
  const int32_t* ti[2];
  int32_t* to[2];   // tet, particle id
};

__global__ void k_sort_scatter(SortArgs a) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  int t = a.tet_in[i];
  int pos = atomicAdd(a.cursor + t, 1);
#pragma unroll
  for (int k = 0; k < 6; ++k) a.dst[k][pos] = a.src[k][i];
  a.to[0][pos] = t;
  a.to[1][pos] = a.ti[1][i];
}

// Validation of a staged transfer: the lowest index of an element that is not
// finite (exponent bits all set) or, for tet ids, outside [0, n_tets), kept by
// atomicMin in *first (all ones = none found).
__global__ void k_first_nonfinite(int64_t m, const double* v, unsigned long long* first) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v[i]);
    if ((u & 0x7FF0000000000000ull) == 0x7FF0000000000000ull) atomicMin(first, (unsigned long long)i);
  }
}
__global__ void k_first_bad_tet(int64_t m, const int32_t* t, int32_t n_tets, unsigned long long* first) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    if (t[i] < 0 || t[i] >= n_tets) atomicMin(first, (unsigned long long)i);
}

// particle-id order <-> device order; a gather with a veto word writes nothing
// once the validation above found a bad element
__global__ void k_gather_by_id(int64_t n, const int32_t* pid, const double* src_il, double* d0, double* d1,
                               double* d2, const unsigned long long* veto = nullptr) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || (veto && *veto != ~0ull)) return;
  int64_t p = pid[i];
  d0[i] = src_il[3 * p];
  d1[i] = src_il[3 * p + 1];
  d2[i] = src_il[3 * p + 2];
}
__global__ void k_scatter_by_id(int64_t n, const int32_t* pid, const double* s0, const double* s1,
                                const double* s2, double* dst_il) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t p = pid[i];
  dst_il[3 * p] = s0[i];
  dst_il[3 * p + 1] = s1[i];
  dst_il[3 * p + 2] = s2[i];
}
template <class T>
__global__ void k_scatter1_by_id(int64_t n, const int32_t* pid, const T* s, T* dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[pid[i]] = s[i];
}
template <class T>
__global__ void k_gather1_by_id(int64_t n, const int32_t* pid, const T* s, T* dst,
                                const unsigned long long* veto = nullptr) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(veto && *veto != ~0ull)) dst[i] = s[pid[i]];
}

// ---- diagnostics ----------------------------------------------------------------
// out[0] += sum over mask of a^2, out[1] += sum of b^2 where a = x1 - x0 - y, b = x1 - x0
__global__ void k_norms2(int32_t n, const uint8_t* mask, const double* u, const double* w, const double* y,
                         double c_y, double c_w2, const double* w2, double* out) {
  double s[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (!mask[i]) continue;
    double base = u[i] - (w ? w[i] : 0.0);
    double res = base + c_y * y[i] + (w2 ? c_w2 * w2[i] : 0.0);
    s[0] += res * res;
    s[1] += base * base;
  }
  for (int k = 0; k < 2; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out + k, s[k]);
  }
}

}  // namespace dev
}  // namespace fempic
