// Batched execution of many independent EM-FEMPIC instances ("members") of
// different meshes, orders, precisions and particle counts on one GPU.
//
// Every member keeps its own device state; a device-resident descriptor per
// member holds all pointers the kernels need.  Work is cut into fixed-size work
// blocks tagged with a member (prefix tables), so one launch covers all
// members and every warp works on one member.  The per-step buffer rotations
// are done by tiny kernels on the descriptors, so a whole batched step is a
// fixed launch sequence that can be captured once in a CUDA graph and
// replayed.  The field solve is one cooperative, block-diagonal PCG: each
// member owns a contiguous range of CTAs, has its own reductions and
// convergence test, and the launch ends once every member has converged.
#pragma once

#include "linalg.cuh"
#include "particle_fast.cuh"

namespace fempic {
namespace dev {

struct MemberDesc {
  int32_t order, mixed, max_cross, max_it;
  int32_t n1, n2, n0, nt;
  int64_t np;
  double qw, h, dt, rtol;
  double B0[3];
  const double* geom;
  const int32_t* nbr;
  const int32_t* dof0;
  const int32_t* dof1;
  const int32_t* dof2;
  const uint8_t* pec;
  double* x[3];
  double* v[3];
  int32_t* tet;
  int32_t* pid;
  double* xa[3];
  double* va[3];
  int32_t* teta;
  int32_t* pida;
  int32_t* ncross;
  unsigned long long* hash;
  int32_t* cnt;
  int32_t* off;
  double *e, *e_prev, *e_new, *b, *dg, *dg_prev, *rho, *rho_prev;
  CsrView A, R1, Q, C;
  const double* dinvA;
  CsrView32 D, DT, Pi, PiT;  // FP32 preconditioner operators
  const float* dinvL;
  const float* dinvV;
  float* t;
  float* u;
  // Chebyshev smoothing of the auxiliary problems (as in k_pcg)
  CsrView32 L, V;
  float *tf, *td, *t2, *uf, *ud, *u2;
  int32_t cheb_k;
  float chebL[3][kMaxCheb];
  float chebV[3][kMaxCheb];
  double* rhs;
  double* r[2];
  double* z;
  double* p[2];
  double* q;
  float* q32;    // FP32 shadows of q and r (auxiliary products)
  float* r32;    // [2][n1]
  BsrView Ab;    // order 2: 2x2-block system matrix (nb = 0 otherwise)
  const double* binv;
  int32_t* status;
  int32_t* cg_iters;
  double* cg_res;
  unsigned long long* crossings;
};

struct BatchWork {
  int32_t n;                // members
  MemberDesc* d;            // [n]
  const int32_t* pblk;      // [n+1] particle work blocks (256 particles) of the sort kernels
  const int32_t* ppblk;     // [n+1] particle work blocks of the particle kernel (pbs particles)
  int32_t pbs;              // particles per work block of the particle kernel = its CTA size
  const int32_t* tblk;      // [n+1] tet tiles (1024 tets)
  const int32_t* r1blk;     // [n+1] W1 row blocks (32 rows: 8 lanes per row)
  const int32_t* r2blk;     // [n+1] W2 row blocks (64 rows: 4 lanes per row)
  const int32_t* zblk;      // [n+1] zeroing blocks (256 entries of dg | rho | counts)
  const int32_t* cgblk;     // [n+1] CTAs of the cooperative PCG per member
  int32_t* tile_sums;       // [total tiles]
  GridBarrier* bar;
  double* partials;         // [2][grid * 4]
  double* red;              // [3][n + 1][4] reduction ring (per member, then the working count)
  int32_t* status;          // batch-level status (barrier timeouts)
};

// largest m with pref[m] <= wb
__device__ __forceinline__ int member_of(const int32_t* pref, int n, int wb) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(pref + mid) <= wb)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__global__ void k_batch_begin(BatchWork w) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= w.n) return;
  MemberDesc& d = w.d[m];
  double* t = d.dg;
  d.dg = d.dg_prev;
  d.dg_prev = t;
  t = d.rho;
  d.rho = d.rho_prev;
  d.rho_prev = t;
}

__global__ void k_batch_zero(BatchWork w) {
  const int total = __ldg(w.zblk + w.n);
  for (int wb = blockIdx.x; wb < total; wb += gridDim.x) {
    const int m = member_of(w.zblk, w.n, wb);
    const MemberDesc& d = w.d[m];
    int64_t k = (int64_t)(wb - __ldg(w.zblk + m)) * 256 + threadIdx.x;
    if (k < d.n1)
      d.dg[k] = 0.0;
    else if (k < d.n1 + d.n0)
      d.rho[k - d.n1] = 0.0;
    else if (k < d.n1 + d.n0 + d.nt)
      d.cnt[k - d.n1 - d.n0] = 0;
  }
}

__global__ void k_batch_hist(BatchWork w) {
  const int total = __ldg(w.pblk + w.n);
  for (int wb = blockIdx.x; wb < total; wb += gridDim.x) {
    const int m = member_of(w.pblk, w.n, wb);
    const MemberDesc& d = w.d[m];
    int64_t i = (int64_t)(wb - __ldg(w.pblk + m)) * 256 + threadIdx.x;
    if (i < d.np) atomicAdd(d.cnt + d.tet[i], 1);
  }
}

// exclusive scan of one 1024-tet tile; tile total into tile_sums (global tile id)
__global__ void k_batch_scan_tiles(BatchWork w) {
  __shared__ int32_t warp_tot[32];
  const int tile = blockIdx.x;
  const int m = member_of(w.tblk, w.n, tile);
  const MemberDesc& d = w.d[m];
  const int local = tile - __ldg(w.tblk + m);
  const int i = local * 1024 + threadIdx.x;
  int v = i < d.nt ? d.cnt[i] : 0;
  int l = threadIdx.x & 31, wi = threadIdx.x >> 5;
  int s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, s, o);
    if (l >= o) s += t;
  }
  if (l == 31) warp_tot[wi] = s;
  __syncthreads();
  if (wi == 0) {
    int t = warp_tot[l];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, t, o);
      if (l >= o) t += u;
    }
    warp_tot[l] = t;
  }
  __syncthreads();
  int excl = s - v + (wi > 0 ? warp_tot[wi - 1] : 0);
  if (i < d.nt) d.off[i] = excl;
  if (threadIdx.x == 1023) w.tile_sums[tile] = excl + v;
}

// one CTA per member: exclusive scan of its tile totals (at most 1024 tiles)
__global__ void k_batch_scan_sums(BatchWork w) {
  __shared__ int32_t warp_tot[32];
  const int m = blockIdx.x;
  const int t0 = __ldg(w.tblk + m), nt = __ldg(w.tblk + m + 1) - t0;
  int v = threadIdx.x < nt ? w.tile_sums[t0 + threadIdx.x] : 0;
  int l = threadIdx.x & 31, wi = threadIdx.x >> 5;
  int s = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, s, o);
    if (l >= o) s += t;
  }
  if (l == 31) warp_tot[wi] = s;
  __syncthreads();
  if (wi == 0) {
    int t = warp_tot[l];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, t, o);
      if (l >= o) t += u;
    }
    warp_tot[l] = t;
  }
  __syncthreads();
  if (threadIdx.x < nt) w.tile_sums[t0 + threadIdx.x] = s - v + (wi > 0 ? warp_tot[wi - 1] : 0);
}

__global__ void k_batch_scan_add(BatchWork w) {
  const int tile = blockIdx.x;
  const int m = member_of(w.tblk, w.n, tile);
  const MemberDesc& d = w.d[m];
  const int i = (tile - __ldg(w.tblk + m)) * 1024 + threadIdx.x;
  if (i < d.nt) d.off[i] += w.tile_sums[tile];
}

__global__ void k_batch_scatter(BatchWork w) {
  const int total = __ldg(w.pblk + w.n);
  for (int wb = blockIdx.x; wb < total; wb += gridDim.x) {
    const int m = member_of(w.pblk, w.n, wb);
    const MemberDesc& d = w.d[m];
    int64_t i = (int64_t)(wb - __ldg(w.pblk + m)) * 256 + threadIdx.x;
    if (i >= d.np) continue;
    int t = d.tet[i];
    int pos = atomicAdd(d.off + t, 1);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      d.xa[k][pos] = d.x[k][i];
      d.va[k][pos] = d.v[k][i];
    }
    d.teta[pos] = t;
    d.pida[pos] = d.pid[i];
  }
}

__global__ void k_batch_swap_particles(BatchWork w) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= w.n) return;
  MemberDesc& d = w.d[m];
  for (int k = 0; k < 3; ++k) {
    double* t = d.x[k];
    d.x[k] = d.xa[k];
    d.xa[k] = t;
    t = d.v[k];
    d.v[k] = d.va[k];
    d.va[k] = t;
  }
  int32_t* ti = d.tet;
  d.tet = d.teta;
  d.teta = ti;
  ti = d.pid;
  d.pid = d.pida;
  d.pida = ti;
}

__device__ __forceinline__ ParticleArgs member_particle_args(const MemberDesc& d) {
  ParticleArgs a;
  a.n = d.np;
  for (int k = 0; k < 3; ++k) {
    a.x[k] = d.x[k];
    a.v[k] = d.v[k];
    a.B0[k] = d.B0[k];
  }
  a.tet = d.tet;
  a.ncross = d.ncross;
  a.hash = d.hash;
  a.geom = d.geom;
  a.nbr = d.nbr;
  a.dof0 = d.dof0;
  a.dof1 = d.dof1;
  a.dof2 = d.dof2;
  a.e = d.e;
  a.b = d.b;
  a.dg = d.dg;
  a.rho = d.rho;
  a.h = d.h;
  a.dt = d.dt;
  a.qw = d.qw;
  a.pid = d.pid;
  a.sp.n = 1;
  a.max_cross = d.max_cross;
  a.status = d.status;
  a.n_tets = d.nt;
  a.crossings = d.crossings;
  return a;
}

// persistent: CTAs loop over the particle work blocks of all members
// (CTA size w.pbs and grid picked by the batch's autotuner)
__global__ void __launch_bounds__(256, 2) k_batch_particles(BatchWork w) {
  const int total = __ldg(w.ppblk + w.n);
  for (int wb = blockIdx.x; wb < total; wb += gridDim.x) {
    const int m = member_of(w.ppblk, w.n, wb);
    const MemberDesc& d = w.d[m];
    const ParticleArgs a = member_particle_args(d);
    const int64_t i = (int64_t)(wb - __ldg(w.ppblk + m)) * w.pbs + threadIdx.x;
    if (d.order == 1) {
      if (d.mixed)
        particle_step<1, (bool)FEMPIC_PARTICLE_AGG, true>(a, i);
      else
        particle_step<1, (bool)FEMPIC_PARTICLE_AGG, false>(a, i);
    } else {
      if (d.mixed)
        particle_step<2, (bool)FEMPIC_PARTICLE_AGG, true>(a, i);
      else
        particle_step<2, (bool)FEMPIC_PARTICLE_AGG, false>(a, i);
    }
  }
}

// initial guess e_new = 2 e - e_prev, over W1 row blocks (32 rows each)
__global__ void k_batch_guess(BatchWork w) {
  const int total = __ldg(w.r1blk + w.n);
  for (int wb = blockIdx.x; wb < total; wb += gridDim.x) {
    const int m = member_of(w.r1blk, w.n, wb);
    const MemberDesc& d = w.d[m];
    int base = (wb - __ldg(w.r1blk + m)) * 32;
    for (int r = base + threadIdx.x; r < base + 32 && r < d.n1; r += blockDim.x)
      d.e_new[r] = 2.0 * d.e[r] - d.e_prev[r];
  }
}

// trapezoidal right-hand side, 8 lanes per row
__global__ void k_batch_rhs(BatchWork w) {
  const int total = __ldg(w.r1blk + w.n);
  const int lane = threadIdx.x & 7;
  for (int wb = blockIdx.x; wb < total; wb += gridDim.x) {
    const int m = member_of(w.r1blk, w.n, wb);
    const MemberDesc& d = w.d[m];
    const int r = (wb - __ldg(w.r1blk + m)) * 32 + (threadIdx.x >> 3);
    const bool act = r < d.n1;
    double s = 0.0;
    if (act) {
      for (int k = __ldg(d.R1.rp + r) + lane; k < __ldg(d.R1.rp + r + 1); k += 8)
        s = fma(__ldg(d.R1.v + k), __ldg(d.e + __ldg(d.R1.ci + k)), s);
      double t = 0.0;
      for (int k = __ldg(d.Q.rp + r) + lane; k < __ldg(d.Q.rp + r + 1); k += 8)
        t = fma(__ldg(d.Q.v + k), __ldg(d.b + __ldg(d.Q.ci + k)), t);
      s = fma(d.dt, t, s);
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, 8);
    if (act && lane == 0) d.rhs[r] = d.pec[r] ? 0.0 : s - d.dg[r];
  }
}

// b -= dt/2 C (e_new + e), 4 lanes per row
__global__ void k_batch_bupdate(BatchWork w) {
  const int total = __ldg(w.r2blk + w.n);
  const int lane = threadIdx.x & 3;
  for (int wb = blockIdx.x; wb < total; wb += gridDim.x) {
    const int m = member_of(w.r2blk, w.n, wb);
    const MemberDesc& d = w.d[m];
    const int r = (wb - __ldg(w.r2blk + m)) * 64 + (threadIdx.x >> 2);
    const bool act = r < d.n2;
    double s = 0.0;
    if (act) {
      for (int k = __ldg(d.C.rp + r) + lane; k < __ldg(d.C.rp + r + 1); k += 4) {
        int c = __ldg(d.C.ci + k);
        s = fma(__ldg(d.C.v + k), __ldg(d.e_new + c) + __ldg(d.e + c), s);
      }
    }
#pragma unroll
    for (int o = 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, 4);
    if (act && lane == 0) d.b[r] = fma(-0.5 * d.dt, s, d.b[r]);
  }
}

__global__ void k_batch_end(BatchWork w) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= w.n) return;
  MemberDesc& d = w.d[m];
  double* old_prev = d.e_prev;
  d.e_prev = d.e;
  d.e = d.e_new;
  d.e_new = old_prev;
}

// ---- block-diagonal PCG ---------------------------------------------------------
// member totals: sum of the member's CTA partials in CTA order
template <int NV>
__device__ __forceinline__ void member_totals(const double* partials, int b0, int b1, double (&tot)[NV]) {
  __shared__ double res[4];
  if (threadIdx.x < 32) {
    int l = threadIdx.x;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int b = b0 + l; b < b1; b += 32) s += __ldcg(partials + b * 4 + k);
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

// rows of one member, LPR lanes per row, spread over the member's CTAs
template <int LPR, class X, class F>
__device__ __forceinline__ void member_rows(const CsrView& A, int tid, int tcount, X x_of, F emit) {
  const int lane = tid % LPR;
  const int groups = tcount / LPR;
  for (int r0 = tid / LPR; ; r0 += groups) {
    bool act = r0 < A.n_rows;
    if (!__any_sync(0xffffffffu, act)) break;
    double s = 0.0;
    if (act) {
      int beg = __ldg(A.rp + r0), end = __ldg(A.rp + r0 + 1);
      for (int k = beg + lane; k < end; k += LPR) s = fma(__ldg(A.v + k), x_of(__ldg(A.ci + k)), s);
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LPR);
    if (act && lane == 0) emit(r0, s);
  }
}

// z_i = (block-)Jacobi + (D t)_i + (Pi u)_i over the member's rows; returns r.z part
__device__ __forceinline__ double member_z(const MemberDesc& d, const double* rvec, const float* tv, const float* uv,
                                           int tid, int tcount) {
  const int lane = tid % 4;
  const int groups = tcount / 4;
  double rz = 0.0;
  for (int i = tid / 4; ; i += groups) {
    bool act = i < d.n1;
    if (!__any_sync(0xffffffffu, act)) break;
    float s = 0.f;
    if (act) {
      for (int k = __ldg(d.D.rp + i) + lane; k < __ldg(d.D.rp + i + 1); k += 4)
        s = fmaf(__ldg(d.D.v + k), __ldcg(tv + __ldg(d.D.ci + k)), s);
      for (int k = __ldg(d.Pi.rp + i) + lane; k < __ldg(d.Pi.rp + i + 1); k += 4)
        s = fmaf(__ldg(d.Pi.v + k), __ldcg(uv + __ldg(d.Pi.ci + k)), s);
    }
#pragma unroll
    for (int o = 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, 4);
    if (act && (tid & 3) == 0) {
      double rr = __ldcg(rvec + i);
      double zz;
      if (d.Ab.nb > 0) {
        const int k = i >> 1, par = i & 1;
        double r0 = __ldcg(rvec + 2 * k), r1 = __ldcg(rvec + 2 * k + 1);
        zz = fma(__ldg(d.binv + 4 * k + 2 * par), r0, fma(__ldg(d.binv + 4 * k + 2 * par + 1), r1, (double)s));
      } else {
        zz = fma(__ldg(d.dinvA + i), rr, (double)s);
      }
      d.z[i] = zz;
      rz += rr * zz;
    }
  }
  return rz;
}

// FP32 rows of one member
template <int LPR, class X, class F>
__device__ __forceinline__ void member_rows32(const CsrView32& A, int tid, int tcount, X x_of, F emit) {
  const int lane = tid % LPR;
  const int groups = tcount / LPR;
  for (int r0 = tid / LPR; ; r0 += groups) {
    bool act = r0 < A.n_rows;
    if (!__any_sync(0xffffffffu, act)) break;
    float s = 0.f;
    if (act) {
      int beg = __ldg(A.rp + r0), end = __ldg(A.rp + r0 + 1);
      for (int k = beg + lane; k < end; k += LPR) s = fmaf(__ldg(A.v + k), x_of(__ldg(A.ci + k)), s);
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LPR);
    if (act && lane == 0) emit(r0, s);
  }
}

// first Chebyshev iterate of the member's auxiliary problems from their right-hand sides
__device__ __forceinline__ void member_first_t(const MemberDesc& d, int k, float f) {
  const float y = d.chebL[0][0] * __ldg(d.dinvL + k) * f;
  d.t[k] = y;
  if (d.cheb_k > 1) {
    d.tf[k] = f;
    d.td[k] = y;
  }
}
__device__ __forceinline__ void member_first_u(const MemberDesc& d, int k, float f) {
  const float y = d.chebV[0][0] * __ldg(d.dinvV + k) * f;
  d.u[k] = y;
  if (d.cheb_k > 1) {
    d.uf[k] = f;
    d.ud[k] = y;
  }
}

// The remaining Chebyshev steps of the member's auxiliary problems.  Every CTA
// passes kc - 1 grid barriers (kc: largest degree in the batch); a member works
// in the first cheb_k - 1 of them while it is still iterating.
__device__ bool member_cheb(const BatchWork& w, const MemberDesc& d, bool work, int kc, int tid, int tcount,
                            const float*& tfin, const float*& ufin) {
  float* ty[2] = {d.t, d.t2};
  float* uy[2] = {d.u, d.u2};
  int cur = 0;
  for (int i = 1; i < kc; ++i) {
    if (!grid_sync(w.bar, w.status)) return false;
    if (!work || i >= d.cheb_k) continue;
    const float* yc = ty[cur];
    float* yn = ty[cur ^ 1];
    const float c1 = d.chebL[1][i], c2 = d.chebL[2][i];
    member_rows32<8>(d.L, tid, tcount, [&](int c) { return __ldcg(yc + c); }, [&](int k, float s) {
      const float dd = fmaf(c1, __ldcg(d.td + k), c2 * __ldg(d.dinvL + k) * (__ldcg(d.tf + k) - s));
      d.td[k] = dd;
      yn[k] = __ldcg(yc + k) + dd;
    });
    if (d.V.n_rows > 0) {
      const float* vc = uy[cur];
      float* vn = uy[cur ^ 1];
      const float e1 = d.chebV[1][i], e2 = d.chebV[2][i];
      member_rows32<16>(d.V, tid, tcount, [&](int c) { return __ldcg(vc + c); }, [&](int k, float s) {
        const float dd = fmaf(e1, __ldcg(d.ud + k), e2 * __ldg(d.dinvV + k) * (__ldcg(d.uf + k) - s));
        d.ud[k] = dd;
        vn[k] = __ldcg(vc + k) + dd;
      });
    }
    cur ^= 1;
  }
  tfin = ty[cur];
  ufin = uy[cur];
  return true;
}

// q = A x over one member's rows (2x2 blocks at order 2); emit(row, value)
template <class F>
__device__ __forceinline__ void member_matvec(const MemberDesc& d, const double* x, int tid, int tcount, F emit) {
  if (d.Ab.nb > 0)
    rows_bspmv<4>(d.Ab, x, tid, tcount / 4, [&](int k, double s0, double s1) {
      emit(2 * k, s0);
      emit(2 * k + 1, s1);
    });
  else
    member_rows<8>(d.A, tid, tcount, [&](int c) { return __ldcg(x + c); }, emit);
}

// per-member sums through the reduction ring: CTA totals are added atomically
// into slot k of the member; the last entry of each slot counts CTAs whose
// member is still working.  CTA 0 clears slot k+1 (its readers are done).
template <int NV>
__device__ __forceinline__ void member_sum_add(double (&v)[NV], double working, const BatchWork& w, int m, int k) {
  __shared__ double wsum[32][4];
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) wsum[wi][q] = v[q];
  __syncthreads();
  const int stride = (w.n + 1) * 4;
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < stride; j += blockDim.x) w.red[((k + 1) % 3) * stride + j] = 0.0;
  if (wi == 0) {
    int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = l < nw ? wsum[l][q] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (l == 0) atomicAdd(w.red + (k % 3) * stride + m * 4 + q, s);
    }
    if (l == 0 && working != 0.0) atomicAdd(w.red + (k % 3) * stride + w.n * 4, working);
  }
  __syncthreads();
}

__device__ __forceinline__ double member_sum_read(const BatchWork& w, int m, int k, int q) {
  return __ldcg(w.red + (k % 3) * (w.n + 1) * 4 + m * 4 + q);
}

// 6 co-resident 256-thread CTAs per SM (<= 40 registers)
#ifndef FEMPIC_BATCH_PCG_MIN_BLOCKS
#define FEMPIC_BATCH_PCG_MIN_BLOCKS 6
#endif

// Every CTA runs the same number of iterations and barriers; a CTA whose
// member has converged skips the work.  The exit test counts members still
// working at the start of the iteration (summed after the barrier), so every
// CTA leaves at the same iteration.
__global__ void __launch_bounds__(256, FEMPIC_BATCH_PCG_MIN_BLOCKS) k_batch_pcg(BatchWork w, int max_it_all, int kc) {
  const int m = member_of(w.cgblk, w.n, blockIdx.x);
  const MemberDesc& d = w.d[m];
  const int b0 = __ldg(w.cgblk + m), b1 = __ldg(w.cgblk + m + 1);
  const int tid = (blockIdx.x - b0) * blockDim.x + threadIdx.x;
  const int tcount = (b1 - b0) * blockDim.x;
  const int n = d.n1;
  double* x = d.e_new;
  double* r_cur = d.r[0];
  float* r32_cur = d.r32;
  float* r32_alt = d.r32 + n;
  int kred = 0;
  double acc[3] = {0.0, 0.0, 0.0};  // r.z, r.r, rhs.rhs
  member_matvec(d, x, tid, tcount, [&](int r0, double s) {
    double b = d.rhs[r0];
    double rr = b - s;
    r_cur[r0] = rr;
    r32_cur[r0] = (float)rr;
    acc[1] += rr * rr;
    acc[2] += b * b;
  });
  if (!grid_sync(w.bar, w.status)) return;
  member_rows32<FEMPIC_LPR_DT>(d.DT, tid, tcount, [&](int c) { return __ldcg(r32_cur + c); },
                   [&](int k, float s) { member_first_t(d, k, s); });
  member_rows32<16>(d.PiT, tid, tcount, [&](int c) { return __ldcg(r32_cur + c); },
                    [&](int k, float s) { member_first_u(d, k, s); });
  {
    const float *tv, *uv;
    if (!member_cheb(w, d, true, kc, tid, tcount, tv, uv)) return;
    if (!grid_sync(w.bar, w.status)) return;
    acc[0] += member_z(d, r_cur, tv, uv, tid, tcount);
  }
  member_sum_add<3>(acc, 0.0, w, m, kred);
  if (!grid_sync(w.bar, w.status)) return;
  double rz = member_sum_read(w, m, kred, 0);
  const double bnorm = sqrt(member_sum_read(w, m, kred, 2));
  double rnorm = sqrt(member_sum_read(w, m, kred, 1));
  ++kred;
  const double thresh = d.rtol * bnorm;
  bool conv = rnorm <= thresh || bnorm == 0.0;
  int it_m = 0;
  double beta = 0.0;
  int pb = 0;
  for (int it = 0; it < max_it_all; ++it) {
    const bool work = !conv && it_m < d.max_it;
    const double* p_old = d.p[pb];
    double* p_new = d.p[pb ^ 1];
    const bool first = it_m == 0;
    if (work) {
      if (first) {
        for (int i = tid; i < n; i += tcount) p_new[i] = __ldcg(d.z + i);
      } else {
        for (int i = tid; i < n; i += tcount) p_new[i] = fma(beta, __ldcg(p_old + i), __ldcg(d.z + i));
      }
    }
    if (!grid_sync(w.bar, w.status)) return;
    double acc1[1] = {0.0};
    if (work)
      member_matvec(d, p_new, tid, tcount, [&](int r0, double s) {
        d.q[r0] = s;
        d.q32[r0] = (float)s;
        acc1[0] += __ldcg(p_new + r0) * s;
      });
    member_sum_add<1>(acc1, work ? 1.0 : 0.0, w, m, kred);
    if (!grid_sync(w.bar, w.status)) return;
    // every CTA: is any member still working?  (state at this iteration's start)
    if (__ldcg(w.red + (kred % 3) * (w.n + 1) * 4 + w.n * 4) == 0.0) break;
    const double pq = member_sum_read(w, m, kred, 0);
    ++kred;
    const double alpha = (work && pq != 0.0) ? rz / pq : 0.0;
    double* r_new = d.r[(it_m + 1) & 1];
    const double* r_old = r_cur;
    double acc2[2] = {0.0, 0.0};
    if (work) {
      for (int i = tid; i < n; i += tcount) {
        x[i] = fma(alpha, __ldcg(p_new + i), __ldcg(x + i));
        double rr = fma(-alpha, __ldcg(d.q + i), __ldcg(r_old + i));
        r_new[i] = rr;
        r32_alt[i] = (float)rr;
        acc2[1] += rr * rr;
      }
      const float a32 = (float)alpha;
      const float* r32o = r32_cur;
      member_rows32<FEMPIC_LPR_DT>(d.DT, tid, tcount, [&](int c) { return fmaf(-a32, __ldcg(d.q32 + c), __ldcg(r32o + c)); },
                       [&](int k, float s) { member_first_t(d, k, s); });
      member_rows32<16>(d.PiT, tid, tcount, [&](int c) { return fmaf(-a32, __ldcg(d.q32 + c), __ldcg(r32o + c)); },
                        [&](int k, float s) { member_first_u(d, k, s); });
    }
    const float *tv, *uv;
    if (!member_cheb(w, d, work, kc, tid, tcount, tv, uv)) return;
    if (!grid_sync(w.bar, w.status)) return;
    if (work) acc2[0] += member_z(d, r_new, tv, uv, tid, tcount);
    member_sum_add<2>(acc2, 0.0, w, m, kred);
    if (!grid_sync(w.bar, w.status)) return;
    const double rzn = member_sum_read(w, m, kred, 0), rrn = member_sum_read(w, m, kred, 1);
    ++kred;
    if (work) {
      ++it_m;
      r_cur = r_new;
      float* t32 = r32_cur;
      r32_cur = r32_alt;
      r32_alt = t32;
      pb ^= 1;
      rnorm = sqrt(rrn);
      conv = rnorm <= thresh;
      beta = rz != 0.0 ? rzn / rz : 0.0;
      rz = rzn;
    }
  }
  if (blockIdx.x == b0 && threadIdx.x == 0) {
    *d.cg_iters = it_m;
    *d.cg_res = bnorm > 0.0 ? rnorm / bnorm : 0.0;
    if (!conv) atomicOr(d.status, kStatusCG);
  }
}

}  // namespace dev
}  // namespace fempic
