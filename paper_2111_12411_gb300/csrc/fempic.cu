// C-ABI entry points of the EM-FEMPIC library (see include/fempic.h): handle
// life cycle, the per-step launch sequence, state transfer and operators.
//
// Step sequence (Section III-B; the PIC cycle of Section II):
//   [sort particles by tet] -> zero Delta g, rho ->
//   k_particle: gather E^n, B^n; Boris push; walk; deposit Delta g^{n+1}; rho^{n+1}
//   -> k_rhs: Newmark right-hand side -> k_pcg: ([*eps] + dt^2/4 K) e^{n+1} = rhs
//   -> k_bupdate: b^{n+1} = b^n - dt/2 C (e^{n+1} + e^n) -> [diagnostics]

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fempic.h"
#include "internal.h"
#include "kernels.cuh"
#include "linalg.cuh"
#include "particle_fast.cuh"
#include "batch.cuh"
#include "particle_ab4.cuh"
#include "project.cuh"
#include "inject.cuh"

namespace {
// Device allocations made by this library in this process (all handles and
// batches): reported by femPIC_get_info, so a caller can check that a call
// allocated nothing.
std::atomic<long long> g_device_allocations{0};

template <typename T>
cudaError_t counted_malloc(T** p, size_t bytes) {
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  if (e == cudaSuccess) g_device_allocations.fetch_add(1, std::memory_order_relaxed);
  return e;
}
}  // namespace

using namespace fempic;
using namespace fempic::dev;

namespace {

struct DevCSR {
  int32_t n_rows = 0, n_cols = 0;
  int64_t nnz = 0;
  int32_t* rp = nullptr;
  int32_t* ci = nullptr;
  double* v = nullptr;
  CsrView view(const double* vals = nullptr) const { return CsrView{n_rows, rp, ci, vals ? vals : v}; }
};

}  // namespace

struct FemPIC {
  femPIC_opts opts;
  std::string err;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  size_t bytes = 0;
  std::vector<void*> allocs;
  // model sizes
  int order = 1, nl0 = 4, nl1 = 6, nl2 = 4;
  int32_t n_nodes = 0, n_tets = 0, n_edges = 0, n_faces = 0, n0 = 0, n1 = 0, n2 = 0, n_bfaces = 0;
  // species
  double q = 0, m = 0, weight = 0;
  int64_t np = 0;
  // device mesh
  double* geom = nullptr;
  float* geom32 = nullptr;  // mixed precision: barycentric gradients [nt][12] in FP32
  float* e32 = nullptr;     // mixed precision: e and the sampled b rounded to FP32,
  float* b32 = nullptr;     // refreshed before every particle launch
  int32_t *nbr = nullptr, *dof0 = nullptr, *dof1 = nullptr, *dof2 = nullptr;
  uint8_t *pec1 = nullptr, *int0 = nullptr;
  double* load0 = nullptr;
  // matrices
  DevCSR M, K, Q, C, M2, D, DT, L, Pi, PiT;
  // order 2: the W1 system in 2x2 blocks (DOF pairs of one edge or face)
  int32_t nb = 0;
  int64_t nnzb = 0;
  int32_t *brp = nullptr, *bci = nullptr;
  double *bM = nullptr, *bK = nullptr, *bA = nullptr, *binv = nullptr;
  float* bA32 = nullptr;   // FP32 copy of bA: the CG's direction products (FEMPIC_PCG_FP32A)
  // Chebyshev smoother on B^-1 A (order 2, FP32 A): degree, whether it is in
  // use for the current system, its coefficients and its vectors
  int smooth_k = 1;
  bool smooth_on = false;
  float* chebS = nullptr;  // [3 * kMaxCheb] coefficients, written on the device
  uint16_t* bA16 = nullptr;  // bfloat16 copy of bA for the smoother's products
  float* binv32 = nullptr;   // FP32 copy of binv for the smoother
  float *sy = nullptr, *sd = nullptr;
  double kdiag_med = 0.0;  // median over W1 rows of K_ii / M_ii: the coefficient of K in A
                           // times it is the typical ratio of the curl-curl to the mass term
  bool pcg_fp32 = false;   // this dt's solves use the FP32 direction products
  double *dvM = nullptr, *dvK = nullptr;
  // FP32 copies for the preconditioner's auxiliary-space corrections
  float *D32 = nullptr, *DT32 = nullptr, *Pi32 = nullptr, *PiT32 = nullptr;
  float *dinvL32 = nullptr, *dinvV = nullptr, *aux_t = nullptr, *aux_u = nullptr;
  // Chebyshev smoothing of the auxiliary problems: V = Pi^T (M + c K) Pi on
  // the pattern of V_M = Pi^T M Pi (values of V_K beside it), FP32 copies of
  // V and L, the Chebyshev buffers, and host copies of V for its eigenvalue
  // bound (recomputed when dt changes)
  DevCSR V;
  double* VKv = nullptr;
  float *V32 = nullptr, *L32 = nullptr;
  float *aux_tf = nullptr, *aux_td = nullptr, *aux_t2 = nullptr, *aux_uf = nullptr, *aux_ud = nullptr,
        *aux_u2 = nullptr;
  std::vector<int32_t> hV_rp, hV_ci;
  std::vector<double> hV_m, hV_k;
  int cheb_k = 1;
  float chebL[3][kMaxCheb] = {}, chebV[3][kMaxCheb] = {};
  double *Aval = nullptr, *R1val = nullptr, *R2val = nullptr, *dinvA = nullptr, *dinvL = nullptr;
  // fields
  double *e = nullptr, *e_prev = nullptr, *e_new = nullptr, *b = nullptr, *dg = nullptr, *dg_prev = nullptr;
  double *rho = nullptr, *rho_prev = nullptr, *phi = nullptr, *rhs = nullptr;
  // CG scratch
  double *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_q = nullptr, *partials = nullptr;
  double *cg_r2 = nullptr, *cg_p2 = nullptr, *cg_red = nullptr;
  float *cg_q32 = nullptr, *cg_r32 = nullptr;
  float* cg_p32 = nullptr;  // FP32 copy of the search direction (FEMPIC_PCG_FP32A)
  GridBarrier* bar = nullptr;
  int pcg_blocks_w1 = 0, pcg_blocks_w0 = 0;
  int32_t* apart = nullptr;  // [pcg_blocks_w1 + 1] per-CTA row ranges of A in the CG
  // impedance (first-order absorbing) faces: Y0 <n x W1, n x W1> on M's pattern
  // and, at order 2, in 2x2 blocks; null without such faces
  int32_t n_imp_faces = 0;
  double *Iv = nullptr, *bI = nullptr;
  // with impedance faces: the preconditioner's gradient space (W0 DOFs off
  // PEC faces), its Laplacian L_a = D_a^T ([*eps] + c_I [*_I]) D_a formed when
  // dt changes (values LA.v + c_I LAI in LAdt), FP32 copies, Chebyshev
  // coefficients, host copies for the eigenvalue bound
  // order 3: block Jacobi of A over the W1 DOF groups (edge, face, interior)
  int32_t n_groups = 0;
  int32_t* gstart = nullptr;
  uint8_t* gsize = nullptr;
  DevCSR Bg;
  DevCSR DA, DAT, LA;
  double *LAI = nullptr, *LAdt = nullptr, *dinvLA = nullptr;
  float *DA32 = nullptr, *DAT32 = nullptr, *LA32 = nullptr, *dinvLA32 = nullptr;
  std::vector<int32_t> hLA_rp, hLA_ci;
  std::vector<double> hLA_m, hLA_i;
  float chebLA[3][kMaxCheb] = {};
  // with the smoother: the degree of the auxiliary Chebyshev steps and their
  // coefficients (same bounds, more steps), and the bounds they come from
  int cheb_k_sm = 1;
  float chebL_sm[3][kMaxCheb] = {}, chebV_sm[3][kMaxCheb] = {}, chebLA_sm[3][kMaxCheb] = {};
  double lmaxL = 0.0;
  // species: ids [sp_off[k], sp_off[k+1]) belong to species k
  // Adams-Bashforth push: history v^{n-1-j}, a^{n-1-j} per particle (device
  // order; the particles are not re-sorted), entries filled so far
  double* ab_vh[3][3] = {};
  double* ab_ah[3][3] = {};
  int ab_count = 0;
  int n_species = 1;
  int64_t sp_off[kMaxSpecies + 1] = {};
  double sp_q[kMaxSpecies] = {}, sp_m[kMaxSpecies] = {}, sp_w[kMaxSpecies] = {};
  // particles (device order), SoA
  double* px[3] = {nullptr, nullptr, nullptr};
  double* pv[3] = {nullptr, nullptr, nullptr};
  double* alt[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* stage = nullptr;  // [3*np] staging for particle-id ordered transfers
  int32_t *ptet = nullptr, *pid = nullptr, *ptet_alt = nullptr, *pid_alt = nullptr;
  int32_t *pncross = nullptr;
  unsigned long long* phash = nullptr;
  int32_t *sort_cnt = nullptr, *sort_off = nullptr, *sort_sums = nullptr, *sort_sums2 = nullptr;
  // status / counters
  int32_t* d_status = nullptr;
  int32_t* d_cg_iters = nullptr;
  double* d_cg_res = nullptr;
  double* d_norms = nullptr;  // [6]: continuity abs^2, ref^2, gauss abs^2, ref^2, div b abs^2, ref^2
  double* divref = nullptr;   // [n3][nl2] int_ref W3_i div W2_j (div b diagnostic)
  int32_t n3 = 0;
  unsigned long long* d_cross = nullptr;
  unsigned long long* d_first = nullptr;  // first bad element of a staged host transfer (all ones: none)
  double* d_tmp1 = nullptr;  // N1 scratch
  double* d_tmp0 = nullptr;  // N0 scratch
  double dt_cur = -1.0;
  int64_t steps = 0;
  int64_t since_sort = 0;
  // timing of the last femPIC_step call
  std::vector<cudaEvent_t> ev;
  double t_particle_ms = 0, t_field_ms = 0;
  double t_sort_ms = 0, t_push_ms = 0, t_rhs_ms = 0, t_pcg_ms = 0, t_bupd_ms = 0;
  int64_t cg_iters_sum = 0;
  int32_t* d_cg_iters_acc = nullptr;  // sum of CG iterations since the last sync
  int launches = 0;
  int pending_steps = 0;
  // impressed magnetic flux density (Section III-C): W2 coefficients bimp and
  // the sum btot = b + bimp the particles sample; null until one is set.  The
  // mesh as given (sorted tets) is kept for the projection's quadrature points.
  double *bimp = nullptr, *btot = nullptr;
  std::vector<double> hxyz;
  std::vector<int32_t> htets;
  // particle walls: absorbing faces (nbr = -2), injection faces (sorted
  // vertices, owning tet, running area), per-particle absorbed flags of the
  // last step, the injectors and the absorbed count of the last call
  int32_t n_absorb_faces = 0, n_inj_faces = 0;
  double *inj_xyz = nullptr, *inj_cum = nullptr;
  int32_t* inj_tet = nullptr;
  uint8_t* pabs = nullptr;
  bool inj_has[kMaxSpecies] = {};
  double inj_drift[kMaxSpecies][3] = {}, inj_sigma[kMaxSpecies][3] = {};
  uint64_t inj_seed = 0;
  unsigned long long* d_absorbed = nullptr;
};

// the flux the particles see (self field, plus the impressed one if set)
inline const double* b_gather(const FemPIC* h) { return h->bimp ? h->btot : h->b; }

static_assert(kMaxSpecies == FEMPIC_MAX_SPECIES, "species table size");

namespace {

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
      return FEMPIC_ERR_CUDA;                                                      \
    }                                                                              \
  } while (0)

template <class T>
int dalloc(FemPIC* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = counted_malloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    h->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? FEMPIC_ERR_OOM : FEMPIC_ERR_CUDA;
  }
  h->allocs.push_back(*p);
  h->bytes += count * sizeof(T);
  return FEMPIC_OK;
}

template <class T>
int upload(FemPIC* h, T** p, const std::vector<T>& src) {
  int rc = dalloc(h, p, src.size());
  if (rc) return rc;
  if (!src.empty()) CK(cudaMemcpy(*p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FEMPIC_OK;
}

int upload_csr(FemPIC* h, DevCSR* d, const HostCSR& s) {
  d->n_rows = s.n_rows;
  d->n_cols = s.n_cols;
  d->nnz = s.nnz();
  int rc = upload(h, &d->rp, s.rowptr);
  if (!rc) rc = upload(h, &d->ci, s.col);
  if (!rc) rc = upload(h, &d->v, s.val);
  return rc;
}

CsrView32 view32(const DevCSR& m, const float* v) { return CsrView32{m.n_rows, m.rp, m.ci, v}; }

inline int grid_for(int64_t work, int block, int cap) {
  int64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  return (int)std::min<int64_t>(g, cap);
}

// Degree of the Chebyshev smoothing of the auxiliary problems and the ratio
// lambda_max / lambda_min of the interval it damps.  Degree 4 cuts the CG
// iterations of the drift-tube (p = 2) and box (p = 1, 2) systems by 2.0-2.4x
// against diagonal scaling (degree 1); higher degrees gain little because the
// block-Jacobi part then limits.
#ifndef FEMPIC_AUX_CHEB
#define FEMPIC_AUX_CHEB 4
#endif
constexpr double kChebRatio = 100.0;

// Chebyshev smoother on B^-1 A (order 2): degree (1 = block Jacobi alone),
// power-iteration steps for its largest eigenvalue, the margin put on that
// estimate (the power iteration approaches it from below) and the ratio of
// the damped interval.  Each degree above 1 costs one A product per
// iteration (bfloat16 values), run in a phase of the auxiliary Chebyshev
// steps.  The degree is odd: the smoother's polynomial p(lambda) then stays
// positive for every lambda > 0, beyond the damped interval too, so the
// preconditioner is positive definite whatever the eigenvalue estimate (at
// even degrees p turns negative just above the interval).  Drift tube at
// p = 2 (full size, live timing, ms per step): block Jacobi with 4 auxiliary
// steps 55.3 (173.8 iterations); degree 3, 6 steps 46.1 (100.5); degree 5,
// 8 steps 45.0 (73.5); degree 4, 8 steps 45.0 (79.5).
#ifndef FEMPIC_SMOOTH_DEG
#define FEMPIC_SMOOTH_DEG 5
#endif
// auxiliary Chebyshev degree while the smoother is in use
#ifndef FEMPIC_AUX_CHEB_SMOOTH
#define FEMPIC_AUX_CHEB_SMOOTH 8
#endif
constexpr int kSmoothPower = 40;
constexpr double kSmoothMargin = 1.1;
constexpr double kSmoothRatio = 10.0;

// Chebyshev iteration for a Jacobi-scaled SPD matrix whose scaled spectrum is
// taken as [lmax / kChebRatio, lmax]: step 0 sets y = dinv f / theta; step i
// sets d <- c1_i d + c2_i dinv (f - A y), y <- y + d.  Degree 1 (or no bound)
// leaves the diagonal scaling y = dinv f.
void cheb_coeffs(double lmax, int k, float (&c)[3][kMaxCheb], double ratio = kChebRatio) {
  for (auto& row : c)
    for (float& v : row) v = 0.f;
  if (k <= 1 || !(lmax > 0.0)) {
    c[0][0] = 1.f;
    return;
  }
  const double lmin = lmax / ratio, th = 0.5 * (lmax + lmin), de = 0.5 * (lmax - lmin);
  const double sig = th / de;
  double rho = 1.0 / sig;
  c[0][0] = (float)(1.0 / th);
  for (int i = 1; i < k; ++i) {
    const double rn = 1.0 / (2.0 * sig - rho);
    c[1][i] = (float)(rn * rho);
    c[2][i] = (float)(2.0 * rn / de);
    rho = rn;
  }
}

// species table of a launch: q w and q dt / 2m per species (the same
// expressions as the single-species scalars)
SpeciesTable species_table(const FemPIC* h, double dt) {
  SpeciesTable t;
  memset(&t, 0, sizeof(t));
  t.n = h->n_species;
  for (int k = 0; k <= h->n_species && k <= kMaxSpecies; ++k) t.off[k] = (int32_t)h->sp_off[k];
  for (int k = 0; k < h->n_species; ++k) {
    t.qw[k] = h->sp_q[k] * h->sp_w[k];
    t.h[k] = ((h->sp_q[k] / h->sp_m[k]) * dt) * 0.5;
  }
  return t;
}

// Cut rows 0..n-1 (prefix of stored entries `pre`, pre[n] = total) into
// `parts` contiguous ranges of about equal cost, a row costing its entries
// plus two (its pointer loads and result store); returns parts + 1 bounds.
std::vector<int32_t> balanced_ranges(const std::vector<int64_t>& pre, int parts) {
  const int64_t n = (int64_t)pre.size() - 1;
  const int64_t total = pre[n] + 2 * n;
  std::vector<int32_t> out((size_t)parts + 1, 0);
  int64_t r = 0;
  for (int b = 1; b < parts; ++b) {
    const int64_t target = total * b / parts;
    while (r < n && pre[r] + 2 * r < target) ++r;
    out[b] = (int32_t)r;
  }
  out[parts] = (int32_t)n;
  return out;
}

// Gershgorin bound of the spectrum of diag(A)^-1 A, A = a + c b on one CSR
// pattern (b may be null): max over rows with a positive diagonal of
// sum_j |A_ij| / A_ii.
double gershgorin_scaled(const std::vector<int32_t>& rp, const std::vector<int32_t>& ci, const double* a,
                         const double* b, double c) {
  double best = 0.0;
  const int32_t n = (int32_t)rp.size() - 1;
  for (int32_t i = 0; i < n; ++i) {
    double sum = 0.0, diag = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const double v = b ? a[k] + c * b[k] : a[k];
      sum += std::fabs(v);
      if (ci[k] == i) diag = v;
    }
    if (diag > 0.0) best = std::max(best, sum / diag);
  }
  return best;
}


// lanes per CSR row of the order-2 system matrix (rows of ~30-75 entries);
// 4 measured faster than 8 and 16 in the persistent CG
#ifndef FEMPIC_LPR_P2
#define FEMPIC_LPR_P2 4
#endif
int lpr_w1(const FemPIC* h) { return h->order == 1 ? 4 : FEMPIC_LPR_P2; }

int latch_status(FemPIC* h) {
  int32_t st = 0;
  CK(cudaMemcpyAsync(&st, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (st & kStatusBarrier) {
    h->err = "device grid barrier timed out";
    return FEMPIC_ERR_BARRIER;
  }
  if (st & kStatusWalk) {
    h->err = "a particle reached the face-crossing cap (max_cross)";
    return FEMPIC_ERR_WALK;
  }
  if (st & kStatusCG) {
    h->err = "CG reached its iteration cap before the tolerance";
    return FEMPIC_ERR_CG;
  }
  if (st & kStatusBounds) {
    h->err = "a tet id or DOF index was out of range (checked build)";
    return FEMPIC_ERR_BOUNDS;
  }
  return FEMPIC_OK;
}

template <int LPR>
int launch_spmv(FemPIC* h, const CsrView& A, const double* x, double* y, double alpha, double beta) {
  int grid = grid_for((int64_t)A.n_rows * LPR, 256, h->num_sms * 16);
  k_spmv<LPR><<<grid, 256, 0, h->stream>>>(A, x, y, alpha, beta);
  h->launches++;
  CK(cudaGetLastError());
  return FEMPIC_OK;
}

int spmv(FemPIC* h, const CsrView& A, const double* x, double* y, double alpha = 1.0, double beta = 0.0) {
  return h->order == 1 ? launch_spmv<4>(h, A, x, y, alpha, beta) : launch_spmv<8>(h, A, x, y, alpha, beta);
}

// co-resident blocks of the persistent PCG kernel, or -1 on error
template <int LPR>
int pcg_blocks(FemPIC* h) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<LPR>, FEMPIC_PCG_THREADS, 0);
  if (e != cudaSuccess) {
    h->err = std::string("occupancy query: ") + cudaGetErrorString(e);
    return -1;
  }
  return std::max(1, per_sm) * h->num_sms;
}

// Solve A x = rhs (x holds the initial guess) on the device; with nodal, the
// preconditioner adds the auxiliary nodal correction D L_diag^-1 D^T.
int run_pcg(FemPIC* h, const CsrView& A, const double* dinv, const double* rhs, double* x, int blocks,
            bool nodal) {
  PcgArgs a;
  a.A = A;
  a.dinv = dinv;
  const bool imp = nodal && h->LA.nnz > 0;  // gradient space with the impedance faces' W0 DOFs
  a.D = imp ? view32(h->DA, h->DA32) : nodal ? view32(h->D, h->D32) : CsrView32{0, nullptr, nullptr, nullptr};
  a.DT = imp ? view32(h->DAT, h->DAT32) : nodal ? view32(h->DT, h->DT32) : CsrView32{0, nullptr, nullptr, nullptr};
  a.dinvL = imp ? h->dinvLA32 : h->dinvL32;
  a.t = h->aux_t;
  a.Pi = nodal ? view32(h->Pi, h->Pi32) : CsrView32{0, nullptr, nullptr, nullptr};
  a.PiT = nodal ? view32(h->PiT, h->PiT32) : CsrView32{0, nullptr, nullptr, nullptr};
  a.dinvV = h->dinvV;
  a.u = h->aux_u;
  a.L = imp ? view32(h->LA, h->LA32) : nodal ? view32(h->L, h->L32) : CsrView32{0, nullptr, nullptr, nullptr};
  a.V = (nodal && h->V.nnz > 0) ? view32(h->V, h->V32) : CsrView32{0, nullptr, nullptr, nullptr};
  a.tf = h->aux_tf;
  a.td = h->aux_td;
  a.t2 = h->aux_t2;
  a.uf = h->aux_uf;
  a.ud = h->aux_ud;
  a.u2 = h->aux_u2;
  // the smoother runs with cheb_k_sm auxiliary steps (its products share their phases)
  const bool smooth = nodal && h->nb > 0 && h->smooth_on;
  a.cheb_k = !nodal ? 1 : smooth ? h->cheb_k_sm : h->cheb_k;
  memcpy(a.chebL, imp ? (smooth ? h->chebLA_sm : h->chebLA) : (smooth ? h->chebL_sm : h->chebL), sizeof(a.chebL));
  memcpy(a.chebV, smooth ? h->chebV_sm : h->chebV, sizeof(a.chebV));
  a.Bg = (nodal && h->Bg.nnz > 0) ? h->Bg.view() : CsrView{0, nullptr, nullptr, nullptr};
  a.Ab = (nodal && h->nb > 0) ? BsrView{h->nb, h->brp, h->bci, h->bA} : BsrView{0, nullptr, nullptr, nullptr};
  a.Ab32 = (nodal && h->nb > 0 && h->pcg_fp32) ? BsrView32{h->nb, h->brp, h->bci, h->bA32}
                                               : BsrView32{0, nullptr, nullptr, nullptr};
  a.p32 = h->cg_p32;
  a.repl = kPcgReplacePeriod;
  a.smooth_k = (smooth && a.cheb_k >= h->smooth_k) ? h->smooth_k : 1;
  a.chebS = h->chebS;
  a.As16 = a.smooth_k > 1 ? BsrView16{h->nb, h->brp, h->bci, h->bA16} : BsrView16{0, nullptr, nullptr, nullptr};
  a.binv32 = h->binv32;
  a.sy = h->sy;
  a.sd = h->sd;
  a.q32 = h->cg_q32;
  a.r32 = h->cg_r32;
  a.red = h->cg_red;
  a.binv = h->binv;
  a.Apart = (nodal && blocks == h->pcg_blocks_w1) ? h->apart : nullptr;
  a.rhs = rhs;
  a.x = x;
  a.r[0] = h->cg_r;
  a.r[1] = h->cg_r2;
  a.z = h->cg_z;
  a.p[0] = h->cg_p;
  a.p[1] = h->cg_p2;
  a.q = h->cg_q;
  a.partials[0] = h->partials;
  a.partials[1] = h->partials + 4 * (size_t)blocks;
  a.bar = h->bar;
  a.status = h->d_status;
  a.iters_out = h->d_cg_iters;
  a.res_out = h->d_cg_res;
  a.rtol = h->opts.cg_rtol;
  a.max_it = h->opts.cg_max_it;
  CK(cudaMemsetAsync(h->bar, 0, sizeof(GridBarrier), h->stream));
  CK(cudaMemsetAsync(h->cg_red, 0, 12 * sizeof(double), h->stream));
  void* args[] = {&a};
  if (h->order == 1)
    CK(cudaLaunchCooperativeKernel((void*)k_pcg<4>, blocks, FEMPIC_PCG_THREADS, args, 0, h->stream));
  else
    CK(cudaLaunchCooperativeKernel((void*)k_pcg<FEMPIC_LPR_P2>, blocks, FEMPIC_PCG_THREADS, args, 0, h->stream));
  h->launches++;
  return FEMPIC_OK;
}

// Coefficients of the Chebyshev smoother for the current system, all on the
// device: the largest eigenvalue of B^-1 A (B: A's 2x2 diagonal blocks) by
// kSmoothPower steps of the power iteration from a hashed start vector, as
// the Rayleigh quotient x.(A x) / x.(B x) of the last iterate (B x is the
// A x_prev of the step before, since x = B^-1 (A x_prev)), then the
// coefficients from it.  Uses the CG's scratch vectors; no host synchronisation.
int smoother_coeffs(FemPIC* h) {
  const int32_t n = 2 * h->nb;
  const CsrView A = h->M.view(h->Aval);
  double* x = h->cg_z;
  double* yp = h->cg_q;
  double* yc = h->cg_r;
  const int g = grid_for(n, 256, h->num_sms * 8);
  k_hash_vector<<<g, 256, 0, h->stream>>>(n, x);
  int rc = 0;
  for (int it = 0; it < kSmoothPower; ++it) {
    if ((rc = spmv(h, A, x, yp))) return rc;
    k_block_apply<<<g, 256, 0, h->stream>>>(h->nb, h->binv, yp, x);
  }
  if ((rc = spmv(h, A, x, yc))) return rc;
  CK(cudaMemsetAsync(h->cg_red, 0, 2 * sizeof(double), h->stream));
  k_dot2<<<g, 256, 0, h->stream>>>(n, x, yc, yp, h->cg_red);
  k_smooth_coeffs<<<1, 32, 0, h->stream>>>(h->cg_red, h->smooth_k, kSmoothMargin, kSmoothRatio, h->chebS);
  CK(cudaGetLastError());
  h->launches += 2 * kSmoothPower + 3;
  return FEMPIC_OK;
}

int form_system(FemPIC* h, double dt) {
  double c1;
  double cr1, cr2 = 0.0;
  if (h->opts.scheme == FEMPIC_SCHEME_TRAPEZOID) {
    c1 = 0.25 * dt * dt;
    cr1 = -0.25 * dt * dt;  // R1 = M - dt^2/4 K
  } else {
    double g = h->opts.gamma, be = h->opts.beta;
    c1 = be * dt * dt;
    double c2 = 0.5 + g - 2.0 * be, c3 = 0.5 - g + be;
    cr1 = -c2 * dt * dt;  // R1 = 2M - c2 dt^2 K  (M part doubled below)
    cr2 = c3 * dt * dt;   // R2 = M + c3 dt^2 K
  }
  int grid = grid_for(h->n1, 256, 1 << 30);
  // impedance faces (trapezoid only): A += dt/2 I, R1 -= dt/2 I
  const double ci_imp = h->Iv ? 0.5 * dt : 0.0;
  // FP32 direction products only while the curl-curl term stays within
  // kPcgFp32MaxRatio of the mass term (median over the rows): beyond it the
  // cancellation in A x of gradient fields outgrows what FP32 products and
  // the FP64 residual replacement can follow
  h->pcg_fp32 = h->bA32 && h->kdiag_med * c1 <= kPcgFp32MaxRatio;
  k_form_system<<<grid, 256, 0, h->stream>>>(h->n1, h->M.rp, h->M.ci, h->M.v, h->K.v, c1, cr1, h->Aval, h->R1val,
                                             h->dinvA, h->Iv, ci_imp, -ci_imp);
  h->launches++;
  CK(cudaGetLastError());
  if (h->opts.scheme == FEMPIC_SCHEME_WAVE) {
    // R1 = 2M - c2 dt^2 K = (M - c2 dt^2 K) + M: form as M*2 via a second pass
    // using R2 scratch: R2 <- M + cr2 K; R1 <- R1 + M
    k_form_system<<<grid, 256, 0, h->stream>>>(h->n1, h->M.rp, h->M.ci, h->M.v, h->K.v, cr2, 0.0, h->R2val, nullptr,
                                               h->d_tmp1);
    h->launches++;
    CK(cudaGetLastError());
    // R1 += M (reuse k_form_system with a = R1 + 1*M by passing m=R1 and k=M)
    k_form_system<<<grid, 256, 0, h->stream>>>(h->n1, h->M.rp, h->M.ci, h->R1val, h->M.v, 1.0, 0.0, h->R1val,
                                               nullptr, h->d_tmp1);
    h->launches++;
    CK(cudaGetLastError());
  }
  k_form_dv<<<grid_for(h->PiT.n_rows, 256, 1 << 30), 256, 0, h->stream>>>(h->PiT.n_rows, h->dvM, h->dvK, c1,
                                                                            h->dinvV);
  if (h->V.nnz > 0) {
    k_axpy_to_f32<<<grid_for(h->V.nnz, 256, 4096), 256, 0, h->stream>>>(h->V.nnz, h->V.v, h->VKv, c1, h->V32);
    h->launches++;
    const double lv = gershgorin_scaled(h->hV_rp, h->hV_ci, h->hV_m.data(), h->hV_k.data(), c1);
    cheb_coeffs(lv, h->cheb_k, h->chebV);
    cheb_coeffs(lv, h->cheb_k_sm, h->chebV_sm);
  }
  if (h->nb > 0) {
    k_form_blocks<<<grid_for(h->nb, 256, 1 << 30), 256, 0, h->stream>>>(h->nb, h->brp, h->bci, h->bM, h->bK, c1,
                                                                        h->bA, h->binv, h->bI, ci_imp);
    h->launches++;
    if (h->bA32 && (h->pcg_fp32 || (h->smooth_k > 1 && h->sy))) {
      k_to_f32<<<grid_for(4 * h->nnzb, 256, 4096), 256, 0, h->stream>>>(4 * h->nnzb, h->bA, h->bA32);
      h->launches++;
    }
  }
  // the smoother's products take bfloat16 values of A whether or not the
  // direction products are FP32: it is a fixed symmetric operator either way
  // (host study, 12^3 box at c dt / h = 150 with FP64 direction products:
  // 94 iterations with block Jacobi, 44 with the degree-5 smoother)
  h->smooth_on = h->smooth_k > 1 && h->sy;
  if (h->smooth_on) {
    k_to_bf16<<<grid_for(4 * h->nnzb, 256, 4096), 256, 0, h->stream>>>(4 * h->nnzb, h->bA32, h->bA16);
    k_to_f32<<<grid_for(4 * h->nb, 256, 4096), 256, 0, h->stream>>>(4 * h->nb, h->binv, h->binv32);
    h->launches += 2;
    int rc = smoother_coeffs(h);
    if (rc) return rc;
  }
  if (h->Bg.nnz > 0) {
    k_group_inverse<<<grid_for(h->n_groups, 128, 1 << 30), 128, 0, h->stream>>>(
        h->n_groups, h->gstart, h->gsize, h->M.view(h->Aval), h->Bg.rp, h->Bg.v);
    h->launches++;
    CK(cudaGetLastError());
  }
  if (h->LA.nnz > 0) {
    // L_a = D_a^T ([*eps] + dt/2 [*_I]) D_a: the gradients of W0 on impedance faces see the boundary term
    const int32_t nnz = (int32_t)h->LA.nnz;
    k_lincomb<<<grid_for(nnz, 256, 4096), 256, 0, h->stream>>>(nnz, h->LA.v, h->LAI, 1.0, ci_imp, h->LAdt);
    k_to_f32<<<grid_for(nnz, 256, 4096), 256, 0, h->stream>>>(nnz, h->LAdt, h->LA32);
    k_inv_diag<<<grid_for(h->n0, 256, 1 << 30), 256, 0, h->stream>>>(h->n0, h->LA.rp, h->LA.ci, h->LAdt, h->dinvLA);
    k_to_f32<<<grid_for(h->n0, 256, 4096), 256, 0, h->stream>>>(h->n0, h->dinvLA, h->dinvLA32);
    h->launches += 4;
    CK(cudaGetLastError());
    if (h->cheb_k > 1) {
      const double la = gershgorin_scaled(h->hLA_rp, h->hLA_ci, h->hLA_m.data(), h->hLA_i.data(), ci_imp);
      cheb_coeffs(la, h->cheb_k, h->chebLA);
      cheb_coeffs(la, h->cheb_k_sm, h->chebLA_sm);
    } else {
      cheb_coeffs(0.0, 1, h->chebLA);
      cheb_coeffs(0.0, 1, h->chebLA_sm);
    }
  }
  h->launches++;
  CK(cudaGetLastError());
  h->dt_cur = dt;
  return FEMPIC_OK;
}

int measure_rho(FemPIC* h, double* rho_out) {
  CK(cudaMemsetAsync(rho_out, 0, sizeof(double) * h->n0, h->stream));
  if (h->np == 0) return FEMPIC_OK;
  int grid = grid_for(h->np, 256, 1 << 30);
  double qw = h->q * h->weight;
  const SpeciesTable st = species_table(h, 0.0);
  if (h->order == 1)
    k_rho<1><<<grid, 256, 0, h->stream>>>(h->np, h->px[0], h->px[1], h->px[2], h->ptet, h->geom, h->dof0, qw,
                                          rho_out, h->pid, st);
  else if (h->order == 2)
    k_rho<2><<<grid, 256, 0, h->stream>>>(h->np, h->px[0], h->px[1], h->px[2], h->ptet, h->geom, h->dof0, qw,
                                          rho_out, h->pid, st);
  else
    k_rho<3><<<grid, 256, 0, h->stream>>>(h->np, h->px[0], h->px[1], h->px[2], h->ptet, h->geom, h->dof0, qw,
                                          rho_out, h->pid, st);
  h->launches++;
  CK(cudaGetLastError());
  return FEMPIC_OK;
}

// exclusive scan of cnt[0..n) into off (recursive over 1024-element tiles)
int scan_excl(FemPIC* h, int32_t n, const int32_t* in, int32_t* out, int32_t* sums, int32_t* sums2) {
  int tiles = (n + 1023) / 1024;
  k_scan_tiles<<<tiles, 1024, 0, h->stream>>>(n, in, out, tiles > 1 ? sums : nullptr);
  h->launches++;
  CK(cudaGetLastError());
  if (tiles > 1) {
    if (tiles > 1024 * 1024) {
      h->err = "too many tets for the scan";
      return FEMPIC_ERR_ARG;
    }
    int t2 = (tiles + 1023) / 1024;
    k_scan_tiles<<<t2, 1024, 0, h->stream>>>(tiles, sums, sums, t2 > 1 ? sums2 : nullptr);
    h->launches++;
    if (t2 > 1) {
      k_scan_tiles<<<1, 1024, 0, h->stream>>>(t2, sums2, sums2, nullptr);
      k_scan_add<<<t2, 1024, 0, h->stream>>>(tiles, sums, sums2);
      h->launches += 2;
    }
    k_scan_add<<<tiles, 1024, 0, h->stream>>>(n, out, sums);
    h->launches++;
    CK(cudaGetLastError());
  }
  return FEMPIC_OK;
}

int sort_particles(FemPIC* h) {
  if (h->np == 0) return FEMPIC_OK;
  CK(cudaMemsetAsync(h->sort_cnt, 0, sizeof(int32_t) * h->n_tets, h->stream));
  int grid = grid_for(h->np, 256, 1 << 30);
  k_hist<<<grid, 256, 0, h->stream>>>(h->np, h->ptet, h->sort_cnt);
  h->launches++;
  CK(cudaGetLastError());
  int rc = scan_excl(h, h->n_tets, h->sort_cnt, h->sort_off, h->sort_sums, h->sort_sums2);
  if (rc) return rc;
  SortArgs a;
  a.n = h->np;
  a.tet_in = h->ptet;
  a.cursor = h->sort_off;
  for (int k = 0; k < 3; ++k) {
    a.src[k] = h->px[k];
    a.src[3 + k] = h->pv[k];
    a.dst[k] = h->alt[k];
    a.dst[3 + k] = h->alt[3 + k];
  }
  a.ti[0] = h->ptet;
  a.ti[1] = h->pid;
  a.to[0] = h->ptet_alt;
  a.to[1] = h->pid_alt;
  k_sort_scatter<<<grid, 256, 0, h->stream>>>(a);
  h->launches++;
  CK(cudaGetLastError());
  for (int k = 0; k < 3; ++k) {
    std::swap(h->px[k], h->alt[k]);
    std::swap(h->pv[k], h->alt[3 + k]);
  }
  std::swap(h->ptet, h->ptet_alt);
  std::swap(h->pid, h->pid_alt);
  return FEMPIC_OK;
}

int launch_particles(FemPIC* h, double dt) {
  ParticleArgs a;
  a.n = h->np;
  for (int k = 0; k < 3; ++k) {
    a.x[k] = h->px[k];
    a.v[k] = h->pv[k];
  }
  a.tet = h->ptet;
  a.ncross = h->pncross;
  a.hash = h->phash;
  a.geom = h->geom;
  a.nbr = h->nbr;
  a.dof0 = h->dof0;
  a.dof1 = h->dof1;
  a.dof2 = h->dof2;
  a.e = h->e;
  a.b = b_gather(h);
  a.dg = h->dg;
  a.rho = h->rho;
  for (int k = 0; k < 3; ++k) a.B0[k] = h->opts.B0[k];
  a.h = ((h->q / h->m) * dt) * 0.5;
  a.dt = dt;
  a.qw = h->q * h->weight;
  a.max_cross = h->opts.max_cross;
  a.status = h->d_status;
  a.crossings = h->d_cross;
  a.pid = h->pid;
  a.sp = species_table(h, dt);
  a.absorbed = h->pabs;
  a.n_tets = h->n_tets;
  if (h->np == 0) return FEMPIC_OK;
  if (h->e32 && h->opts.precision == FEMPIC_MIXED && h->opts.push != FEMPIC_PUSH_AB4 && h->order <= 2) {
    // the mixed gather's FP32 copies of this step's e and sampled b
    k_to_f32<<<grid_for(h->n1, 256, 4096), 256, 0, h->stream>>>(h->n1, h->e, h->e32);
    k_to_f32<<<grid_for(h->n2, 256, 4096), 256, 0, h->stream>>>(h->n2, a.b, h->b32);
    h->launches += 2;
    CK(cudaGetLastError());
    a.e32 = h->e32;
    a.b32 = h->b32;
    a.geom32 = h->geom32;
  }
  if (h->opts.push == FEMPIC_PUSH_AB4) {
    Ab4Args A;
    A.p = a;
    for (int j = 0; j < 3; ++j)
      for (int c = 0; c < 3; ++c) {
        A.vh[j][c] = h->ab_vh[j][c];
        A.ah[j][c] = h->ab_ah[j][c];
      }
    A.k = std::min(4, h->ab_count + 1);
    A.qm = h->q / h->m;
    for (int k = 0; k < kMaxSpecies; ++k) A.qm_s[k] = k < h->n_species ? h->sp_q[k] / h->sp_m[k] : 0.0;
    const int g128 = grid_for(h->np, 128, 1 << 30);
    auto launch = [&](auto kern) { kern<<<g128, 128, 0, h->stream>>>(A); };
    if (h->order == 1) {
      switch (A.k) {
        case 1: launch(k_particle_ab4<1, 1>); break;
        case 2: launch(k_particle_ab4<1, 2>); break;
        case 3: launch(k_particle_ab4<1, 3>); break;
        default: launch(k_particle_ab4<1, 4>); break;
      }
    } else {
      switch (A.k) {
        case 1: launch(k_particle_ab4<2, 1>); break;
        case 2: launch(k_particle_ab4<2, 2>); break;
        case 3: launch(k_particle_ab4<2, 3>); break;
        default: launch(k_particle_ab4<2, 4>); break;
      }
    }
    h->launches++;
    CK(cudaGetLastError());
    h->ab_count = std::min(3, h->ab_count + 1);
    return FEMPIC_OK;
  }
  int grid = grid_for(h->np, 256, 1 << 30);
  bool strict = h->opts.precision == FEMPIC_FP64_STRICT;
  // lanes share tets only right after a sort
  const bool agg = FEMPIC_PARTICLE_AGG && h->opts.sort_period == 1;
  const bool mixed = h->opts.precision == FEMPIC_MIXED;
  if (h->order == 1) {
    if (strict)
      k_particle<1, Strict><<<grid, 256, 0, h->stream>>>(a);
    else if (mixed)
      agg ? k_particle_fast<1, true, true><<<grid, 256, 0, h->stream>>>(a)
          : k_particle_fast<1, false, true><<<grid, 256, 0, h->stream>>>(a);
    else
      agg ? k_particle_fast<1, true, false><<<grid, 256, 0, h->stream>>>(a)
          : k_particle_fast<1, false, false><<<grid, 256, 0, h->stream>>>(a);
  } else if (h->order == 3) {
    // order 3 has no hand-factored fast forms: the generic kernel, one rounding
    // per operation when strict, contracted otherwise
    if (strict)
      k_particle<3, Strict><<<grid, 256, 0, h->stream>>>(a);
    else
      k_particle<3, Fast><<<grid, 256, 0, h->stream>>>(a);
  } else {
    if (strict)
      k_particle<2, Strict><<<grid, 256, 0, h->stream>>>(a);
    else if (mixed)
      agg ? k_particle_fast<2, true, true><<<grid, 256, 0, h->stream>>>(a)
          : k_particle_fast<2, false, true><<<grid, 256, 0, h->stream>>>(a);
    else
      agg ? k_particle_fast<2, true, false><<<grid, 256, 0, h->stream>>>(a)
          : k_particle_fast<2, false, false><<<grid, 256, 0, h->stream>>>(a);
  }
  h->launches++;
  CK(cudaGetLastError());
  if (h->n_absorb_faces > 0) {
    InjectArgs in;
    in.n = h->np;
    for (int k = 0; k < 3; ++k) {
      in.x[k] = h->px[k];
      in.v[k] = h->pv[k];
    }
    in.tet = h->ptet;
    in.absorbed = h->pabs;
    in.pid = h->pid;
    in.geom = h->geom;
    in.dof0 = h->dof0;
    in.rho = h->rho;
    in.face_xyz = h->inj_xyz;
    in.face_tet = h->inj_tet;
    in.face_cum = h->inj_cum;
    in.n_faces = h->n_inj_faces;
    in.seed = h->inj_seed;
    in.step = (uint64_t)h->steps;
    in.sp = species_table(h, dt);
    for (int k = 0; k < kMaxSpecies; ++k)
      for (int c = 0; c < 3; ++c) {
        in.drift[k][c] = h->inj_drift[k][c];
        in.sigma[k][c] = h->inj_sigma[k][c];
      }
    in.count = h->d_absorbed;
    if (h->order == 1)
      k_inject<1><<<grid, 256, 0, h->stream>>>(in);
    else if (h->order == 2)
      k_inject<2><<<grid, 256, 0, h->stream>>>(in);
    else
      k_inject<3><<<grid, 256, 0, h->stream>>>(in);
    h->launches++;
    CK(cudaGetLastError());
  }
  return FEMPIC_OK;
}

// field evaluation at given points: order and arithmetic picked at run time
template <int P>
void launch_eval_fields_p(FemPIC* h, int grid, bool strict, int64_t n, const double* x, const int32_t* tet, double* E,
                          double* B) {
  const double* B0 = h->opts.B0;
  if (strict)
    k_eval_fields<P, Strict><<<grid, 128, 0, h->stream>>>(n, x, tet, h->geom, h->dof1, h->dof2, h->e, b_gather(h), B0[0],
                                                          B0[1], B0[2], E, B);
  else
    k_eval_fields<P, Fast><<<grid, 128, 0, h->stream>>>(n, x, tet, h->geom, h->dof1, h->dof2, h->e, b_gather(h), B0[0], B0[1],
                                                        B0[2], E, B);
}

void launch_eval_fields(FemPIC* h, int grid, bool strict, int64_t n, const double* x, const int32_t* tet, double* E,
                        double* B) {
  if (h->order == 1)
    launch_eval_fields_p<1>(h, grid, strict, n, x, tet, E, B);
  else if (h->order == 2)
    launch_eval_fields_p<2>(h, grid, strict, n, x, tet, E, B);
  else
    launch_eval_fields_p<3>(h, grid, strict, n, x, tet, E, B);
}

int field_update(FemPIC* h, double dt, cudaEvent_t ev_pcg0, cudaEvent_t ev_pcg1) {
  bool trap = h->opts.scheme == FEMPIC_SCHEME_TRAPEZOID;
  // initial guess: linear extrapolation 2 e^n - e^{n-1}
  {
    int g = grid_for(h->n1, 256, h->num_sms * 8);
    k_lincomb<<<g, 256, 0, h->stream>>>(h->n1, h->e, h->e_prev, 2.0, -1.0, h->e_new);
    h->launches++;
    CK(cudaGetLastError());
  }
  CsrView R1 = h->M.view(h->R1val);
  CsrView Qv = h->Q.view();
  int grid = grid_for((int64_t)h->n1 * lpr_w1(h), 256, h->num_sms * 16);
  if (h->order == 1)
    k_rhs<4><<<grid, 256, 0, h->stream>>>(R1, trap ? nullptr : h->R2val, Qv, h->e, h->e_prev, h->b, trap ? dt : 0.0,
                                          h->dg, h->dg_prev, trap ? 0.0 : 1.0, h->pec1, h->rhs);
  else
    k_rhs<8><<<grid, 256, 0, h->stream>>>(R1, trap ? nullptr : h->R2val, Qv, h->e, h->e_prev, h->b, trap ? dt : 0.0,
                                          h->dg, h->dg_prev, trap ? 0.0 : 1.0, h->pec1, h->rhs);
  h->launches++;
  CK(cudaGetLastError());
  CK(cudaEventRecord(ev_pcg0, h->stream));
  int rc = run_pcg(h, h->M.view(h->Aval), h->dinvA, h->rhs, h->e_new, h->pcg_blocks_w1, true);
  if (rc) return rc;
  CK(cudaEventRecord(ev_pcg1, h->stream));
  k_accumulate_iters<<<1, 1, 0, h->stream>>>(h->d_cg_iters, h->d_cg_iters_acc);
  h->launches++;
  int gridc = grid_for((int64_t)h->n2 * 4, 256, h->num_sms * 16);
  k_bupdate<4><<<gridc, 256, 0, h->stream>>>(h->C.view(), h->e_new, h->e, 0.5 * dt, h->b);
  h->launches++;
  CK(cudaGetLastError());
  if (h->bimp) {
    k_lincomb<<<grid_for(h->n2, 256, h->num_sms * 8), 256, 0, h->stream>>>(h->n2, h->b, h->bimp, 1.0, 1.0, h->btot);
    h->launches++;
    CK(cudaGetLastError());
  }
  return FEMPIC_OK;
}

int diagnostics(FemPIC* h) {
  // continuity: (rho - rho_prev) - D^T dg ; Gauss: D^T M e + rho + rho_ion load
  CK(cudaMemsetAsync(h->d_norms, 0, sizeof(double) * 6, h->stream));
  int rc = spmv(h, h->DT.view(), h->dg, h->d_tmp0);
  if (rc) return rc;
  int grid = grid_for(h->n0, 256, h->num_sms * 8);
  k_norms2<<<grid, 256, 0, h->stream>>>(h->n0, h->int0, h->rho, h->rho_prev, h->d_tmp0, -1.0, 0.0, nullptr,
                                        h->d_norms);
  h->launches++;
  rc = spmv(h, h->M.view(), h->e, h->d_tmp1);
  if (rc) return rc;
  rc = spmv(h, h->DT.view(), h->d_tmp1, h->d_tmp0);
  if (rc) return rc;
  k_norms2<<<grid, 256, 0, h->stream>>>(h->n0, h->int0, h->rho, nullptr, h->d_tmp0, 1.0, h->opts.rho_ion, h->load0,
                                        h->d_norms + 2);
  h->launches++;
  // Gauss's magnetic law of the flux the particles see (self plus impressed)
  const int gt = grid_for(h->n_tets, 256, h->num_sms * 8);
  if (h->order == 1)
    k_divb<1><<<gt, 256, 0, h->stream>>>(h->n_tets, h->geom, h->dof2, b_gather(h), h->divref, h->n3, h->d_norms + 4);
  else if (h->order == 2)
    k_divb<2><<<gt, 256, 0, h->stream>>>(h->n_tets, h->geom, h->dof2, b_gather(h), h->divref, h->n3, h->d_norms + 4);
  else
    k_divb<3><<<gt, 256, 0, h->stream>>>(h->n_tets, h->geom, h->dof2, b_gather(h), h->divref, h->n3, h->d_norms + 4);
  h->launches++;
  CK(cudaGetLastError());
  return FEMPIC_OK;
}

cudaEvent_t event_at(FemPIC* h, size_t i) {
  while (h->ev.size() <= i) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->ev.push_back(e);
  }
  return h->ev[i];
}

// NVTX range for profilers (a no-op without an attached tool)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

int do_steps(FemPIC* h, double dt, int32_t n) {
  if (!(dt > 0.0) || !std::isfinite(dt) || n < 0) {
    h->err = "dt must be positive and finite, n_steps >= 0";
    return FEMPIC_ERR_ARG;
  }
  CK(cudaSetDevice(h->device));
  h->launches = 0;
  if (dt != h->dt_cur) {
    int rc = form_system(h, dt);
    if (rc) return rc;
  }
  if (h->n_absorb_faces > 0) {
    for (int k = 0; k < h->n_species; ++k)
      if (!h->inj_has[k]) {
        h->err = "absorbing faces need an injector for every species (femPIC_set_injection)";
        return FEMPIC_ERR_STATE;
      }
  }
  CK(cudaMemsetAsync(h->d_cross, 0, sizeof(unsigned long long), h->stream));
  CK(cudaMemsetAsync(h->d_absorbed, 0, sizeof(unsigned long long), h->stream));
  CK(cudaMemsetAsync(h->d_cg_iters_acc, 0, sizeof(int32_t), h->stream));
  constexpr int kEv = 6;
  for (int32_t s = 0; s < n; ++s) {
    cudaEvent_t e[kEv];
    for (int k = 0; k < kEv; ++k) {
      e[k] = event_at(h, (size_t)kEv * s + k);
      if (!e[k]) {
        h->err = "cudaEventCreate failed";
        return FEMPIC_ERR_CUDA;
      }
    }
    CK(cudaEventRecord(e[0], h->stream));
    NvtxRange step_range("femPIC_step");
    if (h->opts.sort_period > 0 && h->since_sort >= h->opts.sort_period && h->opts.push != FEMPIC_PUSH_AB4) {
      int rc = sort_particles(h);
      if (rc) return rc;
      h->since_sort = 0;
    }
    std::swap(h->dg, h->dg_prev);
    std::swap(h->rho, h->rho_prev);
    CK(cudaMemsetAsync(h->dg, 0, sizeof(double) * h->n1, h->stream));
    CK(cudaMemsetAsync(h->rho, 0, sizeof(double) * h->n0, h->stream));
    CK(cudaEventRecord(e[1], h->stream));
    nvtxRangePushA("particles");
    int rc = launch_particles(h, dt);
    nvtxRangePop();
    if (rc) return rc;
    CK(cudaEventRecord(e[2], h->stream));
    nvtxRangePushA("field_update");
    rc = field_update(h, dt, e[3], e[4]);
    nvtxRangePop();
    if (rc) return rc;
    CK(cudaEventRecord(e[5], h->stream));
    // rotate e: e_prev <- e, e <- e_new
    double* old_prev = h->e_prev;
    h->e_prev = h->e;
    h->e = h->e_new;
    h->e_new = old_prev;
    if (h->opts.diagnostics) {
      rc = diagnostics(h);
      if (rc) return rc;
    }
    h->steps++;
    h->since_sort++;
  }
  h->pending_steps = n;
  return FEMPIC_OK;
}

int collect_timing(FemPIC* h) {
  h->t_particle_ms = h->t_field_ms = 0.0;
  h->t_sort_ms = h->t_push_ms = h->t_rhs_ms = h->t_pcg_ms = h->t_bupd_ms = 0.0;
  for (int s = 0; s < h->pending_steps; ++s) {
    float t[5];
    for (int k = 0; k < 5; ++k) CK(cudaEventElapsedTime(&t[k], h->ev[6 * s + k], h->ev[6 * s + k + 1]));
    h->t_sort_ms += t[0];
    h->t_push_ms += t[1];
    h->t_rhs_ms += t[2];
    h->t_pcg_ms += t[3];
    h->t_bupd_ms += t[4];
    h->t_particle_ms += t[0] + t[1];
    h->t_field_ms += t[2] + t[3] + t[4];
  }
  int32_t it = 0;
  CK(cudaMemcpy(&it, h->d_cg_iters_acc, sizeof(int32_t), cudaMemcpyDeviceToHost));
  h->cg_iters_sum = it;
  h->pending_steps = 0;
  return FEMPIC_OK;
}

size_t what_bytes(const FemPIC* h, int32_t what) {
  switch (what) {
    case FEMPIC_E:
    case FEMPIC_DG:
    case FEMPIC_J:
    case FEMPIC_E_PREV:
    case FEMPIC_DG_PREV:
      return sizeof(double) * (size_t)h->n1;
    case FEMPIC_B:
    case FEMPIC_B_IMPRESSED:
      return sizeof(double) * (size_t)h->n2;
    case FEMPIC_RHO:
    case FEMPIC_PHI:
      return sizeof(double) * (size_t)h->n0;
    case FEMPIC_X:
    case FEMPIC_V:
      return sizeof(double) * 3 * (size_t)h->np;
    case FEMPIC_TET:
    case FEMPIC_NCROSS:
    case FEMPIC_SPECIES:
      return sizeof(int32_t) * (size_t)h->np;
    case FEMPIC_HASH:
      return sizeof(uint64_t) * (size_t)h->np;
    case FEMPIC_DIAG:
      return sizeof(femPIC_diag);
    default:
      return 0;
  }
}

double* field_ptr(FemPIC* h, int32_t what) {
  switch (what) {
    case FEMPIC_E:
      return h->e;
    case FEMPIC_B:
      return h->b;
    case FEMPIC_DG:
      return h->dg;
    case FEMPIC_RHO:
      return h->rho;
    case FEMPIC_E_PREV:
      return h->e_prev;
    case FEMPIC_DG_PREV:
      return h->dg_prev;
    case FEMPIC_PHI:
      return h->phi;
    default:
      return nullptr;
  }
}

// allocate the impressed-field coefficients (zero) and the sampled sum
int ensure_impressed(FemPIC* h) {
  if (h->bimp) return FEMPIC_OK;
  int rc = dalloc(h, &h->bimp, h->n2);
  if (!rc) rc = dalloc(h, &h->btot, h->n2);
  if (rc) return rc;
  CK(cudaMemsetAsync(h->bimp, 0, sizeof(double) * h->n2, h->stream));
  return FEMPIC_OK;
}

// btot = b + bimp (stream-ordered)
int refresh_btot(FemPIC* h) {
  if (!h->bimp) return FEMPIC_OK;
  k_lincomb<<<grid_for(h->n2, 256, h->num_sms * 8), 256, 0, h->stream>>>(h->n2, h->b, h->bimp, 1.0, 1.0, h->btot);
  h->launches++;
  CK(cudaGetLastError());
  return FEMPIC_OK;
}

// move a quantity between the handle and a buffer (host or device)
int transfer(FemPIC* h, int32_t what, void* buf, size_t bytes, bool to_handle, bool buf_on_device) {
  if (!h) return FEMPIC_ERR_ARG;
  size_t need = what_bytes(h, what);
  if (need == 0 || (to_handle && (what == FEMPIC_DIAG || what == FEMPIC_PHI || what == FEMPIC_NCROSS ||
                                  what == FEMPIC_SPECIES || what == FEMPIC_J ||
                                  what == FEMPIC_HASH))) {
    h->err = "unknown or read-only quantity";
    return FEMPIC_ERR_ARG;
  }
  if (bytes != need) {
    h->err = "buffer is " + std::to_string(bytes) + " bytes, quantity needs " + std::to_string(need);
    return FEMPIC_ERR_SIZE;
  }
  if (!buf && need) {
    h->err = "NULL buffer";
    return FEMPIC_ERR_ARG;
  }
  CK(cudaSetDevice(h->device));
#if FEMPIC_CHECKS
  if (to_handle && what == FEMPIC_TET && buf_on_device && h->np > 0) {
    // the device path's tet ids are checked before anything is copied
    k_check_ids<<<grid_for(h->np, 256, 1 << 20), 256, 0, h->stream>>>(h->np, static_cast<const int32_t*>(buf),
                                                                     h->n_tets, h->d_status);
    CK(cudaGetLastError());
    int32_t st = 0;
    CK(cudaMemcpyAsync(&st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (st & kStatusBounds) {
      st &= ~kStatusBounds;
      CK(cudaMemcpyAsync(h->d_status, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      h->err = "tet id out of range in the device buffer (checked build)";
      return FEMPIC_ERR_BOUNDS;
    }
  }
#endif
  if (what == FEMPIC_SPECIES) {  // fixed by the particle-id ranges
    std::vector<int32_t> sp((size_t)h->np);
    for (int k = 0; k < h->n_species; ++k)
      for (int64_t i = h->sp_off[k]; i < h->sp_off[k + 1]; ++i) sp[(size_t)i] = k;
    if (buf_on_device)
      CK(cudaMemcpy(buf, sp.data(), need, cudaMemcpyHostToDevice));
    else if (need)
      memcpy(buf, sp.data(), need);
    return FEMPIC_OK;
  }
  cudaMemcpyKind up = buf_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyKind down = buf_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (what == FEMPIC_DIAG) {
    femPIC_diag d;
    memset(&d, 0, sizeof(d));
    if (h->steps > 0 && h->opts.diagnostics) {  // residuals of the state as it is now (after any femPIC_set)
      const int rc = diagnostics(h);
      if (rc) return rc;
    }
    double norms[6];
    CK(cudaMemcpyAsync(norms, h->d_norms, sizeof(norms), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&d.cg_iterations, h->d_cg_iters, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&d.cg_residual, h->d_cg_res, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    unsigned long long cr = 0, nab = 0;
    CK(cudaMemcpyAsync(&cr, h->d_cross, sizeof(cr), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&nab, h->d_absorbed, sizeof(nab), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&d.status, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    d.steps = h->steps;
    d.continuity_abs = std::sqrt(norms[0]);
    d.continuity_ref = std::sqrt(norms[1]);
    d.gauss_abs = std::sqrt(norms[2]);
    d.gauss_ref = std::sqrt(norms[3]);
    d.divb_abs = std::sqrt(norms[4]);
    d.divb_ref = std::sqrt(norms[5]);
    d.crossings = (double)cr;
    d.absorbed = (double)nab;
    if (buf_on_device)
      CK(cudaMemcpy(buf, &d, sizeof(d), cudaMemcpyHostToDevice));
    else
      memcpy(buf, &d, sizeof(d));
    return FEMPIC_OK;
  }
  if (what == FEMPIC_J) {  // Delta g / dt, scaled on the device into the scratch vector
    if (h->dt_cur <= 0.0) {
      h->err = "no current before the first step";
      return FEMPIC_ERR_STATE;
    }
    k_lincomb<<<grid_for(h->n1, 256, h->num_sms * 8), 256, 0, h->stream>>>(h->n1, h->dg, h->dg, 1.0 / h->dt_cur, 0.0,
                                                                           h->d_tmp1);
    h->launches++;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(buf, h->d_tmp1, need, down, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return FEMPIC_OK;
  }
  if (what == FEMPIC_B_IMPRESSED) {
    if (!to_handle && !h->bimp) {  // none set: zeros
      if (buf_on_device)
        CK(cudaMemset(buf, 0, need));
      else
        memset(buf, 0, need);
      return FEMPIC_OK;
    }
    if (to_handle) {
      int rc = ensure_impressed(h);
      if (rc) return rc;
      CK(cudaMemcpyAsync(h->bimp, buf, need, up, h->stream));
      if ((rc = refresh_btot(h))) return rc;
    } else {
      CK(cudaMemcpyAsync(buf, h->bimp, need, down, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    return FEMPIC_OK;
  }
  if (double* f = field_ptr(h, what)) {
    if (to_handle)
      CK(cudaMemcpyAsync(f, buf, need, up, h->stream));
    else
      CK(cudaMemcpyAsync(buf, f, need, down, h->stream));
    if (to_handle && what == FEMPIC_B) {
      int rc = refresh_btot(h);
      if (rc) return rc;
    }
    CK(cudaStreamSynchronize(h->stream));
    return FEMPIC_OK;
  }
  if (h->np == 0) return FEMPIC_OK;
  int grid = grid_for(h->np, 256, 1 << 30);
  double* stage = h->stage;
  // Host X, V and TET are validated on the device after the staging copy: the
  // first non-finite value or out-of-range tet id vetoes the gather into the
  // particle state, so a refused transfer leaves the state as it was.
  const bool check = to_handle && !buf_on_device && (what == FEMPIC_X || what == FEMPIC_V || what == FEMPIC_TET);
  const unsigned long long* veto = check ? h->d_first : nullptr;
  const int vgrid = grid_for(3 * h->np, 256, h->num_sms * 8);
  if (what == FEMPIC_X || what == FEMPIC_V) {
    double** dst = what == FEMPIC_X ? h->px : h->pv;
    if (to_handle) {
      CK(cudaMemcpyAsync(stage, buf, need, up, h->stream));
      if (check) k_first_nonfinite<<<vgrid, 256, 0, h->stream>>>(3 * h->np, stage, h->d_first);
      k_gather_by_id<<<grid, 256, 0, h->stream>>>(h->np, h->pid, stage, dst[0], dst[1], dst[2], veto);
    } else {
      k_scatter_by_id<<<grid, 256, 0, h->stream>>>(h->np, h->pid, dst[0], dst[1], dst[2], stage);
      CK(cudaMemcpyAsync(buf, stage, need, down, h->stream));
    }
  } else if (what == FEMPIC_TET || what == FEMPIC_NCROSS) {
    int32_t* src = what == FEMPIC_TET ? h->ptet : h->pncross;
    int32_t* st = reinterpret_cast<int32_t*>(stage);
    if (to_handle) {
      CK(cudaMemcpyAsync(st, buf, need, up, h->stream));
      if (check) k_first_bad_tet<<<vgrid, 256, 0, h->stream>>>(h->np, st, h->n_tets, h->d_first);
      k_gather1_by_id<int32_t><<<grid, 256, 0, h->stream>>>(h->np, h->pid, st, src, veto);
    } else {
      k_scatter1_by_id<int32_t><<<grid, 256, 0, h->stream>>>(h->np, h->pid, src, st);
      CK(cudaMemcpyAsync(buf, st, need, down, h->stream));
    }
  } else if (what == FEMPIC_HASH) {
    auto* st = reinterpret_cast<unsigned long long*>(stage);
    k_scatter1_by_id<unsigned long long><<<grid, 256, 0, h->stream>>>(h->np, h->pid, h->phash, st);
    CK(cudaMemcpyAsync(buf, st, need, down, h->stream));
  }
  CK(cudaGetLastError());
  unsigned long long first = ~0ull;
  if (check) CK(cudaMemcpyAsync(&first, h->d_first, sizeof(first), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (first != ~0ull) {
    CK(cudaMemsetAsync(h->d_first, 0xFF, sizeof(unsigned long long), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->err = what == FEMPIC_TET ? "tet id out of range at particle " + std::to_string(first)
                                : "non-finite value at particle " + std::to_string(first / 3);
    return FEMPIC_ERR_ARG;
  }
  if (to_handle && (what == FEMPIC_X || what == FEMPIC_V || what == FEMPIC_TET)) h->ab_count = 0;
  if (to_handle && (what == FEMPIC_X || what == FEMPIC_TET)) {
    int rc = measure_rho(h, h->rho);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
  }
  return FEMPIC_OK;
}

int create_impl(const femPIC_mesh* mesh, int32_t order, const femPIC_species* sp, const femPIC_opts* opts,
                FemPIC* h, const int32_t* bface_tag) {
  if (opts)
    h->opts = *opts;
  else
    femPIC_default_opts(&h->opts);
  const femPIC_opts& o = h->opts;
  if (!mesh || !sp) {
    h->err = "NULL mesh or species";
    return FEMPIC_ERR_ARG;
  }
  if (order < 1 || order > 3) {
    h->err = "order must be 1, 2 or 3";
    return FEMPIC_ERR_ARG;
  }
  if (order == 3 && opts && opts->push == FEMPIC_PUSH_AB4) {
    h->err = "the Adams-Bashforth push is built for orders 1 and 2";
    return FEMPIC_ERR_ARG;
  }
  if (o.precision < 0 || o.precision > 2 || o.scheme < 0 || o.scheme > 1 || !(o.cg_rtol > 0) ||
      o.cg_max_it < 1 || o.max_cross < 1 || o.sort_period < 0 || o.push < 0 || o.push > 1) {
    h->err = "invalid option";
    return FEMPIC_ERR_ARG;
  }
  if (sp->n < 0 || (sp->n > 0 && (!sp->x_host || !sp->v_host || !sp->tet_host)) || !(sp->m > 0) ||
      sp->n > INT32_MAX) {
    h->err = "invalid species";
    return FEMPIC_ERR_ARG;
  }
  HostModel hm;
  std::string err;
  int code = build_model(mesh->xyz_host, mesh->n_nodes, mesh->tets_host, mesh->n_tets, order, &hm, &err, bface_tag);
  if (code) {
    h->err = err;
    return code == 2 ? FEMPIC_ERR_MESH : FEMPIC_ERR_ARG;
  }
  if (hm.n_imp_faces > 0 && o.scheme != FEMPIC_SCHEME_TRAPEZOID) {
    h->err = "impedance (absorbing) faces need the trapezoid scheme";
    return FEMPIC_ERR_ARG;
  }
  h->n_imp_faces = hm.n_imp_faces;
  if (hm.n_absorb_faces > 0 && o.push == FEMPIC_PUSH_AB4) {
    h->err = "absorbing faces are built for the Boris push only";
    return FEMPIC_ERR_ARG;
  }
  h->n_absorb_faces = hm.n_absorb_faces;
  h->n_inj_faces = (int32_t)hm.inj_tet.size();
  // particle ownership check on the host: lambda >= -1e-9 in the given tet
  for (int64_t i = 0; i < sp->n; ++i) {
    int32_t t = sp->tet_host[i];
    if (t < 0 || t >= hm.n_tets) {
      h->err = "particle " + std::to_string(i) + " has a tet id out of range";
      return FEMPIC_ERR_ARG;
    }
    const double* g = &hm.geom[(size_t)t * 16];
    const double* x = sp->x_host + 3 * i;
    const double* v = sp->v_host + 3 * i;
    if (!std::isfinite(v[0]) || !std::isfinite(v[1]) || !std::isfinite(v[2])) {
      h->err = "particle " + std::to_string(i) + " has a non-finite velocity";
      return FEMPIC_ERR_ARG;
    }
    for (int k = 0; k < 4; ++k) {
      double l = ((g[3 * k] * x[0] + g[3 * k + 1] * x[1]) + g[3 * k + 2] * x[2]) + g[12 + k];
      if (!(l >= -1e-9)) {
        h->err = "particle " + std::to_string(i) + " is not inside its tet";
        return FEMPIC_ERR_ARG;
      }
    }
  }
  h->order = order;
  h->hxyz.assign(mesh->xyz_host, mesh->xyz_host + 3 * (size_t)mesh->n_nodes);
  h->htets = hm.tets;
  h->nl0 = hm.nl0;
  h->nl1 = hm.nl1;
  h->nl2 = hm.nl2;
  h->n_nodes = hm.n_nodes;
  h->n_tets = hm.n_tets;
  h->n_edges = hm.n_edges;
  h->n_faces = hm.n_faces;
  h->n0 = hm.n0;
  h->n1 = hm.n1;
  h->n2 = hm.n2;
  h->n_bfaces = hm.n_bfaces;
  h->q = sp->q;
  h->m = sp->m;
  h->weight = sp->weight;
  h->np = sp->n;

  h->device = o.device;
  CK(cudaSetDevice(h->device));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, h->device));
  h->num_sms = prop.multiProcessorCount;
  if (o.stream) {
    h->stream = (cudaStream_t)o.stream;
  } else {
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  int rc = 0;
#define UP(dst, src)             \
  rc = upload(h, &(dst), (src)); \
  if (rc) return rc;
  UP(h->geom, hm.geom);
  if (o.precision == FEMPIC_MIXED) {
    std::vector<float> g32((size_t)hm.n_tets * 12);
    for (size_t t = 0; t < (size_t)hm.n_tets; ++t)
      for (int k = 0; k < 12; ++k) g32[t * 12 + k] = (float)hm.geom[t * 16 + k];
    UP(h->geom32, g32);
    if ((rc = dalloc(h, &h->e32, std::max(1, hm.n1))) || (rc = dalloc(h, &h->b32, std::max(1, hm.n2)))) return rc;
  }
  UP(h->nbr, hm.nbr);
  UP(h->dof0, hm.dof0);
  UP(h->dof1, hm.dof1);
  UP(h->dof2, hm.dof2);
  UP(h->pec1, hm.pec1);
  {
    std::vector<uint8_t> i0(hm.n0);
    for (int32_t i = 0; i < hm.n0; ++i) i0[i] = !hm.bnd0[i];
    UP(h->int0, i0);
  }
  UP(h->load0, hm.load0);
#undef UP
  {  // typical curl-curl to mass ratio per unit dt^2 (decides the FP32 direction products)
    std::vector<double> ratio;
    ratio.reserve(hm.M.n_rows);
    for (int32_t i = 0; i < hm.M.n_rows; ++i) {
      double m = 0.0, k = 0.0;
      for (int32_t j = hm.M.rowptr[i]; j < hm.M.rowptr[i + 1]; ++j)
        if (hm.M.col[j] == i) {
          m = hm.M.val[j];
          k = hm.K.val[j];
        }
      if (m > 0.0) ratio.push_back(k / m);
    }
    if (!ratio.empty()) {
      std::nth_element(ratio.begin(), ratio.begin() + ratio.size() / 2, ratio.end());
      h->kdiag_med = ratio[ratio.size() / 2];
    }
  }
  if ((rc = upload_csr(h, &h->M, hm.M)) || (rc = upload_csr(h, &h->K, hm.K)) || (rc = upload_csr(h, &h->Q, hm.Q)) ||
      (rc = upload_csr(h, &h->C, hm.C)) || (rc = upload_csr(h, &h->M2, hm.M2)) || (rc = upload_csr(h, &h->D, hm.D)) ||
      (rc = upload_csr(h, &h->DT, hm.DT)) || (rc = upload_csr(h, &h->L, hm.L)) ||
      (rc = upload_csr(h, &h->Pi, hm.Pi)) || (rc = upload_csr(h, &h->PiT, hm.PiT)) ||
      (rc = upload(h, &h->dvM, hm.dvM)) || (rc = upload(h, &h->dvK, hm.dvK)) ||
      (rc = dalloc(h, &h->dinvV, hm.PiT.n_rows)) || (rc = dalloc(h, &h->aux_u, hm.PiT.n_rows)) ||
      (rc = dalloc(h, &h->aux_t, hm.n0)) || (rc = dalloc(h, &h->dinvL32, hm.n0)) ||
      (rc = dalloc(h, &h->D32, hm.D.col.size())) || (rc = dalloc(h, &h->DT32, hm.DT.col.size())) ||
      (rc = dalloc(h, &h->Pi32, hm.Pi.col.size())) || (rc = dalloc(h, &h->PiT32, hm.PiT.col.size())))
    return rc;
  h->cheb_k = std::max(1, std::min(FEMPIC_AUX_CHEB, kMaxCheb));
  if (h->cheb_k > 1) {
    const size_t nv = hm.PiT.n_rows;
    if ((rc = upload_csr(h, &h->V, hm.VM)) || (rc = upload(h, &h->VKv, hm.VK)) ||
        (rc = dalloc(h, &h->V32, hm.VM.col.size())) || (rc = dalloc(h, &h->L32, hm.L.col.size())) ||
        (rc = dalloc(h, &h->aux_tf, hm.n0)) || (rc = dalloc(h, &h->aux_td, hm.n0)) ||
        (rc = dalloc(h, &h->aux_t2, hm.n0)) || (rc = dalloc(h, &h->aux_uf, nv)) || (rc = dalloc(h, &h->aux_ud, nv)) ||
        (rc = dalloc(h, &h->aux_u2, nv)))
      return rc;
    if (h->L.nnz > 0) k_to_f32<<<grid_for(h->L.nnz, 256, 4096), 256, 0, h->stream>>>(h->L.nnz, h->L.v, h->L32);
    CK(cudaGetLastError());
    h->hV_rp = hm.VM.rowptr;
    h->hV_ci = hm.VM.col;
    h->hV_m = hm.VM.val;
    h->hV_k = hm.VK;
    h->lmaxL = gershgorin_scaled(hm.L.rowptr, hm.L.col, hm.L.val.data(), nullptr, 0.0);
    cheb_coeffs(h->lmaxL, h->cheb_k, h->chebL);
  } else {
    cheb_coeffs(0.0, 1, h->chebL);
  }
  cheb_coeffs(0.0, 1, h->chebV);
  {
    const std::pair<const double*, float*> cv[] = {{h->D.v, h->D32}, {h->DT.v, h->DT32}, {h->Pi.v, h->Pi32},
                                                   {h->PiT.v, h->PiT32}};
    const int64_t nn[] = {h->D.nnz, h->DT.nnz, h->Pi.nnz, h->PiT.nnz};
    for (int k = 0; k < 4; ++k)
      if (nn[k] > 0) k_to_f32<<<grid_for(nn[k], 256, 4096), 256, 0, h->stream>>>(nn[k], cv[k].first, cv[k].second);
    CK(cudaGetLastError());
  }
  if (order == 2) {
    // DOFs 2k, 2k+1 belong to one edge or face and share their couplings
    const int32_t nb = hm.n1 / 2;
    std::vector<int32_t> brp(nb + 1, 0), bci;
    std::vector<double> bM, bK, bI;
    const bool imp = !hm.Ival.empty();
    bool ok = (hm.n1 % 2) == 0;
    for (int32_t k = 0; k < nb && ok; ++k) {
      int32_t r0 = 2 * k, r1 = 2 * k + 1;
      int32_t b0 = hm.M.rowptr[r0], e0 = hm.M.rowptr[r0 + 1], b1 = hm.M.rowptr[r1];
      if (e0 - b0 != hm.M.rowptr[r1 + 1] - b1 || (e0 - b0) % 2) {
        ok = false;
        break;
      }
      for (int32_t j = b0; j < e0; j += 2) {
        int32_t c = hm.M.col[j];
        if ((c & 1) || hm.M.col[j + 1] != c + 1 || hm.M.col[b1 + (j - b0)] != c ||
            hm.M.col[b1 + (j - b0) + 1] != c + 1) {
          ok = false;
          break;
        }
        bci.push_back(c / 2);
        const int32_t q0 = j, q1 = b1 + (j - b0);
        bM.insert(bM.end(), {hm.M.val[q0], hm.M.val[q0 + 1], hm.M.val[q1], hm.M.val[q1 + 1]});
        bK.insert(bK.end(), {hm.K.val[q0], hm.K.val[q0 + 1], hm.K.val[q1], hm.K.val[q1 + 1]});
        if (imp) bI.insert(bI.end(), {hm.Ival[q0], hm.Ival[q0 + 1], hm.Ival[q1], hm.Ival[q1 + 1]});
      }
      brp[k + 1] = (int32_t)bci.size();
    }
    if (ok) {
      h->nb = nb;
      h->nnzb = (int64_t)bci.size();
      if ((rc = upload(h, &h->brp, brp)) || (rc = upload(h, &h->bci, bci)) || (rc = upload(h, &h->bM, bM)) ||
          (rc = upload(h, &h->bK, bK)) || (rc = dalloc(h, &h->bA, bM.size())) || (rc = dalloc(h, &h->binv, 4 * (size_t)nb)) ||
          (FEMPIC_PCG_FP32A && (rc = dalloc(h, &h->bA32, bM.size()))))
        return rc;
      h->cheb_k_sm = h->cheb_k > 1 ? std::max(h->cheb_k, std::min(FEMPIC_AUX_CHEB_SMOOTH, kMaxCheb)) : 1;
      h->smooth_k = std::max(1, std::min(FEMPIC_SMOOTH_DEG, h->cheb_k_sm));
      cheb_coeffs(h->lmaxL, h->cheb_k_sm, h->chebL_sm);
      if (FEMPIC_PCG_FP32A && h->smooth_k > 1 &&
          ((rc = dalloc(h, &h->sy, 4 * (size_t)nb)) || (rc = dalloc(h, &h->sd, 2 * (size_t)nb)) ||
           (rc = dalloc(h, &h->chebS, 3 * kMaxCheb)) || (rc = dalloc(h, &h->bA16, bM.size())) ||
           (rc = dalloc(h, &h->binv32, 4 * (size_t)nb))))
        return rc;
      if (imp && (rc = upload(h, &h->bI, bI))) return rc;
    }
  }
  const size_t nnz = hm.M.col.size();
  if (!hm.Ival.empty() && (rc = upload(h, &h->Iv, hm.Ival))) return rc;
  if (order == 3) {
    // W1 DOF groups, contiguous: 3 per edge, 6 per face, 3 per tet interior
    std::vector<int32_t> gs, rp(1, 0), ci;
    std::vector<uint8_t> gz;
    auto add = [&](int32_t start, int size) {
      gs.push_back(start);
      gz.push_back((uint8_t)size);
      for (int r = 0; r < size; ++r) {
        for (int c = 0; c < size; ++c) ci.push_back(start + c);
        rp.push_back((int32_t)ci.size());
      }
    };
    for (int32_t e = 0; e < hm.n_edges; ++e) add(3 * e, 3);
    for (int32_t f = 0; f < hm.n_faces; ++f) add(3 * hm.n_edges + 6 * f, 6);
    for (int32_t t = 0; t < hm.n_tets; ++t) add(3 * hm.n_edges + 6 * hm.n_faces + 3 * t, 3);
    if ((int32_t)rp.size() != hm.n1 + 1) {
      h->err = "order-3 DOF groups do not cover the W1 DOFs";
      return FEMPIC_ERR_ARG;
    }
    HostCSR bg;
    bg.n_rows = bg.n_cols = hm.n1;
    bg.rowptr = rp;
    bg.col = ci;
    bg.val.assign(ci.size(), 0.0);
    h->n_groups = (int32_t)gs.size();
    if ((rc = upload(h, &h->gstart, gs)) || (rc = upload(h, &h->gsize, gz)) || (rc = upload_csr(h, &h->Bg, bg)))
      return rc;
  }
  if (!hm.LA.col.empty()) {
    const size_t nl = hm.LA.col.size();
    if ((rc = upload_csr(h, &h->DA, hm.DA)) || (rc = upload_csr(h, &h->DAT, hm.DAT)) ||
        (rc = upload_csr(h, &h->LA, hm.LA)) || (rc = upload(h, &h->LAI, hm.LAI)) || (rc = dalloc(h, &h->LAdt, nl)) ||
        (rc = dalloc(h, &h->dinvLA, h->n0)) || (rc = dalloc(h, &h->DA32, hm.DA.col.size())) ||
        (rc = dalloc(h, &h->DAT32, hm.DAT.col.size())) || (rc = dalloc(h, &h->LA32, nl)) ||
        (rc = dalloc(h, &h->dinvLA32, h->n0)))
      return rc;
    if (h->DA.nnz > 0) k_to_f32<<<grid_for(h->DA.nnz, 256, 4096), 256, 0, h->stream>>>(h->DA.nnz, h->DA.v, h->DA32);
    if (h->DAT.nnz > 0)
      k_to_f32<<<grid_for(h->DAT.nnz, 256, 4096), 256, 0, h->stream>>>(h->DAT.nnz, h->DAT.v, h->DAT32);
    CK(cudaGetLastError());
    h->hLA_rp = hm.LA.rowptr;
    h->hLA_ci = hm.LA.col;
    h->hLA_m = hm.LA.val;
    h->hLA_i = hm.LAI;
  }
  if ((rc = dalloc(h, &h->Aval, nnz)) || (rc = dalloc(h, &h->R1val, nnz)) ||
      (rc = dalloc(h, &h->R2val, o.scheme == FEMPIC_SCHEME_WAVE ? nnz : 1)) || (rc = dalloc(h, &h->dinvA, h->n1)) ||
      (rc = dalloc(h, &h->dinvL, h->n0)))
    return rc;
  double** vec1[] = {&h->e, &h->e_prev, &h->e_new, &h->dg, &h->dg_prev, &h->d_tmp1};
  for (auto p : vec1)
    if ((rc = dalloc(h, p, h->n1))) return rc;
  double** vec0[] = {&h->rho, &h->rho_prev, &h->phi, &h->d_tmp0};
  for (auto p : vec0)
    if ((rc = dalloc(h, p, h->n0))) return rc;
  if ((rc = dalloc(h, &h->b, h->n2))) return rc;
  int32_t nmax = std::max(h->n1, h->n0);
  if ((rc = dalloc(h, &h->rhs, nmax))) return rc;
  double** cgv[] = {&h->cg_r, &h->cg_z, &h->cg_p, &h->cg_q, &h->cg_r2, &h->cg_p2};
  for (auto p : cgv)
    if ((rc = dalloc(h, p, nmax))) return rc;
  if (order == 1) {
    int bl = pcg_blocks<4>(h);
    if (bl < 0) return FEMPIC_ERR_CUDA;
    h->pcg_blocks_w1 = h->pcg_blocks_w0 = bl;
  } else {
    int bl = pcg_blocks<FEMPIC_LPR_P2>(h);
    if (bl < 0) return FEMPIC_ERR_CUDA;
    h->pcg_blocks_w1 = h->pcg_blocks_w0 = bl;
  }
  {
    // CG row ranges of A per CTA, balanced by stored entries (block rows at order 2)
    std::vector<int64_t> pre;
    if (h->nb > 0) {
      pre.assign((size_t)h->nb + 1, 0);
      for (int32_t k = 0; k < h->nb; ++k) pre[k + 1] = pre[k] + (hm.M.rowptr[2 * k + 1] - hm.M.rowptr[2 * k]) / 2;
    } else {
      pre.assign(hm.M.rowptr.begin(), hm.M.rowptr.end());
    }
    std::vector<int32_t> part = balanced_ranges(pre, h->pcg_blocks_w1);
    if ((rc = upload(h, &h->apart, part))) return rc;
  }
  if ((rc = dalloc(h, &h->cg_q32, nmax)) || (rc = dalloc(h, &h->cg_r32, 4 * (size_t)nmax)) ||
      (rc = dalloc(h, &h->cg_p32, nmax)) || (rc = dalloc(h, &h->cg_red, 12)))
    return rc;
  if ((rc = dalloc(h, &h->partials, 8 * (size_t)h->pcg_blocks_w1)) || (rc = dalloc(h, &h->bar, 1)) ||
      (rc = dalloc(h, &h->d_status, 1)) || (rc = dalloc(h, &h->d_cg_iters, 1)) || (rc = dalloc(h, &h->d_cg_res, 1)) ||
      (rc = dalloc(h, &h->d_cg_iters_acc, 1)) ||
      (rc = dalloc(h, &h->d_norms, 6)) || (rc = dalloc(h, &h->d_cross, 1)) || (rc = dalloc(h, &h->d_first, 1)))
    return rc;
  CK(cudaMemset(h->d_first, 0xFF, sizeof(unsigned long long)));
  for (void* p : std::vector<void*>{h->e, h->e_prev, h->e_new, h->dg, h->dg_prev})
    CK(cudaMemset(p, 0, sizeof(double) * h->n1));
  CK(cudaMemset(h->b, 0, sizeof(double) * h->n2));
  CK(cudaMemset(h->phi, 0, sizeof(double) * h->n0));
  CK(cudaMemset(h->rho_prev, 0, sizeof(double) * h->n0));
  CK(cudaMemset(h->d_status, 0, sizeof(int32_t)));
#if FEMPIC_CHECKS
  CK(cudaDeviceSynchronize());
  k_check_tables<<<grid_for(h->n_tets, 256, 4096), 256, 0, h->stream>>>(
      h->n_tets, h->nl0, h->nl1, h->nl2, h->dof0, h->dof1, h->dof2, h->nbr, h->n0, h->n1, h->n2, h->d_status);
  CK(cudaGetLastError());
  if ((rc = latch_status(h))) return rc;
#endif
  CK(cudaMemset(h->d_cg_iters, 0, sizeof(int32_t)));
  CK(cudaMemset(h->d_cg_res, 0, sizeof(double)));
  CK(cudaMemset(h->d_norms, 0, 4 * sizeof(double)));
  CK(cudaMemset(h->d_cross, 0, sizeof(unsigned long long)));
  // particles
  const int64_t n = h->np;
  for (int k = 0; k < 3; ++k) {
    if ((rc = dalloc(h, &h->px[k], n)) || (rc = dalloc(h, &h->pv[k], n))) return rc;
  }
  double* altblock = nullptr;
  if ((rc = dalloc(h, &altblock, 6 * (size_t)std::max<int64_t>(n, 1)))) return rc;
  for (int k = 0; k < 6; ++k) h->alt[k] = altblock + (size_t)k * std::max<int64_t>(n, 1);
  if ((rc = dalloc(h, &h->stage, 3 * (size_t)std::max<int64_t>(n, 1)))) return rc;
  if ((rc = dalloc(h, &h->ptet, n)) || (rc = dalloc(h, &h->pid, n)) || (rc = dalloc(h, &h->ptet_alt, n)) ||
      (rc = dalloc(h, &h->pid_alt, n)) || (rc = dalloc(h, &h->pncross, n)) || (rc = dalloc(h, &h->phash, n)) ||
      (rc = dalloc(h, &h->sort_cnt, h->n_tets)) || (rc = dalloc(h, &h->sort_off, h->n_tets)) ||
      (rc = dalloc(h, &h->sort_sums, (h->n_tets + 1023) / 1024 + 1)) ||
      (rc = dalloc(h, &h->sort_sums2, (h->n_tets + 1023) / 1024 / 1024 + 2)))
    return rc;
  {
    std::vector<double> dref;
    int n3 = 0;
    div_table(order, &dref, &n3);
    h->n3 = n3;
    if ((rc = upload(h, &h->divref, dref))) return rc;
  }
  if ((rc = dalloc(h, &h->d_absorbed, 1))) return rc;
  CK(cudaMemset(h->d_absorbed, 0, sizeof(unsigned long long)));
  if (h->n_absorb_faces > 0 && (rc = dalloc(h, &h->pabs, n))) return rc;
  if (h->n_inj_faces > 0 && ((rc = upload(h, &h->inj_xyz, hm.inj_xyz)) || (rc = upload(h, &h->inj_tet, hm.inj_tet)) ||
                             (rc = upload(h, &h->inj_cum, hm.inj_cum))))
    return rc;
  if (o.push == FEMPIC_PUSH_AB4) {
    for (int j = 0; j < 3; ++j)
      for (int c = 0; c < 3; ++c) {
        if ((rc = dalloc(h, &h->ab_vh[j][c], n)) || (rc = dalloc(h, &h->ab_ah[j][c], n))) return rc;
        if (n > 0) {
          CK(cudaMemset(h->ab_vh[j][c], 0, n * sizeof(double)));
          CK(cudaMemset(h->ab_ah[j][c], 0, n * sizeof(double)));
        }
      }
    h->ab_count = 0;
  }
  if (n > 0) {
    std::vector<double> tmp((size_t)n);
    for (int k = 0; k < 3; ++k) {
      for (int64_t i = 0; i < n; ++i) tmp[i] = sp->x_host[3 * i + k];
      CK(cudaMemcpy(h->px[k], tmp.data(), n * sizeof(double), cudaMemcpyHostToDevice));
      for (int64_t i = 0; i < n; ++i) tmp[i] = sp->v_host[3 * i + k];
      CK(cudaMemcpy(h->pv[k], tmp.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(h->ptet, sp->tet_host, n * sizeof(int32_t), cudaMemcpyHostToDevice));
    std::vector<int32_t> ids((size_t)n);
    for (int64_t i = 0; i < n; ++i) ids[i] = (int32_t)i;
    CK(cudaMemcpy(h->pid, ids.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(cudaMemset(h->pncross, 0, n * sizeof(int32_t)));
    CK(cudaMemset(h->phash, 0, n * sizeof(unsigned long long)));
  }
  h->since_sort = h->opts.sort_period;  // sort before the first step
  rc = measure_rho(h, h->rho);
  if (rc) return rc;
  {
    int grid = grid_for(h->n0, 256, 1 << 30);
    k_inv_diag<<<grid, 256, 0, h->stream>>>(h->n0, h->L.rp, h->L.ci, h->L.v, h->dinvL);
    k_to_f32<<<grid, 256, 0, h->stream>>>(h->n0, h->dinvL, h->dinvL32);
    CK(cudaGetLastError());
  }
  // electrostatic start: L phi = rho + rho_ion <W0, 1> on interior DOFs, e = -D phi
  if (o.es_init) {
    // rhs0 = (rho + rho_ion load) masked to interior: use k_norms2-free path on the host side
    CK(cudaStreamSynchronize(h->stream));
    std::vector<double> rho_h(h->n0), rhs0(h->n0);
    CK(cudaMemcpy(rho_h.data(), h->rho, sizeof(double) * h->n0, cudaMemcpyDeviceToHost));
    for (int32_t i = 0; i < h->n0; ++i) rhs0[i] = hm.bnd0[i] ? 0.0 : rho_h[i] + o.rho_ion * hm.load0[i];
    CK(cudaMemcpy(h->d_tmp0, rhs0.data(), sizeof(double) * h->n0, cudaMemcpyHostToDevice));
    CK(cudaMemcpyAsync(h->rhs, h->d_tmp0, sizeof(double) * h->n0, cudaMemcpyDeviceToDevice, h->stream));
    rc = run_pcg(h, h->L.view(), h->dinvL, h->rhs, h->phi, h->pcg_blocks_w0, false);
    if (rc) return rc;
    rc = spmv(h, h->D.view(), h->phi, h->e, -1.0, 0.0);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->e_prev, h->e, sizeof(double) * h->n1, cudaMemcpyDeviceToDevice, h->stream));
    rc = latch_status(h);
    if (rc) {
      h->err = "electrostatic start: " + h->err;
      return rc;
    }
  }
  CK(cudaStreamSynchronize(h->stream));
  return FEMPIC_OK;
}

}  // namespace

// =============================================================================
extern "C" {

void femPIC_default_opts(femPIC_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = FEMPIC_FP64;
  o->scheme = FEMPIC_SCHEME_TRAPEZOID;
  o->gamma = 0.5;
  o->beta = 0.25;
  o->cg_rtol = 1e-12;
  o->cg_max_it = 2000;
  o->max_cross = 4096;
  o->sort_period = 1;
  o->es_init = 1;
  o->diagnostics = 0;
  o->device = 0;
  o->stream = nullptr;
}

int femPIC_create(const femPIC_mesh* mesh, int32_t order, const femPIC_species* species, const femPIC_opts* opts,
                  FemPIC** out) {
  if (!out) return FEMPIC_ERR_ARG;
  *out = nullptr;
  FemPIC* h = new (std::nothrow) FemPIC();
  if (!h) return FEMPIC_ERR_OOM;
  h->n_species = 1;
  if (species) {
    h->sp_q[0] = species->q;
    h->sp_m[0] = species->m;
    h->sp_w[0] = species->weight;
    h->sp_off[1] = species->n;
  }
  int rc = create_impl(mesh, order, species, opts, h, nullptr);
  *out = h;  // the handle carries the error message even on failure
  return rc;
}

int femPIC_create_ext(const femPIC_mesh* mesh, int32_t order, const femPIC_species* species, int32_t n_species,
                      const int32_t* bface_tag_host, const femPIC_opts* opts, FemPIC** out) {
  if (!out) return FEMPIC_ERR_ARG;
  *out = nullptr;
  FemPIC* h = new (std::nothrow) FemPIC();
  if (!h) return FEMPIC_ERR_OOM;
  *out = h;  // the handle carries the error message even on failure
  if (!species || n_species < 1 || n_species > FEMPIC_MAX_SPECIES) {
    h->err = "n_species must be 1.." + std::to_string(FEMPIC_MAX_SPECIES) + " with a species array";
    return FEMPIC_ERR_ARG;
  }
  int64_t total = 0;
  for (int32_t k = 0; k < n_species; ++k) {
    const femPIC_species& sk = species[k];
    if (sk.n < 0 || (sk.n > 0 && (!sk.x_host || !sk.v_host || !sk.tet_host)) || !(sk.m > 0) ||
        !std::isfinite(sk.q) || !(sk.weight >= 0)) {
      h->err = "invalid species " + std::to_string(k);
      return FEMPIC_ERR_ARG;
    }
    h->sp_q[k] = sk.q;
    h->sp_m[k] = sk.m;
    h->sp_w[k] = sk.weight;
    h->sp_off[k] = total;
    total += sk.n;
  }
  h->sp_off[n_species] = total;
  h->n_species = n_species;
  if (total > INT32_MAX) {
    h->err = "too many particles";
    return FEMPIC_ERR_ARG;
  }
  if (n_species == 1) return create_impl(mesh, order, species, opts, h, bface_tag_host);
  // one particle array in species order; species 0's constants stand as the scalars
  std::vector<double> xs((size_t)3 * total), vs((size_t)3 * total);
  std::vector<int32_t> ts((size_t)total);
  for (int32_t k = 0; k < n_species; ++k) {
    const femPIC_species& sk = species[k];
    const int64_t o = h->sp_off[k];
    if (sk.n > 0) {
      std::copy(sk.x_host, sk.x_host + 3 * sk.n, xs.begin() + 3 * o);
      std::copy(sk.v_host, sk.v_host + 3 * sk.n, vs.begin() + 3 * o);
      std::copy(sk.tet_host, sk.tet_host + sk.n, ts.begin() + o);
    }
  }
  femPIC_species all = species[0];
  all.n = total;
  all.x_host = xs.data();
  all.v_host = vs.data();
  all.tet_host = ts.data();
  return create_impl(mesh, order, &all, opts, h, bface_tag_host);
}

int femPIC_step_async(FemPIC* h, double dt, int32_t n) {
  if (!h) return FEMPIC_ERR_ARG;
  if (!h->stream) {
    h->err = "handle was not created";
    return FEMPIC_ERR_STATE;
  }
  return do_steps(h, dt, n);
}

int femPIC_sync(FemPIC* h) {
  if (!h) return FEMPIC_ERR_ARG;
  if (!h->stream) return FEMPIC_ERR_STATE;
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->stream));
  int rc = collect_timing(h);
  if (rc) return rc;
  return latch_status(h);
}

int femPIC_step(FemPIC* h, double dt, int32_t n) {
  int rc = femPIC_step_async(h, dt, n);
  if (rc) return rc;
  return femPIC_sync(h);
}

int femPIC_get(FemPIC* h, int32_t what, void* dst, size_t bytes) {
  if (!h || !h->stream) return FEMPIC_ERR_ARG;
  return transfer(h, what, dst, bytes, false, false);
}
int femPIC_set(FemPIC* h, int32_t what, const void* src, size_t bytes) {
  if (!h || !h->stream) return FEMPIC_ERR_ARG;
  return transfer(h, what, const_cast<void*>(src), bytes, true, false);
}
int femPIC_get_device(FemPIC* h, int32_t what, void* dst, size_t bytes) {
  if (!h || !h->stream) return FEMPIC_ERR_ARG;
  return transfer(h, what, dst, bytes, false, true);
}
int femPIC_set_device(FemPIC* h, int32_t what, const void* src, size_t bytes) {
  if (!h || !h->stream) return FEMPIC_ERR_ARG;
  return transfer(h, what, const_cast<void*>(src), bytes, true, true);
}

int femPIC_apply(FemPIC* h, int32_t op, const double* x_host, size_t nx, double* y_host, size_t ny) {
  if (!h || !h->stream || !x_host || !y_host) return FEMPIC_ERR_ARG;
  const DevCSR* A = nullptr;
  const double* vals = nullptr;
  switch (op) {
    case FEMPIC_OP_M1: A = &h->M; break;
    case FEMPIC_OP_K: A = &h->K; break;
    case FEMPIC_OP_C: A = &h->C; break;
    case FEMPIC_OP_D: A = &h->D; break;
    case FEMPIC_OP_DT: A = &h->DT; break;
    case FEMPIC_OP_M2: A = &h->M2; break;
    case FEMPIC_OP_A:
      A = &h->M;
      vals = h->Aval;
      if (h->dt_cur < 0) {
        h->err = "no system matrix before the first step";
        return FEMPIC_ERR_STATE;
      }
      break;
    case FEMPIC_OP_L: A = &h->L; break;
    case FEMPIC_OP_PI: A = &h->Pi; break;
    case FEMPIC_OP_PIT: A = &h->PiT; break;
    default:
      h->err = "unknown operator";
      return FEMPIC_ERR_ARG;
  }
  if (nx != (size_t)A->n_cols || ny != (size_t)A->n_rows) {
    h->err = "operator size mismatch";
    return FEMPIC_ERR_SIZE;
  }
  CK(cudaSetDevice(h->device));
  double *dx = nullptr, *dy = nullptr;
  CK(counted_malloc(&dx, sizeof(double) * std::max<size_t>(nx, 1)));
  if (counted_malloc(&dy, sizeof(double) * std::max<size_t>(ny, 1)) != cudaSuccess) {
    cudaFree(dx);
    h->err = "cudaMalloc failed";
    return FEMPIC_ERR_OOM;
  }
  int rc = FEMPIC_OK;
  if (cudaMemcpy(dx, x_host, sizeof(double) * nx, cudaMemcpyHostToDevice) != cudaSuccess) rc = FEMPIC_ERR_CUDA;
  if (!rc) rc = spmv(h, A->view(vals), dx, dy);
  if (!rc && cudaMemcpyAsync(y_host, dy, sizeof(double) * ny, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    rc = FEMPIC_ERR_CUDA;
  if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = FEMPIC_ERR_CUDA;
  cudaFree(dx);
  cudaFree(dy);
  if (rc == FEMPIC_ERR_CUDA) h->err = "operator application failed";
  return rc;
}

int femPIC_eval_fields(FemPIC* h, int64_t n, const double* x_host, const int32_t* tet_host, double* E_host,
                       double* B_host) {
  if (!h || !h->stream || n < 0 || (n > 0 && (!x_host || !tet_host || !E_host || !B_host))) return FEMPIC_ERR_ARG;
  if (n == 0) return FEMPIC_OK;
  for (int64_t i = 0; i < n; ++i)
    if (tet_host[i] < 0 || tet_host[i] >= h->n_tets) {
      h->err = "tet id out of range";
      return FEMPIC_ERR_ARG;
    }
  CK(cudaSetDevice(h->device));
  double *dx = nullptr, *dE = nullptr, *dB = nullptr;
  int32_t* dt = nullptr;
  CK(counted_malloc(&dx, sizeof(double) * 3 * n));
  CK(counted_malloc(&dE, sizeof(double) * 3 * n));
  CK(counted_malloc(&dB, sizeof(double) * 3 * n));
  CK(counted_malloc(&dt, sizeof(int32_t) * n));
  CK(cudaMemcpy(dx, x_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dt, tet_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  int grid = grid_for(n, 128, 1 << 30);
  bool strict = h->opts.precision == FEMPIC_FP64_STRICT;
  launch_eval_fields(h, grid, strict, n, dx, dt, dE, dB);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(E_host, dE, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(B_host, dB, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  cudaFree(dx);
  cudaFree(dE);
  cudaFree(dB);
  cudaFree(dt);
  return FEMPIC_OK;
}

}  // extern "C"

// ---- field probe without device allocation ------------------------------------------
// One fixed staging array per loaded library (and per device that uses it):
// x [3n] doubles, E [3n], B [3n], then tet [n] int32.  Its device address is
// looked up once per device, with that device current.
namespace {
constexpr size_t kProbeBytes = (size_t)FEMPIC_PROBE_MAX_POINTS * (9 * sizeof(double) + sizeof(int32_t));
static __device__ __align__(256) unsigned char g_probe_scratch[kProbeBytes];

constexpr int kProbeMaxDevices = 64;
std::mutex g_probe_mutex;
struct ProbeSlot {
  unsigned long long ctx_id = 0;  // context the address belongs to (0: none yet)
  void* ptr = nullptr;
};
ProbeSlot g_probe_slot[kProbeMaxDevices];

// Unique id of the calling thread's current CUDA context, through the driver
// entry points the runtime hands out (the library does not link libcuda);
// 0 when it cannot be read.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    looked_up = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// device address of g_probe_scratch in the current context of `device`
// (nullptr on error).  The address is cached per device together with the
// context it was read in, and read again when the context changed (after a
// cudaDeviceReset, say), or every time if the context id cannot be read.
void* probe_scratch(int device, std::string* err) {
  if (device < 0 || device >= kProbeMaxDevices) {
    *err = "device ordinal out of range for the probe scratch table";
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_probe_mutex);
  const unsigned long long ctx = current_context_id();
  ProbeSlot& slot = g_probe_slot[device];
  if (!slot.ptr || ctx == 0 || slot.ctx_id != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_probe_scratch);
    if (e != cudaSuccess || !p) {
      *err = std::string("cudaGetSymbolAddress(probe scratch): ") + cudaGetErrorString(e);
      slot = ProbeSlot();
      return nullptr;
    }
    slot.ptr = p;
    slot.ctx_id = ctx;
  }
  return slot.ptr;
}
}  // namespace

extern "C" {

int femPIC_eval_fields_noalloc(FemPIC* h, int64_t n, const double* x_host, const int32_t* tet_host, double* E_host,
                               double* B_host) {
  if (!h || !h->stream || n < 0 || (n > 0 && (!x_host || !tet_host || !E_host || !B_host))) return FEMPIC_ERR_ARG;
  if (n > FEMPIC_PROBE_MAX_POINTS) {
    h->err = "femPIC_eval_fields_noalloc: " + std::to_string(n) + " points exceed FEMPIC_PROBE_MAX_POINTS (" +
             std::to_string(FEMPIC_PROBE_MAX_POINTS) + ")";
    return FEMPIC_ERR_SIZE;
  }
  if (n == 0) return FEMPIC_OK;
  for (int64_t i = 0; i < n; ++i)
    if (tet_host[i] < 0 || tet_host[i] >= h->n_tets) {
      h->err = "tet id out of range";
      return FEMPIC_ERR_ARG;
    }
  CK(cudaSetDevice(h->device));
  void* base = probe_scratch(h->device, &h->err);
  if (!base) return FEMPIC_ERR_CUDA;
  const size_t cap = FEMPIC_PROBE_MAX_POINTS;
  double* dx = static_cast<double*>(base);
  double* dE = dx + 3 * cap;
  double* dB = dE + 3 * cap;
  int32_t* dt = reinterpret_cast<int32_t*>(dB + 3 * cap);
  CK(cudaMemcpyAsync(dx, x_host, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(dt, tet_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->stream));
  int grid = grid_for(n, 128, 1 << 30);
  bool strict = h->opts.precision == FEMPIC_FP64_STRICT;
  launch_eval_fields(h, grid, strict, n, dx, dt, dE, dB);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(E_host, dE, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(B_host, dB, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return FEMPIC_OK;
}

int femPIC_get_info(const FemPIC* h, femPIC_info* info) {
  if (!h || !info) return FEMPIC_ERR_ARG;
  memset(info, 0, sizeof(*info));
  info->n_nodes = h->n_nodes;
  info->n_tets = h->n_tets;
  info->n_edges = h->n_edges;
  info->n_faces = h->n_faces;
  info->order = h->order;
  info->n0 = h->n0;
  info->n1 = h->n1;
  info->n2 = h->n2;
  info->nl0 = h->nl0;
  info->nl1 = h->nl1;
  info->nl2 = h->nl2;
  info->n_particles = h->np;
  info->device_allocations = g_device_allocations.load(std::memory_order_relaxed);
  info->cg_fp32_products = h->pcg_fp32 ? 1 : 0;
  info->cg_replace_period = kPcgReplacePeriod;
  info->cg_smooth_degree = h->smooth_on ? h->smooth_k : 1;
  info->nnz_A = h->M.nnz;
  info->nnz_C = h->C.nnz;
  info->nnz_Q = h->Q.nnz;
  info->nnz_D = h->D.nnz;
  info->nnz_DT = h->DT.nnz;
  info->nnz_Pi = h->Pi.nnz;
  info->n_boundary_faces = h->n_bfaces;
  info->device_bytes = h->bytes;
  info->nnz_L = h->L.nnz;
  info->nnz_V = h->V.nnz;
  info->aux_cheb_degree = h->smooth_on ? h->cheb_k_sm : h->cheb_k;
  info->n_species = h->n_species;
  info->n_impedance_faces = h->n_imp_faces;
  info->n_absorb_faces = h->n_absorb_faces;
  info->n_inject_faces = h->n_inj_faces;
  return FEMPIC_OK;
}

int femPIC_last_timing(const FemPIC* h, double* times, int32_t n) {
  if (!h || !times || n < 1) return FEMPIC_ERR_ARG;
  const double v[10] = {h->t_particle_ms, h->t_field_ms, (double)h->launches, h->t_sort_ms, h->t_push_ms,
                        h->t_rhs_ms,      h->t_pcg_ms,   h->t_bupd_ms,         (double)h->cg_iters_sum, 0.0};
  for (int32_t k = 0; k < n && k < 10; ++k) times[k] = v[k];
  return FEMPIC_OK;
}

void femPIC_destroy(FemPIC* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (void* p : h->allocs) cudaFree(p);
  for (auto e : h->ev) cudaEventDestroy(e);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

const char* femPIC_last_error(const FemPIC* h) { return h ? h->err.c_str() : "NULL handle"; }

}  // extern "C"

// =============================================================================
// Batched execution of several handles (members) on one stream.
struct FemPICBatch {
  std::vector<FemPIC*> m;
  std::string err;
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  std::vector<MemberDesc> hd;
  MemberDesc* dd = nullptr;
  int32_t *pblk = nullptr, *tblk = nullptr, *r1blk = nullptr, *r2blk = nullptr, *zblk = nullptr, *cgblk = nullptr;
  int32_t* tile_sums = nullptr;
  GridBarrier* bar = nullptr;
  double* partials = nullptr;
  double* red = nullptr;
  int32_t* status = nullptr;
  int total_tiles = 0, cg_grid = 0, persist_grid = 0;
  cudaGraphExec_t graph = nullptr;
  bool graph_failed = false;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  double t_particle_ms = 0, t_field_ms = 0;
  int launches_per_step = 0;
  bool used_graph = false;
  std::vector<void*> allocs;
  // launch shapes picked by femPIC_batch_autotune: CTA size and grid of the
  // particle kernel (work-block tables for 128 and 256 particles), CTAs per SM
  // of the cooperative CG; events around those two kernels while tuning
  int32_t *ppblk128 = nullptr, *ppblk256 = nullptr;
  int part_block = 256, part_grid = 0, cg_per_sm = 0, cg_max_per_sm = 0;
  std::vector<int64_t> wnnz;
  bool time_kernels = false, tuning = false;
  cudaEvent_t kev[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

#define BCK(call)                                                \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) {                                     \
      b->err = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return FEMPIC_ERR_CUDA;                                    \
    }                                                            \
  } while (0)

template <class T>
int balloc(FemPICBatch* b, T** p, size_t n) {
  cudaError_t e = counted_malloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) {
    b->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FEMPIC_ERR_OOM : FEMPIC_ERR_CUDA;
  }
  b->allocs.push_back(*p);
  return FEMPIC_OK;
}

MemberDesc describe(FemPIC* h, double dt) {
  MemberDesc d;
  memset(&d, 0, sizeof(d));
  d.order = h->order;
  d.mixed = h->opts.precision == FEMPIC_MIXED;
  d.max_cross = h->opts.max_cross;
  d.max_it = h->opts.cg_max_it;
  d.n1 = h->n1;
  d.n2 = h->n2;
  d.n0 = h->n0;
  d.nt = h->n_tets;
  d.np = h->np;
  d.qw = h->q * h->weight;
  d.h = ((h->q / h->m) * dt) * 0.5;
  d.dt = dt;
  d.rtol = h->opts.cg_rtol;
  for (int k = 0; k < 3; ++k) d.B0[k] = h->opts.B0[k];
  d.geom = h->geom;
  d.nbr = h->nbr;
  d.dof0 = h->dof0;
  d.dof1 = h->dof1;
  d.dof2 = h->dof2;
  d.pec = h->pec1;
  for (int k = 0; k < 3; ++k) {
    d.x[k] = h->px[k];
    d.v[k] = h->pv[k];
    d.xa[k] = h->alt[k];
    d.va[k] = h->alt[3 + k];
  }
  d.tet = h->ptet;
  d.pid = h->pid;
  d.teta = h->ptet_alt;
  d.pida = h->pid_alt;
  d.ncross = h->pncross;
  d.hash = h->phash;
  d.cnt = h->sort_cnt;
  d.off = h->sort_off;
  d.e = h->e;
  d.e_prev = h->e_prev;
  d.e_new = h->e_new;
  d.b = h->b;
  d.dg = h->dg;
  d.dg_prev = h->dg_prev;
  d.rho = h->rho;
  d.rho_prev = h->rho_prev;
  d.A = h->M.view(h->Aval);
  d.R1 = h->M.view(h->R1val);
  d.Q = h->Q.view();
  d.C = h->C.view();
  d.dinvA = h->dinvA;
  d.D = view32(h->D, h->D32);
  d.DT = view32(h->DT, h->DT32);
  d.dinvL = h->dinvL32;
  d.t = h->aux_t;
  d.Pi = view32(h->Pi, h->Pi32);
  d.PiT = view32(h->PiT, h->PiT32);
  d.dinvV = h->dinvV;
  d.u = h->aux_u;
  d.L = h->cheb_k > 1 ? view32(h->L, h->L32) : CsrView32{0, nullptr, nullptr, nullptr};
  d.V = h->cheb_k > 1 ? view32(h->V, h->V32) : CsrView32{0, nullptr, nullptr, nullptr};
  d.tf = h->aux_tf;
  d.td = h->aux_td;
  d.t2 = h->aux_t2;
  d.uf = h->aux_uf;
  d.ud = h->aux_ud;
  d.u2 = h->aux_u2;
  d.cheb_k = h->cheb_k;
  memcpy(d.chebL, h->chebL, sizeof(d.chebL));
  memcpy(d.chebV, h->chebV, sizeof(d.chebV));
  d.rhs = h->rhs;
  d.r[0] = h->cg_r;
  d.r[1] = h->cg_r2;
  d.z = h->cg_z;
  d.p[0] = h->cg_p;
  d.p[1] = h->cg_p2;
  d.q = h->cg_q;
  d.q32 = h->cg_q32;
  d.r32 = h->cg_r32;
  d.Ab = h->nb > 0 ? BsrView{h->nb, h->brp, h->bci, h->bA} : BsrView{0, nullptr, nullptr, nullptr};
  d.binv = h->binv;
  d.status = h->d_status;
  d.cg_iters = h->d_cg_iters;
  d.cg_res = h->d_cg_res;
  d.crossings = h->d_cross;
  return d;
}

void write_back(FemPIC* h, const MemberDesc& d) {
  for (int k = 0; k < 3; ++k) {
    h->px[k] = d.x[k];
    h->pv[k] = d.v[k];
    h->alt[k] = d.xa[k];
    h->alt[3 + k] = d.va[k];
  }
  h->ptet = d.tet;
  h->pid = d.pid;
  h->ptet_alt = d.teta;
  h->pid_alt = d.pida;
  h->e = d.e;
  h->e_prev = d.e_prev;
  h->e_new = d.e_new;
  h->dg = d.dg;
  h->dg_prev = d.dg_prev;
  h->rho = d.rho;
  h->rho_prev = d.rho_prev;
}

std::vector<int32_t> prefix_blocks(const std::vector<int64_t>& work, int64_t per_block) {
  std::vector<int32_t> p(work.size() + 1, 0);
  for (size_t i = 0; i < work.size(); ++i) p[i + 1] = p[i] + (int32_t)((work[i] + per_block - 1) / per_block);
  return p;
}

// CTAs of the block-diagonal CG: per_sm per SM, each member at least one and
// the rest in proportion to its matrix entries
int set_cg_grid(FemPICBatch* b, int per_sm) {
  const int n = (int)b->m.size();
  b->cg_per_sm = per_sm;
  b->cg_grid = per_sm * b->num_sms;
  std::vector<int32_t> pc(n + 1, 0);
  double tot = 0;
  for (auto v : b->wnnz) tot += (double)v;
  const int spare = b->cg_grid - n;
  std::vector<int32_t> cnt(n, 1);
  int used = 0;
  for (int i = 0; i < n; ++i) {
    const int extra = tot > 0 ? (int)std::floor(spare * (double)b->wnnz[i] / tot) : 0;
    cnt[i] += extra;
    used += extra;
  }
  for (int i = 0; used < spare; i = (i + 1) % n, ++used) cnt[i]++;
  for (int i = 0; i < n; ++i) pc[i + 1] = pc[i] + cnt[i];
  BCK(cudaMemcpy(b->cgblk, pc.data(), pc.size() * 4, cudaMemcpyHostToDevice));
  return FEMPIC_OK;
}

BatchWork batch_work(FemPICBatch* b) {
  BatchWork w;
  w.n = (int32_t)b->m.size();
  w.d = b->dd;
  w.pblk = b->pblk;
  w.ppblk = b->part_block == 128 ? b->ppblk128 : b->ppblk256;
  w.pbs = b->part_block;
  w.tblk = b->tblk;
  w.r1blk = b->r1blk;
  w.r2blk = b->r2blk;
  w.zblk = b->zblk;
  w.cgblk = b->cgblk;
  w.tile_sums = b->tile_sums;
  w.bar = b->bar;
  w.partials = b->partials;
  w.red = b->red;
  w.status = b->status;
  return w;
}

// one batched step: 13 launches (+1 memset), no host synchronisation
int batch_launch_step(FemPICBatch* b, int max_it_all) {
  BatchWork w = batch_work(b);
  const int n = (int)b->m.size();
  const int g1 = (n + 127) / 128;
  const int pg = b->persist_grid;
  cudaStream_t s = b->stream;
  k_batch_begin<<<g1, 128, 0, s>>>(w);
  k_batch_zero<<<pg, 256, 0, s>>>(w);
  k_batch_hist<<<pg, 256, 0, s>>>(w);
  k_batch_scan_tiles<<<b->total_tiles, 1024, 0, s>>>(w);
  k_batch_scan_sums<<<n, 1024, 0, s>>>(w);
  k_batch_scan_add<<<b->total_tiles, 1024, 0, s>>>(w);
  k_batch_scatter<<<pg, 256, 0, s>>>(w);
  k_batch_swap_particles<<<g1, 128, 0, s>>>(w);
  if (b->time_kernels) BCK(cudaEventRecord(b->kev[0], s));
  k_batch_particles<<<b->part_grid, b->part_block, 0, s>>>(w);
  if (b->time_kernels) BCK(cudaEventRecord(b->kev[1], s));
  BCK(cudaGetLastError());
  BCK(cudaEventRecord(b->ev[1], s));
  k_batch_guess<<<pg, 256, 0, s>>>(w);
  k_batch_rhs<<<pg, 256, 0, s>>>(w);
  BCK(cudaMemsetAsync(b->bar, 0, sizeof(GridBarrier), s));
  BCK(cudaMemsetAsync(b->red, 0, 12 * (size_t)(n + 1) * sizeof(double), s));
  int kc = 1;
  for (FemPIC* h : b->m) kc = std::max(kc, h->cheb_k);
  void* args[] = {&w, &max_it_all, &kc};
  if (b->time_kernels) BCK(cudaEventRecord(b->kev[2], s));
  BCK(cudaLaunchCooperativeKernel((void*)k_batch_pcg, b->cg_grid, 256, args, 0, s));
  if (b->time_kernels) BCK(cudaEventRecord(b->kev[3], s));
  k_batch_bupdate<<<pg, 256, 0, s>>>(w);
  k_batch_end<<<g1, 128, 0, s>>>(w);
  BCK(cudaGetLastError());
  b->launches_per_step = 14;
  return FEMPIC_OK;
}

}  // namespace

extern "C" {

int femPIC_batch_create(FemPIC* const* members, int32_t n, FemPICBatch** out) {
  if (!out) return FEMPIC_ERR_ARG;
  *out = nullptr;
  FemPICBatch* b = new (std::nothrow) FemPICBatch();
  if (!b) return FEMPIC_ERR_OOM;
  *out = b;
  if (!members || n < 1) {
    b->err = "a batch needs at least one member";
    return FEMPIC_ERR_ARG;
  }
  for (int32_t i = 0; i < n; ++i) {
    FemPIC* h = members[i];
    if (!h || !h->stream) {
      b->err = "member " + std::to_string(i) + " is not a created handle";
      return FEMPIC_ERR_ARG;
    }
    if (h->opts.precision == FEMPIC_FP64_STRICT || h->opts.scheme != FEMPIC_SCHEME_TRAPEZOID) {
      b->err = "batched members must use FEMPIC_FP64 or FEMPIC_MIXED and the trapezoid scheme";
      return FEMPIC_ERR_ARG;
    }
    if (h->n_species != 1 || h->opts.push != FEMPIC_PUSH_BORIS) {
      b->err = "batched members must have a single species and the Boris push";
      return FEMPIC_ERR_ARG;
    }
    if (h->order > 2) {
      b->err = "batched members must be of order 1 or 2";
      return FEMPIC_ERR_ARG;
    }
    if (h->bimp) {
      b->err = "batched members cannot carry an impressed flux density";
      return FEMPIC_ERR_ARG;
    }
    if (h->n_absorb_faces > 0) {
      b->err = "batched members cannot have absorbing faces";
      return FEMPIC_ERR_ARG;
    }
    if (h->n_tets > 1024 * 1024) {
      b->err = "batched members are limited to 1048576 tets";
      return FEMPIC_ERR_ARG;
    }
    if (i > 0 && h->device != members[0]->device) {
      b->err = "all members must be on one device";
      return FEMPIC_ERR_ARG;
    }
    b->m.push_back(h);
  }
  b->device = members[0]->device;
  BCK(cudaSetDevice(b->device));
  cudaDeviceProp prop;
  BCK(cudaGetDeviceProperties(&prop, b->device));
  b->num_sms = prop.multiProcessorCount;
  BCK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
  for (auto& e : b->ev) BCK(cudaEventCreate(&e));
  std::vector<int64_t> wp, wt, w1, w2, wz, wnnz;
  for (FemPIC* h : b->m) {
    wp.push_back(h->np);
    wt.push_back(h->n_tets);
    w1.push_back(h->n1);
    w2.push_back(h->n2);
    wz.push_back((int64_t)h->n1 + h->n0 + h->n_tets);
    wnnz.push_back(h->M.nnz + h->D.nnz + h->DT.nnz + 2 * h->Pi.nnz + (h->cheb_k - 1) * (h->L.nnz + h->V.nnz));
  }
  auto pp = prefix_blocks(wp, 256), pt = prefix_blocks(wt, 1024), p1 = prefix_blocks(w1, 32),
       p2 = prefix_blocks(w2, 64), pz = prefix_blocks(wz, 256);
  b->total_tiles = pt.back();
  int per_sm = 0;
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_pcg, 256, 0));
  b->cg_max_per_sm = std::max(1, per_sm);
  if (b->cg_max_per_sm * b->num_sms < n) {
    b->err = "more members than co-resident CTAs for the batched CG";
    return FEMPIC_ERR_ARG;
  }
  b->wnnz = wnnz;
  int per_sm_p = 0;
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_p, k_batch_particles, 256, 0));
  b->persist_grid = std::max(1, per_sm_p) * b->num_sms;
  b->part_block = 256;
  b->part_grid = b->persist_grid;
  auto pp128 = prefix_blocks(wp, 128);
  int rc;
  if ((rc = balloc(b, &b->dd, n)) || (rc = balloc(b, &b->pblk, n + 1)) || (rc = balloc(b, &b->tblk, n + 1)) ||
      (rc = balloc(b, &b->r1blk, n + 1)) || (rc = balloc(b, &b->r2blk, n + 1)) || (rc = balloc(b, &b->zblk, n + 1)) ||
      (rc = balloc(b, &b->cgblk, n + 1)) || (rc = balloc(b, &b->tile_sums, b->total_tiles)) ||
      (rc = balloc(b, &b->bar, 1)) ||
      (rc = balloc(b, &b->partials, 8 * (size_t)b->cg_max_per_sm * b->num_sms)) ||
      (rc = balloc(b, &b->red, 12 * (size_t)(n + 1))) || (rc = balloc(b, &b->ppblk128, n + 1)) ||
      (rc = balloc(b, &b->ppblk256, n + 1)) || (rc = balloc(b, &b->status, 1)))
    return rc;
  BCK(cudaMemcpy(b->ppblk128, pp128.data(), pp128.size() * 4, cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->ppblk256, pp.data(), pp.size() * 4, cudaMemcpyHostToDevice));
  if ((rc = set_cg_grid(b, b->cg_max_per_sm))) return rc;
  BCK(cudaMemcpy(b->pblk, pp.data(), pp.size() * 4, cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->tblk, pt.data(), pt.size() * 4, cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->r1blk, p1.data(), p1.size() * 4, cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->r2blk, p2.data(), p2.size() * 4, cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->zblk, pz.data(), pz.size() * 4, cudaMemcpyHostToDevice));
  BCK(cudaMemset(b->status, 0, sizeof(int32_t)));
  return FEMPIC_OK;
}

int femPIC_batch_step(FemPICBatch* b, const double* dt, int32_t n_steps) {
  if (!b || !b->stream || !dt || n_steps < 0) return FEMPIC_ERR_ARG;
  const int n = (int)b->m.size();
  BCK(cudaSetDevice(b->device));
  int max_it_all = 1;
  b->hd.resize(n);
  for (int i = 0; i < n; ++i) {
    FemPIC* h = b->m[i];
    if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) {
      b->err = "dt must be positive and finite";
      return FEMPIC_ERR_ARG;
    }
    int rc = FEMPIC_OK;
    if (dt[i] != h->dt_cur) rc = form_system(h, dt[i]);
    if (rc) {
      b->err = h->err;
      return rc;
    }
    BCK(cudaStreamSynchronize(h->stream));
    BCK(cudaMemsetAsync(h->d_cross, 0, sizeof(unsigned long long), b->stream));
    b->hd[i] = describe(h, dt[i]);
    max_it_all = std::max(max_it_all, h->opts.cg_max_it);
  }
  BCK(cudaMemcpyAsync(b->dd, b->hd.data(), sizeof(MemberDesc) * n, cudaMemcpyHostToDevice, b->stream));
  BCK(cudaEventRecord(b->ev[0], b->stream));
  // capture one step in a CUDA graph the first time; replay it n_steps times
  if (!b->graph && !b->graph_failed && !b->tuning && n_steps > 0) {
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int rc = ok ? batch_launch_step(b, max_it_all) : FEMPIC_ERR_CUDA;
    ok = (cudaStreamEndCapture(b->stream, &g) == cudaSuccess) && ok && rc == FEMPIC_OK;
    if (ok) ok = cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      b->graph = nullptr;
      b->graph_failed = true;
      cudaGetLastError();
    }
  }
  double tp = 0, tf = 0;
  for (int32_t s = 0; s < n_steps; ++s) {
    if (b->graph) {
      BCK(cudaGraphLaunch(b->graph, b->stream));
      b->used_graph = true;
    } else {
      int rc = batch_launch_step(b, max_it_all);
      if (rc) return rc;
      b->used_graph = false;
    }
  }
  BCK(cudaEventRecord(b->ev[2], b->stream));
  BCK(cudaMemcpyAsync(b->hd.data(), b->dd, sizeof(MemberDesc) * n, cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  float tot = 0.f;
  BCK(cudaEventElapsedTime(&tot, b->ev[0], b->ev[2]));
  if (!b->graph) {
    float a = 0.f;
    BCK(cudaEventElapsedTime(&a, b->ev[0], b->ev[1]));
    tp = a;
    tf = tot - a;
  } else {
    tp = 0.0;
    tf = tot;
  }
  b->t_particle_ms = tp;
  b->t_field_ms = tf;
  int32_t bst = 0;
  BCK(cudaMemcpy(&bst, b->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  int worst = FEMPIC_OK;
  for (int i = 0; i < n; ++i) {
    FemPIC* h = b->m[i];
    write_back(h, b->hd[i]);
    h->steps += n_steps;
    h->since_sort = 1;
    h->dt_cur = dt[i];
    int rc = latch_status(h);
    if (rc && !worst) {
      worst = rc;
      b->err = "member " + std::to_string(i) + ": " + h->err;
    }
  }
  if (bst & kStatusBarrier) {
    b->err = "batched CG grid barrier timed out";
    return FEMPIC_ERR_BARRIER;
  }
  return worst;
}

int femPIC_batch_timing(const FemPICBatch* b, double* times, int32_t n) {
  if (!b || !times || n < 1) return FEMPIC_ERR_ARG;
  const double v[4] = {b->t_particle_ms + b->t_field_ms, (double)b->launches_per_step, b->used_graph ? 1.0 : 0.0,
                       (double)b->cg_grid};
  for (int32_t k = 0; k < n && k < 4; ++k) times[k] = v[k];
  return FEMPIC_OK;
}

void femPIC_batch_destroy(FemPICBatch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void* p : b->allocs) cudaFree(p);
  for (auto e : b->ev)
    if (e) cudaEventDestroy(e);
  for (auto e : b->kev)
    if (e) cudaEventDestroy(e);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* femPIC_batch_last_error(const FemPICBatch* b) { return b ? b->err.c_str() : "NULL batch"; }

int femPIC_batch_autotune(FemPICBatch* b, const double* dt, int32_t steps_per_candidate, femPIC_batch_tuning* out) {
  if (!b || !b->stream || !dt || steps_per_candidate < 1) return FEMPIC_ERR_ARG;
  BCK(cudaSetDevice(b->device));
  const int n = (int)b->m.size();
  // candidates: particle kernel CTA size x CTAs per SM (persistent) or one CTA
  // per work block; CG CTAs per SM that still give every member one CTA
  struct PartCfg {
    int block, grid;
  };
  std::vector<PartCfg> pcs;
  int64_t np_total = 0;
  for (FemPIC* h : b->m) np_total += h->np;
  for (int block : {128, 256}) {
    int per_sm = 0;
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_particles, block, 0));
    for (int k = 1; k <= std::max(1, per_sm); ++k) pcs.push_back({block, k * b->num_sms});
    int64_t blocks = 0;
    for (FemPIC* h : b->m) blocks += (h->np + block - 1) / block;
    if (blocks > (int64_t)std::max(1, per_sm) * b->num_sms) pcs.push_back({block, (int)std::min<int64_t>(blocks, 1 << 30)});
  }
  std::vector<int> ccs;
  for (int k = 1; k <= b->cg_max_per_sm; ++k)
    if (k * b->num_sms >= n) ccs.push_back(k);
  const int def_block = b->part_block, def_grid = b->part_grid, def_cg = b->cg_per_sm;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->graph_failed = false;
  for (auto& e : b->kev)
    if (!e) BCK(cudaEventCreate(&e));
  b->tuning = b->time_kernels = true;
  std::vector<double> pt(pcs.size(), 0.0), ct(ccs.size(), 0.0);
  std::vector<int> pn(pcs.size(), 0), cn(ccs.size(), 0);
  const size_t rounds = std::max(pcs.size(), ccs.size());
  int rc = FEMPIC_OK;
  for (size_t r = 0; r < rounds && !rc; ++r) {
    const size_t ip = r % pcs.size(), ic = r % ccs.size();
    b->part_block = pcs[ip].block;
    b->part_grid = pcs[ip].grid;
    if ((rc = set_cg_grid(b, ccs[ic]))) break;
    for (int32_t k = 0; k < steps_per_candidate && !rc; ++k) {
      rc = femPIC_batch_step(b, dt, 1);
      if (rc) break;
      float a = 0.f, c = 0.f;
      if (cudaEventElapsedTime(&a, b->kev[0], b->kev[1]) != cudaSuccess ||
          cudaEventElapsedTime(&c, b->kev[2], b->kev[3]) != cudaSuccess) {
        b->err = "autotune: kernel timing failed";
        rc = FEMPIC_ERR_CUDA;
        break;
      }
      pt[ip] += a;
      ct[ic] += c;
      pn[ip]++;
      cn[ic]++;
    }
  }
  b->tuning = b->time_kernels = false;
  if (rc) {
    b->part_block = def_block;
    b->part_grid = def_grid;
    set_cg_grid(b, def_cg);
    return rc;
  }
  size_t bp = 0, bc = 0;
  for (size_t i = 0; i < pcs.size(); ++i)
    if (pt[i] / pn[i] < pt[bp] / pn[bp]) bp = i;
  for (size_t i = 0; i < ccs.size(); ++i)
    if (ct[i] / cn[i] < ct[bc] / cn[bc]) bc = i;
  b->part_block = pcs[bp].block;
  b->part_grid = pcs[bp].grid;
  if ((rc = set_cg_grid(b, ccs[bc]))) return rc;
  if (out) {
    memset(out, 0, sizeof(*out));
    out->particle_block = pcs[bp].block;
    out->particle_grid = pcs[bp].grid;
    out->cg_ctas_per_sm = ccs[bc];
    out->particle_candidates = (int32_t)pcs.size();
    out->cg_candidates = (int32_t)ccs.size();
    out->steps = (int32_t)(rounds * steps_per_candidate);
    out->particle_ms = pt[bp] / pn[bp];
    out->cg_ms = ct[bc] / cn[bc];
    for (size_t i = 0; i < pcs.size(); ++i)
      if (pcs[i].block == def_block && pcs[i].grid == def_grid) out->particle_ms_default = pt[i] / pn[i];
    for (size_t i = 0; i < ccs.size(); ++i)
      if (ccs[i] == def_cg) out->cg_ms_default = ct[i] / cn[i];
  }
  return FEMPIC_OK;
}

}  // extern "C"

// ---- measurement: arithmetic throughput -----------------------------------
namespace {

constexpr int kAluChains = 8;
constexpr int kAluUnroll = 16;

// kAluChains independent chains x = x * m + c per thread; the final sum is
// written only if it equals an impossible value, so the chains stay live
template <class T>
__global__ void __launch_bounds__(256) k_alu_fma(int iters, T m, T c, T* out) {
  T a[kAluChains];
#pragma unroll
  for (int j = 0; j < kAluChains; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kAluUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kAluChains; ++j) a[j] = fma(a[j], m, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kAluChains; ++j) s += a[j];
  if (s == (T)-12345.0) out[0] = s;
}

// kAluChains independent chains x = c / (x + d) per thread (division as the
// compiler implements it)
__global__ void __launch_bounds__(256) k_alu_div(int iters, double c, double d, double* out) {
  double a[kAluChains];
#pragma unroll
  for (int j = 0; j < kAluChains; ++j) a[j] = 1.0 + (threadIdx.x + j) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kAluChains; ++j) a[j] = c / (a[j] + d);
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < kAluChains; ++j) s += a[j];
  if (s == -12345.0) out[0] = s;
}

}  // namespace

extern "C" int femPIC_measure_alu(int32_t device, int32_t kind, double* ops_per_second) {
  if (!ops_per_second || kind < FEMPIC_ALU_FP64_FMA || kind > FEMPIC_ALU_FP64_DIV) return FEMPIC_ERR_ARG;
  *ops_per_second = 0.0;
  if (cudaSetDevice(device) != cudaSuccess) return FEMPIC_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return FEMPIC_ERR_CUDA;
  const int blocks = prop.multiProcessorCount * 4, threads = 256;
  void* buf = nullptr;
  if (counted_malloc(&buf, 64) != cudaSuccess) return FEMPIC_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = FEMPIC_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = FEMPIC_ERR_CUDA;
  auto launch = [&](int iters) {
    if (kind == FEMPIC_ALU_FP64_FMA)
      k_alu_fma<double><<<blocks, threads>>>(iters, 0.999999, 1e-7, (double*)buf);
    else if (kind == FEMPIC_ALU_FP32_FMA)
      k_alu_fma<float><<<blocks, threads>>>(iters, 0.999999f, 1e-7f, (float*)buf);
    else
      k_alu_div<<<blocks, threads>>>(iters, 1.5, 0.75, (double*)buf);
  };
  // per-thread operations of one loop pass
  const double per_pass = kind == FEMPIC_ALU_FP64_DIV ? kAluChains : (double)kAluChains * kAluUnroll;
  int iters = 64;
  float ms = 0.f;
  for (int round = 0; round < 12 && rc == FEMPIC_OK; ++round) {
    launch(iters);  // warm-up (and first estimate)
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      rc = FEMPIC_ERR_CUDA;
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms >= 50.f) break;
    iters = (int)std::min<double>(1 << 26, iters * std::max(2.0, 80.0 / std::max(ms, 0.01f)));
  }
  if (rc == FEMPIC_OK && ms > 0.f)
    *ops_per_second = per_pass * iters * (double)blocks * threads / (ms * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  return rc;
}

// ---- impressed magnetic flux density (Section III-C, eq. conB) -----------
namespace {

// frees the allocations made after it (temporaries of one call), after the
// stream has drained
struct ScratchScope {
  FemPIC* h;
  size_t mark, bytes;
  explicit ScratchScope(FemPIC* hh) : h(hh), mark(hh->allocs.size()), bytes(hh->bytes) {}
  ~ScratchScope() {
    cudaStreamSynchronize(h->stream);
    for (size_t i = mark; i < h->allocs.size(); ++i) cudaFree(h->allocs[i]);
    h->allocs.resize(mark);
    h->bytes = bytes;
  }
};

// lanes per row in the projection's products: [*mu^-1] and [~div] rows, and
// the block-diagonal preconditioners' rows
#ifndef FEMPIC_PROJ_LPR_A
#define FEMPIC_PROJ_LPR_A 2
#endif
#ifndef FEMPIC_PROJ_LPR_P
#define FEMPIC_PROJ_LPR_P 1
#endif
constexpr int kProjChunk = 16;

// four timing events, destroyed with the scope
struct ScopedEvents {
  cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
  int create(FemPIC* h) {
    for (auto& x : e) CK(cudaEventCreate(&x));
    return FEMPIC_OK;
  }
  ~ScopedEvents() {
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
};  // CG iterations launched between convergence reads

struct ProjBuffers {
  double *r, *z, *p, *q, *sc, *part;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around each chunk of inner iterations
  double inner_ms = 0.0;
};

// x = A^-1 rhs by CG from x = 0, preconditioned by the product with P; every
// scalar on the device, the host reading the flag every kProjChunk iterations
int proj_pcg(FemPIC* h, const CsrView& A, const CsrView& P, const double* rhs, double* x, int32_t n, double rtol,
             int32_t max_it, ProjBuffers& w, int32_t* iters) {
  cudaStream_t st = h->stream;
  const int gv = grid_for(n, 256, h->num_sms * 8);
  CK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
  CK(cudaMemcpyAsync(w.r, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  k_spmv_dot<FEMPIC_PROJ_LPR_P, true><<<kRedGrid, kRedThreads, 0, st>>>(P, w.r, w.z, w.r, w.part, nullptr);
  k_cg_start<<<1, kRedThreads, 0, st>>>(w.sc, w.part, rtol * rtol);
  CK(cudaMemcpyAsync(w.p, w.z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  h->launches += 2;
  CK(cudaGetLastError());
  double hs[kCgN];
  bool timed = false;
  for (;;) {
    CK(cudaMemcpyAsync(hs, w.sc, sizeof(hs), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (timed) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, w.ev0, w.ev1));
      w.inner_ms += ms;
    }
    if (hs[kCgDone] != 0.0) break;
    CK(cudaEventRecord(w.ev0, st));
    for (int k = 0; k < kProjChunk; ++k) {
      k_spmv_dot<FEMPIC_PROJ_LPR_A, false><<<kRedGrid, kRedThreads, 0, st>>>(A, w.p, w.q, w.p, w.part, w.sc);
      k_cg_alpha<<<1, kRedThreads, 0, st>>>(w.sc, w.part);
      k_cg_xr<<<gv, 256, 0, st>>>(n, w.sc, w.p, w.q, x, w.r);
      k_spmv_dot<FEMPIC_PROJ_LPR_P, true><<<kRedGrid, kRedThreads, 0, st>>>(P, w.r, w.z, w.r, w.part, w.sc);
      k_cg_beta<<<1, kRedThreads, 0, st>>>(w.sc, w.part, max_it);
      k_cg_p<<<gv, 256, 0, st>>>(n, w.sc, w.z, w.p);
    }
    CK(cudaEventRecord(w.ev1, st));
    timed = true;
    h->launches += 6 * kProjChunk;
    CK(cudaGetLastError());
  }
  *iters = (int32_t)hs[kCgIt];
  if (hs[kCgDone] == 2.0) {
    h->err = "projection CG: the operator is not positive definite on the search direction";
    return FEMPIC_ERR_CG;
  }
  if (hs[kCgDone] == 3.0) {
    h->err = "projection CG reached its iteration cap before the tolerance";
    return FEMPIC_ERR_CG;
  }
  return FEMPIC_OK;
}

double host_norm(const std::vector<double>& v) {
  double s = 0.0;
  for (double x : v) s += x * x;
  return std::sqrt(s);
}

// || |A| |x| ||: the size of the terms of A x, the scale rounding errors of A x live on
double abs_product_norm(const HostCSR& A, const std::vector<double>& x) {
  double s = 0.0;
  for (int32_t r = 0; r < A.n_rows; ++r) {
    double t = 0.0;
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) t += std::fabs(A.val[k]) * std::fabs(x[A.col[k]]);
    s += t * t;
  }
  return std::sqrt(s);
}

int project_impressed(FemPIC* h, const double* B_host, int64_t n_points, int32_t constrained,
                      femPIC_projection* stats) {
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->stream));
  // host structures: M2 and the W2 numbering come back from the device
  HostCSR M2;
  M2.n_rows = h->M2.n_rows;
  M2.n_cols = h->M2.n_cols;
  M2.rowptr.resize((size_t)M2.n_rows + 1);
  M2.col.resize((size_t)h->M2.nnz);
  M2.val.resize((size_t)h->M2.nnz);
  std::vector<int32_t> dof2((size_t)h->n_tets * h->nl2);
  CK(cudaMemcpy(M2.rowptr.data(), h->M2.rp, sizeof(int32_t) * M2.rowptr.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(M2.col.data(), h->M2.ci, sizeof(int32_t) * M2.col.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(M2.val.data(), h->M2.v, sizeof(double) * M2.val.size(), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(dof2.data(), h->dof2, sizeof(int32_t) * dof2.size(), cudaMemcpyDeviceToHost));
  ProjModel P;
  const auto th0 = std::chrono::steady_clock::now();
  std::string err = build_projection(h->order, h->n_tets, h->n_faces, h->n2, h->hxyz.data(), h->htets.data(),
                                     dof2.data(), M2, &P);
  const double host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - th0).count();
  if (!err.empty()) {
    h->err = err;
    return FEMPIC_ERR_MESH;
  }
  const int64_t need = (int64_t)h->n_tets * P.nq;
  if (n_points != need) {
    h->err = "impressed B: " + std::to_string(n_points) + " points given, the rule has " + std::to_string(need);
    return FEMPIC_ERR_SIZE;
  }
  int rc = ensure_impressed(h);
  if (rc) return rc;
  double* b = h->bimp;
  ScratchScope scope(h);
  const int32_t n2 = h->n2, N3 = P.Dv.n_rows, nl2 = h->nl2;
  DevCSR Dv, DvT, Bm, Bs, Asm;
  double *qlam, *qw, *vol6, *Bq, *fl, *f, *t2, *wv, *r3, *z3, *p3, *q3, *sc3;
  ProjBuffers w;
  if ((rc = upload_csr(h, &Dv, P.Dv)) || (rc = upload_csr(h, &DvT, P.DvT)) || (rc = upload_csr(h, &Bm, P.Bm)) ||
      (rc = upload_csr(h, &Bs, P.Bs)) || (rc = upload_csr(h, &Asm, P.Asm)) || (rc = upload(h, &qlam, P.qlam)) ||
      (rc = upload(h, &qw, P.qw)) || (rc = upload(h, &vol6, P.vol6)) || (rc = dalloc(h, &Bq, 3 * (size_t)need)) ||
      (rc = dalloc(h, &fl, (size_t)h->n_tets * nl2)) || (rc = dalloc(h, &f, n2)) || (rc = dalloc(h, &t2, n2)) ||
      (rc = dalloc(h, &wv, n2)) || (rc = dalloc(h, &w.r, n2)) || (rc = dalloc(h, &w.z, n2)) ||
      (rc = dalloc(h, &w.p, n2)) || (rc = dalloc(h, &w.q, n2)) || (rc = dalloc(h, &w.sc, kCgN)) ||
      (rc = dalloc(h, &w.part, 2 * kRedGrid)) || (rc = dalloc(h, &r3, std::max(N3, 1))) ||
      (rc = dalloc(h, &z3, std::max(N3, 1))) || (rc = dalloc(h, &p3, std::max(N3, 1))) ||
      (rc = dalloc(h, &q3, std::max(N3, 1))) || (rc = dalloc(h, &sc3, kCgN)))
    return rc;
  cudaStream_t st = h->stream;
  ScopedEvents evs;
  if ((rc = evs.create(h))) return rc;
  w.ev0 = evs.e[2];
  w.ev1 = evs.e[3];
  CK(cudaMemcpyAsync(Bq, B_host, sizeof(double) * 3 * (size_t)need, cudaMemcpyHostToDevice, st));
  CK(cudaEventRecord(evs.e[0], st));
  // load f = <W2, B> / mu0, per tet then assembled
  const int gt = grid_for(h->n_tets, 128, 1 << 30);
  const double inv_mu0 = 1.0 / kMu0;
  if (h->order == 1)
    k_w2_load<1><<<gt, 128, 0, st>>>(h->n_tets, P.nq, qlam, qw, vol6, inv_mu0, h->geom, Bq, fl);
  else if (h->order == 2)
    k_w2_load<2><<<gt, 128, 0, st>>>(h->n_tets, P.nq, qlam, qw, vol6, inv_mu0, h->geom, Bq, fl);
  else
    k_w2_load<3><<<gt, 128, 0, st>>>(h->n_tets, P.nq, qlam, qw, vol6, inv_mu0, h->geom, Bq, fl);
  k_spmv<4><<<grid_for((int64_t)n2 * 4, 256, h->num_sms * 16), 256, 0, st>>>(Asm.view(), fl, f, 1.0, 0.0);
  h->launches += 2;
  CK(cudaGetLastError());
  // Galerkin projection b_G = M2^-1 f
  const double rtol_in = 1e-2 * h->opts.cg_rtol, rtol_out = h->opts.cg_rtol;
  const int32_t max_in = std::max(1000, 4 * h->opts.cg_max_it), max_out = std::max(1000, 10 * h->opts.cg_max_it);
  femPIC_projection S;
  memset(&S, 0, sizeof(S));
  S.host_ms = host_ms;
  S.bytes_per_inner_iteration = 12.0 * ((double)h->M2.nnz + (double)Bm.nnz) + 8.0 * (n2 + 1.0) + 104.0 * n2;
  int32_t it = 0;
  if ((rc = proj_pcg(h, h->M2.view(), Bm.view(), f, b, n2, rtol_in, max_in, w, &it))) return rc;
  S.inner_iterations += it;
  // the constraint residual Dv b_G against the size of its terms || |Dv| |b_G| ||:
  // a Galerkin projection that is divergence free up to rounding needs no correction
  std::vector<double> hr((size_t)N3), hb((size_t)n2);
  k_spmv<8><<<grid_for((int64_t)N3 * 8, 256, h->num_sms * 16), 256, 0, st>>>(Dv.view(), b, r3, 1.0, 0.0);
  h->launches++;
  CK(cudaMemcpyAsync(hr.data(), r3, sizeof(double) * N3, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hb.data(), b, sizeof(double) * n2, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double div0 = host_norm(hr), scale0 = abs_product_norm(P.Dv, hb);
  // reduce ||Dv b|| by rtol_out, but not below the rounding floor of its terms
  const double target = std::max(rtol_out * div0, 1e2 * 2.220446049250313e-16 * scale0);
  if (constrained && div0 > target) {
    // CG on S lambda = Dv b_G carried as b = b_G - M2^-1 Dv^T lambda; its residual is Dv b
    const double tol = target / div0;
    k_spmv_dot<FEMPIC_PROJ_LPR_P, true><<<kRedGrid, kRedThreads, 0, st>>>(Bs.view(), r3, z3, r3, w.part, nullptr);
    k_cg_start<<<1, kRedThreads, 0, st>>>(sc3, w.part, tol * tol);
    CK(cudaMemcpyAsync(p3, z3, sizeof(double) * N3, cudaMemcpyDeviceToDevice, st));
    h->launches += 2;
    const int g3 = grid_for(N3, 256, h->num_sms * 8), g2 = grid_for(n2, 256, h->num_sms * 8);
    double hs[kCgN];
    for (;;) {
      CK(cudaMemcpyAsync(hs, sc3, sizeof(hs), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (hs[kCgDone] != 0.0) break;
      k_spmv<8><<<grid_for((int64_t)n2 * 8, 256, h->num_sms * 16), 256, 0, st>>>(DvT.view(), p3, t2, 1.0, 0.0);
      h->launches++;
      if ((rc = proj_pcg(h, h->M2.view(), Bm.view(), t2, wv, n2, rtol_in, max_in, w, &it))) return rc;
      S.inner_iterations += it;
      k_spmv_dot<FEMPIC_PROJ_LPR_A, false><<<kRedGrid, kRedThreads, 0, st>>>(Dv.view(), wv, q3, p3, w.part, sc3);
      k_cg_alpha<<<1, kRedThreads, 0, st>>>(sc3, w.part);
      k_cg_sub<<<g2, 256, 0, st>>>(n2, sc3, wv, b);
      k_cg_sub<<<g3, 256, 0, st>>>(N3, sc3, q3, r3);
      k_spmv_dot<FEMPIC_PROJ_LPR_P, true><<<kRedGrid, kRedThreads, 0, st>>>(Bs.view(), r3, z3, r3, w.part, sc3);
      k_cg_beta<<<1, kRedThreads, 0, st>>>(sc3, w.part, max_out);
      k_cg_p<<<g3, 256, 0, st>>>(N3, sc3, z3, p3);
      h->launches += 7;
      CK(cudaGetLastError());
    }
    S.outer_iterations = (int32_t)hs[kCgIt];
    if (hs[kCgDone] == 2.0 || hs[kCgDone] == 3.0) {
      h->err = hs[kCgDone] == 2.0 ? "projection: the divergence Schur complement lost positivity"
                                  : "projection: outer CG reached its iteration cap before the tolerance";
      return FEMPIC_ERR_CG;
    }
  }
  // true constraint residual of the result, against the size of its terms
  k_spmv<8><<<grid_for((int64_t)N3 * 8, 256, h->num_sms * 16), 256, 0, st>>>(Dv.view(), b, r3, 1.0, 0.0);
  h->launches++;
  CK(cudaMemcpyAsync(hr.data(), r3, sizeof(double) * N3, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hb.data(), b, sizeof(double) * n2, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  {
    const double sc_end = abs_product_norm(P.Dv, hb);
    S.div_residual = sc_end > 0.0 ? host_norm(hr) / sc_end : 0.0;
  }
  if ((rc = refresh_btot(h))) return rc;
  CK(cudaEventRecord(evs.e[1], st));
  CK(cudaStreamSynchronize(st));
  float dms = 0.f;
  CK(cudaEventElapsedTime(&dms, evs.e[0], evs.e[1]));
  S.device_ms = dms;
  S.inner_ms = w.inner_ms;
  if (stats) *stats = S;
  return FEMPIC_OK;
}

}  // namespace

extern "C" {

int femPIC_impressed_points(FemPIC* h, double* xyz_host, int64_t* n_points) {
  if (!h || !h->stream || !n_points) return FEMPIC_ERR_ARG;
  const int n1d = h->order + 3;
  const int64_t nq = (int64_t)n1d * n1d * n1d, need = (int64_t)h->n_tets * nq;
  if (!xyz_host) {
    *n_points = need;
    return FEMPIC_OK;
  }
  if (*n_points != need) {
    h->err = "impressed points: buffer holds " + std::to_string(*n_points) + " points, the rule has " +
             std::to_string(need);
    return FEMPIC_ERR_SIZE;
  }
  // the rule of the projection's load, mapped into every tet (sorted vertices)
  ProjModel P;
  projection_rule(h->order, &P);
  for (int32_t t = 0; t < h->n_tets; ++t) {
    const int32_t* v = &h->htets[(size_t)t * 4];
    for (int64_t q = 0; q < nq; ++q) {
      const double* l = &P.qlam[(size_t)q * 4];
      for (int d = 0; d < 3; ++d)
        xyz_host[((size_t)t * nq + q) * 3 + d] =
            ((l[0] * h->hxyz[3 * (size_t)v[0] + d] + l[1] * h->hxyz[3 * (size_t)v[1] + d]) +
             l[2] * h->hxyz[3 * (size_t)v[2] + d]) +
            l[3] * h->hxyz[3 * (size_t)v[3] + d];
    }
  }
  return FEMPIC_OK;
}

int femPIC_set_impressed_B(FemPIC* h, const double* B_host, int64_t n_points, int32_t constrained,
                           femPIC_projection* stats) {
  if (!h || !h->stream) return FEMPIC_ERR_ARG;
  if (!B_host) {
    if (n_points != 0) return FEMPIC_ERR_ARG;
    if (h->bimp) {
      CK(cudaSetDevice(h->device));
      CK(cudaMemsetAsync(h->bimp, 0, sizeof(double) * h->n2, h->stream));
      int rc = refresh_btot(h);
      if (rc) return rc;
      CK(cudaStreamSynchronize(h->stream));
    }
    if (stats) memset(stats, 0, sizeof(*stats));
    return FEMPIC_OK;
  }
  return project_impressed(h, B_host, n_points, constrained, stats);
}

}  // extern "C"

extern "C" int femPIC_set_injection(FemPIC* h, const femPIC_injector* inj, int32_t n, uint64_t seed) {
  if (!h || !h->stream || n < 0 || (n > 0 && !inj)) return FEMPIC_ERR_ARG;
  bool has[kMaxSpecies] = {};
  double drift[kMaxSpecies][3] = {}, sigma[kMaxSpecies][3] = {};
  for (int32_t k = 0; k < n; ++k) {
    const int32_t s = inj[k].species;
    if (s < 0 || s >= h->n_species || has[s]) {
      h->err = "injector " + std::to_string(k) + ": species out of range or given twice";
      return FEMPIC_ERR_ARG;
    }
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(inj[k].v_drift[c]) || !std::isfinite(inj[k].v_sigma[c])) {
        h->err = "injector " + std::to_string(k) + ": non-finite velocity";
        return FEMPIC_ERR_ARG;
      }
    has[s] = true;
    for (int c = 0; c < 3; ++c) {
      drift[s][c] = inj[k].v_drift[c];
      sigma[s][c] = inj[k].v_sigma[c];
    }
  }
  if (n > 0 && h->n_inj_faces == 0) {
    h->err = "injectors need FEMPIC_FACE_INJECT faces";
    return FEMPIC_ERR_ARG;
  }
  for (int k = 0; k < kMaxSpecies; ++k) {
    h->inj_has[k] = has[k];
    for (int c = 0; c < 3; ++c) {
      h->inj_drift[k][c] = drift[k][c];
      h->inj_sigma[k][c] = sigma[k][c];
    }
  }
  h->inj_seed = seed;
  return FEMPIC_OK;
}
