/*
 * fempic.h -- C ABI of the GB300 EM-FEMPIC library.
 *
 * The library advances one charged species and the electromagnetic field on an
 * unstructured tetrahedral mesh with the higher-order, charge-conserving
 * finite-element particle-in-cell method of Crawford, Ramachandran, O'Connor,
 * Luginsland and Shanker, "Higher Order Charge Conserving Electromagnetic
 * Finite Element Particle in Cell Method" (arXiv 2111.12411):
 *
 *   - E is expanded in order-p interpolatory Whitney edge functions W1 and B in
 *     face functions W2 (Section III-A, Appendix), p = 1, 2 or 3;
 *   - each step gathers E and B at every particle, applies the Lorentz force
 *     (Section II), moves the particle on a straight chord, walks the chord
 *     through the tets by ray-face intersection, and deposits the exact path
 *     integral q w int W1_i . dr of every edge function into the current DOFs
 *     g (Section III-B, g_i = <W1_i, G>), which conserves charge;
 *   - the fields advance with the implicit Newmark (average acceleration)
 *     scheme, gamma = 1/2, beta = 1/4 (Section III-B), solved on the device by
 *     preconditioned conjugate gradients;
 *   - charge is measured with the order-p nodal functions W0 (Section III-A).
 *
 * Conventions shared by every entry point:
 *   - All pointers named *_host are host memory owned by the caller; the
 *     library copies from/to them and never keeps them.  All device memory is
 *     owned by the library and released by femPIC_destroy.
 *   - Every function returns FEMPIC_OK (0) or one of the FEMPIC_ERR_* codes and
 *     never exits, aborts or traps; femPIC_last_error gives a message.
 *   - Device-side failures (crossing cap, CG iteration cap, barrier timeout)
 *     are latched in a device status word and reported by the next call that
 *     synchronises (femPIC_step, femPIC_sync, femPIC_get).
 *   - DOF numbering: tet vertices are sorted by global node id; edges (sorted
 *     node pairs) and faces (sorted triples) are numbered in lexicographic
 *     order.  Order 1: W1 DOF = edge, W2 DOF = face, W0 DOF = node.  Order 2:
 *     W1 DOFs 2*edge+v (v=0: (3 l_lo - 1) w, v=1: (3 l_hi - 1) w) then
 *     2*N_e + 2*face + v (v=0: 3 l_u w_st, v=1: 3 l_t w_su for face s<t<u);
 *     W2 DOFs 3*face + v ((4 l_v - 1) w_stu for the v-th face vertex) then
 *     3*N_f + 3*tet + i (4 l_i w_(face opposite local vertex i), i = 0..2);
 *     W0 DOFs nodes then N_n + edge (mid-edge Lagrange nodes).  Order 3
 *     (Appendix; P_i / P^_i the Silvester polynomials at scale = index sum):
 *     W1 DOFs 3*edge + v (P^_a(l_lo) P^_b(l_hi) w, (a,b) = (3,1), (2,2),
 *     (1,3)), then 3*N_e + 6*face + v (pairs (s,t) then (s,u) of face s<t<u,
 *     each with (a,b,c) = (2,1,1), (1,2,1), (1,1,2) on the pair's first and
 *     second vertex and the face's third, the third as P_c), then 3*N_e +
 *     6*N_f + 3*tet + v (pairs (0,1), (0,2), (0,3) of the sorted tet, all
 *     indices 1); W2 DOFs 6*face + v ((a,b,c) = (3,1,1), (1,3,1), (1,1,3),
 *     (2,2,1), (2,1,2), (1,2,2)) then 6*N_f + 12*tet + 4*i + v (faces
 *     opposite local vertices i = 0..2, index 2 on the v-th of face vertex
 *     0, 1, 2 or the opposite vertex); W0 DOFs nodes, then N_n + 2*edge + v
 *     (lattice point nearer the lower vertex first), then N_n + 2*N_e + face.
 *   - Units are SI.  Boundary faces are perfect electric conductors (W1 DOFs
 *     on them held at 0) unless femPIC_create_ext tags them impedance
 *     (first-order absorbing).  Particles reflect specularly at a wall unless
 *     femPIC_create_ext tags its face absorbing: there the path ends at the
 *     wall and the particle is re-injected on the faces tagged injecting
 *     (femPIC_set_injection).
 *   - Besides the Boris push on a straight chord (the default), opts.push
 *     selects the paper's Adams-Bashforth 4 push on a polynomial path
 *     (Section III-B), orders 1 and 2.
 */
#ifndef FEMPIC_H
#define FEMPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
  FEMPIC_OK = 0,
  FEMPIC_ERR_ARG = 1,    /* bad argument (NULL, size, order, option)            */
  FEMPIC_ERR_MESH = 2,   /* degenerate tet, node out of range, non-manifold face */
  FEMPIC_ERR_OOM = 3,    /* device allocation failed                             */
  FEMPIC_ERR_CUDA = 4,   /* a CUDA call failed (message has the CUDA error)      */
  FEMPIC_ERR_CG = 5,     /* CG hit its iteration cap before the tolerance        */
  FEMPIC_ERR_WALK = 6,   /* a particle hit the face-crossing cap in one step     */
  FEMPIC_ERR_SIZE = 7,   /* caller buffer size does not match the quantity       */
  FEMPIC_ERR_STATE = 8,  /* call not valid in the current state                  */
  FEMPIC_ERR_BARRIER = 9, /* a device grid barrier timed out                     */
  FEMPIC_ERR_BOUNDS = 10  /* an index out of range (builds with -DFEMPIC_CHECKS=1) */
};

/* ---- precision modes (set at create) ------------------------------------ */
enum {
  FEMPIC_FP64_STRICT = 0, /* all FP64, every operation rounded separately in the
                             order the reference evaluation uses (no FMA): the
                             walk's decisions are bit-reproducible             */
  FEMPIC_FP64 = 1,        /* all FP64, fused multiply-add and factored forms   */
  FEMPIC_MIXED = 2        /* FP32 gather and push; FP64 positions, walk,
                             deposit, charge and CG (order 3 has no FP32
                             kernel: it runs as FEMPIC_FP64)                  */
};

/* ---- field time schemes ------------------------------------------------- */
enum {
  FEMPIC_SCHEME_TRAPEZOID = 0, /* gamma = 1/2, beta = 1/4 on the [b; e] system */
  FEMPIC_SCHEME_WAVE = 1       /* second-order e form with free gamma, beta    */
};

/* ---- particle push (set at create) --------------------------------------- */
enum {
  FEMPIC_PUSH_BORIS = 0, /* Boris rotation, straight chord x^{n+1} = x^n + dt v^{n+1/2};
                            FEMPIC_V holds v^{n-1/2}                           */
  FEMPIC_PUSH_AB4 = 1    /* the paper's Adams-Bashforth push (Section III-B): v^{n+1}
                            = v^n + dt sum_j beta_j a^{n-j}, path x(s) = x^n + dt
                            int_0^s V, V the Lagrange polynomial through the last
                            velocities (quartic in s); orders 1..3 while the history
                            fills; the walk samples the path at 8 steps per tet and
                            bisects the crossings; walls mirror the path and the
                            history; current by the (2p+2)-point Gauss-Legendre
                            rule.  FEMPIC_V holds v^n.  One kernel with every
                            operation rounded separately, whatever the precision
                            mode; particles are not re-sorted; setting X, V or TET
                            restarts the history.                                */
};

/* ---- quantities for femPIC_get / femPIC_set ----------------------------- */
enum {
  FEMPIC_E = 0,        /* double[N1]  electric field DOFs e^n                   */
  FEMPIC_B = 1,        /* double[N2]  magnetic flux DOFs b^n (self field only;
                          the uniform B0 and FEMPIC_B_IMPRESSED are added at
                          the gather)                                           */
  FEMPIC_DG = 2,       /* double[N1]  g^n - g^{n-1} deposited by the last step  */
  FEMPIC_RHO = 3,      /* double[N0]  rho_k = q w sum_p W0_k(x_p)               */
  FEMPIC_X = 4,        /* double[3*Np] positions, particle-id order, xyz interleaved */
  FEMPIC_V = 5,        /* double[3*Np] velocities v^{n-1/2}                     */
  FEMPIC_TET = 6,      /* int32[Np]   owning tet                                */
  FEMPIC_NCROSS = 7,   /* int32[Np]   face crossings (incl. wall hits), last step */
  FEMPIC_HASH = 8,     /* uint64[Np]  FNV-1a style hash of the last step's crossing
                          events: h = (h ^ code) * 1099511628211 from
                          14695981039346656037, code = new tet id, or
                          0x80000000 | local face for a wall reflection        */
  FEMPIC_E_PREV = 9,   /* double[N1]  e^{n-1} (wave scheme, CG initial guess)    */
  FEMPIC_DG_PREV = 10, /* double[N1]  Delta g of the step before (wave scheme)   */
  FEMPIC_DIAG = 11,    /* femPIC_diag (get only)                                */
  FEMPIC_PHI = 12,     /* double[N0]  potential of the electrostatic start (get) */
  FEMPIC_SPECIES = 13, /* int32[Np]   species index of each particle (get)      */
  FEMPIC_B_IMPRESSED = 14, /* double[N2] W2 coefficients of an impressed flux
                          density (zeros when none is set): added to b wherever
                          the particles sample B, absent from the field update */
  FEMPIC_J = 15          /* double[N1]  (g^n - g^{n-1}) / dt of the last step: the
                          W1 moments <W1_i, J> of the current averaged over the
                          step (get only; FEMPIC_ERR_STATE before the first step) */
};

/* ---- operators for femPIC_apply ----------------------------------------- */
enum {
  FEMPIC_OP_M1 = 0,  /* [*eps]    N1 x N1 (PEC rows/cols removed)              */
  FEMPIC_OP_K = 1,   /* K = C^T [*mu^-1] C, N1 x N1 (PEC rows/cols removed)    */
  FEMPIC_OP_C = 2,   /* curl map C, N2 x N1: curl W1_j = sum_f C_fj W2_f        */
  FEMPIC_OP_D = 3,   /* grad map D, N1 x N0: grad W0_k = sum_i D_ik W1_i        */
  FEMPIC_OP_DT = 4,  /* D^T, N0 x N1                                            */
  FEMPIC_OP_M2 = 5,  /* [*mu^-1], N2 x N2                                       */
  FEMPIC_OP_A = 6,   /* system matrix of the last dt, N1 x N1                   */
  FEMPIC_OP_L = 7,   /* nodal Laplacian D^T [*eps] D on interior W0 DOFs        */
  FEMPIC_OP_PI = 8,  /* vector nodal interpolation Pi, N1 x 3*n_nodes: W1
                        coefficients of hat_v e_c (exact at order 2; edge
                        moments at order 1), PEC rows removed; an auxiliary
                        space of the CG preconditioner                        */
  FEMPIC_OP_PIT = 9  /* Pi^T, 3*n_nodes x N1                                   */
};

typedef struct FemPIC FemPIC; /* opaque handle */

/* Mesh (Section III-A: K = {N, E, F, T}).  Vertex order inside a tet is free. */
typedef struct {
  int32_t n_nodes;
  int32_t n_tets;
  const double* xyz_host;   /* [3*n_nodes] node coordinates (m)               */
  const int32_t* tets_host; /* [4*n_tets] node ids                             */
} femPIC_mesh;

/* One species of macro particles (Section II: a single species). */
typedef struct {
  double q;                 /* charge of one physical particle (C)             */
  double m;                 /* mass of one physical particle (kg)              */
  double weight;            /* physical particles per macro particle           */
  int64_t n;                /* number of macro particles (>= 0)                */
  const double* x_host;     /* [3n] positions                                  */
  const double* v_host;     /* [3n] velocities, taken as v^{-1/2}              */
  const int32_t* tet_host;  /* [n] tet containing each position (checked)      */
} femPIC_species;

typedef struct {
  int32_t precision;    /* FEMPIC_FP64_STRICT / FEMPIC_FP64 / FEMPIC_MIXED     */
  int32_t scheme;       /* FEMPIC_SCHEME_*                                     */
  double gamma, beta;   /* Newmark parameters of the wave scheme               */
  double cg_rtol;       /* stop when ||r|| <= cg_rtol ||rhs||                   */
  int32_t cg_max_it;    /* iteration cap (FEMPIC_ERR_CG when reached)          */
  int32_t max_cross;    /* face crossings per particle per step (FEMPIC_ERR_WALK) */
  int32_t sort_period;  /* re-sort particles by tet every this many steps (0 = never) */
  double B0[3];         /* uniform impressed magnetic flux density (T)         */
  double rho_ion;       /* uniform neutralising charge density (C/m^3)         */
  int32_t es_init;      /* 1: solve the electrostatic start at create          */
  int32_t diagnostics;  /* 1: compute continuity/Gauss residuals every step    */
  int32_t device;       /* CUDA device ordinal                                  */
  void* stream;         /* cudaStream_t to run on; NULL = library-owned stream */
  int32_t push;         /* FEMPIC_PUSH_* (default FEMPIC_PUSH_BORIS)           */
} femPIC_opts;

/* Per-step diagnostics (Section IV-D): continuity and Gauss residuals.
   With opts.diagnostics set, femPIC_get(FEMPIC_DIAG) computes the continuity,
   Gauss and div b residuals of the state as it is at the call (after the first
   step; zeros before it), so a state changed by femPIC_set shows in them;
   without it they are zero.  The CG figures, crossings and absorbed counts are
   those of the last step. */
typedef struct {
  int64_t steps;            /* steps taken since create                        */
  int32_t status;           /* latched FEMPIC_* status of the device            */
  int32_t cg_iterations;    /* iterations of the last field solve              */
  double cg_residual;       /* ||r|| / ||rhs|| of the last field solve          */
  double continuity_abs;    /* ||rho^{n+1} - rho^n - D^T Delta g||_2, interior W0 */
  double continuity_ref;    /* ||rho^{n+1} - rho^n||_2, interior W0             */
  double gauss_abs;         /* ||D^T [*eps] e + rho + rho_ion <W0,1>||_2, interior */
  double gauss_ref;         /* ||rho||_2, interior                             */
  double crossings;         /* face crossings in the last step (all particles) */
  double absorbed;          /* particles absorbed on walls (and re-injected) by the
                               last femPIC_step call, all its steps           */
  double divb_abs;          /* Gauss's magnetic law of b (+ the impressed part):
                               ||m||_2, m_ti = sign(det J_t) int_ref W3_i div W2 . b
                               per tet (zero iff div b = 0)                    */
  double divb_ref;          /* the size of the terms of m: || sum_j |.| ||_2    */
} femPIC_diag;

typedef struct {
  int32_t n_nodes, n_tets, n_edges, n_faces;
  int32_t order;
  int32_t n0, n1, n2;       /* global W0, W1, W2 DOF counts                     */
  int32_t nl0, nl1, nl2;    /* local DOFs per tet                               */
  int64_t n_particles;
  int64_t nnz_A, nnz_C, nnz_Q;  /* stored entries of A, C, C^T [*mu^-1] */
  int64_t nnz_D, nnz_DT;        /* stored entries of D and D^T          */
  int64_t nnz_Pi;               /* stored entries of the vector nodal interpolation */
  int32_t n_boundary_faces;
  size_t device_bytes;      /* device memory held by the handle                */
  int64_t nnz_L;            /* stored entries of the nodal Laplacian D^T [*eps] D */
  int64_t nnz_V;            /* stored entries of Pi^T A Pi (0 without smoothing) */
  int32_t aux_cheb_degree;  /* Chebyshev degree of the auxiliary-space solves
                               in the CG preconditioner (1 = diagonal only)  */
  int32_t n_species;        /* species of the handle                          */
  int32_t n_impedance_faces; /* boundary faces with the absorbing condition   */
  int32_t n_absorb_faces;   /* boundary faces that absorb particles            */
  int32_t n_inject_faces;   /* boundary faces particles are re-injected on     */
  int64_t device_allocations; /* device allocations (cudaMalloc) this library has
                               made in the process so far, all handles and
                               batches together (not a per-handle figure)     */
  int32_t cg_fp32_products; /* 1: the field solve's direction products run in
                               FP32, the residual recomputed in FP64 every
                               cg_replace_period iterations and before a solve
                               is accepted (order 2); 0: FP64 products        */
  int32_t cg_replace_period;
  int32_t cg_smooth_degree; /* degree of the Chebyshev smoother on B^-1 A that
                               replaces the block-Jacobi term of the CG
                               preconditioner (1: block Jacobi; > 1 at order 2,
                               whose 2x2 blocks it works on)                  */
} femPIC_info;

/* Fill *opts with defaults: FP64, trapezoid, cg_rtol 1e-12, cg_max_it 2000,
 * max_cross 4096, sort_period 1, B0 = 0, rho_ion = 0, es_init 1,
 * diagnostics 0, device 0, stream NULL. */
void femPIC_default_opts(femPIC_opts* opts);

/* Build the mesh complex, DOF numbering, Hodge/curl/gradient matrices (Section
 * III-A) and upload mesh, matrices and particles to the device.  order is p
 * (1, 2 or 3; FEMPIC_PUSH_AB4 and batching take 1 or 2 only).  opts may be
 * NULL for defaults.  On success *out holds a handle.
 * On failure *out may still hold a handle that only carries the error message
 * (femPIC_last_error); release it with femPIC_destroy. */
int femPIC_create(const femPIC_mesh* mesh, int32_t order, const femPIC_species* species,
                  const femPIC_opts* opts, FemPIC** out);

/* As femPIC_create, with two additions of the paper's problem statement:
 *   - several species (up to FEMPIC_MAX_SPECIES, e.g. the ions and electrons
 *     of the plasma-ball example, Section IV): species[k] has its own q, m and
 *     weight; particle ids run through the species in order (species 0's
 *     particles first), the order of FEMPIC_X/V/TET; their currents and charges
 *     add;
 *   - impedance faces (Section II, eq. impedanceBC with Psi_I = 0, the
 *     first-order absorbing condition): bface_tag_host (NULL = all PEC) is
 *     int32[4*n_tets], the tag of the face opposite the i-th vertex of each tet
 *     as given in the mesh, read for boundary faces only, a sum of bits:
 *     FEMPIC_FACE_IMPEDANCE (else PEC), FEMPIC_FACE_ABSORB (particles whose
 *     path reaches the face stop on it, their current deposited up to the
 *     wall, and are re-injected, see femPIC_set_injection; else they reflect
 *     specularly), FEMPIC_FACE_INJECT (re-injection happens on such faces).
 *     The surface matrix [*_I]_ij = Y0 <n x W1_i, n x W1_j> (Section III-A;
 *     Y0 = sqrt(eps0/mu0), free-space admittance) enters the trapezoid rule as
 *     ([*eps] + dt^2/4 K + dt/2 [*_I]) e^{n+1} = ([*eps] - dt^2/4 K -
 *     dt/2 [*_I]) e^n + dt C^T [*mu^-1] b^n - Delta g.  W1 DOFs on impedance
 *     faces are free; an edge shared with a PEC face stays PEC.  Needs the
 *     trapezoid scheme (FEMPIC_ERR_ARG otherwise).
 * Errors as femPIC_create; n_species outside 1..FEMPIC_MAX_SPECIES, a NULL
 * species array or a species with m <= 0, weight < 0 or a non-finite q, a
 * tag outside 0..7, or absorbing faces with FEMPIC_PUSH_AB4 give
 * FEMPIC_ERR_ARG.  Handles with several species or absorbing faces cannot
 * join a batch. */
#define FEMPIC_MAX_SPECIES 8
enum { FEMPIC_FACE_IMPEDANCE = 1, FEMPIC_FACE_ABSORB = 2, FEMPIC_FACE_INJECT = 4 };
int femPIC_create_ext(const femPIC_mesh* mesh, int32_t order, const femPIC_species* species, int32_t n_species,
                      const int32_t* bface_tag_host, const femPIC_opts* opts, FemPIC** out);

/* Re-injection of absorbed particles (the paper's drift-tube beam enters at
 * one end; it does not say how): a particle absorbed by a FEMPIC_FACE_ABSORB
 * face during a step is replaced in its slot (same id, same species) at the
 * end of that step by a sample of its species' injector on the
 * FEMPIC_FACE_INJECT faces, and its charge q w W0(x) is added to rho (the
 * absorbed particle's is not); the particle count stays fixed.  Sampling,
 * with every operation rounded once whatever the precision mode: u_d = top 53
 * bits of SplitMix64 (Steele, Lea and Flood) at state seed + (c + 1)
 * 0x9E3779B97F4A7C15, c = (step << 40) + (particle id << 6) + d, step the
 * 0-based index of the step since create; the face is the first (in global
 * face order) whose running area sum exceeds u_0 times the total; the point
 * (a + u1 (b - a)) + u2 (c - a) on its sorted vertices, (u1, u2) = (u_1, u_2)
 * or (1 - u_1, 1 - u_2) when u_1 + u_2 > 1; the tet is the face's; velocity
 * component j = v_drift[j] + v_sigma[j] ((u_(3+12j) + ... + u_(14+12j)) - 6).
 * inj[k] configures species inj[k].species; n = 0 clears.  A step of a
 * handle with absorbing faces and a species without an injector returns
 * FEMPIC_ERR_STATE.  Errors: FEMPIC_ERR_ARG (species out of range, given
 * twice, non-finite values, or injectors without FEMPIC_FACE_INJECT faces). */
typedef struct {
  int32_t species;   /* species index (0 for femPIC_create handles)          */
  double v_drift[3]; /* m/s                                                   */
  double v_sigma[3]; /* m/s, spread of each component (Irwin-Hall, 12 uniforms) */
} femPIC_injector;
int femPIC_set_injection(FemPIC* h, const femPIC_injector* inj, int32_t n, uint64_t seed);

/* Advance n_steps PIC steps of size dt (s): gather, Lorentz push, walk,
 * charge-conserving deposit, Newmark field solve, b update, rho measurement
 * (Section III-B); with absorbing faces, the absorbed particles' slots are
 * refilled before rho is measured (femPIC_set_injection).  Returns after the
 * device finished; the return value is the latched device status
 * (FEMPIC_ERR_WALK crossing cap, FEMPIC_ERR_CG iteration cap,
 * FEMPIC_ERR_BARRIER grid-barrier timeout; FEMPIC_ERR_BOUNDS in a checked
 * build), FEMPIC_ERR_ARG for a bad dt, or FEMPIC_ERR_STATE for absorbing
 * faces with a species that has no injector. */
int femPIC_step(FemPIC* h, double dt, int32_t n_steps);

/* Same as femPIC_step but returns as soon as the work is enqueued on the
 * handle's stream; femPIC_sync collects the status. */
int femPIC_step_async(FemPIC* h, double dt, int32_t n_steps);
int femPIC_sync(FemPIC* h);

/* Copy a quantity to/from caller memory; bytes must equal its size
 * (FEMPIC_ERR_SIZE otherwise), read-only quantities reject femPIC_set
 * (FEMPIC_ERR_ARG), and a tet id out of range in FEMPIC_TET or a non-finite
 * value in FEMPIC_X or FEMPIC_V is rejected (FEMPIC_ERR_ARG) before anything
 * is copied.  X and TET are set one at a time: the caller keeps every
 * position inside its owning tet, as femPIC_create checks (barycentric
 * coordinates >= -1e-9).  Particle quantities are in particle-id order. */
int femPIC_get(FemPIC* h, int32_t what, void* host_dst, size_t bytes);
int femPIC_set(FemPIC* h, int32_t what, const void* host_src, size_t bytes);

/* Copy the same quantities to/from device memory the caller owns (same
 * device, ordered on the handle's stream; synchronous on return).  Unlike
 * femPIC_set, femPIC_set_device does not range-check tet ids: the caller
 * guarantees 0 <= tet < n_tets.  A library built with -DFEMPIC_CHECKS=1
 * checks them on the device before copying (FEMPIC_ERR_BOUNDS, nothing
 * copied), again in the particle kernels (the particle is skipped and the
 * step returns FEMPIC_ERR_BOUNDS), and checks the per-tet DOF and neighbour
 * tables once at create. */
int femPIC_get_device(FemPIC* h, int32_t what, void* dev_dst, size_t bytes);
int femPIC_set_device(FemPIC* h, int32_t what, const void* dev_src, size_t bytes);

/* y = Op x for one of the FEMPIC_OP_* operators (host vectors). */
int femPIC_apply(FemPIC* h, int32_t op, const double* x_host, size_t nx,
                 double* y_host, size_t ny);

/* E(x) and B(x) (B includes B0) at n points with known owning tets, evaluated
 * with the handle's precision mode (Section III-A field expansions). */
int femPIC_eval_fields(FemPIC* h, int64_t n, const double* x_host, const int32_t* tet_host,
                       double* E_host, double* B_host);

/* Field probe that makes no device allocation.  The paper has no counterpart;
 * this is a library service for callers that must not allocate device memory
 * while they run: a serving loop that has handed its whole HBM budget to
 * simulation instances, or a latency-critical host loop that cannot afford the
 * device-wide synchronisation that cudaMalloc/cudaFree bring with them.
 *
 * Same inputs, outputs and result as femPIC_eval_fields (the same kernel runs),
 * but the points, tet ids and results are staged in one fixed device array
 * that lives in the library for as long as it is loaded (on every device that
 * uses it), instead of buffers allocated per call.  Limits and rules:
 *   - at most FEMPIC_PROBE_MAX_POINTS points per call; larger n returns
 *     FEMPIC_ERR_SIZE and touches nothing;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current, and so does the first
 *     call after that device's context was created anew (a cudaDeviceReset,
 *     say): the address is cached with the id of the context it belongs to;
 *     under CUDA's lazy module loading the first call per device, order and
 *     precision mode also loads the field kernel, which may allocate and
 *     synchronise inside the CUDA runtime: make these first calls before any
 *     stream capture or latency-critical work starts;
 *   - femPIC_info.device_allocations does not change across a call after
 *     those first ones;
 *   - all calls share the array and it keeps the last call's contents; every
 *     output value is rewritten by each call, so nothing needs clearing.
 *     Calls that overlap on the GPU (from several host threads or handles at
 *     once) race on the array: serialise them per device.
 *   - returns after the results are in E_host and B_host. */
#define FEMPIC_PROBE_MAX_POINTS 65536
int femPIC_eval_fields_noalloc(FemPIC* h, int64_t n, const double* x_host, const int32_t* tet_host,
                               double* E_host, double* B_host);

int femPIC_get_info(const FemPIC* h, femPIC_info* info);

/* ---- impressed magnetic flux density (Section III-C, eq. conB) ------------
 * A static, externally produced B^i (e.g. magnets) enters the particle push
 * through its W2 coefficients b^i: the particles sample B0 + (b + b^i) . W2
 * while the field update sees b alone.  The coefficients come from a
 * projection of B^i given at quadrature points:
 *
 *   femPIC_impressed_points: the points at which the caller evaluates B^i.
 *     Per tet (input order) the conical-product rule of p + 3 Gauss-Legendre
 *     points per direction on the tet with its vertices sorted by node id,
 *     (p + 3)^3 points per tet, exact for polynomials of degree 2p + 3.  With
 *     xyz_host NULL only *n_points is written; otherwise *n_points must equal
 *     that count (FEMPIC_ERR_SIZE if not) and xyz_host [3 * n_points]
 *     receives the points, xyz interleaved, tet-major.
 *
 *   femPIC_set_impressed_B: B_host [3 * n_points] holds B^i at those points
 *     (T).  The load f_i = <W2_i, B^i> is integrated with the same rule.
 *     constrained = 0: the Galerkin projection [*mu^-1] b^i = f / mu0.
 *     constrained = 1: eq. conB, the same energy minimised under Gauss's
 *     magnetic law imposed against the order-p volume functions W3 (products
 *     P^_a(l0) P^_b(l1) P^_c(l2) P^_d(l3), a..d >= 1, a+b+c+d = p+3), which
 *     span the degree p-1 polynomials where div W2 lives, so div b^i = 0
 *     exactly up to the solver tolerance: the saddle-point system
 *     [[*mu^-1], [~div]^T; [~div], 0] is solved on the device by CG on its
 *     Schur complement (preconditioned by per-tet inverses) around inner CG
 *     solves of [*mu^-1] (block-Jacobi by face and interior DOF groups);
 *     tolerances: ||[~div] b|| reduced by opts.cg_rtol from the Galerkin
 *     projection's, but not below 100 eps || |[~div]| |b_Galerkin| || (the
 *     rounding floor of its terms; no outer iteration if the Galerkin
 *     projection is already there: a field the space reproduces), inner
 *     0.01 cg_rtol.
 *     B_host NULL (n_points 0) clears b^i.  The result replaces any earlier
 *     b^i (readable and settable as FEMPIC_B_IMPRESSED).  stats_out
 *     (nullable) receives the iteration counts, timings and the relative
 *     constraint residual.  Synchronous; allocates its work
 *     space for the call (a few times N2 doubles, the point values and the
 *     W3 operators) and frees it before returning.  Errors: FEMPIC_ERR_SIZE
 *     (point count), FEMPIC_ERR_CG (a solve hit its cap), FEMPIC_ERR_CUDA. */
typedef struct {
  int32_t outer_iterations; /* CG iterations on the Schur complement (0 if unconstrained) */
  int32_t inner_iterations; /* CG iterations of all [*mu^-1] solves                     */
  double div_residual;      /* ||[~div] b^i|| / || |[~div]| |b^i| || (entrywise absolute
                               values: the size of the terms whose sum is [~div] b^i)  */
  double host_ms;           /* host time of the W3 operators and preconditioners        */
  double device_ms;         /* device time from the load to the last kernel (CUDA events,
                               idle gaps at the host's convergence reads included)      */
  double inner_ms;          /* device time of the inner iterations alone (events around
                               each chunk of iterations)                                */
  double bytes_per_inner_iteration; /* algorithmic: 12 (nnz(M2) + nnz(Bm)) + 8 (N2 + 1)
                               + 104 N2 (CSR values and columns, row pointers, and the
                               products' and updates' vector passes)                    */
} femPIC_projection;
int femPIC_impressed_points(FemPIC* h, double* xyz_host, int64_t* n_points);
int femPIC_set_impressed_B(FemPIC* h, const double* B_host, int64_t n_points, int32_t constrained,
                           femPIC_projection* stats_out);

/* Device time of the work of the last femPIC_step / femPIC_sync, measured with
 * CUDA events on the handle's stream, summed over its steps.  Fills up to n
 * of: [0] particle loop ms (sort + gather/push/walk/deposit/charge),
 * [1] field update ms (right-hand side + CG + b update), [2] kernel launches
 * of the call, [3] sort ms, [4] particle kernel ms, [5] right-hand side ms,
 * [6] CG ms, [7] b update ms, [8] CG iterations (sum over the steps). */
int femPIC_last_timing(const FemPIC* h, double* times, int32_t n);

void femPIC_destroy(FemPIC* h);
const char* femPIC_last_error(const FemPIC* h);

/* ---- batching: many independent instances advanced together -------------
 * The paper runs one simulation at a time; this is a systems extension for
 * many small, uneven instances on one GPU.  A batch groups created handles
 * (FEMPIC_FP64 or FEMPIC_MIXED, trapezoid scheme, order 1 or 2, Boris push,
 * one species, at most 2^20 tets each, one device).  femPIC_batch_step advances every member by n_steps steps of its
 * own dt (dt_host[i]) with one launch per kernel for all members: a batched
 * counting sort, one persistent gather/push/walk/deposit kernel, batched
 * right-hand side and b update, and one cooperative block-diagonal PCG in
 * which each member owns a range of CTAs, its own reductions and its own
 * convergence test.  The step's launch sequence is captured once in a CUDA
 * graph and replayed (plain launches if capture is refused).  Each member's
 * result is the same as stepping it alone, up to the order of floating-point
 * atomic sums.  Between batch calls the members can be read (femPIC_get) and
 * stepped alone; the batch does not own them (destroy it before them).
 * femPIC_batch_step returns the first member error (message in
 * femPIC_batch_last_error). */
typedef struct FemPICBatch FemPICBatch;
int femPIC_batch_create(FemPIC* const* members, int32_t n, FemPICBatch** out);
int femPIC_batch_step(FemPICBatch* b, const double* dt_host, int32_t n_steps);
/* times: [0] device ms of the last femPIC_batch_step call, [1] launches per
 * step, [2] 1 if the CUDA graph was used, [3] CTAs of the batched CG. */
int femPIC_batch_timing(const FemPICBatch* b, double* times, int32_t n);
/* Autotuner of the batch's launch shapes: advances every member by
 * steps_per_candidate real steps per tuning round (results differ from
 * untuned steps only in the order of floating-point atomic sums), timing the
 * batched particle kernel and the batched CG with CUDA events under each
 * candidate: particle kernel CTAs of 128 or 256 threads (= particles per work
 * block), 1 .. max co-resident CTAs per SM or one CTA per work block; CG
 * CTAs per SM from 1 (as long as every member gets one) to the co-resident
 * maximum.  Rounds = the larger candidate count (the shorter list cycles);
 * the fastest mean of each kernel is kept, and the next femPIC_batch_step
 * captures its CUDA graph with it.  dt_host as femPIC_batch_step.  out
 * (nullable) receives the choice, the candidate counts, the steps taken and
 * the kernels' mean device ms per step chosen and at the creation-time
 * default (256 threads, max co-resident CTAs; CG at its co-resident maximum). */
typedef struct {
  int32_t particle_block, particle_grid, cg_ctas_per_sm;
  int32_t particle_candidates, cg_candidates, steps;
  double particle_ms, cg_ms;                 /* chosen, mean per step          */
  double particle_ms_default, cg_ms_default; /* creation-time shapes           */
} femPIC_batch_tuning;
int femPIC_batch_autotune(FemPICBatch* b, const double* dt_host, int32_t steps_per_candidate,
                          femPIC_batch_tuning* out);
void femPIC_batch_destroy(FemPICBatch* b);
const char* femPIC_batch_last_error(const FemPICBatch* b);

/* ---- measurement: arithmetic throughput of the device --------------------
 * Not part of the method: the denominator of the arithmetic roofline of the
 * particle kernel, whose walk and deposit are FP64 by design (charge
 * conservation to 1e-12) on a part with a narrow FP64 pipe.  Runs one kernel
 * of independent chains on every SM of `device` (about 0.1 s after a warm-up
 * launch) and returns the operations per second of the whole device in
 * *ops_per_second: FEMPIC_ALU_FP64_FMA and FEMPIC_ALU_FP32_FMA count one fused
 * multiply-add as one operation (two flops), FEMPIC_ALU_FP64_DIV counts one
 * correctly rounded FP64 division.  Allocates 64 bytes of device memory for the
 * call.  Returns FEMPIC_ERR_ARG for an unknown kind or a NULL pointer,
 * FEMPIC_ERR_CUDA if the device or the launch fails. */
enum { FEMPIC_ALU_FP64_FMA = 0, FEMPIC_ALU_FP32_FMA = 1, FEMPIC_ALU_FP64_DIV = 2 };
int femPIC_measure_alu(int32_t device, int32_t kind, double* ops_per_second);

#ifdef __cplusplus
}
#endif

#endif /* FEMPIC_H */
