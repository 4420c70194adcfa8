/*
 * fe.h -- C ABI of the GB300 nonlinear-elasticity solver library (libfe.so).
 *
 * The library solves the quasi-static hyperelastic problem of the paper
 * (arxiv 2203.05610, Section "The hyperelasticity problem"): find the
 * displacement d with R(d) = f - div P(F) = 0, F = I + grad d, P = dPsi/dF,
 * with Dirichlet data d = d_D and Neumann data P n = t, on P1 or P2
 * tetrahedra (and a P1 pressure for the Taylor-Hood u-p form).  It provides
 * the four nonlinear solvers the paper compares (Section "Numerical solvers"
 * and Appendix A): Newton-Krylov (NK), inexact Newton-Krylov with
 * Eisenstat-Walker forcing (iNK), BFGS-preonly (B) and inexact BFGS (iB).
 *
 * Conventions for every call:
 *  - All functions return int: 0 = FE_OK, < 0 = API error (FE_ERR_*),
 *    > 0 = solver outcome (NL_*, only from nl_solve).  A message for the
 *    last error of the calling thread is returned by fe_last_error().
 *  - "device" pointers are CUDA device addresses on the mesh's device;
 *    "host" pointers are ordinary host memory.  The caller owns every
 *    buffer it passes; the library never keeps a caller pointer after the
 *    call returns.  The library owns everything reachable from an fe_mesh
 *    (mesh, pattern, tangent, solver workspace) and frees it in
 *    fe_mesh_destroy.
 *  - Vectors of unknowns have length ndof = 3*nn (+ np for the u-p form),
 *    laid out node-major: u[3*a + c] for node a, component c, followed by
 *    the np pressure values.  Nodes 0..nv-1 are the vertices; for P2 the
 *    edge nodes follow, numbered by the ascending (min, max) vertex pair of
 *    their edge.  Local node order in an element is v0..v3 then the edges
 *    01, 02, 03, 12, 13, 23.
 *  - Calls are stream-ordered on the stream given at fe_mesh_create and are
 *    synchronous with respect to the host unless stated otherwise.
 *  - Kernels never trap.  A device-side check that fails (bounds, a bounded
 *    wait that ran out) sets an error word that the host reads after the
 *    launch, and the call returns FE_ERR_DEVICE_FLAG or FE_ERR_TIMEOUT.
 */
#ifndef FE_H
#define FE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FE_OK 0
#define FE_ERR_ARG (-1)          /* invalid argument (message says which) */
#define FE_ERR_OOM (-2)          /* device or host allocation failed */
#define FE_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define FE_ERR_TIMEOUT (-4)      /* a bounded device wait ran out */
#define FE_ERR_DEVICE_FLAG (-5)  /* a device-side check failed */
#define FE_ERR_STATE (-6)        /* call out of order (e.g. no tangent yet) */
#define NL_DIVERGED 1            /* ||R|| > dtol*||R0|| */
#define NL_MAX_IT 2              /* max_it nonlinear iterations without convergence */
#define NL_NONFINITE 3           /* a residual norm became NaN or Inf */
#define KSP_BREAKDOWN 4          /* the Krylov solver broke down (non-finite) */

/* ---- enums ------------------------------------------------------------- */
typedef enum { NL_NK = 0, NL_INK = 1, NL_B = 2, NL_IB = 3 } nl_method;
typedef enum {
  FE_PREC_FP64 = 0,       /* tangent, SpMV, preconditioner in FP64 */
  FE_PREC_MIXED_FP32 = 1, /* tangent assembled and stored in FP32; the Krylov
                             SpMV and preconditioner in FP32; Arnoldi,
                             residual, update and BFGS products stay FP64.
                             GMRES's restart residual b - K x and iNK's
                             linear residual use the stored values with FP64
                             vectors and accumulation, and a residual
                             estimate at the target is confirmed on that
                             residual (restarted GMRES as iterative
                             refinement), so Krylov tolerances are met as
                             in FP64 */
  FE_PREC_MIXED_BF16 = 2  /* as MIXED_FP32 with BF16 tangent storage */
} fe_precision;
typedef enum {
  FE_MAT_COOK_NH = 0,  /* Psi = mu/2 (tr(Fbar^T Fbar) - 3) + c_vol (J^2 - 1 - 2 ln J),
                          Fbar = J^{-1/3} F, mu = E/(2(1+nu)), lambda = 2 mu nu/(1-2nu),
                          kappa = lambda + 2mu/3; c_vol = kappa/4 (vol_literal = 0,
                          small-strain consistent reading) or kappa (vol_literal = 1,
                          as printed).  Paper: Cook test, Psi_Cook. */
  FE_MAT_TH_NH = 1,    /* Psi = mu/2 (tr(F^T F) - 3) - mu ln J - p (J - 1); with
                          pressure_order = 1 this is the Taylor-Hood u-p form
                          (twist test stand-in).  Without pressure, p = 0. */
  FE_MAT_GUCCIONE = 2, /* Psi = C/2 (e^Q - 1) + kappa/2 (J - 1) ln J, Q in the fibre
                          frame with b_ff = bf, b_ss = b_nn = b_sn = bt,
                          b_fs = b_fn = bfs; plus active stress
                          P_act = gamma(t) (F f) x f / |F f|,
                          gamma(t) = Ta_peak max(sin(2 pi t / period), 0).
                          Paper: Heartbeat test. */
  FE_MAT_POLYCONVEX = 3 /* Psi = alpha_p (F:F - 3) + beta_p (cof F : cof F - 3)
                          - c_log ln J - p (J - 1), cof F = J F^{-T}; the paper's
                          twist potential (Section "Test problems", Psi_Twist, with
                          c_log = 4 beta_s + 2 alpha_s and its "log(F)" read as
                          ln det F).  With pressure_order = 1 the u-p form. */
} fe_material_kind;
typedef enum {
  FE_FACE_TRACTION = 0, /* dead traction t = load * data[0..2] per unit reference area */
  FE_FACE_PRESSURE = 1, /* dead pressure: t = -load * data[0] * N (reference outward normal) */
  FE_FACE_ROBIN = 2,    /* springs: t = -(kperp N x N + kpar (I - N x N)) d,
                           data = {kperp, kpar, 0}; not scaled by load */
  FE_FACE_FOLLOWER = 3, /* follower pressure: t da = -load * data[0] * n da on the
                           DEFORMED face (n its outward normal), i.e. nodal forces
                           load * data[0] * int N_a (x_xi x x_eta) dxi deta over the
                           reference triangle; its tangent is not symmetric and it
                           has no potential (fe_energy leaves it out).  The
                           pressure on the moving endocardium of the paper's
                           heartbeat test. */
  FE_FACE_DASHPOT = 4,  /* dashpots of the epicardial Robin condition (Eq. "bc epi",
                           the C terms): t = -(cperp N x N + cpar (I - N x N)) v,
                           v the velocity of the Newmark step, data = {cperp, cpar, 0};
                           inactive until fe_set_dynamics turns inertia on */
  FE_FACE_TRACTION_DEFORMED = 5 /* traction load * data[0..2] per unit DEFORMED area (the
                           Cook load "in the deformed configuration"): nodal forces
                           load * t int N_a |x_xi x x_eta| dxi deta; not symmetric, no
                           potential (fe_energy leaves it out) */
} fe_face_kind;

/* ---- mesh description (host data, copied by fe_mesh_create) ------------ */
typedef struct {
  int32_t kind;        /* fe_material_kind */
  int32_t vol_literal; /* COOK_NH only, see above */
  double E, nu;        /* COOK_NH */
  double mu;           /* TH_NH */
  double C, bf, bt, bfs, kappa, Ta_peak, period; /* GUCCIONE */
  double alpha_p, beta_p, c_log;                 /* POLYCONVEX */
} fe_material;

typedef struct {
  uint32_t comp_mask;    /* bit c set: component c of d is prescribed */
  double center[3];      /* a point on the rotation axis (axis parallel to z) */
  double angle;          /* rotation angle in radians at load factor 1 */
  double translation[3]; /* translation at load factor 1 */
} fe_dirichlet_group;    /* prescribed d(X) = load-scaled rigid motion of X minus X */

typedef struct {
  int32_t order;          /* displacement order: 1 (P1) or 2 (P2) */
  int32_t pressure_order; /* 0: displacement only; 1: P1 pressure (vertex values, Taylor-Hood);
                             2: P0 pressure (one constant per element, the paper's P2-P0
                             twist pair); 1 and 2 need order 2 and TH_NH or POLYCONVEX */
  int32_t nv;             /* number of vertices */
  int32_t ne;             /* number of tetrahedra */
  const double* coords;   /* host [nv][3] vertex coordinates */
  const int32_t* tets;    /* host [ne][4] vertex ids, positively oriented */
  const uint8_t* dir_group; /* host [nv]: 0 = free, g = member of groups[g-1];
                             a P2 edge node belongs to group g when both of its
                             end vertices do */
  int32_t ngroups;
  const fe_dirichlet_group* groups; /* host [ngroups] */
  int32_t nf;                /* boundary faces carrying loads or springs */
  const int32_t* faces;      /* host [nf][3] vertex ids, (x1-x0)x(x2-x0) outward */
  const int32_t* face_kind;  /* host [nf] fe_face_kind */
  const double* face_data;   /* host [nf][3] */
  fe_material material;
  const double* fibers;      /* host [ne][9] rows f, s, n (GUCCIONE), else NULL */
  int32_t device;            /* CUDA device ordinal */
  void* stream;              /* cudaStream_t; NULL = legacy default stream */
} fe_mesh_desc;

typedef struct fe_mesh_s* fe_mesh; /* opaque, library-owned */

typedef struct {
  int32_t order, pressure_order;
  int32_t nv, ne, nn;  /* vertices, elements, displacement nodes */
  int32_t np;          /* pressure unknowns (nv for P1 pressure, else 0) */
  int64_t ndof;        /* 3*nn + np */
  int32_t nen;         /* nodes per element: 4 or 10 */
  int64_t nnzb;        /* 3x3 blocks in the displacement BCSR pattern */
  int64_t nnz_up;      /* 3x1 blocks of the u-p coupling (0 without pressure) */
  int32_t ncolors;     /* colours of the element colouring */
  int64_t device_bytes;/* device memory held by the mesh and its workspace */
} fe_mesh_info;

/* Create a mesh: copies the description to the device, builds the P2 edge
 * nodes, the element colouring (first-fit greedy in descending
 * splitmix64(element id) priority, ties by id) and the block-CSR pattern
 * (one 3x3 block per pair of nodes that share an element, columns
 * ascending).  Paper: FE discretisation of the quasi-static problem
 * (Sections "The hyperelasticity problem" and "Test problems").
 * Returns FE_ERR_ARG on inconsistent sizes or ids out of range. */
int fe_mesh_create(const fe_mesh_desc* desc, fe_mesh* out);
int fe_mesh_destroy(fe_mesh m);
int fe_mesh_get_info(fe_mesh m, fe_mesh_info* out);

/* Copy the mesh topology to host buffers (each may be NULL):
 * conn [ne][nen], colors [ne], row_ptr [nn+1], col [nnzb],
 * node_coords [nn][3]. */
int fe_mesh_get_topology(fe_mesh m, int32_t* conn, int32_t* colors,
                         int32_t* row_ptr, int32_t* col, double* node_coords);

/* Set the load factor (scales tractions, pressures and prescribed motions)
 * and the time (activation gamma(t) of the GUCCIONE material).  Paper:
 * quasi-static problem with time-dependent data; load stepping of the
 * tests. */
int fe_set_load(fe_mesh m, double load, double time);

/* ---- elastodynamics: Newmark average acceleration ------------------------
 * The momentum equation with its inertia term (Section "Problem
 * formulation", Eq. "momentum strong"; the paper keeps unit density and
 * names no time integrator).  Readings: density rho per unit reference
 * volume, consistent mass M = rho int N_a N_b I dV, Newmark's average
 * acceleration rule (beta = 1/4, gamma = 1/2).  With the state d_n, v_n,
 * a_n, a time step is one nl_solve of
 *   R(d) + M a(d) + C v(d) = 0,  a(d) = 4/dt^2 (d - dhat),  v(d) = 2/dt (d - dtil),
 *   dhat = d_n + dt v_n + dt^2/4 a_n,  dtil = d_n + dt/2 v_n,
 * C the dashpots of the FE_FACE_DASHPOT faces.  The tangent gains
 * 4/dt^2 M + 2/dt C, fe_energy the step functional
 * 2/dt^2 (d - dhat)^T M (d - dhat) + 1/dt (d - dtil)^T C (d - dtil).
 * Prescribed components keep R = 0 as in the static problem.
 *
 * fe_set_dynamics: rho > 0 and dt > 0 turn inertia on with the state at
 *   rest (d_n = v_n = a_n = 0); rho <= 0 or dt <= 0 turns it off.
 *   FE_ERR_ARG for non-finite values.  The first call allocates 6 vectors
 *   of 3 nn doubles on the mesh's device (kept until fe_mesh_destroy).
 * fe_dynamics_set: d_n, v_n, a_n from device arrays of 3 nn doubles (node
 *   major, the displacement part of a solution vector); NULL = zero.
 * fe_dynamics_advance: after a converged step with solution d (device,
 *   [ndof], its displacement part read) moves the state to a_{n+1} = a(d),
 *   v_{n+1} = v(d), d_{n+1} = d.
 * fe_dynamics_get: copies v_n and a_n into device arrays of 3 nn doubles
 *   (NULL skips one).
 * The last three return FE_ERR_STATE while dynamics is off. */
int fe_set_dynamics(fe_mesh m, double rho, double dt);
int fe_dynamics_set(fe_mesh m, const double* d, const double* v, const double* a);
int fe_dynamics_advance(fe_mesh m, const double* d);
int fe_dynamics_get(fe_mesh m, double* v, double* a);

/* Write the prescribed Dirichlet values of the current load into d
 * (device, [ndof]); other entries are left unchanged. */
int fe_apply_dirichlet(fe_mesh m, double* d);

/* Residual R(d) = internal - external forces (the gradient of Pi), with
 * R = 0 at prescribed components.  d, r: device [ndof] FP64.  norm_out
 * (host, nullable) receives ||R||_2 (paper, the l2 norm of the EW
 * definition).  Paper: residual form R(d) = f - div P (sign: gradient of
 * the energy, Eq. "minimization"). */
int fe_assemble_residual(fe_mesh m, const double* d, double* r, double* norm_out);

/* Energy Pi(d) = int Psi(F) - external work + spring energy (host out).
 * Paper: Eq. "minimization". */
int fe_energy(fe_mesh m, const double* d, double* pi_out);

/* Assemble the consistent tangent dR/dd at d (device [ndof]) into the
 * library-owned block-CSR matrix in the given fe_precision, and set up the
 * preconditioner (nodal block-Jacobi: inverse 3x3 diagonal blocks; for the
 * u-p form the lower Schur preconditioner of Appendix B with the SIMPLE
 * approximation S = -B2 diag(A)^{-1} B1 and point Jacobi on S).
 * Prescribed components get zero rows and columns and a unit diagonal.
 * Paper: Eq. "newton" (tangent problem). */
int fe_assemble_tangent(fe_mesh m, const double* d, int precision);

/* Copy the assembled tangent to host as FP64 (any of the pointers may be
 * NULL): val [nnzb][9] row-major 3x3 blocks, bup [nnz_up][3] (u-p
 * coupling, u rows), dinv [nn][9] (inverse diagonal blocks). */
int fe_tangent_copy(fe_mesh m, double* val, double* bup, double* dinv);

/* y = K x with the assembled tangent (device [ndof] FP64 in and out). */
int fe_spmv(fe_mesh m, const double* x, double* y);

/* y = M^{-1} x with the preconditioner of the assembled tangent. */
int fe_pc_apply(fe_mesh m, const double* x, double* y);

/* y = K x like fe_spmv, without allocating device memory during the call.
 * The paper has no counterpart.  For callers that cannot call cudaMalloc
 * while they run: a serving loop whose memory pool already owns the free
 * device memory, a latency-bound loop that cannot afford the device-wide
 * synchronisation an allocation may cause, or a host thread that another
 * allocator (PyTorch's caching allocator, a custom arena) must remain the
 * only owner for.  fe_spmv converts x to the SpMV's input precision in a
 * buffer it allocates on first use; this call stages that input in a fixed
 * device array of the library instead: 2^20 FP64 entries (8 MiB), held on
 * every GPU where a mesh was created (with eager module loading, on every
 * GPU the process uses) until the process exits.  Limits and rules:
 *  - ndof must be at most 1,048,576; larger meshes get FE_ERR_ARG.
 *  - fe_mesh_create brings the array into device memory on the mesh's
 *    device (CUDA loads it lazily, on first use), looks its address up and
 *    loads the kernels this call launches, so no call of this function
 *    loads or allocates anything; a mesh that could not do so is not
 *    created (FE_ERR_CUDA).
 *  - All calls share the array and each overwrites it: calls that overlap
 *    on the GPU (other streams or threads) race; serialise them.
 *  - The tangent must be assembled (fe_assemble_tangent); mesh and tangent
 *    memory are allocated by those earlier calls, not by this one.
 * x, y: device [ndof] FP64.  Returns FE_ERR_STATE without a tangent. */
int fe_spmv_noalloc(fe_mesh m, const double* x, double* y);

/* ---- solvers ----------------------------------------------------------- */
typedef struct {
  int32_t precision;   /* fe_precision (default FE_PREC_FP64) */
  double ksp_rtol;     /* NK 1e-6, iB 1e-2 (Appendix A); < 0 = default */
  double ksp_atol;     /* NK 1e-10, iNK/iB 1e-14; < 0 = default */
  double ew_rtol0;     /* iNK first forcing term, default 0.1 */
  double ew_rtolmax;   /* iNK forcing cap, default 0.1 */
  int32_t ksp_restart; /* GMRES restart length, default 500 */
  int32_t ksp_max_it;  /* GMRES iteration cap per solve, default 10000 */
  int32_t lbfgs_m;     /* stored secant pairs, default 50 */
  double dtol;         /* divergence: ||R|| > dtol*||R0||, default 1e4 */
  int32_t apply_dirichlet; /* 1 (default): write prescribed values into d first */
  int32_t orthog;      /* Arnoldi orthogonalisation: 0 (default) the sequential modified
                          Gram-Schmidt sweep the paper uses (j+2 grid reductions per step);
                          1 the same MGS projections in compact-WY form (2 grid
                          reductions per step, ~1.5x the FP64 work, restart <= 128);
                          2 MGS over blocks of 8 basis vectors, the block's
                          coefficients from its cached Gram entries (ceil((j+1)/8)+1
                          grid reductions per step, same FP64 work; vectors too long
                          for one co-resident grid take the sequential sweep) */
  int32_t jac_lag;     /* NK/iNK: assemble the tangent (and its block-Jacobi) only at
                          iterations 1, 1+L, 1+2L, ... and solve with the last one in
                          between (Jacobian lagging, named as an extension in the
                          paper's conclusions); 1 (default, 0 means 1) = every iteration */
  int32_t hess_reassemble; /* B/iB: every R iterations re-assemble the tangent at the
                          current d (new H0) and restart the L-BFGS memory (the
                          conclusions' occasional Jacobian re-assembly for BFGS);
                          0 (default) = only at d_0 */
  int32_t ib_adaptive; /* iB: 1 = adaptive H0 tolerance of Eisenstat-Walker type (the
                          alternative to the fixed 1e-2 that the paper leaves for future
                          work), reading: EW choice 2, eta_1 = ksp_rtol,
                          eta_k = min(ew_rtolmax, max(0.9 (|R_{k-1}|/|R_{k-2}|)^a,
                          0.9 eta_{k-1}^a if that exceeds 0.1)), a = (1+sqrt 5)/2;
                          0 (default) = fixed ksp_rtol */
  int32_t pc_type;     /* preconditioner of the displacement block (GMRES and the B/iB H0):
                          0 (default) nodal block-Jacobi; 1 algebraic multigrid, one
                          smoothed-aggregation V-cycle on the nodal blocks (the class of
                          the paper's BoomerAMG with block size 3, Appendix A); 2 that
                          V-cycle with a BF16 fine-level smoother (mixed FP32); see
                          fe_set_pc */
} nl_opts;

#define NL_HIST 1024
typedef struct {
  int32_t status;      /* same as the return value of nl_solve */
  int32_t nit;         /* nonlinear iterations */
  int64_t lit_total;   /* Krylov iterations summed over the solve */
  int32_t assemblies;  /* tangent assemblies */
  double r0, rfinal;   /* ||R(d_0)||, ||R(d_final)|| */
  double time_s;       /* wall time of the solve */
  int32_t hist_len;
  double res_hist[NL_HIST]; /* ||R_k||, k = 0..nit */
  int32_t lit_hist[NL_HIST];/* Krylov iterations of iteration k */
  double eta_hist[NL_HIST]; /* relative Krylov tolerance used at iteration k */
  double lres_hist[NL_HIST];/* NK/iNK: linear residual ||R_{k-1} + K_{k-1} delta_k|| of
                               iteration k (the Eisenstat-Walker forcing term's second
                               norm); 0 for B/iB */
} nl_stats;

/* Fill opts with the defaults of the given method (Appendix A options). */
int nl_opts_default(nl_method method, nl_opts* opts);

/* Solve R(d) = 0 from the initial guess in d (device [ndof], overwritten
 * with the last iterate) with the given method, until
 * ||R_k|| <= tol*||R_0|| or max_it iterations.  Line search "basic" (full
 * step).  NK/iNK: Eq. "newton" with GMRES (right block-Jacobi / Schur
 * preconditioning, MGS Arnoldi, restarted every ksp_restart), iNK forcing
 * by Eisenstat-Walker choice 1 with the safeguard; B/iB: limited-memory
 * BFGS two-loop (Nocedal 1980) with H0 = preconditioner (B) or GMRES at
 * ksp_rtol (iB) on the tangent assembled once at d_0.  opts may be NULL
 * (method defaults); stats may be NULL.  Returns 0 on convergence or an
 * NL_* outcome (> 0) or an FE_ERR_* (< 0). */
int nl_solve(fe_mesh m, int method, double tol, int max_it, double* d,
             const nl_opts* opts, nl_stats* stats);

/* Solve K x = b with GMRES on the assembled tangent (device [ndof] FP64;
 * x holds the initial guess and is overwritten); orthog as in nl_opts.
 * iters/res_out (host, nullable) receive the iteration count and the final
 * residual estimate.  Paper: GMRES with modified Gram-Schmidt (Section
 * "Test problems and solvers details"), right preconditioning (reading). */
int fe_gmres(fe_mesh m, const double* b, double* x, double rtol, double atol,
             int restart, int max_it, int orthog, int* iters, double* res_out);

/* One L-BFGS two-loop application z = H q over k stored pairs (device
 * pointers: S, Y [k][ndof] row-major oldest first, rho [k], q, z [ndof]),
 * with H0 = the preconditioner of the assembled tangent (h0 = 0) or
 * identity (h0 = 1).  Paper: BFGS update formula and its two-loop
 * recursion (Section "Numerical solvers", BFGS method). */
int fe_lbfgs_apply(fe_mesh m, const double* S, const double* Y, const double* rho,
                   int k, const double* q, double* z, int h0);

/* ---- instrumentation ----------------------------------------------------
 * Measurement support (no counterpart in the paper).  Every kernel launch
 * of the library is counted per class; with timing on, each launch is also
 * bracketed by CUDA events on the mesh's stream and credited with the
 * algorithmic bytes it must move (inputs read once, outputs written once)
 * and the floating-point operations it must perform. */
#define FE_PROF_CLASSES 8
enum {
  FE_PROF_RESIDUAL = 0, /* element residual + node gather */
  FE_PROF_TANGENT = 1,  /* coloured tangent assembly, springs, diagonal inverse */
  FE_PROF_SPMV = 2,     /* block-CSR SpMV */
  FE_PROF_PC = 3,       /* block-Jacobi / Schur preconditioner, AMG V-cycle (one launch of its graph) */
  FE_PROF_ARNOLDI = 4,  /* persistent MGS Arnoldi step */
  FE_PROF_TWOLOOP = 5,  /* L-BFGS two-loop recursion */
  FE_PROF_VECTOR = 6,   /* dots, axpys, copies, GMRES update */
  FE_PROF_OTHER = 7     /* mesh set-up and the AMG hierarchy's numbers after each assembly */
};
typedef struct {
  int64_t launches[FE_PROF_CLASSES]; /* kernel launches since the last reset */
  int64_t timed[FE_PROF_CLASSES];    /* launches timed with events */
  double ms[FE_PROF_CLASSES];        /* summed event time of the timed launches */
  double bytes[FE_PROF_CLASSES];     /* summed algorithmic bytes of the timed launches */
  double flops[FE_PROF_CLASSES];     /* summed algorithmic floating-point operations (FMA = 2) */
} fe_profile_info;
/* Zero the counters; timing = 1 also times every launch with CUDA events. */
int fe_profile_reset(fe_mesh m, int timing);
/* Synchronise the stream and read the counters (host out). */
int fe_profile_read(fe_mesh m, fe_profile_info* out);

/* Preconditioner of the displacement block for the following tangent
 * assemblies (and, with a tangent assembled, set up now): 0 nodal
 * block-Jacobi (default), 1 algebraic multigrid.  The paper preconditions
 * with BoomerAMG on blocks of 3 (Section "Test problems and solvers
 * details", Appendix A); this library's AMG is a smoothed-aggregation
 * V-cycle: aggregates from a greedy distance-2 independent set of the block
 * graph, the six rigid motions as near null space (tentative prolongator by
 * per-aggregate QR), P = (I - 4/(3 rho) D^-1 A) T, Galerkin coarse
 * operators, degree-2 Chebyshev smoothing, an exact coarsest solve.  Its
 * structure is built once per mesh (host), its numbers after every tangent
 * assembly (device, FP64 for an FP64 tangent, FP32 for the mixed forms; the
 * V-cycle runs in the tangent's precision).  For the u-p form it replaces
 * the block-Jacobi of the displacement block inside the lower Schur
 * preconditioner.  2: the same V-cycle whose fine-level smoother reads a
 * BF16 copy of the FP32 tangent (made after each assembly; the V-cycle's
 * dominant passes then move 22 instead of 40 bytes per block, the coarse
 * levels, transfers and vectors stay FP32; the GMRES operator stays the
 * FP32 tangent, so the solution's accuracy is unchanged); with an FP64 or
 * BF16 tangent 2 acts as 1.  FE_ERR_ARG for pc_type outside {0, 1, 2}. */
int fe_set_pc(fe_mesh m, int pc_type);

/* The AMG hierarchy of the last assembly, for inspection and tests:
 * fe_amg_levels returns the number of levels (0 without a hierarchy);
 * fe_amg_get_level copies level `level` to host buffers, each nullable:
 * info [5] = n (block rows), b (components per node: 3 at level 0, 6 below),
 * nnz(A_l), nc (aggregates; 0 on the coarsest level), nnz(P_l); rho (the
 * spectral-radius estimate of D^-1 A_l); for level >= 1 the operator A_l:
 * ptr [n+1], col [nnz], val [nnz][b*b] FP64 row-major blocks (level 0 is the
 * tangent, see fe_tangent_copy); absent [n] (bit c: component c absent);
 * agg [n] (aggregate of each node, -1 none); pptr [n+1], pcol [nnz(P_l)],
 * pval [nnz(P_l)][b*6] the smoothed prolongator in FP64. */
int fe_amg_levels(fe_mesh m);
int fe_amg_get_level(fe_mesh m, int level, int64_t* info, double* rho, int32_t* ptr, int32_t* col,
                     double* val, uint8_t* absent, int32_t* agg, int32_t* pptr, int32_t* pcol, double* pval);

/* Bounded device waits (no counterpart in the paper).  The persistent
 * kernels' grid barriers poll for a published value at most `polls` times
 * before they give up: the kernel then records a timeout in the mesh's
 * error word and ends, and the call returns FE_ERR_TIMEOUT with the mesh
 * still usable.  Default 2^26 polls (seconds); polls < 0 restores it; 0 makes
 * every wait that does not find its value at the first poll give up (how
 * the tests drive the timeout path).  Returns FE_ERR_ARG for polls >= 2^32. */
int fe_set_wait_limit(fe_mesh m, int64_t polls);

/* Thread-local message describing the last error. */
const char* fe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FE_H */
