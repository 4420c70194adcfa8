/*
 * oracle.h -- plain, slow, single-threaded FP64 CPU oracle of the
 * paper's nonlinear-elasticity solver hot path (arxiv 2203.05610).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may call this code.  It shares no code,
 * header or table with the CUDA library; both consume the same synthetic
 * inputs.  Every function follows the paper's definitions step by step
 * with plain loops, in the paper's order, so that it can be checked by eye.
 *
 * Material parameter array matp[15]:
 *   [0] kind (0 Cook neo-Hookean, 1 Taylor-Hood neo-Hookean, 2 Guccione,
 *       3 polyconvex twist potential)
 *   [1] vol_literal  [2] E  [3] nu  [4] mu  [5] C  [6] bf  [7] bt  [8] bfs
 *   [9] kappa  [10] Ta_peak  [11] period  [12] alpha_p  [13] beta_p
 *   [14] c_log = 4 beta_s + 2 alpha_s
 * Dirichlet group array groups[ngroups][8]:
 *   mask, center x, y, z, angle, translation x, y, z
 * Solver option array opts[14]:
 *   precision(ignored: FP64), ksp_rtol, ksp_atol, ew_rtol0, ew_rtolmax,
 *   ksp_restart, ksp_max_it, lbfgs_m, dtol, apply_dirichlet,
 *   jac_lag (NK/iNK: tangent assembled every jac_lag iterations, >= 1),
 *   hess_reassemble (B/iB: tangent re-assembled and memory restarted every
 *   hess_reassemble iterations, 0 = never),
 *   ib_adaptive (iB: 1 = Eisenstat-Walker choice-2 tolerance for the H0 solve),
 *   pc_type (0 nodal block-Jacobi, 1 algebraic multigrid V-cycle)
 * Stats array (6 + 5*OM_HIST doubles):
 *   status, nit, lit_total, assemblies, r0, rfinal,
 *   res_hist[OM_HIST], lit_hist[OM_HIST], eta_hist[OM_HIST],
 *   lres_hist[OM_HIST] (NK/iNK: linear residual ||R_{k-1} + K_{k-1} delta_k||
 *   of iteration k, the second norm of the Eisenstat-Walker forcing term),
 *   time_hist[OM_HIST] (seconds from the start of the solve to the end of
 *   iteration k; instrumentation for the timed CPU baseline)
 */
#ifndef ORACLE_H
#define ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

#define OM_HIST 1024

typedef struct om_mesh om_mesh;

/* pressure_order: 0 none, 1 P1 (vertex values, Taylor-Hood), 2 P0 (one
 * constant per element, the paper's P2-P0 twist pair) */
om_mesh* om_create(int order, int pressure_order, int nv, int ne, const double* coords,
                   const int* tets, const unsigned char* dir_group, int ngroups,
                   const double* groups, int nf, const int* faces, const int* face_kind,
                   const double* face_data, const double* matp, const double* fibers);
void om_destroy(om_mesh* m);
/* out: nn, np, ndof, nnzb, nnz_up, ncolors, nen */
void om_info(const om_mesh* m, long long* out);
void om_topology(const om_mesh* m, int* conn, int* colors, int* row_ptr, int* col, double* X);
void om_set_load(om_mesh* m, double load, double time);
void om_apply_dirichlet(const om_mesh* m, double* d);
double om_residual(om_mesh* m, const double* d, double* r);
double om_energy(om_mesh* m, const double* d);
void om_tangent(om_mesh* m, const double* d);
void om_tangent_copy(const om_mesh* m, double* val, double* bup, double* dinv);
void om_spmv(const om_mesh* m, const double* x, double* y);
void om_pc(const om_mesh* m, const double* x, double* y);
int om_gmres(om_mesh* m, const double* b, double* x, double rtol, double atol, int restart,
             int max_it, double* res_out);
int om_solve(om_mesh* m, int method, double tol, int max_it, double* d, const double* opts,
             double* stats);
void om_lbfgs_apply(om_mesh* m, const double* S, const double* Y, const double* rho, int k,
                    const double* q, double* z, int h0);

/* elastodynamics (Newmark average acceleration): rho > 0 and dt > 0 enable
 * it (mass and dashpot matrices assembled here, state at rest);
 * om_dynamics_set sets d_n, v_n, a_n (nullable: zero; [3 nn]); after a
 * converged step om_dynamics_advance(d) moves the state to d;
 * om_dynamics_get reads v_n, a_n.  Face kinds 3 (follower pressure, data
 * p), 4 (dashpots, data c_perp, c_par) and 5 (traction t per unit deformed
 * area, data t) join 0-2. */
void om_set_dynamics(om_mesh* m, double rho, double dt);
void om_dynamics_set(om_mesh* m, const double* d, const double* v, const double* a);
void om_dynamics_advance(om_mesh* m, const double* d);
void om_dynamics_get(const om_mesh* m, double* v, double* a);

/* preconditioner of the displacement block: 0 nodal block-Jacobi, 1 the
 * smoothed-aggregation AMG V-cycle (set up by om_tangent) */
void om_set_pc(om_mesh* m, int pc_type);
int om_amg_levels(const om_mesh* m);
/* out: n, b (components per node), nnz(A_l), nc, nnz(P_l) */
void om_amg_level_info(const om_mesh* m, int l, long long* out);
void om_amg_copy(const om_mesh* m, int l, int* ptr, int* col, double* val, unsigned char* absent, double* ns,
                 int* agg, int* pptr, int* pcol, double* pval, double* tval, double* rho, double* inv);
void om_amg_smooth(const om_mesh* m, int l, const double* b, double* x, int deg);
void om_amg_vcycle(const om_mesh* m, const double* b, double* x);

/* pointwise pieces, exposed for the pins */
void om_material(const double* matp, const double* F, const double* fib, double gamma, double p,
                 double* psi, double* P, double* A, double* dPdp);
int om_tet_rule(int order, double* lam, double* w);   /* barycentric points, weights (sum 1) */
int om_tri_rule(double* lam, double* w);              /* degree-4 triangle rule, weights sum 1 */
unsigned long long om_splitmix64(unsigned long long x);

#ifdef __cplusplus
}
#endif
#endif
