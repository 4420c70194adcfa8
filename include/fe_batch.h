/*
 * fe_batch.h -- many small nonlinear solves in one kernel launch.
 *
 * One CTA solves one request (a mesh created by fe_mesh_create, its load
 * already set by fe_set_load, a method, a tolerance and options) from its
 * first residual to convergence, with the solvers of nl_solve (arxiv
 * 2203.05610, Section "Numerical solvers": NK, iNK with the Eisenstat-Walker
 * forcing, B and iB with the L-BFGS two-loop; the options of Appendix A),
 * so that a batch of small solves costs one launch instead of thousands of
 * launches and host round trips.  Results are independent of the batch: a
 * request solved alone and in a batch gives bit-identical results (CTA
 * reductions in a fixed order).  They agree with nl_solve to rounding (the
 * reductions differ in order).  The batching itself has no counterpart in
 * the paper.
 *
 * Supported requests (fe_batch_supported): displacement form (no pressure
 * space), no follower faces, inertia off, nodal block-Jacobi (pc_type 0),
 * FP64 or mixed FP32 precision, 1 <= ksp_restart <= 100, lbfgs_m <=
 * FE_BATCH_HIST, no Jacobian lagging, re-assembly or adaptive iB, at most
 * 64 element colours, and explicit options (opts != NULL).
 *
 * Errors follow fe.h: 0 = FE_OK, < 0 = FE_ERR_*, message in fe_last_error().
 */
#ifndef FE_BATCH_H
#define FE_BATCH_H

#include "fe.h"

#ifdef __cplusplus
extern "C" {
#endif

#define FE_BATCH_HIST 64

typedef struct {
  int32_t status;       /* nl_solve's return value for this request */
  int32_t nit;          /* nonlinear iterations */
  int32_t assemblies;   /* tangent assemblies */
  int32_t hist_len;     /* valid entries of the histories */
  int64_t lit_total;    /* Krylov iterations */
  double r0, rfinal;    /* ||R(d_0)||, final ||R|| */
  double res_hist[FE_BATCH_HIST];  /* ||R_k|| */
  int32_t lit_hist[FE_BATCH_HIST]; /* Krylov iterations of iteration k */
  double eta_hist[FE_BATCH_HIST];  /* forcing term of iteration k */
} fe_batch_out;

/* 1 when nl_solve(m, method, ..., opts) can run in a batch, else 0. */
int fe_batch_supported(fe_mesh m, int method, const nl_opts* opts);

/* Solve nreq requests with `threads` threads per CTA (128 or 256): one
 * launch per (order, precision) present, in order of first appearance.
 * meshes[i]: request i's mesh (all on one device); methods/tols/max_its/
 * opts[i] as for nl_solve (opts required); the result does not depend on
 * `threads` (the CTA reductions use a fixed set of 256 virtual lanes);
 * d[i]: device [ndof] initial guess, overwritten by the solution (prescribed
 * values written first when opts[i].apply_dirichlet).  out: host
 * [nreq].  Each launch runs on its first mesh's stream; the call returns
 * when every request is done;
 * workspace is allocated for the call and freed before it returns.
 * FE_ERR_ARG for an unsupported or inconsistent request (nothing runs). */
int fe_batch_solve(int nreq, fe_mesh* meshes, const int* methods, const double* tols, const int* max_its,
                   const nl_opts* opts, double** d, int threads, fe_batch_out* out);

#ifdef __cplusplus
}
#endif
#endif /* FE_BATCH_H */
