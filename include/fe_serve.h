/*
 * fe_serve.h -- continuous-batching request loop over libfe.so solves.
 *
 * A server owns one GPU.  Clients submit nonlinear solves (a mesh
 * description, a method, tolerances, a load step) at any time; a scheduler
 * thread admits queued requests in arrival order as soon as a slot is free
 * and their estimated device footprint fits the HBM budget, and runs every
 * admitted request on its own CUDA stream, so the work of all admitted
 * requests overlaps on the device.  Small requests (fe_batch.h) are instead
 * handed to batcher threads that solve all such requests waiting at that
 * moment in one launch (one CTA per request), so requests that arrive while
 * a batch runs form the next one.  Meshes stay resident between requests
 * with the same description (fe_server_opts.mesh_cache).  Results are the same as a solve of the
 * same request alone (same kernels, same launch shapes, deterministic
 * reductions; a batched request's result does not depend on its batch).
 * Each request is one call of nl_solve (include/fe.h) or its batched form,
 * i.e. one load step of the paper's quasi-static problem (arxiv 2203.05610,
 * Section "Numerical solvers"); the serving loop itself has no counterpart
 * in the paper.
 *
 * Errors follow fe.h: 0 = FE_OK, < 0 = FE_ERR_*, message in fe_last_error().
 */
#ifndef FE_SERVE_H
#define FE_SERVE_H

#include "fe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe_server_s* fe_server;

typedef struct {
  int32_t device;      /* CUDA device ordinal */
  int64_t hbm_budget;  /* bytes admitted requests may hold together; 0 = 80% of free memory */
  int32_t max_active;  /* requests solved concurrently (slots); <= 0 means 8 */
  int64_t batch_max_dofs; /* requests up to this many unknowns that fe_batch_supported
                             accepts are solved in shared launches (fe_batch.h), one
                             launch per size class (order, precision, floor(log2
                             ndof)); 0 = 1000 (up to where one CTA solves a
                             request about as fast as the whole GPU does; a launch
                             lasts as long as its slowest request and holds its SMs
                             meanwhile), < 0 = never */
  int32_t mesh_cache;     /* 0 = a mesh whose solve ran stays resident on the device
                             (pattern, colouring, AMG structure, workspace) and the
                             next request with a byte-identical description reuses
                             it; resident meshes keep their admission charge and
                             are evicted least recently used when a request needs
                             the room; < 0 = every request builds and frees its own */
} fe_server_opts;

/* One entry of the launch-shape autotuner of the batched path: per size
 * class (order, precision, floor(log2 ndof)) the first batches try 128 and
 * 256 threads per CTA, each timed per unit of work (sum over the batch's
 * requests of ndof x (nonlinear + Krylov iterations)); later batches of the
 * class use the cheaper shape. */
typedef struct {
  int32_t order, precision, size_class; /* the class */
  int32_t threads;                      /* chosen threads per CTA (0: still trying) */
  int32_t batches[2];                   /* batches timed with 128 and 256 threads */
  double cost[2];                       /* best seconds per unit of work, 128 and 256 threads (0: none) */
} fe_tuning_entry;

typedef struct {
  const fe_mesh_desc* mesh; /* copied by serve_submit (device/stream fields ignored) */
  int32_t method;           /* nl_method */
  double tol;               /* relative residual target */
  int32_t max_it;           /* nonlinear iteration cap */
  const nl_opts* opts;      /* NULL = method defaults (copied) */
  double load, time;        /* load factor and time of the step (fe_set_load) */
  const double* d0;         /* host [ndof] initial guess, NULL = zeros (copied) */
} fe_request;

enum { FE_REQ_QUEUED = 0, FE_REQ_RUNNING = 1, FE_REQ_DONE = 2, FE_REQ_FAILED = 3 };

typedef struct {
  int32_t state;         /* FE_REQ_* */
  int32_t result;        /* nl_solve's return value (DONE), or the FE_ERR_* of a failure */
  int64_t ndof;          /* unknowns of the request's mesh (0 before admission) */
  int64_t footprint;     /* admission estimate of its device bytes */
  double t_submit, t_start, t_end; /* seconds on the server's steady clock */
  nl_stats stats;        /* filled when DONE */
  int32_t mesh_reused;   /* 1: ran on a resident mesh of an earlier request */
} fe_request_status;

/* Create a server and start its scheduler thread. */
int serve_create(const fe_server_opts* opts, fe_server* out);

/* Queue a request (non-blocking; the request and its arrays are copied).
 * id_out receives the request id.  A request whose footprint can never fit
 * the budget is failed at admission with FE_ERR_OOM. */
int serve_submit(fe_server s, const fe_request* req, int64_t* id_out);

/* Status of a request; wait = 1 blocks until it is DONE or FAILED.  d_out
 * (host [ndof], nullable) receives the solution once DONE. */
int serve_poll(fe_server s, int64_t id, int wait, fe_request_status* status, double* d_out);

/* The autotuner's table: up to cap entries into out (host); returns the
 * number of classes seen (may exceed cap). */
int serve_tuning(fe_server s, fe_tuning_entry* out, int cap);

/* Seconds on the server's steady clock (the clock of t_submit etc.). */
double serve_clock(fe_server s);

/* Wait for all requests to finish, stop the scheduler, free everything. */
int serve_destroy(fe_server s);

#ifdef __cplusplus
}
#endif
#endif /* FE_SERVE_H */
