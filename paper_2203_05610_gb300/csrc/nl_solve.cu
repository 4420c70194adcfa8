// nl_solve.cu -- the four nonlinear solvers of arxiv 2203.05610 (Section
// "Numerical solvers", options of Appendix A) on the device path:
//   NK : solve K(d) delta = -R(d) with GMRES at ksp_rtol/ksp_atol (Eq. "newton")
//   iNK: as NK with the Eisenstat-Walker forcing term (choice 1 with the
//        safeguard, capped at ew_rtolmax) -- reading of the garbled formula
//   B  : L-BFGS (m pairs) with H0 = preconditioner of K(d_0), one assembly
//   iB : L-BFGS with H0 = GMRES on K(d_0) at ksp_rtol
// All four use the basic line search (full step) and the test
// ||R_k|| <= tol ||R_0||; divergence when ||R_k|| > dtol ||R_0|| or non-finite.
// The host only sequences kernels and reads one scalar per convergence test.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "fe_internal.h"

extern "C" int nl_opts_default(nl_method method, nl_opts* o) {
  if (!o) return fe_set_error("NULL opts"), FE_ERR_ARG;
  if (method < NL_NK || method > NL_IB) return fe_set_error("bad method"), FE_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->precision = FE_PREC_FP64;
  o->ksp_rtol = method == NL_NK ? 1e-6 : (method == NL_B ? 0.0 : 1e-2);
  o->ksp_atol = method == NL_NK ? 1e-10 : (method == NL_B ? 0.0 : 1e-14);
  o->ew_rtol0 = 0.1;
  o->ew_rtolmax = 0.1;
  o->ksp_restart = 500;
  o->ksp_max_it = 10000;
  o->lbfgs_m = 50;
  o->dtol = 1e4;
  o->apply_dirichlet = 1;
  o->orthog = 0;
  o->jac_lag = 1;
  o->hess_reassemble = 0;
  o->ib_adaptive = 0;
  o->pc_type = 0;
  return FE_OK;
}

// y = x_new - x_old into dst, and s = delta; returns y.s on the device slot
__global__ void k_diff(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = a[i] - b[i];
}
// delta = -z; d += delta
__global__ void k_step(int64_t n, const double* __restrict__ z, double* __restrict__ delta, double* __restrict__ d) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double v = -z[i];
    delta[i] = v;
    d[i] += v;
  }
}

static int residual_norm(fe_mesh m, const double* d, double* r, double* out) {
  FE_TRY(fe_residual_dev(m, d, r, true));
  FE_CUDA(cudaMemcpyAsync(m->h_scal, m->scal, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  FE_TRY(fe_check_device_error(m));
  *out = sqrt(m->h_scal[0]);
  return FE_OK;
}

static int solve_impl(fe_mesh m, int method, double tol, int max_it, double* d, const nl_opts& o, nl_stats& st) {
  const int64_t n = m->ndof;
  const unsigned g1 = (unsigned)((n + 255) / 256);
  if (!m->nl_R) FE_TRY(fe_alloc_t(m, &m->nl_R, (size_t)n));
  if (!m->nl_Rn) FE_TRY(fe_alloc_t(m, &m->nl_Rn, (size_t)n));
  if (!m->nl_dl) FE_TRY(fe_alloc_t(m, &m->nl_dl, (size_t)n));
  if (!m->nl_t) FE_TRY(fe_alloc_t(m, &m->nl_t, (size_t)n));
  if (!m->rho_d) FE_TRY(fe_alloc_t(m, &m->rho_d, LBFGS_MAX));
  m->orthog = o.orthog;
  FE_TRY(fe_workspace(m, o.ksp_restart));
  if (o.apply_dirichlet) FE_TRY(fe_apply_dirichlet(m, d));
  double* R = m->nl_R;
  double* Rn = m->nl_Rn;
  double* dl = m->nl_dl;
  double* t = m->nl_t;
  double r0 = 0.0, rk = 0.0;
  FE_TRY(residual_norm(m, d, R, &r0));
  rk = r0;
  st.r0 = r0;
  st.res_hist[0] = r0;
  st.hist_len = 1;
  st.nit = 0;
  st.lit_total = 0;
  st.assemblies = 0;
  int status = NL_MAX_IT;
  if (!std::isfinite(r0)) {
    st.rfinal = r0;
    return NL_NONFINITE;
  }
  if (r0 == 0.0) {
    st.rfinal = 0.0;
    return FE_OK;
  }
  if (method == NL_NK || method == NL_INK) {
    double eta = method == NL_NK ? o.ksp_rtol : o.ew_rtol0;
    const double alpha2 = 0.5 * (1.0 + sqrt(5.0));
    for (int k = 1; k <= max_it; k++) {
      if ((k - 1) % o.jac_lag == 0) {  // Jacobian lagging: reuse the tangent in between
        FE_TRY(fe_tangent_dev(m, d, o.precision));
        st.assemblies++;
      }
      // K delta = -R
      FE_TRY(fe_axpby_dev(m, -1.0, R, 0.0, t, n));
      FE_CUDA(cudaMemsetAsync(dl, 0, n * sizeof(double), m->stream));
      int its = 0;
      double lres = 0.0;
      FE_TRY(fe_gmres_dev(m, t, dl, eta, o.ksp_atol, o.ksp_restart, o.ksp_max_it, &its, &lres));
      st.lit_total += its;
      if (k < NL_HIST) {
        st.lit_hist[k] = its;
        st.eta_hist[k] = eta;
      }
      // linear residual ||R_{k-1} + K delta|| for Eisenstat-Walker (FP64
      // vectors and accumulation in every precision)
      FE_TRY(fe_spmv_acc_dev(m, dl, Rn));
      FE_TRY(fe_axpby_dev(m, 1.0, R, 1.0, Rn, n));
      double ln2 = 0.0;
      FE_TRY(fe_dot_dev(m, Rn, Rn, n, &ln2));
      double lnorm = sqrt(ln2);
      if (k < NL_HIST) st.lres_hist[k] = lnorm;
      FE_TRY(fe_axpby_dev(m, 1.0, dl, 1.0, d, n));  // basic line search: full step
      double rprev = rk;
      FE_TRY(residual_norm(m, d, R, &rk));
      st.nit = k;
      if (k < NL_HIST) {
        st.res_hist[k] = rk;
        st.hist_len = k + 1;
      }
      if (!std::isfinite(rk)) { status = NL_NONFINITE; break; }
      if (rk <= tol * r0) { status = FE_OK; break; }
      if (rk > o.dtol * r0) { status = NL_DIVERGED; break; }
      if (method == NL_INK) {
        double eta_prev = eta;
        eta = fabs(rk - lnorm) / rprev;
        double stol = pow(eta_prev, alpha2);
        if (stol > 0.1) eta = fmax(eta, stol);
        eta = fmin(eta, o.ew_rtolmax);
      }
    }
  } else {
    const int mcap = o.lbfgs_m;
    if (mcap < 1 || mcap > LBFGS_MAX) return fe_set_error("lbfgs_m must lie in [1, %d]", LBFGS_MAX), FE_ERR_ARG;
    if (m->lb_m < mcap) {
      if (m->S) {
        cudaFreeAsync(m->S, m->stream);
        cudaFreeAsync(m->Yv, m->stream);
        m->device_bytes -= 2LL * m->lb_m * n * 8;
        m->S = m->Yv = nullptr;
      }
      FE_TRY(fe_alloc_t(m, &m->S, (size_t)mcap * n));
      FE_TRY(fe_alloc_t(m, &m->Yv, (size_t)mcap * n));
      m->lb_m = mcap;
    }
    FE_TRY(fe_tangent_dev(m, d, o.precision));  // the one Hessian assembly at d_0
    st.assemblies = 1;
    int head = 0, np = 0;
    double eta = o.ksp_rtol, rprev2 = 0.0;  // iB H0 tolerance; ||R_{k-2}||
    const double alpha2 = 0.5 * (1.0 + sqrt(5.0));
    for (int k = 1; k <= max_it; k++) {
      if (method == NL_IB && o.ib_adaptive && k > 1) {  // EW choice 2 on the nonlinear residuals
        const double eta_prev = eta;
        eta = 0.9 * pow(rk / rprev2, alpha2);
        const double sg = 0.9 * pow(eta_prev, alpha2);
        if (sg > 0.1) eta = fmax(eta, sg);
        eta = fmin(eta, o.ew_rtolmax);
      }
      if (o.hess_reassemble > 0 && k > 1 && (k - 1) % o.hess_reassemble == 0) {
        // new H0 from the tangent at the current iterate; the stored pairs
        // belonged to the old one, so the memory restarts
        FE_TRY(fe_tangent_dev(m, d, o.precision));
        st.assemblies++;
        head = 0;
        np = 0;
      }
      int lit = 0;
      FE_TRY(fe_lbfgs_dev(m, m->S, m->Yv, m->rho_d, head, mcap, np, n, R, t, method == NL_B ? 0 : 2,
                          eta, o.ksp_atol, o.ksp_restart, o.ksp_max_it, &lit));
      st.lit_total += lit;
      if (k < NL_HIST) {
        st.lit_hist[k] = lit;
        st.eta_hist[k] = method == NL_B ? 0.0 : eta;
      }
      rprev2 = rk;
      {
        FE_SCOPE(m, FE_PROF_VECTOR, 32.0 * n);
        k_step<<<g1, 256, 0, m->stream>>>(n, t, dl, d);  // delta = -H R; d += delta
      }
      FE_CUDA(cudaGetLastError());
      FE_TRY(residual_norm(m, d, Rn, &rk));
      st.nit = k;
      if (k < NL_HIST) {
        st.res_hist[k] = rk;
        st.hist_len = k + 1;
      }
      // secant pair: s = delta, y = R_{k+1} - R_k, rho = 1/(y.s), skipped if y.s <= 0
      {
        FE_SCOPE(m, FE_PROF_VECTOR, 24.0 * n);
        k_diff<<<g1, 256, 0, m->stream>>>(n, Rn, R, t);
      }
      FE_CUDA(cudaGetLastError());
      double ys = 0.0;
      FE_TRY(fe_dot_dev(m, t, dl, n, &ys));
      if (ys > 0.0) {
        int slot = np < mcap ? (head + np) % mcap : head;
        FE_CUDA(cudaMemcpyAsync(m->S + (int64_t)slot * n, dl, n * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
        FE_CUDA(cudaMemcpyAsync(m->Yv + (int64_t)slot * n, t, n * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
        m->h_scal[8] = 1.0 / ys;
        FE_CUDA(cudaMemcpyAsync(m->rho_d + slot, m->h_scal + 8, sizeof(double), cudaMemcpyHostToDevice, m->stream));
        FE_CUDA(cudaStreamSynchronize(m->stream));
        if (np < mcap) np++;
        else head = (head + 1) % mcap;
      }
      std::swap(R, Rn);
      if (!std::isfinite(rk)) { status = NL_NONFINITE; break; }
      if (rk <= tol * r0) { status = FE_OK; break; }
      if (rk > o.dtol * r0) { status = NL_DIVERGED; break; }
      status = NL_MAX_IT;
    }
    m->nl_R = R;
    m->nl_Rn = Rn;
  }
  st.rfinal = rk;
  FE_CUDA(cudaStreamSynchronize(m->stream));
  return status;
}

extern "C" int nl_solve(fe_mesh m, int method, double tol, int max_it, double* d, const nl_opts* opts,
                        nl_stats* stats) {
  if (!m || !d) return fe_set_error("NULL argument"), FE_ERR_ARG;
  if (method < NL_NK || method > NL_IB) return fe_set_error("method must be 0..3"), FE_ERR_ARG;
  if (!(tol >= 0.0) || max_it < 0) return fe_set_error("bad tol/max_it"), FE_ERR_ARG;
  nl_opts o;
  nl_opts_default((nl_method)method, &o);
  if (opts) {
    o.precision = opts->precision;
    if (opts->ksp_rtol >= 0) o.ksp_rtol = opts->ksp_rtol;
    if (opts->ksp_atol >= 0) o.ksp_atol = opts->ksp_atol;
    if (opts->ew_rtol0 > 0) o.ew_rtol0 = opts->ew_rtol0;
    if (opts->ew_rtolmax > 0) o.ew_rtolmax = opts->ew_rtolmax;
    if (opts->ksp_restart > 0) o.ksp_restart = opts->ksp_restart;
    if (opts->ksp_max_it > 0) o.ksp_max_it = opts->ksp_max_it;
    if (opts->lbfgs_m > 0) o.lbfgs_m = opts->lbfgs_m;
    if (opts->dtol > 0) o.dtol = opts->dtol;
    o.apply_dirichlet = opts->apply_dirichlet;
    o.orthog = opts->orthog;
    o.jac_lag = opts->jac_lag > 0 ? opts->jac_lag : 1;
    o.hess_reassemble = opts->hess_reassemble;
    o.ib_adaptive = opts->ib_adaptive;
    o.pc_type = opts->pc_type;
  }
  if (o.jac_lag < 1 || o.hess_reassemble < 0)
    return fe_set_error("jac_lag must be >= 1 (0 = 1) and hess_reassemble >= 0"), FE_ERR_ARG;
  if (o.orthog < 0 || o.orthog > 2) return fe_set_error("orthog must be 0, 1 or 2"), FE_ERR_ARG;
  if (o.precision < 0 || o.precision > 2) return fe_set_error("bad precision"), FE_ERR_ARG;
  if (o.pc_type < 0 || o.pc_type > 2) return fe_set_error("pc_type must be 0, 1 or 2"), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  nl_stats local;
  nl_stats& st = stats ? *stats : local;
  std::memset(&st, 0, sizeof(st));
  auto t0 = std::chrono::steady_clock::now();
  m->pc_type = o.pc_type;  // used by every tangent assembly of the solve
  int rc = solve_impl(m, method, tol, max_it, d, o, st);
  auto t1 = std::chrono::steady_clock::now();
  st.time_s = std::chrono::duration<double>(t1 - t0).count();
  st.status = rc;
  return rc;
}
