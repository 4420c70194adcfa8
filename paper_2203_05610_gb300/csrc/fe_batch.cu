// fe_batch.cu -- many small nonlinear solves in one launch: one CTA solves
// one request from its first residual to convergence, so a batch of up to
// (SMs x CTAs per SM) requests runs as a single kernel with no host round
// trip per iteration.  The solvers are those of nl_solve.cu (arxiv
// 2203.05610, Section "Numerical solvers", Appendix A options):
//   NK / iNK: Newton with GMRES(restart) right-preconditioned by the nodal
//             block-Jacobi, fixed ksp_rtol or the Eisenstat-Walker forcing
//             (choice 1 with the safeguard and the cap), full step;
//   B / iB  : L-BFGS two-loop over the stored pairs with H0 = block-Jacobi
//             of K(d_0) (B) or GMRES on K(d_0) at ksp_rtol (iB), full step.
// Every step is a CTA-level loop over the request's elements, nodes or
// unknowns, with the element bodies of fe_element.cuh; reductions are CTA
// sums in a fixed order, so a request's result does not depend on the
// other requests of its batch.  Residuals, Krylov vectors, the Arnoldi
// orthogonalisation and the L-BFGS inner products are FP64; the tangent,
// its block-Jacobi and the SpMV are in T (float: the mixed form, double:
// FP64 throughout).  Displacement-form meshes with nodal block-Jacobi only
// (no pressure space, AMG, follower faces or inertia).
#include <cstring>

#include "../../include/fe_batch.h"
#include "fe_element.cuh"

namespace {

constexpr int BATCH_MAX_COLORS = 64;
constexpr int BATCH_HIST = FE_BATCH_HIST;       // history entries and the L-BFGS pair cap
constexpr int BATCH_MAX_RESTART = 100;

}  // namespace

// one request of a batch: its mesh's device arrays, options and workspace
struct BatchReq {
  // mesh
  int nn, ne, ncolors;
  int64_t nnzb;
  const int *conn, *perm, *node_ptr, *node_list, *row_ptr, *col, *emap, *diag_pos;
  const int *ks_ptr, *ks_col, *ks_kpos;
  const double *geo, *X, *fib, *fext1, *ks_val;
  const uint8_t* fixmask;
  MatParams mp;
  double load;
  int cstart[BATCH_MAX_COLORS + 1];
  // solver
  int method, max_it, restart, kmaxit, mcap;
  double tol, ksp_rtol, ksp_atol, ew0, ewmax, dtol;
  // workspace: d (in/out) and the rest
  double *d, *r, *rn, *dl, *t, *w, *zb, *gr, *rel, *V, *S, *Y;
  void *K, *Dinv;
  fe_batch_out* out;
};

// CTA reductions that do not depend on the CTA's shape: 256 virtual lanes,
// lane v summing the terms i = v, v + 256, ... in order, each group of 32
// lanes reduced by the same shuffle tree, the 8 group sums added in order by
// one thread.  A request therefore gets bit-identical results with 128 or
// 256 threads per CTA (the launch shape the autotuner picks).
constexpr int VLANES = 256;
template <class F>
__device__ __forceinline__ double cta_vsum(int64_t n, F f, double* sh8, double* slot) {
  const int lane = threadIdx.x & 31;
  for (int vw = threadIdx.x >> 5; vw < VLANES / 32; vw += blockDim.x >> 5) {
    double s = 0.0;
    for (int64_t i = vw * 32 + lane; i < n; i += VLANES) s += f(i);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) sh8[vw] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < VLANES / 32; k++) t += sh8[k];
    *slot = t;
  }
  __syncthreads();
  const double r = *slot;
  __syncthreads();
  return r;
}

__device__ __forceinline__ double cta_dot(const double* a, const double* b, int64_t n, double* sh8, double* slot) {
  return cta_vsum(n, [&](int64_t i) { return a[i] * b[i]; }, sh8, slot);
}

// y = a x + b y over the CTA (no trailing barrier: callers sync before reading y elsewhere)
__device__ __forceinline__ void cta_axpby(double a, const double* x, double b, double* y, int64_t n) {
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

// R(d) into r; returns ||R||
template <int ORDER>
__device__ double cta_residual(const BatchReq& q, const double* d, double* r, double* sh8, double* slot) {
  constexpr int NQ = ORDER == 1 ? 1 : 4;
  constexpr int NEN = ORDER == 1 ? 4 : 10;
  const int nitems = q.ne * NQ;
  for (int base = 0; base < nitems; base += blockDim.x)
    elem_residual_item<ORDER, false>(base + (int)threadIdx.x, q.ne, q.conn, q.geo, d, q.nn, 0, q.mp, q.fib, 0.0,
                                     q.rel, nullptr);
  __syncthreads();
  const FollowerFaces none{0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int a = threadIdx.x; a < q.nn; a += blockDim.x)
    gather_node<ORDER, false>(a, q.nn, NEN, q.node_ptr, q.node_list, q.rel, q.fext1, q.load, q.ks_ptr, q.ks_col,
                              q.ks_val, d, q.fixmask, 0, nullptr, nullptr, nullptr, none, nullptr, r,
                              (int64_t)q.ne * NEN);
  __syncthreads();
  return sqrt(cta_dot(r, r, 3 * (int64_t)q.nn, sh8, slot));
}

// tangent K(d) in T with its block-Jacobi inverse
template <int ORDER, class T>
__device__ void cta_tangent(const BatchReq& q, const double* d) {
  using C = TanCfg<ORDER, T>;
  T* K = (T*)q.K;
  const int64_t nval = ((q.nnzb + 31) / 32) * 288;  // kv_count
  for (int64_t i = threadIdx.x; i < nval; i += blockDim.x) K[i] = T(0);
  __syncthreads();
  for (int c = 0; c < q.ncolors; c++) {
    const int start = q.cstart[c], nel = q.cstart[c + 1] - start;
    const int ntiles = (nel + C::EPB - 1) / C::EPB;
    for (int tile = 0; tile < ntiles; tile++) {
      tangent_tile<ORDER, T>(tile, nel, q.perm + start, q.conn, q.geo, d, q.nn, 0, q.mp, q.fib, q.emap, nullptr,
                             q.fixmask, 0.0, K, nullptr, q.nnzb);
      __syncthreads();
    }
  }
  const FollowerFaces none{0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int a = threadIdx.x; a < q.nn; a += blockDim.x)
    face_blocks_row<ORDER, T>(a, q.nn, q.ks_ptr, q.ks_col, q.ks_val, q.ks_kpos, q.fixmask, none, d, q.load, K);
  __syncthreads();
  for (int a = threadIdx.x; a < q.nn; a += blockDim.x)
    diag_inverse_row<T, T>(a, q.nn, q.diag_pos, q.fixmask, K, (T*)q.Dinv);
  __syncthreads();
}

// z = D^{-1} x (nodal 3x3 blocks, arithmetic in T)
template <class T>
__device__ __forceinline__ void cta_pc(const BatchReq& q, const double* x, double* z) {
  const T* Dv = (const T*)q.Dinv;
  for (int a = threadIdx.x; a < q.nn; a += blockDim.x) {
    const T* D = Dv + (int64_t)a * 9;
    const T x0 = (T)x[3 * (int64_t)a], x1 = (T)x[3 * (int64_t)a + 1], x2 = (T)x[3 * (int64_t)a + 2];
    z[3 * (int64_t)a] = (double)(D[0] * x0 + D[1] * x1 + D[2] * x2);
    z[3 * (int64_t)a + 1] = (double)(D[3] * x0 + D[4] * x1 + D[5] * x2);
    z[3 * (int64_t)a + 2] = (double)(D[6] * x0 + D[7] * x1 + D[8] * x2);
  }
}

// y = K x: a warp per node row, its lanes over the row's blocks; arithmetic
// in A (T, or double for the FP64-accumulated products of the EW test)
template <class T, class A>
__device__ void cta_spmv(const BatchReq& q, const double* x, double* y) {
  const T* K = (const T*)q.K;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int a = warp; a < q.nn; a += nw) {
    A s0 = A(0), s1 = A(0), s2 = A(0);
    const int p1 = q.row_ptr[a + 1];
    for (int p = q.row_ptr[a] + lane; p < p1; p += 32) {
      const double* xb = x + 3 * (int64_t)q.col[p];
      const A x0 = (A)xb[0], x1 = (A)xb[1], x2 = (A)xb[2];
      s0 += (A)K[kv_index(p, 0)] * x0 + (A)K[kv_index(p, 1)] * x1 + (A)K[kv_index(p, 2)] * x2;
      s1 += (A)K[kv_index(p, 3)] * x0 + (A)K[kv_index(p, 4)] * x1 + (A)K[kv_index(p, 5)] * x2;
      s2 += (A)K[kv_index(p, 6)] * x0 + (A)K[kv_index(p, 7)] * x1 + (A)K[kv_index(p, 8)] * x2;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s0 += __shfl_down_sync(0xffffffffu, s0, off);
      s1 += __shfl_down_sync(0xffffffffu, s1, off);
      s2 += __shfl_down_sync(0xffffffffu, s2, off);
    }
    if (lane == 0) {
      y[3 * (int64_t)a] = (double)s0;
      y[3 * (int64_t)a + 1] = (double)s1;
      y[3 * (int64_t)a + 2] = (double)s2;
    }
  }
}

// Restarted GMRES, right-preconditioned by the block-Jacobi, modified
// Gram-Schmidt (FP64), Givens rotations; solves K x = b from x = 0 to
// ||b - K x|| <= max(rtol ||b||, atol) or kmaxit iterations, as fe_gmres:
// every cycle starts from the residual b - K x, and in the mixed form with a
// target below 1e-4 ||b|| that residual takes FP64 products and an estimate
// at the target sends the iterate back to it (mixed-precision iterative
// refinement).  H, the rotations and the projected right-hand side live in
// shared memory.  Returns the iterations; *res the final residual (estimate).
template <class T>
__device__ int cta_gmres(const BatchReq& q, const double* b, double* x, double rtol, double atol, double* sh,
                         double* sh8, double* slot, double* res) {
  const int64_t n = 3 * (int64_t)q.nn;
  const int m = q.restart;
  double* H = sh;                // [(m+1) m] column j at H + j (m+1)
  double* cs = H + (m + 1) * m;  // [m]
  double* sn = cs + m;           // [m]
  double* g = sn + m;            // [m+1]
  double* y = g + m + 1;         // [m]
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = 0.0;
  const double bnorm = sqrt(cta_dot(b, b, n, sh8, slot));
  const double target = fmax(rtol * bnorm, atol);
  const bool refine = sizeof(T) == 4 && target < 1e-4 * bnorm;
  double* r = q.gr;  // residual of the current iterate
  int its = 0;
  bool first = true;
  for (;;) {
    // r = b - K x (x = 0 on the first cycle)
    if (first) {
      cta_axpby(1.0, b, 0.0, r, n);
    } else {
      if (refine) cta_spmv<T, double>(q, x, r);
      else cta_spmv<T, T>(q, x, r);
      __syncthreads();
      for (int64_t k = threadIdx.x; k < n; k += blockDim.x) r[k] = b[k] - r[k];
    }
    __syncthreads();
    const double beta = first ? bnorm : sqrt(cta_dot(r, r, n, sh8, slot));
    first = false;
    *res = beta;
    if (beta <= target || beta == 0.0 || its >= q.kmaxit || !isfinite(beta)) break;
    double* v0 = q.V;
    cta_axpby(1.0 / beta, r, 0.0, v0, n);
    if (threadIdx.x == 0) g[0] = beta;
    __syncthreads();
    int j = 0;
    bool stop = false;
    for (; j < m && its < q.kmaxit; j++) {
      double* vj = q.V + (int64_t)j * n;
      double* w = q.V + (int64_t)(j + 1) * n;
      cta_pc<T>(q, vj, q.zb);
      __syncthreads();
      cta_spmv<T, T>(q, q.zb, w);
      __syncthreads();
      for (int i = 0; i <= j; i++) {
        const double* vi = q.V + (int64_t)i * n;
        const double h = cta_dot(w, vi, n, sh8, slot);
        for (int64_t k = threadIdx.x; k < n; k += blockDim.x) w[k] -= h * vi[k];
        if (threadIdx.x == 0) H[j * (m + 1) + i] = h;
        __syncthreads();
      }
      const double hn = sqrt(cta_dot(w, w, n, sh8, slot));
      if (hn > 0.0)
        for (int64_t k = threadIdx.x; k < n; k += blockDim.x) w[k] /= hn;
      if (threadIdx.x == 0) {
        double* hc = H + j * (m + 1);
        hc[j + 1] = hn;
        for (int i = 0; i < j; i++) {  // previous rotations
          const double a = hc[i], c = hc[i + 1];
          hc[i] = cs[i] * a + sn[i] * c;
          hc[i + 1] = -sn[i] * a + cs[i] * c;
        }
        const double a = hc[j], c = hc[j + 1];
        const double den = sqrt(a * a + c * c);
        cs[j] = den > 0.0 ? a / den : 1.0;
        sn[j] = den > 0.0 ? c / den : 0.0;
        hc[j] = den;
        hc[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
      }
      __syncthreads();
      its++;
      if (fabs(g[j + 1]) <= target || hn == 0.0) {
        stop = hn == 0.0;
        j++;
        break;
      }
    }
    const int kdim = j;
    const double est = fabs(g[kdim]);
    if (threadIdx.x == 0) {  // back substitution H y = g
      for (int i = kdim - 1; i >= 0; i--) {
        double s = g[i];
        for (int l = i + 1; l < kdim; l++) s -= H[l * (m + 1) + i] * y[l];
        y[i] = s / H[i * (m + 1) + i];
      }
    }
    __syncthreads();
    // x += D^{-1} (V y)
    double* u = q.zb;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
      double s = 0.0;
      for (int i = 0; i < kdim; i++) s += y[i] * q.V[(int64_t)i * n + k];
      u[k] = s;
    }
    __syncthreads();
    double* pu = q.V;  // the basis is spent: preconditioned correction
    cta_pc<T>(q, u, pu);
    __syncthreads();
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) x[k] += pu[k];
    __syncthreads();
    *res = est;
    // the estimate decides, except in the refined mixed form, where an
    // estimate at the target goes back to the top for the FP64-product residual
    if (its >= q.kmaxit || stop || !isfinite(est) || (est <= target && !refine)) break;
  }
  return its;
}

template <int ORDER, class T>
__device__ void cta_record(const BatchReq& q, int k, double rk, int lit, double eta) {
  if (threadIdx.x == 0 && k < BATCH_HIST) {
    q.out->res_hist[k] = rk;
    q.out->lit_hist[k] = lit;
    q.out->eta_hist[k] = eta;
    q.out->hist_len = k + 1;
  }
}

template <int ORDER, class T, int NT>
__global__ void __launch_bounds__(NT) k_batch_solve(const BatchReq* __restrict__ reqs) {
  __shared__ BatchReq q;
  __shared__ double slot;
  __shared__ double sh8[VLANES / 32];
  extern __shared__ __align__(16) unsigned char smraw[];
  if (threadIdx.x == 0) q = reqs[blockIdx.x];
  __syncthreads();
  // GMRES scratch after the tangent's staging area
  double* sh = (double*)(smraw + ((sizeof(T) * TanCfg<ORDER, T>::EPB * TanCfg<ORDER, T>::PER_E + 15) / 16) * 16);
  const int64_t n = 3 * (int64_t)q.nn;
  double* d = q.d;
  double rk = cta_residual<ORDER>(q, d, q.r, sh8, &slot);
  const double r0 = rk;
  int status = NL_MAX_IT, nit = 0, assemblies = 0;
  int64_t lit_total = 0;
  cta_record<ORDER, T>(q, 0, r0, 0, 0.0);
  if (!isfinite(r0)) status = NL_NONFINITE;
  else if (r0 == 0.0) status = FE_OK;
  else if (q.method == NL_NK || q.method == NL_INK) {
    double eta = q.method == NL_NK ? q.ksp_rtol : q.ew0;
    const double alpha2 = 0.5 * (1.0 + sqrt(5.0));
    for (int k = 1; k <= q.max_it; k++) {
      cta_tangent<ORDER, T>(q, d);
      assemblies++;
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) q.t[i] = -q.r[i];
      __syncthreads();
      double lres_est = 0.0;
      const int its = cta_gmres<T>(q, q.t, q.dl, eta, q.ksp_atol, sh, sh8, &slot, &lres_est);
      lit_total += its;
      // linear residual ||R + K delta|| with FP64 products (Eisenstat-Walker)
      cta_spmv<T, double>(q, q.dl, q.rn);
      __syncthreads();
      const double* rr = q.r;
      const double* rl = q.rn;
      const double lnorm = sqrt(cta_vsum(
          n, [&](int64_t i) { const double v = rl[i] + rr[i]; return v * v; }, sh8, &slot));
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) d[i] += q.dl[i];
      __syncthreads();
      const double rprev = rk;
      rk = cta_residual<ORDER>(q, d, q.r, sh8, &slot);
      nit = k;
      cta_record<ORDER, T>(q, k, rk, its, eta);
      if (!isfinite(rk)) { status = NL_NONFINITE; break; }
      if (rk <= q.tol * r0) { status = FE_OK; break; }
      if (rk > q.dtol * r0) { status = NL_DIVERGED; break; }
      if (q.method == NL_INK) {
        const double eta_prev = eta;
        eta = fabs(rk - lnorm) / rprev;
        const double stol = pow(eta_prev, alpha2);
        if (stol > 0.1) eta = fmax(eta, stol);
        eta = fmin(eta, q.ewmax);
      }
    }
  } else {  // B / iB
    cta_tangent<ORDER, T>(q, d);
    assemblies = 1;
    __shared__ double alpha[BATCH_HIST];
    __shared__ double rho[BATCH_HIST];
    int head = 0, np = 0;
    const int mcap = min(q.mcap, BATCH_HIST);
    for (int k = 1; k <= q.max_it; k++) {
      // two-loop: z = H R, newest pair first
      double* z = q.t;
      cta_axpby(1.0, q.r, 0.0, q.w, n);  // q-vector of the recursion
      __syncthreads();
      for (int l = np - 1; l >= 0; l--) {
        const int sl = (head + l) % mcap;
        const double* s = q.S + (int64_t)sl * n;
        const double* yv = q.Y + (int64_t)sl * n;
        const double a = rho[sl] * cta_dot(s, q.w, n, sh8, &slot);
        if (threadIdx.x == 0) alpha[sl] = a;
        cta_axpby(-a, yv, 1.0, q.w, n);
        __syncthreads();
      }
      int its = 0;
      if (q.method == NL_B) {
        cta_pc<T>(q, q.w, z);
      } else {
        double est = 0.0;
        its = cta_gmres<T>(q, q.w, z, q.ksp_rtol, q.ksp_atol, sh, sh8, &slot, &est);
      }
      __syncthreads();
      lit_total += its;
      for (int l = 0; l < np; l++) {
        const int sl = (head + l) % mcap;
        const double* s = q.S + (int64_t)sl * n;
        const double* yv = q.Y + (int64_t)sl * n;
        const double bcoef = rho[sl] * cta_dot(yv, z, n, sh8, &slot);
        cta_axpby(alpha[sl] - bcoef, s, 1.0, z, n);
        __syncthreads();
      }
      // delta = -z; d += delta; new residual; secant pair
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        q.dl[i] = -z[i];
        d[i] -= z[i];
      }
      __syncthreads();
      rk = cta_residual<ORDER>(q, d, q.rn, sh8, &slot);
      nit = k;
      cta_record<ORDER, T>(q, k, rk, its, q.method == NL_B ? 0.0 : q.ksp_rtol);
      const double* rr = q.r;
      const double* rl = q.rn;
      const double* dd = q.dl;
      const double ys = cta_vsum(n, [&](int64_t i) { return (rl[i] - rr[i]) * dd[i]; }, sh8, &slot);
      if (ys > 0.0) {
        const int sl = np < mcap ? (head + np) % mcap : head;
        double* s = q.S + (int64_t)sl * n;
        double* yv = q.Y + (int64_t)sl * n;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
          s[i] = q.dl[i];
          yv[i] = q.rn[i] - q.r[i];
        }
        if (threadIdx.x == 0) rho[sl] = 1.0 / ys;
        if (np < mcap) np++;
        else head = (head + 1) % mcap;
      }
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) q.r[i] = q.rn[i];
      __syncthreads();
      if (!isfinite(rk)) { status = NL_NONFINITE; break; }
      if (rk <= q.tol * r0) { status = FE_OK; break; }
      if (rk > q.dtol * r0) { status = NL_DIVERGED; break; }
      status = NL_MAX_IT;
    }
  }
  if (threadIdx.x == 0) {
    fe_batch_out* o = q.out;
    o->status = status;
    o->nit = nit;
    o->lit_total = lit_total;
    o->assemblies = assemblies;
    o->r0 = r0;
    o->rfinal = rk;
  }
}

// ---------------------------------------------------------------- host side
static size_t batch_smem(int order, int prec, int restart) {
  const size_t tan = order == 1 ? (prec == FE_PREC_FP64 ? sizeof(double) * TanCfg<1, double>::EPB * TanCfg<1, double>::PER_E
                                                       : sizeof(float) * TanCfg<1, float>::EPB * TanCfg<1, float>::PER_E)
                                : (prec == FE_PREC_FP64 ? sizeof(double) * TanCfg<2, double>::EPB * TanCfg<2, double>::PER_E
                                                       : sizeof(float) * TanCfg<2, float>::EPB * TanCfg<2, float>::PER_E);
  const size_t gm = sizeof(double) * ((size_t)(restart + 1) * restart + 4 * (size_t)restart + 1);
  return (tan + 15) / 16 * 16 + gm;
}

template <int ORDER, class T, int NT>
static const void* batch_kernel() {
  return (const void*)k_batch_solve<ORDER, T, NT>;
}

static const void* pick_kernel(int order, int prec, int nt) {
  const bool f64 = prec == FE_PREC_FP64;
  if (order == 1) {
    if (f64) return nt == 128 ? batch_kernel<1, double, 128>() : batch_kernel<1, double, 256>();
    return nt == 128 ? batch_kernel<1, float, 128>() : batch_kernel<1, float, 256>();
  }
  if (f64) return nt == 128 ? batch_kernel<2, double, 128>() : batch_kernel<2, double, 256>();
  return nt == 128 ? batch_kernel<2, float, 128>() : batch_kernel<2, float, 256>();
}

extern "C" int fe_batch_supported(fe_mesh m, int method, const nl_opts* o) {
  if (!m) return 0;
  if (m->pres || m->nff || m->dyn || m->ncolors > BATCH_MAX_COLORS) return 0;
  if (method < NL_NK || method > NL_IB) return 0;
  if (o && (o->pc_type != 0 || o->precision == FE_PREC_MIXED_BF16 || o->jac_lag > 1 || o->hess_reassemble > 0 ||
            o->ib_adaptive))
    return 0;
  // the Hessenberg matrix lives in shared memory: GMRES(m) with m <= BATCH_MAX_RESTART
  if (!o || o->ksp_restart <= 0 || o->ksp_restart > BATCH_MAX_RESTART) return 0;
  if ((method == NL_B || method == NL_IB) && o && o->lbfgs_m > BATCH_HIST) return 0;
  return 1;
}

// workspace of one request (device), allocated per batch call
struct BatchWork {
  double* base = nullptr;
  void* K = nullptr;
  void* Dinv = nullptr;
};

// one launch for requests of one order and one precision
static int batch_group(int nreq, fe_mesh* meshes, const int* methods, const double* tols, const int* max_its,
                       const nl_opts* opts, double** d, int threads, fe_batch_out* out_host) {
  const fe_mesh m0 = meshes[0];
  const int order = m0->order;
  const int prec = opts[0].precision;
  std::vector<BatchReq> h(nreq);
  std::vector<void*> allocs;
  cudaStream_t stream = m0->stream;
  // stream-ordered allocations: no device-wide synchronisation, so batches
  // on other streams keep running
  auto cleanup = [&]() {
    for (void* p : allocs) cudaFreeAsync(p, stream);
  };
  std::vector<size_t> off_base(nreq), off_K(nreq), off_D(nreq);
  size_t total = 0;
  auto take = [&](size_t bytes) {
    const size_t o = total;
    total += (bytes + 255) / 256 * 256;
    return o;
  };
  int restart_max = 1;
  for (int i = 0; i < nreq; i++) {
    fe_mesh m = meshes[i];
    nl_opts o;
    nl_opts_default((nl_method)methods[i], &o);
    if (opts) {
      const nl_opts& u = opts[i];
      o.precision = u.precision;
      if (u.ksp_rtol >= 0) o.ksp_rtol = u.ksp_rtol;
      if (u.ksp_atol >= 0) o.ksp_atol = u.ksp_atol;
      if (u.ew_rtol0 > 0) o.ew_rtol0 = u.ew_rtol0;
      if (u.ew_rtolmax > 0) o.ew_rtolmax = u.ew_rtolmax;
      if (u.ksp_restart > 0) o.ksp_restart = u.ksp_restart;
      if (u.ksp_max_it > 0) o.ksp_max_it = u.ksp_max_it;
      if (u.lbfgs_m > 0) o.lbfgs_m = u.lbfgs_m;
      if (u.dtol > 0) o.dtol = u.dtol;
      o.apply_dirichlet = u.apply_dirichlet;
    }
    if (m->order != order || o.precision != prec) {
      cleanup();
      return fe_set_error("internal: a launch group needs one order and one precision"), FE_ERR_ARG;
    }
    restart_max = std::max(restart_max, o.ksp_restart);
    BatchReq& q = h[i];
    std::memset(&q, 0, sizeof(q));
    q.nn = m->nn;
    q.ne = m->ne;
    q.ncolors = m->ncolors;
    q.nnzb = m->nnzb;
    q.conn = m->conn;
    q.perm = m->perm;
    q.node_ptr = m->node_ptr;
    q.node_list = m->node_list;
    q.row_ptr = m->row_ptr;
    q.col = m->col;
    q.emap = m->emap;
    q.diag_pos = m->diag_pos;
    q.ks_ptr = m->ks_ptr;
    q.ks_col = m->ks_col;
    q.ks_kpos = m->ks_kpos;
    q.geo = m->geo;
    q.X = m->X;
    q.fib = m->fib;
    q.fext1 = m->fext1;
    q.ks_val = m->ks_val;
    q.fixmask = m->fixmask;
    q.mp = m->mp;
    q.load = m->load;
    for (int c = 0; c <= m->ncolors; c++) q.cstart[c] = m->h_color_start[c];
    q.method = methods[i];
    q.max_it = max_its[i];
    q.restart = o.ksp_restart;
    q.kmaxit = o.ksp_max_it;
    q.mcap = o.lbfgs_m;
    q.tol = tols[i];
    q.ksp_rtol = o.ksp_rtol;
    q.ksp_atol = o.ksp_atol;
    q.ew0 = o.ew_rtol0;
    q.ewmax = o.ew_rtolmax;
    q.dtol = o.dtol;
    const int64_t n = 3 * (int64_t)m->nn;
    const int64_t nvec = 7 + (q.restart + 1) + ((q.method >= NL_B) ? 2 * (int64_t)std::min(q.mcap, BATCH_HIST) : 0);
    const int64_t nrel = (int64_t)m->ne * m->nen * 3;
    const size_t sval = prec == FE_PREC_FP64 ? 8 : 4;
    off_base[i] = take(sizeof(double) * (size_t)(nvec * n + nrel));
    off_K[i] = take(sval * kv_count(m->nnzb));
    off_D[i] = take(sval * 9 * (size_t)m->nn);
  }
  FE_CUDA(cudaSetDevice(m0->device));
  char* pool = nullptr;
  if (cudaMallocAsync((void**)&pool, total, stream) != cudaSuccess)
    return fe_set_error("batch workspace allocation failed"), FE_ERR_OOM;
  allocs.push_back(pool);
  for (int i = 0; i < nreq; i++) {
    BatchReq& q = h[i];
    const int64_t n = 3 * (int64_t)meshes[i]->nn;
    const int64_t nrel = (int64_t)meshes[i]->ne * meshes[i]->nen * 3;
    double* base = (double*)(pool + off_base[i]);
    q.d = d[i];
    q.r = base;
    q.rn = base + n;
    q.dl = base + 2 * n;
    q.t = base + 3 * n;
    q.w = base + 4 * n;
    q.zb = base + 5 * n;
    q.gr = base + 6 * n;
    q.rel = base + 7 * n;
    q.V = q.rel + nrel;
    q.S = q.V + (int64_t)(q.restart + 1) * n;
    q.Y = q.S + (int64_t)std::min(q.mcap, BATCH_HIST) * n;
    q.K = pool + off_K[i];
    q.Dinv = pool + off_D[i];
  }
  BatchReq* dq = nullptr;
  fe_batch_out* dout = nullptr;
  if (cudaMallocAsync((void**)&dq, sizeof(BatchReq) * nreq, stream) != cudaSuccess) {
    cleanup();
    return fe_set_error("batch table allocation failed"), FE_ERR_OOM;
  }
  allocs.push_back(dq);
  if (cudaMallocAsync((void**)&dout, sizeof(fe_batch_out) * nreq, stream) != cudaSuccess) {
    cleanup();
    return fe_set_error("batch table allocation failed"), FE_ERR_OOM;
  }
  allocs.push_back(dout);
  for (int i = 0; i < nreq; i++) h[i].out = dout + i;
  // Dirichlet values of each request's load first (on each mesh's stream),
  // then the batch on the first mesh's stream
  for (int i = 0; i < nreq; i++) {
    if (!opts || opts[i].apply_dirichlet) {
      int rc = fe_apply_dirichlet(meshes[i], d[i]);
      if (rc != FE_OK) {
        cleanup();
        return rc;
      }
    }
    if (meshes[i]->stream != stream) {
      cudaError_t e = cudaStreamSynchronize(meshes[i]->stream);
      if (e != cudaSuccess) {
        cleanup();
        return fe_set_error("%s", cudaGetErrorString(e)), FE_ERR_CUDA;
      }
    }
  }
  cudaError_t e = cudaMemcpyAsync(dq, h.data(), sizeof(BatchReq) * nreq, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dout, 0, sizeof(fe_batch_out) * nreq, stream);
  const size_t smem = batch_smem(order, prec, restart_max);
  const void* fn = pick_kernel(order, prec, threads);
  if (e == cudaSuccess && fe_kernel_smem(fn, (int)smem) != FE_OK) {
    cleanup();
    return FE_ERR_CUDA;
  }
  if (e == cudaSuccess) {
    void* args[] = {(void*)&dq};
    e = cudaLaunchKernel(fn, dim3(nreq), dim3(threads), args, smem, stream);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, dout, sizeof(fe_batch_out) * nreq, cudaMemcpyDeviceToHost, stream);
  cleanup();  // stream-ordered: after the kernel and the copy-back
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fe_set_error("batch solve: %s", cudaGetErrorString(e)), FE_ERR_CUDA;
  return FE_OK;
}

extern "C" int fe_batch_solve(int nreq, fe_mesh* meshes, const int* methods, const double* tols,
                              const int* max_its, const nl_opts* opts, double** d, int threads,
                              fe_batch_out* out_host) {
  if (nreq <= 0) return FE_OK;
  if (!meshes || !methods || !tols || !max_its || !opts || !d || !out_host)
    return fe_set_error("NULL argument"), FE_ERR_ARG;
  if (threads != 128 && threads != 256) return fe_set_error("threads must be 128 or 256"), FE_ERR_ARG;
  for (int i = 0; i < nreq; i++) {
    if (!meshes[i] || !d[i]) return fe_set_error("NULL mesh or vector of request %d", i), FE_ERR_ARG;
    if (meshes[i]->device != meshes[0]->device) return fe_set_error("a batch runs on one device"), FE_ERR_ARG;
    if (!fe_batch_supported(meshes[i], methods[i], &opts[i]))
      return fe_set_error("request %d is not supported by the batched solver", i), FE_ERR_ARG;
  }
  // one launch per (order, precision), in order of first appearance
  std::vector<int> done(nreq, 0);
  for (int i0 = 0; i0 < nreq; i0++) {
    if (done[i0]) continue;
    std::vector<int> idx;
    for (int i = i0; i < nreq; i++)
      if (!done[i] && meshes[i]->order == meshes[i0]->order && opts[i].precision == opts[i0].precision) {
        idx.push_back(i);
        done[i] = 1;
      }
    const size_t g = idx.size();
    std::vector<fe_mesh> gm(g);
    std::vector<int> gmeth(g), gmax(g);
    std::vector<double> gtol(g);
    std::vector<nl_opts> gopt(g);
    std::vector<double*> gd(g);
    std::vector<fe_batch_out> gout(g);
    for (size_t k = 0; k < g; k++) {
      gm[k] = meshes[idx[k]];
      gmeth[k] = methods[idx[k]];
      gmax[k] = max_its[idx[k]];
      gtol[k] = tols[idx[k]];
      gopt[k] = opts[idx[k]];
      gd[k] = d[idx[k]];
    }
    FE_TRY(batch_group((int)g, gm.data(), gmeth.data(), gtol.data(), gmax.data(), gopt.data(), gd.data(), threads,
                       gout.data()));
    for (size_t k = 0; k < g; k++) out_host[idx[k]] = gout[k];
  }
  return FE_OK;
}

FE_DBG_BOUNDS_READER(fe_dbg_bounds_batch)
