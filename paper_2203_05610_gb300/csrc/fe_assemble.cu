// fe_assemble.cu -- residual, energy and consistent-tangent assembly on
// P1/P2 tetrahedra (arxiv 2203.05610: residual form R(d) = f - div P(F),
// F = I + grad d, P = dPsi/dF; energy of Eq. "minimization"; tangent of
// Eq. "newton"), materials of Section "Test problems and solvers details".
//
// Residual: one thread per (element, quadrature point) writes element-local
// contributions (QP lanes reduced with warp shuffles), then one thread per
// node gathers its incident contributions in a fixed order, adds loads and
// springs, masks prescribed components and reduces ||R||^2 deterministically.
// Tangent: elements in colour order (no two elements of a colour share a
// node), a CTA per group of elements: material tangent per QP in shared
// memory, then G_a^T A G_b block products written straight into the
// block-CSR values (read-modify-write, no atomics).
#include <cmath>

#include "fe_element.cuh"

// ---------------------------------------------------------------- residual
static FollowerFaces follower_faces(fe_mesh m) {
  return FollowerFaces{m->nff, m->ff_nodes, m->ff_kind, m->ff_data, m->fn_ptr, m->fn_list, m->fk_ptr, m->fk_list,
                       m->X};
}

// MASS adds the inertia of a Newmark step, mass_c M d with mass_c = 4 rho /
// dt^2 (the step's constant part 4/dt^2 M dhat enters in the gather); the
// static instantiation carries none of its registers.
template <int ORDER, bool MASS>
__global__ void __launch_bounds__(128) k_elem_residual(int ne, const int* __restrict__ conn,
                                                       const double* __restrict__ geo,
                                                       const double* __restrict__ d, int nn, int pres,
                                                       MatParams mp, const double* __restrict__ fib,
                                                       double mass_c, double* __restrict__ rel,
                                                       double* __restrict__ relp) {
  elem_residual_item<ORDER, MASS>(blockIdx.x * blockDim.x + threadIdx.x, ne, conn, geo, d, nn, pres, mp, fib, mass_c, rel, relp);
}

// Node-wise gather of the element contributions plus the boundary and
// Newmark terms: R = sum rel - load fext1 + Ks d + follower forces - fdyn
// (fdyn = 4/dt^2 M dhat + 2/dt C dtil, nullptr when static; the dashpots'
// 2/dt C d sits in ks_val while dynamics is on).  FOLLOW: the mesh has
// follower faces (the instantiation without them keeps the plain gather's
// registers).
template <int ORDER, bool FOLLOW>
__global__ void __launch_bounds__(256) k_gather_residual(
    int nn, int nen, const int* __restrict__ node_ptr, const int* __restrict__ node_list,
    const double* __restrict__ rel, const double* __restrict__ fext1, double load,
    const int* __restrict__ ks_ptr, const int* __restrict__ ks_col, const double* __restrict__ ks_val,
    const double* __restrict__ d, const uint8_t* __restrict__ fixmask, int np,
    const int* __restrict__ vert_ptr, const int* __restrict__ vert_list, const double* __restrict__ relp,
    FollowerFaces ff, const double* __restrict__ fdyn,
    double* __restrict__ r, double* red, unsigned* ticket, double* norm2, int64_t nrel) {
  const double acc = gather_node<ORDER, FOLLOW>(blockIdx.x * blockDim.x + threadIdx.x, nn, nen, node_ptr, node_list, rel, fext1, load, ks_ptr, ks_col, ks_val, d, fixmask, np, vert_ptr, vert_list, relp, ff, fdyn, r, nrel);
  if (norm2) grid_sum_finish(acc, red, ticket, norm2);
}

int fe_residual_dev(fe_mesh m, const double* d, double* r, bool want_norm) {
  int nthr = m->ne * m->nq;
  double eb = (double)m->ne * (4.0 * m->nen + 80.0 + 24.0 * m->nen + (m->fib ? 72.0 : 0.0) + (m->pres ? 32.0 : 0.0)) +
              8.0 * (double)m->ndof;
  {
    FE_SCOPE(m, FE_PROF_RESIDUAL, eb);
    const bool dyn = m->dyn != nullptr;
    auto kern = m->order == 1 ? (dyn ? k_elem_residual<1, true> : k_elem_residual<1, false>)
                              : (dyn ? k_elem_residual<2, true> : k_elem_residual<2, false>);
    kern<<<(nthr + 127) / 128, 128, 0, m->stream>>>(m->ne, m->conn, m->geo, d, m->nn, m->pres, m->mp, m->fib,
                                                    m->mass_c, m->rel, m->relp);
  }
  FE_CUDA(cudaGetLastError());
  int rows = m->nn + m->np;
  int grid = (rows + 255) / 256;
  if (grid > RED_SLOTS) return fe_set_error("mesh too large for the reduction buffer"), FE_ERR_ARG;
  double gb = (double)m->ne * m->nen * 28.0 + 4.0 * (m->nn + 1) + 25.0 * m->nn + 8.0 * (double)m->ndof +
              (m->pres ? (double)m->ne * 4 * 12.0 + 4.0 * (m->np + 1) : 0.0);
  if (m->dyn) gb += 24.0 * m->nn;
  FE_SCOPE(m, FE_PROF_RESIDUAL, gb);
  const double* fdyn = m->dyn ? m->dyn + 5 * 3 * (size_t)m->nn : nullptr;
  const bool fol = m->nff > 0;
  auto gather = m->order == 1 ? (fol ? k_gather_residual<1, true> : k_gather_residual<1, false>)
                              : (fol ? k_gather_residual<2, true> : k_gather_residual<2, false>);
  gather<<<grid, 256, 0, m->stream>>>(m->nn, m->nen, m->node_ptr, m->node_list, m->rel, m->fext1, m->load,
                                      m->ks_ptr, m->ks_col, m->ks_val, d, m->fixmask, m->np, m->vert_ptr,
                                      m->vert_list, m->relp, follower_faces(m), fdyn, r, m->red, m->red_ticket,
                                      want_norm ? m->scal : nullptr, (int64_t)m->ne * m->nen);
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// ---------------------------------------------------------------- energy
template <int ORDER>
__global__ void __launch_bounds__(128) k_elem_energy(int ne, const int* __restrict__ conn,
                                                     const double* __restrict__ geo, const double* __restrict__ d,
                                                     int nn, int pres, MatParams mp, const double* __restrict__ fib,
                                                     double mass_c, double* red, unsigned* ticket, double* out) {
  constexpr int NEN = ORDER == 1 ? 4 : 10;
  constexpr int NQ = ORDER == 1 ? 1 : 4;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int e = t / NQ, q = t % NQ;
  double val = 0.0;
  if (e < ne) {
    const int* c = conn + (size_t)e * NEN;
    double G[4][3], vol;
    load_G(geo, e, G, vol);
    double lam[4];
    for (int k = 0; k < 4; k++) lam[k] = lam_q<ORDER>(q, k);
    QPState<double> s;
    for (int k = 0; k < 9; k++) s.F[k] = (k % 4 == 0) ? 1.0 : 0.0;
    for (int a = 0; a < NEN; a++) {
      double g[3];
      shape_grad<ORDER>(a, lam, G, g);
      for (int i = 0; i < 3; i++)
        for (int J = 0; J < 3; J++) s.F[3 * i + J] += d[3 * (size_t)c[a] + i] * g[J];
    }
    s.p = 0.0;
    if (pres == 1)
      for (int v = 0; v < 4; v++) s.p += d[3 * (size_t)nn + c[v]] * lam[v];
    else if (pres == 2)
      s.p = d[3 * (size_t)nn + e];
    const double* fe = fib ? fib + (size_t)e * 9 : nullptr;
    qp_prepare(mp, fe, s);
    val = vol / NQ * qp_energy(mp, s);
    if (mass_c != 0.0 && q == 0)  // inertia of the step: mass_c / 2 d^T M d
      for (int a = 0; a < NEN; a++)
        for (int b = 0; b < NEN; b++) {
          const double* ua = d + 3 * (size_t)c[a];
          const double* ub = d + 3 * (size_t)c[b];
          val += 0.5 * mass_c * vol * mass_hat(ORDER, a, b) * (ua[0] * ub[0] + ua[1] * ub[1] + ua[2] * ub[2]);
        }
  }
  grid_sum_finish(val, red, ticket, out);
}

// boundary part of the energy: -load fext.d + d.Ks d / 2, and -fdyn.d of a
// Newmark step (fdyn nullptr when static)
__global__ void k_node_energy(int nn, const double* __restrict__ fext1, double load, const int* __restrict__ ks_ptr,
                              const int* __restrict__ ks_col, const double* __restrict__ ks_val,
                              const double* __restrict__ fdyn, const double* __restrict__ d, double* red,
                              unsigned* ticket, double* out) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (a < nn) {
    const double* u = d + 3 * (size_t)a;
    v = -load * (fext1[3 * a] * u[0] + fext1[3 * a + 1] * u[1] + fext1[3 * a + 2] * u[2]);
    if (fdyn) v -= fdyn[3 * (size_t)a] * u[0] + fdyn[3 * (size_t)a + 1] * u[1] + fdyn[3 * (size_t)a + 2] * u[2];
    for (int k = ks_ptr[a]; k < ks_ptr[a + 1]; k++) {
      const double* kv = ks_val + (size_t)k * 9;
      const double* w = d + 3 * (size_t)ks_col[k];
      for (int i = 0; i < 3; i++) v += 0.5 * u[i] * (kv[3 * i] * w[0] + kv[3 * i + 1] * w[1] + kv[3 * i + 2] * w[2]);
    }
  }
  grid_sum_finish(v, red, ticket, out);
}

int fe_energy_dev(fe_mesh m, const double* d, double* out) {
  int nthr = m->ne * m->nq;
  int grid = (nthr + 127) / 128;
  if (grid > RED_SLOTS) {
    // large meshes: the element sum in two halves would change the order; keep one pass
    return fe_set_error("mesh too large for the energy reduction"), FE_ERR_ARG;
  }
  const double mass_c = m->dyn ? m->mass_c : 0.0;
  if (m->order == 1)
    k_elem_energy<1><<<grid, 128, 0, m->stream>>>(m->ne, m->conn, m->geo, d, m->nn, m->pres, m->mp, m->fib,
                                                  mass_c, m->red, m->red_ticket, m->scal + 1);
  else
    k_elem_energy<2><<<grid, 128, 0, m->stream>>>(m->ne, m->conn, m->geo, d, m->nn, m->pres, m->mp, m->fib,
                                                  mass_c, m->red, m->red_ticket, m->scal + 1);
  FE_CUDA(cudaGetLastError());
  const double* fdyn = m->dyn ? m->dyn + 5 * 3 * (size_t)m->nn : nullptr;
  k_node_energy<<<(m->nn + 255) / 256, 256, 0, m->stream>>>(m->nn, m->fext1, m->load, m->ks_ptr, m->ks_col,
                                                            m->ks_val, fdyn, d, m->red, m->red_ticket, m->scal + 2);
  FE_CUDA(cudaGetLastError());
  FE_CUDA(cudaMemcpyAsync(m->h_scal + 1, m->scal + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  *out = m->h_scal[1] + m->h_scal[2] + (m->dyn ? m->dyn_const : 0.0);
  return FE_OK;
}

// ---------------------------------------------------------------- tangent

// One CTA assembles EPB elements of one colour into the block-CSR values.
template <int ORDER, class T>
__global__ void __launch_bounds__(256) k_elem_tangent(
    int nel, const int* __restrict__ elems, const int* __restrict__ conn, const double* __restrict__ geo,
    const double* __restrict__ d, int nn, int pres, MatParams mp, const double* __restrict__ fib,
    const int* __restrict__ emap, const int* __restrict__ upmap, const uint8_t* __restrict__ fixmask,
    double mass_c, T* __restrict__ K, T* __restrict__ B, int64_t nnzb) {
  tangent_tile<ORDER, T>(blockIdx.x, nel, elems, conn, geo, d, nn, pres, mp, fib, emap, upmap, fixmask, mass_c, K, B, nnzb);
}

// face-pattern blocks: springs (plus 2/dt dashpots while dynamics is on)
// and the follower-pressure blocks at d, in FP64, prescribed components
// masked; one thread per node row, the faces of an entry in a fixed order
template <int ORDER, class T>
__global__ void k_add_face_blocks(int nn, const int* __restrict__ ks_ptr, const int* __restrict__ ks_col,
                                  const double* __restrict__ ks_val, const int* __restrict__ ks_kpos,
                                  const uint8_t* __restrict__ fixmask, FollowerFaces ff,
                                  const double* __restrict__ d, double load, T* K) {
  face_blocks_row<ORDER, T>(blockIdx.x * blockDim.x + threadIdx.x, nn, ks_ptr, ks_col, ks_val, ks_kpos, fixmask, ff, d, load, K);
}

// unit diagonal at prescribed components, then invert each 3x3 diagonal block
template <class T, class DT>
__global__ void k_diag_inverse(int nn, const int* __restrict__ diag_pos, const uint8_t* __restrict__ fixmask,
                               T* K, DT* Dinv) {
  diag_inverse_row<T, DT>(blockIdx.x * blockDim.x + threadIdx.x, nn, diag_pos, fixmask, K, Dinv);
}

// SIMPLE Schur diagonal: S_vv = -sum_{(a,v)} sum_i B[a,v]_i^2 / A_(ai,ai)
template <class T>
__global__ void k_schur_diag(int np, const int* __restrict__ pu_ptr, const int* __restrict__ pu_col,
                             const int* __restrict__ pu_src, const int* __restrict__ diag_pos,
                             const T* __restrict__ K, const T* __restrict__ B, double* Sd) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= np) return;
  double s = 0.0;
  for (int k = pu_ptr[v]; k < pu_ptr[v + 1]; k++) {
    const int p = diag_pos[pu_col[k]];
    const T* b = B + (size_t)pu_src[k] * 3;
    for (int i = 0; i < 3; i++) s -= (double)b[i] * (double)b[i] / (double)K[kv_index(p, 4 * i)];
  }
  Sd[v] = s;
}

__global__ void k_to_bf16(int64_t n, const float* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

template <int ORDER, class T>
static int launch_tangent(fe_mesh m, const double* d, T* K, T* B) {
  using C = TanCfg<ORDER, T>;
  size_t smem = sizeof(T) * C::EPB * C::PER_E;
  FE_TRY(fe_kernel_smem((const void*)k_elem_tangent<ORDER, T>, (int)smem));
  for (int c = 0; c < m->ncolors; c++) {
    int start = m->h_color_start[c], nel = m->h_color_start[c + 1] - start;
    if (nel == 0) continue;
    int grid = (nel + C::EPB - 1) / C::EPB;
    const double nen = C::NEN;
    FE_SCOPE(m, FE_PROF_TANGENT, (double)nel * (4 * nen + 84 + 4 + 24 * nen + 4 * nen * nen + nen +
                                                2.0 * 9 * sizeof(T) * nen * nen + (m->pres ? 16.0 * nen * 4 * sizeof(T) : 0)));
    k_elem_tangent<ORDER, T><<<grid, 256, smem, m->stream>>>(nel, m->perm + start, m->conn, m->geo, d, m->nn,
                                                             m->pres, m->mp, m->fib, m->emap, m->upmap,
                                                             m->fixmask, m->dyn ? m->mass_c : 0.0, K, B,
                                                             m->nnzb);
    FE_CUDA(cudaGetLastError());
  }
  return FE_OK;
}

template <class T>
static int add_face_blocks(fe_mesh m, const double* d, T* K) {
  FE_SCOPE(m, FE_PROF_TANGENT, (double)m->nnz_ks * (4 + 4 + 72 + 2 * 9 * sizeof(T)));
  auto kern = m->order == 1 ? k_add_face_blocks<1, T> : k_add_face_blocks<2, T>;
  kern<<<(m->nn + 255) / 256, 256, 0, m->stream>>>(m->nn, m->ks_ptr, m->ks_col, m->ks_val, m->ks_kpos, m->fixmask,
                                                   follower_faces(m), d, m->load, K);
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

int fe_tangent_dev(fe_mesh m, const double* d, int precision) {
  if (precision < 0 || precision > 2) return fe_set_error("bad precision %d", precision), FE_ERR_ARG;
  if (precision == FE_PREC_MIXED_BF16 && m->pres)
    return fe_set_error("BF16 tangent storage is offered for the displacement form only"), FE_ERR_ARG;
  const size_t nval = kv_count(m->nnzb);  // tiles of 32 blocks (the last one zero-padded)
  const size_t nb = (size_t)(m->nnz_up > 0 ? m->nnz_up : 1) * 3;
  if (precision == FE_PREC_FP64) {
    if (!m->K64) FE_TRY(fe_alloc_t(m, &m->K64, nval));
    if (!m->Dinv64) FE_TRY(fe_alloc_t(m, &m->Dinv64, (size_t)m->nn * 9));
    if (m->pres && !m->B64) FE_TRY(fe_alloc_t(m, &m->B64, nb));
    FE_CUDA(cudaMemsetAsync(m->K64, 0, nval * sizeof(double), m->stream));
    if (m->pres) FE_CUDA(cudaMemsetAsync(m->B64, 0, nb * sizeof(double), m->stream));
    if (m->order == 1) FE_TRY((launch_tangent<1, double>(m, d, m->K64, m->B64)));
    else FE_TRY((launch_tangent<2, double>(m, d, m->K64, m->B64)));
    if (m->nnz_ks) FE_TRY(add_face_blocks(m, d, m->K64));
    FE_SCOPE(m, FE_PROF_TANGENT, (double)m->nn * (4 + 1 + 72 + 72 + 72));
    k_diag_inverse<double, double><<<(m->nn + 255) / 256, 256, 0, m->stream>>>(m->nn, m->diag_pos, m->fixmask,
                                                                               m->K64, m->Dinv64);
  } else {
    if (!m->K32) FE_TRY(fe_alloc_t(m, &m->K32, nval));
    if (!m->Dinv32) FE_TRY(fe_alloc_t(m, &m->Dinv32, (size_t)m->nn * 9));
    if (m->pres && !m->B32) FE_TRY(fe_alloc_t(m, &m->B32, nb));
    FE_CUDA(cudaMemsetAsync(m->K32, 0, nval * sizeof(float), m->stream));
    if (m->pres) FE_CUDA(cudaMemsetAsync(m->B32, 0, nb * sizeof(float), m->stream));
    if (m->order == 1) FE_TRY((launch_tangent<1, float>(m, d, m->K32, m->B32)));
    else FE_TRY((launch_tangent<2, float>(m, d, m->K32, m->B32)));
    if (m->nnz_ks) FE_TRY(add_face_blocks(m, d, m->K32));
    {
      FE_SCOPE(m, FE_PROF_TANGENT, (double)m->nn * (4 + 1 + 36 + 36 + 36));
      k_diag_inverse<float, float><<<(m->nn + 255) / 256, 256, 0, m->stream>>>(m->nn, m->diag_pos, m->fixmask,
                                                                             m->K32, m->Dinv32);
    }
    if (precision == FE_PREC_MIXED_BF16) {
      if (!m->K16) FE_TRY(fe_alloc_t(m, &m->K16, nval));
      FE_SCOPE(m, FE_PROF_TANGENT, 6.0 * nval);
      k_to_bf16<<<(unsigned)((nval + 255) / 256), 256, 0, m->stream>>>((int64_t)nval, m->K32, m->K16);
    }
  }
  FE_CUDA(cudaGetLastError());
  if (m->pres) {
    if (!m->Sd) FE_TRY(fe_alloc_t(m, &m->Sd, (size_t)m->np));
    FE_SCOPE(m, FE_PROF_TANGENT, (double)m->nnz_up * (8 + 3.0 * (precision == FE_PREC_FP64 ? 8 : 4) + 4) + 12.0 * m->np);
    if (precision == FE_PREC_FP64)
      k_schur_diag<double><<<(m->np + 255) / 256, 256, 0, m->stream>>>(m->np, m->pu_ptr, m->pu_col, m->pu_src,
                                                                       m->diag_pos, m->K64, m->B64, m->Sd);
    else
      k_schur_diag<float><<<(m->np + 255) / 256, 256, 0, m->stream>>>(m->np, m->pu_ptr, m->pu_col, m->pu_src,
                                                                      m->diag_pos, m->K32, m->B32, m->Sd);
    FE_CUDA(cudaGetLastError());
  }
  m->prec = precision;
  if (m->pc_type == 2 && precision == FE_PREC_MIXED_FP32) {  // BF16 fine level for the V-cycle's smoother
    const size_t nval = kv_count(m->nnzb);
    if (!m->K16) FE_TRY(fe_alloc_t(m, &m->K16, nval));
    FE_SCOPE(m, FE_PROF_TANGENT, 6.0 * nval);
    k_to_bf16<<<(unsigned)((nval + 255) / 256), 256, 0, m->stream>>>((int64_t)nval, m->K32, m->K16);
    FE_CUDA(cudaGetLastError());
  }
  if (m->pc_type >= 1) FE_TRY(fe_amg_setup(m));  // the AMG hierarchy of this tangent
  return FE_OK;
}

// ---------------------------------------------------------------- C ABI
extern "C" int fe_assemble_residual(fe_mesh m, const double* d, double* r, double* norm_out) {
  if (!m || !d || !r) return fe_set_error("NULL argument"), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  FE_TRY(fe_residual_dev(m, d, r, norm_out != nullptr));
  if (norm_out) {
    FE_CUDA(cudaMemcpyAsync(m->h_scal, m->scal, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  }
  FE_TRY(fe_check_device_error(m));
  if (norm_out) *norm_out = sqrt(m->h_scal[0]);
  return FE_OK;
}

extern "C" int fe_energy(fe_mesh m, const double* d, double* pi_out) {
  if (!m || !d || !pi_out) return fe_set_error("NULL argument"), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  FE_TRY(fe_energy_dev(m, d, pi_out));
  return fe_check_device_error(m);
}

extern "C" int fe_assemble_tangent(fe_mesh m, const double* d, int precision) {
  if (!m || !d) return fe_set_error("NULL argument"), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  FE_TRY(fe_tangent_dev(m, d, precision));
  return fe_check_device_error(m);
}

__global__ void k_widen(int64_t n, const float* __restrict__ s, double* __restrict__ d) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = (double)s[i];
}
__global__ void k_widen_bf(int64_t n, const __nv_bfloat16* __restrict__ s, double* __restrict__ d) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = (double)__bfloat162float(s[i]);
}

static int copy_out(fe_mesh m, double* host, const double* d64, const float* d32, const __nv_bfloat16* d16,
                    int64_t n) {
  if (!host) return FE_OK;
  if (d64) {
    FE_CUDA(cudaMemcpy(host, d64, n * sizeof(double), cudaMemcpyDeviceToHost));
    return FE_OK;
  }
  double* tmp = nullptr;
  FE_CUDA(cudaMallocAsync((void**)&tmp, n * sizeof(double), m->stream));
  if (d16) k_widen_bf<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(n, d16, tmp);
  else k_widen<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(n, d32, tmp);
  cudaError_t e = cudaStreamSynchronize(m->stream);
  if (e == cudaSuccess) e = cudaMemcpy(host, tmp, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFreeAsync(tmp, m->stream);
  cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return fe_set_error("%s", cudaGetErrorString(e)), FE_ERR_CUDA;
  return FE_OK;
}

extern "C" int fe_tangent_copy(fe_mesh m, double* val, double* bup, double* dinv) {
  if (!m) return fe_set_error("NULL mesh"), FE_ERR_ARG;
  if (m->prec < 0) return fe_set_error("no tangent assembled"), FE_ERR_STATE;
  FE_CUDA(cudaSetDevice(m->device));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  bool f64 = m->prec == FE_PREC_FP64;
  bool b16 = m->prec == FE_PREC_MIXED_BF16;
  if (val) {  // device values are tiled (kv_index); the copy is block-major [nnzb][3][3]
    std::vector<double> tv(kv_count(m->nnzb));
    FE_TRY(copy_out(m, tv.data(), f64 ? m->K64 : nullptr, f64 ? nullptr : m->K32, b16 ? m->K16 : nullptr,
                    (int64_t)tv.size()));
    for (int64_t p = 0; p < m->nnzb; p++)
      for (int c = 0; c < 9; c++) val[p * 9 + c] = tv[kv_index(p, c)];
  }
  if (m->pres) FE_TRY(copy_out(m, bup, f64 ? m->B64 : nullptr, f64 ? nullptr : m->B32, nullptr, m->nnz_up * 3));
  FE_TRY(copy_out(m, dinv, f64 ? m->Dinv64 : nullptr, f64 ? nullptr : m->Dinv32, nullptr, (int64_t)m->nn * 9));
  return FE_OK;
}

// ---------------------------------------------------------------- elastodynamics
// Newmark average acceleration (beta = 1/4, gamma = 1/2): the state d_n,
// v_n, a_n gives the predictors dhat = d_n + dt v_n + dt^2/4 a_n and
// dtil = d_n + dt/2 v_n; the step's residual is R(d) + 4/dt^2 M (d - dhat)
// + 2/dt C (d - dtil).  Layout of m->dyn: [6][3 nn] d_n, v_n, a_n, dhat,
// dtil, fdyn.

int fe_upload_face_values(fe_mesh m) {
  const size_t n = m->h_ks_spring.size();
  std::vector<double> v(m->h_ks_spring);
  if (m->dyn && m->has_dashpots)
    for (size_t i = 0; i < n; i++) v[i] += 2.0 / m->dyn_dt * m->h_ks_dashpot[i];
  if (!m->ks_val) FE_TRY(fe_alloc_t(m, &m->ks_val, n ? n : 1));
  if (n) FE_CUDA(cudaMemcpyAsync(m->ks_val, v.data(), n * sizeof(double), cudaMemcpyHostToDevice, m->stream));
  if (m->has_dashpots && !m->kc_val) {
    FE_TRY(fe_alloc_t(m, &m->kc_val, n));
    FE_CUDA(cudaMemcpyAsync(m->kc_val, m->h_ks_dashpot.data(), n * sizeof(double), cudaMemcpyHostToDevice,
                            m->stream));
  }
  FE_CUDA(cudaStreamSynchronize(m->stream));  // v is a host temporary
  return FE_OK;
}

// mode 0 (set): the state from d, v, a (nullptr: zero); mode 1 (advance):
// a = 4/dt^2 (d - dhat), v = 2/dt (d - dtil) from the converged d, then d_n = d.
// Either way the predictors of the next step follow.
__global__ void k_newmark_state(int64_t n3, int mode, double dt, const double* __restrict__ d,
                                const double* __restrict__ v, const double* __restrict__ a,
                                double* __restrict__ st) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  double* dn = st;
  double* vn = st + n3;
  double* an = st + 2 * n3;
  double* dhat = st + 3 * n3;
  double* dtil = st + 4 * n3;
  double di, vi, ai;
  if (mode == 0) {
    di = d ? d[i] : 0.0;
    vi = v ? v[i] : 0.0;
    ai = a ? a[i] : 0.0;
  } else {
    di = d[i];
    ai = 4.0 / (dt * dt) * (di - dhat[i]);
    vi = 2.0 / dt * (di - dtil[i]);
  }
  dn[i] = di;
  vn[i] = vi;
  an[i] = ai;
  dhat[i] = di + dt * vi + 0.25 * dt * dt * ai;
  dtil[i] = di + 0.5 * dt * vi;
}

// fdyn = mass_c M dhat + 2/dt C dtil per node (M gathered from the
// elements of the node in node_list order, C from the face pattern) and the
// constant of the step functional, (mass_c dhat.M dhat + 2/dt dtil.C dtil) / 2
template <int ORDER>
__global__ void __launch_bounds__(256) k_newmark_load(int nn, const int* __restrict__ node_ptr,
                                                      const int* __restrict__ node_list, const int* __restrict__ conn,
                                                      const double* __restrict__ geo, double mass_c, double cc,
                                                      const int* __restrict__ ks_ptr, const int* __restrict__ ks_col,
                                                      const double* __restrict__ kc_val, double* __restrict__ st,
                                                      double* red, unsigned* ticket, double* out) {
  constexpr int NEN = ORDER == 1 ? 4 : 10;
  const int64_t n3 = 3 * (int64_t)nn;
  const double* dhat = st + 3 * n3;
  const double* dtil = st + 4 * n3;
  double* fdyn = st + 5 * n3;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (t < nn) {
    double mh[3] = {0.0, 0.0, 0.0}, ch[3] = {0.0, 0.0, 0.0};
    for (int k = node_ptr[t]; k < node_ptr[t + 1]; k++) {
      const int slot = node_list[k], e = slot / NEN, a = slot % NEN;
      const double vol = geo[(size_t)e * 10 + 9];
      const int* c = conn + (size_t)e * NEN;
      for (int b = 0; b < NEN; b++) {
        const double w = vol * mass_hat(ORDER, a, b);
        const double* u = dhat + 3 * (size_t)c[b];
        for (int i = 0; i < 3; i++) mh[i] += w * u[i];
      }
    }
    if (kc_val)
      for (int k = ks_ptr[t]; k < ks_ptr[t + 1]; k++) {
        const double* kv = kc_val + (size_t)k * 9;
        const double* u = dtil + 3 * (size_t)ks_col[k];
        for (int i = 0; i < 3; i++) ch[i] += kv[3 * i] * u[0] + kv[3 * i + 1] * u[1] + kv[3 * i + 2] * u[2];
      }
    for (int i = 0; i < 3; i++) {
      fdyn[3 * (size_t)t + i] = mass_c * mh[i] + cc * ch[i];
      acc += 0.5 * (mass_c * dhat[3 * (size_t)t + i] * mh[i] + cc * dtil[3 * (size_t)t + i] * ch[i]);
    }
  }
  grid_sum_finish(acc, red, ticket, out);
}

static int newmark_update(fe_mesh m, int mode, const double* d, const double* v, const double* a) {
  const int64_t n3 = 3 * (int64_t)m->nn;
  const int grid = (m->nn + 255) / 256;
  if (grid > RED_SLOTS) return fe_set_error("mesh too large for the reduction buffer"), FE_ERR_ARG;
  {
    FE_SCOPE(m, FE_PROF_OTHER, (mode == 0 ? 3.0 : 1.0) * 8 * n3 + (mode == 0 ? 0.0 : 16.0 * n3) + 40.0 * n3);
    k_newmark_state<<<(unsigned)((n3 + 255) / 256), 256, 0, m->stream>>>(n3, mode, m->dyn_dt, d, v, a, m->dyn);
  }
  FE_CUDA(cudaGetLastError());
  {
    FE_SCOPE(m, FE_PROF_OTHER, (double)m->ne * m->nen * (8.0 + 4.0 * m->nen + 24.0 * m->nen) + 72.0 * m->nnz_ks);
    auto kern = m->order == 1 ? k_newmark_load<1> : k_newmark_load<2>;
    kern<<<grid, 256, 0, m->stream>>>(m->nn, m->node_ptr, m->node_list, m->conn, m->geo, m->mass_c,
                                      2.0 / m->dyn_dt, m->ks_ptr, m->ks_col, m->kc_val, m->dyn, m->red,
                                      m->red_ticket, m->scal + 40);
  }
  FE_CUDA(cudaGetLastError());
  FE_CUDA(cudaMemcpyAsync(m->h_scal + 40, m->scal + 40, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  FE_TRY(fe_check_device_error(m));
  m->dyn_const = m->h_scal[40];
  return FE_OK;
}

extern "C" int fe_set_dynamics(fe_mesh m, double rho, double dt) {
  if (!m) return fe_set_error("NULL mesh"), FE_ERR_ARG;
  if (!std::isfinite(rho) || !std::isfinite(dt)) return fe_set_error("rho and dt must be finite"), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  if (rho <= 0.0 || dt <= 0.0) {  // static again; the state storage stays allocated
    const bool was = m->dyn != nullptr;
    m->dyn_rho = m->dyn_dt = m->mass_c = m->dyn_const = 0.0;
    if (was) {
      double* keep = m->dyn;
      m->dyn = nullptr;
      FE_TRY(fe_upload_face_values(m));
      m->dyn_keep = keep;
    }
    return FE_OK;
  }
  if (!m->dyn) {
    if (!m->dyn_keep) FE_TRY(fe_alloc_t(m, &m->dyn_keep, 6 * 3 * (size_t)m->nn));
    m->dyn = m->dyn_keep;
  }
  m->dyn_rho = rho;
  m->dyn_dt = dt;
  m->mass_c = 4.0 * rho / (dt * dt);
  FE_TRY(fe_upload_face_values(m));
  return newmark_update(m, 0, nullptr, nullptr, nullptr);
}

extern "C" int fe_dynamics_set(fe_mesh m, const double* d, const double* v, const double* a) {
  if (!m) return fe_set_error("NULL mesh"), FE_ERR_ARG;
  if (!m->dyn) return fe_set_error("dynamics is off (fe_set_dynamics)"), FE_ERR_STATE;
  FE_CUDA(cudaSetDevice(m->device));
  return newmark_update(m, 0, d, v, a);
}

extern "C" int fe_dynamics_advance(fe_mesh m, const double* d) {
  if (!m || !d) return fe_set_error("NULL argument"), FE_ERR_ARG;
  if (!m->dyn) return fe_set_error("dynamics is off (fe_set_dynamics)"), FE_ERR_STATE;
  FE_CUDA(cudaSetDevice(m->device));
  return newmark_update(m, 1, d, nullptr, nullptr);
}

extern "C" int fe_dynamics_get(fe_mesh m, double* v, double* a) {
  if (!m) return fe_set_error("NULL mesh"), FE_ERR_ARG;
  if (!m->dyn) return fe_set_error("dynamics is off (fe_set_dynamics)"), FE_ERR_STATE;
  FE_CUDA(cudaSetDevice(m->device));
  const size_t n3 = 3 * (size_t)m->nn;
  if (v) FE_CUDA(cudaMemcpyAsync(v, m->dyn + n3, n3 * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  if (a) FE_CUDA(cudaMemcpyAsync(a, m->dyn + 2 * n3, n3 * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  return fe_check_device_error(m);
}

FE_DBG_BOUNDS_READER(fe_dbg_bounds_assemble)
