// fe_internal.h -- internal types shared by the translation units of libfe.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fe.h"

// ---------------------------------------------------------------- errors
void fe_set_error(const char* fmt, ...);
#define FE_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      fe_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));   \
      return FE_ERR_CUDA;                                                                \
    }                                                                                    \
  } while (0)
#define FE_TRY(expr)            \
  do {                          \
    int r_ = (expr);            \
    if (r_ != FE_OK) return r_; \
  } while (0)

// device error word values (written by kernels, read by the host)
enum { DEV_OK = 0, DEV_ERR_TIMEOUT = 1, DEV_ERR_BOUNDS = 2, DEV_ERR_COLORS = 3 };

// Index checks of the FE_DEBUG_BOUNDS build.  fe_idx(i, n) returns i when
// 0 <= i < n; in the debug build an index outside the range raises this
// translation unit's device flag and is replaced by 0, so the access stays
// in bounds and the kernel runs to its end; every call then reports
// FE_ERR_DEVICE_FLAG (fe_check_device_error reads and clears the flags).  In
// the normal build fe_idx is the identity and costs nothing.
#ifdef FE_DEBUG_BOUNDS
static __device__ unsigned g_fe_dbg_bounds;
__device__ __forceinline__ int fe_idx(int i, int64_t n) {
  if (i < 0 || (int64_t)i >= n) {
    atomicExch(&g_fe_dbg_bounds, 1u);
    return 0;
  }
  return i;
}
// defines the host reader of this translation unit's flag (reads and clears it)
#define FE_DBG_BOUNDS_READER(name)                                                  \
  int name(void) {                                                                  \
    unsigned v = 0, z = 0;                                                          \
    if (cudaMemcpyFromSymbol(&v, g_fe_dbg_bounds, sizeof(v)) != cudaSuccess) return 1; \
    cudaMemcpyToSymbol(g_fe_dbg_bounds, &z, sizeof(z));                             \
    return v != 0;                                                                  \
  }
int fe_dbg_bounds_mesh(void);
int fe_dbg_bounds_assemble(void);
int fe_dbg_bounds_krylov(void);
int fe_dbg_bounds_amg(void);
int fe_dbg_bounds_batch(void);
#else
__device__ __forceinline__ int fe_idx(int i, int64_t) { return i; }
#define FE_DBG_BOUNDS_READER(name)
#endif

// ---------------------------------------------------------------- material parameters
struct MatParams {
  int kind;
  double mu, cvol;                // COOK_NH (mu, c_vol), TH_NH (mu)
  double C, bf, bt, bfs, kappa;   // GUCCIONE
  double gamma;                   // active tension at the current time
  double ap, bp, clog;            // POLYCONVEX: alpha_p, beta_p, c_log
};

// ---------------------------------------------------------------- mesh object
struct fe_mesh_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  int order = 1, pres = 0, nv = 0, ne = 0, nn = 0, np = 0, nen = 4, nq = 1;
  int64_t ndof = 0;
  fe_material mat{};
  double load = 0.0, time = 0.0;
  MatParams mp{};

  // host copies kept for queries
  std::vector<int> h_color_start;  // [ncolors+1] offsets into perm
  int ncolors = 0;
  int ngroups = 0;
  std::vector<fe_dirichlet_group> groups;

  // device topology / geometry
  double* X = nullptr;        // [nn][3]
  int* conn = nullptr;        // [ne][nen]
  int* colors = nullptr;      // [ne]
  int* perm = nullptr;        // [ne] element ids sorted by (colour, id)
  double* geo = nullptr;      // [ne][10]: grad lambda_1..3 (rows, 9) + volume
  double* fib = nullptr;      // [ne][9] or null
  uint8_t* fixmask = nullptr; // [nn] bit c: component c prescribed
  uint8_t* dgroup = nullptr;  // [nn]
  fe_dirichlet_group* d_groups = nullptr;

  // displacement block pattern
  int64_t nnzb = 0;
  int* row_ptr = nullptr;  // [nn+1]
  int* col = nullptr;      // [nnzb]
  int* diag_pos = nullptr; // [nn]
  int* emap = nullptr;     // [ne][nen*nen]
  // u-p coupling pattern (u rows, vertex columns) and its transpose
  int64_t nnz_up = 0;
  int* up_ptr = nullptr;   // [nn+1]
  int* up_col = nullptr;   // [nnz_up]
  int* upmap = nullptr;    // [ne][nen*4]
  int* pu_ptr = nullptr;   // [np+1]
  int* pu_col = nullptr;   // [nnz_up] u node of the entry
  int* pu_src = nullptr;   // [nnz_up] index of the entry in the u-row storage

  // residual gather lists: node -> (element*nen + local) ; vertex -> (element*4 + local)
  int* node_ptr = nullptr;
  int* node_list = nullptr;
  int* vert_ptr = nullptr;
  int* vert_list = nullptr;

  // boundary data precomputed at creation (constant in d)
  double* fext1 = nullptr;   // [nn][3] external load at load factor 1
  int64_t nnz_ks = 0;
  int* ks_ptr = nullptr;     // [nn+1] spring matrix (Robin faces)
  int* ks_col = nullptr;
  double* ks_val = nullptr;  // [nnz_ks][9]
  int* ks_kpos = nullptr;    // [nnz_ks] block index in the tangent pattern
  // The face pattern (ks_*) covers the node pairs of every face of kind 2
  // (springs), 3 (follower pressure) and 4 (dashpots).  ks_val holds the
  // springs, plus 2/dt times the dashpots while dynamics is on; the host
  // keeps both parts to rebuild it when dt changes.
  std::vector<double> h_ks_spring, h_ks_dashpot;  // [nnz_ks][9] each
  bool has_dashpots = false;
  double* kc_val = nullptr;  // [nnz_ks][9] the dashpots alone (device, while dynamics is on)
  // follower faces, evaluated on the deformed surface: kind 3 (pressure)
  // and kind 5 (traction per unit deformed area)
  int nff = 0;
  int* ff_nodes = nullptr;   // [nff][6] face nodes (vertices, then P2 edge nodes (0,1), (1,2), (2,0))
  int* ff_kind = nullptr;    // [nff] 3 or 5
  double* ff_data = nullptr; // [nff][3] p (kind 3) or t (kind 5) at load factor 1
  int* fn_ptr = nullptr;     // [nn+1] node -> its (follower face, local node) slots
  int* fn_list = nullptr;    // face * 8 + local node
  int* fk_ptr = nullptr;     // [nnz_ks+1] face-pattern entry -> its follower blocks
  int* fk_list = nullptr;    // face * 64 + a * 8 + b (block (a, b) of that face)

  // Newmark average-acceleration state (fe_set_dynamics); dyn == nullptr: static
  double dyn_rho = 0.0, dyn_dt = 0.0;
  double mass_c = 0.0;       // 4 rho / dt^2: the inertia weight of the step
  double dyn_const = 0.0;    // constant of the step functional (energy only)
  double* dyn = nullptr;     // [6][3 nn]: d_n, v_n, a_n, dhat, dtil, fdyn = 4/dt^2 M dhat + 2/dt C dtil
  double* dyn_keep = nullptr;  // the state storage, kept while dynamics is off

  // tangent and preconditioner
  int prec = -1;             // precision of the assembled tangent (-1 none)
  double* K64 = nullptr;     // [kv_count(nnzb)] tiles of 32 blocks, component-major inside a tile (kv_index)
  float* K32 = nullptr;
  __nv_bfloat16* K16 = nullptr;
  double* B64 = nullptr;     // [nnz_up][3]
  float* B32 = nullptr;
  double* Dinv64 = nullptr;  // [nn][9]
  float* Dinv32 = nullptr;
  double* Sd = nullptr;      // [np] SIMPLE Schur diagonal

  // workspace
  double* rel = nullptr;     // [ne][nen*3] element-local residual contributions
  double* relp = nullptr;    // [ne][4]
  double* red = nullptr;     // reduction partials [RED_SLOTS]
  unsigned* red_ticket = nullptr;
  double* scal = nullptr;    // device scalars [64]
  int* err = nullptr;        // device error word
  unsigned* bar = nullptr;   // grid reduction state [BAR_WORDS]: count, seq, slot[2] (u64); blocked-MGS seq, pub[2][8] (u64)
  double* h_scal = nullptr;  // pinned host mirror [64]

  // solver workspace (lazy)
  int ws_restart = 0;
  double* V = nullptr;       // [(restart+1)][ldv], rows zero-padded
  int64_t ldv = 0;           // leading dimension of V: ndof rounded up to 32
  int orthog = 0;            // 0: sequential MGS sweep, 1: low-synchronisation MGS, 2: blocked MGS
  double* Lmat = nullptr;    // [(restart+1)^2] strictly lower triangle of V^T V (low-sync MGS)
  double* hpub = nullptr;    // [restart+1] published MGS coefficients
  double* partv = nullptr;   // [partv_blocks][2 restart + 1] per-block inner products
  int partv_blocks = 0;
  double* Tbm = nullptr;     // [(restart+2)][BMGS_P] strictly lower rows of (I + L_B)^{-1} (blocked MGS)
  double* H = nullptr;       // [(restart+1)][restart] column-major by step
  double* gv = nullptr;      // Givens: cs, sn, g, y [4][restart+1]
  double* w64 = nullptr;     // [ndof]
  double* t64 = nullptr;     // [ndof]
  double* u64 = nullptr;     // [ndof]
  void* zx = nullptr;        // [ndof] SpMV input (FP32 or FP64)
  int lb_m = 0;
  double* S = nullptr;       // [m][ndof]
  double* Yv = nullptr;      // [m][ndof]
  double* nl_R = nullptr, *nl_Rn = nullptr, *nl_dl = nullptr, *nl_t = nullptr;
  double* rho_d = nullptr;   // [LBFGS_MAX] curvature scalars 1/(y.s) of the stored pairs
  double* alpha_d = nullptr; // [LBFGS_MAX] two-loop coefficients alpha_i
  double* lb_x = nullptr;    // [ndof] GMRES iterate of the inexact-BFGS H0

  // instrumentation
  int prof_timing = 0;
  int prof_suspend = 0;      // > 0 while kernels are captured into a CUDA graph
  int64_t prof_launches[FE_PROF_CLASSES] = {};
  int64_t prof_timed[FE_PROF_CLASSES] = {};
  double prof_ms[FE_PROF_CLASSES] = {};
  double prof_bytes[FE_PROF_CLASSES] = {};
  double prof_flops[FE_PROF_CLASSES] = {};
  struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    double bytes, flops;
  };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> ev_free;

  int pc_type = 0;           // displacement-block preconditioner: 0 nodal block-Jacobi, 1 AMG V-cycle,
                             // 2 AMG V-cycle with a BF16 copy of the fine level in its smoother
  struct AmgHier* amg = nullptr;  // AMG hierarchy (fe_amg.cu), built at the first AMG tangent
  unsigned wait_limit = 1u << 26;  // polls before a bounded device wait gives up
  int coop_blocks = 0;       // co-resident blocks for the persistent kernels
  int sm_count = 0;
  int64_t device_bytes = 0;
};

constexpr int RED_SLOTS = 16384;
constexpr int SCAL_N = 64;
constexpr int LBFGS_MAX = 1000;  // largest number of stored secant pairs
constexpr int BMGS_P = 8;        // basis vectors per block of the blocked MGS step
constexpr int BAR_WORDS = 64;    // u32 words of the grid reduction state

// Tangent values: tiles of 32 consecutive blocks, component-major inside a
// tile.  Entry c = 3i + k of block p lives at (p / 32) 288 + 32 c + p % 32,
// so a warp reading one component of 32 consecutive blocks reads at most two
// 128-byte runs of one 1,152-byte tile region (block-major storage made each
// such load touch the warp's whole value segment; fully component-major
// storage spread the warp over 9 distant DRAM pages).
__host__ __device__ __forceinline__ int64_t kv_index(int64_t p, int c) { return (p >> 5) * 288 + 32 * c + (p & 31); }
inline size_t kv_count(int64_t nnzb) { return (size_t)((nnzb + 31) / 32) * 288; }

// Consistent mass of one tet: int_T N_a N_b dV = V * mass_hat(order, a, b)
// (local nodes: vertices 0..3, then the P2 edge nodes (0,1), (0,2), (0,3),
// (1,2), (1,3), (2,3)).  Closed forms from int_T l1^i l2^j l3^k l4^l dV =
// 6 V i! j! k! l! / (i + j + k + l + 3)!: P1 (1 + delta_ab) / 20; P2 over
// 420: vertex-vertex 6 (a = b) or 1, vertex-edge -4 (the vertex is an end
// of the edge) or -6, edge-edge 32 (a = b), 16 (one shared vertex) or 8.
__host__ __device__ __forceinline__ double mass_hat(int order, int a, int b) {
  if (order == 1) return a == b ? 0.1 : 0.05;
  // end vertices of edge k, packed one per nibble: (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
  auto e0 = [](int k) { return (0x211000 >> (4 * k)) & 15; };
  auto e1 = [](int k) { return (0x332321 >> (4 * k)) & 15; };
  double c;
  if (a < 4 && b < 4) {
    c = a == b ? 6.0 : 1.0;
  } else if (a >= 4 && b >= 4) {
    int p = a - 4, q = b - 4;
    int shared = (e0(p) == e0(q)) + (e0(p) == e1(q)) + (e1(p) == e0(q)) + (e1(p) == e1(q));
    c = p == q ? 32.0 : (shared ? 16.0 : 8.0);
  } else {
    int v = a < 4 ? a : b, ed = (a < 4 ? b : a) - 4;
    c = (e0(ed) == v || e1(ed) == v) ? -4.0 : -6.0;
  }
  return c / 420.0;
}

// Counts one kernel launch of class `cls` and, with timing on, brackets it
// with events on the mesh stream: open the scope, launch, close the scope.
struct LaunchScope {
  fe_mesh m;
  int cls;
  double bytes, flops;
  cudaEvent_t a = nullptr;
  LaunchScope(fe_mesh m_, int cls_, double bytes_, double flops_ = 0.0);
  ~LaunchScope();
};
#define FE_CAT2(a, b) a##b
#define FE_CAT(a, b) FE_CAT2(a, b)
#define FE_SCOPE(m, cls, bytes) LaunchScope FE_CAT(fe_scope_, __LINE__)(m, cls, (double)(bytes))
#define FE_SCOPE_F(m, cls, bytes, flops) \
  LaunchScope FE_CAT(fe_scope_, __LINE__)(m, cls, (double)(bytes), (double)(flops))

// allocation helper that tracks the mesh's device footprint
int fe_alloc(fe_mesh m, void** p, size_t bytes);
template <class T>
int fe_alloc_t(fe_mesh m, T** p, size_t count) {
  return fe_alloc(m, reinterpret_cast<void**>(p), count * sizeof(T));
}
int fe_check_device_error(fe_mesh m);  // syncs the stream and reads the error word
// Kernel launch facts cached per (kernel, device, shape), safe from several
// host threads (the serving loop) and from several devices in one process:
// the dynamic shared memory opt-in of a kernel (set once per device) and its
// resident blocks per SM for a block size and dynamic shared memory size.
int fe_kernel_smem(const void* fn, int smem_bytes);
int fe_kernel_occupancy(const void* fn, int threads, size_t smem_bytes, int* blocks_per_sm);
int fe_reset_grid_sync(fe_mesh m);     // arrival counter, step sequence, published-value slots

// ---------------------------------------------------------------- internal entry points
// assembly (fe_assemble.cu)
int fe_residual_dev(fe_mesh m, const double* d, double* r, bool want_norm);  // norm^2 -> scal[0]
int fe_tangent_dev(fe_mesh m, const double* d, int precision);
int fe_energy_dev(fe_mesh m, const double* d, double* out);
// linear algebra (fe_krylov.cu)
int fe_spmv_dev(fe_mesh m, const double* x, double* y);           // FP64 in/out, current tangent
int fe_spmv_acc_dev(fe_mesh m, const double* x, double* y);       // FP64 in/out and accumulation, any storage
int fe_pc_dev(fe_mesh m, const double* x, double* y);             // FP64 in/out
int fe_gmres_dev(fe_mesh m, const double* b, double* x, double rtol, double atol, int restart,
                 int max_it, int* iters, double* res);
int fe_dot_dev(fe_mesh m, const double* a, const double* b, int64_t n, double* out_host);
int fe_axpby_dev(fe_mesh m, double a, const double* x, double b, double* y, int64_t n);
int fe_lbfgs_dev(fe_mesh m, const double* S, const double* Y, const double* rho, int head, int mcap,
                 int k, int64_t ld, const double* q, double* z, int h0, double ksp_rtol,
                 double ksp_atol, int restart, int kmaxit, int* lit);
int fe_workspace(fe_mesh m, int restart);
int fe_spmv_from_input(fe_mesh m, const void* xin, double* y);  // input already in the SpMV precision
int fe_spmv_preload(fe_mesh m);  // loads every SpMV kernel and caches its launch facts
// fe_amg.cu: smoothed-aggregation AMG.  fe_amg_setup builds the hierarchy
// for the tangent just assembled (its structure once per mesh, on the host;
// its numbers every time, on the device); fe_amg_apply runs one V-cycle on
// the displacement part of x (FP64) into z (FP64 or FP32, z_double says
// which); fe_amg_free releases everything.
int fe_amg_setup(fe_mesh m);
int fe_amg_apply(fe_mesh m, const double* x, void* z, bool z_double);
void fe_amg_free(fe_mesh m);
// fe_assemble.cu: uploads the face-pattern values (springs plus 2/dt times
// the dashpots while dynamics is on)
int fe_upload_face_values(fe_mesh m);
// fe_noalloc.cu: resolves the fixed array of fe_spmv_noalloc on the mesh's
// device and loads the kernels that entry point launches (called by
// fe_mesh_create with the mesh's device current)
int fe_noalloc_prepare(fe_mesh m);
