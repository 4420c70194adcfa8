// fe_mesh.cu -- mesh creation: P2 edge nodes, GPU Jones-Plassmann colouring,
// block-CSR pattern, element -> block maps, element geometry, boundary data.
//
// Discretisation of the quasi-static problem of arxiv 2203.05610 (Sections
// "The hyperelasticity problem" and "Test problems and solvers details"):
// P1/P2 displacement on tetrahedra, optional P1 pressure (Taylor-Hood),
// Dirichlet data by rigid motions, dead tractions and pressures, epicardial
// springs.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <array>
#include <climits>
#include <map>
#include <mutex>
#include <numeric>

#include "fe_internal.h"

// ---------------------------------------------------------------- errors
static thread_local char g_err[1024] = "";
void fe_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
extern "C" const char* fe_last_error(void) { return g_err; }

// Stream-ordered allocations on the mesh's stream: freeing them does not
// synchronise the device, so meshes created and destroyed by the serving
// loop's workers do not stall the kernels of other requests.
int fe_alloc(fe_mesh m, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(p, bytes, m->stream);
  if (e != cudaSuccess) {
    fe_set_error("cudaMallocAsync(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    cudaGetLastError();
    return FE_ERR_OOM;
  }
  m->device_bytes += (int64_t)bytes;
  return FE_OK;
}

// grid-reduction state of the persistent kernels: arrival counter, step
// sequence, and two published-value slots holding the "not yet" sentinel;
// then the blocked-MGS step's own sequence and its two sets of 8 slots
int fe_reset_grid_sync(fe_mesh m) {
  static const unsigned long long sentinel = 0x7FF4DEAD5EEDF00DULL;
  unsigned long long init[BAR_WORDS / 2] = {};
  init[1] = init[2] = sentinel;                                 // {count, seq}, slot0, slot1
  for (int i = 4; i < 4 + 2 * BMGS_P; i++) init[i] = sentinel;  // {bseq, pad}, pub[2][8]
  FE_CUDA(cudaMemcpyAsync(m->bar, init, sizeof(init), cudaMemcpyHostToDevice, m->stream));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  return FE_OK;
}

namespace {
struct KernelKey {
  const void* fn;
  int device, threads;
  size_t smem;
  bool operator<(const KernelKey& o) const {
    if (fn != o.fn) return fn < o.fn;
    if (device != o.device) return device < o.device;
    if (threads != o.threads) return threads < o.threads;
    return smem < o.smem;
  }
};
std::mutex g_kernel_mu;
std::map<KernelKey, int> g_kernel_cache;  // smem opt-ins (threads = -1) and occupancies
}  // namespace

// The opt-in is one value per kernel and device: raise it to the largest
// size asked for so far (a smaller later request must not lower it below a
// size an earlier launch of that kernel still uses).
int fe_kernel_smem(const void* fn, int smem_bytes) {
  int dev = 0;
  FE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_kernel_mu);
  KernelKey k{fn, dev, -1, 0};
  auto it = g_kernel_cache.find(k);
  if (it != g_kernel_cache.end() && it->second >= smem_bytes) return FE_OK;
  FE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes));
  g_kernel_cache[k] = smem_bytes;
  return FE_OK;
}

int fe_kernel_occupancy(const void* fn, int threads, size_t smem_bytes, int* blocks_per_sm) {
  int dev = 0;
  FE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_kernel_mu);
  KernelKey k{fn, dev, threads, smem_bytes};
  auto it = g_kernel_cache.find(k);
  if (it != g_kernel_cache.end()) {
    *blocks_per_sm = it->second;
    return FE_OK;
  }
  int b = 0;
  FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem_bytes));
  g_kernel_cache[k] = b;
  *blocks_per_sm = b;
  return FE_OK;
}

FE_DBG_BOUNDS_READER(fe_dbg_bounds_mesh)

int fe_check_device_error(fe_mesh m) {
  int h = 0;
  FE_CUDA(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  FE_CUDA(cudaStreamSynchronize(m->stream));
#ifdef FE_DEBUG_BOUNDS
  if (h == DEV_OK && (fe_dbg_bounds_mesh() | fe_dbg_bounds_assemble() | fe_dbg_bounds_krylov() | fe_dbg_bounds_amg() |
                        fe_dbg_bounds_batch()))
    h = DEV_ERR_BOUNDS;
#endif
  if (h == DEV_OK) return FE_OK;
  // clear the error word and the grid-synchronisation state for later calls
  cudaMemsetAsync(m->err, 0, sizeof(int), m->stream);
  fe_reset_grid_sync(m);
  cudaStreamSynchronize(m->stream);
  if (h == DEV_ERR_TIMEOUT) {
    fe_set_error("a bounded device wait ran out (grid barrier)");
    return FE_ERR_TIMEOUT;
  }
  if (h == DEV_ERR_BOUNDS) {
    fe_set_error("device-side index check failed (an index outside its array)");
    return FE_ERR_DEVICE_FLAG;
  }
  fe_set_error("device-side check failed (code %d)", h);
  return FE_ERR_DEVICE_FLAG;
}

// ---------------------------------------------------------------- instrumentation
static cudaEvent_t ev_get(fe_mesh m) {
  if (!m->ev_free.empty()) {
    cudaEvent_t e = m->ev_free.back();
    m->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static void prof_resolve(fe_mesh m) {
  for (auto& r : m->prof_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      m->prof_ms[r.cls] += ms;
      m->prof_bytes[r.cls] += r.bytes;
      m->prof_flops[r.cls] += r.flops;
      m->prof_timed[r.cls]++;
    }
    m->ev_free.push_back(r.a);
    m->ev_free.push_back(r.b);
  }
  m->prof_pending.clear();
}

LaunchScope::LaunchScope(fe_mesh m_, int cls_, double bytes_, double flops_)
    : m(m_), cls(cls_), bytes(bytes_), flops(flops_) {
  if (m->prof_suspend) return;  // launches captured into a graph are counted at its launch
  m->prof_launches[cls]++;
  if (m->prof_timing) {
    a = ev_get(m);
    cudaEventRecord(a, m->stream);
  }
}

LaunchScope::~LaunchScope() {
  if (!a) return;
  cudaEvent_t b = ev_get(m);
  cudaEventRecord(b, m->stream);
  m->prof_pending.push_back({cls, a, b, bytes, flops});
  if (m->prof_pending.size() > 50000) prof_resolve(m);
}

extern "C" int fe_profile_reset(fe_mesh m, int timing) {
  if (!m) return fe_set_error("NULL mesh"), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  prof_resolve(m);
  for (int c = 0; c < FE_PROF_CLASSES; c++) {
    m->prof_launches[c] = m->prof_timed[c] = 0;
    m->prof_ms[c] = m->prof_bytes[c] = m->prof_flops[c] = 0.0;
  }
  m->prof_timing = timing ? 1 : 0;
  return FE_OK;
}

extern "C" int fe_profile_read(fe_mesh m, fe_profile_info* out) {
  if (!m || !out) return fe_set_error("NULL argument"), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  prof_resolve(m);
  for (int c = 0; c < FE_PROF_CLASSES; c++) {
    out->launches[c] = m->prof_launches[c];
    out->timed[c] = m->prof_timed[c];
    out->ms[c] = m->prof_ms[c];
    out->bytes[c] = m->prof_bytes[c];
    out->flops[c] = m->prof_flops[c];
  }
  return FE_OK;
}

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  // splitmix64 output function (Vigna), priority of the colouring
  unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// One Jones-Plassmann round: an uncoloured element whose higher-priority
// neighbours (sharing a vertex) are all coloured takes the smallest colour
// none of its coloured neighbours uses.  This reproduces sequential first-fit
// greedy colouring in descending priority order exactly.
__global__ void k_jp_round(int ne, int nen, const int* __restrict__ conn,
                           const int* __restrict__ vptr, const int* __restrict__ vel,
                           int* color, int* remaining, int* err) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  if (((volatile int*)color)[e] >= 0) return;
  unsigned long long pe = mix64((unsigned long long)e);
  unsigned long long used[2] = {0ull, 0ull};
  for (int a = 0; a < 4; a++) {
    int v = conn[(size_t)e * nen + a];
    for (int k = vptr[v]; k < vptr[v + 1]; k++) {
      int f = vel[k];
      if (f == e) continue;
      int cf = ((volatile int*)color)[f];
      if (cf < 0) {
        unsigned long long pf = mix64((unsigned long long)f);
        if (pf > pe || (pf == pe && f < e)) {
          atomicAdd(remaining, 1);
          return;
        }
      } else if (cf < 128) {
        used[cf >> 6] |= 1ull << (cf & 63);
      }
    }
  }
  int c;
  if (~used[0]) c = __ffsll((long long)~used[0]) - 1;
  else if (~used[1]) c = 64 + __ffsll((long long)~used[1]) - 1;
  else {
    atomicExch(err, DEV_ERR_COLORS);
    return;
  }
  color[e] = c;
}

// element geometry: gradients of the barycentric coordinates 1..3 (rows of
// the inverse Jacobian of the affine map) and the volume
__global__ void k_geometry(int ne, int nen, const int* __restrict__ conn,
                           const double* __restrict__ X, double* geo) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int* c = conn + (size_t)e * nen;
  double J[3][3];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) J[i][j] = X[3 * c[j + 1] + i] - X[3 * c[0] + i];
  double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  double id = 1.0 / det;
  // inverse = adj/det; row r of inverse = gradient of lambda_{r+1}
  double inv[3][3];
  inv[0][0] = c00 * id;
  inv[1][0] = c01 * id;
  inv[2][0] = c02 * id;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  double* g = geo + (size_t)e * 10;
  for (int r = 0; r < 3; r++)
    for (int i = 0; i < 3; i++) g[3 * r + i] = inv[r][i];
  g[9] = det / 6.0;
}

// position of block (conn[e][a], conn[e][b]) in the pattern (binary search)
__global__ void k_emap(int ne, int nen, int ncolk, const int* __restrict__ conn,
                       const int* __restrict__ ptr, const int* __restrict__ col, int* map,
                       int* err, int col_is_element) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = (int64_t)ne * nen * ncolk;
  if (t >= total) return;
  int e = (int)(t / (nen * ncolk));
  int ab = (int)(t % (nen * ncolk));
  int a = ab / ncolk, b = ab % ncolk;
  int r = conn[(size_t)e * nen + a];
  // u-p map: a vertex id (P1 pressure) or the element itself (P0)
  int c = col_is_element ? e : conn[(size_t)e * nen + b];
  int lo = ptr[r], hi = ptr[r + 1] - 1, pos = -1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int v = col[mid];
    if (v == c) {
      pos = mid;
      break;
    }
    if (v < c) lo = mid + 1;
    else hi = mid - 1;
  }
  if (pos < 0) {
    atomicExch(err, DEV_ERR_BOUNDS);
    pos = 0;
  }
  map[t] = pos;
}

__global__ void k_apply_dirichlet(int nn, const double* __restrict__ X, const uint8_t* __restrict__ dgroup,
                                  const fe_dirichlet_group* __restrict__ groups, double load,
                                  double* d) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nn) return;
  int g = dgroup[a];
  if (!g) return;
  fe_dirichlet_group G = groups[g - 1];
  double th = load * G.angle;
  double s, c;
  sincos(th, &s, &c);
  double x = X[3 * a] - G.center[0], y = X[3 * a + 1] - G.center[1];
  double T[3] = {G.center[0] + c * x - s * y + load * G.translation[0],
                 G.center[1] + s * x + c * y + load * G.translation[1],
                 X[3 * a + 2] + load * G.translation[2]};
  for (int k = 0; k < 3; k++)
    if ((G.comp_mask >> k) & 1u) d[3 * (size_t)a + k] = T[k] - X[3 * a + k];
}

// ---------------------------------------------------------------- host helpers
template <class T>
static int upload(fe_mesh m, T** dst, const std::vector<T>& src) {
  FE_TRY(fe_alloc_t(m, dst, src.size() ? src.size() : 1));
  if (!src.empty())
    FE_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice,
                            m->stream));
  return FE_OK;
}

static MatParams make_params(const fe_material& mt, double time) {
  MatParams p{};
  p.kind = mt.kind;
  if (mt.kind == FE_MAT_COOK_NH) {
    double mu = mt.E / (2.0 * (1.0 + mt.nu));
    double lam = 2.0 * mu * mt.nu / (1.0 - 2.0 * mt.nu);
    double kap = lam + 2.0 * mu / 3.0;
    p.mu = mu;
    p.cvol = mt.vol_literal ? kap : 0.25 * kap;
  } else if (mt.kind == FE_MAT_TH_NH) {
    p.mu = mt.mu;
  } else if (mt.kind == FE_MAT_POLYCONVEX) {
    p.ap = mt.alpha_p;
    p.bp = mt.beta_p;
    p.clog = mt.c_log;
  } else {
    p.C = mt.C;
    p.bf = mt.bf;
    p.bt = mt.bt;
    p.bfs = mt.bfs;
    p.kappa = mt.kappa;
    double s = sin(2.0 * M_PI * time / mt.period);
    p.gamma = mt.Ta_peak * (s > 0.0 ? s : 0.0);
  }
  return p;
}

// node rows -> sorted unique neighbour columns, from node -> element lists
static void build_rows(int nrow, const std::vector<int>& nptr, const std::vector<int>& nlist,
                       const std::vector<int>& conn, int nen, int cstride, int ncols_per_e,
                       std::vector<int>& ptr, std::vector<int>& col) {
  ptr.assign(nrow + 1, 0);
  col.clear();
  std::vector<int> buf;
  for (int a = 0; a < nrow; a++) {
    buf.clear();
    for (int k = nptr[a]; k < nptr[a + 1]; k++) {
      int e = nlist[k] / nen;
      for (int b = 0; b < ncols_per_e; b++) buf.push_back(conn[(size_t)e * cstride + b]);
    }
    std::sort(buf.begin(), buf.end());
    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    col.insert(col.end(), buf.begin(), buf.end());
    ptr[a + 1] = (int)col.size();
  }
}

static int validate(const fe_mesh_desc* d) {
  if (!d) return fe_set_error("desc is NULL"), FE_ERR_ARG;
  if (d->order != 1 && d->order != 2) return fe_set_error("order must be 1 or 2"), FE_ERR_ARG;
  if (d->pressure_order < 0 || d->pressure_order > 2)
    return fe_set_error("pressure_order must be 0, 1 (P1) or 2 (P0)"), FE_ERR_ARG;
  if (d->pressure_order != 0 &&
      (d->order != 2 || (d->material.kind != FE_MAT_TH_NH && d->material.kind != FE_MAT_POLYCONVEX)))
    return fe_set_error("a pressure space needs order 2 and the TH_NH or POLYCONVEX material"), FE_ERR_ARG;
  if (d->nv < 4 || d->ne < 1 || !d->coords || !d->tets)
    return fe_set_error("need nv >= 4, ne >= 1, coords and tets"), FE_ERR_ARG;
  if (d->material.kind < 0 || d->material.kind > 3) return fe_set_error("bad material kind"), FE_ERR_ARG;
  if (d->material.kind == FE_MAT_GUCCIONE && !d->fibers)
    return fe_set_error("GUCCIONE needs fibers"), FE_ERR_ARG;
  if (d->material.kind == FE_MAT_COOK_NH && !(d->material.nu < 0.5 && d->material.nu > -1.0))
    return fe_set_error("nu must lie in (-1, 0.5)"), FE_ERR_ARG;
  if (d->nf < 0 || (d->nf > 0 && (!d->faces || !d->face_kind || !d->face_data)))
    return fe_set_error("faces, face_kind and face_data are required when nf > 0"), FE_ERR_ARG;
  if (d->ngroups < 0 || (d->ngroups > 0 && !d->groups) || d->ngroups > 255)
    return fe_set_error("bad Dirichlet groups"), FE_ERR_ARG;
  for (int64_t i = 0; i < 4LL * d->ne; i++)
    if (d->tets[i] < 0 || d->tets[i] >= d->nv) return fe_set_error("tet vertex id out of range"), FE_ERR_ARG;
  for (int64_t i = 0; i < 3LL * d->nf; i++)
    if (d->faces[i] < 0 || d->faces[i] >= d->nv) return fe_set_error("face vertex id out of range"), FE_ERR_ARG;
  for (int i = 0; i < d->nf; i++)
    if (d->face_kind[i] < 0 || d->face_kind[i] > 5) return fe_set_error("bad face kind"), FE_ERR_ARG;
  for (int64_t i = 0; i < 3LL * d->nf; i++)
    if (!std::isfinite(d->face_data[i])) return fe_set_error("face data must be finite"), FE_ERR_ARG;
  if (d->dir_group)
    for (int i = 0; i < d->nv; i++)
      if (d->dir_group[i] > d->ngroups) return fe_set_error("dir_group id beyond ngroups"), FE_ERR_ARG;
  for (int e = 0; e < d->ne; e++) {
    const double* x0 = d->coords + 3 * (size_t)d->tets[4 * e];
    double J[3][3];
    for (int j = 0; j < 3; j++)
      for (int i = 0; i < 3; i++) J[i][j] = d->coords[3 * (size_t)d->tets[4 * e + j + 1] + i] - x0[i];
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                 J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                 J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (!(det > 0.0)) return fe_set_error("tet %d is not positively oriented", e), FE_ERR_ARG;
  }
  return FE_OK;
}

static const int kTetEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

static int create_impl(const fe_mesh_desc* desc, fe_mesh m) {
  const int nv = desc->nv, ne = desc->ne;
  m->order = desc->order;
  m->pres = desc->pressure_order;
  m->nv = nv;
  m->ne = ne;
  m->nen = m->order == 1 ? 4 : 10;
  m->nq = m->order == 1 ? 1 : 4;
  m->mat = desc->material;
  m->mp = make_params(m->mat, 0.0);
  m->device = desc->device;
  m->stream = (cudaStream_t)desc->stream;
  FE_CUDA(cudaSetDevice(m->device));
  cudaDeviceProp prop;
  FE_CUDA(cudaGetDeviceProperties(&prop, m->device));
  m->sm_count = prop.multiProcessorCount;

  // ---- P2 edge nodes: unique (min, max) vertex pairs in ascending order
  std::vector<uint64_t> ekeys;
  if (m->order == 2) {
    ekeys.resize((size_t)ne * 6);
    for (int e = 0; e < ne; e++)
      for (int k = 0; k < 6; k++) {
        uint64_t a = (uint64_t)desc->tets[4 * e + kTetEdge[k][0]];
        uint64_t b = (uint64_t)desc->tets[4 * e + kTetEdge[k][1]];
        ekeys[(size_t)e * 6 + k] = (std::min(a, b) << 32) | std::max(a, b);
      }
    std::sort(ekeys.begin(), ekeys.end());
    ekeys.erase(std::unique(ekeys.begin(), ekeys.end()), ekeys.end());
  }
  auto edge_id = [&](int a, int b) -> int {
    uint64_t key = ((uint64_t)std::min(a, b) << 32) | (uint64_t)std::max(a, b);
    auto it = std::lower_bound(ekeys.begin(), ekeys.end(), key);
    if (it == ekeys.end() || *it != key) return -1;  // not an edge of the mesh
    return nv + (int)(it - ekeys.begin());
  };
  const int nn = nv + (int)ekeys.size();
  m->nn = nn;
  m->np = m->pres == 1 ? nv : (m->pres == 2 ? ne : 0);  // P1: vertex values; P0: one per element
  m->ndof = 3LL * nn + m->np;
  std::vector<int> conn((size_t)ne * m->nen);
  for (int e = 0; e < ne; e++) {
    for (int a = 0; a < 4; a++) conn[(size_t)e * m->nen + a] = desc->tets[4 * e + a];
    if (m->order == 2)
      for (int k = 0; k < 6; k++)
        conn[(size_t)e * m->nen + 4 + k] =
            edge_id(desc->tets[4 * e + kTetEdge[k][0]], desc->tets[4 * e + kTetEdge[k][1]]);
  }
  std::vector<double> X((size_t)nn * 3);
  std::memcpy(X.data(), desc->coords, sizeof(double) * 3 * nv);
  for (size_t k = 0; k < ekeys.size(); k++) {
    int a = (int)(ekeys[k] >> 32), b = (int)(ekeys[k] & 0xffffffffu);
    for (int i = 0; i < 3; i++) X[3 * (nv + k) + i] = 0.5 * (desc->coords[3 * a + i] + desc->coords[3 * b + i]);
  }
  // Dirichlet groups: an edge node belongs to the common group of its ends
  std::vector<uint8_t> dgroup(nn, 0), fixmask(nn, 0);
  for (int a = 0; a < nv; a++) dgroup[a] = desc->dir_group ? desc->dir_group[a] : 0;
  for (size_t k = 0; k < ekeys.size(); k++) {
    int a = (int)(ekeys[k] >> 32), b = (int)(ekeys[k] & 0xffffffffu);
    if (dgroup[a] && dgroup[a] == dgroup[b]) dgroup[nv + k] = dgroup[a];
  }
  m->ngroups = desc->ngroups;
  m->groups.assign(desc->groups, desc->groups + desc->ngroups);
  for (int a = 0; a < nn; a++)
    if (dgroup[a]) fixmask[a] = (uint8_t)(m->groups[dgroup[a] - 1].comp_mask & 7u);

  // ---- node -> (element, local) lists; vertex -> element lists
  std::vector<int> nptr(nn + 1, 0), nlist((size_t)ne * m->nen);
  for (size_t t = 0; t < conn.size(); t++) nptr[conn[t] + 1]++;
  for (int a = 0; a < nn; a++) nptr[a + 1] += nptr[a];
  {
    std::vector<int> fill(nptr.begin(), nptr.end() - 1);
    for (int e = 0; e < ne; e++)
      for (int a = 0; a < m->nen; a++) nlist[fill[conn[(size_t)e * m->nen + a]]++] = e * m->nen + a;
  }
  std::vector<int> vptr(nv + 1, 0), vlist((size_t)ne * 4), vel((size_t)ne * 4);
  for (int e = 0; e < ne; e++)
    for (int a = 0; a < 4; a++) vptr[desc->tets[4 * e + a] + 1]++;
  for (int v = 0; v < nv; v++) vptr[v + 1] += vptr[v];
  {
    std::vector<int> fill(vptr.begin(), vptr.end() - 1);
    for (int e = 0; e < ne; e++)
      for (int a = 0; a < 4; a++) {
        int v = desc->tets[4 * e + a];
        int slot = fill[v]++;
        vlist[slot] = e * 4 + a;
        vel[slot] = e;
      }
  }

  // ---- block pattern (one block per node pair sharing an element)
  std::vector<int> row_ptr, col;
  build_rows(nn, nptr, nlist, conn, m->nen, m->nen, m->nen, row_ptr, col);
  m->nnzb = (int64_t)col.size();
  std::vector<int> diag(nn);
  for (int a = 0; a < nn; a++)
    diag[a] = (int)(std::lower_bound(col.begin() + row_ptr[a], col.begin() + row_ptr[a + 1], a) - col.begin());
  std::vector<int> up_ptr, up_col, pu_ptr, pu_col, pu_src;
  if (m->pres) {
    if (m->pres == 1) {
      build_rows(nn, nptr, nlist, conn, m->nen, m->nen, 4, up_ptr, up_col);  // columns: the element's vertices
    } else {
      std::vector<int> eid(ne);
      for (int e = 0; e < ne; e++) eid[e] = e;
      build_rows(nn, nptr, nlist, eid, m->nen, 1, 1, up_ptr, up_col);  // columns: the element itself
    }
    m->nnz_up = (int64_t)up_col.size();
    // transpose: pressure rows, u-node columns, with the index of the source entry
    pu_ptr.assign(m->np + 1, 0);
    for (int64_t k = 0; k < m->nnz_up; k++) pu_ptr[up_col[k] + 1]++;
    for (int v = 0; v < m->np; v++) pu_ptr[v + 1] += pu_ptr[v];
    pu_col.resize(m->nnz_up);
    pu_src.resize(m->nnz_up);
    std::vector<int> fill(pu_ptr.begin(), pu_ptr.end() - 1);
    for (int a = 0; a < nn; a++)
      for (int k = up_ptr[a]; k < up_ptr[a + 1]; k++) {
        int s = fill[up_col[k]]++;
        pu_col[s] = a;
        pu_src[s] = k;
      }
  }

  // ---- boundary data: dead loads at load 1 and the spring matrix
  //   triangle integrals: P1 int phi_a = A/3, M_ab = A(1+delta_ab)/12;
  //   P2 (vertices 0..2, edges (0,1),(1,2),(2,0)): int phi_vertex = 0,
  //   int phi_edge = A/3, M = A/180 [6 on vertex diagonal, -1 vertex-vertex,
  //   -4 vertex-opposite edge, 0 vertex-adjacent edge, 32 edge diagonal,
  //   16 edge-edge]
  // Face pattern: node pairs of the faces of kinds 2 (springs), 3 (follower
  // pressure) and 4 (dashpots); springs and dashpots keep separate values.
  struct FaceBlock {
    std::array<double, 9> spring{}, dashpot{};
    std::vector<int> follower;  // face * 64 + a * 8 + b
  };
  std::vector<double> fext((size_t)nn * 3, 0.0);
  std::map<std::pair<int, int>, FaceBlock> fpat;
  std::vector<int> ff_nodes, ff_kind, fn_count(nn, 0);
  std::vector<double> ff_data;
  for (int f = 0; f < desc->nf; f++) {
    const int* v = desc->faces + 3 * f;
    const double* x0 = desc->coords + 3 * (size_t)v[0];
    const double* x1 = desc->coords + 3 * (size_t)v[1];
    const double* x2 = desc->coords + 3 * (size_t)v[2];
    double a[3] = {x1[0] - x0[0], x1[1] - x0[1], x1[2] - x0[2]};
    double b[3] = {x2[0] - x0[0], x2[1] - x0[1], x2[2] - x0[2]};
    double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    double ln = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(ln > 0.0)) return fe_set_error("face %d is degenerate", f), FE_ERR_ARG;
    double A = 0.5 * ln;
    double N[3] = {n[0] / ln, n[1] / ln, n[2] / ln};
    int nodes[6];
    int nfn = m->order == 1 ? 3 : 6;
    for (int k = 0; k < 3; k++) nodes[k] = v[k];
    if (m->order == 2)
      for (int k = 0; k < 3; k++) {
        nodes[3 + k] = edge_id(v[k], v[(k + 1) % 3]);
        if (nodes[3 + k] < 0) return fe_set_error("face %d is not a face of the mesh", f), FE_ERR_ARG;
      }
    double intphi[6], M[6][6];
    for (int p = 0; p < nfn; p++)
      for (int q = 0; q < nfn; q++) {
        if (m->order == 1) {
          M[p][q] = A * (p == q ? 2.0 : 1.0) / 12.0;
        } else {
          double c;
          if (p < 3 && q < 3) c = (p == q) ? 6.0 : -1.0;
          else if (p >= 3 && q >= 3) c = (p == q) ? 32.0 : 16.0;
          else {
            int vtx = p < 3 ? p : q, ed = (p < 3 ? q : p) - 3;
            c = ((ed + 2) % 3 == vtx) ? -4.0 : 0.0;  // edge (k, k+1) is opposite vertex k+2
          }
          M[p][q] = A * c / 180.0;
        }
      }
    for (int p = 0; p < nfn; p++) intphi[p] = m->order == 1 ? A / 3.0 : (p < 3 ? 0.0 : A / 3.0);
    const double* fd = desc->face_data + 3 * f;
    int kind = desc->face_kind[f];
    if (kind == FE_FACE_TRACTION || kind == FE_FACE_PRESSURE) {
      double t[3];
      for (int i = 0; i < 3; i++) t[i] = kind == FE_FACE_TRACTION ? fd[i] : -fd[0] * N[i];
      for (int p = 0; p < nfn; p++)
        for (int i = 0; i < 3; i++) fext[3 * (size_t)nodes[p] + i] += t[i] * intphi[p];
    } else if (kind == FE_FACE_FOLLOWER || kind == FE_FACE_TRACTION_DEFORMED) {
      int ff = (int)ff_kind.size();
      ff_kind.push_back(kind);
      for (int i = 0; i < 3; i++) ff_data.push_back(fd[i]);
      for (int p = 0; p < 6; p++) ff_nodes.push_back(p < nfn ? nodes[p] : nodes[0]);
      for (int p = 0; p < nfn; p++) {
        fn_count[nodes[p]]++;
        for (int q = 0; q < nfn; q++) fpat[{nodes[p], nodes[q]}].follower.push_back(ff * 64 + p * 8 + q);
      }
    } else {  // springs or dashpots: (c_perp N x N + c_par (I - N x N)) times the face mass
      double Ks[9];
      for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) Ks[3 * i + k] = fd[0] * N[i] * N[k] + fd[1] * ((i == k) - N[i] * N[k]);
      for (int p = 0; p < nfn; p++)
        for (int q = 0; q < nfn; q++) {
          FaceBlock& fb = fpat[{nodes[p], nodes[q]}];
          auto& blk = kind == FE_FACE_ROBIN ? fb.spring : fb.dashpot;
          for (int k = 0; k < 9; k++) blk[k] += M[p][q] * Ks[k];
        }
      if (kind == FE_FACE_DASHPOT) m->has_dashpots = true;
    }
  }
  std::vector<int> ks_ptr(nn + 1, 0), ks_col, ks_kpos, fk_ptr(1, 0), fk_list;
  for (auto& kv : fpat) {
    ks_ptr[kv.first.first + 1]++;
    ks_col.push_back(kv.first.second);
    m->h_ks_spring.insert(m->h_ks_spring.end(), kv.second.spring.begin(), kv.second.spring.end());
    m->h_ks_dashpot.insert(m->h_ks_dashpot.end(), kv.second.dashpot.begin(), kv.second.dashpot.end());
    fk_list.insert(fk_list.end(), kv.second.follower.begin(), kv.second.follower.end());
    fk_ptr.push_back((int)fk_list.size());
    int a = kv.first.first, b = kv.first.second;
    ks_kpos.push_back((int)(std::lower_bound(col.begin() + row_ptr[a], col.begin() + row_ptr[a + 1], b) - col.begin()));
  }
  for (int a = 0; a < nn; a++) ks_ptr[a + 1] += ks_ptr[a];
  m->nnz_ks = (int64_t)ks_col.size();
  m->nff = (int)ff_kind.size();
  std::vector<int> fn_ptr(nn + 1, 0), fn_list;
  if (m->nff) {  // node -> (follower face, local node), faces in order
    for (int a = 0; a < nn; a++) fn_ptr[a + 1] = fn_ptr[a] + fn_count[a];
    fn_list.resize(fn_ptr[nn]);
    std::vector<int> fill(fn_ptr.begin(), fn_ptr.end() - 1);
    int nfn = m->order == 1 ? 3 : 6;
    for (int ff = 0; ff < m->nff; ff++)
      for (int p = 0; p < nfn; p++) fn_list[fill[ff_nodes[6 * ff + p]]++] = ff * 8 + p;
  }

  // ---- uploads
  FE_TRY(upload(m, &m->X, X));
  FE_TRY(upload(m, &m->conn, conn));
  FE_TRY(upload(m, &m->row_ptr, row_ptr));
  {  // column indices padded to whole 32-block tiles: the SpMV copies them tile by tile
    std::vector<int> colp(col);
    colp.resize((col.size() + 31) / 32 * 32, 0);
    FE_TRY(upload(m, &m->col, colp));
  }
  FE_TRY(upload(m, &m->diag_pos, diag));
  FE_TRY(upload(m, &m->dgroup, dgroup));
  FE_TRY(upload(m, &m->fixmask, fixmask));
  FE_TRY(upload(m, &m->d_groups, m->groups));
  FE_TRY(upload(m, &m->node_ptr, nptr));
  FE_TRY(upload(m, &m->node_list, nlist));
  FE_TRY(upload(m, &m->fext1, fext));
  FE_TRY(upload(m, &m->ks_ptr, ks_ptr));
  FE_TRY(upload(m, &m->ks_col, ks_col));
  FE_TRY(fe_upload_face_values(m));
  FE_TRY(upload(m, &m->ks_kpos, ks_kpos));
  if (m->nff) {
    FE_TRY(upload(m, &m->ff_nodes, ff_nodes));
    FE_TRY(upload(m, &m->ff_kind, ff_kind));
    FE_TRY(upload(m, &m->ff_data, ff_data));
    FE_TRY(upload(m, &m->fn_ptr, fn_ptr));
    FE_TRY(upload(m, &m->fn_list, fn_list));
    FE_TRY(upload(m, &m->fk_ptr, fk_ptr));
    FE_TRY(upload(m, &m->fk_list, fk_list));
  }
  if (m->pres) {
    FE_TRY(upload(m, &m->up_ptr, up_ptr));
    FE_TRY(upload(m, &m->up_col, up_col));
    FE_TRY(upload(m, &m->pu_ptr, pu_ptr));
    FE_TRY(upload(m, &m->pu_col, pu_col));
    FE_TRY(upload(m, &m->pu_src, pu_src));
    if (m->pres == 1) {  // pressure residual gather: vertex -> (element, local vertex) slots
      FE_TRY(upload(m, &m->vert_ptr, vptr));
      FE_TRY(upload(m, &m->vert_list, vlist));
    } else {  // P0: element e's pressure residual sits in its slot 0
      std::vector<int> pptr(ne + 1), plist(ne);
      for (int e = 0; e <= ne; e++) pptr[e] = e;
      for (int e = 0; e < ne; e++) plist[e] = 4 * e;
      FE_TRY(upload(m, &m->vert_ptr, pptr));
      FE_TRY(upload(m, &m->vert_list, plist));
    }
  }
  if (desc->fibers) {
    std::vector<double> fib(desc->fibers, desc->fibers + 9 * (size_t)ne);
    FE_TRY(upload(m, &m->fib, fib));
  }

  FE_TRY(fe_alloc_t(m, &m->bar, BAR_WORDS));
  FE_TRY(fe_reset_grid_sync(m));
  FE_TRY(fe_alloc_t(m, &m->red, RED_SLOTS));
  FE_TRY(fe_alloc_t(m, &m->red_ticket, 4));
  FE_CUDA(cudaMemsetAsync(m->red_ticket, 0, 4 * sizeof(unsigned), m->stream));
  FE_TRY(fe_alloc_t(m, &m->scal, SCAL_N));
  FE_CUDA(cudaMemsetAsync(m->scal, 0, SCAL_N * sizeof(double), m->stream));
  m->err = (int*)(m->scal + SCAL_N - 1);  // read back together with the solver scalars
  FE_CUDA(cudaMallocHost(&m->h_scal, SCAL_N * sizeof(double)));
  FE_TRY(fe_alloc_t(m, &m->rel, (size_t)ne * m->nen * 3));
  if (m->pres) FE_TRY(fe_alloc_t(m, &m->relp, (size_t)ne * 4));

  // ---- device work: geometry, colouring, block maps
  FE_TRY(fe_alloc_t(m, &m->geo, (size_t)ne * 10));
  {
    FE_SCOPE(m, FE_PROF_OTHER, 0);
    k_geometry<<<(ne + 127) / 128, 128, 0, m->stream>>>(ne, m->nen, m->conn, m->X, m->geo);
  }
  FE_CUDA(cudaGetLastError());

  int *d_vptr = nullptr, *d_vel = nullptr, *d_rem = nullptr;
  FE_TRY(upload(m, &d_vptr, vptr));
  FE_TRY(upload(m, &d_vel, vel));
  FE_TRY(fe_alloc_t(m, &d_rem, 1));
  FE_TRY(fe_alloc_t(m, &m->colors, ne));
  FE_CUDA(cudaMemsetAsync(m->colors, 0xff, sizeof(int) * ne, m->stream));
  for (int round = 0; round <= ne; round++) {
    FE_CUDA(cudaMemsetAsync(d_rem, 0, sizeof(int), m->stream));
    {
      FE_SCOPE(m, FE_PROF_OTHER, 0);
      k_jp_round<<<(ne + 255) / 256, 256, 0, m->stream>>>(ne, m->nen, m->conn, d_vptr, d_vel, m->colors,
                                                          d_rem, m->err);
    }
    FE_CUDA(cudaGetLastError());
    int rem = 0;
    FE_CUDA(cudaMemcpyAsync(&rem, d_rem, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    FE_CUDA(cudaStreamSynchronize(m->stream));
    if (rem == 0) break;
  }
  FE_TRY(fe_check_device_error(m));
  cudaFreeAsync(d_vptr, m->stream);
  cudaFreeAsync(d_vel, m->stream);
  cudaFreeAsync(d_rem, m->stream);
  m->device_bytes -= (int64_t)(vptr.size() + vel.size() + 1) * sizeof(int);
  std::vector<int> colors(ne);
  FE_CUDA(cudaMemcpy(colors.data(), m->colors, sizeof(int) * ne, cudaMemcpyDeviceToHost));
  int nc = 0;
  for (int e = 0; e < ne; e++) nc = std::max(nc, colors[e] + 1);
  m->ncolors = nc;
  m->h_color_start.assign(nc + 1, 0);
  for (int e = 0; e < ne; e++) m->h_color_start[colors[e] + 1]++;
  for (int c = 0; c < nc; c++) m->h_color_start[c + 1] += m->h_color_start[c];
  std::vector<int> perm(ne);
  {
    std::vector<int> fill(m->h_color_start.begin(), m->h_color_start.end() - 1);
    for (int e = 0; e < ne; e++) perm[fill[colors[e]]++] = e;
  }
  FE_TRY(upload(m, &m->perm, perm));

  int64_t tot = (int64_t)ne * m->nen * m->nen;
  FE_TRY(fe_alloc_t(m, &m->emap, (size_t)tot));
  {
    FE_SCOPE(m, FE_PROF_OTHER, 0);
    k_emap<<<(unsigned)((tot + 255) / 256), 256, 0, m->stream>>>(ne, m->nen, m->nen, m->conn, m->row_ptr,
                                                                 m->col, m->emap, m->err, 0);
  }
  FE_CUDA(cudaGetLastError());
  if (m->pres) {
    const int npl = m->pres == 2 ? 1 : 4;  // local pressure values per element
    int64_t tu = (int64_t)ne * m->nen * npl;
    FE_TRY(fe_alloc_t(m, &m->upmap, (size_t)tu));
    FE_SCOPE(m, FE_PROF_OTHER, 0);
    k_emap<<<(unsigned)((tu + 255) / 256), 256, 0, m->stream>>>(ne, m->nen, npl, m->conn, m->up_ptr,
                                                                m->up_col, m->upmap, m->err, m->pres == 2);
    FE_CUDA(cudaGetLastError());
  }
  FE_TRY(fe_check_device_error(m));
  return FE_OK;
}

static void free_all(fe_mesh m) {
  fe_amg_free(m);
  prof_resolve(m);
  for (cudaEvent_t e : m->ev_free) cudaEventDestroy(e);
  m->ev_free.clear();
  void* ptrs[] = {m->X, m->conn, m->colors, m->perm, m->geo, m->fib, m->fixmask, m->dgroup,
                  m->d_groups, m->row_ptr, m->col, m->diag_pos, m->emap, m->up_ptr, m->up_col,
                  m->upmap, m->pu_ptr, m->pu_col, m->pu_src, m->node_ptr, m->node_list,
                  m->vert_ptr, m->vert_list, m->fext1, m->ks_ptr, m->ks_col, m->ks_val,
                  m->ks_kpos, m->K64, m->K32, m->K16, m->B64, m->B32, m->Dinv64, m->Dinv32,
                  m->Sd, m->rel, m->relp, m->red, m->red_ticket, m->scal, m->bar, m->V,
                  m->H, m->gv, m->w64, m->t64, m->u64, m->zx, m->S, m->Yv, m->nl_R, m->nl_Rn,
                  m->nl_dl, m->nl_t, m->rho_d, m->lb_x, m->alpha_d, m->Lmat, m->hpub, m->partv, m->Tbm,
                  m->ff_nodes, m->ff_kind, m->ff_data, m->fn_ptr, m->fn_list, m->fk_ptr, m->fk_list, m->kc_val,
                  m->dyn_keep};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, m->stream);
  cudaStreamSynchronize(m->stream);
  if (m->h_scal) cudaFreeHost(m->h_scal);
}

extern "C" int fe_mesh_create(const fe_mesh_desc* desc, fe_mesh* out) {
  if (!out) return fe_set_error("out is NULL"), FE_ERR_ARG;
  *out = nullptr;
  FE_TRY(validate(desc));
  fe_mesh m = new fe_mesh_s();
  int rc = create_impl(desc, m);
  // bring the fixed array of fe_spmv_noalloc and the kernels it launches
  // into memory now, while allocating is allowed (see fe_noalloc.cu)
  if (rc == FE_OK) rc = fe_noalloc_prepare(m);
  if (rc != FE_OK) {
    free_all(m);
    delete m;
    return rc;
  }
  *out = m;
  return FE_OK;
}

extern "C" int fe_set_pc(fe_mesh m, int pc_type) {
  if (!m) return fe_set_error("NULL mesh"), FE_ERR_ARG;
  if (pc_type < 0 || pc_type > 2)
    return fe_set_error("pc_type must be 0 (block-Jacobi), 1 (AMG) or 2 (AMG, BF16 fine-level smoother)"), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  const bool rebuild = pc_type >= 1 && m->pc_type != pc_type && m->prec >= 0;
  m->pc_type = pc_type;
  if (rebuild) FE_TRY(fe_amg_setup(m));  // a tangent is assembled already
  return FE_OK;
}

extern "C" int fe_set_wait_limit(fe_mesh m, int64_t polls) {
  if (!m) return fe_set_error("NULL mesh"), FE_ERR_ARG;
  if (polls > (int64_t)UINT32_MAX) return fe_set_error("polls must be < 2^32"), FE_ERR_ARG;
  m->wait_limit = polls < 0 ? (1u << 26) : (unsigned)polls;
  return FE_OK;
}

extern "C" int fe_mesh_destroy(fe_mesh m) {
  if (!m) return FE_OK;
  cudaSetDevice(m->device);
  cudaStreamSynchronize(m->stream);
  free_all(m);
  delete m;
  return FE_OK;
}

extern "C" int fe_mesh_get_info(fe_mesh m, fe_mesh_info* out) {
  if (!m || !out) return fe_set_error("NULL argument"), FE_ERR_ARG;
  out->order = m->order;
  out->pressure_order = m->pres;
  out->nv = m->nv;
  out->ne = m->ne;
  out->nn = m->nn;
  out->np = m->np;
  out->ndof = m->ndof;
  out->nen = m->nen;
  out->nnzb = m->nnzb;
  out->nnz_up = m->nnz_up;
  out->ncolors = m->ncolors;
  out->device_bytes = m->device_bytes;
  return FE_OK;
}

extern "C" int fe_mesh_get_topology(fe_mesh m, int32_t* conn, int32_t* colors, int32_t* row_ptr,
                                    int32_t* col, double* node_coords) {
  if (!m) return fe_set_error("NULL mesh"), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  if (conn) FE_CUDA(cudaMemcpy(conn, m->conn, sizeof(int) * (size_t)m->ne * m->nen, cudaMemcpyDeviceToHost));
  if (colors) FE_CUDA(cudaMemcpy(colors, m->colors, sizeof(int) * (size_t)m->ne, cudaMemcpyDeviceToHost));
  if (row_ptr) FE_CUDA(cudaMemcpy(row_ptr, m->row_ptr, sizeof(int) * (size_t)(m->nn + 1), cudaMemcpyDeviceToHost));
  if (col) FE_CUDA(cudaMemcpy(col, m->col, sizeof(int) * (size_t)m->nnzb, cudaMemcpyDeviceToHost));
  if (node_coords) FE_CUDA(cudaMemcpy(node_coords, m->X, sizeof(double) * 3 * (size_t)m->nn, cudaMemcpyDeviceToHost));
  return FE_OK;
}

extern "C" int fe_set_load(fe_mesh m, double load, double time) {
  if (!m) return fe_set_error("NULL mesh"), FE_ERR_ARG;
  if (!std::isfinite(load) || !std::isfinite(time)) return fe_set_error("load/time not finite"), FE_ERR_ARG;
  m->load = load;
  m->time = time;
  m->mp = make_params(m->mat, time);
  return FE_OK;
}

extern "C" int fe_apply_dirichlet(fe_mesh m, double* d) {
  if (!m || !d) return fe_set_error("NULL argument"), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  if (m->ngroups == 0) return FE_OK;
  {
    FE_SCOPE(m, FE_PROF_VECTOR, 0);
    k_apply_dirichlet<<<(m->nn + 255) / 256, 256, 0, m->stream>>>(m->nn, m->X, m->dgroup, m->d_groups,
                                                                  m->load, d);
  }
  FE_CUDA(cudaGetLastError());
  FE_CUDA(cudaStreamSynchronize(m->stream));
  return FE_OK;
}
