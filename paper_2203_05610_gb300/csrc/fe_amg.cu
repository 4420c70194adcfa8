// fe_amg.cu -- smoothed-aggregation algebraic multigrid (AMG) on the nodal
// blocks, as the preconditioner of the displacement block.
//
// The paper preconditions its Krylov solves with algebraic multigrid on
// blocks of size 3 (BoomerAMG with bs = 3, Section "Test problems and
// solvers details" and Appendix A) without describing it; this is a
// smoothed-aggregation V-cycle of that class:
//   - aggregation on the block graph of A_l (nodes whose components are all
//     absent -- Dirichlet at level 0 -- left out, no strength filter): roots
//     = greedy maximal distance-2 independent set in descending
//     splitmix64(node) priority, ties by id; a root takes its neighbours;
//     every other node joins the aggregate of its smallest-id neighbour
//     taken so; aggregates numbered by root id;
//   - near null space: the six rigid motions (translations, rotations
//     (-y, x, 0), (0, -z, y), (z, 0, -x)); tentative prolongator T by
//     modified Gram-Schmidt QR of each aggregate's rows (columns left with
//     <= 1e-8 of their norm are dropped and that coarse component is
//     absent); coarse nodes carry 6 components;
//   - P = (I - omega D^-1 A) T, omega = 4 / (3 rho), rho from 15 power steps
//     on D^-1 A (D the block diagonal) from x_k = u(splitmix64(k)) - 1/2;
//   - Galerkin A_{l+1} = P^T A_l P, absent components with a unit diagonal;
//   - Chebyshev smoothing of degree 2 in D^-1 A on [rho/30, 1.1 rho] before
//     and after the coarse correction; exact solve on the coarsest level
//     (<= 16 nodes) with the inverse from Gauss-Jordan elimination.
//
// GB300 design.  Everything that depends only on the mesh -- the
// aggregates, T (rigid motions at the node coordinates), the patterns of P,
// A P, P^T and every coarse operator, and the index lists of the Galerkin
// products -- is built once per mesh on the host (native C++, like the
// mesh's own block pattern) and kept resident.  What depends on the
// tangent's values runs on the device after every assembly: block
// inverses, power iterations, P, A P, P^T A P and the coarsest inverse,
// each output entry computed by one thread from a fixed gather list (no
// atomics: deterministic, and the same summation order as a plain loop).
// The numbers are formed in FP64 for an FP64 tangent and in FP32 for the
// mixed forms (GB300's FP32 rate is tens of times its FP64 rate); the
// V-cycle runs in the tangent's precision (FP32 values, vectors and
// accumulation in the mixed forms), the coarsest inverse is formed in FP64.  A
// Chebyshev step is one fused kernel: the SpMV with A_l, the residual update,
// the block-Jacobi product and the direction and iterate updates of its
// rows (r stays b - A x throughout, so the residual for the restriction
// comes for free); level 0 reads the tangent in its tiled layout, coarser
// levels their 6x6 blocks block-major with 16-byte loads.  The levels of at
// most a few hundred nodes below level 0 run in one block (one launch
// instead of seven or more latency-bound ones), and the whole V-cycle is
// captured as one CUDA graph.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <numeric>
#include <type_traits>
#include <vector>

#include "fe_internal.h"

namespace {

constexpr int AMG_MAXLEV = 12;
constexpr int AMG_COARSE = 16;   // the coarsest level has at most this many nodes
constexpr int AMG_NS = 6;        // near null space vectors
constexpr int AMG_DENSE_MAX = 96;
constexpr int AMG_POWER_STEPS = 15;
constexpr double AMG_QR_DROP = 1e-8;
constexpr int AMG_RED_BLOCKS = 256;

uint64_t mix64(uint64_t z) {  // splitmix64 (Steele, Lea and Flood; Vigna's constants)
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t mix64_d(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace

struct AmgLevel {
  int n = 0, b = 3, nc = 0;
  int64_t nnz = 0, nnzp = 0, nnzap = 0, nnzr = 0;
  // structure (device)
  const int* ptr = nullptr;  // A_l pattern (level 0: the mesh's)
  const int* col = nullptr;
  const int* diag = nullptr; // [n] diagonal block positions
  int* own = nullptr;        // one allocation holding this level's int arrays
  unsigned char* absent = nullptr;
  int *agg = nullptr, *pptr = nullptr, *pcol = nullptr, *prow = nullptr;
  int *rptr = nullptr, *rcol = nullptr, *rsrc = nullptr;
  int *apptr = nullptr, *apcol = nullptr, *aprow = nullptr;
  int* crow = nullptr;       // row of each entry of A_l (level >= 1)
  double* tnode = nullptr;   // [n][b*6] tentative block of each node
  // numbers (device)
  double* val64 = nullptr;  // level >= 1: [nnz][b*b]
  float* val32 = nullptr;
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  double *p64 = nullptr, *r64 = nullptr, *ap64 = nullptr;
  float *p32 = nullptr, *r32 = nullptr, *ap32 = nullptr;
  double* inv64 = nullptr;
  float* inv32 = nullptr;
  double rho = 0.0;
  double* pt64 = nullptr;    // tiled V-cycle copy of P_l
  float* pt32 = nullptr;
  double* coef64 = nullptr;  // Chebyshev coefficients {1/theta, c1, c2} in device memory, so
  float* coef32 = nullptr;   // a captured V-cycle stays valid when a new tangent changes them
  // V-cycle vectors [n*b] in the V-cycle precision
  void *x = nullptr, *r = nullptr, *d0 = nullptr, *d1 = nullptr, *e = nullptr;
};

struct AmgHier {
  int nlev = 0;
  AmgLevel lev[AMG_MAXLEV];
  int vec_elem = 0;          // bytes per V-cycle vector element allocated (0: none yet)
  double* pw = nullptr;      // power iterations: x, y [2][max n*b]
  double* part = nullptr;    // [2][AMG_RED_BLOCKS] partial sums
  double* scal = nullptr;    // [4] rho, 1/|y|
  std::vector<void*> allocs; // device buffers owned by the hierarchy
  int64_t bytes = 0;         // their size (counted in the mesh's device bytes)
  bool ready = false;        // numbers formed for the current tangent
  // the V-cycle captured as a CUDA graph: input vin (FP64), output lev[0].x
  double* vin = nullptr;
  cudaStream_t cap = nullptr;       // capture stream (the mesh's may be the legacy stream)
  cudaGraphExec_t exec = nullptr;
  int exec_prec = -1;               // tangent precision the graph was captured for
  double vc_bytes = 0, vc_flops = 0; // algorithmic bytes and flops of one V-cycle
  unsigned grid0 = 0;               // one wave of the streamed level-0 kernel
};

namespace {

// ---------------------------------------------------------------- host structure
struct HostLevel {
  int n = 0, b = 3, nc = 0;
  std::vector<int> ptr, col, diag;
  std::vector<uint8_t> absent;
  std::vector<double> ns;  // [n*b][6]
  std::vector<int> agg, pptr, pcol, rptr, rcol, rsrc, apptr, apcol;
  std::vector<double> tnode;  // [n][b*6]
};

uint8_t full_mask(int b) { return (uint8_t)((1u << b) - 1u); }

// sorted unique values of v[beg, end) appended to out; returns the new size
void sort_unique(std::vector<int>& tmp) {
  std::sort(tmp.begin(), tmp.end());
  tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
}

void aggregate(HostLevel& L) {
  const int n = L.n;
  const uint8_t full = full_mask(L.b);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::vector<uint64_t> pri(n);
  for (int i = 0; i < n; i++) pri[i] = mix64((uint64_t)i);
  std::sort(order.begin(), order.end(), [&](int a, int c) { return pri[a] != pri[c] ? pri[a] > pri[c] : a < c; });
  std::vector<int> root(n, -1);  // root whose neighbourhood took the node
  for (int i : order) {
    if (L.absent[i] == full || root[i] >= 0) continue;
    bool taken = false;
    for (int k = L.ptr[i]; k < L.ptr[i + 1] && !taken; k++) {
      const int j = L.col[k];
      taken = j != i && L.absent[j] != full && root[j] >= 0;
    }
    if (taken) continue;
    for (int k = L.ptr[i]; k < L.ptr[i + 1]; k++)
      if (L.absent[L.col[k]] != full) root[L.col[k]] = i;
    root[i] = i;
  }
  std::vector<int> id(n, -1);
  L.nc = 0;
  for (int i = 0; i < n; i++)
    if (root[i] == i) id[i] = L.nc++;
  L.agg.assign(n, -1);
  for (int i = 0; i < n; i++)
    if (root[i] >= 0) L.agg[i] = id[root[i]];
  for (int i = 0; i < n; i++) {  // nodes at distance 2 from every root
    if (L.absent[i] == full || root[i] >= 0) continue;
    for (int k = L.ptr[i]; k < L.ptr[i + 1]; k++) {
      const int j = L.col[k];
      if (j != i && root[j] >= 0) {
        L.agg[i] = id[root[j]];
        break;
      }
    }
  }
}

// T per node, coarse near null space and absent components, all patterns
// of the level's products and the coarse level's pattern
void coarsen(HostLevel& L, HostLevel& C) {
  const int n = L.n, nc = L.nc, b = L.b, K = AMG_NS;
  std::vector<std::vector<int>> members(nc);
  for (int i = 0; i < n; i++)
    if (L.agg[i] >= 0) members[L.agg[i]].push_back(i);
  C.n = nc;
  C.b = K;
  C.absent.assign(nc, 0);
  C.ns.assign((size_t)nc * K * K, 0.0);
  L.tnode.assign((size_t)n * b * K, 0.0);
  std::vector<double> Q;
  for (int a = 0; a < nc; a++) {
    const std::vector<int>& mem = members[a];
    const int rows = (int)mem.size() * b;
    Q.assign((size_t)rows * K, 0.0);  // column c at Q[c * rows ...]
    for (size_t s = 0; s < mem.size(); s++)
      for (int i = 0; i < b; i++)
        for (int c = 0; c < K; c++) Q[(size_t)c * rows + s * b + i] = L.ns[((size_t)mem[s] * b + i) * K + c];
    double* R = C.ns.data() + (size_t)a * K * K;  // R(p, c) at R[p K + c]
    for (int c = 0; c < K; c++) {
      double* v = Q.data() + (size_t)c * rows;
      double n0 = 0.0;
      for (int t = 0; t < rows; t++) n0 += v[t] * v[t];
      n0 = std::sqrt(n0);
      for (int p = 0; p < c; p++) {
        const double* q = Q.data() + (size_t)p * rows;
        double h = 0.0;
        for (int t = 0; t < rows; t++) h += q[t] * v[t];
        R[p * K + c] = h;
        for (int t = 0; t < rows; t++) v[t] -= h * q[t];
      }
      double nv = 0.0;
      for (int t = 0; t < rows; t++) nv += v[t] * v[t];
      nv = std::sqrt(nv);
      if (n0 == 0.0 || nv <= AMG_QR_DROP * n0) {
        std::fill(v, v + rows, 0.0);
        R[c * K + c] = 0.0;
        C.absent[a] |= (uint8_t)(1u << c);
      } else {
        for (int t = 0; t < rows; t++) v[t] /= nv;
        R[c * K + c] = nv;
      }
    }
    for (size_t s = 0; s < mem.size(); s++)
      for (int i = 0; i < b; i++)
        for (int c = 0; c < K; c++) L.tnode[((size_t)mem[s] * b + i) * K + c] = Q[(size_t)c * rows + s * b + i];
  }
  const uint8_t full = full_mask(b);
  std::vector<int> tmp;
  // P: row i takes the aggregates of its neighbours
  L.pptr.assign(n + 1, 0);
  L.pcol.clear();
  for (int i = 0; i < n; i++) {
    tmp.clear();
    if (L.absent[i] != full)
      for (int k = L.ptr[i]; k < L.ptr[i + 1]; k++)
        if (L.agg[L.col[k]] >= 0) tmp.push_back(L.agg[L.col[k]]);
    sort_unique(tmp);
    L.pcol.insert(L.pcol.end(), tmp.begin(), tmp.end());
    L.pptr[i + 1] = (int)L.pcol.size();
  }
  // A P: row i takes the P rows of its neighbours
  L.apptr.assign(n + 1, 0);
  L.apcol.clear();
  for (int i = 0; i < n; i++) {
    tmp.clear();
    for (int k = L.ptr[i]; k < L.ptr[i + 1]; k++) {
      const int j = L.col[k];
      tmp.insert(tmp.end(), L.pcol.begin() + L.pptr[j], L.pcol.begin() + L.pptr[j + 1]);
    }
    sort_unique(tmp);
    L.apcol.insert(L.apcol.end(), tmp.begin(), tmp.end());
    L.apptr[i + 1] = (int)L.apcol.size();
  }
  // P^T: row a lists (fine node, P entry) by ascending fine node
  L.rptr.assign(nc + 1, 0);
  for (int q = 0; q < L.pptr[n]; q++) L.rptr[L.pcol[q] + 1]++;
  for (int a = 0; a < nc; a++) L.rptr[a + 1] += L.rptr[a];
  L.rcol.assign(L.pptr[n], 0);
  L.rsrc.assign(L.pptr[n], 0);
  {
    std::vector<int> fill(L.rptr.begin(), L.rptr.end() - 1);
    for (int i = 0; i < n; i++)
      for (int q = L.pptr[i]; q < L.pptr[i + 1]; q++) {
        const int s = fill[L.pcol[q]]++;
        L.rcol[s] = i;
        L.rsrc[s] = q;
      }
  }
  // coarse pattern: row a takes the A P rows of its P^T row, and the diagonal
  C.ptr.assign(nc + 1, 0);
  C.col.clear();
  for (int a = 0; a < nc; a++) {
    tmp.clear();
    tmp.push_back(a);
    for (int s = L.rptr[a]; s < L.rptr[a + 1]; s++) {
      const int i = L.rcol[s];
      tmp.insert(tmp.end(), L.apcol.begin() + L.apptr[i], L.apcol.begin() + L.apptr[i + 1]);
    }
    sort_unique(tmp);
    C.col.insert(C.col.end(), tmp.begin(), tmp.end());
    C.ptr[a + 1] = (int)C.col.size();
  }
  C.diag.assign(nc, -1);
  for (int a = 0; a < nc; a++)
    for (int k = C.ptr[a]; k < C.ptr[a + 1]; k++)
      if (C.col[k] == a) C.diag[a] = k;
}

// ---------------------------------------------------------------- device helpers
// V-cycle copies of the operators are tiled like the tangent: tiles of 32
// consecutive blocks, component-major inside a tile, so the lanes of a warp
// reading one component of consecutive blocks read one 128-byte run
template <int NV>
__host__ __device__ __forceinline__ int64_t tix(int64_t k, int c) {
  return (k >> 5) * (NV * 32) + 32 * c + (k & 31);
}
inline int64_t tiled_count(int64_t nblocks, int nv) { return (nblocks + 31) / 32 * 32 * nv; }

// a stored value in the V-cycle's arithmetic type T (FP32 values stay FP32)
template <class T, class V>
__device__ __forceinline__ T ldt(const V* p) {
  if constexpr (std::is_same<V, __nv_bfloat16>::value) return (T)__bfloat162float(*p);
  else return (T)__ldg(p);
}

// entry c of block k in the setup's arithmetic type C: level 0 reads the
// tangent in its tiled layout, coarser levels their block-major values
template <class C, class V, int B>
struct Vals {
  const V* v;
  bool tiled;
  __device__ __forceinline__ C operator()(int64_t k, int c) const {
    return tiled ? ldt<C, V>(v + kv_index(k, c)) : ldt<C, V>(v + k * (B * B) + c);
  }
};

__device__ __forceinline__ int find_col(const int* __restrict__ col, int lo, int hi, int c) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int v = __ldg(col + mid);
    if (v == c) return mid;
    if (v < c) lo = mid + 1;
    else hi = mid;
  }
  return -1;
}

// inverse of a B x B matrix by Gauss-Jordan elimination with partial pivoting
template <int B>
__device__ void gj_inverse(double (&a)[B][B], double (&inv)[B][B]) {
  for (int i = 0; i < B; i++)
    for (int j = 0; j < B; j++) inv[i][j] = i == j ? 1.0 : 0.0;
  for (int c = 0; c < B; c++) {
    int p = c;
    for (int r = c + 1; r < B; r++)
      if (fabs(a[r][c]) > fabs(a[p][c])) p = r;
    if (p != c)
      for (int j = 0; j < B; j++) {
        double t = a[c][j];
        a[c][j] = a[p][j];
        a[p][j] = t;
        t = inv[c][j];
        inv[c][j] = inv[p][j];
        inv[p][j] = t;
      }
    const double piv = a[c][c];
    for (int j = 0; j < B; j++) {
      a[c][j] /= piv;
      inv[c][j] /= piv;
    }
    for (int r = 0; r < B; r++) {
      if (r == c) continue;
      const double f = a[r][c];
      if (f == 0.0) continue;
      for (int j = 0; j < B; j++) {
        a[r][j] -= f * a[c][j];
        inv[r][j] -= f * inv[c][j];
      }
    }
  }
}

// ---------------------------------------------------------------- numeric setup kernels
// C is the setup's arithmetic type: FP64 for an FP64 tangent, FP32 for the
// mixed forms (whose V-cycle runs in FP32; GB300's FP32 rate is tens of
// times its FP64 rate).  The dense coarsest inverse is always formed in FP64.
template <class C, class V, int B>
__global__ void k_amg_dinv(int n, const int* __restrict__ diag, Vals<C, V, B> A, C* __restrict__ dinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a[B][B], inv[B][B];
  const int64_t k = diag[i];
  for (int r = 0; r < B; r++)
    for (int c = 0; c < B; c++) a[r][c] = (double)A(k, B * r + c);
  gj_inverse<B>(a, inv);
  for (int r = 0; r < B; r++)
    for (int c = 0; c < B; c++) dinv[(int64_t)i * B * B + B * r + c] = (C)inv[r][c];
}

// y = D^-1 (A x), one warp per block row
template <class C, class V, int B>
__global__ void __launch_bounds__(256) k_amg_dmv(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                                                 Vals<C, V, B> A, const C* __restrict__ dinv,
                                                 const C* __restrict__ x, C* __restrict__ y) {
  const int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  C s[B];
  for (int r = 0; r < B; r++) s[r] = C(0);
  for (int k = ptr[row] + lane; k < ptr[row + 1]; k += 32) {
    const int c = col[k];
    for (int r = 0; r < B; r++)
      for (int j = 0; j < B; j++) s[r] += A(k, B * r + j) * x[(int64_t)B * c + j];
  }
  for (int r = 0; r < B; r++)
    for (int off = 16; off > 0; off >>= 1) s[r] += __shfl_xor_sync(0xffffffffu, s[r], off);
  if (lane == 0)
    for (int r = 0; r < B; r++) {
      C t = C(0);
      for (int j = 0; j < B; j++) t += dinv[(int64_t)row * B * B + B * r + j] * s[j];
      y[(int64_t)B * row + r] = t;
    }
}

template <class C>
__global__ void k_amg_start(int64_t N, C* __restrict__ x) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) x[k] = (C)((double)(mix64_d((uint64_t)k) >> 11) * (1.0 / 9007199254740992.0) - 0.5);
}

// partial sums of x.x and y.y over a fixed grid (fixed order: deterministic), in FP64
template <class C>
__global__ void __launch_bounds__(256) k_amg_sumsq2(int64_t N, const C* __restrict__ x, const C* __restrict__ y,
                                                    double* __restrict__ part) {
  __shared__ double sh[2][8];
  double sx = 0.0, sy = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const double a = (double)x[k], c = (double)y[k];
    sx += a * a;
    sy += c * c;
  }
  for (int off = 16; off > 0; off >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, off);
    sy += __shfl_xor_sync(0xffffffffu, sy, off);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sh[0][w] = sx;
    sh[1][w] = sy;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
      a += sh[0][i];
      c += sh[1][i];
    }
    part[blockIdx.x] = a;
    part[gridDim.x + blockIdx.x] = c;
  }
}

// rho = |y| / |x|, x = y / |y|
template <class C>
__global__ void k_amg_power_step(int64_t N, int nblk, const double* __restrict__ part, const C* __restrict__ y,
                                 C* __restrict__ x, double* __restrict__ scal) {
  __shared__ double s_inv;
  if (threadIdx.x == 0) {
    double xx = 0.0, yy = 0.0;
    for (int i = 0; i < nblk; i++) {
      xx += part[i];
      yy += part[nblk + i];
    }
    scal[0] = sqrt(yy) / sqrt(xx);
    s_inv = 1.0 / sqrt(yy);
  }
  __syncthreads();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
    x[k] = (C)((double)y[k] * s_inv);
}

// P entry q = (row i, aggregate a): [agg(i) = a] T_i - omega sum_{k: agg(col k) = a} D_i^-1 A_k T_col(k)
template <class C, class V, int B>
__global__ void k_amg_pvals(int64_t nnzp, const int* __restrict__ prow, const int* __restrict__ pcol,
                            const int* __restrict__ ptr, const int* __restrict__ col, Vals<C, V, B> A,
                            const int* __restrict__ agg, const C* __restrict__ dinv,
                            const double* __restrict__ tnode, C omega, C* __restrict__ p) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nnzp) return;
  const int i = prow[q], a = pcol[q];
  C acc[B][AMG_NS];
  for (int r = 0; r < B; r++)
    for (int c = 0; c < AMG_NS; c++)
      acc[r][c] = agg[i] == a ? (C)tnode[(int64_t)i * B * AMG_NS + AMG_NS * r + c] : C(0);
  C D[B][B];
  for (int r = 0; r < B; r++)
    for (int c = 0; c < B; c++) D[r][c] = dinv[(int64_t)i * B * B + B * r + c];
  for (int k = ptr[i]; k < ptr[i + 1]; k++) {
    const int j = col[k];
    if (agg[j] != a) continue;
    C DA[B][B];
    for (int r = 0; r < B; r++)
      for (int c = 0; c < B; c++) {
        C s = C(0);
        for (int l = 0; l < B; l++) s += D[r][l] * A(k, B * l + c);
        DA[r][c] = s;
      }
    const double* T = tnode + (int64_t)j * B * AMG_NS;
    for (int r = 0; r < B; r++)
      for (int c = 0; c < AMG_NS; c++) {
        C s = C(0);
        for (int l = 0; l < B; l++) s += DA[r][l] * (C)T[AMG_NS * l + c];
        acc[r][c] -= omega * s;
      }
  }
  for (int r = 0; r < B; r++)
    for (int c = 0; c < AMG_NS; c++) p[q * B * AMG_NS + AMG_NS * r + c] = acc[r][c];
}

// A P entry (row i, aggregate a) = sum_k A_k P_(col k, a)
template <class C, class V, int B>
__global__ void k_amg_ap(int64_t nnzap, const int* __restrict__ aprow, const int* __restrict__ apcol,
                         const int* __restrict__ ptr, const int* __restrict__ col, Vals<C, V, B> A,
                         const int* __restrict__ pptr, const int* __restrict__ pcol, const C* __restrict__ p,
                         C* __restrict__ ap) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnzap) return;
  const int i = aprow[e], a = apcol[e];
  C acc[B][AMG_NS];
  for (int r = 0; r < B; r++)
    for (int c = 0; c < AMG_NS; c++) acc[r][c] = C(0);
  for (int k = ptr[i]; k < ptr[i + 1]; k++) {
    const int j = col[k];
    const int q = find_col(pcol, pptr[j], pptr[j + 1], a);
    if (q < 0) continue;
    const C* P = p + (int64_t)q * B * AMG_NS;
    for (int r = 0; r < B; r++) {
      C Ar[B];
      for (int l = 0; l < B; l++) Ar[l] = A(k, B * r + l);
      for (int c = 0; c < AMG_NS; c++) {
        C s = C(0);
        for (int l = 0; l < B; l++) s += Ar[l] * P[AMG_NS * l + c];
        acc[r][c] += s;
      }
    }
  }
  for (int r = 0; r < B; r++)
    for (int c = 0; c < AMG_NS; c++) ap[e * B * AMG_NS + AMG_NS * r + c] = acc[r][c];
}

// coarse entry (a, c) = sum over P^T row a (fine node i, P entry q) of P_q^T (A P)_(i, c);
// absent coarse components get a unit diagonal
template <class C, int B>
__global__ void k_amg_rap(int64_t nnzc, const int* __restrict__ crow, const int* __restrict__ ccol,
                          const int* __restrict__ rptr, const int* __restrict__ rcol, const int* __restrict__ rsrc,
                          const int* __restrict__ apptr, const int* __restrict__ apcol, const C* __restrict__ p,
                          const C* __restrict__ ap, const unsigned char* __restrict__ cabsent, C* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnzc) return;
  const int a = crow[e], cc = ccol[e];
  C acc[AMG_NS][AMG_NS];
  for (int r = 0; r < AMG_NS; r++)
    for (int c = 0; c < AMG_NS; c++) acc[r][c] = C(0);
  for (int s = rptr[a]; s < rptr[a + 1]; s++) {
    const int i = rcol[s];
    const int pe = find_col(apcol, apptr[i], apptr[i + 1], cc);
    if (pe < 0) continue;
    const C* P = p + (int64_t)rsrc[s] * B * AMG_NS;
    const C* Q = ap + (int64_t)pe * B * AMG_NS;
    for (int r = 0; r < AMG_NS; r++)
      for (int c = 0; c < AMG_NS; c++) {
        C v = C(0);
        for (int l = 0; l < B; l++) v += P[AMG_NS * l + r] * Q[AMG_NS * l + c];
        acc[r][c] += v;
      }
  }
  if (a == cc) {
    const unsigned m = cabsent[a];
    for (int c = 0; c < AMG_NS; c++)
      if ((m >> c) & 1u) acc[c][c] = C(1);
  }
  for (int r = 0; r < AMG_NS; r++)
    for (int c = 0; c < AMG_NS; c++) out[e * AMG_NS * AMG_NS + AMG_NS * r + c] = acc[r][c];
}

// R = P^T values: R entry s holds the transpose of P entry rsrc[s]
template <class C, int B>
__global__ void k_amg_rvals(int64_t nnzr, const int* __restrict__ rsrc, const C* __restrict__ p, C* __restrict__ rv) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nnzr) return;
  const C* P = p + (int64_t)rsrc[s] * B * AMG_NS;
  for (int c = 0; c < AMG_NS; c++)
    for (int r = 0; r < B; r++) rv[s * B * AMG_NS + B * c + r] = P[AMG_NS * r + c];
}

// dense inverse of the coarsest operator (N <= 96): one block, Gauss-Jordan
// with partial pivoting in shared memory (first maximal pivot on ties), FP64
template <class C, class V, int B>
__global__ void __launch_bounds__(1024) k_amg_dense_inverse(int n, const int* __restrict__ ptr,
                                                            const int* __restrict__ col, Vals<C, V, B> A,
                                                            double* __restrict__ inv) {
  extern __shared__ double sm[];
  const int N = n * B;
  double* M = sm;
  double* I = sm + N * N;
  double* fac = sm + 2 * N * N;  // column c before the elimination step
  __shared__ int s_piv;
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    M[t] = 0.0;
    I[t] = (t / N == t % N) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int a = threadIdx.x; a < n; a += blockDim.x)
    for (int k = ptr[a]; k < ptr[a + 1]; k++)
      for (int r = 0; r < B; r++)
        for (int c = 0; c < B; c++) M[(B * a + r) * N + B * col[k] + c] = (double)A(k, B * r + c);
  __syncthreads();
  for (int c = 0; c < N; c++) {
    if (threadIdx.x == 0) {
      int p = c;
      for (int r = c + 1; r < N; r++)
        if (fabs(M[r * N + c]) > fabs(M[p * N + c])) p = r;
      s_piv = p;
    }
    __syncthreads();
    const int p = s_piv;
    if (p != c)
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double t = M[c * N + j];
        M[c * N + j] = M[p * N + j];
        M[p * N + j] = t;
        t = I[c * N + j];
        I[c * N + j] = I[p * N + j];
        I[p * N + j] = t;
      }
    __syncthreads();
    const double piv = M[c * N + c];
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      M[c * N + j] /= piv;
      I[c * N + j] /= piv;
    }
    for (int r = threadIdx.x; r < N; r += blockDim.x) fac[r] = M[r * N + c];
    __syncthreads();
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
      const int r = t / N, j = t % N;
      const double f = fac[r];
      if (r == c || f == 0.0) continue;
      M[r * N + j] -= f * M[c * N + j];
      I[r * N + j] -= f * I[c * N + j];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) inv[t] = I[t];
}

__global__ void k_amg_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// block-major blocks of nv values -> the tiled layout
template <int NV, class T>
__global__ void k_amg_tile(int64_t nblocks, const T* __restrict__ src, T* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nblocks * NV) return;
  const int64_t k = i / NV;
  const int c = (int)(i % NV);
  dst[tix<NV>(k, c)] = (T)src[i];
}

// ---------------------------------------------------------------- V-cycle kernels
// One Chebyshev step of level l, fused (row i of n block rows, B components):
//   t = (A g)_i; x_i = (setx ? 0 : x_i) + cx g_i; r_i -= t;
//   dout_i = c1 g_i + c2 D_i^-1 r_i; final: x_i += dout_i.
// One warp per block row, one lane per block; level 0 reads the tangent
// in its tiled layout.
enum { VC_SETX = 1, VC_FINAL = 2, VC_KEEPX = 4, VC_START = 8 };


// Chebyshev epilogue of block row `row` with row sum s = (A g)_row
template <class T, int B>
__device__ __forceinline__ void cheb_rows(int64_t row, const T (&s)[B], const T* __restrict__ dinv,
                                          const T* __restrict__ g, T* __restrict__ x, T* __restrict__ r,
                                          T* __restrict__ dout, T cx, const T* __restrict__ coef, int flags) {
  const int64_t o = (int64_t)B * row;
  T rn[B], gi[B], xi[B];
#pragma unroll
  for (int q = 0; q < B; q++) {
    gi[q] = g[o + q];
    rn[q] = r[o + q] - s[q];
    r[o + q] = rn[q];
  }
  const bool wx = !(flags & VC_KEEPX);
#pragma unroll
  for (int q = 0; q < B; q++) xi[q] = ((flags & VC_SETX) ? T(0) : (wx ? x[o + q] : T(0))) + cx * gi[q];
  if (dout) {
    const T c1 = (flags & VC_START) ? T(0) : coef[1];
    const T c2 = (flags & VC_START) ? coef[0] : coef[2];
#pragma unroll
    for (int q = 0; q < B; q++) {
      T t = T(0);
#pragma unroll
      for (int j = 0; j < B; j++) t += dinv[row * B * B + B * q + j] * rn[j];
      const T dn = c1 * gi[q] + c2 * t;
      dout[o + q] = dn;
      if (flags & VC_FINAL) xi[q] += dn;
    }
  }
  if (wx)
#pragma unroll
    for (int q = 0; q < B; q++) x[o + q] = xi[q];
}

// Level-0 Chebyshev step, streamed like the SpMV: a warp takes groups of 16
// consecutive block rows and walks their (contiguous) blocks in chunks of 32,
// one block per lane, forming the row sums by a segmented scan across the
// lanes and carrying a row's partial sum into the next chunk; values, column
// indices and the gather of g run two chunks ahead.  A row's sum goes to
// shared memory when its last block is reached; the group's 16 Chebyshev
// row updates (cheb_rows' arithmetic) run together after its last chunk,
// lane i on row i, with the rows' g, r, x and block-Jacobi inverse loaded
// when the group starts: one memory latency per group for the updates
// instead of one per chunk that ends a row.  Every row of A holds its
// diagonal block, so no row is empty.
constexpr int VC_RPW = 16;

template <class V, class T>
__device__ __forceinline__ void vc_load_chunk(const int* __restrict__ col, const V* __restrict__ val, int64_t k,
                                              int64_t kend, int& c, T (&v)[9]) {
  if (k < kend) {
    c = __ldg(col + k);
#pragma unroll
    for (int t = 0; t < 9; t++) v[t] = ldt<T, V>(val + tix<9>(k, t));
  } else {
    c = -1;
#pragma unroll
    for (int t = 0; t < 9; t++) v[t] = T(0);
  }
}

template <class T>
__device__ __forceinline__ void vc_load_g(const T* __restrict__ g, int c, T (&x)[3], int n) {
  const int64_t cc = c >= 0 ? fe_idx(c, n) : 0;
#pragma unroll
  for (int j = 0; j < 3; j++) x[j] = c >= 0 ? g[3 * cc + j] : T(0);
}

template <class V, class T>
__global__ void __launch_bounds__(256) k_vc_cheb0(int n, const int* __restrict__ row_ptr, const int* __restrict__ col,
                                                  const V* __restrict__ val, const T* __restrict__ dinv,
                                                  const T* __restrict__ g, T* __restrict__ x, T* __restrict__ r,
                                                  T* __restrict__ dout, T cx, const T* __restrict__ coef,
                                                  int flags) {
  __shared__ T rsum[8][VC_RPW][3];  // row sums of each warp's current group
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool wx = !(flags & VC_KEEPX), rx = wx && !(flags & VC_SETX);
  const int ngroups = (n + VC_RPW - 1) / VC_RPW;
  const int nwarps = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
  for (int grp = (int)((((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5)); grp < ngroups; grp += nwarps) {
    const int r0 = grp * VC_RPW;
    const int nr = min(VC_RPW, n - r0);
    const int rpl = lane < nr ? __ldg(row_ptr + r0 + lane) : INT_MAX;  // start of row r0 + lane
    const int kstart = __shfl_sync(0xffffffffu, rpl, 0);
    const int kend = __ldg(row_ptr + r0 + nr);
    // this lane's row of the group (lane < nr): its update operands, loaded now
    T gi[3] = {T(0), T(0), T(0)}, ri[3] = {T(0), T(0), T(0)}, xo[3] = {T(0), T(0), T(0)}, di[9];
#pragma unroll
    for (int q = 0; q < 9; q++) di[q] = T(0);
    if (lane < nr) {
      const int64_t o = 3 * (int64_t)(r0 + lane);
#pragma unroll
      for (int q = 0; q < 3; q++) {
        gi[q] = g[o + q];
        ri[q] = r[o + q];
        if (rx) xo[q] = x[o + q];
      }
      if (dout)
#pragma unroll
        for (int q = 0; q < 9; q++) di[q] = dinv[9 * (int64_t)(r0 + lane) + q];
    }
    int c0, c1;
    T v0[9], v1[9];
    vc_load_chunk<V, T>(col, val, (int64_t)kstart + lane, kend, c0, v0);
    vc_load_chunk<V, T>(col, val, (int64_t)kstart + 32 + lane, kend, c1, v1);
    T xa[3];
    vc_load_g<T>(g, c0, xa, n);
    T carry[3] = {T(0), T(0), T(0)};
    int rowbase = r0 - 1;
    for (int kc = kstart; kc < kend; kc += 32) {
      int c2;
      T v2[9];
      vc_load_chunk<V, T>(col, val, (int64_t)kc + 64 + lane, kend, c2, v2);
      T xb[3];
      vc_load_g<T>(g, c1, xb, n);
      T p[3] = {T(0), T(0), T(0)};
      if (c0 >= 0)
#pragma unroll
        for (int q = 0; q < 3; q++) p[q] = v0[3 * q] * xa[0] + v0[3 * q + 1] * xa[1] + v0[3 * q + 2] * xa[2];
      const unsigned bit = (rpl >= kc && rpl - kc < 32) ? (1u << (rpl - kc)) : 0u;
      const unsigned heads = __reduce_or_sync(0xffffffffu, bit);
      const unsigned below = heads & (0xffffffffu >> (31 - lane));
      const int sstart = below ? 31 - __clz(below) : -1;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        T t[3];
#pragma unroll
        for (int q = 0; q < 3; q++) t[q] = __shfl_up_sync(0xffffffffu, p[q], off);
        if (lane >= off && lane - off >= sstart)
#pragma unroll
          for (int q = 0; q < 3; q++) p[q] += t[q];
      }
      const int nvalid = min(32, kend - kc);
      const bool cont = nvalid == 32 && kc + 32 < kend && !__any_sync(0xffffffffu, rpl == kc + 32);
      const bool tail = lane < nvalid && ((lane < 31 && ((heads >> (lane + 1)) & 1u)) || (lane == nvalid - 1 && !cont));
      if (tail) {
        const int row = rowbase + __popc(below);
        const bool add = sstart < 0;
#pragma unroll
        for (int q = 0; q < 3; q++) rsum[wid][row - r0][q] = p[q] + (add ? carry[q] : T(0));
      }
      T l[3];
#pragma unroll
      for (int q = 0; q < 3; q++) l[q] = __shfl_sync(0xffffffffu, p[q], 31);
      if (cont) {
        const bool whole = heads == 0u;  // lane 31's segment started before this chunk
#pragma unroll
        for (int q = 0; q < 3; q++) carry[q] = l[q] + (whole ? carry[q] : T(0));
      } else {
#pragma unroll
        for (int q = 0; q < 3; q++) carry[q] = T(0);
      }
      rowbase += __popc(heads);
      c0 = c1;
      c1 = c2;
#pragma unroll
      for (int t = 0; t < 9; t++) {
        v0[t] = v1[t];
        v1[t] = v2[t];
      }
#pragma unroll
      for (int j = 0; j < 3; j++) xa[j] = xb[j];
    }
    __syncwarp();
    if (lane < nr) {  // the group's row updates (cheb_rows' arithmetic, operands preloaded)
      const int64_t row = r0 + lane, o = 3 * row;
      T rn[3], xi[3];
#pragma unroll
      for (int q = 0; q < 3; q++) {
        rn[q] = ri[q] - rsum[wid][lane][q];
        r[o + q] = rn[q];
        xi[q] = xo[q] + cx * gi[q];
      }
      if (dout) {
        const T k1 = (flags & VC_START) ? T(0) : coef[1];
        const T k2 = (flags & VC_START) ? coef[0] : coef[2];
#pragma unroll
        for (int q = 0; q < 3; q++) {
          T t = T(0);
#pragma unroll
          for (int jj = 0; jj < 3; jj++) t += di[3 * q + jj] * rn[jj];
          const T dn = k1 * gi[q] + k2 * t;
          dout[o + q] = dn;
          if (flags & VC_FINAL) xi[q] += dn;
        }
      }
      if (wx)
#pragma unroll
        for (int q = 0; q < 3; q++) x[o + q] = xi[q];
    }
    __syncwarp();
  }
}

// Chebyshev step of a coarse level, one block row per warp (coarse rows
// are few and long), one lane per block; a lane reads its 6x6 block
// (block-major, from a device allocation, so 16-byte aligned) with 16-byte
// loads: nine load instructions in FP32 instead of 36.  Device function of
// warp-uniform `row` (< n): the kernel below runs it for its warp's row, the
// fused bottom of the V-cycle (k_vc_bottom) for rows strided over its warps;
// both sum in the same order, so their results are identical.  Vectors are
// read with plain loads: in k_vc_bottom they were written by the same block.
template <class T, int B>
__device__ __forceinline__ void vc_cheb_row(int row, int lane, int n, const int* ptr, const int* col, const T* val,
                                            const T* dinv, const T* g, T* x, T* r, T* dout, T cx, const T* coef,
                                            int flags) {
  // lane q < B updates component q of the row (cheb_rows' arithmetic); its
  // operands are loaded before the row's products, so their latency overlaps
  const bool wx = !(flags & VC_KEEPX), rx = wx && !(flags & VC_SETX);
  const int64_t o = (int64_t)B * row;
  T gq = T(0), rq = T(0), xq = T(0), dq[B];
#pragma unroll
  for (int j = 0; j < B; j++) dq[j] = T(0);
  if (lane < B) {
    gq = g[o + lane];
    rq = r[o + lane];
    if (rx) xq = x[o + lane];
    if (dout)
#pragma unroll
      for (int j = 0; j < B; j++) dq[j] = dinv[(int64_t)row * B * B + B * lane + j];
  }
  T s[B];
#pragma unroll
  for (int q = 0; q < B; q++) s[q] = T(0);
  for (int k = ptr[row] + lane; k < ptr[row + 1]; k += 32) {
    const int c = fe_idx(__ldg(col + k), n);
    T v[B * B];  // the block, block-major: B * B * sizeof(T) bytes, a multiple of 16
    if constexpr (sizeof(T) == 4) {
      const float4* p4 = reinterpret_cast<const float4*>(val + (int64_t)k * B * B);
#pragma unroll
      for (int t = 0; t < B * B / 4; t++) {
        const float4 u = __ldg(p4 + t);
        v[4 * t] = u.x;
        v[4 * t + 1] = u.y;
        v[4 * t + 2] = u.z;
        v[4 * t + 3] = u.w;
      }
    } else {
      const double2* p2 = reinterpret_cast<const double2*>(val + (int64_t)k * B * B);
#pragma unroll
      for (int t = 0; t < B * B / 2; t++) {
        const double2 u = __ldg(p2 + t);
        v[2 * t] = u.x;
        v[2 * t + 1] = u.y;
      }
    }
    T gv[B];
#pragma unroll
    for (int j = 0; j < B; j++) gv[j] = g[(int64_t)B * c + j];
#pragma unroll
    for (int q = 0; q < B; q++)
#pragma unroll
      for (int j = 0; j < B; j++) s[q] += v[B * q + j] * gv[j];
  }
#pragma unroll
  for (int q = 0; q < B; q++)
    for (int off = 16; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
  // this lane's component of the new residual, then every lane gets all of them
  T sq = T(0);
#pragma unroll
  for (int q = 0; q < B; q++)
    if (q == lane) sq = s[q];
  const T rn_q = rq - sq;
  T rn[B];
#pragma unroll
  for (int j = 0; j < B; j++) rn[j] = __shfl_sync(0xffffffffu, rn_q, j);
  if (lane < B) {
    r[o + lane] = rn_q;
    T xi = xq + cx * gq;
    if (dout) {
      const T c1 = (flags & VC_START) ? T(0) : coef[1];
      const T c2 = (flags & VC_START) ? coef[0] : coef[2];
      T t = T(0);
#pragma unroll
      for (int j = 0; j < B; j++) t += dq[j] * rn[j];
      const T dn = c1 * gq + c2 * t;
      dout[o + lane] = dn;
      if (flags & VC_FINAL) xi += dn;
    }
    if (wx) x[o + lane] = xi;
  }
}

template <class T, int B>
__global__ void __launch_bounds__(256) k_vc_cheb(int n, const int* __restrict__ ptr, const int* __restrict__ col,
                                                 const T* __restrict__ val, const T* __restrict__ dinv,
                                                 const T* __restrict__ g, T* __restrict__ x, T* __restrict__ r,
                                                 T* __restrict__ dout, T cx, const T* __restrict__ coef,
                                                 int flags) {
  const int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  vc_cheb_row<T, B>(row, lane, n, ptr, col, val, dinv, g, x, r, dout, cx, coef, flags);
}

// level-0 start of the pre-smoothing: r = b, d = D^-1 b / theta
template <class T>
__global__ void k_vc_init0(int n, const T* __restrict__ dinv, const double* __restrict__ b, T* __restrict__ r,
                           T* __restrict__ d, const T* __restrict__ coef) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T inv_theta = coef[0];
  T bi[3];
  for (int q = 0; q < 3; q++) {
    bi[q] = (T)b[3 * (int64_t)i + q];
    r[3 * (int64_t)i + q] = bi[q];
  }
  for (int q = 0; q < 3; q++) {
    T t = T(0);
    for (int j = 0; j < 3; j++) t += dinv[(int64_t)i * 9 + 3 * q + j] * bi[j];
    d[3 * (int64_t)i + q] = t * inv_theta;
  }
}

// restriction to the coarse level (6 components): s = (P^T r)_a;
// coarsest: bout = s; else: rc = s, dc = D_c^-1 s / theta_c.  A block of 128
// threads per coarse row: P^T rows are long (an aggregate's nodes and their
// neighbours, hundreds of blocks at level 0), so a warp per row would leave
// too few warps in flight; the block's partial sums are reduced in a fixed
// order (deterministic).
constexpr int VC_RESTRICT_THREADS = 128;

// thread t's partial sums of coarse row a (entries t, t + 128, ...)
template <class T, int BF>
__device__ __forceinline__ void vc_restrict_part(int a, int t, T (&s)[AMG_NS], const int* rptr, const int* rcol,
                                                 const T* rv, const T* rf, int nfine) {
#pragma unroll
  for (int q = 0; q < AMG_NS; q++) s[q] = T(0);
  for (int k = rptr[a] + t; k < rptr[a + 1]; k += VC_RESTRICT_THREADS) {
    const int i = fe_idx(__ldg(rcol + k), nfine);
    T f[BF];
#pragma unroll
    for (int j = 0; j < BF; j++) f[j] = rf[(int64_t)BF * i + j];
#pragma unroll
    for (int q = 0; q < AMG_NS; q++)
#pragma unroll
      for (int j = 0; j < BF; j++) s[q] += __ldg(rv + (int64_t)k * BF * AMG_NS + BF * q + j) * f[j];
  }
#pragma unroll
  for (int q = 0; q < AMG_NS; q++)
    for (int off = 16; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off);
}

// coarse row a from its four warps' sums sh[w][q] (one thread)
template <class T>
__device__ __forceinline__ void vc_restrict_finish(int a, const T (*sh)[AMG_NS], const T* dinvc, T* rc, T* dc,
                                                   const T* coefc) {
  T s[AMG_NS];
#pragma unroll
  for (int q = 0; q < AMG_NS; q++) s[q] = (sh[0][q] + sh[1][q]) + (sh[2][q] + sh[3][q]);
  const int64_t o = (int64_t)AMG_NS * a;
#pragma unroll
  for (int q = 0; q < AMG_NS; q++) rc[o + q] = s[q];
  if (dc) {
    const T inv_theta = coefc[0];
#pragma unroll
    for (int q = 0; q < AMG_NS; q++) {
      T t = T(0);
#pragma unroll
      for (int j = 0; j < AMG_NS; j++) t += dinvc[(int64_t)a * AMG_NS * AMG_NS + AMG_NS * q + j] * s[j];
      dc[o + q] = t * inv_theta;
    }
  }
}

template <class T, int BF>
__global__ void __launch_bounds__(VC_RESTRICT_THREADS) k_vc_restrict(int nc, const int* __restrict__ rptr,
                                                                     const int* __restrict__ rcol,
                                                                     const T* __restrict__ rv, const T* __restrict__ rf,
                                                                     const T* __restrict__ dinvc, T* __restrict__ rc,
                                                                     T* __restrict__ dc, const T* __restrict__ coefc,
                                                                     int nfine) {
  __shared__ T sh[4][AMG_NS];
  const int a = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T s[AMG_NS];
  vc_restrict_part<T, BF>(a, threadIdx.x, s, rptr, rcol, rv, rf, nfine);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < AMG_NS; q++) sh[w][q] = s[q];
  __syncthreads();
  if (threadIdx.x == 0) vc_restrict_finish<T>(a, sh, dinvc, rc, dc, coefc);
}

// coarsest solve: x = inv b (one block)
template <class T>
__global__ void k_vc_dense(int N, const T* __restrict__ inv, const T* __restrict__ b, T* __restrict__ x) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    T s = T(0);
    for (int j = 0; j < N; j++) s += inv[(int64_t)i * N + j] * b[j];
    x[i] = s;
  }
}

// prolongation: e_i = (P xc)_i, x_i += e_i.  LPR lanes per fine row: a P row
// holds the few aggregates around the node (about 7 at level 0), so a whole
// warp per row would idle most lanes (4 lanes: two blocks each, in flight
// together); P is tiled, so the lanes of a warp
// (consecutive rows, consecutive blocks) read each component in one run.
// Rows of wholly absent nodes have no blocks: their e stays zero.
// thread t of the prolongation (row t / LPR, lane t % LPR); every lane of
// the warp calls it (the row sums are reduced across the row's lanes)
template <class T, int BF, int LPR>
__device__ __forceinline__ void vc_prolong_thread(int64_t t, int n, const int* pptr, const int* pcol, const T* pv,
                                                  const T* xc, T* x, T* e, int ncoarse) {
  const int i = (int)(t / LPR);
  const int l = (int)(t % LPR);
  const bool active = i < n;
  T s[BF], xo[BF];
#pragma unroll
  for (int q = 0; q < BF; q++) s[q] = xo[q] = T(0);
  if (active && l == 0)  // the row's x, loaded ahead of its products
#pragma unroll
    for (int q = 0; q < BF; q++) xo[q] = x[(int64_t)BF * i + q];
  if (active)
    for (int k = pptr[i] + l; k < pptr[i + 1]; k += LPR) {
      const int a = fe_idx(__ldg(pcol + k), ncoarse);
      T c[AMG_NS];
#pragma unroll
      for (int j = 0; j < AMG_NS; j++) c[j] = xc[(int64_t)AMG_NS * a + j];
#pragma unroll
      for (int q = 0; q < BF; q++)
#pragma unroll
        for (int j = 0; j < AMG_NS; j++) s[q] += __ldg(pv + tix<BF * AMG_NS>(k, AMG_NS * q + j)) * c[j];
    }
#pragma unroll
  for (int q = 0; q < BF; q++)
    for (int off = LPR / 2; off > 0; off >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], off, LPR);
  if (!active || l != 0) return;
#pragma unroll
  for (int q = 0; q < BF; q++) {
    e[(int64_t)BF * i + q] = s[q];
    x[(int64_t)BF * i + q] = xo[q] + s[q];
  }
}

template <class T, int BF, int LPR>
__global__ void __launch_bounds__(256) k_vc_prolong(int n, const int* __restrict__ pptr, const int* __restrict__ pcol,
                                                    const T* __restrict__ pv, const T* __restrict__ xc,
                                                    T* __restrict__ x, T* __restrict__ e, int ncoarse) {
  vc_prolong_thread<T, BF, LPR>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, n, pptr, pcol, pv, xc, x, e, ncoarse);
}

// The bottom of the V-cycle in one block.  Below a few hundred nodes per
// level the coarse kernels are a few blocks each, and their cost is launch
// latency, not bytes: levels q0..L-1 (each at most VC_BOTTOM_MAXN nodes,
// q0 >= 1) run as one launch of one block -- smoothing, restriction, the
// coarsest solve, prolongation and smoothing again, separated by block
// barriers.  Each stage runs the same device functions as the per-level
// kernels, with the same assignment of rows and entries to warps, lanes and
// 128-thread groups, so the result is identical to theirs.
template <class T>
__host__ __device__ constexpr int vc_bottom_threads() { return sizeof(T) == 8 ? 512 : 1024; }
constexpr int VC_BOTTOM_MAXN = 256;

template <class T>
struct VcLevelArgs {  // one level of the bottom (device pointers)
  int n, nc;
  const int *ptr, *col;            // A_l pattern, tiled values, block-Jacobi inverse, Chebyshev coefficients
  const T *val, *dinv, *coef;
  const int *rptr, *rcol;          // P_l^T (l below the coarsest)
  const T* rv;
  const int *pptr, *pcol;          // P_l, tiled
  const T* pv;
  const T* inv;                    // coarsest: dense inverse
  T *x, *r, *d0, *d1, *e;          // V-cycle vectors
};
template <class T>
struct VcBottomArgs {
  int nb;                          // levels q0 .. q0 + nb - 1, the last one the coarsest
  VcLevelArgs<T> lev[AMG_MAXLEV];
};

template <class T>
__global__ void __launch_bounds__(vc_bottom_threads<T>()) k_vc_bottom(const VcBottomArgs<T> P) {
  constexpr int NT = vc_bottom_threads<T>();
  constexpr int NW = NT / 32;
  constexpr int NG = NT / VC_RESTRICT_THREADS;
  __shared__ T sh[NG][4][AMG_NS];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // one Chebyshev step of a level: rows strided over the warps
  auto cheb = [&](const VcLevelArgs<T>& L, const T* g, T* dout, T cx, int flags) {
    for (int row = wid; row < L.n; row += NW)
      vc_cheb_row<T, AMG_NS>(row, lane, L.n, L.ptr, L.col, L.val, L.dinv, g, L.x, L.r, dout, cx, L.coef, flags);
    __syncthreads();
  };
  const int nb = P.nb;
  for (int l = 0; l < nb - 1; l++) {  // downward
    const VcLevelArgs<T>& L = P.lev[l];
    const VcLevelArgs<T>& C = P.lev[l + 1];
    cheb(L, L.d0, L.d1, T(1), VC_SETX);
    cheb(L, L.d1, nullptr, T(1), 0);
    const bool coarsest = l + 1 == nb - 1;
    const int grp = tid / VC_RESTRICT_THREADS, t = tid % VC_RESTRICT_THREADS, w = t >> 5;
    for (int a0 = 0; a0 < C.n; a0 += NG) {  // coarse rows, one per 128-thread group
      const int a = a0 + grp;
      if (a < C.n) {
        T s[AMG_NS];
        vc_restrict_part<T, AMG_NS>(a, t, s, L.rptr, L.rcol, L.rv, L.r, L.n);
        if (lane == 0)
#pragma unroll
          for (int q = 0; q < AMG_NS; q++) sh[grp][w][q] = s[q];
      }
      __syncthreads();
      if (t == 0 && a < C.n) vc_restrict_finish<T>(a, sh[grp], C.dinv, C.r, coarsest ? nullptr : C.d0, C.coef);
      __syncthreads();
    }
  }
  {  // coarsest: x = inv r
    const VcLevelArgs<T>& Lc = P.lev[nb - 1];
    const int N = Lc.n * AMG_NS;
    for (int i = tid; i < N; i += NT) {
      T s = T(0);
      for (int j = 0; j < N; j++) s += Lc.inv[(int64_t)i * N + j] * Lc.r[j];
      Lc.x[i] = s;
    }
    __syncthreads();
  }
  for (int l = nb - 2; l >= 0; l--) {  // upward
    const VcLevelArgs<T>& L = P.lev[l];
    const VcLevelArgs<T>& C = P.lev[l + 1];
    constexpr int LPR = 4;
    for (int64_t t0 = 0; t0 < (int64_t)L.n * LPR; t0 += NT)
      vc_prolong_thread<T, AMG_NS, LPR>(t0 + tid, L.n, L.pptr, L.pcol, L.pv, C.x, L.x, L.e, L.nc);
    __syncthreads();
    cheb(L, L.e, L.d0, T(0), VC_KEEPX | VC_START);
    cheb(L, L.d0, L.d1, T(1), VC_FINAL);
  }
}

template <class A, class B>
__global__ void k_vc_convert(int64_t n, const A* __restrict__ a, B* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (B)a[i];
}

// ---------------------------------------------------------------- host drivers
template <class X>
int dev_alloc(fe_mesh m, X** p, size_t count) {
  count = count ? count : 1;
  FE_TRY(fe_alloc_t(m, p, count));
  m->amg->allocs.push_back((void*)*p);
  m->amg->bytes += (int64_t)(count * sizeof(X));
  return FE_OK;
}

template <class X>
int upload(fe_mesh m, X** p, const std::vector<X>& v) {
  FE_TRY(dev_alloc(m, p, v.size()));
  if (!v.empty()) FE_CUDA(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice, m->stream));
  return FE_OK;
}

unsigned blocks_for(int64_t n, int per) { return (unsigned)std::max<int64_t>(1, (n + per - 1) / per); }

// structure of every level, once per mesh
int build_structure(fe_mesh m) {
  AmgHier* h = m->amg;
  std::vector<HostLevel> hl(1);
  HostLevel& L0 = hl[0];
  const int nn = m->nn;
  L0.n = nn;
  L0.b = 3;
  L0.ptr.resize(nn + 1);
  L0.col.resize(m->nnzb);
  std::vector<uint8_t> fix(nn);
  std::vector<double> X((size_t)nn * 3);
  FE_CUDA(cudaMemcpyAsync(L0.ptr.data(), m->row_ptr, sizeof(int) * (nn + 1), cudaMemcpyDeviceToHost, m->stream));
  FE_CUDA(cudaMemcpyAsync(L0.col.data(), m->col, sizeof(int) * m->nnzb, cudaMemcpyDeviceToHost, m->stream));
  FE_CUDA(cudaMemcpyAsync(fix.data(), m->fixmask, nn, cudaMemcpyDeviceToHost, m->stream));
  FE_CUDA(cudaMemcpyAsync(X.data(), m->X, sizeof(double) * 3 * nn, cudaMemcpyDeviceToHost, m->stream));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  L0.absent = fix;
  L0.ns.assign((size_t)nn * 3 * AMG_NS, 0.0);
  for (int a = 0; a < nn; a++) {
    const double x = X[3 * a], y = X[3 * a + 1], z = X[3 * a + 2];
    const double rb[3][AMG_NS] = {{1, 0, 0, -y, 0, z}, {0, 1, 0, x, -z, 0}, {0, 0, 1, 0, y, -x}};
    for (int c = 0; c < 3; c++)
      for (int k = 0; k < AMG_NS; k++) L0.ns[((size_t)3 * a + c) * AMG_NS + k] = ((fix[a] >> c) & 1) ? 0.0 : rb[c][k];
  }
  int l = 0;
  for (;;) {
    HostLevel& L = hl[l];
    if (L.n <= AMG_COARSE || l == AMG_MAXLEV - 1) break;
    aggregate(L);
    if (L.nc == 0 || L.nc > 0.9 * L.n) {
      L.agg.clear();
      L.nc = 0;
      break;
    }
    hl.emplace_back();
    coarsen(hl[l], hl[l + 1]);
    l++;
  }
  const int nlev = l + 1;
  const HostLevel& Lc = hl[nlev - 1];
  if (Lc.n * Lc.b > AMG_DENSE_MAX)
    return fe_set_error("AMG: the coarsest level has %d unknowns (at most %d)", Lc.n * Lc.b, AMG_DENSE_MAX),
           FE_ERR_ARG;
  h->nlev = nlev;
  for (int q = 0; q < nlev; q++) {
    HostLevel& H = hl[q];
    AmgLevel& A = h->lev[q];
    A.n = H.n;
    A.b = H.b;
    A.nc = q < nlev - 1 ? H.nc : 0;
    if (q == 0) {
      A.ptr = m->row_ptr;
      A.col = m->col;
      A.diag = m->diag_pos;
      A.nnz = m->nnzb;
    } else {
      int *p = nullptr, *c = nullptr, *d = nullptr, *cr = nullptr;
      FE_TRY(upload(m, &p, H.ptr));
      FE_TRY(upload(m, &c, H.col));
      FE_TRY(upload(m, &d, H.diag));
      std::vector<int> crow(H.col.size());
      for (int a = 0; a < H.n; a++)
        for (int k = H.ptr[a]; k < H.ptr[a + 1]; k++) crow[k] = a;
      FE_TRY(upload(m, &cr, crow));
      A.ptr = p;
      A.col = c;
      A.diag = d;
      A.crow = cr;
      A.nnz = (int64_t)H.col.size();
    }
    FE_TRY(upload(m, &A.absent, H.absent));
    if (q < nlev - 1) {
      FE_TRY(upload(m, &A.agg, H.agg));
      FE_TRY(upload(m, &A.pptr, H.pptr));
      FE_TRY(upload(m, &A.pcol, H.pcol));
      std::vector<int> prow(H.pcol.size()), aprow(H.apcol.size());
      for (int i = 0; i < H.n; i++) {
        for (int k = H.pptr[i]; k < H.pptr[i + 1]; k++) prow[k] = i;
        for (int k = H.apptr[i]; k < H.apptr[i + 1]; k++) aprow[k] = i;
      }
      FE_TRY(upload(m, &A.prow, prow));
      FE_TRY(upload(m, &A.rptr, H.rptr));
      FE_TRY(upload(m, &A.rcol, H.rcol));
      FE_TRY(upload(m, &A.rsrc, H.rsrc));
      FE_TRY(upload(m, &A.apptr, H.apptr));
      FE_TRY(upload(m, &A.apcol, H.apcol));
      FE_TRY(upload(m, &A.aprow, aprow));
      FE_TRY(upload(m, &A.tnode, H.tnode));
      A.nnzp = (int64_t)H.pcol.size();
      A.nnzr = A.nnzp;
      A.nnzap = (int64_t)H.apcol.size();
    }
  }
  int64_t maxN = 0;
  for (int q = 0; q < nlev; q++) maxN = std::max<int64_t>(maxN, (int64_t)h->lev[q].n * h->lev[q].b);
  FE_TRY(dev_alloc(m, &h->pw, (size_t)2 * maxN));
  FE_TRY(dev_alloc(m, &h->part, (size_t)2 * AMG_RED_BLOCKS));
  FE_TRY(dev_alloc(m, &h->scal, 4));
  FE_CUDA(cudaStreamSynchronize(m->stream));  // host vectors above go out of scope
  return FE_OK;
}

int to_f32(fe_mesh m, const double* a, float** b, int64_t n) {
  if (!*b) FE_TRY(dev_alloc(m, b, (size_t)n));
  k_amg_to_f32<<<blocks_for(n, 256), 256, 0, m->stream>>>(n, a, *b);
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// the arrays of the setup's arithmetic type C
template <class C>
struct Arr {
  static C*& val(AmgLevel& L);
  static C*& dinv(AmgLevel& L);
  static C*& p(AmgLevel& L);
  static C*& ap(AmgLevel& L);
  static C*& r(AmgLevel& L);
};
template <>
struct Arr<double> {
  static double*& val(AmgLevel& L) { return L.val64; }
  static double*& dinv(AmgLevel& L) { return L.dinv64; }
  static double*& p(AmgLevel& L) { return L.p64; }
  static double*& ap(AmgLevel& L) { return L.ap64; }
  static double*& r(AmgLevel& L) { return L.r64; }
};
template <>
struct Arr<float> {
  static float*& val(AmgLevel& L) { return L.val32; }
  static float*& dinv(AmgLevel& L) { return L.dinv32; }
  static float*& p(AmgLevel& L) { return L.p32; }
  static float*& ap(AmgLevel& L) { return L.ap32; }
  static float*& r(AmgLevel& L) { return L.r32; }
};

// numbers of level q (A_q already numeric) in arithmetic type C: D^-1, rho,
// P, AP, R and A_{q+1}; the coarsest level's dense inverse (FP64, with an
// FP32 copy for the mixed forms)
template <class C, class V, int B>
int numeric_level(fe_mesh m, int q, Vals<C, V, B> A) {
  AmgHier* h = m->amg;
  AmgLevel& L = h->lev[q];
  const int64_t N = (int64_t)L.n * L.b;
  C*& dinv = Arr<C>::dinv(L);
  if (!dinv) FE_TRY(dev_alloc(m, &dinv, (size_t)L.n * B * B));
  {
    FE_SCOPE(m, FE_PROF_OTHER, (double)L.n * B * B * (8 + sizeof(C)));
    k_amg_dinv<C, V, B><<<blocks_for(L.n, 128), 128, 0, m->stream>>>(L.n, L.diag, A, dinv);
  }
  FE_CUDA(cudaGetLastError());
  if (q == h->nlev - 1) {  // coarsest: dense inverse
    const int Nd = L.n * B;
    if (!L.inv64) FE_TRY(dev_alloc(m, &L.inv64, (size_t)Nd * Nd));
    const int smem = (2 * Nd * Nd + Nd) * (int)sizeof(double);
    FE_TRY(fe_kernel_smem((const void*)k_amg_dense_inverse<C, V, B>, smem));
    {
      FE_SCOPE(m, FE_PROF_OTHER, 8.0 * Nd * Nd);
      k_amg_dense_inverse<C, V, B><<<1, 1024, smem, m->stream>>>(L.n, L.ptr, L.col, A, L.inv64);
    }
    FE_CUDA(cudaGetLastError());
    if (!std::is_same<C, double>::value) FE_TRY(to_f32(m, L.inv64, &L.inv32, (int64_t)Nd * Nd));
    return FE_OK;
  }
  // rho: power steps on D^-1 A
  C* x = (C*)h->pw;
  C* y = x + N;
  k_amg_start<C><<<blocks_for(N, 256), 256, 0, m->stream>>>(N, x);
  for (int it = 0; it < AMG_POWER_STEPS; it++) {
    {
      FE_SCOPE(m, FE_PROF_OTHER, (double)L.nnz * (B * B * sizeof(V) + 4) + 2.0 * sizeof(C) * N);
      k_amg_dmv<C, V, B><<<blocks_for((int64_t)L.n * 32, 256), 256, 0, m->stream>>>(L.n, L.ptr, L.col, A, dinv, x, y);
    }
    k_amg_sumsq2<C><<<AMG_RED_BLOCKS, 256, 0, m->stream>>>(N, x, y, h->part);
    k_amg_power_step<C><<<blocks_for(N, 256), 256, 0, m->stream>>>(N, AMG_RED_BLOCKS, h->part, y, x, h->scal);
  }
  FE_CUDA(cudaGetLastError());
  FE_CUDA(cudaMemcpyAsync(m->h_scal + 20, h->scal, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  L.rho = m->h_scal[20];
  if (!(L.rho > 0.0) || !std::isfinite(L.rho))
    return fe_set_error("AMG: spectral radius estimate %g on level %d", L.rho, q), FE_ERR_STATE;
  const C omega = (C)(4.0 / (3.0 * L.rho));
  C*& p = Arr<C>::p(L);
  C*& ap = Arr<C>::ap(L);
  C*& r = Arr<C>::r(L);
  if (!p) FE_TRY(dev_alloc(m, &p, (size_t)L.nnzp * B * AMG_NS));
  if (!ap) FE_TRY(dev_alloc(m, &ap, (size_t)L.nnzap * B * AMG_NS));
  if (!r) FE_TRY(dev_alloc(m, &r, (size_t)L.nnzr * B * AMG_NS));
  AmgLevel& Cq = h->lev[q + 1];
  C*& cval = Arr<C>::val(Cq);
  if (!cval) FE_TRY(dev_alloc(m, &cval, (size_t)Cq.nnz * AMG_NS * AMG_NS));
  {
    FE_SCOPE(m, FE_PROF_OTHER, (double)L.nnzp * B * AMG_NS * sizeof(C));
    k_amg_pvals<C, V, B><<<blocks_for(L.nnzp, 128), 128, 0, m->stream>>>(L.nnzp, L.prow, L.pcol, L.ptr, L.col, A,
                                                                        L.agg, dinv, L.tnode, omega, p);
  }
  FE_CUDA(cudaGetLastError());
  {
    FE_SCOPE(m, FE_PROF_OTHER, (double)L.nnzap * B * AMG_NS * sizeof(C));
    k_amg_ap<C, V, B><<<blocks_for(L.nnzap, 128), 128, 0, m->stream>>>(L.nnzap, L.aprow, L.apcol, L.ptr, L.col, A,
                                                                      L.pptr, L.pcol, p, ap);
  }
  FE_CUDA(cudaGetLastError());
  {
    FE_SCOPE(m, FE_PROF_OTHER, (double)Cq.nnz * AMG_NS * AMG_NS * sizeof(C));
    k_amg_rap<C, B><<<blocks_for(Cq.nnz, 128), 128, 0, m->stream>>>(Cq.nnz, Cq.crow, Cq.col, L.rptr, L.rcol, L.rsrc,
                                                                    L.apptr, L.apcol, p, ap, Cq.absent, cval);
  }
  FE_CUDA(cudaGetLastError());
  k_amg_rvals<C, B><<<blocks_for(L.nnzr, 256), 256, 0, m->stream>>>(L.nnzr, L.rsrc, p, r);
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

int store_coeffs(fe_mesh m);

template <int NV, class T>
int tile_one(fe_mesh m, const T* src, T** dst, int64_t nblocks) {
  if (!*dst) FE_TRY(dev_alloc(m, dst, (size_t)tiled_count(nblocks, NV)));
  k_amg_tile<NV, T><<<blocks_for(nblocks * NV, 256), 256, 0, m->stream>>>(nblocks, src, *dst);
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// tiled V-cycle copies of the prolongators
template <class C>
int tile_copies(fe_mesh m) {
  AmgHier* h = m->amg;
  for (int q = 0; q < h->nlev; q++) {
    AmgLevel& L = h->lev[q];
    C** pt = std::is_same<C, double>::value ? (C**)&L.pt64 : (C**)&L.pt32;
    if (q < h->nlev - 1) {
      if (L.b == 3) FE_TRY((tile_one<3 * AMG_NS, C>(m, Arr<C>::p(L), pt, L.nnzp)));
      else FE_TRY((tile_one<AMG_NS * AMG_NS, C>(m, Arr<C>::p(L), pt, L.nnzp)));
    }
  }
  return FE_OK;
}

// the whole hierarchy's numbers: FP64 for an FP64 tangent, FP32 otherwise
template <class C, class V>
int numeric_all(fe_mesh m, const V* K0) {
  AmgHier* h = m->amg;
  FE_TRY((numeric_level<C, V, 3>(m, 0, Vals<C, V, 3>{K0, true})));
  for (int q = 1; q < h->nlev; q++)
    FE_TRY((numeric_level<C, C, AMG_NS>(m, q, Vals<C, C, AMG_NS>{Arr<C>::val(h->lev[q]), false})));
  FE_TRY(store_coeffs(m));
  return tile_copies<C>(m);
}

int ensure_vectors(fe_mesh m, int elem) {
  AmgHier* h = m->amg;
  if (h->vec_elem == elem) return FE_OK;  // (a precision change allocates a new set)
  for (int q = 0; q < h->nlev; q++) {
    AmgLevel& L = h->lev[q];
    const size_t bytes = (size_t)L.n * L.b * elem;
    void** vs[5] = {&L.x, &L.r, &L.d0, &L.d1, &L.e};
    for (void** v : vs) {
      char* p = nullptr;
      FE_TRY(dev_alloc(m, &p, bytes));
      *v = p;
    }
  }
  h->vec_elem = elem;
  return FE_OK;
}

struct Cheb {
  double inv_theta, c1, c2;
};
Cheb cheb_coeffs(double rho) {
  const double lo = rho / 30.0, hi = 1.1 * rho;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  const double r0 = 1.0 / sigma, r1 = 1.0 / (2.0 * sigma - r0);
  return Cheb{1.0 / theta, r1 * r0, 2.0 * r1 / delta};
}

// Chebyshev coefficients of every smoothed level into device memory
int store_coeffs(fe_mesh m) {
  AmgHier* h = m->amg;
  for (int q = 0; q < h->nlev - 1; q++) {
    AmgLevel& L = h->lev[q];
    if (!L.coef64) FE_TRY(dev_alloc(m, &L.coef64, 4));
    if (!L.coef32) FE_TRY(dev_alloc(m, &L.coef32, 4));
    const Cheb c = cheb_coeffs(L.rho);
    double* hd = m->h_scal + 24;  // pinned staging, consumed before the next sync
    float* hf = (float*)(m->h_scal + 28);
    hd[0] = c.inv_theta;
    hd[1] = c.c1;
    hd[2] = c.c2;
    hf[0] = (float)c.inv_theta;
    hf[1] = (float)c.c1;
    hf[2] = (float)c.c2;
    FE_CUDA(cudaMemcpyAsync(L.coef64, hd, 3 * sizeof(double), cudaMemcpyHostToDevice, m->stream));
    FE_CUDA(cudaMemcpyAsync(L.coef32, hf, 3 * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    FE_CUDA(cudaStreamSynchronize(m->stream));
  }
  return FE_OK;
}

// The kernels of one V-cycle in precision T, level-0 values of type V
// (tiled), on stream st: input b (FP64 [3 nn]), result in lev[0].x.  Adds
// the algorithmic bytes and flops of its kernels to *bytes, *flops.
template <class T, class V>
int vcycle_launches(fe_mesh m, cudaStream_t st, const V* K0, const double* b, double* bytes, double* flops) {
  AmgHier* h = m->amg;
  const int L = h->nlev;
  constexpr bool D = sizeof(T) == 8;
  auto vals = [&](int q) -> const T* { return D ? (const T*)h->lev[q].val64 : (const T*)h->lev[q].val32; };
  auto dinv = [&](int q) -> const T* { return D ? (const T*)h->lev[q].dinv64 : (const T*)h->lev[q].dinv32; };
  auto pv = [&](int q) -> const T* { return D ? (const T*)h->lev[q].pt64 : (const T*)h->lev[q].pt32; };
  auto rv = [&](int q) -> const T* { return D ? (const T*)h->lev[q].r64 : (const T*)h->lev[q].r32; };
  auto inv = [&](int q) -> const T* { return D ? (const T*)h->lev[q].inv64 : (const T*)h->lev[q].inv32; };
  auto coef = [&](int q) -> const T* { return D ? (const T*)h->lev[q].coef64 : (const T*)h->lev[q].coef32; };
  auto X = [&](int q) { return (T*)h->lev[q].x; };
  const double sv = sizeof(T), s0 = sizeof(V);
  // Chebyshev step on level q (fused SpMV)
  auto step = [&](int q, const T* g, T* dout, double cx, int flags) -> int {
    AmgLevel& Lq = h->lev[q];
    const int B = Lq.b;
    *bytes += (double)Lq.nnz * (B * B * (q == 0 ? s0 : sv) + 4) + 4.0 * (Lq.n + 1) + (double)Lq.n * B * (sv * 5 + B * sv);
    *flops += 2.0 * Lq.nnz * B * B;
    if (q == 0)
      k_vc_cheb0<V, T><<<h->grid0, 256, 0, st>>>(Lq.n, Lq.ptr, Lq.col, K0, dinv(0), g, X(0), (T*)Lq.r, dout, (T)cx,
                                                 coef(0), flags);
    else
      k_vc_cheb<T, AMG_NS><<<blocks_for((int64_t)Lq.n * 32, 256), 256, 0, st>>>(
          Lq.n, Lq.ptr, Lq.col, vals(q), dinv(q), g, X(q), (T*)Lq.r, dout, (T)cx, coef(q), flags);
    FE_CUDA(cudaGetLastError());
    return FE_OK;
  };
  if (L == 1) {  // one level: the exact solve
    AmgLevel& L0 = h->lev[0];
    const int64_t N = (int64_t)L0.n * 3;
    k_vc_convert<double, T><<<blocks_for(N, 256), 256, 0, st>>>(N, b, (T*)L0.r);
    k_vc_dense<T><<<1, 256, 0, st>>>((int)N, inv(0), (const T*)L0.r, X(0));
    FE_CUDA(cudaGetLastError());
    *bytes += (double)N * N * sv + 8.0 * N;
    *flops += 2.0 * N * N;
    return FE_OK;
  }
  // the bottom levels q0..L-1 (at most VC_BOTTOM_MAXN nodes each, q0 >= 1)
  // run in one block when at least one of them is smoothed
  int q0 = L - 1;
  while (q0 > 1 && h->lev[q0 - 1].n <= VC_BOTTOM_MAXN) q0--;
  const bool fused = q0 <= L - 2;
  const int qf = fused ? q0 : L - 1;  // the per-level kernels run on levels 0..qf-1
  // downward: pre-smoothing, restriction
  for (int q = 0; q < qf; q++) {
    AmgLevel& Lq = h->lev[q];
    if (q == 0) {
      k_vc_init0<T><<<blocks_for(Lq.n, 256), 256, 0, st>>>(Lq.n, dinv(0), b, (T*)Lq.r, (T*)Lq.d0, coef(0));
      FE_CUDA(cudaGetLastError());
      *bytes += (double)Lq.n * (24 + 9 * sv + 6 * sv);
    }
    // x = d0; r -= A d0; d1 = c1 d0 + c2 D^-1 r
    FE_TRY(step(q, (const T*)Lq.d0, (T*)Lq.d1, 1.0, VC_SETX));
    // x += d1; r -= A d1 (r = b - A x for the restriction)
    FE_TRY(step(q, (const T*)Lq.d1, nullptr, 1.0, 0));
    AmgLevel& Cq = h->lev[q + 1];
    const bool coarsest = q + 1 == L - 1;
    *bytes += (double)Lq.nnzr * (Lq.b * AMG_NS * sv + 4) + (double)Lq.n * Lq.b * sv + (double)Cq.n * AMG_NS * sv * 2;
    *flops += 2.0 * Lq.nnzr * Lq.b * AMG_NS;
    if (Lq.b == 3)
      k_vc_restrict<T, 3><<<Cq.n, 128, 0, st>>>(Cq.n, Lq.rptr, Lq.rcol, rv(q), (const T*)Lq.r, dinv(q + 1), (T*)Cq.r,
                                                coarsest ? nullptr : (T*)Cq.d0, coef(q + 1), Lq.n);
    else
      k_vc_restrict<T, AMG_NS><<<Cq.n, 128, 0, st>>>(Cq.n, Lq.rptr, Lq.rcol, rv(q), (const T*)Lq.r, dinv(q + 1),
                                                     (T*)Cq.r, coarsest ? nullptr : (T*)Cq.d0, coef(q + 1), Lq.n);
    FE_CUDA(cudaGetLastError());
  }
  if (fused) {  // levels q0..L-1 in one block (the bytes and flops of the kernels it replaces)
    VcBottomArgs<T> a{};
    a.nb = L - q0;
    for (int l = 0; l < a.nb; l++) {
      AmgLevel& Lq = h->lev[q0 + l];
      VcLevelArgs<T>& A = a.lev[l];
      A.n = Lq.n;
      A.nc = Lq.nc;
      A.ptr = Lq.ptr;
      A.col = Lq.col;
      A.val = vals(q0 + l);
      A.dinv = dinv(q0 + l);
      A.coef = coef(q0 + l);
      A.rptr = Lq.rptr;
      A.rcol = Lq.rcol;
      A.rv = rv(q0 + l);
      A.pptr = Lq.pptr;
      A.pcol = Lq.pcol;
      A.pv = pv(q0 + l);
      A.inv = l == a.nb - 1 ? inv(q0 + l) : nullptr;
      A.x = X(q0 + l);
      A.r = (T*)Lq.r;
      A.d0 = (T*)Lq.d0;
      A.d1 = (T*)Lq.d1;
      A.e = (T*)Lq.e;
      if (l < a.nb - 1) {
        const AmgLevel& Cq = h->lev[q0 + l + 1];
        const int B = Lq.b;
        *bytes += 4 * ((double)Lq.nnz * (B * B * sv + 4) + 4.0 * (Lq.n + 1) + (double)Lq.n * B * (sv * 5 + B * sv));
        *flops += 4 * 2.0 * Lq.nnz * B * B;
        *bytes += (double)Lq.nnzr * (B * AMG_NS * sv + 4) + (double)Lq.n * B * sv + (double)Cq.n * AMG_NS * sv * 2;
        *flops += 2.0 * Lq.nnzr * B * AMG_NS;
        *bytes += (double)Lq.nnzp * (B * AMG_NS * sv + 4) + (double)Lq.n * B * sv * 3;
        *flops += 2.0 * Lq.nnzp * B * AMG_NS;
      } else {
        const int N = Lq.n * Lq.b;
        *bytes += (double)N * N * sv;
        *flops += 2.0 * N * N;
      }
    }
    k_vc_bottom<T><<<1, vc_bottom_threads<T>(), 0, st>>>(a);
    FE_CUDA(cudaGetLastError());
  } else {  // coarsest
    AmgLevel& Lc = h->lev[L - 1];
    const int N = Lc.n * Lc.b;
    k_vc_dense<T><<<1, 256, 0, st>>>(N, inv(L - 1), (const T*)Lc.r, X(L - 1));
    FE_CUDA(cudaGetLastError());
    *bytes += (double)N * N * sv;
    *flops += 2.0 * N * N;
  }
  // upward: prolongation, post-smoothing
  for (int q = qf - 1; q >= 0; q--) {
    AmgLevel& Lq = h->lev[q];
    *bytes += (double)Lq.nnzp * (Lq.b * AMG_NS * sv + 4) + (double)Lq.n * Lq.b * sv * 3;
    *flops += 2.0 * Lq.nnzp * Lq.b * AMG_NS;
    const unsigned grid = blocks_for((int64_t)Lq.n * 4, 256);
    if (Lq.b == 3)
      k_vc_prolong<T, 3, 4><<<grid, 256, 0, st>>>(Lq.n, Lq.pptr, Lq.pcol, pv(q), X(q + 1), X(q), (T*)Lq.e, Lq.nc);
    else
      k_vc_prolong<T, AMG_NS, 4><<<grid, 256, 0, st>>>(Lq.n, Lq.pptr, Lq.pcol, pv(q), X(q + 1), X(q), (T*)Lq.e,
                                                       Lq.nc);
    FE_CUDA(cudaGetLastError());
    // r -= A e; d0 = D^-1 r / theta
    FE_TRY(step(q, (const T*)Lq.e, (T*)Lq.d0, 0.0, VC_KEEPX | VC_START));
    // x += d0; r -= A d0; d1 = c1 d0 + c2 D^-1 r; x += d1
    FE_TRY(step(q, (const T*)Lq.d0, (T*)Lq.d1, 1.0, VC_FINAL));
  }
  return FE_OK;
}

// capture the V-cycle of the current precision into a CUDA graph
template <class T, class V>
int capture(fe_mesh m, const V* K0) {
  AmgHier* h = m->amg;
  if (h->exec) {
    cudaGraphExecDestroy(h->exec);
    h->exec = nullptr;
  }
  if (!h->cap) FE_CUDA(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  {  // one wave of resident blocks, no more warps than 16-row groups
    int per_sm = 0;
    FE_TRY(fe_kernel_occupancy((const void*)k_vc_cheb0<V, T>, 256, 0, &per_sm));
    const int64_t groups = ((int64_t)m->nn + VC_RPW - 1) / VC_RPW;
    h->grid0 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((groups + 7) / 8, (int64_t)std::max(per_sm, 1) * m->sm_count));
  }
  double bytes = 0.0, flops = 0.0;
  m->prof_suspend++;
  cudaGraph_t g = nullptr;
  cudaError_t e0 = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
  int rc = e0 == cudaSuccess ? vcycle_launches<T, V>(m, h->cap, K0, h->vin, &bytes, &flops) : FE_ERR_CUDA;
  cudaError_t e1 = e0 == cudaSuccess ? cudaStreamEndCapture(h->cap, &g) : e0;
  m->prof_suspend--;
  if (rc != FE_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e1 != cudaSuccess)
    return fe_set_error("capturing the V-cycle failed: %s", cudaGetErrorString(e1)), FE_ERR_CUDA;
  cudaError_t e2 = cudaGraphInstantiate(&h->exec, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) return fe_set_error("instantiating the V-cycle graph failed: %s", cudaGetErrorString(e2)), FE_ERR_CUDA;
  h->exec_prec = m->prec;
  h->vc_bytes = bytes;
  h->vc_flops = flops;
  return FE_OK;
}

}  // namespace

int fe_amg_setup(fe_mesh m) {
  if (!m->amg) {
    m->amg = new AmgHier();
    int rc = build_structure(m);
    if (rc != FE_OK) {
      fe_amg_free(m);
      return rc;
    }
  }
  m->amg->ready = false;
  if (m->prec == FE_PREC_FP64) FE_TRY((numeric_all<double, double>(m, m->K64)));
  else if (m->prec == FE_PREC_MIXED_BF16) FE_TRY((numeric_all<float, __nv_bfloat16>(m, m->K16)));
  else FE_TRY((numeric_all<float, float>(m, m->K32)));
  m->amg->ready = true;
  return FE_OK;
}

int fe_amg_apply(fe_mesh m, const double* x, void* z, bool z_double) {
  if (!m->amg || !m->amg->ready) return fe_set_error("AMG hierarchy not set up"), FE_ERR_STATE;
  AmgHier* h = m->amg;
  const int64_t N = (int64_t)m->nn * 3;
  const bool d64 = m->prec == FE_PREC_FP64;
  FE_TRY(ensure_vectors(m, d64 ? 8 : 4));
  if (!h->vin) FE_TRY(dev_alloc(m, &h->vin, (size_t)N));
  // pc_type 2 with the FP32 tangent: the smoother reads a BF16 copy of the
  // fine level (half the bytes of the V-cycle's dominant passes); coarse
  // levels, transfers and vectors stay FP32
  const bool bf_smooth = m->pc_type == 2 && m->prec == FE_PREC_MIXED_FP32;
  const int variant = bf_smooth ? 16 : m->prec;
  if (!h->exec || h->exec_prec != variant) {
    if (d64) FE_TRY((capture<double, double>(m, m->K64)));
    else if (m->prec == FE_PREC_MIXED_BF16 || bf_smooth) FE_TRY((capture<float, __nv_bfloat16>(m, m->K16)));
    else FE_TRY((capture<float, float>(m, m->K32)));
    h->exec_prec = variant;
  }
  FE_CUDA(cudaMemcpyAsync(h->vin, x, N * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  {
    FE_SCOPE_F(m, FE_PROF_PC, h->vc_bytes, h->vc_flops);
    FE_CUDA(cudaGraphLaunch(h->exec, m->stream));
  }
  const unsigned g = blocks_for(N, 256);
  if (d64) {
    if (z_double) FE_CUDA(cudaMemcpyAsync(z, h->lev[0].x, N * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
    else k_vc_convert<double, float><<<g, 256, 0, m->stream>>>(N, (const double*)h->lev[0].x, (float*)z);
  } else {
    if (z_double) k_vc_convert<float, double><<<g, 256, 0, m->stream>>>(N, (const float*)h->lev[0].x, (double*)z);
    else FE_CUDA(cudaMemcpyAsync(z, h->lev[0].x, N * sizeof(float), cudaMemcpyDeviceToDevice, m->stream));
  }
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

void fe_amg_free(fe_mesh m) {
  if (!m->amg) return;
  if (m->amg->exec) cudaGraphExecDestroy(m->amg->exec);
  if (m->amg->cap) cudaStreamDestroy(m->amg->cap);
  for (void* p : m->amg->allocs) cudaFreeAsync(p, m->stream);
  m->device_bytes -= m->amg->bytes;
  delete m->amg;
  m->amg = nullptr;
}

// Copy of level `level` of the hierarchy to host buffers (each may be NULL):
// info [5] = n, b, nnz(A_l), nc, nnz(P_l); rho; A_l pattern and FP64 values
// (level 0: the tangent's own pattern and values are not copied), absent
// components, aggregates, and P_l's pattern and FP64 values.
extern "C" int fe_amg_get_level(fe_mesh m, int level, int64_t* info, double* rho, int32_t* ptr, int32_t* col,
                                double* val, uint8_t* absent, int32_t* agg, int32_t* pptr, int32_t* pcol,
                                double* pval) {
  if (!m) return fe_set_error("NULL mesh"), FE_ERR_ARG;
  if (!m->amg || !m->amg->ready) return fe_set_error("no AMG hierarchy"), FE_ERR_STATE;
  AmgHier* h = m->amg;
  if (level < 0 || level >= h->nlev) return fe_set_error("level %d outside [0, %d)", level, h->nlev), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  const AmgLevel& L = h->lev[level];
  const bool last = level == h->nlev - 1;
  if (info) {
    info[0] = L.n;
    info[1] = L.b;
    info[2] = L.nnz;
    info[3] = last ? 0 : L.nc;
    info[4] = last ? 0 : L.nnzp;
  }
  if (rho) *rho = L.rho;
  // values in FP64 (widened from the FP32 numbers of the mixed forms)
  auto copy_vals = [&](double* dst, const double* s64, const float* s32, int64_t count) -> int {
    if (s64) {
      FE_CUDA(cudaMemcpy(dst, s64, sizeof(double) * count, cudaMemcpyDeviceToHost));
    } else {
      std::vector<float> tmp(count);
      FE_CUDA(cudaMemcpy(tmp.data(), s32, sizeof(float) * count, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < count; i++) dst[i] = (double)tmp[i];
    }
    return FE_OK;
  };
  if (level > 0) {
    if (ptr) FE_CUDA(cudaMemcpy(ptr, L.ptr, sizeof(int) * (L.n + 1), cudaMemcpyDeviceToHost));
    if (col) FE_CUDA(cudaMemcpy(col, L.col, sizeof(int) * L.nnz, cudaMemcpyDeviceToHost));
    if (val) FE_TRY(copy_vals(val, L.val64, L.val32, L.nnz * L.b * L.b));
  }
  if (absent) FE_CUDA(cudaMemcpy(absent, L.absent, L.n, cudaMemcpyDeviceToHost));
  if (!last) {
    if (agg) FE_CUDA(cudaMemcpy(agg, L.agg, sizeof(int) * L.n, cudaMemcpyDeviceToHost));
    if (pptr) FE_CUDA(cudaMemcpy(pptr, L.pptr, sizeof(int) * (L.n + 1), cudaMemcpyDeviceToHost));
    if (pcol) FE_CUDA(cudaMemcpy(pcol, L.pcol, sizeof(int) * L.nnzp, cudaMemcpyDeviceToHost));
    if (pval) FE_TRY(copy_vals(pval, L.p64, L.p32, L.nnzp * L.b * AMG_NS));
  }
  return FE_OK;
}

extern "C" int fe_amg_levels(fe_mesh m) { return (m && m->amg && m->amg->ready) ? m->amg->nlev : 0; }

FE_DBG_BOUNDS_READER(fe_dbg_bounds_amg)
