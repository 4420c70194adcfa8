// fe_krylov.cu -- block-CSR SpMV, nodal block-Jacobi and lower-Schur
// preconditioners, reductions, GMRES with modified Gram-Schmidt Arnoldi
// (paper: GMRES with MGS, Section "Test problems and solvers details"), and
// the L-BFGS two-loop recursion (Section "Numerical solvers", BFGS method).
//
// The Arnoldi step is one persistent cooperative kernel: each block keeps
// its slice of w on chip (shared memory for the sequential sweep, registers
// for the blocked one) for the whole orthogonalisation, so each basis vector
// v_i leaves HBM once per step; the inner products are reduced in a fixed
// order (block tree, then block partials in block order) between bounded
// grid barriers -- one per inner product for the sequential MGS sweep, one
// per block of 8 basis vectors for the blocked form.  The SpMV streams block
// rows in 32-block chunks with a segmented row-sum scan.  The two-loop
// recursion uses the persistent structure with q (or z) held in registers.
#include <algorithm>
#include <climits>
#include <cmath>

#include "fe_internal.h"

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// block sum, result broadcast to all threads
__device__ __forceinline__ double block_sum_all(double v, double* sh) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  double t = lane < nw ? sh[lane] : 0.0;
  t = warp_sum(t);
  return t;
}

// sum of the per-block partials in block order (every block gets the same value)
__device__ __forceinline__ double sum_partials(const double* part, double* sh) {
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += ((volatile const double*)part)[b];
  return block_sum_all(s, sh);
}

// ---------------------------------------------------------------- grid reduction with publish
// Sequential inner products of the persistent kernels, one grid-wide
// reduction each.  Warp 0 of every block does the synchronisation:
//   arrive : lane 0 stores the block partial and increments the arrival
//            counter with acq_rel semantics (atom.inc wraps to 0 on the last
//            arrival, so the counter needs no reset);
//   publish: the last block to arrive adds the partials in block order
//            (fixed order: deterministic for a given grid), resets the slot
//            of the next step to a sentinel and stores the total with
//            release semantics into this step's slot;
//   wait   : the other blocks poll this step's slot (acquire loads) until it
//            holds a value instead of the sentinel.
// Two slots alternate by the global step sequence number seq, which lives in
// device memory across launches.  The sentinel is a NaN payload that no
// arithmetic produces.  The wait is bounded (2^26 polls, seconds): on
// timeout the block records DEV_ERR_TIMEOUT and the kernel ends.  The
// limit is the mesh's (fe_set_wait_limit; 2^26 polls by default).
constexpr unsigned long long kSentinel = 0x7FF4DEAD5EEDF00DULL;

__device__ __forceinline__ unsigned atom_inc_acq_rel(unsigned* p, unsigned lim) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.inc.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(lim) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ double ld_relaxed_f64(const double* p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}

struct GridSync {
  unsigned* count;           // arrival counter
  unsigned* seq;             // global step sequence
  unsigned long long* slot;  // [2] published totals
  int* err;
  unsigned limit;            // polls before a wait gives up (fe_set_wait_limit)
};

// lane 0 of warp 0 only: returns 1 for the last block to arrive
__device__ __forceinline__ int grid_arrive(const GridSync& gs, double* part, double bsum) {
  part[blockIdx.x] = bsum;
  if (gridDim.x == 1) return 1;  // one block: nothing to synchronise with
  return atom_inc_acq_rel(gs.count, gridDim.x - 1) == gridDim.x - 1;
}

// warp 0: publish (last block) or wait; all threads: the total in `out`
__device__ __forceinline__ bool grid_complete(const GridSync& gs, const double* part, unsigned seq, int last,
                                              double* s_val, int* s_fail, double& out) {
  if (gridDim.x == 1) {  // one block: its own partial is the total
    if (threadIdx.x == 0) {
      *s_val = part[0];
      *s_fail = 0;
    }
    __syncthreads();
    out = *s_val;
    return true;
  }
  if (threadIdx.x < 32) {
    last = __shfl_sync(0xffffffffu, last, 0);
    unsigned long long* slot = gs.slot + (seq & 1u);
    if (last) {
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
      double s = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) s += ld_relaxed_f64(part + b);
      s = warp_sum(s);
      if (threadIdx.x == 0) {
        st_relaxed_u64(gs.slot + ((seq + 1u) & 1u), kSentinel);
        *(volatile unsigned*)gs.seq = seq + 1u;
        st_release_u64(slot, (unsigned long long)__double_as_longlong(s));
        *s_val = s;
        *s_fail = 0;
      }
    } else if (threadIdx.x == 0) {
      unsigned spins = 0;
      unsigned long long v;
      *s_fail = 0;
      while ((v = ld_acquire_u64(slot)) == kSentinel) {
        if (++spins > gs.limit || *(volatile int*)gs.err != DEV_OK) {
          atomicCAS(gs.err, DEV_OK, DEV_ERR_TIMEOUT);
          *s_fail = 1;
          break;
        }
      }
      *s_val = __longlong_as_double((long long)v);
    }
  }
  __syncthreads();
  out = *s_val;
  return *s_fail == 0;
}

// block sum with the result in thread 0 (others: partial garbage)
__device__ __forceinline__ double block_sum0(double v, double* sh) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// ---------------------------------------------------------------- persistent Arnoldi (MGS)
// Step j.  Block b owns the contiguous slice [b*S, min((b+1)*S, n)) of every
// vector (S = NPT*blockDim values, NPT a multiple of 3, so slices hold whole
// nodes); w's slice lives in shared memory for the whole sweep.  For
// i = 0..j: h_ij = <w, V_i> (warp sums -> one block barrier -> warp 0 adds the
// warp sums and runs the grid reduction -> one block barrier), w -= h_ij V_i;
// V_{i+1}'s slice is loaded into registers before the reduction.  Then
// h_{j+1,j} = ||w||, V_{j+1} = w / h_{j+1,j}, optionally z = D^{-1} V_{j+1}
// (nodal block-Jacobi, the input of the next SpMV), and block 0 applies the
// previous Givens rotations to column j, forms the new one and updates g.
// Rows of V have a leading dimension rounded up to 32 values (256 bytes).
// warp 0 only: grid reduction of the block total `b` (valid in every lane);
// publishes or waits; lane 0 leaves the total in *s_val
__device__ __forceinline__ void grid_reduce_w0(const GridSync& gs, double* part, unsigned seq, double b, double* s_val,
                                               int* s_fail) {
  if (gridDim.x == 1) {  // one block: the block total is the result, no grid traffic
    if (threadIdx.x == 0) *s_val = b;
    return;
  }
  int last = 0;
  if (threadIdx.x == 0) last = grid_arrive(gs, part, b);
  last = __shfl_sync(0xffffffffu, last, 0);
  unsigned long long* slot = gs.slot + (seq & 1u);
  if (last) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    double s = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += 32) s += ld_relaxed_f64(part + k);
    s = warp_sum(s);
    if (threadIdx.x == 0) {
      st_relaxed_u64(gs.slot + ((seq + 1u) & 1u), kSentinel);
      *(volatile unsigned*)gs.seq = seq + 1u;
      st_release_u64(slot, (unsigned long long)__double_as_longlong(s));
      *s_val = s;
    }
  } else if (threadIdx.x == 0) {
    unsigned spins = 0;
    unsigned long long v;
    while ((v = ld_acquire_u64(slot)) == kSentinel) {
      if (++spins > gs.limit || *(volatile int*)gs.err != DEV_OK) {
        atomicCAS(gs.err, DEV_OK, DEV_ERR_TIMEOUT);
        *s_fail = 1;
        break;
      }
    }
    *s_val = __longlong_as_double((long long)v);
  }
}

template <int NPT, class DT, class ZT>
__global__ void __launch_bounds__(NPT <= 6 ? 1024 : (NPT <= 12 ? 512 : 256))
    k_arnoldi(int64_t n, int j, double* __restrict__ V, int64_t ldv, const double* __restrict__ w,
              double* __restrict__ Hcol, double* part, GridSync gs,
              double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g, double* __restrict__ out,
              const DT* __restrict__ Dinv, ZT* __restrict__ z, double target, int kmax, int it0, int max_it) {
  extern __shared__ __align__(16) double ws[];
  __shared__ double wpart[32];
  __shared__ double s_val;
  __shared__ int s_fail;
  // speculative batches: a step queued after the cycle ended does nothing
  if (*(volatile double*)(out + 7) != 0.0) return;
  unsigned seq = *(volatile unsigned*)gs.seq;  // no reduction completes before every block has read it
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t S = (int64_t)NPT * blockDim.x;
  const int64_t base = (int64_t)blockIdx.x * S;
  const int64_t len = n - base < S ? n - base : S;
  for (int64_t k = threadIdx.x; k < S; k += blockDim.x) ws[k] = k < len ? w[base + k] : 0.0;
  if (threadIdx.x == 0) s_fail = 0;
  double vc[NPT], vn[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    int64_t k = threadIdx.x + (int64_t)s * blockDim.x;
    vc[s] = k < len ? V[base + k] : 0.0;
  }
  __syncthreads();
  for (int i = 0; i <= j; i++) {
    double loc = 0.0;
#pragma unroll
    for (int s = 0; s < NPT; s++) loc += ws[threadIdx.x + s * blockDim.x] * vc[s];
    loc = warp_sum(loc);
    if (lane == 0) wpart[wid] = loc;
    if (i < j) {
      const double* vi = V + (int64_t)(i + 1) * ldv + base;
#pragma unroll
      for (int s = 0; s < NPT; s++) {
        int64_t k = threadIdx.x + (int64_t)s * blockDim.x;
        vn[s] = k < len ? vi[k] : 0.0;
      }
    }
    __syncthreads();
    if (wid == 0) grid_reduce_w0(gs, part, seq, warp_sum(lane < nw ? wpart[lane] : 0.0), &s_val, &s_fail);
    seq++;
    __syncthreads();
    if (s_fail) return;
    const double h = s_val;
    if (blockIdx.x == 0 && threadIdx.x == 0) Hcol[i] = h;
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      ws[threadIdx.x + s * blockDim.x] -= h * vc[s];
      vc[s] = vn[s];
    }
  }
  double loc = 0.0;
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    double a = ws[threadIdx.x + s * blockDim.x];
    loc += a * a;
  }
  loc = warp_sum(loc);
  if (lane == 0) wpart[wid] = loc;
  __syncthreads();
  if (wid == 0) grid_reduce_w0(gs, part, seq, warp_sum(lane < nw ? wpart[lane] : 0.0), &s_val, &s_fail);
  __syncthreads();
  if (s_fail) return;
  const double hn = sqrt(s_val);
  if (hn > 0.0) {
    const double inv = 1.0 / hn;
    double* vnx = V + (int64_t)(j + 1) * ldv + base;
    for (int64_t k = threadIdx.x; k < len; k += blockDim.x) {
      double v = ws[k] * inv;
      ws[k] = v;
      vnx[k] = v;
    }
    if (z) {
      __syncthreads();
      for (int64_t a = threadIdx.x; a < len / 3; a += blockDim.x) {
        const DT* D = Dinv + ((base / 3) + a) * 9;
        double x0 = ws[3 * a], x1 = ws[3 * a + 1], x2 = ws[3 * a + 2];
        ZT* zo = z + base + 3 * a;
        if constexpr (sizeof(DT) == 8) {
          zo[0] = (ZT)(D[0] * x0 + D[1] * x1 + D[2] * x2);
          zo[1] = (ZT)(D[3] * x0 + D[4] * x1 + D[5] * x2);
          zo[2] = (ZT)(D[6] * x0 + D[7] * x1 + D[8] * x2);
        } else {
          float f0 = (float)x0, f1 = (float)x1, f2 = (float)x2;
          zo[0] = (ZT)(D[0] * f0 + D[1] * f1 + D[2] * f2);
          zo[1] = (ZT)(D[3] * f0 + D[4] * f1 + D[5] * f2);
          zo[2] = (ZT)(D[6] * f0 + D[7] * f1 + D[8] * f2);
        }
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Hcol[j + 1] = hn;
    for (int i = 0; i < j; i++) {
      double a = Hcol[i], c = Hcol[i + 1];
      Hcol[i] = cs[i] * a + sn[i] * c;
      Hcol[i + 1] = -sn[i] * a + cs[i] * c;
    }
    double a = Hcol[j], c = Hcol[j + 1];
    double r = hypot(a, c);
    cs[j] = a / r;
    sn[j] = c / r;
    Hcol[j] = r;
    Hcol[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    double res = fabs(g[j + 1]);
    out[0] = res;
    out[1] = hn;
    out[8] = (double)(j + 1);  // steps completed in this cycle
    if (!(res > target) || hn == 0.0 || j + 1 >= kmax || it0 + j + 1 >= max_it) out[7] = 1.0;
  }
}

// ---------------------------------------------------------------- low-synchronisation MGS step
// Modified Gram-Schmidt in its compact-WY form: the product of the j+1 MGS
// projectors (I - q_j q_j^T) ... (I - q_0 q_0^T) equals I - Q T Q^T with
// T = (I + L)^{-1}, L the strictly lower triangle of Q^T Q, Q = [V_0 .. V_j].
// The MGS coefficients are therefore h = (I + L)^{-1} Q^T w: one grid
// reduction of the j+1 inner products Q^T w together with the j products
// V_j^T V_i (row j of L), a triangular solve, and one more sweep w -= Q h.
// In exact arithmetic the step equals the sequential MGS sweep; it takes 2
// grid reductions instead of j + 2, at about 1.5x the FP64 work (published:
// Swirydowicz, Langou, Ananthan, Yang and Thomas, low-synchronisation
// Gram-Schmidt and GMRES, 2020).
//
// Block b owns the same contiguous slice as k_arnoldi; the slices of w and
// V_j live in shared memory.  Per-warp partials of all 2j+1 inner products
// go to shared memory without block barriers; the block sums go to
// part[block][2j+1]; the last block to arrive adds them in block order,
// stores row j of L, solves (I + L) h = s with one warp and publishes h.
__device__ __forceinline__ void publish_seq(const GridSync& gs, unsigned seq) {
  st_relaxed_u64(gs.slot + ((seq + 1u) & 1u), kSentinel);
  *(volatile unsigned*)gs.seq = seq + 1u;
  st_release_u64(gs.slot + (seq & 1u), (unsigned long long)seq);
}

__device__ __forceinline__ bool wait_seq(const GridSync& gs, unsigned seq) {
  unsigned spins = 0;
  while (ld_acquire_u64(gs.slot + (seq & 1u)) == kSentinel) {
    if (++spins > gs.limit || *(volatile int*)gs.err != DEV_OK) {
      atomicCAS(gs.err, DEV_OK, DEV_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

template <int NPT, class DT, class ZT>
__global__ void __launch_bounds__(NPT <= 6 ? 1024 : (NPT <= 12 ? 512 : 256))
    k_arnoldi_ls(int64_t n, int j, double* __restrict__ V, int64_t ldv, const double* __restrict__ w,
                 double* __restrict__ Hcol, double* part, double* partv, GridSync gs, double* __restrict__ Lmat,
                 int ldl, double* hpub, double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                 double* __restrict__ out, const DT* __restrict__ Dinv, ZT* __restrict__ z, double target, int kmax,
                 int it0, int max_it) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double wpart[32];
  __shared__ double s_val;
  __shared__ int s_fail, s_last;
  if (*(volatile double*)(out + 7) != 0.0) return;
  unsigned seq = *(volatile unsigned*)gs.seq;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t S = (int64_t)NPT * blockDim.x;
  const int64_t base = (int64_t)blockIdx.x * S;
  const int64_t len = n - base < S ? n - base : S;
  const int nv = 2 * j + 1;  // s_0..s_j, then l_0..l_{j-1}
  double* ws = sm;           // [S]  w
  double* vj = sm + S;       // [S]  V_j
  double* pw = sm + 2 * S;   // [nv][32] per-warp partials
  for (int64_t k = threadIdx.x; k < S; k += blockDim.x) {
    ws[k] = k < len ? w[base + k] : 0.0;
    vj[k] = k < len ? V[(int64_t)j * ldv + base + k] : 0.0;
  }
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  double vc[NPT], vn[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    int64_t k = threadIdx.x + (int64_t)s * blockDim.x;
    vc[s] = k < len ? V[base + k] : 0.0;
  }
  for (int i = 0; i <= j; i++) {
    if (i < j) {
      const double* vi = V + (int64_t)(i + 1) * ldv + base;
#pragma unroll
      for (int s = 0; s < NPT; s++) {
        int64_t k = threadIdx.x + (int64_t)s * blockDim.x;
        vn[s] = k < len ? vi[k] : 0.0;
      }
    }
    double ps = 0.0, pl = 0.0;
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      const int64_t k = threadIdx.x + (int64_t)s * blockDim.x;
      ps += ws[k] * vc[s];
      pl += vj[k] * vc[s];
    }
    ps = warp_sum(ps);
    if (i < j) pl = warp_sum(pl);
    if (lane == 0) {
      pw[i * 32 + wid] = ps;
      if (i < j) pw[(j + 1 + i) * 32 + wid] = pl;
    }
#pragma unroll
    for (int s = 0; s < NPT; s++) vc[s] = vn[s];
  }
  __syncthreads();
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double t = 0.0;
    for (int q = 0; q < nw; q++) t += pw[v * 32 + q];
    partv[(int64_t)blockIdx.x * nv + v] = t;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_last = gridDim.x == 1 ? 1 : (atom_inc_acq_rel(gs.count, gridDim.x - 1) == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      double t = 0.0;
      for (int b = 0; b < (int)gridDim.x; b++) t += ld_relaxed_f64(partv + (int64_t)b * nv + v);
      if (v <= j) hpub[v] = t;
      else Lmat[(int64_t)j * ldl + (v - j - 1)] = t;
    }
    __threadfence();
    __syncthreads();
    if (wid == 0) {  // forward substitution (I + L) h = s, column by column
      for (int i = 0; i <= j; i++) {
        const double hi = ld_relaxed_f64(hpub + i);
        for (int r = i + 1 + lane; r <= j; r += 32) hpub[r] -= ld_relaxed_f64(Lmat + (int64_t)r * ldl + i) * hi;
        __threadfence();
        __syncwarp();
      }
      if (lane == 0 && gridDim.x > 1) publish_seq(gs, seq);
    }
  } else if (threadIdx.x == 0) {
    if (!wait_seq(gs, seq)) s_fail = 1;
  }
  if (gridDim.x > 1) seq++;
  __syncthreads();
  if (s_fail) return;
  for (int i = 0; i <= j; i++) {  // w -= sum_i h_i V_i
    const double hi = ld_relaxed_f64(hpub + i);
    const double* vi = V + (int64_t)i * ldv + base;
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      const int64_t k = threadIdx.x + (int64_t)s * blockDim.x;
      if (k < len) ws[k] -= hi * vi[k];
    }
  }
  double loc = 0.0;
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    const int64_t k = threadIdx.x + (int64_t)s * blockDim.x;
    loc += ws[k] * ws[k];
  }
  loc = warp_sum(loc);
  if (lane == 0) wpart[wid] = loc;
  __syncthreads();
  if (wid == 0) grid_reduce_w0(gs, part, seq, warp_sum(lane < nw ? wpart[lane] : 0.0), &s_val, &s_fail);
  __syncthreads();
  if (s_fail) return;
  const double hn = sqrt(s_val);
  if (hn > 0.0) {
    const double inv = 1.0 / hn;
    double* vnx = V + (int64_t)(j + 1) * ldv + base;
    for (int64_t k = threadIdx.x; k < len; k += blockDim.x) {
      double v = ws[k] * inv;
      ws[k] = v;
      vnx[k] = v;
    }
    if (z) {
      __syncthreads();
      for (int64_t a = threadIdx.x; a < len / 3; a += blockDim.x) {
        const DT* D = Dinv + ((base / 3) + a) * 9;
        double x0 = ws[3 * a], x1 = ws[3 * a + 1], x2 = ws[3 * a + 2];
        ZT* zo = z + base + 3 * a;
        if constexpr (sizeof(DT) == 8) {
          zo[0] = (ZT)(D[0] * x0 + D[1] * x1 + D[2] * x2);
          zo[1] = (ZT)(D[3] * x0 + D[4] * x1 + D[5] * x2);
          zo[2] = (ZT)(D[6] * x0 + D[7] * x1 + D[8] * x2);
        } else {
          float f0 = (float)x0, f1 = (float)x1, f2 = (float)x2;
          zo[0] = (ZT)(D[0] * f0 + D[1] * f1 + D[2] * f2);
          zo[1] = (ZT)(D[3] * f0 + D[4] * f1 + D[5] * f2);
          zo[2] = (ZT)(D[6] * f0 + D[7] * f1 + D[8] * f2);
        }
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int i = 0; i <= j; i++) Hcol[i] = ld_relaxed_f64(hpub + i);
    Hcol[j + 1] = hn;
    for (int i = 0; i < j; i++) {
      double a = Hcol[i], c = Hcol[i + 1];
      Hcol[i] = cs[i] * a + sn[i] * c;
      Hcol[i + 1] = -sn[i] * a + cs[i] * c;
    }
    double a = Hcol[j], c = Hcol[j + 1];
    double r = hypot(a, c);
    cs[j] = a / r;
    sn[j] = c / r;
    Hcol[j] = r;
    Hcol[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    double res = fabs(g[j + 1]);
    out[0] = res;
    out[1] = hn;
    out[8] = (double)(j + 1);
    if (!(res > target) || hn == 0.0 || j + 1 >= kmax || it0 + j + 1 >= max_it) out[7] = 1.0;
  }
}

// ---------------------------------------------------------------- blocked MGS step
// Modified Gram-Schmidt over the basis in blocks of P vectors.  Inside a
// block the sequential MGS coefficients follow from the block's inner
// products with the current w and from the block's own Gram entries:
//   <w - sum_{l<m} h_l v_l, v_m> = <w, v_m> - sum_{l<m} h_l <v_l, v_m>,
// i.e. h_B = (I + L_B)^{-1} V_B^T w with L_B the strictly lower triangle of
// V_B^T V_B (the compact-WY identity of the low-synchronisation step,
// applied per block; equal to the MGS coefficients in exact arithmetic, the
// sequential MGS sweep for P = 1).  Between blocks w is updated before the
// next block's inner products, as in MGS.  The entries <v_{j+1}, v_l>, v_l in
// the block of v_{j+1}, are reduced together with ||w||^2 at the end of step
// j, and the new row of T_B = (I + L_B)^{-1} is stored, so step j takes
// ceil((j+1)/P) + 1 grid reductions instead of j + 2, at the same 2 FMAs per
// entry and basis vector (plus at most P - 1 inner products for the Gram
// row).  w stays in registers; each sweep applies the previous block's
// update and accumulates the current block's inner products, one vector per
// pass, with the next pass's vector loaded while the current one is used.
//
// The reductions have their own step sequence and two sets of P published
// slots (bar[6], bar[8..]) so that other persistent kernels' use of the
// shared slots cannot leave a stale value in a slot this kernel polls.
struct BlockSync {
  unsigned* count;           // arrival counter (shared with GridSync)
  unsigned* seq;             // this kernel's step sequence
  unsigned long long* pub;   // [2][BMGS_P] published values, kSentinel when not yet
  int* err;
  unsigned limit;            // polls before a wait gives up (fe_set_wait_limit)
};

// Warp reduce-scatter of P values per lane: returns, in every lane, the warp
// total of value index lane / (32 / P).  Each of the first log2(P) exchange
// steps halves the values a lane carries (it keeps the half selected by its
// lane bit and adds the partner's copy of that half), then plain xor steps
// finish the sum: P - 1 + 5 - log2(P) shuffles instead of 5 P.
template <int P>
__device__ __forceinline__ double warp_reduce_scatter(double (&v)[P], int lane) {
#pragma unroll
  for (int cnt = P, o = 16; cnt > 1; cnt >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < cnt / 2; k++) {
      const double send = up ? v[k] : v[k + cnt / 2];
      const double keep = up ? v[k + cnt / 2] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double t = v[0];
#pragma unroll
  for (int o = 16 / P; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// warp 0 of every block.  Lane l holds the block total of value l % P.  The
// last block to arrive adds the partials of all blocks in block order, and
// when `solve` is set (trow[m][l], l < m < nc: the block's rows of T_B)
// turns the totals s into h = T_B s; lanes m < P of every block end with the
// value m in out_sh[m].  false: the wait timed out (error word set).
template <int P>
__device__ __forceinline__ bool bm_reduce_w0(const BlockSync& bs, double* part, unsigned seq, double t,
                                             const double (*trow)[P], bool solve, int nc, double* out_sh) {
  const int lane = threadIdx.x & 31;
  if (gridDim.x > 1) {
    if (lane < P) part[(int64_t)blockIdx.x * P + lane] = t;
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0) last = atom_inc_acq_rel(bs.count, gridDim.x - 1) == gridDim.x - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) {
      bool ok = true;
      if (lane < P) {
        const unsigned long long* slot = bs.pub + (seq & 1u) * BMGS_P + lane;
        unsigned spins = 0;
        unsigned long long u;
        while ((u = ld_acquire_u64(slot)) == kSentinel) {
          if (++spins > bs.limit || *(volatile int*)bs.err != DEV_OK) {
            atomicCAS(bs.err, DEV_OK, DEV_ERR_TIMEOUT);
            ok = false;
            break;
          }
        }
        out_sh[lane] = __longlong_as_double((long long)u);
      }
      return __all_sync(0xffffffffu, ok);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    t = 0.0;
    for (int b = lane / P; b < (int)gridDim.x; b += 32 / P) t += ld_relaxed_f64(part + (int64_t)b * P + (lane % P));
#pragma unroll
    for (int o = P; o < 32; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  if (solve) {  // h_m = s_m + sum_{l<m} T[m][l] s_l
    double h = t;
#pragma unroll
    for (int l = 0; l < P - 1; l++) {
      const double sl = __shfl_sync(0xffffffffu, t, l);
      if (lane > l && lane < nc) h += trow[lane][l] * sl;
    }
    t = h;
  }
  if (lane < P) {
    out_sh[lane] = t;
    if (gridDim.x > 1) {
      st_relaxed_u64(bs.pub + ((seq + 1u) & 1u) * BMGS_P + lane, kSentinel);
      st_release_u64(bs.pub + (seq & 1u) * BMGS_P + lane, (unsigned long long)__double_as_longlong(t));
    }
  }
  if (lane == 0 && gridDim.x > 1) *(volatile unsigned*)bs.seq = seq + 1u;
  return true;
}

__device__ __forceinline__ void prefetch_l2(const double* p, int64_t count) {
  // bulk L2 prefetch of a 16-byte aligned run (rows of V are 256-byte aligned
  // and zero-padded, so rounding the size up stays inside the row)
  const uint32_t bytes = (uint32_t)(((count * 8) + 15) & ~(int64_t)15);
  if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// A thread owns NPT / 2 pairs of consecutive values of its block's slice:
// values s = 2q, 2q + 1 sit at slice offset bm_off(q) and bm_off(q) + 1, so
// each pair is one 16-byte load (slices start at even offsets of 256-byte
// aligned rows).
__device__ __forceinline__ int64_t bm_off(int q) { return 2 * (threadIdx.x + (int64_t)q * blockDim.x); }

// this thread's NPT values of a vector slice (0 past its end)
template <int NPT>
__device__ __forceinline__ void load_slice(double (&r)[NPT], const double* __restrict__ v, int64_t len) {
#pragma unroll
  for (int q = 0; q < NPT / 2; q++) {
    const int64_t k = bm_off(q);
    if (k + 1 < len) {
      const double2 p = __ldcg(reinterpret_cast<const double2*>(v + k));
      r[2 * q] = p.x;
      r[2 * q + 1] = p.y;
    } else {
      r[2 * q] = k < len ? __ldcg(v + k) : 0.0;
      r[2 * q + 1] = 0.0;
    }
  }
}

template <int NPT, int P, class DT, class ZT>
__global__ void __launch_bounds__(NPT <= 12 ? 512 : 256)
    k_arnoldi_bm(int64_t n, int j, double* __restrict__ V, int64_t ldv, const double* __restrict__ w,
                 double* __restrict__ Hcol, double* part, BlockSync bs, double* __restrict__ T,
                 double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g, double* __restrict__ out,
                 const DT* __restrict__ Dinv, ZT* __restrict__ z, double target, int kmax, int it0, int max_it) {
  static_assert(P == 2 || P == 4 || P == 8, "block of 2, 4 or 8 basis vectors");
  extern __shared__ __align__(16) double ws[];
  __shared__ double wpart[P][32];
  __shared__ double s_h[P];       // the last reduction's results (h of the block, or the final norm/Gram row)
  __shared__ double s_trow[P][P];
  __shared__ int s_fail;
  if (*(volatile double*)(out + 7) != 0.0) return;
  unsigned seq = *(volatile unsigned*)bs.seq;  // no reduction completes before every block has read it
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t S = (int64_t)NPT * blockDim.x;
  const int64_t base = (int64_t)blockIdx.x * S;
  const int64_t len = n - base < S ? n - base : S;
  const int nb = j / P + 1;                // blocks of the basis v_0..v_j
  const int nlast = j + 1 - (nb - 1) * P;  // vectors in the last block
  const int ng = (j + 1) % P ? nlast : 0;  // Gram entries of v_{j+1} (its block is the last one)
  if (threadIdx.x == 0) s_fail = 0;
  if (threadIdx.x < P) s_h[threadIdx.x] = 0.0;
  if (threadIdx.x < P && (int)threadIdx.x <= j) prefetch_l2(V + (int64_t)threadIdx.x * ldv + base, len);
  double wr[NPT];
  load_slice<NPT>(wr, w + base, len);
  double cur[NPT], nxt[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) nxt[s] = 0.0;
  load_slice<NPT>(cur, V + base, len);  // first pass: the inner product with v_0
  for (int kb = 0; kb <= nb; kb++) {
    const int np = kb == 0 ? 0 : (kb == nb ? nlast : P);        // previous block: update
    const int nc = kb == nb ? ng : (kb == nb - 1 ? nlast : P);  // current block (final sweep: Gram row)
    const double* Vp = V + (int64_t)(kb > 0 ? kb - 1 : 0) * P * ldv + base;
    const double* Vc = kb < nb ? V + (int64_t)kb * P * ldv + base : Vp;
    // Passes over one vector each: np update passes (w -= h_m v_m, block B-1),
    // then nc inner-product passes (block B; final sweep: the Gram row against
    // block B-1).  The slice of the next pass's vector is loaded into registers
    // while the current one is used.
    const int nq = np + nc;
#pragma unroll
    for (int m = 0; m < P; m++) {
      if (m < np) {
        if (m + 1 < nq) load_slice<NPT>(nxt, m + 1 < np ? Vp + (int64_t)(m + 1) * ldv : Vc, len);
        const double h = s_h[m];
#pragma unroll
        for (int s = 0; s < NPT; s++) wr[s] -= h * cur[s];
#pragma unroll
        for (int s = 0; s < NPT; s++) cur[s] = nxt[s];
      }
    }
    double loc[P];
#pragma unroll
    for (int m = 0; m < P; m++) loc[m] = 0.0;
#pragma unroll
    for (int m = 0; m < P; m++) {
      if (m < nc) {
        if (m + 1 < nc) load_slice<NPT>(nxt, Vc + (int64_t)(m + 1) * ldv, len);
        double a[2] = {0.0, 0.0};  // two chains: each extra one costs an FP64 add per vector
#pragma unroll
        for (int s = 0; s < NPT; s++) a[s & 1] += wr[s] * cur[s];
        loc[m] = a[0] + a[1];
#pragma unroll
        for (int s = 0; s < NPT; s++) cur[s] = nxt[s];
      }
    }
    if (kb == nb) {  // final sweep: [||w||^2, Gram row]
      double a[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int s = 0; s < NPT; s++) a[s & 3] += wr[s] * wr[s];
#pragma unroll
      for (int m = P - 1; m > 0; m--) loc[m] = loc[m - 1];
      loc[0] = (a[0] + a[1]) + (a[2] + a[3]);
    } else {
      // first pass of the next sweep: the update with this block's v_{kb P}
      load_slice<NPT>(cur, V + (int64_t)kb * P * ldv + base, len);
    }
    // the next block's vectors are read from HBM by the next sweep: start them now
    if (kb + 1 < nb && threadIdx.x < P && (kb + 1) * P + (int)threadIdx.x <= j)
      prefetch_l2(V + (int64_t)((kb + 1) * P + threadIdx.x) * ldv + base, len);
    // T rows of the current block (lane m: row kb P + m, entries l < m)
    const bool solve = kb < nb;
    if (wid == 0 && solve && lane < nc) {
      const double* tr = T + (int64_t)(kb * P + lane) * P;
#pragma unroll
      for (int l = 0; l < P - 1; l++)
        if (l < lane) s_trow[lane][l] = tr[l];
    }
    const double r = warp_reduce_scatter<P>(loc, lane);
    if ((lane & (32 / P - 1)) == 0) wpart[lane / (32 / P)][wid] = r;
    __syncthreads();
    if (wid == 0) {
      double t = 0.0;
      for (int q = lane / P; q < nw; q += 32 / P) t += wpart[lane % P][q];
#pragma unroll
      for (int x = P; x < 32; x <<= 1) t += __shfl_xor_sync(0xffffffffu, t, x);
      __syncwarp();
      if (!bm_reduce_w0<P>(bs, part, seq, t, s_trow, solve, nc, s_h) && lane == 0) s_fail = 1;
    }
    if (gridDim.x > 1) seq++;
    __syncthreads();
    if (s_fail) return;
    if (solve && blockIdx.x == 0 && threadIdx.x < nc) Hcol[kb * P + threadIdx.x] = s_h[threadIdx.x];
  }
  // s_h[0] = ||w||^2, s_h[1..ng] = <w, v_l> for the last block's vectors
  const double hn = sqrt(s_h[0]);
  if (hn > 0.0) {
    const double inv = 1.0 / hn;
    double* vnx = V + (int64_t)(j + 1) * ldv + base;
#pragma unroll
    for (int q = 0; q < NPT / 2; q++) {
      const int64_t k = bm_off(q);
      const double v0 = wr[2 * q] * inv, v1 = wr[2 * q + 1] * inv;
      ws[k] = v0;
      ws[k + 1] = v1;
      if (k + 1 < len) *reinterpret_cast<double2*>(vnx + k) = make_double2(v0, v1);
      else if (k < len) vnx[k] = v0;
    }
    if (z) {
      __syncthreads();
      for (int64_t a = threadIdx.x; a < len / 3; a += blockDim.x) {
        const DT* D = Dinv + ((base / 3) + a) * 9;
        double x0 = ws[3 * a], x1 = ws[3 * a + 1], x2 = ws[3 * a + 2];
        ZT* zo = z + base + 3 * a;
        if constexpr (sizeof(DT) == 8) {
          zo[0] = (ZT)(D[0] * x0 + D[1] * x1 + D[2] * x2);
          zo[1] = (ZT)(D[3] * x0 + D[4] * x1 + D[5] * x2);
          zo[2] = (ZT)(D[6] * x0 + D[7] * x1 + D[8] * x2);
        } else {
          float f0 = (float)x0, f1 = (float)x1, f2 = (float)x2;
          zo[0] = (ZT)(D[0] * f0 + D[1] * f1 + D[2] * f2);
          zo[1] = (ZT)(D[3] * f0 + D[4] * f1 + D[5] * f2);
          zo[2] = (ZT)(D[6] * f0 + D[7] * f1 + D[8] * f2);
        }
      }
    }
    // new row of T_B: T[j+1][c] = -(g_c + sum_{c<l<ng} g_l T[b0+l][c]), g_l = <v_{j+1}, v_{b0+l}>
    if (blockIdx.x == 0 && threadIdx.x < ng) {
      const int c = threadIdx.x, b0 = (nb - 1) * P;
      double acc = s_h[1 + c] * inv;
      for (int l = c + 1; l < ng; l++) acc += s_h[1 + l] * inv * T[(int64_t)(b0 + l) * P + c];
      T[(int64_t)(j + 1) * P + c] = -acc;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Hcol[j + 1] = hn;
    for (int i = 0; i < j; i++) {
      double a = Hcol[i], c = Hcol[i + 1];
      Hcol[i] = cs[i] * a + sn[i] * c;
      Hcol[i + 1] = -sn[i] * a + cs[i] * c;
    }
    double a = Hcol[j], c = Hcol[j + 1];
    double r = hypot(a, c);
    cs[j] = a / r;
    sn[j] = c / r;
    Hcol[j] = r;
    Hcol[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    double res = fabs(g[j + 1]);
    out[0] = res;
    out[1] = hn;
    out[8] = (double)(j + 1);
    if (!(res > target) || hn == 0.0 || j + 1 >= kmax || it0 + j + 1 >= max_it) out[7] = 1.0;
  }
}

// The blocked MGS step for vectors too long for a register-resident grid:
// the same passes, reductions and tail as k_arnoldi_bm, with the block's
// slice of w in shared memory (NPT values per thread, up to 18,432 per
// block) and each basis slice read straight from L2/HBM in 16-byte pairs
// (the next block of basis vectors is prefetched into L2 as before).  One
// block per SM holds 152 x 18,432 = 2.8 M unknowns.
template <int NPT, int P, class DT, class ZT>
__global__ void __launch_bounds__(256)
    k_arnoldi_bm_ws(int64_t n, int j, double* __restrict__ V, int64_t ldv, const double* __restrict__ w,
                    double* __restrict__ Hcol, double* part, BlockSync bs, double* __restrict__ T,
                    double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g, double* __restrict__ out,
                    const DT* __restrict__ Dinv, ZT* __restrict__ z, double target, int kmax, int it0, int max_it) {
  static_assert(P == 2 || P == 4 || P == 8, "block of 2, 4 or 8 basis vectors");
  extern __shared__ __align__(16) double ws[];
  __shared__ double wpart[P][32];
  __shared__ double s_h[P];
  __shared__ double s_trow[P][P];
  __shared__ int s_fail;
  if (*(volatile double*)(out + 7) != 0.0) return;
  unsigned seq = *(volatile unsigned*)bs.seq;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t S = (int64_t)NPT * blockDim.x;
  const int64_t base = (int64_t)blockIdx.x * S;
  const int64_t len = n - base < S ? n - base : S;
  const int nb = j / P + 1;
  const int nlast = j + 1 - (nb - 1) * P;
  const int ng = (j + 1) % P ? nlast : 0;
  if (threadIdx.x == 0) s_fail = 0;
  if (threadIdx.x < P) s_h[threadIdx.x] = 0.0;
  if (threadIdx.x < P && (int)threadIdx.x <= j) prefetch_l2(V + (int64_t)threadIdx.x * ldv + base, len);
  // w's slice into shared memory (pairs at the register variant's offsets; 0 past the end)
  for (int q = 0; q < NPT / 2; q++) {
    const int64_t k = bm_off(q);
    double2 p = make_double2(0.0, 0.0);
    if (k + 1 < len) p = __ldcg(reinterpret_cast<const double2*>(w + base + k));
    else if (k < len) p.x = __ldcg(w + base + k);
    ws[k] = p.x;
    ws[k + 1] = p.y;
  }
  auto pair = [&](const double* v, int64_t k) {
    double2 p = make_double2(0.0, 0.0);
    if (k + 1 < len) p = __ldcg(reinterpret_cast<const double2*>(v + k));
    else if (k < len) p.x = __ldcg(v + k);
    return p;
  };
  for (int kb = 0; kb <= nb; kb++) {
    const int np = kb == 0 ? 0 : (kb == nb ? nlast : P);
    const int nc = kb == nb ? ng : (kb == nb - 1 ? nlast : P);
    const double* Vp = V + (int64_t)(kb > 0 ? kb - 1 : 0) * P * ldv + base;
    const double* Vc = kb < nb ? V + (int64_t)kb * P * ldv + base : Vp;
    // update passes w -= h_m v_m (previous block), each thread on its own pairs
    for (int m = 0; m < np; m++) {
      const double h = s_h[m];
      const double* vm = Vp + (int64_t)m * ldv;
      for (int q = 0; q < NPT / 2; q++) {
        const int64_t k = bm_off(q);
        const double2 p = pair(vm, k);
        ws[k] -= h * p.x;
        ws[k + 1] -= h * p.y;
      }
    }
    double loc[P];
#pragma unroll
    for (int m = 0; m < P; m++) loc[m] = 0.0;
#pragma unroll
    for (int m = 0; m < P; m++) {
      if (m < nc) {
        const double* vm = Vc + (int64_t)m * ldv;
        double a[2] = {0.0, 0.0};
        for (int q = 0; q < NPT / 2; q++) {
          const int64_t k = bm_off(q);
          const double2 p = pair(vm, k);
          a[0] += ws[k] * p.x;
          a[1] += ws[k + 1] * p.y;
        }
        loc[m] = a[0] + a[1];
      }
    }
    if (kb == nb) {  // final sweep: [||w||^2, Gram row]
      double a[4] = {0.0, 0.0, 0.0, 0.0};
      for (int q = 0; q < NPT / 2; q++) {
        const int64_t k = bm_off(q);
        a[(2 * q) & 3] += ws[k] * ws[k];
        a[(2 * q + 1) & 3] += ws[k + 1] * ws[k + 1];
      }
#pragma unroll
      for (int m = P - 1; m > 0; m--) loc[m] = loc[m - 1];
      loc[0] = (a[0] + a[1]) + (a[2] + a[3]);
    }
    if (kb + 1 < nb && threadIdx.x < P && (kb + 1) * P + (int)threadIdx.x <= j)
      prefetch_l2(V + (int64_t)((kb + 1) * P + threadIdx.x) * ldv + base, len);
    const bool solve = kb < nb;
    if (wid == 0 && solve && lane < nc) {
      const double* tr = T + (int64_t)(kb * P + lane) * P;
#pragma unroll
      for (int l = 0; l < P - 1; l++)
        if (l < lane) s_trow[lane][l] = tr[l];
    }
    const double r = warp_reduce_scatter<P>(loc, lane);
    if ((lane & (32 / P - 1)) == 0) wpart[lane / (32 / P)][wid] = r;
    __syncthreads();
    if (wid == 0) {
      double t = 0.0;
      for (int q = lane / P; q < nw; q += 32 / P) t += wpart[lane % P][q];
#pragma unroll
      for (int x = P; x < 32; x <<= 1) t += __shfl_xor_sync(0xffffffffu, t, x);
      __syncwarp();
      if (!bm_reduce_w0<P>(bs, part, seq, t, s_trow, solve, nc, s_h) && lane == 0) s_fail = 1;
    }
    if (gridDim.x > 1) seq++;
    __syncthreads();
    if (s_fail) return;
    if (solve && blockIdx.x == 0 && threadIdx.x < nc) Hcol[kb * P + threadIdx.x] = s_h[threadIdx.x];
  }
  const double hn = sqrt(s_h[0]);
  if (hn > 0.0) {
    const double inv = 1.0 / hn;
    double* vnx = V + (int64_t)(j + 1) * ldv + base;
    for (int q = 0; q < NPT / 2; q++) {
      const int64_t k = bm_off(q);
      const double v0 = ws[k] * inv, v1 = ws[k + 1] * inv;
      ws[k] = v0;
      ws[k + 1] = v1;
      if (k + 1 < len) *reinterpret_cast<double2*>(vnx + k) = make_double2(v0, v1);
      else if (k < len) vnx[k] = v0;
    }
    if (z) {
      __syncthreads();
      for (int64_t a = threadIdx.x; a < len / 3; a += blockDim.x) {
        const DT* D = Dinv + ((base / 3) + a) * 9;
        double x0 = ws[3 * a], x1 = ws[3 * a + 1], x2 = ws[3 * a + 2];
        ZT* zo = z + base + 3 * a;
        if constexpr (sizeof(DT) == 8) {
          zo[0] = (ZT)(D[0] * x0 + D[1] * x1 + D[2] * x2);
          zo[1] = (ZT)(D[3] * x0 + D[4] * x1 + D[5] * x2);
          zo[2] = (ZT)(D[6] * x0 + D[7] * x1 + D[8] * x2);
        } else {
          float f0 = (float)x0, f1 = (float)x1, f2 = (float)x2;
          zo[0] = (ZT)(D[0] * f0 + D[1] * f1 + D[2] * f2);
          zo[1] = (ZT)(D[3] * f0 + D[4] * f1 + D[5] * f2);
          zo[2] = (ZT)(D[6] * f0 + D[7] * f1 + D[8] * f2);
        }
      }
    }
    if (blockIdx.x == 0 && threadIdx.x < ng) {
      const int c = threadIdx.x, b0 = (nb - 1) * P;
      double acc = s_h[1 + c] * inv;
      for (int l = c + 1; l < ng; l++) acc += s_h[1 + l] * inv * T[(int64_t)(b0 + l) * P + c];
      T[(int64_t)(j + 1) * P + c] = -acc;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Hcol[j + 1] = hn;
    for (int i = 0; i < j; i++) {
      double a = Hcol[i], c = Hcol[i + 1];
      Hcol[i] = cs[i] * a + sn[i] * c;
      Hcol[i + 1] = -sn[i] * a + cs[i] * c;
    }
    double a = Hcol[j], c = Hcol[j + 1];
    double r = hypot(a, c);
    cs[j] = a / r;
    sn[j] = c / r;
    Hcol[j] = r;
    Hcol[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    double res = fabs(g[j + 1]);
    out[0] = res;
    out[1] = hn;
    out[8] = (double)(j + 1);
    if (!(res > target) || hn == 0.0 || j + 1 >= kmax || it0 + j + 1 >= max_it) out[7] = 1.0;
  }
}

// ---------------------------------------------------------------- SpMV
// float -> double widening with integer operations only.  GB300's FP64 pipe
// issues ~2 lane-operations per clock per SM, so the three hardware
// conversions of every row result of the FP32 SpMV cost about half of the
// kernel's time.  The conversion is exact for every float: normal numbers
// rebias the exponent (+896) and shift the mantissa (<< 29), subnormals are
// normalised with a leading-zero count, zeros keep their sign, infinities
// and NaNs map to the all-ones exponent with the payload in place.
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  uint32_t mant = u & 0x7fffffu;
  uint32_t de;                           // biased double exponent
  if (e == 0xffu) de = 0x7ffu;           // Inf / NaN (payload and quiet bit keep their place)
  else if (e != 0u) de = e + 896u;       // normal: rebias 127 -> 1023
  else if (mant == 0u) de = 0u;          // signed zero
  else {                                 // subnormal: normalise; value = mant 2^-149
    const uint32_t lz = __clz(mant);     // >= 9; leading one moves to bit 23
    de = 905u - lz;
    mant = (mant << (lz - 8u)) & 0x7fffffu;
  }
  const uint64_t bits = ((uint64_t)(u >> 31) << 63) | ((uint64_t)de << 52) | ((uint64_t)mant << 29);
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double widen(double d) { return d; }

template <class V>
__device__ __forceinline__ float ld_val(const V* p);
template <>
__device__ __forceinline__ float ld_val<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ld_val<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

// y_u = K x_u (+ B1 x_p): one warp per block row, one lane per 3x3 block.
// A lane loads its block's column index, its 9 values and the 3 entries of
// x, then accumulates the 3 row sums; the warp reduces them with shuffles.
// The values are tiled (kv_index: 32 blocks per tile, component-major
// inside it), so each of the 9 value loads of a warp reads at most two
// 128-byte runs: with block-major storage every load touched the warp's
// whole 1,152-byte segment and the L1 request rate, not HBM, bounded the
// kernel (ncu: 9x more L1 sectors than DRAM sectors).  Few registers keep
// the SM full of warps, which hides the HBM latency.
template <class VT, class XT, class AT>
__global__ void __launch_bounds__(256) k_spmv(int nn, const int* __restrict__ row_ptr, const int* __restrict__ col,
                                              const VT* __restrict__ val, const XT* __restrict__ x,
                                              double* __restrict__ y, const int* __restrict__ up_ptr,
                                              const int* __restrict__ up_col, const VT* __restrict__ B,
                                              const XT* __restrict__ xp) {
  int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (row >= nn) return;
  const int rs = row_ptr[row], re = row_ptr[row + 1];
  AT a0 = AT(0), a1 = AT(0), a2 = AT(0);
  for (int k = rs + lane; k < re; k += 32) {
    const int c = fe_idx(__ldg(col + k), nn);
    const VT* b = val + kv_index(k, 0);
    AT v[9];
#pragma unroll
    for (int t = 0; t < 9; t++) {
      if constexpr (sizeof(VT) == 8) v[t] = __ldg(b + 32 * t);
      else v[t] = (AT)ld_val<VT>(b + 32 * t);
    }
    const XT* xc = x + 3 * (int64_t)c;
    AT x0 = (AT)xc[0], x1 = (AT)xc[1], x2 = (AT)xc[2];
    a0 += v[0] * x0 + v[1] * x1 + v[2] * x2;
    a1 += v[3] * x0 + v[4] * x1 + v[5] * x2;
    a2 += v[6] * x0 + v[7] * x1 + v[8] * x2;
  }
  if (up_ptr) {
    for (int k = up_ptr[row] + lane; k < up_ptr[row + 1]; k += 32) {
      AT xv = (AT)xp[up_col[k]];
      const VT* b = B + (int64_t)k * 3;
      if constexpr (sizeof(VT) == 8) {
        a0 += b[0] * xv;
        a1 += b[1] * xv;
        a2 += b[2] * xv;
      } else {
        a0 += (AT)ld_val<VT>(b) * xv;
        a1 += (AT)ld_val<VT>(b + 1) * xv;
        a2 += (AT)ld_val<VT>(b + 2) * xv;
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, off);
    a1 += __shfl_xor_sync(0xffffffffu, a1, off);
    a2 += __shfl_xor_sync(0xffffffffu, a2, off);
  }
  if (lane == 0) {
    y[3 * (int64_t)row] = widen(a0);
    y[3 * (int64_t)row + 1] = widen(a1);
    y[3 * (int64_t)row + 2] = widen(a2);
  }
}

// y = K x for the displacement form, streamed: a warp takes groups of 16
// consecutive block rows, whose blocks are contiguous in memory, and walks
// each group in chunks of 32 blocks (one block per lane) regardless of where
// rows start.  The grid is one wave of resident blocks; warps stride over
// the groups, so no half-empty second wave idles the SMs.  Row sums are
// formed by a segmented inclusive scan across the lanes (segment heads = row
// starts inside the chunk, found from the group's row pointers); the last
// lane of each segment writes its row, and a row that runs past the chunk
// carries its partial sum into the next chunk.  Loads run two chunks ahead:
// while chunk i is multiplied and reduced, the x gather of chunk i + 1 and
// the column indices and values of chunk i + 2 are in flight, so each warp
// keeps HBM and L2 requests outstanding across its rows instead of one
// dependent row-pointer -> values -> x chain per row, and no lane idles on
// rows shorter than 32 blocks.  Summation order is fixed by the chunking, so
// results are deterministic.
constexpr int SPMV_RPW = 16;  // block rows per group (<= 32)

template <class VT, class AT>
__device__ __forceinline__ void spmv_load_chunk(const int* __restrict__ col, const VT* __restrict__ val, int64_t k,
                                                int64_t kend, int& c, AT (&v)[9]) {
  if (k < kend) {
    c = __ldg(col + k);
    const VT* b = val + kv_index(k, 0);
#pragma unroll
    for (int t = 0; t < 9; t++) {
      if constexpr (sizeof(VT) == 8) v[t] = __ldg(b + 32 * t);
      else v[t] = (AT)ld_val<VT>(b + 32 * t);
    }
  } else {
    c = -1;
#pragma unroll
    for (int t = 0; t < 9; t++) v[t] = AT(0);
  }
}

template <class XT, class AT>
__device__ __forceinline__ void spmv_load_x(const XT* __restrict__ x, int c, AT& x0, AT& x1, AT& x2, int ncol) {
  if (c >= 0) {
    const XT* xc = x + 3 * (int64_t)fe_idx(c, ncol);
    x0 = (AT)xc[0];
    x1 = (AT)xc[1];
    x2 = (AT)xc[2];
  } else {
    x0 = x1 = x2 = AT(0);
  }
}

template <class VT, class XT, class AT>
__global__ void __launch_bounds__(256) k_spmv_stream(int nn, const int* __restrict__ row_ptr,
                                                     const int* __restrict__ col, const VT* __restrict__ val,
                                                     const XT* __restrict__ x, double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int ngroups = (nn + SPMV_RPW - 1) / SPMV_RPW;
  const int nwarps = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
  for (int g = (int)((((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5)); g < ngroups; g += nwarps) {
    const int r0 = g * SPMV_RPW;
    const int nr = min(SPMV_RPW, nn - r0);
    const int rpl = lane < nr ? __ldg(row_ptr + r0 + lane) : INT_MAX;  // start of row r0 + lane
    const int kstart = __shfl_sync(0xffffffffu, rpl, 0);
    const int kend = __ldg(row_ptr + r0 + nr);
    // three chunks in flight: the current one (values and x in registers), the
    // next one (values in registers, x gather issued) and the one after (column
    // indices and values issued)
    int c0, c1;
    AT v0[9], v1[9];
    spmv_load_chunk<VT, AT>(col, val, (int64_t)kstart + lane, kend, c0, v0);
    spmv_load_chunk<VT, AT>(col, val, (int64_t)kstart + 32 + lane, kend, c1, v1);
    AT xa0, xa1, xa2;
    spmv_load_x<XT, AT>(x, c0, xa0, xa1, xa2, nn);
    AT carry0 = AT(0), carry1 = AT(0), carry2 = AT(0);
    int rowbase = r0 - 1;  // the row in progress before the current chunk
    for (int kc = kstart; kc < kend; kc += 32) {
      int c2;
      AT v2[9];
      spmv_load_chunk<VT, AT>(col, val, (int64_t)kc + 64 + lane, kend, c2, v2);
      AT xb0, xb1, xb2;
      spmv_load_x<XT, AT>(x, c1, xb0, xb1, xb2, nn);
      AT p0 = AT(0), p1 = AT(0), p2 = AT(0);
      if (c0 >= 0) {
        p0 = v0[0] * xa0 + v0[1] * xa1 + v0[2] * xa2;
        p1 = v0[3] * xa0 + v0[4] * xa1 + v0[5] * xa2;
        p2 = v0[6] * xa0 + v0[7] * xa1 + v0[8] * xa2;
      }
      // row starts inside the chunk, and this lane's segment start (-1: before the chunk)
      const unsigned bit = (rpl >= kc && rpl - kc < 32) ? (1u << (rpl - kc)) : 0u;
      const unsigned heads = __reduce_or_sync(0xffffffffu, bit);
      const unsigned below = heads & (0xffffffffu >> (31 - lane));
      const int sstart = below ? 31 - __clz(below) : -1;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const AT t0 = __shfl_up_sync(0xffffffffu, p0, off);
        const AT t1 = __shfl_up_sync(0xffffffffu, p1, off);
        const AT t2 = __shfl_up_sync(0xffffffffu, p2, off);
        if (lane >= off && lane - off >= sstart) {
          p0 += t0;
          p1 += t1;
          p2 += t2;
        }
      }
      const int nvalid = min(32, kend - kc);
      const bool cont = nvalid == 32 && kc + 32 < kend && !__any_sync(0xffffffffu, rpl == kc + 32);
      const bool tail = lane < nvalid && ((lane < 31 && ((heads >> (lane + 1)) & 1u)) || (lane == nvalid - 1 && !cont));
      if (tail) {
        const int row = rowbase + __popc(below);
        const bool add = sstart < 0;
        y[3 * (int64_t)row] = widen(p0 + (add ? carry0 : AT(0)));
        y[3 * (int64_t)row + 1] = widen(p1 + (add ? carry1 : AT(0)));
        y[3 * (int64_t)row + 2] = widen(p2 + (add ? carry2 : AT(0)));
      }
      const AT l0 = __shfl_sync(0xffffffffu, p0, 31), l1 = __shfl_sync(0xffffffffu, p1, 31),
               l2 = __shfl_sync(0xffffffffu, p2, 31);
      if (cont) {
        const bool whole = heads == 0u;  // lane 31's segment started before this chunk
        carry0 = l0 + (whole ? carry0 : AT(0));
        carry1 = l1 + (whole ? carry1 : AT(0));
        carry2 = l2 + (whole ? carry2 : AT(0));
      } else {
        carry0 = carry1 = carry2 = AT(0);
      }
      rowbase += __popc(heads);
      c0 = c1;
      c1 = c2;
#pragma unroll
      for (int t = 0; t < 9; t++) {
        v0[t] = v1[t];
        v1[t] = v2[t];
      }
      xa0 = xb0;
      xa1 = xb1;
      xa2 = xb2;
    }
  }
}

// pressure rows: y_p[v] = sum over (u node a, v) of B[a,v] . x_u[a]  (B2 = B1^T)
template <class VT, class XT, class AT>
__global__ void __launch_bounds__(256) k_spmv_p(int np, const int* __restrict__ pu_ptr, const int* __restrict__ pu_col,
                                                const int* __restrict__ pu_src, const VT* __restrict__ B,
                                                const XT* __restrict__ xu, double* __restrict__ yp) {
  int v = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (v >= np) return;
  AT acc = AT(0);
  for (int k = pu_ptr[v] + lane; k < pu_ptr[v + 1]; k += 32) {
    const VT* b = B + (int64_t)pu_src[k] * 3;
    const XT* u = xu + 3 * (int64_t)pu_col[k];
    if constexpr (sizeof(VT) == 8) acc += b[0] * u[0] + b[1] * u[1] + b[2] * u[2];
    else acc += (AT)ld_val<VT>(b) * (AT)u[0] + (AT)ld_val<VT>(b + 1) * (AT)u[1] + (AT)ld_val<VT>(b + 2) * (AT)u[2];
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) yp[v] = widen(acc);
}

// ---------------------------------------------------------------- preconditioner
// nodal block-Jacobi z_a = D_a^{-1} x_a (displacement part)
template <class DT, class OT>
__global__ void k_pc_bj(int nn, const DT* __restrict__ Dinv, const double* __restrict__ x, OT* __restrict__ z) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nn) return;
  const DT* D = Dinv + (int64_t)a * 9;
  double x0 = x[3 * (int64_t)a], x1 = x[3 * (int64_t)a + 1], x2 = x[3 * (int64_t)a + 2];
  if constexpr (sizeof(DT) == 8) {
    z[3 * (int64_t)a] = (OT)(D[0] * x0 + D[1] * x1 + D[2] * x2);
    z[3 * (int64_t)a + 1] = (OT)(D[3] * x0 + D[4] * x1 + D[5] * x2);
    z[3 * (int64_t)a + 2] = (OT)(D[6] * x0 + D[7] * x1 + D[8] * x2);
  } else {
    float f0 = (float)x0, f1 = (float)x1, f2 = (float)x2;
    z[3 * (int64_t)a] = (OT)(D[0] * f0 + D[1] * f1 + D[2] * f2);
    z[3 * (int64_t)a + 1] = (OT)(D[3] * f0 + D[4] * f1 + D[5] * f2);
    z[3 * (int64_t)a + 2] = (OT)(D[6] * f0 + D[7] * f1 + D[8] * f2);
  }
}

// lower Schur (SIMPLE): z_p = S^{-1} (x_p - B2 z_u), point-Jacobi S
template <class VT, class OT>
__global__ void __launch_bounds__(256) k_pc_schur(int np, int nn, const int* __restrict__ pu_ptr,
                                                  const int* __restrict__ pu_col, const int* __restrict__ pu_src,
                                                  const VT* __restrict__ B, const double* __restrict__ Sd,
                                                  const double* __restrict__ x, OT* __restrict__ z) {
  int v = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (v >= np) return;
  double acc = 0.0;
  for (int k = pu_ptr[v] + lane; k < pu_ptr[v + 1]; k += 32) {
    const VT* b = B + (int64_t)pu_src[k] * 3;
    const OT* u = z + 3 * (int64_t)pu_col[k];
    double b0, b1, b2;
    if constexpr (sizeof(VT) == 8) {
      b0 = b[0]; b1 = b[1]; b2 = b[2];
    } else {
      b0 = ld_val<VT>(b); b1 = ld_val<VT>(b + 1); b2 = ld_val<VT>(b + 2);
    }
    acc += b0 * (double)u[0] + b1 * (double)u[1] + b2 * (double)u[2];
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    double t = x[3 * (int64_t)nn + v] - acc;
    double s = Sd[v];
    z[3 * (int64_t)nn + v] = (OT)(s != 0.0 ? t / s : t);
  }
}

template <class OT>
static int pc_apply_t(fe_mesh m, const double* x, OT* z) {
  if (m->pc_type >= 1) {  // one AMG V-cycle on the displacement block
    FE_TRY(fe_amg_apply(m, x, z, sizeof(OT) == 8));
    if (!m->pres) return FE_OK;
    // u-p form: the lower Schur step z_p = S^-1 (x_p - B2 z_u) with the V-cycle's z_u
    FE_SCOPE(m, FE_PROF_PC, (double)m->nnz_up * (8 + 12.0 * (m->prec == FE_PREC_FP64 ? 8 : 4)) + 24.0 * m->np);
    const unsigned grid = (unsigned)(((int64_t)m->np * 32 + 255) / 256);
    if (m->prec == FE_PREC_FP64)
      k_pc_schur<double, OT><<<grid, 256, 0, m->stream>>>(m->np, m->nn, m->pu_ptr, m->pu_col, m->pu_src, m->B64,
                                                          m->Sd, x, z);
    else
      k_pc_schur<float, OT><<<grid, 256, 0, m->stream>>>(m->np, m->nn, m->pu_ptr, m->pu_col, m->pu_src, m->B32,
                                                         m->Sd, x, z);
    FE_CUDA(cudaGetLastError());
    return FE_OK;
  }
  FE_SCOPE(m, FE_PROF_PC, (double)m->nn * (9.0 * (m->prec == FE_PREC_FP64 ? 8 : 4) + 24 + 3.0 * sizeof(OT)) +
                              (m->pres ? (double)m->nnz_up * (8 + 12.0 * (m->prec == FE_PREC_FP64 ? 8 : 4)) + 24.0 * m->np
                                       : 0.0));
  if (m->prec == FE_PREC_FP64)
    k_pc_bj<double, OT><<<(m->nn + 255) / 256, 256, 0, m->stream>>>(m->nn, m->Dinv64, x, z);
  else
    k_pc_bj<float, OT><<<(m->nn + 255) / 256, 256, 0, m->stream>>>(m->nn, m->Dinv32, x, z);
  FE_CUDA(cudaGetLastError());
  if (m->pres) {
    unsigned grid = (unsigned)(((int64_t)m->np * 32 + 255) / 256);
    if (m->prec == FE_PREC_FP64)
      k_pc_schur<double, OT><<<grid, 256, 0, m->stream>>>(m->np, m->nn, m->pu_ptr, m->pu_col, m->pu_src, m->B64,
                                                          m->Sd, x, z);
    else
      k_pc_schur<float, OT><<<grid, 256, 0, m->stream>>>(m->np, m->nn, m->pu_ptr, m->pu_col, m->pu_src, m->B32,
                                                         m->Sd, x, z);
    FE_CUDA(cudaGetLastError());
  }
  return FE_OK;
}

int fe_pc_dev(fe_mesh m, const double* x, double* y) { return pc_apply_t<double>(m, x, y); }

// z (SpMV input type) = M^{-1} x
static int pc_to_zx(fe_mesh m, const double* x) {
  if (m->prec == FE_PREC_FP64) return pc_apply_t<double>(m, x, (double*)m->zx);
  return pc_apply_t<float>(m, x, (float*)m->zx);
}

// one wave of the streamed SpMV: resident 256-thread blocks on every SM, but
// no more warps than row groups
template <class VT, class XT, class AT>
static unsigned stream_grid_t(fe_mesh m) {
  int per_sm = 0;
  if (fe_kernel_occupancy((const void*)k_spmv_stream<VT, XT, AT>, 256, 0, &per_sm) != FE_OK) per_sm = 4;
  const int64_t groups = ((int64_t)m->nn + SPMV_RPW - 1) / SPMV_RPW;
  const int64_t need = (groups + 7) / 8;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)std::max(per_sm, 1) * m->sm_count));
}
static unsigned spmv_stream_grid(fe_mesh m) {
  if (m->prec == FE_PREC_FP64) return stream_grid_t<double, double, double>(m);
  if (m->prec == FE_PREC_MIXED_BF16) return stream_grid_t<__nv_bfloat16, float, float>(m);
  return stream_grid_t<float, float, float>(m);
}

// y = K xin with xin in the SpMV input type (FP64 for an FP64 tangent, FP32
// otherwise).  The displacement form streams its blocks (k_spmv_stream);
// the u-p form adds the coupling B1 x_p per row (k_spmv) and the pressure
// rows (k_spmv_p); the u-p coupling is kept in the tangent's precision.
static int launch_spmv(fe_mesh m, const void* xin, double* y) {
  const unsigned grid = (unsigned)(((int64_t)m->nn * 32 + 255) / 256);
  const unsigned gridp = (unsigned)(((int64_t)m->np * 32 + 255) / 256);
  const unsigned grids = spmv_stream_grid(m);
  if (m->prec == FE_PREC_FP64) {
    const double* x = (const double*)xin;
    if (!m->pres) {
      k_spmv_stream<double, double, double><<<grids, 256, 0, m->stream>>>(m->nn, m->row_ptr, m->col, m->K64, x, y);
    } else {
      k_spmv<double, double, double><<<grid, 256, 0, m->stream>>>(m->nn, m->row_ptr, m->col, m->K64, x, y, m->up_ptr,
                                                                  m->up_col, m->B64, x + 3 * (int64_t)m->nn);
      k_spmv_p<double, double, double><<<gridp, 256, 0, m->stream>>>(m->np, m->pu_ptr, m->pu_col, m->pu_src, m->B64,
                                                                     x, y + 3 * (int64_t)m->nn);
    }
  } else if (m->prec == FE_PREC_MIXED_BF16) {
    const float* x = (const float*)xin;
    k_spmv_stream<__nv_bfloat16, float, float><<<grids, 256, 0, m->stream>>>(m->nn, m->row_ptr, m->col, m->K16, x, y);
  } else {
    const float* x = (const float*)xin;
    if (!m->pres) {
      k_spmv_stream<float, float, float><<<grids, 256, 0, m->stream>>>(m->nn, m->row_ptr, m->col, m->K32, x, y);
    } else {
      k_spmv<float, float, float><<<grid, 256, 0, m->stream>>>(m->nn, m->row_ptr, m->col, m->K32, x, y, m->up_ptr,
                                                               m->up_col, m->B32, x + 3 * (int64_t)m->nn);
      k_spmv_p<float, float, float><<<gridp, 256, 0, m->stream>>>(m->np, m->pu_ptr, m->pu_col, m->pu_src, m->B32, x,
                                                                  y + 3 * (int64_t)m->nn);
    }
  }
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// y = K zx (zx already in the SpMV input type)
static int spmv_zx(fe_mesh m, double* y) {
  const double sv = m->prec == FE_PREC_FP64 ? 8 : (m->prec == FE_PREC_MIXED_BF16 ? 2 : 4);
  const double sx = m->prec == FE_PREC_FP64 ? 8 : 4;
  FE_SCOPE_F(m, FE_PROF_SPMV, (double)m->nnzb * (9 * sv + 4) + 4.0 * (m->nn + 1) + sx * (double)m->ndof + 8.0 * (double)m->ndof +
                                  (m->pres ? (double)m->nnz_up * 2 * (3 * sv + 8) + 4.0 * (m->nn + m->np + 2) : 0.0),
             18.0 * (double)m->nnzb + (m->pres ? 12.0 * (double)m->nnz_up : 0.0));
  return launch_spmv(m, m->zx, y);
}

__global__ void k_narrow(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}
__global__ void k_copy(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i];
}

static int ensure_zx(fe_mesh m) {
  if (!m->zx) FE_TRY(fe_alloc(m, &m->zx, (size_t)m->ndof * sizeof(double)));
  return FE_OK;
}

// y = K x for FP64 x, y
int fe_spmv_dev(fe_mesh m, const double* x, double* y) {
  if (m->prec < 0) return fe_set_error("no tangent assembled"), FE_ERR_STATE;
  FE_TRY(ensure_zx(m));
  unsigned g = (unsigned)((m->ndof + 255) / 256);
  FE_SCOPE(m, FE_PROF_VECTOR, (m->prec == FE_PREC_FP64 ? 16.0 : 12.0) * m->ndof);
  if (m->prec == FE_PREC_FP64) k_copy<<<g, 256, 0, m->stream>>>(m->ndof, x, (double*)m->zx);
  else k_narrow<<<g, 256, 0, m->stream>>>(m->ndof, x, (float*)m->zx);
  FE_CUDA(cudaGetLastError());
  return spmv_zx(m, y);
}

// y = K x with FP64 input and FP64 accumulation whatever the storage of the
// tangent values (FP32 and BF16 values widen exactly to FP64).  The
// residuals that decide the stopping tests of the mixed forms -- GMRES's
// restart residual b - K x and iNK's linear residual R + K delta -- then
// carry no rounding beyond the stored tangent's, so restarted GMRES refines
// its iterate in FP64 (mixed-precision iterative refinement) instead of
// stalling at the FP32 SpMV's accuracy.  The FP64 form is fe_spmv_dev.
template <class VT>
static int spmv_acc_t(fe_mesh m, const VT* K, const VT* B, const double* x, double* y) {
  const double sv = sizeof(VT);
  FE_SCOPE_F(m, FE_PROF_SPMV, (double)m->nnzb * (9 * sv + 4) + 4.0 * (m->nn + 1) + 16.0 * (double)m->ndof +
                                  (m->pres ? (double)m->nnz_up * 2 * (3 * sv + 8) + 4.0 * (m->nn + m->np + 2) : 0.0),
             18.0 * (double)m->nnzb + (m->pres ? 12.0 * (double)m->nnz_up : 0.0));
  if (!m->pres) {
    const unsigned grids = stream_grid_t<VT, double, double>(m);
    k_spmv_stream<VT, double, double><<<grids, 256, 0, m->stream>>>(m->nn, m->row_ptr, m->col, K, x, y);
  } else {
    const unsigned grid = (unsigned)(((int64_t)m->nn * 32 + 255) / 256);
    const unsigned gridp = (unsigned)(((int64_t)m->np * 32 + 255) / 256);
    k_spmv<VT, double, double><<<grid, 256, 0, m->stream>>>(m->nn, m->row_ptr, m->col, K, x, y, m->up_ptr, m->up_col,
                                                            B, x + 3 * (int64_t)m->nn);
    k_spmv_p<VT, double, double><<<gridp, 256, 0, m->stream>>>(m->np, m->pu_ptr, m->pu_col, m->pu_src, B, x,
                                                               y + 3 * (int64_t)m->nn);
  }
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

int fe_spmv_acc_dev(fe_mesh m, const double* x, double* y) {
  if (m->prec < 0) return fe_set_error("no tangent assembled"), FE_ERR_STATE;
  if (m->prec == FE_PREC_FP64) return fe_spmv_dev(m, x, y);
  if (m->prec == FE_PREC_MIXED_BF16) return spmv_acc_t<__nv_bfloat16>(m, m->K16, nullptr, x, y);
  return spmv_acc_t<float>(m, m->K32, m->B32, x, y);
}

// y = K xin where xin already holds the input in the SpMV's input precision
// (FP64 for an FP64 tangent, FP32 otherwise).  Used by the allocation-free
// entry point, which stages the input in its own fixed device array.
int fe_spmv_from_input(fe_mesh m, const void* xin, double* y) { return launch_spmv(m, xin, y); }

// Under CUDA's lazy loading a kernel's code is placed in device memory at
// its first launch.  Loading every SpMV kernel here (and caching the
// occupancy the streamed launch reads) lets a caller that must not allocate
// launch them later without that first-use cost.
int fe_spmv_preload(fe_mesh m) {
  const void* fns[] = {(const void*)k_spmv_stream<double, double, double>,
                       (const void*)k_spmv_stream<float, float, float>,
                       (const void*)k_spmv_stream<__nv_bfloat16, float, float>,
                       (const void*)k_spmv<double, double, double>,
                       (const void*)k_spmv<float, float, float>,
                       (const void*)k_spmv_p<double, double, double>,
                       (const void*)k_spmv_p<float, float, float>};
  for (const void* fn : fns) {
    cudaFuncAttributes a;
    FE_CUDA(cudaFuncGetAttributes(&a, fn));
  }
  int per_sm = 0;
  FE_TRY(fe_kernel_occupancy((const void*)k_spmv_stream<double, double, double>, 256, 0, &per_sm));
  FE_TRY(fe_kernel_occupancy((const void*)k_spmv_stream<float, float, float>, 256, 0, &per_sm));
  FE_TRY(fe_kernel_occupancy((const void*)k_spmv_stream<__nv_bfloat16, float, float>, 256, 0, &per_sm));
  (void)m;
  return FE_OK;
}

// ---------------------------------------------------------------- vectors
__global__ void k_dot(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* red,
                      unsigned* ticket, double* out) {
  __shared__ double sh[32];
  __shared__ bool last;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  s = block_sum_all(s, sh);
  if (threadIdx.x == 0) {
    red[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = sum_partials(red, sh);
  if (threadIdx.x == 0) {
    *out = t;
    *ticket = 0u;
  }
}

static unsigned dot_grid(fe_mesh m) { return (unsigned)(m->sm_count * 4); }

// dot product into device scalar slot `slot` (no host sync)
static int dot_async(fe_mesh m, const double* a, const double* b, int64_t n, int slot) {
  FE_SCOPE(m, FE_PROF_VECTOR, (a == b ? 8.0 : 16.0) * n);
  k_dot<<<dot_grid(m), 256, 0, m->stream>>>(n, a, b, m->red, m->red_ticket, m->scal + slot);
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

int fe_dot_dev(fe_mesh m, const double* a, const double* b, int64_t n, double* out_host) {
  FE_TRY(dot_async(m, a, b, n, 5));
  FE_CUDA(cudaMemcpyAsync(m->h_scal + 5, m->scal + 5, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  *out_host = m->h_scal[5];
  return FE_OK;
}

// y = a x + b y
// y = a x + b y; b == 0 overwrites y (the BLAS convention), so a NaN left in
// y by an earlier solve cannot leak into y through 0 * NaN
__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = b == 0.0 ? a * x[i] : a * x[i] + b * y[i];
}
int fe_axpby_dev(fe_mesh m, double a, const double* x, double b, double* y, int64_t n) {
  FE_SCOPE(m, FE_PROF_VECTOR, 24.0 * n);
  k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(n, a, x, b, y);
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// v = (b - w) / beta? -> r = b - w
__global__ void k_sub(int64_t n, const double* __restrict__ b, const double* __restrict__ w, double* __restrict__ r) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = b[i] - w[i];
}
__global__ void k_scale(int64_t n, const double* __restrict__ s, double* __restrict__ v, double* __restrict__ g,
                        int glen) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double beta = sqrt(s[0]);
  if (i < n) v[i] = v[i] / beta;
  if (i < glen) g[i] = (i == 0) ? beta : 0.0;
}

// back substitution y = H^{-1} g on the k x k upper triangle (one block)
// back substitution R y = g (R upper triangular, column j at H + j ldh), one
// block of 1024 threads, thread r owns row r (k <= 1000): g and the diagonal
// sit in shared memory and each thread loads its entry of the next column
// while the current one is applied, so a column costs one block barrier
// instead of a global-memory round trip
__global__ void __launch_bounds__(1024) k_trisolve(int k, int ldh, const double* __restrict__ H,
                                                   const double* __restrict__ g, double* __restrict__ y) {
  __shared__ double gs[1024], dg[1024];
  const int r = threadIdx.x;
  if (r < k) {
    gs[r] = g[r];
    dg[r] = H[(int64_t)r * ldh + r];
  }
  double h = (r < k - 1) ? H[(int64_t)(k - 1) * ldh + r] : 0.0;
  __syncthreads();
  for (int i = k - 1; i >= 0; i--) {
    const double yi = gs[i] / dg[i];
    const double hn = (i >= 1 && r < i - 1) ? H[(int64_t)(i - 1) * ldh + r] : 0.0;
    if (r < i) gs[r] -= h * yi;
    if (r == 0) y[i] = yi;
    h = hn;
    __syncthreads();
  }
}

// u = sum_i y_i V_i
__global__ void k_gemv(int64_t n, int k, const double* __restrict__ V, int64_t ldv, const double* __restrict__ y,
                       double* __restrict__ u) {
  __shared__ double ys[1024];
  for (int i = threadIdx.x; i < k && i < 1024; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  double s = 0.0;
#pragma unroll 8
  for (int i = 0; i < k; i++) s += ys[i] * V[(int64_t)i * ldv + idx];
  u[idx] = s;
}

// ---------------------------------------------------------------- workspace
constexpr int LOWSYNC_MAX_RESTART = 128;  // shared memory holds 32 partials per inner product
int fe_workspace(fe_mesh m, int restart) {
  FE_TRY(ensure_zx(m));
  if (!m->w64) FE_TRY(fe_alloc_t(m, &m->w64, (size_t)m->ndof));
  if (!m->t64) FE_TRY(fe_alloc_t(m, &m->t64, (size_t)m->ndof));
  if (!m->u64) FE_TRY(fe_alloc_t(m, &m->u64, (size_t)m->ndof));
  if (restart > m->ws_restart) {
    // basis rows padded to a multiple of 32 values (256 bytes) and zeroed, so
    // the Arnoldi kernel's 16-byte pair loads stay inside a row
    const int64_t ldv = (m->ndof + 31) / 32 * 32;
    if (m->V) {
      cudaFreeAsync(m->V, m->stream);
      cudaFreeAsync(m->H, m->stream);
      cudaFreeAsync(m->gv, m->stream);
      m->device_bytes -= (int64_t)(m->ws_restart + 1) * m->ldv * 8 + (int64_t)(m->ws_restart + 1) * (m->ws_restart + 1) * 8 +
                         (int64_t)4 * (m->ws_restart + 2) * 8;
      m->V = m->H = m->gv = nullptr;
      cudaFreeAsync(m->Tbm, m->stream);
      m->device_bytes -= (int64_t)(m->ws_restart + 2) * BMGS_P * 8;
      m->Tbm = nullptr;
    }
    FE_TRY(fe_alloc_t(m, &m->V, (size_t)(restart + 1) * ldv));
    FE_CUDA(cudaMemsetAsync(m->V, 0, (size_t)(restart + 1) * ldv * sizeof(double), m->stream));
    FE_TRY(fe_alloc_t(m, &m->H, (size_t)(restart + 1) * (restart + 1)));
    FE_TRY(fe_alloc_t(m, &m->gv, (size_t)4 * (restart + 2)));
    m->ws_restart = restart;
    m->ldv = ldv;
    FE_TRY(fe_alloc_t(m, &m->Tbm, (size_t)(restart + 2) * BMGS_P));
    if (restart <= LOWSYNC_MAX_RESTART) {  // low-synchronisation MGS: L, h, per-block inner products
      if (m->Lmat) {
        cudaFreeAsync(m->Lmat, m->stream);
        cudaFreeAsync(m->hpub, m->stream);
        cudaFreeAsync(m->partv, m->stream);
      }
      m->partv_blocks = 2 * m->sm_count;
      FE_TRY(fe_alloc_t(m, &m->Lmat, (size_t)(restart + 1) * (restart + 1)));
      FE_TRY(fe_alloc_t(m, &m->hpub, (size_t)(restart + 1)));
      FE_TRY(fe_alloc_t(m, &m->partv, (size_t)m->partv_blocks * (2 * restart + 1)));
    }
  }
  return FE_OK;
}

// ---------------------------------------------------------------- persistent launch helpers
struct CoopCfg {
  int npt, grid;
};

static GridSync grid_sync(fe_mesh m) {
  GridSync gs;
  gs.count = m->bar;
  gs.seq = m->bar + 1;
  gs.slot = (unsigned long long*)(m->bar + 2);
  gs.err = m->err;
  gs.limit = m->wait_limit;
  return gs;
}

template <int NPT, class DT, class ZT>
static const void* arnoldi_fn() { return (const void*)k_arnoldi<NPT, DT, ZT>; }

// Picks the smallest slice width (NPT values per thread, a multiple of 3)
// whose grid of ceil(n / S) blocks can be co-resident, then launches the
// step cooperatively.  fuse_pc: also write z = D^{-1} V_{j+1} into zx.
template <class DT, class ZT>
static int launch_arnoldi_t(fe_mesh m, int j, int kmax, bool fuse_pc, const DT* Dinv, double target, int it0,
                            int max_it) {
  const int64_t n = m->ndof;
  const void* fns[3] = {arnoldi_fn<24, DT, ZT>(), arnoldi_fn<12, DT, ZT>(), arnoldi_fn<6, DT, ZT>()};
  const int npts[3] = {24, 12, 6};
  const int bds[3] = {256, 512, 1024};
  int which = -1, grid = 0;
  for (int q = 0; q < 3; q++) {
    size_t smem = (size_t)npts[q] * bds[q] * sizeof(double);
    FE_TRY(fe_kernel_smem(fns[q], (int)smem));
    int per_sm = 0;
    FE_TRY(fe_kernel_occupancy(fns[q], bds[q], smem, &per_sm));
    int64_t need = (n + (int64_t)npts[q] * bds[q] - 1) / ((int64_t)npts[q] * bds[q]);
    if (per_sm >= 1 && need <= (int64_t)per_sm * m->sm_count && need <= RED_SLOTS) {
      which = q;
      grid = (int)need;
      break;
    }
  }
  if (which < 0) return fe_set_error("vector too long for the persistent Arnoldi kernel (n = %lld)", (long long)n), FE_ERR_ARG;
  size_t smem = (size_t)npts[which] * bds[which] * sizeof(double);
  double* V = m->V;
  int64_t ldv = m->ldv;
  double* Hcol = m->H + (int64_t)j * (kmax + 1);
  double* cs = m->gv;
  double* sn = m->gv + (kmax + 2);
  double* g = m->gv + 2 * (kmax + 2);
  double* out = m->scal + 3;
  double* part = m->red;
  const DT* D = fuse_pc ? Dinv : nullptr;
  ZT* z = fuse_pc ? (ZT*)m->zx : nullptr;
  GridSync gs = grid_sync(m);
  void* args[] = {(void*)&n, (void*)&j, (void*)&V, (void*)&ldv, (void*)&m->w64, (void*)&Hcol, (void*)&part,
                  (void*)&gs, (void*)&cs, (void*)&sn, (void*)&g, (void*)&out,
                  (void*)&D, (void*)&z, (void*)&target, (void*)&kmax, (void*)&it0, (void*)&max_it};
  // flops: (j+1) inner products and axpys (4 per entry), the norm (2) and the scaling (1)
  // per entry, plus 18 per node for the fused block-Jacobi product
  FE_SCOPE_F(m, FE_PROF_ARNOLDI, 8.0 * (double)n * (j + 3) + (fuse_pc ? (double)n * (3.0 * sizeof(DT) + sizeof(ZT)) : 0.0),
             (double)n * (4.0 * (j + 1) + 3.0) + (fuse_pc ? 6.0 * n : 0.0));
  FE_CUDA(cudaLaunchCooperativeKernel(fns[which], dim3(grid), dim3(bds[which]), args, smem, m->stream));
  return FE_OK;
}

template <int NPT, class DT, class ZT>
static const void* arnoldi_ls_fn() { return (const void*)k_arnoldi_ls<NPT, DT, ZT>; }

template <class DT, class ZT>
static int launch_arnoldi_ls_t(fe_mesh m, int j, int kmax, bool fuse_pc, const DT* Dinv, double target, int it0,
                               int max_it) {
  const int64_t n = m->ndof;
  const void* fns[3] = {arnoldi_ls_fn<24, DT, ZT>(), arnoldi_ls_fn<12, DT, ZT>(), arnoldi_ls_fn<6, DT, ZT>()};
  const int npts[3] = {24, 12, 6};
  const int bds[3] = {256, 512, 1024};
  const size_t pw_max = (size_t)(2 * LOWSYNC_MAX_RESTART + 1) * 32 * sizeof(double);
  int which = -1, grid = 0;
  for (int q = 0; q < 3; q++) {
    size_t smem = 2 * (size_t)npts[q] * bds[q] * sizeof(double) + pw_max;
    FE_TRY(fe_kernel_smem(fns[q], (int)smem));
    int per_sm = 0;
    FE_TRY(fe_kernel_occupancy(fns[q], bds[q], smem, &per_sm));
    int64_t need = (n + (int64_t)npts[q] * bds[q] - 1) / ((int64_t)npts[q] * bds[q]);
    if (per_sm >= 1 && need <= (int64_t)per_sm * m->sm_count && need <= m->partv_blocks) {
      which = q;
      grid = (int)need;
      break;
    }
  }
  if (which < 0) return fe_set_error("vector too long for the low-synchronisation Arnoldi kernel"), FE_ERR_ARG;
  const int nv = 2 * j + 1;
  size_t smem = 2 * (size_t)npts[which] * bds[which] * sizeof(double) + (size_t)nv * 32 * sizeof(double);
  double* V = m->V;
  int64_t ldv = m->ldv;
  double* Hcol = m->H + (int64_t)j * (kmax + 1);
  double* cs = m->gv;
  double* sn = m->gv + (kmax + 2);
  double* g = m->gv + 2 * (kmax + 2);
  double* out = m->scal + 3;
  double* part = m->red;
  double* partv = m->partv;
  double* Lmat = m->Lmat;
  int ldl = kmax + 1;
  double* hpub = m->hpub;
  const DT* D = fuse_pc ? Dinv : nullptr;
  ZT* z = fuse_pc ? (ZT*)m->zx : nullptr;
  GridSync gs = grid_sync(m);
  void* args[] = {(void*)&n, (void*)&j, (void*)&V, (void*)&ldv, (void*)&m->w64, (void*)&Hcol, (void*)&part,
                  (void*)&partv, (void*)&gs, (void*)&Lmat, (void*)&ldl, (void*)&hpub, (void*)&cs, (void*)&sn,
                  (void*)&g, (void*)&out, (void*)&D, (void*)&z, (void*)&target, (void*)&kmax, (void*)&it0,
                  (void*)&max_it};
  // flops: 2 inner products per basis vector, then the update, the norm and the scaling
  FE_SCOPE_F(m, FE_PROF_ARNOLDI,
             8.0 * (double)n * (2.0 * (j + 1) + 3) + (fuse_pc ? (double)n * (3.0 * sizeof(DT) + sizeof(ZT)) : 0.0),
             (double)n * (6.0 * (j + 1) + 3.0) + (fuse_pc ? 6.0 * n : 0.0));
  FE_CUDA(cudaLaunchCooperativeKernel(fns[which], dim3(grid), dim3(bds[which]), args, smem, m->stream));
  return FE_OK;
}

template <int NPT, class DT, class ZT>
static const void* arnoldi_bm_fn() { return (const void*)k_arnoldi_bm<NPT, BMGS_P, DT, ZT>; }
template <int NPT, class DT, class ZT>
static const void* arnoldi_bm_ws_fn() { return (const void*)k_arnoldi_bm_ws<NPT, BMGS_P, DT, ZT>; }

static BlockSync block_sync(fe_mesh m) {
  BlockSync bs;
  bs.count = m->bar;
  bs.seq = m->bar + 6;
  bs.pub = (unsigned long long*)(m->bar + 8);
  bs.err = m->err;
  bs.limit = m->wait_limit;
  return bs;
}

// Slice selection as in launch_arnoldi_t: first the register-resident
// kernels (w, the current and the next basis slice in registers), then, for
// longer vectors, the shared-memory slices of k_arnoldi_bm_ws (48 or 72
// values per thread); returns 1 without launching when no co-resident grid
// exists, and the caller takes the sequential sweep.
template <class DT, class ZT>
static int launch_arnoldi_bm_t(fe_mesh m, int j, int kmax, bool fuse_pc, const DT* Dinv, double target, int it0,
                               int max_it) {
  const int64_t n = m->ndof;
  // 512 threads of 12 values first: four warps per SM sub-partition keep
  // the FP64 pipe busier than two
  const void* fns[4] = {arnoldi_bm_fn<12, DT, ZT>(), arnoldi_bm_fn<24, DT, ZT>(), arnoldi_bm_ws_fn<48, DT, ZT>(),
                        arnoldi_bm_ws_fn<72, DT, ZT>()};
  const int npts[4] = {12, 24, 48, 72};
  const int bds[4] = {512, 256, 256, 256};
  int which = -1, grid = 0;
  for (int q = 0; q < 4; q++) {
    size_t smem = (size_t)npts[q] * bds[q] * sizeof(double);
    FE_TRY(fe_kernel_smem(fns[q], (int)smem));
    int per_sm = 0;
    FE_TRY(fe_kernel_occupancy(fns[q], bds[q], smem, &per_sm));
    int64_t need = (n + (int64_t)npts[q] * bds[q] - 1) / ((int64_t)npts[q] * bds[q]);
    if (per_sm >= 1 && need <= (int64_t)per_sm * m->sm_count && need * BMGS_P <= RED_SLOTS) {
      which = q;
      grid = (int)need;
      break;
    }
  }
  if (which < 0) return 1;
  size_t smem = (size_t)npts[which] * bds[which] * sizeof(double);
  double* V = m->V;
  int64_t ldv = m->ldv;
  double* Hcol = m->H + (int64_t)j * (kmax + 1);
  double* cs = m->gv;
  double* sn = m->gv + (kmax + 2);
  double* g = m->gv + 2 * (kmax + 2);
  double* out = m->scal + 3;
  double* part = m->red;
  double* T = m->Tbm;
  const DT* D = fuse_pc ? Dinv : nullptr;
  ZT* z = fuse_pc ? (ZT*)m->zx : nullptr;
  BlockSync bs = block_sync(m);
  void* args[] = {(void*)&n, (void*)&j, (void*)&V, (void*)&ldv, (void*)&m->w64, (void*)&Hcol, (void*)&part,
                  (void*)&bs, (void*)&T, (void*)&cs, (void*)&sn, (void*)&g, (void*)&out,
                  (void*)&D, (void*)&z, (void*)&target, (void*)&kmax, (void*)&it0, (void*)&max_it};
  const int ng = (j + 1) % BMGS_P;
  // same algorithmic bytes as the sequential sweep; flops add the Gram row
  FE_SCOPE_F(m, FE_PROF_ARNOLDI, 8.0 * (double)n * (j + 3) + (fuse_pc ? (double)n * (3.0 * sizeof(DT) + sizeof(ZT)) : 0.0),
             (double)n * (4.0 * (j + 1) + 3.0 + 2.0 * ng) + (fuse_pc ? 6.0 * n : 0.0));
  FE_CUDA(cudaLaunchCooperativeKernel(fns[which], dim3(grid), dim3(bds[which]), args, smem, m->stream));
  return FE_OK;
}

static int launch_arnoldi(fe_mesh m, int j, int kmax, bool fuse_pc, double target, int it0, int max_it) {
  if (m->orthog == 2) {
    int r = m->prec == FE_PREC_FP64
                ? launch_arnoldi_bm_t<double, double>(m, j, kmax, fuse_pc, m->Dinv64, target, it0, max_it)
                : launch_arnoldi_bm_t<float, float>(m, j, kmax, fuse_pc, m->Dinv32, target, it0, max_it);
    if (r <= 0) return r;
  }
  if (m->orthog == 1) {
    if (m->prec == FE_PREC_FP64)
      return launch_arnoldi_ls_t<double, double>(m, j, kmax, fuse_pc, m->Dinv64, target, it0, max_it);
    return launch_arnoldi_ls_t<float, float>(m, j, kmax, fuse_pc, m->Dinv32, target, it0, max_it);
  }
  if (m->prec == FE_PREC_FP64)
    return launch_arnoldi_t<double, double>(m, j, kmax, fuse_pc, m->Dinv64, target, it0, max_it);
  return launch_arnoldi_t<float, float>(m, j, kmax, fuse_pc, m->Dinv32, target, it0, max_it);
}

// ---------------------------------------------------------------- GMRES
// Right-preconditioned GMRES(restart) with MGS Arnoldi and Givens rotations.
// Stops when the residual estimate |g_{j+1}| <= max(rtol ||b||, atol), on a
// lucky breakdown, or after max_it iterations; the iterate is updated at the
// end of every cycle with x += M^{-1} V_j y.
constexpr int GMRES_BATCH = 8;

// Steps of the next GMRES batch after j steps of a cycle that started at
// residual beta and now estimates resid: the steps to the target at the
// cycle's mean rate of decrease so far (at least 1, at most GMRES_BATCH;
// GMRES_BATCH when there is no decrease yet to go by).
static int gmres_next_batch(double beta, double resid, double target, int j) {
  if (j < 1 || !(resid > target) || !(resid < beta) || !(target > 0.0)) return GMRES_BATCH;
  const double per_step = std::log(resid / beta) / j;  // < 0
  const double left = std::log(target / resid) / per_step;
  if (!std::isfinite(left)) return GMRES_BATCH;
  return (int)std::min<double>(GMRES_BATCH, std::max(1.0, std::ceil(left)));
}

int fe_gmres_dev(fe_mesh m, const double* b, double* x, double rtol, double atol, int restart, int max_it,
                 int* iters, double* res) {
  if (m->prec < 0) return fe_set_error("no tangent assembled"), FE_ERR_STATE;
  if (restart < 1 || restart > 1000) return fe_set_error("restart must be in [1, 1000]"), FE_ERR_ARG;
  if (m->orthog == 1 && restart > LOWSYNC_MAX_RESTART)
    return fe_set_error("low-synchronisation MGS supports restart <= %d", LOWSYNC_MAX_RESTART), FE_ERR_ARG;
  FE_TRY(fe_workspace(m, restart));
  const int64_t n = m->ndof;
  const unsigned g1 = (unsigned)((n + 255) / 256);
  double bnorm2;
  FE_TRY(fe_dot_dev(m, b, b, n, &bnorm2));
  double bnorm = sqrt(bnorm2);
  double target = fmax(rtol * bnorm, atol);
  int it = 0;
  double resid = 0.0;
  const int kmax = restart;
  double* g = m->gv + 2 * (kmax + 2);  // Givens arrays: cs, sn, g, y
  double* y = m->gv + 3 * (kmax + 2);
  // Mixed forms: the FP32 SpMV resolves residuals to ~1e-6 of |b|; a target
  // below 1e-4 |b| needs the residual with FP64 vectors and accumulation at
  // every restart and the refinement check at the end, a looser one (iB's
  // 1e-2) does not
  const bool refine = m->prec != FE_PREC_FP64 && target < 1e-4 * bnorm;
  for (;;) {
    // r = b - K x -> V_0, beta = ||r||
    if (refine) FE_TRY(fe_spmv_acc_dev(m, x, m->w64));
    else FE_TRY(fe_spmv_dev(m, x, m->w64));
    {
      FE_SCOPE(m, FE_PROF_VECTOR, 24.0 * n);
      k_sub<<<g1, 256, 0, m->stream>>>(n, b, m->w64, m->V);
    }
    FE_TRY(dot_async(m, m->V, m->V, n, 6));
    FE_CUDA(cudaMemcpyAsync(m->h_scal + 6, m->scal + 6, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    FE_CUDA(cudaStreamSynchronize(m->stream));
    double beta = sqrt(m->h_scal[6]);
    resid = beta;
    if (beta <= target || it >= max_it || !std::isfinite(beta)) break;
    unsigned gs = std::max<unsigned>(g1, (unsigned)((kmax + 1 + 255) / 256));
    {
      FE_SCOPE(m, FE_PROF_VECTOR, 16.0 * n);
      k_scale<<<gs, 256, 0, m->stream>>>(n, m->scal + 6, m->V, g, kmax + 1);
    }
    FE_CUDA(cudaGetLastError());
    // the block-Jacobi application is fused into the Arnoldi step (it writes
    // z = D^{-1} V_{j+1} for the next SpMV); the u-p Schur preconditioner
    // (it needs B2 z_u) and the AMG V-cycle run as their own kernels.  Steps are queued in batches
    // of up to GMRES_BATCH; the step that meets the stopping test raises a
    // device flag that turns the rest of its batch's Arnoldi steps into
    // no-ops, so the host reads the scalars once per batch.  The SpMV and the
    // preconditioner of a step queued past the end still run, so after the
    // first step a batch holds the steps that the estimate's decrease so far
    // predicts are left to the target: a batch that falls short costs one
    // more host synchronisation, one that overshoots a V-cycle and an SpMV
    // per extra step.
    const bool fuse = !m->pres && m->pc_type == 0;
    FE_CUDA(cudaMemsetAsync(m->scal + 10, 0, 2 * sizeof(double), m->stream));  // out[7], out[8]
    int batch = 1;
    bool done = false;
    int j = 0;
    while (!done) {
      const int jprev = j;
      int jend = std::min(j + batch, kmax);
      for (int jj = j; jj < jend; jj++) {
        if (jj == 0 || !fuse) FE_TRY(pc_to_zx(m, m->V + (int64_t)jj * m->ldv));
        FE_TRY(spmv_zx(m, m->w64));
        FE_TRY(launch_arnoldi(m, jj, kmax, fuse, target, it, max_it));
      }
      FE_CUDA(cudaMemcpyAsync(m->h_scal + 3, m->scal + 3, (SCAL_N - 3) * sizeof(double), cudaMemcpyDeviceToHost,
                              m->stream));
      FE_CUDA(cudaStreamSynchronize(m->stream));
      if (*(const int*)(m->h_scal + SCAL_N - 1) != DEV_OK) FE_TRY(fe_check_device_error(m));
      done = m->h_scal[10] != 0.0;
      j = (int)m->h_scal[11];
      resid = m->h_scal[3];
      // the batch's Arnoldi launches past the cycle's end did no work: their
      // algorithmic bytes and flops leave the profile (their time stays)
      if (m->prof_timing && !m->prof_suspend) {
        int drop = jend - std::max(j, jprev);
        for (auto r = m->prof_pending.rbegin(); r != m->prof_pending.rend() && drop > 0; ++r)
          if (r->cls == FE_PROF_ARNOLDI) {
            r->bytes = r->flops = 0.0;
            drop--;
          }
      }
      if (!std::isfinite(resid)) done = true;
      if (!done && j <= jprev) return fe_set_error("GMRES made no progress in a batch"), FE_ERR_STATE;
      batch = gmres_next_batch(beta, resid, target, j);
    }
    it += j;
    // FP64 (and loose mixed targets): the residual estimate decides, as in
    // the oracle.  Mixed forms with a tight target: an estimate at the target
    // sends the iterate back to the top of the loop, where its
    // FP64-accumulated residual decides (and, above the target, starts the
    // next refinement cycle)
    done = it >= max_it || m->h_scal[4] == 0.0 || !std::isfinite(resid) || (resid <= target && !refine);
    {
      FE_SCOPE(m, FE_PROF_VECTOR, 8.0 * j * (j + 1));
      k_trisolve<<<1, 1024, 0, m->stream>>>(j, kmax + 1, m->H, g, y);
    }
    {
      FE_SCOPE(m, FE_PROF_VECTOR, 8.0 * n * (j + 1));
      k_gemv<<<g1, 256, 0, m->stream>>>(n, j, m->V, m->ldv, y, m->u64);
    }
    FE_TRY(fe_pc_dev(m, m->u64, m->t64));
    FE_TRY(fe_axpby_dev(m, 1.0, m->t64, 1.0, x, n));
    FE_CUDA(cudaGetLastError());
    if (done) break;
  }
  FE_CUDA(cudaStreamSynchronize(m->stream));
  if (iters) *iters = it;
  if (res) *res = resid;
  return FE_OK;
}

// ---------------------------------------------------------------- L-BFGS two-loop
// loop 1 (newest -> oldest): alpha_i = rho_i s_i . q ; q -= alpha_i y_i
template <int NPT>
__global__ void __launch_bounds__(256) k_twoloop1(int64_t n, int k, int head, int mcap, const double* __restrict__ S,
                                                  const double* __restrict__ Y, int64_t ld,
                                                  const double* __restrict__ rho, const double* __restrict__ qin,
                                                  double* __restrict__ qout, double* __restrict__ alpha, double* part,
                                                  GridSync gs) {
  __shared__ double sh[32];
  __shared__ int s_fail;
  __shared__ double s_val;
  unsigned seq = *(volatile unsigned*)gs.seq;
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double q[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    int64_t idx = tid + s * T;
    q[s] = idx < n ? qin[idx] : 0.0;
  }
  for (int c = k - 1; c >= 0; c--) {
    int slot = (head + c) % mcap;
    const double* si = S + (int64_t)slot * ld;
    const double* yi = Y + (int64_t)slot * ld;
    double loc = 0.0;
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      int64_t idx = tid + s * T;
      if (idx < n) loc += si[idx] * q[s];
    }
    double bs = block_sum0(loc, sh);
    int last = threadIdx.x == 0 ? grid_arrive(gs, part, bs) : 0;
    double yv[NPT];  // streams in while the reduction completes
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      int64_t idx = tid + s * T;
      yv[s] = idx < n ? yi[idx] : 0.0;
    }
    double tot;
    if (!grid_complete(gs, part, seq++, last, &s_val, &s_fail, tot)) return;
    double a = rho[slot] * tot;
    if (blockIdx.x == 0 && threadIdx.x == 0) alpha[c] = a;
#pragma unroll
    for (int s = 0; s < NPT; s++) q[s] -= a * yv[s];
  }
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    int64_t idx = tid + s * T;
    if (idx < n) qout[idx] = q[s];
  }
}

// loop 2 (oldest -> newest): beta = rho_i y_i . z ; z += (alpha_i - beta) s_i
template <int NPT>
__global__ void __launch_bounds__(256) k_twoloop2(int64_t n, int k, int head, int mcap, const double* __restrict__ S,
                                                  const double* __restrict__ Y, int64_t ld,
                                                  const double* __restrict__ rho, const double* __restrict__ alpha,
                                                  const double* __restrict__ zin, double* __restrict__ zout,
                                                  double* part, GridSync gs) {
  __shared__ double sh[32];
  __shared__ int s_fail;
  __shared__ double s_val;
  unsigned seq = *(volatile unsigned*)gs.seq;
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double z[NPT];
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    int64_t idx = tid + s * T;
    z[s] = idx < n ? zin[idx] : 0.0;
  }
  for (int c = 0; c < k; c++) {
    int slot = (head + c) % mcap;
    const double* si = S + (int64_t)slot * ld;
    const double* yi = Y + (int64_t)slot * ld;
    double loc = 0.0;
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      int64_t idx = tid + s * T;
      if (idx < n) loc += yi[idx] * z[s];
    }
    double bs = block_sum0(loc, sh);
    int last = threadIdx.x == 0 ? grid_arrive(gs, part, bs) : 0;
    double sv[NPT];  // streams in while the reduction completes
#pragma unroll
    for (int s = 0; s < NPT; s++) {
      int64_t idx = tid + s * T;
      sv[s] = idx < n ? si[idx] : 0.0;
    }
    double tot;
    if (!grid_complete(gs, part, seq++, last, &s_val, &s_fail, tot)) return;
    double beta = rho[slot] * tot;
    double coef = alpha[c] - beta;
#pragma unroll
    for (int s = 0; s < NPT; s++) z[s] += coef * sv[s];
  }
#pragma unroll
  for (int s = 0; s < NPT; s++) {
    int64_t idx = tid + s * T;
    if (idx < n) zout[idx] = z[s];
  }
}

static int coop_grid(fe_mesh m, const void* fn, int* grid) {
  int per_sm = 0;
  FE_TRY(fe_kernel_occupancy(fn, 256, 0, &per_sm));
  if (per_sm < 1) return fe_set_error("persistent kernel does not fit on an SM"), FE_ERR_CUDA;
  *grid = per_sm * m->sm_count;
  if (*grid > RED_SLOTS) *grid = RED_SLOTS;
  return FE_OK;
}

#define TL_FN(name, N) ((const void*)name<N>)

static int launch_twoloop(fe_mesh m, int which, void** args) {
  const void* f1[6] = {TL_FN(k_twoloop1, 1), TL_FN(k_twoloop1, 2), TL_FN(k_twoloop1, 4),
                       TL_FN(k_twoloop1, 8), TL_FN(k_twoloop1, 16), TL_FN(k_twoloop1, 32)};
  const void* f2[6] = {TL_FN(k_twoloop2, 1), TL_FN(k_twoloop2, 2), TL_FN(k_twoloop2, 4),
                       TL_FN(k_twoloop2, 8), TL_FN(k_twoloop2, 16), TL_FN(k_twoloop2, 32)};
  const int npts[6] = {1, 2, 4, 8, 16, 32};
  const void** fns = which == 1 ? f1 : f2;
  int64_t n = m->ndof;
  int grid = 0, q = 0;
  for (q = 0; q < 6; q++) {
    FE_TRY(coop_grid(m, fns[q], &grid));
    if ((int64_t)grid * 256 * npts[q] >= n) break;
  }
  if (q == 6) return fe_set_error("vector too long for the persistent two-loop kernel"), FE_ERR_ARG;
  int64_t per_block = 256LL * npts[q];
  int need = (int)((n + per_block - 1) / per_block);
  if (need < grid) grid = need;
  int k = *(int*)args[1];
  FE_SCOPE_F(m, FE_PROF_TWOLOOP, 16.0 * (double)n * (k + 1), 4.0 * (double)n * k);
  FE_CUDA(cudaLaunchCooperativeKernel(fns[q], dim3(grid), dim3(256), args, 0, m->stream));
  return FE_OK;
}

// z = H_k q with the pairs at ring slots (head + c) % mcap, c = 0..k-1 oldest
// first; H0 = preconditioner (h0 = 0), identity (h0 = 1) or GMRES (h0 = 2).
int fe_lbfgs_dev(fe_mesh m, const double* S, const double* Y, const double* rho, int head, int mcap, int k,
                 int64_t ld, const double* q, double* z, int h0, double ksp_rtol, double ksp_atol, int restart,
                 int kmaxit, int* lit) {
  FE_TRY(fe_workspace(m, restart > 0 ? restart : 1));
  int64_t n = m->ndof;
  if (k > LBFGS_MAX) return fe_set_error("at most %d stored pairs", LBFGS_MAX), FE_ERR_ARG;
  if (!m->alpha_d) FE_TRY(fe_alloc_t(m, &m->alpha_d, LBFGS_MAX));
  double* alpha = m->alpha_d;
  double* qbuf = m->t64;
  double* part = m->red;
  GridSync gs = grid_sync(m);
  if (k > 0) {
    void* a1[] = {(void*)&n, (void*)&k, (void*)&head, (void*)&mcap, (void*)&S, (void*)&Y, (void*)&ld, (void*)&rho,
                  (void*)&q, (void*)&qbuf, (void*)&alpha, (void*)&part, (void*)&gs};
    FE_TRY(launch_twoloop(m, 1, a1));
  } else {
    FE_SCOPE(m, FE_PROF_VECTOR, 16.0 * n);
    k_copy<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(n, q, qbuf);
  }
  double* zb = m->u64;
  if (h0 == 0) {
    FE_TRY(fe_pc_dev(m, qbuf, zb));
  } else if (h0 == 1) {
    FE_SCOPE(m, FE_PROF_VECTOR, 16.0 * n);
    k_copy<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(n, qbuf, zb);
  } else {
    // GMRES needs t64/u64 itself: move q aside into z's storage first
    {
      FE_SCOPE(m, FE_PROF_VECTOR, 16.0 * n);
      k_copy<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(n, qbuf, z);
    }
    if (!m->lb_x) FE_TRY(fe_alloc_t(m, &m->lb_x, (size_t)n));
    double* xs = m->lb_x;
    FE_CUDA(cudaMemsetAsync(xs, 0, n * sizeof(double), m->stream));
    int its = 0;
    double res = 0.0;
    FE_TRY(fe_gmres_dev(m, z, xs, ksp_rtol, ksp_atol, restart, kmaxit, &its, &res));
    if (lit) *lit += its;
    FE_SCOPE(m, FE_PROF_VECTOR, 16.0 * n);
    k_copy<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(n, xs, zb);
  }
  FE_CUDA(cudaGetLastError());
  if (k > 0) {
    void* a2[] = {(void*)&n, (void*)&k, (void*)&head, (void*)&mcap, (void*)&S, (void*)&Y, (void*)&ld,
                  (void*)&rho, (void*)&alpha, (void*)&zb, (void*)&z, (void*)&part, (void*)&gs};
    FE_TRY(launch_twoloop(m, 2, a2));
  } else {
    FE_SCOPE(m, FE_PROF_VECTOR, 16.0 * n);
    k_copy<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(n, zb, z);
  }
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// ---------------------------------------------------------------- C ABI
extern "C" int fe_spmv(fe_mesh m, const double* x, double* y) {
  if (!m || !x || !y) return fe_set_error("NULL argument"), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  FE_TRY(fe_spmv_dev(m, x, y));
  return fe_check_device_error(m);
}

extern "C" int fe_pc_apply(fe_mesh m, const double* x, double* y) {
  if (!m || !x || !y) return fe_set_error("NULL argument"), FE_ERR_ARG;
  if (m->prec < 0) return fe_set_error("no tangent assembled"), FE_ERR_STATE;
  FE_CUDA(cudaSetDevice(m->device));
  FE_TRY(fe_pc_dev(m, x, y));
  return fe_check_device_error(m);
}

extern "C" int fe_gmres(fe_mesh m, const double* b, double* x, double rtol, double atol, int restart, int max_it,
                        int orthog, int* iters, double* res_out) {
  if (!m || !b || !x) return fe_set_error("NULL argument"), FE_ERR_ARG;
  if (!(rtol >= 0.0) || !(atol >= 0.0) || max_it < 0) return fe_set_error("bad tolerances"), FE_ERR_ARG;
  if (orthog < 0 || orthog > 2) return fe_set_error("orthog must be 0, 1 or 2"), FE_ERR_ARG;
  FE_CUDA(cudaSetDevice(m->device));
  m->orthog = orthog;
  FE_TRY(fe_gmres_dev(m, b, x, rtol, atol, restart, max_it, iters, res_out));
  return fe_check_device_error(m);
}

extern "C" int fe_lbfgs_apply(fe_mesh m, const double* S, const double* Y, const double* rho, int k,
                              const double* q, double* z, int h0) {
  if (!m || !q || !z || k < 0 || (k > 0 && (!S || !Y || !rho))) return fe_set_error("bad arguments"), FE_ERR_ARG;
  if (h0 != 0 && h0 != 1) return fe_set_error("h0 must be 0 or 1"), FE_ERR_ARG;
  if (h0 == 0 && m->prec < 0) return fe_set_error("no tangent assembled"), FE_ERR_STATE;
  FE_CUDA(cudaSetDevice(m->device));
  FE_TRY(fe_lbfgs_dev(m, S, Y, rho, 0, k > 0 ? k : 1, k, m->ndof, q, z, h0, 0.0, 0.0, 1, 1, nullptr));
  return fe_check_device_error(m);
}

FE_DBG_BOUNDS_READER(fe_dbg_bounds_krylov)
