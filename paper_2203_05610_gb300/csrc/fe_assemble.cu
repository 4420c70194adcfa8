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

#include "fe_internal.h"

// ---------------------------------------------------------------- small math
template <class T>
__device__ __forceinline__ T dlog(T x) { return log(x); }
template <>
__device__ __forceinline__ float dlog<float>(float x) { return logf(x); }
template <class T>
__device__ __forceinline__ T dexp(T x) { return exp(x); }
template <>
__device__ __forceinline__ float dexp<float>(float x) { return expf(x); }
template <class T>
__device__ __forceinline__ T dcbrt(T x) { return cbrt(x); }
template <>
__device__ __forceinline__ float dcbrt<float>(float x) { return cbrtf(x); }
template <class T>
__device__ __forceinline__ T dsqrt(T x) { return sqrt(x); }
template <>
__device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }

// state of the material at one quadrature point
template <class T>
struct QPState {
  T F[9], H[9];   // deformation gradient, H = F^{-T}
  T J, I1, p;     // det F, tr(F^T F), pressure
  T S[9], D[9];   // Guccione: S = C e^Q D, D = R (B o E_f) R^T
  T eQ;           // Guccione: e^Q
  T a[3], an;     // Guccione: F f and |F f|
};

template <class T>
__device__ void qp_prepare(const MatParams& mp, const double* __restrict__ fib, QPState<T>& s) {
  const T* F = s.F;
  T c[9];  // cofactor matrix: c_iJ = d det / d F_iJ
  c[0] = F[4] * F[8] - F[5] * F[7];
  c[1] = F[5] * F[6] - F[3] * F[8];
  c[2] = F[3] * F[7] - F[4] * F[6];
  c[3] = F[2] * F[7] - F[1] * F[8];
  c[4] = F[0] * F[8] - F[2] * F[6];
  c[5] = F[1] * F[6] - F[0] * F[7];
  c[6] = F[1] * F[5] - F[2] * F[4];
  c[7] = F[2] * F[3] - F[0] * F[5];
  c[8] = F[0] * F[4] - F[1] * F[3];
  s.J = F[0] * c[0] + F[1] * c[1] + F[2] * c[2];
  T iJ = T(1) / s.J;
  s.I1 = T(0);
  for (int k = 0; k < 9; k++) {
    s.H[k] = c[k] * iJ;
    s.I1 += F[k] * F[k];
  }
  if (mp.kind != FE_MAT_GUCCIONE) return;
  T fr[9];
  for (int k = 0; k < 9; k++) fr[k] = (T)fib[k];  // rows f, s, n
  // E = (F^T F - I)/2, then its fibre-frame components Ef_ab = f_a . E f_b
  T E[9];
  for (int M = 0; M < 3; M++)
    for (int N = 0; N < 3; N++) {
      T v = T(0);
      for (int i = 0; i < 3; i++) v += F[3 * i + M] * F[3 * i + N];
      E[3 * M + N] = T(0.5) * (v - (M == N ? T(1) : T(0)));
    }
  T Ef[9];
  T Bm[9] = {(T)mp.bf, (T)mp.bfs, (T)mp.bfs, (T)mp.bfs, (T)mp.bt, (T)mp.bt, (T)mp.bfs, (T)mp.bt, (T)mp.bt};
  T Q = T(0);
  for (int a = 0; a < 3; a++) {
    T Ef_row[3];
    for (int N = 0; N < 3; N++) {
      T v = T(0);
      for (int M = 0; M < 3; M++) v += fr[3 * a + M] * E[3 * M + N];
      Ef_row[N] = v;
    }
    for (int b = 0; b < 3; b++) {
      T v = Ef_row[0] * fr[3 * b] + Ef_row[1] * fr[3 * b + 1] + Ef_row[2] * fr[3 * b + 2];
      Ef[3 * a + b] = Bm[3 * a + b] * v;  // B o Ef
      Q += Bm[3 * a + b] * v * v;
    }
  }
  s.eQ = dexp(Q);
  // D = R (B o Ef) R^T, R columns f, s, n
  for (int M = 0; M < 3; M++)
    for (int N = 0; N < 3; N++) {
      T v = T(0);
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) v += fr[3 * a + M] * Ef[3 * a + b] * fr[3 * b + N];
      s.D[3 * M + N] = v;
      s.S[3 * M + N] = (T)mp.C * s.eQ * v;
    }
  T an2 = T(0);
  for (int i = 0; i < 3; i++) {
    s.a[i] = F[3 * i] * fr[0] + F[3 * i + 1] * fr[1] + F[3 * i + 2] * fr[2];
    an2 += s.a[i] * s.a[i];
  }
  s.an = dsqrt(an2);
}

// C = F^T F (row-major 3x3)
template <class T>
__device__ __forceinline__ void poly_C(const T* F, T* Cm) {
  for (int M = 0; M < 3; M++)
    for (int N = 0; N < 3; N++) Cm[3 * M + N] = F[M] * F[N] + F[3 + M] * F[3 + N] + F[6 + M] * F[6 + N];
}

// first Piola stress P = dPsi/dF
template <class T>
__device__ void qp_stress(const MatParams& mp, const double* __restrict__ fib, const QPState<T>& s, T* P) {
  if (mp.kind == FE_MAT_COOK_NH) {
    T j13 = dcbrt(s.J);
    T jm23 = T(1) / (j13 * j13);
    T mu = (T)mp.mu, cv = (T)mp.cvol;
    T vol = T(2) * cv * (s.J * s.J - T(1));
    for (int k = 0; k < 9; k++) P[k] = mu * jm23 * (s.F[k] - s.I1 / T(3) * s.H[k]) + vol * s.H[k];
  } else if (mp.kind == FE_MAT_TH_NH) {
    T mu = (T)mp.mu;
    for (int k = 0; k < 9; k++) P[k] = mu * (s.F[k] - s.H[k]) - s.p * s.J * s.H[k];
  } else if (mp.kind == FE_MAT_POLYCONVEX) {
    // P = 2a F + 2b F (tr C I - C) - c H - p J H, C = F^T F
    const T a = (T)mp.ap, b = (T)mp.bp, c = (T)mp.clog;
    T Cm[9];
    poly_C(s.F, Cm);
    for (int i = 0; i < 3; i++)
      for (int Jj = 0; Jj < 3; Jj++) {
        const T fc = s.F[3 * i] * Cm[Jj] + s.F[3 * i + 1] * Cm[3 + Jj] + s.F[3 * i + 2] * Cm[6 + Jj];
        P[3 * i + Jj] = T(2) * a * s.F[3 * i + Jj] + T(2) * b * (s.I1 * s.F[3 * i + Jj] - fc) -
                        (c + s.p * s.J) * s.H[3 * i + Jj];
      }
  } else {
    T kap = (T)mp.kappa, g = (T)mp.gamma;
    T phi = T(0.5) * kap * (s.J * dlog(s.J) + s.J - T(1));
    for (int i = 0; i < 3; i++)
      for (int Jj = 0; Jj < 3; Jj++) {
        T v = s.F[3 * i] * s.S[Jj] + s.F[3 * i + 1] * s.S[3 + Jj] + s.F[3 * i + 2] * s.S[6 + Jj];
        P[3 * i + Jj] = v + phi * s.H[3 * i + Jj] + g * s.a[i] * (T)fib[Jj] / s.an;
      }
  }
}

template <class T>
__device__ T qp_energy(const MatParams& mp, const QPState<T>& s) {
  if (mp.kind == FE_MAT_COOK_NH) {
    T j13 = dcbrt(s.J);
    return T(0.5) * (T)mp.mu * (s.I1 / (j13 * j13) - T(3)) + (T)mp.cvol * (s.J * s.J - T(1) - T(2) * dlog(s.J));
  } else if (mp.kind == FE_MAT_TH_NH) {
    return T(0.5) * (T)mp.mu * (s.I1 - T(3)) - (T)mp.mu * dlog(s.J) - s.p * (s.J - T(1));
  } else if (mp.kind == FE_MAT_POLYCONVEX) {
    // cof F : cof F = ((tr C)^2 - tr(C^2)) / 2
    T Cm[9], trC2 = T(0);
    poly_C(s.F, Cm);
    for (int M = 0; M < 3; M++)
      for (int N = 0; N < 3; N++) trC2 += Cm[3 * M + N] * Cm[3 * N + M];
    const T I2 = T(0.5) * (s.I1 * s.I1 - trC2);
    return (T)mp.ap * (s.I1 - T(3)) + (T)mp.bp * (I2 - T(3)) - (T)mp.clog * dlog(s.J) - s.p * (s.J - T(1));
  }
  return T(0.5) * (T)mp.C * (s.eQ - T(1)) + T(0.5) * (T)mp.kappa * (s.J - T(1)) * dlog(s.J) + (T)mp.gamma * s.an;
}

// column (k, L) of the material tangent: col[iJ] = dP_iJ / dF_kL
template <class T>
__device__ void qp_tangent_col(const MatParams& mp, const double* __restrict__ fib, const QPState<T>& s,
                               int k, int L, T* col) {
  const T* F = s.F;
  const T* H = s.H;
  if (mp.kind == FE_MAT_COOK_NH) {
    T j13 = dcbrt(s.J);
    T mj = (T)mp.mu / (j13 * j13);
    T cv = (T)mp.cvol, J2 = s.J * s.J;
    T HkL = H[3 * k + L], FkL = F[3 * k + L];
    for (int i = 0; i < 3; i++)
      for (int Jj = 0; Jj < 3; Jj++) {
        T HiJ = H[3 * i + Jj];
        T hh = H[3 * i + L] * H[3 * k + Jj];
        T iso = ((i == k && Jj == L) ? T(1) : T(0)) - T(2) / T(3) * (HkL * F[3 * i + Jj] + FkL * HiJ) +
                T(2) / T(9) * s.I1 * HiJ * HkL + s.I1 / T(3) * hh;
        col[3 * i + Jj] = mj * iso + T(4) * cv * J2 * HiJ * HkL - T(2) * cv * (J2 - T(1)) * hh;
      }
  } else if (mp.kind == FE_MAT_TH_NH) {
    T mu = (T)mp.mu, pJ = s.p * s.J;
    for (int i = 0; i < 3; i++)
      for (int Jj = 0; Jj < 3; Jj++) {
        T hh = H[3 * i + L] * H[3 * k + Jj];
        col[3 * i + Jj] = mu * (((i == k && Jj == L) ? T(1) : T(0)) + hh) - pJ * (H[3 * i + Jj] * H[3 * k + L] - hh);
      }
  } else if (mp.kind == FE_MAT_POLYCONVEX) {
    // A_iJkL = 2a d_ik d_JL + 2b (2 F_kL F_iJ + I1 d_ik d_JL - d_ik C_LJ - F_iL F_kJ
    //          - (F F^T)_ik d_JL) + c H_iL H_kJ - p J (H_iJ H_kL - H_iL H_kJ)
    const T a = (T)mp.ap, b = (T)mp.bp, c = (T)mp.clog, pJ = s.p * s.J;
    T CL[3], Bk[3];  // row L of C = F^T F, column k of F F^T
    for (int q = 0; q < 3; q++) {
      CL[q] = F[L] * F[q] + F[3 + L] * F[3 + q] + F[6 + L] * F[6 + q];
      Bk[q] = F[3 * q] * F[3 * k] + F[3 * q + 1] * F[3 * k + 1] + F[3 * q + 2] * F[3 * k + 2];
    }
    const T FkL = F[3 * k + L];
    for (int i = 0; i < 3; i++)
      for (int Jj = 0; Jj < 3; Jj++) {
        const T dik = i == k ? T(1) : T(0), dJL = Jj == L ? T(1) : T(0);
        const T hh = H[3 * i + L] * H[3 * k + Jj];
        const T cof = T(2) * FkL * F[3 * i + Jj] + s.I1 * dik * dJL - dik * CL[Jj] - F[3 * i + L] * F[3 * k + Jj] -
                      Bk[i] * dJL;
        col[3 * i + Jj] = T(2) * a * dik * dJL + T(2) * b * cof + c * hh - pJ * (H[3 * i + Jj] * H[3 * k + L] - hh);
      }
  } else {
    T fr[9];
    for (int q = 0; q < 9; q++) fr[q] = (T)fib[q];
    T Bm[9] = {(T)mp.bf, (T)mp.bfs, (T)mp.bfs, (T)mp.bfs, (T)mp.bt, (T)mp.bt, (T)mp.bfs, (T)mp.bt, (T)mp.bt};
    // dE = (dF^T F + F^T dF)/2 with dF = e_k x e_L: dE_MN = (d_LM F_kN + F_kM d_LN)/2
    T dE[9];
    for (int M = 0; M < 3; M++)
      for (int N = 0; N < 3; N++)
        dE[3 * M + N] = T(0.5) * ((L == M ? F[3 * k + N] : T(0)) + (L == N ? F[3 * k + M] : T(0)));
    T DdE = T(0);
    for (int q = 0; q < 9; q++) DdE += s.D[q] * dE[q];
    // dD = R (B o (R^T dE R)) R^T
    T W[9];
    for (int a = 0; a < 3; a++) {
      T row[3];
      for (int N = 0; N < 3; N++) row[N] = fr[3 * a] * dE[N] + fr[3 * a + 1] * dE[3 + N] + fr[3 * a + 2] * dE[6 + N];
      for (int b = 0; b < 3; b++)
        W[3 * a + b] = Bm[3 * a + b] * (row[0] * fr[3 * b] + row[1] * fr[3 * b + 1] + row[2] * fr[3 * b + 2]);
    }
    T ce = (T)mp.C * s.eQ;
    T dS[9];
    for (int M = 0; M < 3; M++)
      for (int N = 0; N < 3; N++) {
        T v = T(0);
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) v += fr[3 * a + M] * W[3 * a + b] * fr[3 * b + N];
        dS[3 * M + N] = ce * (T(2) * DdE * s.D[3 * M + N] + v);
      }
    T lJ = dlog(s.J);
    T phi = T(0.5) * (T)mp.kappa * (s.J * lJ + s.J - T(1));
    T dphiJ = T(0.5) * (T)mp.kappa * (lJ + T(2)) * s.J;
    T g = (T)mp.gamma / s.an, an2 = s.an * s.an;
    for (int i = 0; i < 3; i++)
      for (int Jj = 0; Jj < 3; Jj++) {
        T v = (i == k) ? s.S[3 * L + Jj] : T(0);
        v += F[3 * i] * dS[Jj] + F[3 * i + 1] * dS[3 + Jj] + F[3 * i + 2] * dS[6 + Jj];
        v += dphiJ * H[3 * i + Jj] * H[3 * k + L] - phi * H[3 * i + L] * H[3 * k + Jj];
        v += g * (((i == k) ? T(1) : T(0)) - s.a[i] * s.a[k] / an2) * fr[L] * fr[Jj];
        col[3 * i + Jj] = v;
      }
  }
}

// ---------------------------------------------------------------- shape functions
// barycentric coordinates of quadrature point q: P1 centroid; P2 the
// symmetric 4-point degree-2 rule (alpha on vertex q, beta elsewhere)
template <int ORDER>
__device__ __forceinline__ double lam_q(int q, int c) {
  if (ORDER == 1) return 0.25;
  return c == q ? 0.5854101966249685 : 0.1381966011250105;
}

// gradient of shape function a at barycentric lam; G[4][3] barycentric gradients
template <int ORDER, class T>
__device__ __forceinline__ void shape_grad(int a, const T* lam, const T (*G)[3], T* g) {
  if (ORDER == 1 || a < 4) {
    T s = ORDER == 1 ? T(1) : T(4) * lam[a] - T(1);
    g[0] = s * G[a][0];
    g[1] = s * G[a][1];
    g[2] = s * G[a][2];
    return;
  }
  // edge nodes 4..9: (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
  const int ep[6] = {0, 0, 0, 1, 1, 2}, eq[6] = {1, 2, 3, 2, 3, 3};
  int p = ep[a - 4], q = eq[a - 4];
  for (int i = 0; i < 3; i++) g[i] = T(4) * (lam[p] * G[q][i] + lam[q] * G[p][i]);
}

template <class T>
__device__ __forceinline__ void load_G(const double* __restrict__ geo, int e, T (*G)[3], T& vol) {
  const double* g = geo + (size_t)e * 10;
  for (int r = 0; r < 3; r++)
    for (int i = 0; i < 3; i++) G[r + 1][i] = (T)g[3 * r + i];
  for (int i = 0; i < 3; i++) G[0][i] = -(G[1][i] + G[2][i] + G[3][i]);
  vol = (T)g[9];
}

// ---------------------------------------------------------------- residual
template <int ORDER>
__global__ void __launch_bounds__(128) k_elem_residual(int ne, const int* __restrict__ conn,
                                                       const double* __restrict__ geo,
                                                       const double* __restrict__ d, int nn, int pres,
                                                       MatParams mp, const double* __restrict__ fib,
                                                       double* __restrict__ rel, double* __restrict__ relp) {
  constexpr int NEN = ORDER == 1 ? 4 : 10;
  constexpr int NQ = ORDER == 1 ? 1 : 4;
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int e = t / NQ, q = t % NQ;
  bool live = e < ne;
  if (!live) e = ne - 1;  // keep the lanes of the warp together for the shuffles
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
    const double* u = d + 3 * (size_t)c[a];
    double u0 = u[0], u1 = u[1], u2 = u[2];
    for (int J = 0; J < 3; J++) {
      s.F[J] += u0 * g[J];
      s.F[3 + J] += u1 * g[J];
      s.F[6 + J] += u2 * g[J];
    }
  }
  s.p = 0.0;
  if (pres == 1)  // P1: vertex pressures with the barycentric shapes
    for (int v = 0; v < 4; v++) s.p += d[3 * (size_t)nn + c[v]] * lam[v];
  else if (pres == 2)  // P0: the element's constant pressure
    s.p = d[3 * (size_t)nn + e];
  const double* fe = fib ? fib + (size_t)e * 9 : nullptr;
  qp_prepare(mp, fe, s);
  double P[9];
  qp_stress(mp, fe, s, P);
  double wq = vol / NQ;
  double r[NEN * 3];
  for (int a = 0; a < NEN; a++) {
    double g[3];
    shape_grad<ORDER>(a, lam, G, g);
    for (int i = 0; i < 3; i++) r[3 * a + i] = wq * (P[3 * i] * g[0] + P[3 * i + 1] * g[1] + P[3 * i + 2] * g[2]);
  }
  double rp[4];  // R_p = -int (J - 1) q_h: P1 slots per vertex, P0 all in slot 0
  for (int v = 0; v < 4; v++)
    rp[v] = pres == 1 ? -wq * (s.J - 1.0) * lam[v] : (pres == 2 && v == 0 ? -wq * (s.J - 1.0) : 0.0);
  if (NQ > 1) {
#pragma unroll
    for (int off = 1; off < NQ; off <<= 1) {
      for (int k = 0; k < NEN * 3; k++) r[k] += __shfl_xor_sync(0xffffffffu, r[k], off);
      for (int v = 0; v < 4; v++) rp[v] += __shfl_xor_sync(0xffffffffu, rp[v], off);
    }
  }
  if (!live) return;
  double* out = rel + (size_t)e * NEN * 3;
#pragma unroll
  for (int k = 0; k < NEN * 3; k++)
    if (k % NQ == q) out[k] = r[k];
  if (pres) relp[(size_t)e * 4 + q] = rp[q];
}

// deterministic block reduction of one double (result valid in thread 0)
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0)
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// partial sums in red[blockIdx]; the last block to finish adds them in
// block order and writes *out (deterministic for a given grid)
__device__ __forceinline__ void grid_sum_finish(double v, double* red, unsigned* ticket, double* out) {
  __shared__ bool last;
  double bs = block_sum(v);
  if (threadIdx.x == 0) {
    red[blockIdx.x] = bs;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += ((volatile double*)red)[b];
  s = block_sum(s);
  if (threadIdx.x == 0) {
    *out = s;
    *ticket = 0u;
  }
}

__global__ void __launch_bounds__(256) k_gather_residual(
    int nn, int nen, const int* __restrict__ node_ptr, const int* __restrict__ node_list,
    const double* __restrict__ rel, const double* __restrict__ fext1, double load,
    const int* __restrict__ ks_ptr, const int* __restrict__ ks_col, const double* __restrict__ ks_val,
    const double* __restrict__ d, const uint8_t* __restrict__ fixmask, int np,
    const int* __restrict__ vert_ptr, const int* __restrict__ vert_list, const double* __restrict__ relp,
    double* __restrict__ r, double* red, unsigned* ticket, double* norm2, int64_t nrel) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (t < nn) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int k = node_ptr[t]; k < node_ptr[t + 1]; k++) {
      const double* c = rel + (size_t)fe_idx(node_list[k], nrel) * 3;
      s0 += c[0];
      s1 += c[1];
      s2 += c[2];
    }
    s0 -= load * fext1[3 * (size_t)t];
    s1 -= load * fext1[3 * (size_t)t + 1];
    s2 -= load * fext1[3 * (size_t)t + 2];
    for (int k = ks_ptr[t]; k < ks_ptr[t + 1]; k++) {
      const double* kv = ks_val + (size_t)k * 9;
      const double* u = d + 3 * (size_t)fe_idx(ks_col[k], nn);
      s0 += kv[0] * u[0] + kv[1] * u[1] + kv[2] * u[2];
      s1 += kv[3] * u[0] + kv[4] * u[1] + kv[5] * u[2];
      s2 += kv[6] * u[0] + kv[7] * u[1] + kv[8] * u[2];
    }
    uint8_t fm = fixmask[t];
    if (fm & 1) s0 = 0.0;
    if (fm & 2) s1 = 0.0;
    if (fm & 4) s2 = 0.0;
    r[3 * (size_t)t] = s0;
    r[3 * (size_t)t + 1] = s1;
    r[3 * (size_t)t + 2] = s2;
    acc = s0 * s0 + s1 * s1 + s2 * s2;
  } else if (t < nn + np) {
    int v = t - nn;
    double s = 0.0;
    for (int k = vert_ptr[v]; k < vert_ptr[v + 1]; k++) s += relp[vert_list[k]];
    r[3 * (size_t)nn + v] = s;
    acc = s * s;
  }
  if (norm2) grid_sum_finish(acc, red, ticket, norm2);
}

int fe_residual_dev(fe_mesh m, const double* d, double* r, bool want_norm) {
  int nthr = m->ne * m->nq;
  double eb = (double)m->ne * (4.0 * m->nen + 80.0 + 24.0 * m->nen + (m->fib ? 72.0 : 0.0) + (m->pres ? 32.0 : 0.0)) +
              8.0 * (double)m->ndof;
  {
    FE_SCOPE(m, FE_PROF_RESIDUAL, eb);
    if (m->order == 1)
    k_elem_residual<1><<<(nthr + 127) / 128, 128, 0, m->stream>>>(m->ne, m->conn, m->geo, d, m->nn, m->pres,
                                                                   m->mp, m->fib, m->rel, m->relp);
  else
    k_elem_residual<2><<<(nthr + 127) / 128, 128, 0, m->stream>>>(m->ne, m->conn, m->geo, d, m->nn, m->pres,
                                                                   m->mp, m->fib, m->rel, m->relp);
  }
  FE_CUDA(cudaGetLastError());
  int rows = m->nn + m->np;
  int grid = (rows + 255) / 256;
  if (grid > RED_SLOTS) return fe_set_error("mesh too large for the reduction buffer"), FE_ERR_ARG;
  double gb = (double)m->ne * m->nen * 28.0 + 4.0 * (m->nn + 1) + 25.0 * m->nn + 8.0 * (double)m->ndof +
              (m->pres ? (double)m->ne * 4 * 12.0 + 4.0 * (m->np + 1) : 0.0);
  FE_SCOPE(m, FE_PROF_RESIDUAL, gb);
  k_gather_residual<<<grid, 256, 0, m->stream>>>(m->nn, m->nen, m->node_ptr, m->node_list, m->rel, m->fext1,
                                                 m->load, m->ks_ptr, m->ks_col, m->ks_val, d, m->fixmask, m->np,
                                                 m->vert_ptr, m->vert_list, m->relp, r, m->red, m->red_ticket,
                                                 want_norm ? m->scal : nullptr, (int64_t)m->ne * m->nen);
  FE_CUDA(cudaGetLastError());
  return FE_OK;
}

// ---------------------------------------------------------------- energy
template <int ORDER>
__global__ void __launch_bounds__(128) k_elem_energy(int ne, const int* __restrict__ conn,
                                                     const double* __restrict__ geo, const double* __restrict__ d,
                                                     int nn, int pres, MatParams mp, const double* __restrict__ fib,
                                                     double* red, unsigned* ticket, double* out) {
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
  }
  grid_sum_finish(val, red, ticket, out);
}

// boundary part of the energy: -load fext.d + d.Ks d / 2
__global__ void k_node_energy(int nn, const double* __restrict__ fext1, double load, const int* __restrict__ ks_ptr,
                              const int* __restrict__ ks_col, const double* __restrict__ ks_val,
                              const double* __restrict__ d, double* red, unsigned* ticket, double* out) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (a < nn) {
    const double* u = d + 3 * (size_t)a;
    v = -load * (fext1[3 * a] * u[0] + fext1[3 * a + 1] * u[1] + fext1[3 * a + 2] * u[2]);
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
  if (m->order == 1)
    k_elem_energy<1><<<grid, 128, 0, m->stream>>>(m->ne, m->conn, m->geo, d, m->nn, m->pres, m->mp, m->fib,
                                                  m->red, m->red_ticket, m->scal + 1);
  else
    k_elem_energy<2><<<grid, 128, 0, m->stream>>>(m->ne, m->conn, m->geo, d, m->nn, m->pres, m->mp, m->fib,
                                                  m->red, m->red_ticket, m->scal + 1);
  FE_CUDA(cudaGetLastError());
  k_node_energy<<<(m->nn + 255) / 256, 256, 0, m->stream>>>(m->nn, m->fext1, m->load, m->ks_ptr, m->ks_col,
                                                            m->ks_val, d, m->red, m->red_ticket, m->scal + 2);
  FE_CUDA(cudaGetLastError());
  FE_CUDA(cudaMemcpyAsync(m->h_scal + 1, m->scal + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  FE_CUDA(cudaStreamSynchronize(m->stream));
  *out = m->h_scal[1] + m->h_scal[2];
  return FE_OK;
}

// ---------------------------------------------------------------- tangent
template <int ORDER, class T>
struct TanCfg {
  static constexpr int NEN = ORDER == 1 ? 4 : 10;
  static constexpr int NQ = ORDER == 1 ? 1 : 4;
  static constexpr int EPB = ORDER == 1 ? 8 : 2;   // elements per CTA
  static constexpr int NPAIR = NEN * (NEN + 1) / 2;
  // shared memory per element
  static constexpr int SZ_A = NQ * 81;
  static constexpr int SZ_G = NQ * NEN * 3;
  static constexpr int SZ_C = NQ * NEN * 27;
  static constexpr int SZ_DP = NQ * 9;
  static constexpr int SZ_L = NQ * 4;
  static constexpr int PER_E = SZ_A + SZ_G + SZ_C + SZ_DP + SZ_L + NQ;
};

// One CTA assembles EPB elements of one colour into the block-CSR values.
template <int ORDER, class T>
__global__ void __launch_bounds__(256) k_elem_tangent(
    int nel, const int* __restrict__ elems, const int* __restrict__ conn, const double* __restrict__ geo,
    const double* __restrict__ d, int nn, int pres, MatParams mp, const double* __restrict__ fib,
    const int* __restrict__ emap, const int* __restrict__ upmap, const uint8_t* __restrict__ fixmask,
    T* __restrict__ K, T* __restrict__ B, int64_t nnzb) {
  using C = TanCfg<ORDER, T>;
  constexpr int NEN = C::NEN, NQ = C::NQ, EPB = C::EPB;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  __shared__ QPState<T> qs[EPB * NQ];
  __shared__ int sconn[EPB][NEN];
  __shared__ int selem[EPB];
  const int e0 = blockIdx.x * EPB;
  for (int k = threadIdx.x; k < EPB * NEN; k += blockDim.x) {
    int le = k / NEN, a = k % NEN;
    int idx = e0 + le;
    int e = idx < nel ? elems[idx] : -1;
    if (a == 0) selem[le] = e;
    sconn[le][a] = e >= 0 ? conn[(size_t)e * NEN + a] : 0;
  }
  __syncthreads();
  auto Abuf = [&](int le, int q) { return sm + le * C::PER_E + q * 81; };
  auto Gbuf = [&](int le, int q) { return sm + le * C::PER_E + C::SZ_A + q * NEN * 3; };
  auto Cbuf = [&](int le, int q) { return sm + le * C::PER_E + C::SZ_A + C::SZ_G + q * NEN * 27; };
  auto DPbuf = [&](int le, int q) { return sm + le * C::PER_E + C::SZ_A + C::SZ_G + C::SZ_C + q * 9; };
  auto Lbuf = [&](int le, int q) { return sm + le * C::PER_E + C::SZ_A + C::SZ_G + C::SZ_C + C::SZ_DP + q * 4; };
  auto Wbuf = [&](int le) { return sm + le * C::PER_E + C::SZ_A + C::SZ_G + C::SZ_C + C::SZ_DP + C::SZ_L; };

  // phase 1a: F and the material state at each (element, QP)
  for (int k = threadIdx.x; k < EPB * NQ; k += blockDim.x) {
    int le = k / NQ, q = k % NQ;
    int e = selem[le];
    if (e < 0) continue;
    T G[4][3], vol;
    load_G(geo, e, G, vol);
    T lam[4];
    for (int c = 0; c < 4; c++) lam[c] = (T)lam_q<ORDER>(q, c);
    T* gb = Gbuf(le, q);
    QPState<T>& s = qs[k];
    for (int j = 0; j < 9; j++) s.F[j] = (j % 4 == 0) ? T(1) : T(0);
    for (int a = 0; a < NEN; a++) {
      T g[3];
      shape_grad<ORDER>(a, lam, G, g);
      gb[3 * a] = g[0];
      gb[3 * a + 1] = g[1];
      gb[3 * a + 2] = g[2];
      const double* u = d + 3 * (size_t)sconn[le][a];
      for (int i = 0; i < 3; i++)
        for (int J = 0; J < 3; J++) s.F[3 * i + J] += (T)u[i] * g[J];
    }
    s.p = T(0);
    if (pres == 1)
      for (int v = 0; v < 4; v++) s.p += (T)d[3 * (size_t)nn + sconn[le][v]] * lam[v];
    else if (pres == 2)
      s.p = (T)d[3 * (size_t)nn + selem[le]];
    qp_prepare(mp, fib ? fib + (size_t)e * 9 : nullptr, s);
    T* lb = Lbuf(le, q);
    // pressure shape functions: P1 the barycentric ones, P0 the constant
    for (int c = 0; c < 4; c++) lb[c] = pres == 2 ? (c == 0 ? T(1) : T(0)) : lam[c];
    if (q == 0) Wbuf(le)[0] = vol / NQ;
    if (pres) {
      T* dp = DPbuf(le, q);
      for (int j = 0; j < 9; j++) dp[j] = -s.J * s.H[j];
    }
  }
  __syncthreads();
  // phase 1b: columns of the material tangent A[iJ][kL]
  for (int k = threadIdx.x; k < EPB * NQ * 9; k += blockDim.x) {
    int lq = k / 9, kl = k % 9;
    int le = lq / NQ, q = lq % NQ;
    if (selem[le] < 0) continue;
    T colv[9];
    qp_tangent_col(mp, fib ? fib + (size_t)selem[le] * 9 : nullptr, qs[lq], kl / 3, kl % 3, colv);
    T* A = Abuf(le, q);
    for (int ij = 0; ij < 9; ij++) A[ij * 9 + kl] = colv[ij];
  }
  __syncthreads();
  // phase 2: C_b[iJ][k] = sum_L A[iJ][kL] g_b[L]
  for (int k = threadIdx.x; k < EPB * NQ * NEN * 9; k += blockDim.x) {
    int ij = k % 9;
    int b = (k / 9) % NEN;
    int q = (k / (9 * NEN)) % NQ;
    int le = k / (9 * NEN * NQ);
    if (selem[le] < 0) continue;
    const T* A = Abuf(le, q) + ij * 9;
    const T* g = Gbuf(le, q) + 3 * b;
    T* Cb = Cbuf(le, q) + b * 27 + ij * 3;
    for (int kk = 0; kk < 3; kk++) Cb[kk] = A[3 * kk] * g[0] + A[3 * kk + 1] * g[1] + A[3 * kk + 2] * g[2];
  }
  __syncthreads();
  // phase 3: K_ab[i][k] = sum_q w sum_J g_a[J] C_b[iJ][k] for a <= b; write
  // block (a,b) and its transpose (b,a); prescribed rows/columns are zeroed
  for (int k = threadIdx.x; k < EPB * C::NPAIR * 3; k += blockDim.x) {
    int i = k % 3;
    int pr = (k / 3) % C::NPAIR;
    int le = k / (3 * C::NPAIR);
    int e = selem[le];
    if (e < 0) continue;
    int a = 0, rem = pr;
    while (rem >= NEN - a) {
      rem -= NEN - a;
      a++;
    }
    int b = a + rem;
    T w = Wbuf(le)[0];
    T acc[3] = {T(0), T(0), T(0)};
    for (int q = 0; q < NQ; q++) {
      const T* ga = Gbuf(le, q) + 3 * a;
      const T* Cb = Cbuf(le, q) + b * 27;
      for (int J = 0; J < 3; J++) {
        T gj = ga[J];
        for (int kk = 0; kk < 3; kk++) acc[kk] += gj * Cb[(3 * i + J) * 3 + kk];
      }
    }
    int na = sconn[le][a], nb = sconn[le][b];
    uint8_t fa = fixmask[na], fb = fixmask[nb];
    const int* em = emap + (size_t)e * NEN * NEN;
    const int pab = fe_idx(em[a * NEN + b], nnzb);
    for (int kk = 0; kk < 3; kk++) {
      T v = w * acc[kk];
      if (((fa >> i) & 1) || ((fb >> kk) & 1)) v = T(0);
      K[kv_index(pab, 3 * i + kk)] += v;
    }
    if (a != b) {
      const int pba = fe_idx(em[b * NEN + a], nnzb);
      for (int kk = 0; kk < 3; kk++) {
        T v = w * acc[kk];
        if (((fa >> i) & 1) || ((fb >> kk) & 1)) v = T(0);
        K[kv_index(pba, 3 * kk + i)] += v;
      }
    }
  }
  // u-p coupling B[a][v][i] = sum_q w sum_J dPdp[iJ] g_a[J] lambda_v over the
  // element's local pressure values (P1: 4 vertices, P0: 1)
  if (pres) {
    const int npl = pres == 2 ? 1 : 4;
    for (int k = threadIdx.x; k < EPB * NEN * npl; k += blockDim.x) {
      int v = k % npl, a = (k / npl) % NEN, le = k / (npl * NEN);
      int e = selem[le];
      if (e < 0) continue;
      T w = Wbuf(le)[0];
      T acc[3] = {T(0), T(0), T(0)};
      for (int q = 0; q < NQ; q++) {
        const T* dp = DPbuf(le, q);
        const T* ga = Gbuf(le, q) + 3 * a;
        T lv = Lbuf(le, q)[v];
        for (int i = 0; i < 3; i++) acc[i] += lv * (dp[3 * i] * ga[0] + dp[3 * i + 1] * ga[1] + dp[3 * i + 2] * ga[2]);
      }
      uint8_t fa = fixmask[sconn[le][a]];
      T* Bv = B + (size_t)upmap[((size_t)e * NEN + a) * npl + v] * 3;
      for (int i = 0; i < 3; i++) Bv[i] += ((fa >> i) & 1) ? T(0) : w * acc[i];
    }
  }
}

// spring blocks (Robin faces), prescribed components masked
template <class T>
__global__ void k_add_springs(int nn, const int* __restrict__ ks_ptr, const int* __restrict__ ks_col,
                              const double* __restrict__ ks_val, const int* __restrict__ ks_kpos,
                              const uint8_t* __restrict__ fixmask, T* K) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nn) return;
  for (int k = ks_ptr[a]; k < ks_ptr[a + 1]; k++) {
    uint8_t fa = fixmask[a], fb = fixmask[ks_col[k]];
    const int p = ks_kpos[k];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++)
        if (!((fa >> i) & 1) && !((fb >> j) & 1)) K[kv_index(p, 3 * i + j)] += (T)ks_val[(size_t)k * 9 + 3 * i + j];
  }
}

// unit diagonal at prescribed components, then invert each 3x3 diagonal block
template <class T, class DT>
__global__ void k_diag_inverse(int nn, const int* __restrict__ diag_pos, const uint8_t* __restrict__ fixmask,
                               T* K, DT* Dinv) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nn) return;
  const int p = diag_pos[a];
  uint8_t fm = fixmask[a];
  for (int i = 0; i < 3; i++)
    if ((fm >> i) & 1) K[kv_index(p, 4 * i)] = T(1);
  T M[9];
  for (int k = 0; k < 9; k++) M[k] = K[kv_index(p, k)];
  T c0 = M[4] * M[8] - M[5] * M[7];
  T c1 = M[5] * M[6] - M[3] * M[8];
  T c2 = M[3] * M[7] - M[4] * M[6];
  T det = M[0] * c0 + M[1] * c1 + M[2] * c2;
  T id = T(1) / det;
  DT* o = Dinv + (size_t)a * 9;
  o[0] = (DT)(c0 * id);
  o[1] = (DT)((M[2] * M[7] - M[1] * M[8]) * id);
  o[2] = (DT)((M[1] * M[5] - M[2] * M[4]) * id);
  o[3] = (DT)(c1 * id);
  o[4] = (DT)((M[0] * M[8] - M[2] * M[6]) * id);
  o[5] = (DT)((M[2] * M[3] - M[0] * M[5]) * id);
  o[6] = (DT)(c2 * id);
  o[7] = (DT)((M[1] * M[6] - M[0] * M[7]) * id);
  o[8] = (DT)((M[0] * M[4] - M[1] * M[3]) * id);
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
                                                             m->fixmask, K, B, m->nnzb);
    FE_CUDA(cudaGetLastError());
  }
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
    if (m->nnz_ks) {
      FE_SCOPE(m, FE_PROF_TANGENT, (double)m->nnz_ks * (4 + 4 + 72 + 2 * 72));
      k_add_springs<double><<<(m->nn + 255) / 256, 256, 0, m->stream>>>(m->nn, m->ks_ptr, m->ks_col, m->ks_val,
                                                                        m->ks_kpos, m->fixmask, m->K64);
    }
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
    if (m->nnz_ks) {
      FE_SCOPE(m, FE_PROF_TANGENT, (double)m->nnz_ks * (4 + 4 + 72 + 2 * 36));
      k_add_springs<float><<<(m->nn + 255) / 256, 256, 0, m->stream>>>(m->nn, m->ks_ptr, m->ks_col, m->ks_val,
                                                                       m->ks_kpos, m->fixmask, m->K32);
    }
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
  if (m->pc_type == 1) FE_TRY(fe_amg_setup(m));  // the AMG hierarchy of this tangent
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
  FE_CUDA(cudaMalloc(&tmp, n * sizeof(double)));
  if (d16) k_widen_bf<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(n, d16, tmp);
  else k_widen<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(n, d32, tmp);
  cudaError_t e = cudaStreamSynchronize(m->stream);
  if (e == cudaSuccess) e = cudaMemcpy(host, tmp, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(tmp);
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

FE_DBG_BOUNDS_READER(fe_dbg_bounds_assemble)
