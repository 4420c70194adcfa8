// fe_element.cuh -- device code of the element level shared by the
// assembly kernels (fe_assemble.cu) and the one-CTA-per-request batched
// solver (fe_batch.cu): material laws at a quadrature point, shape
// functions, the follower-pressure face terms, and per-item bodies of the
// residual (element, node), tangent (element tile, face-pattern row) and
// block-Jacobi (node) kernels, each a function of its item index so that a
// kernel can map items to threads or loop over them.
#pragma once

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

// MASS adds the inertia of a Newmark step, mass_c M d with mass_c = 4 rho /
// dt^2 (the step's constant part 4/dt^2 M dhat enters in the gather); the
// static instantiation carries none of its registers.
template <int ORDER, bool MASS>
__device__ __forceinline__ void elem_residual_item(int t, int ne, const int* __restrict__ conn,
                                                       const double* __restrict__ geo,
                                                       const double* __restrict__ d, int nn, int pres,
                                                       MatParams mp, const double* __restrict__ fib,
                                                       double mass_c, double* __restrict__ rel,
                                                       double* __restrict__ relp) {
  constexpr int NEN = ORDER == 1 ? 4 : 10;
  constexpr int NQ = ORDER == 1 ? 1 : 4;
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
  if (MASS) {  // consistent mass, rows a = q (mod NQ) in this thread
    const double mc = mass_c * vol;
#pragma unroll
    for (int b = 0; b < NEN; b++) {
      const double* u = d + 3 * (size_t)c[b];
      const double u0 = u[0], u1 = u[1], u2 = u[2];
#pragma unroll
      for (int a = 0; a < NEN; a++)
        if (a % NQ == q) {
          const double w = mc * mass_hat(ORDER, a, b);
          r[3 * a] += w * u0;
          r[3 * a + 1] += w * u1;
          r[3 * a + 2] += w * u2;
        }
    }
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

// ---------------------------------------------------------------- follower pressure
// Degree-4 six-point triangle rule (Dunavant 1985, "High degree efficient
// symmetrical Gaussian quadrature rules for the triangle"): barycentric
// points (a, a, 1 - 2a) and their permutations for two values of a; the
// weights integrate over the reference triangle of area 1/2.  The follower
// integrands (degree 4 on P2 faces, 2 on P1) are integrated exactly.
__device__ __forceinline__ void tri_rule6(int q, double l[3], double& w) {
  const double a = q < 3 ? 0.445948490915965 : 0.091576213509771;
  w = q < 3 ? 0.5 * 0.223381589678011 : 0.5 * 0.109951743655322;
  const int k = q % 3;
  for (int i = 0; i < 3; i++) l[i] = i == k ? 1.0 - 2.0 * a : a;
}

// face shapes N_a and their derivatives along xi = l1 and eta = l2 (l0 =
// 1 - xi - eta); local nodes: vertices 0..2, P2 edge nodes (0,1), (1,2), (2,0)
template <int ORDER>
__device__ __forceinline__ void tri_shapes(const double l[3], double N[6], double Nx[6], double Ne[6]) {
  double dN[6][3];
  if (ORDER == 1) {
    for (int a = 0; a < 3; a++) {
      N[a] = l[a];
      for (int c = 0; c < 3; c++) dN[a][c] = a == c ? 1.0 : 0.0;
    }
  } else {
    for (int a = 0; a < 3; a++) {
      N[a] = l[a] * (2.0 * l[a] - 1.0);
      for (int c = 0; c < 3; c++) dN[a][c] = a == c ? 4.0 * l[a] - 1.0 : 0.0;
    }
    for (int k = 0; k < 3; k++) {
      const int i = k, j = (k + 1) % 3;
      N[3 + k] = 4.0 * l[i] * l[j];
      for (int c = 0; c < 3; c++) dN[3 + k][c] = c == i ? 4.0 * l[j] : (c == j ? 4.0 * l[i] : 0.0);
    }
  }
  for (int a = 0; a < (ORDER == 1 ? 3 : 6); a++) {
    Nx[a] = dN[a][1] - dN[a][0];
    Ne[a] = dN[a][2] - dN[a][0];
  }
}

// deformed tangents x_xi, x_eta of follower face f at barycentric point l
template <int ORDER>
__device__ __forceinline__ void face_tangents(const int* __restrict__ fnodes, const double* __restrict__ X,
                                              const double* __restrict__ d, const double Nx[6],
                                              const double Ne[6], double xs[3], double xe[3]) {
  for (int i = 0; i < 3; i++) xs[i] = xe[i] = 0.0;
  for (int c = 0; c < (ORDER == 1 ? 3 : 6); c++) {
    const size_t n = (size_t)fnodes[c];
    for (int i = 0; i < 3; i++) {
      const double x = X[3 * n + i] + d[3 * n + i];
      xs[i] += Nx[c] * x;
      xe[i] += Ne[c] * x;
    }
  }
}

// residual contribution of local node a of a follower face (load factor
// applied): kind 3, p int N_a (x_xi x x_eta); kind 5, -int N_a t |x_xi x x_eta|
template <int ORDER>
__device__ void follower_force(const int* __restrict__ fnodes, int kind, const double* fd, double load, int a,
                               const double* __restrict__ X, const double* __restrict__ d, double f[3]) {
  const double p = load * fd[0];
  f[0] = f[1] = f[2] = 0.0;
  for (int q = 0; q < (ORDER == 1 ? 1 : 6); q++) {
    double l[3], w, N[6], Nx[6], Ne[6], xs[3], xe[3];
    if (ORDER == 1) {  // constant normal: int N_a = 1/6
      l[0] = l[1] = l[2] = 1.0 / 3.0;
      w = 0.5;
    } else {
      tri_rule6(q, l, w);
    }
    tri_shapes<ORDER>(l, N, Nx, Ne);
    face_tangents<ORDER>(fnodes, X, d, Nx, Ne, xs, xe);
    const double n0 = xs[1] * xe[2] - xs[2] * xe[1], n1 = xs[2] * xe[0] - xs[0] * xe[2],
                 n2 = xs[0] * xe[1] - xs[1] * xe[0];
    if (kind == 5) {
      const double s = -w * load * N[a] * sqrt(n0 * n0 + n1 * n1 + n2 * n2);
      f[0] += s * fd[0];
      f[1] += s * fd[1];
      f[2] += s * fd[2];
    } else {
      const double s = w * p * N[a];
      f[0] += s * n0;
      f[1] += s * n1;
      f[2] += s * n2;
    }
  }
}

// derivative of that contribution with respect to the displacement of
// local node b (not symmetric): kind 3, p int N_a skew(Ne_b x_xi - Nx_b
// x_eta) with skew(w) v = w x v; kind 5, -int N_a t (x) g_b with g_b =
// d|n|/d x_b = Nx_b (x_eta x n^) + Ne_b (n^ x x_xi), n^ = n/|n|
template <int ORDER>
__device__ void follower_block(const int* __restrict__ fnodes, int kind, const double* fd, double load, int a, int b,
                               const double* __restrict__ X, const double* __restrict__ d, double K[9]) {
  const double p = load * fd[0];
  for (int k = 0; k < 9; k++) K[k] = 0.0;
  for (int q = 0; q < (ORDER == 1 ? 1 : 6); q++) {
    double l[3], w, N[6], Nx[6], Ne[6], xs[3], xe[3];
    if (ORDER == 1) {
      l[0] = l[1] = l[2] = 1.0 / 3.0;
      w = 0.5;
    } else {
      tri_rule6(q, l, w);
    }
    tri_shapes<ORDER>(l, N, Nx, Ne);
    face_tangents<ORDER>(fnodes, X, d, Nx, Ne, xs, xe);
    if (kind == 5) {
      const double n0 = xs[1] * xe[2] - xs[2] * xe[1], n1 = xs[2] * xe[0] - xs[0] * xe[2],
                   n2 = xs[0] * xe[1] - xs[1] * xe[0];
      const double inl = 1.0 / sqrt(n0 * n0 + n1 * n1 + n2 * n2);
      const double h0 = n0 * inl, h1 = n1 * inl, h2 = n2 * inl;
      const double gb[3] = {Nx[b] * (xe[1] * h2 - xe[2] * h1) + Ne[b] * (h1 * xs[2] - h2 * xs[1]),
                            Nx[b] * (xe[2] * h0 - xe[0] * h2) + Ne[b] * (h2 * xs[0] - h0 * xs[2]),
                            Nx[b] * (xe[0] * h1 - xe[1] * h0) + Ne[b] * (h0 * xs[1] - h1 * xs[0])};
      const double s = -w * load * N[a];
      for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) K[3 * i + k] += s * fd[i] * gb[k];
      continue;
    }
    const double s = w * p * N[a];
    double v[3];
    for (int i = 0; i < 3; i++) v[i] = s * (Ne[b] * xs[i] - Nx[b] * xe[i]);
    K[1] -= v[2];
    K[2] += v[1];
    K[3] += v[2];
    K[5] -= v[0];
    K[6] -= v[1];
    K[7] += v[0];
  }
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

// Follower faces of the mesh, passed by value to the kernels that evaluate them.
struct FollowerFaces {
  int n;                    // number of follower faces (0: none)
  const int* nodes;         // [n][6]
  const int* kind;          // [n] 3 (pressure) or 5 (traction per unit deformed area)
  const double* data;       // [n][3] p or t at load factor 1
  const int* node_ptr;      // [nn+1] node -> slots face * 8 + local node
  const int* node_list;
  const int* blk_ptr;       // [nnz_ks+1] face-pattern entry -> face * 64 + a * 8 + b
  const int* blk_list;
  const double* X;          // [nn][3] reference positions
};

// Node-wise gather of the element contributions plus the boundary and
// Newmark terms: R = sum rel - load fext1 + Ks d + follower forces - fdyn
// (fdyn = 4/dt^2 M dhat + 2/dt C dtil, nullptr when static; the dashpots'
// 2/dt C d sits in ks_val while dynamics is on).  FOLLOW: the mesh has
// follower faces (the instantiation without them keeps the plain gather's
// registers).
// returns this row's ||R||^2 contribution
template <int ORDER, bool FOLLOW>
__device__ __forceinline__ double gather_node(int t, 
    int nn, int nen, const int* __restrict__ node_ptr, const int* __restrict__ node_list,
    const double* __restrict__ rel, const double* __restrict__ fext1, double load,
    const int* __restrict__ ks_ptr, const int* __restrict__ ks_col, const double* __restrict__ ks_val,
    const double* __restrict__ d, const uint8_t* __restrict__ fixmask, int np,
    const int* __restrict__ vert_ptr, const int* __restrict__ vert_list, const double* __restrict__ relp,
    FollowerFaces ff, const double* __restrict__ fdyn,
    double* __restrict__ r, int64_t nrel) {
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
    if (FOLLOW)
      for (int k = ff.node_ptr[t]; k < ff.node_ptr[t + 1]; k++) {
        const int slot = ff.node_list[k], f = fe_idx(slot >> 3, ff.n);
        double fv[3];
        follower_force<ORDER>(ff.nodes + 6 * (size_t)f, ff.kind[f], ff.data + 3 * (size_t)f, load, slot & 7, ff.X,
                              d, fv);
        s0 += fv[0];
        s1 += fv[1];
        s2 += fv[2];
      }
    if (fdyn) {
      s0 -= fdyn[3 * (size_t)t];
      s1 -= fdyn[3 * (size_t)t + 1];
      s2 -= fdyn[3 * (size_t)t + 2];
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
  return acc;
}

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
// One group of EPB elements (tile) of one colour assembled by the whole CTA
// (phases separated by __syncthreads; a caller looping over tiles puts a
// __syncthreads between calls)
template <int ORDER, class T>
__device__ __forceinline__ void tangent_tile(int tile, 
    int nel, const int* __restrict__ elems, const int* __restrict__ conn, const double* __restrict__ geo,
    const double* __restrict__ d, int nn, int pres, MatParams mp, const double* __restrict__ fib,
    const int* __restrict__ emap, const int* __restrict__ upmap, const uint8_t* __restrict__ fixmask,
    double mass_c, T* __restrict__ K, T* __restrict__ B, int64_t nnzb) {
  using C = TanCfg<ORDER, T>;
  constexpr int NEN = C::NEN, NQ = C::NQ, EPB = C::EPB;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  __shared__ QPState<T> qs[EPB * NQ];
  __shared__ int sconn[EPB][NEN];
  __shared__ int selem[EPB];
  const int e0 = tile * EPB;
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
    if (mass_c != 0.0) {  // inertia of a Newmark step: 4 rho / dt^2 M_ab on the block diagonal
      const T mv = (T)(mass_c * NQ * mass_hat(ORDER, a, b));  // w = vol / NQ multiplies acc below
#pragma unroll
      for (int kk = 0; kk < 3; kk++)
        if (kk == i) acc[kk] += mv;
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

// face-pattern blocks: springs (plus 2/dt dashpots while dynamics is on)
// and the follower-pressure blocks at d, in FP64, prescribed components
// masked; one thread per node row, the faces of an entry in a fixed order
template <int ORDER, class T>
__device__ __forceinline__ void face_blocks_row(int a, int nn, const int* __restrict__ ks_ptr, const int* __restrict__ ks_col,
                                  const double* __restrict__ ks_val, const int* __restrict__ ks_kpos,
                                  const uint8_t* __restrict__ fixmask, FollowerFaces ff,
                                  const double* __restrict__ d, double load, T* K) {
  if (a >= nn) return;
  for (int k = ks_ptr[a]; k < ks_ptr[a + 1]; k++) {
    uint8_t fa = fixmask[a], fb = fixmask[ks_col[k]];
    const int p = ks_kpos[k];
    double blk[9];
    for (int c = 0; c < 9; c++) blk[c] = ks_val[(size_t)k * 9 + c];
    if (ff.n)
      for (int j = ff.blk_ptr[k]; j < ff.blk_ptr[k + 1]; j++) {
        const int code = ff.blk_list[j], f = fe_idx(code >> 6, ff.n);
        double fk[9];
        follower_block<ORDER>(ff.nodes + 6 * (size_t)f, ff.kind[f], ff.data + 3 * (size_t)f, load, (code >> 3) & 7,
                              code & 7, ff.X, d, fk);
        for (int c = 0; c < 9; c++) blk[c] += fk[c];
      }
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++)
        if (!((fa >> i) & 1) && !((fb >> j) & 1)) K[kv_index(p, 3 * i + j)] += (T)blk[3 * i + j];
  }
}

// unit diagonal at prescribed components, then invert each 3x3 diagonal block
template <class T, class DT>
__device__ __forceinline__ void diag_inverse_row(int a, int nn, const int* __restrict__ diag_pos, const uint8_t* __restrict__ fixmask,
                               T* K, DT* Dinv) {
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
