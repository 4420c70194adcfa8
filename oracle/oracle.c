/*
 * oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Follows arxiv 2203.05610 step by step:
 *   - problem: quasi-static R(d) = f - div P(F), F = I + grad d, P = dPsi/dF
 *     (Section "The hyperelasticity problem"), energy Pi (Eq. "minimization");
 *   - materials: Cook neo-Hookean Psi_Cook, Taylor-Hood neo-Hookean u-p form
 *     (twist stand-in), Guccione + active stress + epicardial springs
 *     (Section "Test problems and solvers details");
 *   - solvers: NK (Eq. "newton"), iNK with Eisenstat-Walker forcing, BFGS
 *     update and its two-loop recursion, BFGS-preonly and inexact BFGS
 *     (Section "Numerical solvers"), options of Appendix A, lower Schur
 *     preconditioner of Appendix B with the SIMPLE approximation;
 *   - GMRES with modified Gram-Schmidt, no restart in the paper (restart
 *     cap here), right preconditioning.
 * Readings where the paper is silent or garbled are listed in the
 * project's design notes and restated beside the code that takes them.
 */
#include "oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

/* ======================================================================
 * small helpers
 * ====================================================================== */
static void* xcalloc(size_t n, size_t sz) {
  void* p = calloc(n ? n : 1, sz);
  if (!p) abort();
  return p;
}

static double dot(const double* a, const double* b, long n) {
  double s = 0.0;
  for (long i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}

static double nrm2(const double* a, long n) { return sqrt(dot(a, a, n)); }

static double det3(const double M[3][3]) {
  return M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
         M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
         M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
}

/* inverse by the adjugate: Minv = adj(M) / det(M) */
static double inv3(const double M[3][3], double Minv[3][3]) {
  double d = det3(M);
  Minv[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / d;
  Minv[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / d;
  Minv[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / d;
  Minv[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / d;
  Minv[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / d;
  Minv[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / d;
  Minv[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / d;
  Minv[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / d;
  Minv[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / d;
  return d;
}

unsigned long long om_splitmix64(unsigned long long x) {
  /* splitmix64 output function (S. Vigna), applied to state x */
  unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* ======================================================================
 * quadrature (paper silent; readings: P1 one point, P2 the 4-point
 * degree-2 symmetric rule, triangles the 6-point degree-4 rule)
 * ====================================================================== */
int om_tet_rule(int order, double* lam, double* w) {
  if (order == 1) {
    for (int a = 0; a < 4; a++) lam[a] = 0.25;
    w[0] = 1.0;
    return 1;
  }
  const double a = 0.5854101966249685, b = 0.1381966011250105;
  for (int q = 0; q < 4; q++) {
    for (int c = 0; c < 4; c++) lam[4 * q + c] = (c == q) ? a : b;
    w[q] = 0.25;
  }
  return 4;
}

int om_tri_rule(double* lam, double* w) {
  const double a1 = 0.445948490915965, b1 = 0.108103018168070, w1 = 0.223381589678011;
  const double a2 = 0.091576213509771, b2 = 0.816847572980459, w2 = 0.109951743655322;
  int q = 0;
  for (int k = 0; k < 3; k++, q++) {
    for (int c = 0; c < 3; c++) lam[3 * q + c] = (c == k) ? b1 : a1;
    w[q] = w1;
  }
  for (int k = 0; k < 3; k++, q++) {
    for (int c = 0; c < 3; c++) lam[3 * q + c] = (c == k) ? b2 : a2;
    w[q] = w2;
  }
  return 6;
}

/* local edges of a tet and of a triangle */
static const int TET_EDGE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const int TRI_EDGE[3][2] = {{0, 1}, {1, 2}, {0, 2}};

/* values of the nen shape functions at barycentric lam (tet) */
static void tet_shape(int order, const double* lam, double* N) {
  if (order == 1) {
    for (int a = 0; a < 4; a++) N[a] = lam[a];
    return;
  }
  for (int a = 0; a < 4; a++) N[a] = lam[a] * (2.0 * lam[a] - 1.0);
  for (int e = 0; e < 6; e++) N[4 + e] = 4.0 * lam[TET_EDGE[e][0]] * lam[TET_EDGE[e][1]];
}

/* physical gradients of the shape functions given the gradients G[4][3] of
 * the barycentric coordinates */
static void tet_grad(int order, const double* lam, const double G[4][3], double dN[][3]) {
  if (order == 1) {
    for (int a = 0; a < 4; a++)
      for (int i = 0; i < 3; i++) dN[a][i] = G[a][i];
    return;
  }
  for (int a = 0; a < 4; a++)
    for (int i = 0; i < 3; i++) dN[a][i] = (4.0 * lam[a] - 1.0) * G[a][i];
  for (int e = 0; e < 6; e++) {
    int p = TET_EDGE[e][0], q = TET_EDGE[e][1];
    for (int i = 0; i < 3; i++) dN[4 + e][i] = 4.0 * (lam[p] * G[q][i] + lam[q] * G[p][i]);
  }
}

static void tri_shape(int order, const double* lam, double* N) {
  if (order == 1) {
    for (int a = 0; a < 3; a++) N[a] = lam[a];
    return;
  }
  for (int a = 0; a < 3; a++) N[a] = lam[a] * (2.0 * lam[a] - 1.0);
  for (int e = 0; e < 3; e++) N[3 + e] = 4.0 * lam[TRI_EDGE[e][0]] * lam[TRI_EDGE[e][1]];
}

/* ======================================================================
 * materials: Psi, P = dPsi/dF, A = dP/dF (A[9*(3i+J) + 3k+L]) and dP/dp
 * ====================================================================== */
#define IDX(i, J) (3 * (i) + (J))

static void cofactor_H(const double F[9], double* J, double H[9]) {
  /* H = F^{-T} */
  double M[3][3], Mi[3][3];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) M[i][j] = F[IDX(i, j)];
  *J = inv3(M, Mi);
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) H[IDX(i, j)] = Mi[j][i];
}

void om_material(const double* matp, const double* F, const double* fib, double gamma,
                 double p, double* psi, double* P, double* A, double* dPdp) {
  int kind = (int)matp[0];
  double J, H[9];
  cofactor_H(F, &J, H);
  double I1 = 0.0;
  for (int k = 0; k < 9; k++) I1 += F[k] * F[k];
  if (dPdp)
    for (int k = 0; k < 9; k++) dPdp[k] = 0.0;

  if (kind == 0) {
    /* Cook: Psi = C1 (tr(Fbar^T Fbar) - 3) + c_vol (J^2 - 1 - 2 ln J),
     * C1 = mu/2, tr(Fbar^T Fbar) = J^{-2/3} I1, mu = E/(2(1+nu)),
     * lambda = 2 mu nu/(1-2 nu), kappa = lambda + 2 mu/3.
     * Reading: c_vol = kappa/4 (consistent with linear elasticity at small
     * strain); vol_literal = 1 takes the printed coefficient kappa. */
    double E = matp[2], nu = matp[3];
    double mu = E / (2.0 * (1.0 + nu));
    double lam = 2.0 * mu * nu / (1.0 - 2.0 * nu);
    double kap = lam + 2.0 * mu / 3.0;
    double cv = ((int)matp[1]) ? kap : 0.25 * kap;
    double Jm23 = pow(J, -2.0 / 3.0);
    if (psi) *psi = 0.5 * mu * (Jm23 * I1 - 3.0) + cv * (J * J - 1.0 - 2.0 * log(J));
    /* P = mu J^{-2/3} (F - I1/3 H) + 2 c_vol (J^2 - 1) H */
    for (int k = 0; k < 9; k++)
      P[k] = mu * Jm23 * (F[k] - I1 / 3.0 * H[k]) + 2.0 * cv * (J * J - 1.0) * H[k];
    if (A) {
      for (int i = 0; i < 3; i++)
        for (int Jj = 0; Jj < 3; Jj++)
          for (int k = 0; k < 3; k++)
            for (int L = 0; L < 3; L++) {
              double dik = (i == k), dJL = (Jj == L);
              double iso = dik * dJL -
                           2.0 / 3.0 * (H[IDX(k, L)] * F[IDX(i, Jj)] + F[IDX(k, L)] * H[IDX(i, Jj)]) +
                           2.0 / 9.0 * I1 * H[IDX(i, Jj)] * H[IDX(k, L)] +
                           I1 / 3.0 * H[IDX(i, L)] * H[IDX(k, Jj)];
              double vol = 4.0 * cv * J * J * H[IDX(i, Jj)] * H[IDX(k, L)] -
                           2.0 * cv * (J * J - 1.0) * H[IDX(i, L)] * H[IDX(k, Jj)];
              A[9 * IDX(i, Jj) + IDX(k, L)] = mu * Jm23 * iso + vol;
            }
    }
    return;
  }

  if (kind == 1) {
    /* Taylor-Hood neo-Hookean (reading of the twist stand-in):
     * Psi = mu/2 (I1 - 3) - mu ln J - p (J - 1); P = mu (F - H) - p J H */
    double mu = matp[4];
    if (psi) *psi = 0.5 * mu * (I1 - 3.0) - mu * log(J) - p * (J - 1.0);
    for (int k = 0; k < 9; k++) P[k] = mu * (F[k] - H[k]) - p * J * H[k];
    if (dPdp)
      for (int k = 0; k < 9; k++) dPdp[k] = -J * H[k];
    if (A) {
      for (int i = 0; i < 3; i++)
        for (int Jj = 0; Jj < 3; Jj++)
          for (int k = 0; k < 3; k++)
            for (int L = 0; L < 3; L++) {
              double dik = (i == k), dJL = (Jj == L);
              double hh = H[IDX(i, L)] * H[IDX(k, Jj)];
              A[9 * IDX(i, Jj) + IDX(k, L)] =
                  mu * (dik * dJL + hh) - p * J * (H[IDX(i, Jj)] * H[IDX(k, L)] - hh);
            }
    }
    return;
  }

  if (kind == 3) {
    /* Polyconvex u-p potential of the paper's twist test (Section "Test
     * problems", Psi_Twist):
     *   Psi = a (F:F - 3) + b (cof F : cof F - 3) - c ln J - p (J - 1),
     * cof F = J F^{-T}, c = 4 beta_s + 2 alpha_s; the printed "log(F)" is read
     * as ln det F.  With C = F^T F, cof F : cof F = ((tr C)^2 - tr(C^2)) / 2,
     * whose derivative is 2 F (tr C I - C). */
    double a = matp[12], b = matp[13], c = matp[14];
    double Cm[3][3], Bl[3][3], FC[3][3], trC2 = 0.0;
    for (int M = 0; M < 3; M++)
      for (int N = 0; N < 3; N++) {
        double s = 0.0, t = 0.0;
        for (int q = 0; q < 3; q++) {
          s += F[IDX(q, M)] * F[IDX(q, N)];
          t += F[IDX(M, q)] * F[IDX(N, q)];
        }
        Cm[M][N] = s;
        Bl[M][N] = t;
      }
    for (int M = 0; M < 3; M++)
      for (int N = 0; N < 3; N++) trC2 += Cm[M][N] * Cm[N][M];
    for (int i = 0; i < 3; i++)
      for (int N = 0; N < 3; N++) {
        double s = 0.0;
        for (int M = 0; M < 3; M++) s += F[IDX(i, M)] * Cm[M][N];
        FC[i][N] = s;
      }
    double I2 = 0.5 * (I1 * I1 - trC2);
    if (psi) *psi = a * (I1 - 3.0) + b * (I2 - 3.0) - c * log(J) - p * (J - 1.0);
    for (int i = 0; i < 3; i++)
      for (int Jj = 0; Jj < 3; Jj++)
        P[IDX(i, Jj)] = 2.0 * a * F[IDX(i, Jj)] + 2.0 * b * (I1 * F[IDX(i, Jj)] - FC[i][Jj]) -
                        c * H[IDX(i, Jj)] - p * J * H[IDX(i, Jj)];
    if (dPdp)
      for (int k = 0; k < 9; k++) dPdp[k] = -J * H[k];
    if (A) {
      for (int i = 0; i < 3; i++)
        for (int Jj = 0; Jj < 3; Jj++)
          for (int k = 0; k < 3; k++)
            for (int L = 0; L < 3; L++) {
              double dik = (i == k), dJL = (Jj == L);
              double hh = H[IDX(i, L)] * H[IDX(k, Jj)];
              double cof = 2.0 * F[IDX(k, L)] * F[IDX(i, Jj)] + I1 * dik * dJL - dik * Cm[L][Jj] -
                           F[IDX(i, L)] * F[IDX(k, Jj)] - Bl[i][k] * dJL;
              A[9 * IDX(i, Jj) + IDX(k, L)] = 2.0 * a * dik * dJL + 2.0 * b * cof + c * hh -
                                              p * J * (H[IDX(i, Jj)] * H[IDX(k, L)] - hh);
            }
    }
    return;
  }

  /* kind 2: Guccione, Psi = C/2 (e^Q - 1) + kappa/2 (J - 1) ln J + gamma |F f|,
   * Q = sum_ab b_ab E_ab^2 in the fibre frame {f, s, n}, E = (F^T F - I)/2.
   * The active stress gamma (Ff) x f / |Ff| is the derivative of gamma |Ff|. */
  double C = matp[5], bf = matp[6], bt = matp[7], bfs = matp[8], kap = matp[9];
  double Bm[3][3] = {{bf, bfs, bfs}, {bfs, bt, bt}, {bfs, bt, bt}};
  double E[3][3];
  for (int M = 0; M < 3; M++)
    for (int N = 0; N < 3; N++) {
      double s = 0.0;
      for (int a = 0; a < 3; a++) s += F[IDX(a, M)] * F[IDX(a, N)];
      E[M][N] = 0.5 * (s - (M == N));
    }
  /* E in the fibre frame: Ef[a][b] = f_a . E f_b, fib rows are f, s, n */
  double Ef[3][3], Q = 0.0;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double s = 0.0;
      for (int M = 0; M < 3; M++)
        for (int N = 0; N < 3; N++) s += fib[3 * a + M] * E[M][N] * fib[3 * b + N];
      Ef[a][b] = s;
      Q += Bm[a][b] * s * s;
    }
  double eQ = exp(Q);
  /* D = R (B o Ef) R^T in the global frame; dQ/dE = 2 D; S = C e^Q D */
  double D[3][3];
  for (int M = 0; M < 3; M++)
    for (int N = 0; N < 3; N++) {
      double s = 0.0;
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) s += fib[3 * a + M] * Bm[a][b] * Ef[a][b] * fib[3 * b + N];
      D[M][N] = s;
    }
  double S[3][3];
  for (int M = 0; M < 3; M++)
    for (int N = 0; N < 3; N++) S[M][N] = C * eQ * D[M][N];
  double phi = 0.5 * kap * (J * log(J) + J - 1.0); /* dPsi_vol/dJ * J */
  double dphi = 0.5 * kap * (log(J) + 2.0);        /* d phi / dJ */
  double a_[3], an = 0.0;
  for (int i = 0; i < 3; i++) {
    a_[i] = 0.0;
    for (int Jj = 0; Jj < 3; Jj++) a_[i] += F[IDX(i, Jj)] * fib[Jj];
    an += a_[i] * a_[i];
  }
  an = sqrt(an);
  if (psi) *psi = 0.5 * C * (eQ - 1.0) + 0.5 * kap * (J - 1.0) * log(J) + gamma * an;
  for (int i = 0; i < 3; i++)
    for (int Jj = 0; Jj < 3; Jj++) {
      double s = 0.0;
      for (int M = 0; M < 3; M++) s += F[IDX(i, M)] * S[M][Jj];
      P[IDX(i, Jj)] = s + phi * H[IDX(i, Jj)] + gamma * a_[i] * fib[Jj] / an;
    }
  if (!A) return;
  /* A by directional derivatives dP[dF] with dF = e_k x e_L:
   * dE = (dF^T F + F^T dF)/2, dS = C e^Q (2 (D:dE) D + R (B o (R^T dE R)) R^T),
   * dP = dF S + F dS + vol + active parts. */
  for (int k = 0; k < 3; k++)
    for (int L = 0; L < 3; L++) {
      double dE[3][3];
      for (int M = 0; M < 3; M++)
        for (int N = 0; N < 3; N++)
          dE[M][N] = 0.5 * ((L == M) * F[IDX(k, N)] + F[IDX(k, M)] * (L == N));
      double DdE = 0.0;
      for (int M = 0; M < 3; M++)
        for (int N = 0; N < 3; N++) DdE += D[M][N] * dE[M][N];
      double dEf[3][3];
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
          double s = 0.0;
          for (int M = 0; M < 3; M++)
            for (int N = 0; N < 3; N++) s += fib[3 * a + M] * dE[M][N] * fib[3 * b + N];
          dEf[a][b] = s;
        }
      double dS[3][3];
      for (int M = 0; M < 3; M++)
        for (int N = 0; N < 3; N++) {
          double s = 0.0;
          for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) s += fib[3 * a + M] * Bm[a][b] * dEf[a][b] * fib[3 * b + N];
          dS[M][N] = C * eQ * (2.0 * DdE * D[M][N] + s);
        }
      for (int i = 0; i < 3; i++)
        for (int Jj = 0; Jj < 3; Jj++) {
          double v = (i == k) ? S[L][Jj] : 0.0;
          for (int M = 0; M < 3; M++) v += F[IDX(i, M)] * dS[M][Jj];
          v += dphi * J * H[IDX(i, Jj)] * H[IDX(k, L)] - phi * H[IDX(i, L)] * H[IDX(k, Jj)];
          v += gamma / an * ((i == k) - a_[i] * a_[k] / (an * an)) * fib[L] * fib[Jj];
          A[9 * IDX(i, Jj) + IDX(k, L)] = v;
        }
    }
}

/* ======================================================================
 * mesh
 * ====================================================================== */
struct om_mesh {
  int order, pres, nv, ne, nn, nen, np;
  long ndof;
  double* X;   /* [nn][3] */
  int* conn;   /* [ne][nen] */
  int* colors; /* [ne] */
  int ncolors;
  int* row_ptr; /* [nn+1] */
  int* col;     /* [nnzb] */
  long nnzb;
  int* up_ptr; /* [nn+1] u-p coupling rows (u nodes), columns = pressure dofs */
  int* up_col;
  long nnz_up;
  unsigned char* dgroup; /* [nn] */
  int ngroups;
  double* groups; /* [ngroups][8] */
  int nf;
  int* fnodes; /* [nf][6] face nodes (3 vertices, then 3 edge nodes for P2) */
  int* fkind;
  double* fdata;
  double matp[15];
  double* fib; /* [ne][9] or NULL */
  double load, time;
  /* tangent */
  double* K;    /* [nnzb][9] */
  double* B1;   /* [nnz_up][3] */
  double* Dinv; /* [nn][9] */
  double* Sd;   /* [np] Schur diagonal */
  int have_K;
  long long lit; /* Krylov iterations, accumulated by om_gmres */
  int pc_type;   /* displacement block: 0 nodal block-Jacobi, 1 algebraic multigrid */
  struct om_amg* amg;
  /* elastodynamics (om_set_dynamics): density, time step, mass per block
   * (scalar, M_ab = Mm I), dashpot matrix [nnzb][9], the state d_n, v_n, a_n
   * and the Newmark predictors dhat, dtil */
  int dyn;
  double rho, dt;
  double *Mm, *Cd, *dn, *vn, *an, *dhat, *dtil;
};

static int cmp_ll(const void* a, const void* b) {
  long long x = *(const long long*)a, y = *(const long long*)b;
  return (x > y) - (x < y);
}

/* id of the edge node between vertices a and b: binary search in the sorted
 * unique edge list */
static int edge_node(const long long* edges, long nedge, int nv, int a, int b) {
  long long key = (long long)(a < b ? a : b) * nv + (a < b ? b : a);
  long lo = 0, hi = nedge - 1;
  while (lo <= hi) {
    long mid = (lo + hi) / 2;
    if (edges[mid] == key) return nv + (int)mid;
    if (edges[mid] < key) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

typedef struct {
  unsigned long long pri;
  int id;
} pri_t;
static int cmp_pri(const void* a, const void* b) {
  const pri_t* x = (const pri_t*)a;
  const pri_t* y = (const pri_t*)b;
  if (x->pri != y->pri) return x->pri > y->pri ? -1 : 1; /* descending */
  return (x->id > y->id) - (x->id < y->id);
}

static void build_pattern(long nrow, long ncolk, const int* conn, int ne, int nen, int nenc,
                          const int* conn_c, int stride_c, int** ptr_out, int** col_out,
                          long* nnz_out) {
  /* all (row, col) pairs of nodes sharing an element, sorted and made unique */
  long npair = (long)ne * nen * nenc;
  long long* keys = (long long*)xcalloc(npair, sizeof(long long));
  long t = 0;
  for (int e = 0; e < ne; e++)
    for (int a = 0; a < nen; a++)
      for (int b = 0; b < nenc; b++)
        keys[t++] = (long long)conn[(long)e * nen + a] * ncolk + conn_c[(long)e * stride_c + b];
  qsort(keys, npair, sizeof(long long), cmp_ll);
  long nu = 0;
  for (long i = 0; i < npair; i++)
    if (i == 0 || keys[i] != keys[i - 1]) keys[nu++] = keys[i];
  int* ptr = (int*)xcalloc(nrow + 1, sizeof(int));
  int* col = (int*)xcalloc(nu, sizeof(int));
  for (long i = 0; i < nu; i++) {
    long r = keys[i] / ncolk;
    ptr[r + 1]++;
    col[i] = (int)(keys[i] % ncolk);
  }
  for (long r = 0; r < nrow; r++) ptr[r + 1] += ptr[r];
  free(keys);
  *ptr_out = ptr;
  *col_out = col;
  *nnz_out = nu;
}

om_mesh* om_create(int order, int pressure_order, int nv, int ne, const double* coords,
                   const int* tets, const unsigned char* dir_group, int ngroups,
                   const double* groups, int nf, const int* faces, const int* face_kind,
                   const double* face_data, const double* matp, const double* fibers) {
  om_mesh* m = (om_mesh*)xcalloc(1, sizeof(om_mesh));
  m->order = order;
  m->pres = pressure_order;
  m->nv = nv;
  m->ne = ne;
  m->nen = order == 1 ? 4 : 10;
  memcpy(m->matp, matp, 15 * sizeof(double));
  /* P2: unique edges sorted by (min, max) vertex id, numbered after vertices */
  long long* edges = NULL;
  long nedge = 0;
  if (order == 2) {
    edges = (long long*)xcalloc((long)ne * 6, sizeof(long long));
    for (int e = 0; e < ne; e++)
      for (int k = 0; k < 6; k++) {
        int a = tets[4 * e + TET_EDGE[k][0]], b = tets[4 * e + TET_EDGE[k][1]];
        edges[6L * e + k] = (long long)(a < b ? a : b) * nv + (a < b ? b : a);
      }
    qsort(edges, (long)ne * 6, sizeof(long long), cmp_ll);
    for (long i = 0; i < (long)ne * 6; i++)
      if (i == 0 || edges[i] != edges[i - 1]) edges[nedge++] = edges[i];
  }
  m->nn = nv + (int)nedge;
  /* pressure space: 1 = P1 (vertex values, Taylor-Hood), 2 = P0 (one constant
   * per element, the paper's P2-P0 twist discretisation) */
  m->np = pressure_order == 1 ? nv : (pressure_order == 2 ? ne : 0);
  m->ndof = 3L * m->nn + m->np;
  m->X = (double*)xcalloc(3L * m->nn, sizeof(double));
  memcpy(m->X, coords, 3L * nv * sizeof(double));
  for (long k = 0; k < nedge; k++) {
    int a = (int)(edges[k] / nv), b = (int)(edges[k] % nv);
    for (int i = 0; i < 3; i++) m->X[3L * (nv + k) + i] = 0.5 * (coords[3L * a + i] + coords[3L * b + i]);
  }
  m->conn = (int*)xcalloc((long)ne * m->nen, sizeof(int));
  for (int e = 0; e < ne; e++) {
    for (int a = 0; a < 4; a++) m->conn[(long)e * m->nen + a] = tets[4 * e + a];
    if (order == 2)
      for (int k = 0; k < 6; k++)
        m->conn[(long)e * m->nen + 4 + k] =
            edge_node(edges, nedge, nv, tets[4 * e + TET_EDGE[k][0]], tets[4 * e + TET_EDGE[k][1]]);
  }
  /* Dirichlet groups per node: an edge node inherits its vertices' common group */
  m->dgroup = (unsigned char*)xcalloc(m->nn, 1);
  for (int a = 0; a < nv; a++) m->dgroup[a] = dir_group ? dir_group[a] : 0;
  for (long k = 0; k < nedge; k++) {
    int a = (int)(edges[k] / nv), b = (int)(edges[k] % nv);
    if (m->dgroup[a] && m->dgroup[a] == m->dgroup[b]) m->dgroup[nv + k] = m->dgroup[a];
  }
  m->ngroups = ngroups;
  m->groups = (double*)xcalloc(8L * (ngroups > 0 ? ngroups : 1), sizeof(double));
  if (ngroups) memcpy(m->groups, groups, 8L * ngroups * sizeof(double));
  /* faces */
  m->nf = nf;
  m->fnodes = (int*)xcalloc(6L * (nf > 0 ? nf : 1), sizeof(int));
  m->fkind = (int*)xcalloc(nf > 0 ? nf : 1, sizeof(int));
  m->fdata = (double*)xcalloc(3L * (nf > 0 ? nf : 1), sizeof(double));
  for (int f = 0; f < nf; f++) {
    for (int a = 0; a < 3; a++) m->fnodes[6 * f + a] = faces[3 * f + a];
    if (order == 2)
      for (int k = 0; k < 3; k++)
        m->fnodes[6 * f + 3 + k] =
            edge_node(edges, nedge, nv, faces[3 * f + TRI_EDGE[k][0]], faces[3 * f + TRI_EDGE[k][1]]);
    m->fkind[f] = face_kind[f];
    for (int i = 0; i < 3; i++) m->fdata[3 * f + i] = face_data[3 * f + i];
  }
  if (fibers) {
    m->fib = (double*)xcalloc(9L * ne, sizeof(double));
    memcpy(m->fib, fibers, 9L * ne * sizeof(double));
  }
  free(edges);

  /* colouring: first-fit greedy, elements visited by descending
   * splitmix64(id), ties by ascending id; two elements conflict when they
   * share a vertex (equivalently, any node) */
  pri_t* pr = (pri_t*)xcalloc(ne, sizeof(pri_t));
  for (int e = 0; e < ne; e++) {
    pr[e].pri = om_splitmix64((unsigned long long)e);
    pr[e].id = e;
  }
  qsort(pr, ne, sizeof(pri_t), cmp_pri);
  int* vptr = (int*)xcalloc(nv + 1, sizeof(int));
  for (int e = 0; e < ne; e++)
    for (int a = 0; a < 4; a++) vptr[tets[4 * e + a] + 1]++;
  for (int v = 0; v < nv; v++) vptr[v + 1] += vptr[v];
  int* vel = (int*)xcalloc((long)ne * 4, sizeof(int));
  int* fill = (int*)xcalloc(nv, sizeof(int));
  for (int e = 0; e < ne; e++)
    for (int a = 0; a < 4; a++) {
      int v = tets[4 * e + a];
      vel[vptr[v] + fill[v]++] = e;
    }
  m->colors = (int*)xcalloc(ne, sizeof(int));
  for (int e = 0; e < ne; e++) m->colors[e] = -1;
  int maxc = 0;
  unsigned char* used = (unsigned char*)xcalloc(4096, 1);
  for (int t = 0; t < ne; t++) {
    int e = pr[t].id;
    memset(used, 0, 4096);
    for (int a = 0; a < 4; a++) {
      int v = tets[4 * e + a];
      for (int k = vptr[v]; k < vptr[v + 1]; k++) {
        int c = m->colors[vel[k]];
        if (c >= 0) used[c] = 1;
      }
    }
    int c = 0;
    while (used[c]) c++;
    m->colors[e] = c;
    if (c + 1 > maxc) maxc = c + 1;
  }
  m->ncolors = maxc;
  free(used);
  free(fill);
  free(vel);
  free(vptr);
  free(pr);

  /* block pattern */
  build_pattern(m->nn, m->nn, m->conn, ne, m->nen, m->nen, m->conn, m->nen, &m->row_ptr, &m->col,
                &m->nnzb);
  if (m->pres == 1)
    build_pattern(m->nn, nv, m->conn, ne, m->nen, 4, tets, 4, &m->up_ptr, &m->up_col, &m->nnz_up);
  if (m->pres == 2) {
    int* eid = (int*)xcalloc(ne, sizeof(int));
    for (int e = 0; e < ne; e++) eid[e] = e;
    build_pattern(m->nn, ne, m->conn, ne, m->nen, 1, eid, 1, &m->up_ptr, &m->up_col, &m->nnz_up);
    free(eid);
  }
  m->K = (double*)xcalloc(9 * m->nnzb, sizeof(double));
  m->B1 = (double*)xcalloc(3 * (m->nnz_up > 0 ? m->nnz_up : 1), sizeof(double));
  m->Dinv = (double*)xcalloc(9L * m->nn, sizeof(double));
  m->Sd = (double*)xcalloc(m->np > 0 ? m->np : 1, sizeof(double));
  return m;
}

static void amg_free(struct om_amg* h);

void om_destroy(om_mesh* m) {
  if (!m) return;
  free(m->X); free(m->conn); free(m->colors); free(m->row_ptr); free(m->col);
  free(m->up_ptr); free(m->up_col); free(m->dgroup); free(m->groups); free(m->fnodes);
  free(m->fkind); free(m->fdata); free(m->fib); free(m->K); free(m->B1); free(m->Dinv);
  free(m->Sd); amg_free(m->amg);
  free(m->Mm); free(m->Cd); free(m->dn); free(m->vn); free(m->an); free(m->dhat); free(m->dtil);
  free(m);
}

void om_info(const om_mesh* m, long long* out) {
  out[0] = m->nn; out[1] = m->np; out[2] = m->ndof; out[3] = m->nnzb;
  out[4] = m->nnz_up; out[5] = m->ncolors; out[6] = m->nen;
}

void om_topology(const om_mesh* m, int* conn, int* colors, int* row_ptr, int* col, double* X) {
  if (conn) memcpy(conn, m->conn, sizeof(int) * (size_t)m->ne * m->nen);
  if (colors) memcpy(colors, m->colors, sizeof(int) * (size_t)m->ne);
  if (row_ptr) memcpy(row_ptr, m->row_ptr, sizeof(int) * (size_t)(m->nn + 1));
  if (col) memcpy(col, m->col, sizeof(int) * (size_t)m->nnzb);
  if (X) memcpy(X, m->X, sizeof(double) * 3 * (size_t)m->nn);
}

void om_set_load(om_mesh* m, double load, double time) {
  m->load = load;
  m->time = time;
}

static int is_fixed(const om_mesh* m, int node, int c) {
  int g = m->dgroup[node];
  if (!g) return 0;
  unsigned mask = (unsigned)m->groups[8 * (g - 1)];
  return (mask >> c) & 1u;
}

void om_apply_dirichlet(const om_mesh* m, double* d) {
  /* prescribed d(X) = T(X) - X, T = rotation by load*angle about the axis
   * parallel to z through center, followed by load*translation */
  for (int a = 0; a < m->nn; a++) {
    int g = m->dgroup[a];
    if (!g) continue;
    const double* G = m->groups + 8 * (g - 1);
    double th = m->load * G[4];
    double x = m->X[3 * a] - G[1], y = m->X[3 * a + 1] - G[2];
    double T[3] = {G[1] + cos(th) * x - sin(th) * y + m->load * G[5],
                   G[2] + sin(th) * x + cos(th) * y + m->load * G[6],
                   m->X[3 * a + 2] + m->load * G[7]};
    for (int c = 0; c < 3; c++)
      if (is_fixed(m, a, c)) d[3L * a + c] = T[c] - m->X[3 * a + c];
  }
}

/* activation gamma(t) = Ta_peak max(sin(2 pi t / period), 0) */
static double om_gamma(const om_mesh* m) {
  if ((int)m->matp[0] != 2) return 0.0;
  double s = sin(2.0 * M_PI * m->time / m->matp[11]);
  return m->matp[10] * (s > 0.0 ? s : 0.0);
}

/* element geometry: barycentric gradients G[4][3] and volume */
static double elem_geom(const om_mesh* m, int e, double G[4][3]) {
  const int* c = m->conn + (long)e * m->nen;
  double Jm[3][3], Ji[3][3];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) Jm[i][j] = m->X[3 * c[j + 1] + i] - m->X[3 * c[0] + i];
  double det = inv3(Jm, Ji);
  /* grad lambda_{j+1} = row j of J^{-1}; grad lambda_0 = -sum */
  for (int i = 0; i < 3; i++) {
    G[0][i] = 0.0;
    for (int j = 0; j < 3; j++) {
      G[j + 1][i] = Ji[j][i];
      G[0][i] -= Ji[j][i];
    }
  }
  return det / 6.0;
}

/* face geometry: area and unit outward normal */
static double face_geom(const om_mesh* m, int f, double N[3]) {
  const int* v = m->fnodes + 6 * f;
  double a[3], b[3];
  for (int i = 0; i < 3; i++) {
    a[i] = m->X[3 * v[1] + i] - m->X[3 * v[0] + i];
    b[i] = m->X[3 * v[2] + i] - m->X[3 * v[0] + i];
  }
  double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  double ln = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int i = 0; i < 3; i++) N[i] = n[i] / ln;
  return 0.5 * ln;
}

/* per-face: consistent load vector (dead traction / pressure) and spring
 * mass-type matrix M_ab = int phi_a phi_b dA */
static int face_terms(const om_mesh* m, int f, double fvec[6][3], double M[6][6], double Ks[3][3]) {
  int nfn = m->order == 1 ? 3 : 6;
  double N[3];
  double area = face_geom(m, f, N);
  double lam[18], w[6], phi[6];
  int nq = om_tri_rule(lam, w);
  double intphi[6] = {0}, mm[6][6];
  memset(mm, 0, sizeof(mm));
  for (int q = 0; q < nq; q++) {
    tri_shape(m->order, lam + 3 * q, phi);
    for (int a = 0; a < nfn; a++) {
      intphi[a] += w[q] * area * phi[a];
      for (int b = 0; b < nfn; b++) mm[a][b] += w[q] * area * phi[a] * phi[b];
    }
  }
  int kind = m->fkind[f];
  const double* fd = m->fdata + 3 * f;
  double t[3] = {0, 0, 0};
  if (kind == 0)
    for (int i = 0; i < 3; i++) t[i] = m->load * fd[i];
  else if (kind == 1)
    for (int i = 0; i < 3; i++) t[i] = -m->load * fd[0] * N[i];
  for (int a = 0; a < nfn; a++)
    for (int i = 0; i < 3; i++) fvec[a][i] = t[i] * intphi[a];
  memcpy(M, mm, sizeof(mm));
  memset(Ks, 0, 9 * sizeof(double));
  if (kind == 2)
    for (int i = 0; i < 3; i++)
      for (int k = 0; k < 3; k++)
        Ks[i][k] = fd[0] * N[i] * N[k] + fd[1] * ((i == k) - N[i] * N[k]);
  return nfn;
}

/* pressure space of element e: the number of local pressure values, their
 * global indices and their shape functions at barycentric point lamq
 * (P1: the 4 vertices with the barycentric shapes; P0: the element's one
 * constant) */
static int p_count(const om_mesh* m) { return m->pres == 2 ? 1 : 4; }
static int p_index(const om_mesh* m, int e, const int* c, int v) { return m->pres == 2 ? e : c[v]; }
static double p_shape(const om_mesh* m, const double* lamq, int v) { return m->pres == 2 ? 1.0 : lamq[v]; }

static long find_block(const int* ptr, const int* col, int row, int c);

/* ======================================================================
 * Elastodynamics and follower pressure (the paper's momentum equation with
 * its inertia term, Eq. "momentum strong", the Robin condition of the
 * epicardium with its dashpots, Eq. "bc epi", and a pressure that follows
 * the deformed surface).  Readings (the paper names no time integrator and
 * no density):
 *   - density rho per unit reference volume (the printed equation has
 *     rho = 1); consistent mass M_ab = rho int N_a N_b I dV, integrated
 *     exactly (products of the barycentric shape functions, int over the tet
 *     of l1^a l2^b l3^c l4^d = 6 V a! b! c! d! / (a + b + c + d + 3)!);
 *   - Newmark average acceleration (beta = 1/4, gamma = 1/2: trapezoidal,
 *     unconditionally stable, energy conserving for a linear undamped
 *     system): step n -> n+1 solves R(d) + M a(d) + C v(d) = 0 with
 *     a = 4/dt^2 (d - dhat), v = 2/dt (d - dtil),
 *     dhat = d_n + dt v_n + dt^2/4 a_n, dtil = d_n + dt/2 v_n;
 *     tangent K + 4/dt^2 M + 2/dt C;
 *   - dashpots: face kind 4 with data (c_perp, c_par): damping traction
 *     -(c_perp N N^T + c_par (I - N N^T)) v on the reference face (N the
 *     reference normal, like the springs of kind 2);
 *   - follower pressure: face kind 3 with data (p): traction -p n da on the
 *     deformed face, i.e. nodal forces -p int N_a (x_xi x x_eta) dxi deta
 *     over the reference triangle (exact with the degree-4 rule for P1 and
 *     P2 faces); its tangent is not symmetric, and it has no potential, so
 *     om_energy leaves it out.
 * ====================================================================== */
/* d N_a / d lambda_c of the triangle shape functions (face-local nodes) */
static void tri_dshape(int order, const double* lam, double dN[6][3]) {
  memset(dN, 0, sizeof(double) * 18);
  if (order == 1) {
    for (int a = 0; a < 3; a++) dN[a][a] = 1.0;
    return;
  }
  for (int a = 0; a < 3; a++) dN[a][a] = 4.0 * lam[a] - 1.0;
  for (int e = 0; e < 3; e++) {
    int i = TRI_EDGE[e][0], j = TRI_EDGE[e][1];
    dN[3 + e][i] = 4.0 * lam[j];
    dN[3 + e][j] = 4.0 * lam[i];
  }
}

/* follower loads of face f at displacement d: nodal residual rf (R += rf)
 * and, when Kf != NULL, its derivative Kf[a][b][i][k] = d rf_a,i / d d_b,k.
 * Kind 3, follower pressure: rf_a = p int N_a n with n = x_xi x x_eta.
 * Kind 5, traction per unit deformed area (the Cook load "in the deformed
 * configuration"): rf_a = -int N_a t |n|, whose derivative along the
 * displacement of node b is -int N_a t (x) g_b with g_b = d|n|/d x_b =
 * Nx_b (x_eta x n/|n|) + Ne_b (n/|n| x x_xi). */
static int follower_terms(const om_mesh* m, int f, const double* d, double rf[6][3], double Kf[6][6][3][3]) {
  int nfn = m->order == 1 ? 3 : 6;
  const int* v = m->fnodes + 6 * f;
  const int kind = m->fkind[f];
  double p = m->load * m->fdata[3 * f];
  double tr[3] = {m->load * m->fdata[3 * f], m->load * m->fdata[3 * f + 1], m->load * m->fdata[3 * f + 2]};
  double x[6][3];
  for (int a = 0; a < nfn; a++)
    for (int i = 0; i < 3; i++) x[a][i] = m->X[3 * v[a] + i] + d[3L * v[a] + i];
  double lam[18], w[6], N[6], dN[6][3];
  int nq = om_tri_rule(lam, w);
  memset(rf, 0, sizeof(double) * 18);
  if (Kf) memset(Kf, 0, sizeof(double) * 324);
  for (int q = 0; q < nq; q++) {
    tri_shape(m->order, lam + 3 * q, N);
    tri_dshape(m->order, lam + 3 * q, dN);
    /* x(xi, eta) with lambda = (1 - xi - eta, xi, eta): d/dxi = d/dl2 - d/dl1, d/deta = d/dl3 - d/dl1 */
    double Nx[6], Ne[6], xs[3] = {0, 0, 0}, xe[3] = {0, 0, 0};
    for (int a = 0; a < nfn; a++) {
      Nx[a] = dN[a][1] - dN[a][0];
      Ne[a] = dN[a][2] - dN[a][0];
      for (int i = 0; i < 3; i++) {
        xs[i] += Nx[a] * x[a][i];
        xe[i] += Ne[a] * x[a][i];
      }
    }
    double n[3] = {xs[1] * xe[2] - xs[2] * xe[1], xs[2] * xe[0] - xs[0] * xe[2], xs[0] * xe[1] - xs[1] * xe[0]};
    if (kind == 5) {
      double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      double nh[3] = {n[0] / nl, n[1] / nl, n[2] / nl};
      double wt = 0.5 * w[q]; /* reference triangle area 1/2 */
      for (int a = 0; a < nfn; a++)
        for (int i = 0; i < 3; i++) rf[a][i] -= wt * N[a] * tr[i] * nl;
      if (!Kf) continue;
      /* x_eta x nh and nh x x_xi */
      double u1[3] = {xe[1] * nh[2] - xe[2] * nh[1], xe[2] * nh[0] - xe[0] * nh[2], xe[0] * nh[1] - xe[1] * nh[0]};
      double u2[3] = {nh[1] * xs[2] - nh[2] * xs[1], nh[2] * xs[0] - nh[0] * xs[2], nh[0] * xs[1] - nh[1] * xs[0]};
      for (int a = 0; a < nfn; a++)
        for (int b = 0; b < nfn; b++)
          for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) Kf[a][b][i][k] -= wt * N[a] * tr[i] * (Nx[b] * u1[k] + Ne[b] * u2[k]);
      continue;
    }
    double wq = 0.5 * w[q] * p; /* reference triangle area 1/2 */
    for (int a = 0; a < nfn; a++)
      for (int i = 0; i < 3; i++) rf[a][i] += wq * N[a] * n[i];
    if (!Kf) continue;
    /* d n = Nx_b (delta x xe) + Ne_b (xs x delta) */
    for (int a = 0; a < nfn; a++)
      for (int b = 0; b < nfn; b++)
        for (int i = 0; i < 3; i++)
          for (int k = 0; k < 3; k++) {
            double dk[3] = {0, 0, 0};
            dk[k] = 1.0;
            double c1[3] = {dk[1] * xe[2] - dk[2] * xe[1], dk[2] * xe[0] - dk[0] * xe[2], dk[0] * xe[1] - dk[1] * xe[0]};
            double c2[3] = {xs[1] * dk[2] - xs[2] * dk[1], xs[2] * dk[0] - xs[0] * dk[2], xs[0] * dk[1] - xs[1] * dk[0]};
            Kf[a][b][i][k] += wq * N[a] * (Nx[b] * c1[i] + Ne[b] * c2[i]);
          }
  }
  return nfn;
}

/* exact int over a tet of prod of barycentric powers, divided by the volume */
static double bary_moment(const int* e) {
  double num = 6.0;
  int s = 3;
  for (int i = 0; i < 4; i++) {
    for (int k = 2; k <= e[i]; k++) num *= k;
    s += e[i];
  }
  double den = 1.0;
  for (int k = 2; k <= s; k++) den *= k;
  return num / den;
}

/* shape function a of the tet as monomials in the barycentrics: up to 2
 * terms (coefficient, exponents) */
static int tet_shape_poly(int order, int a, double* coef, int (*ex)[4]) {
  memset(ex, 0, sizeof(int) * 8);
  if (order == 1) {
    coef[0] = 1.0;
    ex[0][a] = 1;
    return 1;
  }
  if (a < 4) { /* l_a (2 l_a - 1) */
    coef[0] = 2.0;
    ex[0][a] = 2;
    coef[1] = -1.0;
    ex[1][a] = 1;
    return 2;
  }
  coef[0] = 4.0;
  ex[0][TET_EDGE[a - 4][0]] = 1;
  ex[0][TET_EDGE[a - 4][1]] = 1;
  return 1;
}

void om_set_dynamics(om_mesh* m, double rho, double dt) {
  free(m->Mm); free(m->Cd); free(m->dn); free(m->vn); free(m->an); free(m->dhat); free(m->dtil);
  m->Mm = m->Cd = m->dn = m->vn = m->an = m->dhat = m->dtil = NULL;
  m->dyn = rho > 0.0 && dt > 0.0;
  if (!m->dyn) return;
  m->rho = rho;
  m->dt = dt;
  m->Mm = (double*)xcalloc(m->nnzb, sizeof(double));
  m->Cd = (double*)xcalloc(9 * m->nnzb, sizeof(double));
  long n3 = 3L * m->nn;
  m->dn = (double*)xcalloc(n3, sizeof(double));
  m->vn = (double*)xcalloc(n3, sizeof(double));
  m->an = (double*)xcalloc(n3, sizeof(double));
  m->dhat = (double*)xcalloc(n3, sizeof(double));
  m->dtil = (double*)xcalloc(n3, sizeof(double));
  int nen = m->nen;
  for (int e = 0; e < m->ne; e++) {
    double G[4][3];
    double vol = elem_geom(m, e, G);
    const int* c = m->conn + (long)e * nen;
    for (int a = 0; a < nen; a++) {
      double ca[2];
      int ea[2][4];
      int na = tet_shape_poly(m->order, a, ca, ea);
      for (int b = 0; b < nen; b++) {
        double cb[2];
        int eb[2][4];
        int nb = tet_shape_poly(m->order, b, cb, eb);
        double s = 0.0;
        for (int i = 0; i < na; i++)
          for (int j = 0; j < nb; j++) {
            int ex[4];
            for (int k = 0; k < 4; k++) ex[k] = ea[i][k] + eb[j][k];
            s += ca[i] * cb[j] * bary_moment(ex);
          }
        m->Mm[find_block(m->row_ptr, m->col, c[a], c[b])] += rho * vol * s;
      }
    }
  }
  for (int f = 0; f < m->nf; f++) {
    if (m->fkind[f] != 4) continue;
    double fv[6][3], M[6][6], Ks[3][3], N[3];
    int nfn = face_terms(m, f, fv, M, Ks);
    face_geom(m, f, N);
    const double* fd = m->fdata + 3 * f;
    double Cs[3][3];
    for (int i = 0; i < 3; i++)
      for (int k = 0; k < 3; k++) Cs[i][k] = fd[0] * N[i] * N[k] + fd[1] * ((i == k) - N[i] * N[k]);
    const int* v = m->fnodes + 6 * f;
    for (int a = 0; a < nfn; a++)
      for (int b = 0; b < nfn; b++) {
        long k = find_block(m->row_ptr, m->col, v[a], v[b]);
        for (int i = 0; i < 3; i++)
          for (int kk = 0; kk < 3; kk++) m->Cd[9 * k + 3 * i + kk] += M[a][b] * Cs[i][kk];
      }
  }
}

/* state of the time integration (nullable: zero); the predictors of the next step */
void om_dynamics_set(om_mesh* m, const double* d, const double* v, const double* a) {
  if (!m->dyn) return;
  long n3 = 3L * m->nn;
  double dt = m->dt;
  for (long i = 0; i < n3; i++) {
    m->dn[i] = d ? d[i] : 0.0;
    m->vn[i] = v ? v[i] : 0.0;
    m->an[i] = a ? a[i] : 0.0;
    m->dhat[i] = m->dn[i] + dt * m->vn[i] + 0.25 * dt * dt * m->an[i];
    m->dtil[i] = m->dn[i] + 0.5 * dt * m->vn[i];
  }
}

/* Newmark update from the converged d of the step: v, a of the new state */
void om_dynamics_advance(om_mesh* m, const double* d) {
  if (!m->dyn) return;
  long n3 = 3L * m->nn;
  double dt = m->dt;
  double* v = (double*)xcalloc(n3, sizeof(double));
  double* a = (double*)xcalloc(n3, sizeof(double));
  for (long i = 0; i < n3; i++) {
    a[i] = 4.0 / (dt * dt) * (d[i] - m->dhat[i]);
    v[i] = 2.0 / dt * (d[i] - m->dtil[i]);
  }
  om_dynamics_set(m, d, v, a);
  free(v);
  free(a);
}

void om_dynamics_get(const om_mesh* m, double* v, double* a) {
  if (!m->dyn) return;
  if (v) memcpy(v, m->vn, sizeof(double) * 3 * (size_t)m->nn);
  if (a) memcpy(a, m->an, sizeof(double) * 3 * (size_t)m->nn);
}

/* r += M a(d) + C v(d) (displacement rows) */
static void dyn_residual(const om_mesh* m, const double* d, double* r) {
  double cm = 4.0 / (m->dt * m->dt), cc = 2.0 / m->dt;
  for (int a = 0; a < m->nn; a++)
    for (int k = m->row_ptr[a]; k < m->row_ptr[a + 1]; k++) {
      int b = m->col[k];
      for (int i = 0; i < 3; i++) {
        double s = cm * m->Mm[k] * (d[3L * b + i] - m->dhat[3L * b + i]);
        for (int j = 0; j < 3; j++) s += cc * m->Cd[9L * k + 3 * i + j] * (d[3L * b + j] - m->dtil[3L * b + j]);
        r[3L * a + i] += s;
      }
    }
}

double om_residual(om_mesh* m, const double* d, double* r) {
  memset(r, 0, sizeof(double) * m->ndof);
  int nen = m->nen;
  double gam = om_gamma(m);
  double lam[16], w[4], N[10], dN[10][3], G[4][3];
  int nq = om_tet_rule(m->order, lam, w);
  for (int e = 0; e < m->ne; e++) {
    const int* c = m->conn + (long)e * nen;
    double vol = elem_geom(m, e, G);
    for (int q = 0; q < nq; q++) {
      tet_shape(m->order, lam + 4 * q, N);
      tet_grad(m->order, lam + 4 * q, G, dN);
      double F[9];
      for (int i = 0; i < 3; i++)
        for (int J = 0; J < 3; J++) {
          double s = (i == J);
          for (int a = 0; a < nen; a++) s += d[3L * c[a] + i] * dN[a][J];
          F[IDX(i, J)] = s;
        }
      double p = 0.0;
      if (m->pres)
        for (int a = 0; a < p_count(m); a++) p += d[3L * m->nn + p_index(m, e, c, a)] * p_shape(m, lam + 4 * q, a);
      double P[9];
      om_material(m->matp, F, m->fib ? m->fib + 9L * e : NULL, gam, p, NULL, P, NULL, NULL);
      double wq = w[q] * vol;
      for (int a = 0; a < nen; a++)
        for (int i = 0; i < 3; i++) {
          double s = 0.0;
          for (int J = 0; J < 3; J++) s += P[IDX(i, J)] * dN[a][J];
          r[3L * c[a] + i] += wq * s;
        }
      if (m->pres) {
        double det, H[9];
        cofactor_H(F, &det, H);
        /* R_p = -int (J - 1) q_h */
        for (int a = 0; a < p_count(m); a++)
          r[3L * m->nn + p_index(m, e, c, a)] -= wq * (det - 1.0) * p_shape(m, lam + 4 * q, a);
      }
    }
  }
  /* surface terms: R -= external load; R += springs K_s d */
  for (int f = 0; f < m->nf; f++) {
    double fv[6][3], M[6][6], Ks[3][3];
    int nfn = face_terms(m, f, fv, M, Ks);
    const int* v = m->fnodes + 6 * f;
    for (int a = 0; a < nfn; a++)
      for (int i = 0; i < 3; i++) {
        double s = -fv[a][i];
        for (int b = 0; b < nfn; b++)
          for (int k = 0; k < 3; k++) s += M[a][b] * Ks[i][k] * d[3L * v[b] + k];
        r[3L * v[a] + i] += s;
      }
  }
  /* follower loads: R += p int N_a n da, or R -= int N_a t |n|, on the deformed face */
  for (int f = 0; f < m->nf; f++) {
    if (m->fkind[f] != 3 && m->fkind[f] != 5) continue;
    double rf[6][3];
    int nfn = follower_terms(m, f, d, rf, NULL);
    const int* v = m->fnodes + 6 * f;
    for (int a = 0; a < nfn; a++)
      for (int i = 0; i < 3; i++) r[3L * v[a] + i] += rf[a][i];
  }
  if (m->dyn) dyn_residual(m, d, r);
  for (int a = 0; a < m->nn; a++)
    for (int c = 0; c < 3; c++)
      if (is_fixed(m, a, c)) r[3L * a + c] = 0.0;
  return nrm2(r, m->ndof);
}

double om_energy(om_mesh* m, const double* d) {
  int nen = m->nen;
  double gam = om_gamma(m);
  double lam[16], w[4], N[10], dN[10][3], G[4][3];
  int nq = om_tet_rule(m->order, lam, w);
  double Pi = 0.0;
  for (int e = 0; e < m->ne; e++) {
    const int* c = m->conn + (long)e * nen;
    double vol = elem_geom(m, e, G);
    for (int q = 0; q < nq; q++) {
      tet_shape(m->order, lam + 4 * q, N);
      tet_grad(m->order, lam + 4 * q, G, dN);
      double F[9];
      for (int i = 0; i < 3; i++)
        for (int J = 0; J < 3; J++) {
          double s = (i == J);
          for (int a = 0; a < nen; a++) s += d[3L * c[a] + i] * dN[a][J];
          F[IDX(i, J)] = s;
        }
      double p = 0.0;
      if (m->pres)
        for (int a = 0; a < p_count(m); a++) p += d[3L * m->nn + p_index(m, e, c, a)] * p_shape(m, lam + 4 * q, a);
      double psi, P[9];
      om_material(m->matp, F, m->fib ? m->fib + 9L * e : NULL, gam, p, &psi, P, NULL, NULL);
      Pi += w[q] * vol * psi;
    }
  }
  for (int f = 0; f < m->nf; f++) {
    double fv[6][3], M[6][6], Ks[3][3];
    int nfn = face_terms(m, f, fv, M, Ks);
    const int* v = m->fnodes + 6 * f;
    for (int a = 0; a < nfn; a++)
      for (int i = 0; i < 3; i++) {
        Pi -= fv[a][i] * d[3L * v[a] + i];
        for (int b = 0; b < nfn; b++)
          for (int k = 0; k < 3; k++)
            Pi += 0.5 * M[a][b] * d[3L * v[a] + i] * Ks[i][k] * d[3L * v[b] + k];
      }
  }
  /* Newmark step functional: + 2/dt^2 (d - dhat)^T M (d - dhat) + 1/dt (d - dtil)^T C (d - dtil)
   * (its gradient is the step's M a + C v); the follower pressure has no potential */
  if (m->dyn) {
    double cm = 2.0 / (m->dt * m->dt), cc = 1.0 / m->dt;
    for (int a = 0; a < m->nn; a++)
      for (int k = m->row_ptr[a]; k < m->row_ptr[a + 1]; k++) {
        int b = m->col[k];
        for (int i = 0; i < 3; i++) {
          Pi += cm * (d[3L * a + i] - m->dhat[3L * a + i]) * m->Mm[k] * (d[3L * b + i] - m->dhat[3L * b + i]);
          for (int j = 0; j < 3; j++)
            Pi += cc * (d[3L * a + i] - m->dtil[3L * a + i]) * m->Cd[9L * k + 3 * i + j] *
                  (d[3L * b + j] - m->dtil[3L * b + j]);
        }
      }
  }
  return Pi;
}

static long find_block(const int* ptr, const int* col, int row, int c) {
  for (int k = ptr[row]; k < ptr[row + 1]; k++)
    if (col[k] == c) return k;
  abort();
}

/* ======================================================================
 * Algebraic multigrid preconditioner: smoothed aggregation on the nodal
 * blocks.  The paper preconditions its Krylov solves with algebraic
 * multigrid on blocks of size 3 (BoomerAMG with bs = 3, Section "Test
 * problems and solvers details" and Appendix A) but does not describe the
 * tool, so this is a plain smoothed-aggregation V-cycle of that class; each
 * choice is a stated reading:
 *   - graph of level l: the block pattern of A_l without nodes whose
 *     components are all absent (Dirichlet at level 0); no strength filter;
 *   - aggregation: roots = greedy maximal distance-2 independent set in
 *     descending splitmix64(node) priority, ties by id; phase 1: a root and
 *     its graph neighbours; phase 2: every other node joins the aggregate of
 *     its smallest-id phase-1 neighbour; aggregates numbered by root id;
 *   - near null space: the six rigid motions of linear elasticity (three
 *     translations, rotations (-y, x, 0), (0, -z, y), (z, 0, -x) at the node
 *     coordinates), zero at absent components; tentative prolongator per
 *     aggregate by modified Gram-Schmidt QR of its rows of the near null
 *     space (nodes ascending): B_a = Q_a R_a, T = Q, coarse near null space
 *     R; a column left with norm <= 1e-8 of its original norm is dropped
 *     (zero column of Q and R) and that coarse component is absent; coarse
 *     nodes carry 6 components;
 *   - smoothed prolongator P = (I - omega D^{-1} A) T with D the block
 *     diagonal, omega = 4 / (3 rho), rho = spectral radius of D^{-1} A
 *     estimated by 15 power steps from x_k = u(splitmix64(k)) - 1/2,
 *     u(h) = (h >> 11) 2^-53;
 *   - Galerkin coarse operator A_{l+1} = P^T A_l P, absent components with a
 *     unit diagonal;
 *   - smoother: Chebyshev of degree 2 in D^{-1} A on [rho/30, 1.1 rho],
 *     before and after the coarse correction;
 *   - coarsest level (<= 16 nodes, or aggregation that no longer coarsens
 *     by 10 %): exact solve with the inverse from Gauss-Jordan elimination
 *     with partial pivoting.
 * The V-cycle is a fixed linear operator, so right-preconditioned GMRES
 * and the BFGS initial inverse Hessian use it unchanged.
 * ====================================================================== */
#define OM_AMG_MAXLEV 12
#define OM_AMG_COARSE 16
#define OM_AMG_NS 6

typedef struct {
  int n, b;              /* block rows, components per node (3 at level 0, 6 below) */
  int *ptr, *col;        /* A_l pattern */
  double* val;           /* A_l [nnz][b*b] row-major blocks (level 0: the tangent) */
  double* dinv;          /* [n][b*b] inverse diagonal blocks */
  unsigned char* absent; /* [n] bit c: component c absent */
  double* ns;            /* [n*b][6] near null space */
  double rho;
  int nc;                /* aggregates */
  int* agg;              /* [n], -1 none */
  int *pptr, *pcol;      /* P (and T): n x nc, blocks b x 6 */
  double *pval, *tval;
  double* inv;           /* coarsest: dense (b n)^2 inverse */
} om_amg_level;

struct om_amg {
  int nlev;
  om_amg_level lev[OM_AMG_MAXLEV];
};

static double om_u01(unsigned long long h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

/* y = A x for a block-CSR matrix with br x bc blocks */
static void bsr_mv(int n, int br, int bc, const int* ptr, const int* col, const double* val, const double* x,
                   double* y) {
  for (int a = 0; a < n; a++) {
    double s[OM_AMG_NS] = {0};
    for (int k = ptr[a]; k < ptr[a + 1]; k++)
      for (int i = 0; i < br; i++)
        for (int j = 0; j < bc; j++) s[i] += val[(long)br * bc * k + bc * i + j] * x[(long)bc * col[k] + j];
    for (int i = 0; i < br; i++) y[(long)br * a + i] = s[i];
  }
}

/* y = A^T x (A: n block rows of br x bc blocks, nc block columns) */
static void bsr_tmv(int n, int nc, int br, int bc, const int* ptr, const int* col, const double* val,
                    const double* x, double* y) {
  for (long i = 0; i < (long)bc * nc; i++) y[i] = 0.0;
  for (int a = 0; a < n; a++)
    for (int k = ptr[a]; k < ptr[a + 1]; k++)
      for (int i = 0; i < br; i++)
        for (int j = 0; j < bc; j++)
          y[(long)bc * col[k] + j] += val[(long)br * bc * k + bc * i + j] * x[(long)br * a + i];
}

/* inverse of a dense N x N matrix (row-major) by Gauss-Jordan elimination
 * with partial pivoting */
static void gauss_jordan_inverse(int N, const double* Ain, double* I) {
  double* A = (double*)xcalloc((size_t)N * N, sizeof(double));
  memcpy(A, Ain, sizeof(double) * (size_t)N * N);
  for (size_t i = 0; i < (size_t)N * N; i++) I[i] = 0.0;
  for (int i = 0; i < N; i++) I[(size_t)i * N + i] = 1.0;
  for (int c = 0; c < N; c++) {
    int p = c;
    for (int r = c + 1; r < N; r++)
      if (fabs(A[(size_t)r * N + c]) > fabs(A[(size_t)p * N + c])) p = r;
    if (p != c)
      for (int j = 0; j < N; j++) {
        double t = A[(size_t)c * N + j];
        A[(size_t)c * N + j] = A[(size_t)p * N + j];
        A[(size_t)p * N + j] = t;
        t = I[(size_t)c * N + j];
        I[(size_t)c * N + j] = I[(size_t)p * N + j];
        I[(size_t)p * N + j] = t;
      }
    double piv = A[(size_t)c * N + c];
    for (int j = 0; j < N; j++) {
      A[(size_t)c * N + j] /= piv;
      I[(size_t)c * N + j] /= piv;
    }
    for (int r = 0; r < N; r++) {
      if (r == c) continue;
      double f = A[(size_t)r * N + c];
      if (f == 0.0) continue;
      for (int j = 0; j < N; j++) {
        A[(size_t)r * N + j] -= f * A[(size_t)c * N + j];
        I[(size_t)r * N + j] -= f * I[(size_t)c * N + j];
      }
    }
  }
  free(A);
}

static void amg_block_dinv(om_amg_level* L) {
  int b = L->b;
  L->dinv = (double*)xcalloc((size_t)b * b * (L->n > 0 ? L->n : 1), sizeof(double));
  for (int a = 0; a < L->n; a++) {
    long k = find_block(L->ptr, L->col, a, a);
    gauss_jordan_inverse(b, L->val + (long)b * b * k, L->dinv + (long)b * b * a);
  }
}

static void amg_apply_dinv(const om_amg_level* L, const double* r, double* z) {
  int b = L->b;
  for (int a = 0; a < L->n; a++)
    for (int i = 0; i < b; i++) {
      double s = 0.0;
      for (int j = 0; j < b; j++) s += L->dinv[(long)b * b * a + b * i + j] * r[(long)b * a + j];
      z[(long)b * a + i] = s;
    }
}

/* spectral radius of D^{-1} A by power steps */
static double amg_rho(const om_amg_level* L) {
  long N = (long)L->b * L->n;
  double* x = (double*)xcalloc(N, sizeof(double));
  double* t = (double*)xcalloc(N, sizeof(double));
  double* y = (double*)xcalloc(N, sizeof(double));
  for (long i = 0; i < N; i++) x[i] = om_u01(om_splitmix64((unsigned long long)i)) - 0.5;
  double rho = 0.0;
  for (int it = 0; it < 15; it++) {
    bsr_mv(L->n, L->b, L->b, L->ptr, L->col, L->val, x, t);
    amg_apply_dinv(L, t, y);
    double nx = nrm2(x, N), ny = nrm2(y, N);
    rho = ny / nx;
    for (long i = 0; i < N; i++) x[i] = y[i] / ny;
  }
  free(x); free(t); free(y);
  return rho;
}

static int node_priority_cmp(const void* a, const void* b) {
  const unsigned long long* x = (const unsigned long long*)a;
  const unsigned long long* y = (const unsigned long long*)b;
  if (x[0] != y[0]) return x[0] > y[0] ? -1 : 1; /* descending hash */
  return x[1] < y[1] ? -1 : (x[1] > y[1]);       /* ascending id */
}

static int all_absent(const om_amg_level* L, int i) { return L->absent[i] == (unsigned char)((1u << L->b) - 1u); }

/* aggregation of level L (fills agg, nc) */
static void amg_aggregate(om_amg_level* L) {
  int n = L->n;
  int* root_of = (int*)xcalloc(n > 0 ? n : 1, sizeof(int)); /* phase-1 root, -1 none */
  unsigned long long* ord = (unsigned long long*)xcalloc(2L * (n > 0 ? n : 1), sizeof(unsigned long long));
  for (int i = 0; i < n; i++) {
    ord[2 * i] = om_splitmix64((unsigned long long)i);
    ord[2 * i + 1] = (unsigned long long)i;
    root_of[i] = -1;
  }
  qsort(ord, n, 2 * sizeof(unsigned long long), node_priority_cmp);
  for (int q = 0; q < n; q++) { /* phase 1 in priority order */
    int i = (int)ord[2 * q + 1];
    if (all_absent(L, i) || root_of[i] >= 0) continue;
    int blocked = 0;
    for (int k = L->ptr[i]; k < L->ptr[i + 1] && !blocked; k++) {
      int j = L->col[k];
      if (j != i && !all_absent(L, j) && root_of[j] >= 0) blocked = 1;
    }
    if (blocked) continue;
    for (int k = L->ptr[i]; k < L->ptr[i + 1]; k++)
      if (!all_absent(L, L->col[k])) root_of[L->col[k]] = i;
    root_of[i] = i;
  }
  int* id_of = (int*)xcalloc(n > 0 ? n : 1, sizeof(int)); /* aggregate of each root, roots ascending */
  int nc = 0;
  for (int i = 0; i < n; i++) id_of[i] = root_of[i] == i ? nc++ : -1;
  L->agg = (int*)xcalloc(n > 0 ? n : 1, sizeof(int));
  for (int i = 0; i < n; i++) L->agg[i] = root_of[i] >= 0 ? id_of[root_of[i]] : -1;
  for (int i = 0; i < n; i++) { /* phase 2 */
    if (all_absent(L, i) || root_of[i] >= 0) continue;
    for (int k = L->ptr[i]; k < L->ptr[i + 1]; k++) {
      int j = L->col[k];
      if (j != i && root_of[j] >= 0) {
        L->agg[i] = id_of[root_of[j]];
        break;
      }
    }
  }
  L->nc = nc;
  free(root_of); free(ord); free(id_of);
}

static int cmp_int(const void* a, const void* b) {
  int x = *(const int*)a, y = *(const int*)b;
  return (x > y) - (x < y);
}

/* append c to a growing int array */
static void push_int(int** arr, long* len, long* cap, int c) {
  if (*len == *cap) {
    *cap = 2 * *cap + 16;
    *arr = (int*)realloc(*arr, (size_t)*cap * sizeof(int));
    if (!*arr) abort();
  }
  (*arr)[(*len)++] = c;
}

/* tentative prolongator T, smoothed prolongator P and coarse level
 * C: A_c = P^T A P */
static void amg_coarsen(om_amg_level* L, om_amg_level* C) {
  const int n = L->n, nc = L->nc, b = L->b, K = OM_AMG_NS;
  const int bb = b * K; /* P block size */
  /* members of every aggregate, ascending */
  int* mptr = (int*)xcalloc(nc + 1, sizeof(int));
  for (int i = 0; i < n; i++)
    if (L->agg[i] >= 0) mptr[L->agg[i] + 1]++;
  for (int a = 0; a < nc; a++) mptr[a + 1] += mptr[a];
  int* mem = (int*)xcalloc(mptr[nc] > 0 ? mptr[nc] : 1, sizeof(int));
  int* fill = (int*)xcalloc(nc > 0 ? nc : 1, sizeof(int));
  for (int i = 0; i < n; i++)
    if (L->agg[i] >= 0) mem[mptr[L->agg[i]] + fill[L->agg[i]]++] = i;
  /* QR per aggregate: T rows (tq[i][b][K]) and coarse near null space */
  double* tq = (double*)xcalloc((size_t)n * bb + 1, sizeof(double));
  C->n = nc;
  C->b = K;
  C->ns = (double*)xcalloc((size_t)nc * K * K + 1, sizeof(double));
  C->absent = (unsigned char*)xcalloc(nc > 0 ? nc : 1, 1);
  for (int a = 0; a < nc; a++) {
    int m = mptr[a + 1] - mptr[a];
    int R = m * b;
    double* Q = (double*)xcalloc((size_t)R * K, sizeof(double)); /* column-major R x K */
    for (int c = 0; c < K; c++)
      for (int s = 0; s < m; s++)
        for (int i = 0; i < b; i++) Q[(size_t)c * R + s * b + i] = L->ns[((size_t)mem[mptr[a] + s] * b + i) * K + c];
    double* Rm = C->ns + (size_t)a * K * K; /* R_a, row-major K x K */
    for (int c = 0; c < K; c++) {
      double* v = Q + (size_t)c * R;
      double n0 = nrm2(v, R);
      for (int p = 0; p < c; p++) { /* modified Gram-Schmidt */
        double r = dot(Q + (size_t)p * R, v, R);
        Rm[p * K + c] = r;
        for (int t = 0; t < R; t++) v[t] -= r * Q[(size_t)p * R + t];
      }
      double nv = nrm2(v, R);
      if (n0 == 0.0 || nv <= 1e-8 * n0) {
        for (int t = 0; t < R; t++) v[t] = 0.0;
        Rm[c * K + c] = 0.0;
        C->absent[a] |= (unsigned char)(1u << c);
      } else {
        for (int t = 0; t < R; t++) v[t] /= nv;
        Rm[c * K + c] = nv;
      }
    }
    for (int s = 0; s < m; s++)
      for (int i = 0; i < b; i++)
        for (int c = 0; c < K; c++) tq[((size_t)mem[mptr[a] + s] * b + i) * K + c] = Q[(size_t)c * R + s * b + i];
    free(Q);
  }
  /* pattern of P (= pattern of T widened by one graph step): row i gets the
   * aggregates of its graph neighbours */
  int* mark = (int*)xcalloc(nc > 0 ? nc : 1, sizeof(int));
  for (int a = 0; a < nc; a++) mark[a] = -1;
  L->pptr = (int*)xcalloc(n + 1, sizeof(int));
  long cap = 0, nnz = 0;
  L->pcol = NULL;
  for (int i = 0; i < n; i++) {
    long start = nnz;
    if (!all_absent(L, i))
      for (int k = L->ptr[i]; k < L->ptr[i + 1]; k++) {
        int a = L->agg[L->col[k]];
        if (a >= 0 && mark[a] != i) {
          mark[a] = i;
          push_int(&L->pcol, &nnz, &cap, a);
        }
      }
    qsort(L->pcol + start, nnz - start, sizeof(int), cmp_int);
    L->pptr[i + 1] = (int)nnz;
  }
  if (!L->pcol) L->pcol = (int*)xcalloc(1, sizeof(int));
  L->pval = (double*)xcalloc((size_t)bb * nnz + 1, sizeof(double));
  L->tval = (double*)xcalloc((size_t)bb * nnz + 1, sizeof(double));
  const double omega = 4.0 / (3.0 * L->rho);
  for (int i = 0; i < n; i++) {
    if (all_absent(L, i)) continue;
    if (L->agg[i] >= 0) { /* T block of node i */
      long q = find_block(L->pptr, L->pcol, i, L->agg[i]);
      for (int t = 0; t < bb; t++) {
        L->tval[(size_t)bb * q + t] = tq[(size_t)i * bb + t];
        L->pval[(size_t)bb * q + t] += tq[(size_t)i * bb + t];
      }
    }
    for (int k = L->ptr[i]; k < L->ptr[i + 1]; k++) { /* - omega D_i^{-1} A_ij T_j */
      int j = L->col[k], a = L->agg[j];
      if (a < 0) continue;
      long q = find_block(L->pptr, L->pcol, i, a);
      double DA[OM_AMG_NS * OM_AMG_NS];
      for (int r = 0; r < b; r++)
        for (int c = 0; c < b; c++) {
          double s = 0.0;
          for (int l = 0; l < b; l++) s += L->dinv[(size_t)b * b * i + b * r + l] * L->val[(size_t)b * b * k + b * l + c];
          DA[b * r + c] = s;
        }
      for (int r = 0; r < b; r++)
        for (int c = 0; c < K; c++) {
          double s = 0.0;
          for (int l = 0; l < b; l++) s += DA[b * r + l] * tq[((size_t)j * b + l) * K + c];
          L->pval[(size_t)bb * q + K * r + c] -= omega * s;
        }
    }
  }
  /* AP = A P: n x nc, blocks b x K */
  int* apptr = (int*)xcalloc(n + 1, sizeof(int));
  int* apcol = NULL;
  long apn = 0, apcap = 0;
  for (int a = 0; a < nc; a++) mark[a] = -1;
  for (int i = 0; i < n; i++) {
    long start = apn;
    for (int k = L->ptr[i]; k < L->ptr[i + 1]; k++) {
      int j = L->col[k];
      for (int q = L->pptr[j]; q < L->pptr[j + 1]; q++)
        if (mark[L->pcol[q]] != i) {
          mark[L->pcol[q]] = i;
          push_int(&apcol, &apn, &apcap, L->pcol[q]);
        }
    }
    qsort(apcol + start, apn - start, sizeof(int), cmp_int);
    apptr[i + 1] = (int)apn;
  }
  if (!apcol) apcol = (int*)xcalloc(1, sizeof(int));
  double* apval = (double*)xcalloc((size_t)bb * apn + 1, sizeof(double));
  for (int i = 0; i < n; i++)
    for (int k = L->ptr[i]; k < L->ptr[i + 1]; k++) {
      int j = L->col[k];
      for (int q = L->pptr[j]; q < L->pptr[j + 1]; q++) {
        long p = find_block(apptr, apcol, i, L->pcol[q]);
        for (int r = 0; r < b; r++)
          for (int c = 0; c < K; c++) {
            double s = 0.0;
            for (int l = 0; l < b; l++) s += L->val[(size_t)b * b * k + b * r + l] * L->pval[(size_t)bb * q + K * l + c];
            apval[(size_t)bb * p + K * r + c] += s;
          }
      }
    }
  /* A_c = P^T (AP): entry (a, e) = sum_i P_ia^T AP_ie; rows of P^T first */
  int* tptr = (int*)xcalloc(nc + 1, sizeof(int));
  long np = L->pptr[n];
  for (long q = 0; q < np; q++) tptr[L->pcol[q] + 1]++;
  for (int a = 0; a < nc; a++) tptr[a + 1] += tptr[a];
  int* trow = (int*)xcalloc(np + 1, sizeof(int));
  int* tidx = (int*)xcalloc(np + 1, sizeof(int));
  for (int a = 0; a < nc; a++) fill[a] = 0;
  for (int i = 0; i < n; i++)
    for (int q = L->pptr[i]; q < L->pptr[i + 1]; q++) {
      int a = L->pcol[q], s = tptr[a] + fill[a]++;
      trow[s] = i;
      tidx[s] = q;
    }
  C->ptr = (int*)xcalloc(nc + 1, sizeof(int));
  C->col = NULL;
  long cn = 0, ccap = 0;
  for (int a = 0; a < nc; a++) mark[a] = -1;
  for (int a = 0; a < nc; a++) {
    long start = cn;
    for (int s = tptr[a]; s < tptr[a + 1]; s++)
      for (int p = apptr[trow[s]]; p < apptr[trow[s] + 1]; p++)
        if (mark[apcol[p]] != a) {
          mark[apcol[p]] = a;
          push_int(&C->col, &cn, &ccap, apcol[p]);
        }
    if (mark[a] != a) { /* the diagonal block is always stored */
      mark[a] = a;
      push_int(&C->col, &cn, &ccap, a);
    }
    qsort(C->col + start, cn - start, sizeof(int), cmp_int);
    C->ptr[a + 1] = (int)cn;
  }
  if (!C->col) C->col = (int*)xcalloc(1, sizeof(int));
  C->val = (double*)xcalloc((size_t)K * K * cn + 1, sizeof(double));
  for (int a = 0; a < nc; a++)
    for (int s = tptr[a]; s < tptr[a + 1]; s++) {
      int i = trow[s], q = tidx[s];
      for (int p = apptr[i]; p < apptr[i + 1]; p++) {
        long e = find_block(C->ptr, C->col, a, apcol[p]);
        for (int r = 0; r < K; r++)
          for (int c = 0; c < K; c++) {
            double v = 0.0;
            for (int l = 0; l < b; l++) v += L->pval[(size_t)bb * q + K * l + r] * apval[(size_t)bb * p + K * l + c];
            C->val[(size_t)K * K * e + K * r + c] += v;
          }
      }
    }
  for (int a = 0; a < nc; a++) { /* absent coarse components: unit diagonal */
    long e = find_block(C->ptr, C->col, a, a);
    for (int c = 0; c < K; c++)
      if ((C->absent[a] >> c) & 1) C->val[(size_t)K * K * e + K * c + c] = 1.0;
  }
  free(mptr); free(mem); free(fill); free(tq); free(mark); free(apptr); free(apcol); free(apval);
  free(tptr); free(trow); free(tidx);
}

static void amg_free(struct om_amg* h) {
  if (!h) return;
  for (int l = 0; l < h->nlev; l++) {
    om_amg_level* L = h->lev + l;
    if (l > 0) {
      free(L->ptr);
      free(L->col);
      free(L->val);
    }
    free(L->dinv); free(L->absent); free(L->ns); free(L->agg); free(L->pptr); free(L->pcol);
    free(L->pval); free(L->tval); free(L->inv);
  }
  free(h);
}

/* hierarchy from the assembled tangent (displacement block) */
static void amg_setup(om_mesh* m) {
  amg_free(m->amg);
  struct om_amg* h = (struct om_amg*)xcalloc(1, sizeof(struct om_amg));
  om_amg_level* L = h->lev;
  L->n = m->nn;
  L->b = 3;
  L->ptr = m->row_ptr;
  L->col = m->col;
  L->val = m->K;
  L->absent = (unsigned char*)xcalloc(m->nn, 1);
  L->ns = (double*)xcalloc((size_t)m->nn * 3 * OM_AMG_NS, sizeof(double));
  for (int a = 0; a < m->nn; a++) {
    const double* x = m->X + 3L * a;
    /* rigid motions: translations e_c, rotations (-y, x, 0), (0, -z, y), (z, 0, -x) */
    double rb[3][OM_AMG_NS] = {{1, 0, 0, -x[1], 0, x[2]}, {0, 1, 0, x[0], -x[2], 0}, {0, 0, 1, 0, x[1], -x[0]}};
    for (int c = 0; c < 3; c++) {
      int fixed = is_fixed(m, a, c);
      if (fixed) L->absent[a] |= (unsigned char)(1u << c);
      for (int k = 0; k < OM_AMG_NS; k++) L->ns[(3L * a + c) * OM_AMG_NS + k] = fixed ? 0.0 : rb[c][k];
    }
  }
  int l = 0;
  for (;;) {
    L = h->lev + l;
    amg_block_dinv(L);
    if (L->n <= OM_AMG_COARSE || l == OM_AMG_MAXLEV - 1) break;
    amg_aggregate(L);
    if (L->nc == 0 || L->nc > 0.9 * L->n) {
      free(L->agg);
      L->agg = NULL;
      L->nc = 0;
      break;
    }
    L->rho = amg_rho(L);
    amg_coarsen(L, h->lev + l + 1);
    l++;
  }
  h->nlev = l + 1;
  {
    int N = L->b * L->n;
    double* A = (double*)xcalloc((size_t)N * N + 1, sizeof(double));
    for (int a = 0; a < L->n; a++)
      for (int k = L->ptr[a]; k < L->ptr[a + 1]; k++)
        for (int i = 0; i < L->b; i++)
          for (int j = 0; j < L->b; j++)
            A[(size_t)(L->b * a + i) * N + L->b * L->col[k] + j] = L->val[(size_t)L->b * L->b * k + L->b * i + j];
    L->inv = (double*)xcalloc((size_t)N * N + 1, sizeof(double));
    gauss_jordan_inverse(N, A, L->inv);
    free(A);
  }
  m->amg = h;
}

/* Chebyshev smoothing of A x = b on level L from the given x (deg steps) */
static void amg_cheb(const om_amg_level* L, const double* b, double* x, int deg) {
  long N = (long)L->b * L->n;
  double lo = L->rho / 30.0, hi = 1.1 * L->rho;
  double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta, rho_old = 1.0 / sigma;
  double* r = (double*)xcalloc(N, sizeof(double));
  double* z = (double*)xcalloc(N, sizeof(double));
  double* d = (double*)xcalloc(N, sizeof(double));
  double* t = (double*)xcalloc(N, sizeof(double));
  bsr_mv(L->n, L->b, L->b, L->ptr, L->col, L->val, x, t);
  for (long i = 0; i < N; i++) r[i] = b[i] - t[i];
  amg_apply_dinv(L, r, z);
  for (long i = 0; i < N; i++) d[i] = z[i] / theta;
  for (int k = 1; k <= deg; k++) {
    for (long i = 0; i < N; i++) x[i] += d[i];
    if (k == deg) break;
    bsr_mv(L->n, L->b, L->b, L->ptr, L->col, L->val, d, t);
    for (long i = 0; i < N; i++) r[i] -= t[i];
    amg_apply_dinv(L, r, z);
    double rho_new = 1.0 / (2.0 * sigma - rho_old);
    for (long i = 0; i < N; i++) d[i] = rho_new * rho_old * d[i] + 2.0 * rho_new / delta * z[i];
    rho_old = rho_new;
  }
  free(r); free(z); free(d); free(t);
}

static void amg_vcycle(const struct om_amg* h, int l, const double* b, double* x) {
  const om_amg_level* L = h->lev + l;
  long N = (long)L->b * L->n;
  if (l == h->nlev - 1) {
    for (long i = 0; i < N; i++) {
      double s = 0.0;
      for (long j = 0; j < N; j++) s += L->inv[(size_t)i * N + j] * b[j];
      x[i] = s;
    }
    return;
  }
  const om_amg_level* C = h->lev + l + 1;
  long Nc = (long)C->b * C->n;
  double* r = (double*)xcalloc(N, sizeof(double));
  double* bc = (double*)xcalloc(Nc + 1, sizeof(double));
  double* xc = (double*)xcalloc(Nc + 1, sizeof(double));
  for (long i = 0; i < N; i++) x[i] = 0.0;
  amg_cheb(L, b, x, 2);
  bsr_mv(L->n, L->b, L->b, L->ptr, L->col, L->val, x, r);
  for (long i = 0; i < N; i++) r[i] = b[i] - r[i];
  bsr_tmv(L->n, C->n, L->b, C->b, L->pptr, L->pcol, L->pval, r, bc);
  amg_vcycle(h, l + 1, bc, xc);
  bsr_mv(L->n, L->b, C->b, L->pptr, L->pcol, L->pval, xc, r); /* r = P xc */
  for (long i = 0; i < N; i++) x[i] += r[i];
  amg_cheb(L, b, x, 2);
  free(r); free(bc); free(xc);
}

void om_set_pc(om_mesh* m, int pc_type) {
  m->pc_type = pc_type;
  if (pc_type != 1) {
    amg_free(m->amg);
    m->amg = NULL;
  }
}

int om_amg_levels(const om_mesh* m) { return m->amg ? m->amg->nlev : 0; }

/* out: n, b, nnz(A_l), nc, nnz(P_l) */
void om_amg_level_info(const om_mesh* m, int l, long long* out) {
  const om_amg_level* L = m->amg->lev + l;
  out[0] = L->n;
  out[1] = L->b;
  out[2] = L->ptr[L->n];
  out[3] = L->nc;
  out[4] = L->pptr ? L->pptr[L->n] : 0;
}

/* level l: A_l (ptr, col, val [nnz][b*b]), absent mask, near null space
 * ns [n*b][6], aggregates, P and T (pptr, pcol, pval/tval [nnzP][b*6]),
 * rho, and for the coarsest level the dense inverse inv [(b n)^2] */
void om_amg_copy(const om_mesh* m, int l, int* ptr, int* col, double* val, unsigned char* absent, double* ns,
                 int* agg, int* pptr, int* pcol, double* pval, double* tval, double* rho, double* inv) {
  const om_amg_level* L = m->amg->lev + l;
  long nnz = L->ptr[L->n];
  size_t bb = (size_t)L->b * L->b;
  if (ptr) memcpy(ptr, L->ptr, sizeof(int) * (size_t)(L->n + 1));
  if (col) memcpy(col, L->col, sizeof(int) * (size_t)nnz);
  if (val) memcpy(val, L->val, sizeof(double) * bb * (size_t)nnz);
  if (absent) memcpy(absent, L->absent, (size_t)L->n);
  if (ns && L->ns) memcpy(ns, L->ns, sizeof(double) * (size_t)L->n * L->b * OM_AMG_NS);
  if (agg && L->agg) memcpy(agg, L->agg, sizeof(int) * (size_t)L->n);
  if (L->pptr) {
    long np = L->pptr[L->n];
    if (pptr) memcpy(pptr, L->pptr, sizeof(int) * (size_t)(L->n + 1));
    if (pcol) memcpy(pcol, L->pcol, sizeof(int) * (size_t)np);
    if (pval) memcpy(pval, L->pval, sizeof(double) * (size_t)L->b * OM_AMG_NS * (size_t)np);
    if (tval) memcpy(tval, L->tval, sizeof(double) * (size_t)L->b * OM_AMG_NS * (size_t)np);
  }
  if (rho) *rho = L->rho;
  if (inv && L->inv) memcpy(inv, L->inv, sizeof(double) * (size_t)L->b * L->n * L->b * L->n);
}

/* Chebyshev smoothing on level l (x in/out) and one V-cycle from level 0 */
void om_amg_smooth(const om_mesh* m, int l, const double* b, double* x, int deg) {
  amg_cheb(m->amg->lev + l, b, x, deg);
}

void om_amg_vcycle(const om_mesh* m, const double* b, double* x) { amg_vcycle(m->amg, 0, b, x); }

void om_tangent(om_mesh* m, const double* d) {
  memset(m->K, 0, sizeof(double) * 9 * m->nnzb);
  if (m->pres) memset(m->B1, 0, sizeof(double) * 3 * m->nnz_up);
  int nen = m->nen;
  double gam = om_gamma(m);
  double lam[16], w[4], N[10], dN[10][3], G[4][3];
  int nq = om_tet_rule(m->order, lam, w);
  double Ke[10][10][3][3], Be[10][4][3], A[81], dPdp[9];
  for (int e = 0; e < m->ne; e++) {
    const int* c = m->conn + (long)e * nen;
    double vol = elem_geom(m, e, G);
    memset(Ke, 0, sizeof(Ke));
    memset(Be, 0, sizeof(Be));
    for (int q = 0; q < nq; q++) {
      tet_shape(m->order, lam + 4 * q, N);
      tet_grad(m->order, lam + 4 * q, G, dN);
      double F[9];
      for (int i = 0; i < 3; i++)
        for (int J = 0; J < 3; J++) {
          double s = (i == J);
          for (int a = 0; a < nen; a++) s += d[3L * c[a] + i] * dN[a][J];
          F[IDX(i, J)] = s;
        }
      double p = 0.0;
      if (m->pres)
        for (int a = 0; a < p_count(m); a++) p += d[3L * m->nn + p_index(m, e, c, a)] * p_shape(m, lam + 4 * q, a);
      double P[9];
      om_material(m->matp, F, m->fib ? m->fib + 9L * e : NULL, gam, p, NULL, P, A, dPdp);
      double wq = w[q] * vol;
      /* K_ab[i][k] += w sum_JL dN_a[J] A[iJ][kL] dN_b[L] */
      for (int a = 0; a < nen; a++)
        for (int b = 0; b < nen; b++)
          for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) {
              double s = 0.0;
              for (int J = 0; J < 3; J++)
                for (int L = 0; L < 3; L++) s += dN[a][J] * A[9 * IDX(i, J) + IDX(k, L)] * dN[b][L];
              Ke[a][b][i][k] += wq * s;
            }
      /* coupling dR_u(a,i)/dp_v = w sum_J dPdp[iJ] dN_a[J] lambda_v */
      if (m->pres)
        for (int a = 0; a < nen; a++)
          for (int v = 0; v < p_count(m); v++)
            for (int i = 0; i < 3; i++) {
              double s = 0.0;
              for (int J = 0; J < 3; J++) s += dPdp[IDX(i, J)] * dN[a][J];
              Be[a][v][i] += wq * s * p_shape(m, lam + 4 * q, v);
            }
    }
    for (int a = 0; a < nen; a++)
      for (int b = 0; b < nen; b++) {
        long k = find_block(m->row_ptr, m->col, c[a], c[b]);
        for (int i = 0; i < 3; i++)
          for (int kk = 0; kk < 3; kk++) m->K[9 * k + 3 * i + kk] += Ke[a][b][i][kk];
      }
    if (m->pres)
      for (int a = 0; a < nen; a++)
        for (int v = 0; v < p_count(m); v++) {
          long k = find_block(m->up_ptr, m->up_col, c[a], p_index(m, e, c, v));
          for (int i = 0; i < 3; i++) m->B1[3 * k + i] += Be[a][v][i];
        }
  }
  /* springs */
  for (int f = 0; f < m->nf; f++) {
    double fv[6][3], M[6][6], Ks[3][3];
    int nfn = face_terms(m, f, fv, M, Ks);
    if (m->fkind[f] != 2) continue;
    const int* v = m->fnodes + 6 * f;
    for (int a = 0; a < nfn; a++)
      for (int b = 0; b < nfn; b++) {
        long k = find_block(m->row_ptr, m->col, v[a], v[b]);
        for (int i = 0; i < 3; i++)
          for (int kk = 0; kk < 3; kk++) m->K[9 * k + 3 * i + kk] += M[a][b] * Ks[i][kk];
      }
  }
  /* follower loads (not symmetric) */
  for (int f = 0; f < m->nf; f++) {
    if (m->fkind[f] != 3 && m->fkind[f] != 5) continue;
    double rf[6][3], Kf[6][6][3][3];
    int nfn = follower_terms(m, f, d, rf, Kf);
    const int* v = m->fnodes + 6 * f;
    for (int a = 0; a < nfn; a++)
      for (int b = 0; b < nfn; b++) {
        long k = find_block(m->row_ptr, m->col, v[a], v[b]);
        for (int i = 0; i < 3; i++)
          for (int kk = 0; kk < 3; kk++) m->K[9 * k + 3 * i + kk] += Kf[a][b][i][kk];
      }
  }
  /* inertia and dashpots of the Newmark step: + 4/dt^2 M + 2/dt C */
  if (m->dyn) {
    double cm = 4.0 / (m->dt * m->dt), cc = 2.0 / m->dt;
    for (long k = 0; k < m->nnzb; k++)
      for (int i = 0; i < 3; i++)
        for (int kk = 0; kk < 3; kk++)
          m->K[9 * k + 3 * i + kk] += (i == kk ? cm * m->Mm[k] : 0.0) + cc * m->Cd[9 * k + 3 * i + kk];
  }
  /* Dirichlet: zero rows and columns of prescribed components, unit diagonal */
  for (int a = 0; a < m->nn; a++)
    for (int k = m->row_ptr[a]; k < m->row_ptr[a + 1]; k++) {
      int b = m->col[k];
      for (int i = 0; i < 3; i++)
        for (int kk = 0; kk < 3; kk++)
          if (is_fixed(m, a, i) || is_fixed(m, b, kk))
            m->K[9 * k + 3 * i + kk] = (a == b && i == kk) ? 1.0 : 0.0;
    }
  if (m->pres)
    for (int a = 0; a < m->nn; a++)
      for (int k = m->up_ptr[a]; k < m->up_ptr[a + 1]; k++)
        for (int i = 0; i < 3; i++)
          if (is_fixed(m, a, i)) m->B1[3 * k + i] = 0.0;
  /* nodal block-Jacobi: inverse of each 3x3 diagonal block */
  for (int a = 0; a < m->nn; a++) {
    long k = find_block(m->row_ptr, m->col, a, a);
    double Db[3][3], Di[3][3];
    for (int i = 0; i < 3; i++)
      for (int kk = 0; kk < 3; kk++) Db[i][kk] = m->K[9 * k + 3 * i + kk];
    inv3(Db, Di);
    for (int i = 0; i < 3; i++)
      for (int kk = 0; kk < 3; kk++) m->Dinv[9L * a + 3 * i + kk] = Di[i][kk];
  }
  /* SIMPLE Schur diagonal: S_vv = -sum_{a,i} B1[a,v]_i^2 / A_(ai,ai) */
  if (m->pres) {
    memset(m->Sd, 0, sizeof(double) * m->np);
    for (int a = 0; a < m->nn; a++) {
      long kd = find_block(m->row_ptr, m->col, a, a);
      for (int k = m->up_ptr[a]; k < m->up_ptr[a + 1]; k++)
        for (int i = 0; i < 3; i++) {
          double b = m->B1[3 * k + i];
          m->Sd[m->up_col[k]] -= b * b / m->K[9 * kd + 4 * i];
        }
    }
  }
  if (m->pc_type == 1) amg_setup(m);
  m->have_K = 1;
}

void om_tangent_copy(const om_mesh* m, double* val, double* bup, double* dinv) {
  if (val) memcpy(val, m->K, sizeof(double) * 9 * m->nnzb);
  if (bup && m->pres) memcpy(bup, m->B1, sizeof(double) * 3 * m->nnz_up);
  if (dinv) memcpy(dinv, m->Dinv, sizeof(double) * 9 * (size_t)m->nn);
}

void om_spmv(const om_mesh* m, const double* x, double* y) {
  /* y_u = A x_u + B1 x_p; y_p = B2 x_u with B2 = B1^T */
  for (long i = 0; i < m->ndof; i++) y[i] = 0.0;
  for (int a = 0; a < m->nn; a++)
    for (int k = m->row_ptr[a]; k < m->row_ptr[a + 1]; k++) {
      int b = m->col[k];
      for (int i = 0; i < 3; i++)
        for (int kk = 0; kk < 3; kk++) y[3L * a + i] += m->K[9L * k + 3 * i + kk] * x[3L * b + kk];
    }
  if (m->pres) {
    const double* xp = x + 3L * m->nn;
    double* yp = y + 3L * m->nn;
    for (int a = 0; a < m->nn; a++)
      for (int k = m->up_ptr[a]; k < m->up_ptr[a + 1]; k++) {
        int v = m->up_col[k];
        for (int i = 0; i < 3; i++) {
          y[3L * a + i] += m->B1[3L * k + i] * xp[v];
          yp[v] += m->B1[3L * k + i] * x[3L * a + i];
        }
      }
  }
}

void om_pc(const om_mesh* m, const double* x, double* y) {
  /* displacement: nodal block-Jacobi or one AMG V-cycle; u-p: lower Schur
   * (Appendix B), z_u = M_A^{-1} x_u, z_p = S^{-1} (x_p - B2 z_u), S = point
   * diagonal */
  if (m->pc_type == 1 && m->amg) {
    amg_vcycle(m->amg, 0, x, y);
  } else {
    for (int a = 0; a < m->nn; a++)
      for (int i = 0; i < 3; i++) {
        double s = 0.0;
        for (int k = 0; k < 3; k++) s += m->Dinv[9L * a + 3 * i + k] * x[3L * a + k];
        y[3L * a + i] = s;
      }
  }
  if (m->pres) {
    double* t = (double*)xcalloc(m->np, sizeof(double));
    for (int v = 0; v < m->np; v++) t[v] = x[3L * m->nn + v];
    for (int a = 0; a < m->nn; a++)
      for (int k = m->up_ptr[a]; k < m->up_ptr[a + 1]; k++)
        for (int i = 0; i < 3; i++) t[m->up_col[k]] -= m->B1[3L * k + i] * y[3L * a + i];
    for (int v = 0; v < m->np; v++) y[3L * m->nn + v] = m->Sd[v] != 0.0 ? t[v] / m->Sd[v] : t[v];
    free(t);
  }
}

/* ======================================================================
 * GMRES: right preconditioned, modified Gram-Schmidt Arnoldi, Givens
 * rotations, restart every `restart` steps (the paper uses none; the cap
 * is a reading).  Stops when the residual estimate <= max(rtol ||b||, atol)
 * or after max_it iterations.  Returns the iteration count.
 * ====================================================================== */
int om_gmres(om_mesh* m, const double* b, double* x, double rtol, double atol, int restart,
             int max_it, double* res_out) {
  long n = m->ndof;
  int kmax = restart;
  double* V = (double*)xcalloc((size_t)(kmax + 1) * n, sizeof(double));
  double* H = (double*)xcalloc((size_t)(kmax + 1) * kmax, sizeof(double));
  double* cs = (double*)xcalloc(kmax, sizeof(double));
  double* sn = (double*)xcalloc(kmax, sizeof(double));
  double* g = (double*)xcalloc(kmax + 1, sizeof(double));
  double* yv = (double*)xcalloc(kmax, sizeof(double));
  double* w = (double*)xcalloc(n, sizeof(double));
  double* z = (double*)xcalloc(n, sizeof(double));
  double bnorm = nrm2(b, n);
  double target = fmax(rtol * bnorm, atol);
  int it = 0;
  double res = 0.0;
  for (;;) {
    /* r = b - K x */
    om_spmv(m, x, w);
    for (long i = 0; i < n; i++) V[i] = b[i] - w[i];
    double beta = nrm2(V, n);
    res = beta;
    if (beta <= target || it >= max_it || !isfinite(beta)) break;
    for (long i = 0; i < n; i++) V[i] /= beta;
    memset(g, 0, sizeof(double) * (kmax + 1));
    g[0] = beta;
    int j = 0, done = 0;
    for (j = 0; j < kmax; j++) {
      om_pc(m, V + (size_t)j * n, z);
      om_spmv(m, z, w);
      for (int i = 0; i <= j; i++) { /* modified Gram-Schmidt */
        double h = dot(w, V + (size_t)i * n, n);
        H[(size_t)i * kmax + j] = h;
        for (long l = 0; l < n; l++) w[l] -= h * V[(size_t)i * n + l];
      }
      double hn = nrm2(w, n);
      H[(size_t)(j + 1) * kmax + j] = hn;
      for (int i = 0; i < j; i++) { /* previous rotations */
        double a = H[(size_t)i * kmax + j], c = H[(size_t)(i + 1) * kmax + j];
        H[(size_t)i * kmax + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * kmax + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[(size_t)j * kmax + j], c = H[(size_t)(j + 1) * kmax + j];
      double r = hypot(a, c);
      cs[j] = a / r;
      sn[j] = c / r;
      H[(size_t)j * kmax + j] = r;
      H[(size_t)(j + 1) * kmax + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      it++;
      res = fabs(g[j + 1]);
      if (res <= target || it >= max_it || hn == 0.0 || !isfinite(res)) {
        done = 1;
        j++;
        break;
      }
      for (long l = 0; l < n; l++) V[(size_t)(j + 1) * n + l] = w[l] / hn;
    }
    if (!done) j = kmax;
    /* y = H^{-1} g (upper triangular j x j), x += M^{-1} V y */
    for (int i = j - 1; i >= 0; i--) {
      double s = g[i];
      for (int k = i + 1; k < j; k++) s -= H[(size_t)i * kmax + k] * yv[k];
      yv[i] = s / H[(size_t)i * kmax + i];
    }
    memset(w, 0, sizeof(double) * n);
    for (int i = 0; i < j; i++)
      for (long l = 0; l < n; l++) w[l] += yv[i] * V[(size_t)i * n + l];
    om_pc(m, w, z);
    for (long l = 0; l < n; l++) x[l] += z[l];
    if (done) break;
  }
  m->lit += it;
  if (res_out) *res_out = res;
  free(V); free(H); free(cs); free(sn); free(g); free(yv); free(w); free(z);
  return it;
}

/* L-BFGS two-loop recursion over k pairs stored oldest first:
 * q = input; for i newest..oldest: alpha_i = rho_i s_i.q, q -= alpha_i y_i;
 * z = H0 q; for i oldest..newest: beta = rho_i y_i.z, z += (alpha_i - beta) s_i.
 * This is the product with the BFGS inverse update of the paper applied k
 * times to H0 (Nocedal 1980). */
static void twoloop(om_mesh* m, const double* S, const double* Y, const double* rho, int k,
                    const double* qin, double* z, int h0, double ksp_rtol, double ksp_atol,
                    int restart, int kmaxit) {
  long n = m->ndof;
  double* q = (double*)xcalloc(n, sizeof(double));
  double* alpha = (double*)xcalloc(k > 0 ? k : 1, sizeof(double));
  memcpy(q, qin, sizeof(double) * n);
  for (int i = k - 1; i >= 0; i--) {
    alpha[i] = rho[i] * dot(S + (size_t)i * n, q, n);
    for (long l = 0; l < n; l++) q[l] -= alpha[i] * Y[(size_t)i * n + l];
  }
  if (h0 == 0) {
    om_pc(m, q, z);
  } else if (h0 == 1) {
    memcpy(z, q, sizeof(double) * n);
  } else {
    memset(z, 0, sizeof(double) * n);
    om_gmres(m, q, z, ksp_rtol, ksp_atol, restart, kmaxit, NULL);
  }
  for (int i = 0; i < k; i++) {
    double beta = rho[i] * dot(Y + (size_t)i * n, z, n);
    for (long l = 0; l < n; l++) z[l] += (alpha[i] - beta) * S[(size_t)i * n + l];
  }
  free(q);
  free(alpha);
}

void om_lbfgs_apply(om_mesh* m, const double* S, const double* Y, const double* rho, int k,
                    const double* q, double* z, int h0) {
  twoloop(m, S, Y, rho, k, q, z, h0, 0, 0, 1, 1);
}

/* ======================================================================
 * nonlinear solvers (Section "Numerical solvers", Appendix A)
 * ====================================================================== */
/* seconds since t0 (instrumentation: the per-iteration times of a solve) */
static double om_elapsed(const struct timespec* t0) {
  struct timespec t;
  clock_gettime(CLOCK_MONOTONIC, &t);
  return (double)(t.tv_sec - t0->tv_sec) + 1e-9 * (double)(t.tv_nsec - t0->tv_nsec);
}

int om_solve(om_mesh* m, int method, double tol, int max_it, double* d, const double* opts,
             double* stats) {
  long n = m->ndof;
  double ksp_rtol = opts[1], ksp_atol = opts[2], ew0 = opts[3], ewmax = opts[4];
  int restart = (int)opts[5], kmaxit = (int)opts[6], mm = (int)opts[7];
  double dtol = opts[8];
  int jac_lag = (int)opts[10] > 0 ? (int)opts[10] : 1, hess_re = (int)opts[11];
  int ib_adaptive = (int)opts[12];
  om_set_pc(m, (int)opts[13]);
  double* res_hist = stats + 6;
  double* lit_hist = stats + 6 + OM_HIST;
  double* eta_hist = stats + 6 + 2 * OM_HIST;
  double* lres_hist = stats + 6 + 3 * OM_HIST;
  double* time_hist = stats + 6 + 4 * OM_HIST;
  for (int i = 0; i < 6 + 5 * OM_HIST; i++) stats[i] = 0.0;
  struct timespec ts0;
  clock_gettime(CLOCK_MONOTONIC, &ts0);
  if ((int)opts[9]) om_apply_dirichlet(m, d);
  double* R = (double*)xcalloc(n, sizeof(double));
  double* Rn = (double*)xcalloc(n, sizeof(double));
  double* dl = (double*)xcalloc(n, sizeof(double));
  double* t = (double*)xcalloc(n, sizeof(double));
  m->lit = 0;
  int assemblies = 0, status = 2, nit = 0;
  double r0 = om_residual(m, d, R), rk = r0;
  res_hist[0] = r0;
  time_hist[0] = om_elapsed(&ts0);
  if (!isfinite(r0)) {
    status = 3;
    goto out;
  }
  if (r0 == 0.0) {
    status = 0;
    goto out;
  }
  if (method == 0 || method == 1) {
    double eta = method == 0 ? ksp_rtol : ew0, eta_prev = eta;
    const double alpha2 = 0.5 * (1.0 + sqrt(5.0));
    for (int k = 1; k <= max_it; k++) {
      /* Jacobian lagging (conclusions: an extension for the Newton methods):
       * the tangent is assembled at iterations 1, 1 + L, 1 + 2L, ... and the
       * linear solves in between use the last one */
      if ((k - 1) % jac_lag == 0) {
        om_tangent(m, d);
        assemblies++;
      }
      /* K delta = -R */
      for (long i = 0; i < n; i++) t[i] = -R[i];
      memset(dl, 0, sizeof(double) * n);
      long long lit0 = m->lit;
      om_gmres(m, t, dl, eta, ksp_atol, restart, kmaxit, NULL);
      if (k < OM_HIST) {
        lit_hist[k] = (double)(m->lit - lit0);
        eta_hist[k] = eta;
      }
      /* linear residual ||R_{k-1} + K delta|| (used by Eisenstat-Walker) */
      om_spmv(m, dl, Rn);
      for (long i = 0; i < n; i++) Rn[i] += R[i];
      double lnorm = nrm2(Rn, n);
      if (k < OM_HIST) lres_hist[k] = lnorm;
      for (long i = 0; i < n; i++) d[i] += dl[i]; /* basic line search: full step */
      double rprev = rk;
      rk = om_residual(m, d, R);
      nit = k;
      if (k < OM_HIST) {
        res_hist[k] = rk;
        time_hist[k] = om_elapsed(&ts0);
      }
      if (!isfinite(rk)) { status = 3; goto out; }
      if (rk <= tol * r0) { status = 0; goto out; }
      if (rk > dtol * r0) { status = 1; goto out; }
      if (method == 1) {
        /* Eisenstat-Walker choice 1: eta = | ||R_k|| - ||R_{k-1} + K delta|| | / ||R_{k-1}||,
         * safeguard eta >= eta_prev^((1+sqrt5)/2) when that exceeds 0.1, cap ew_rtolmax.
         * (Reading of the garbled formula of the paper.) */
        eta_prev = eta;
        eta = fabs(rk - lnorm) / rprev;
        double st = pow(eta_prev, alpha2);
        if (st > 0.1) eta = fmax(eta, st);
        eta = fmin(eta, ewmax);
      }
    }
    status = 2;
    goto out;
  } else {
    /* B / iB: K assembled once at d_0; H0 = preconditioner (B) or GMRES (iB) */
    om_tangent(m, d);
    assemblies = 1;
    double* S = (double*)xcalloc((size_t)mm * n, sizeof(double));
    double* Y = (double*)xcalloc((size_t)mm * n, sizeof(double));
    double* rho = (double*)xcalloc(mm, sizeof(double));
    int np = 0;
    /* adaptive H0 tolerance for iB (the paper leaves an Eisenstat-Walker type
     * tolerance for future work); reading: EW choice 2 on the nonlinear
     * residual norms, eta_1 = ksp_rtol,
     *   eta_k = min(ew_rtolmax, max(0.9 (r_{k-1} / r_{k-2})^a, 0.9 eta_{k-1}^a
     *           when the latter exceeds 0.1)),  a = (1 + sqrt 5) / 2 */
    double eta = ksp_rtol, r_km2 = 0.0;
    for (int k = 1; k <= max_it; k++) {
      if (method == 3 && ib_adaptive && k > 1) {
        double eta_prev = eta, a = 0.5 * (1.0 + sqrt(5.0));
        eta = 0.9 * pow(rk / r_km2, a);
        if (0.9 * pow(eta_prev, a) > 0.1) eta = fmax(eta, 0.9 * pow(eta_prev, a));
        eta = fmin(eta, ewmax);
      }
      /* occasional re-assembly for BFGS (conclusions): a new H0 from the
       * tangent at the current iterate, and the memory starts again */
      if (hess_re > 0 && k > 1 && (k - 1) % hess_re == 0) {
        om_tangent(m, d);
        assemblies++;
        np = 0;
      }
      long long lit0 = m->lit;
      twoloop(m, S, Y, rho, np, R, t, method == 2 ? 0 : 2, eta, ksp_atol, restart, kmaxit);
      if (k < OM_HIST) {
        lit_hist[k] = (double)(m->lit - lit0);
        eta_hist[k] = method == 2 ? 0.0 : eta;
      }
      r_km2 = rk;
      for (long i = 0; i < n; i++) {
        dl[i] = -t[i];
        d[i] += dl[i];
      }
      rk = om_residual(m, d, Rn);
      nit = k;
      if (k < OM_HIST) {
        res_hist[k] = rk;
        time_hist[k] = om_elapsed(&ts0);
      }
      /* secant pair s = delta, y = R_{k+1} - R_k, rho = 1/(y.s), skipped when y.s <= 0 */
      for (long i = 0; i < n; i++) t[i] = Rn[i] - R[i];
      double ys = dot(t, dl, n);
      if (ys > 0.0) {
        if (np == mm) {
          memmove(S, S + n, sizeof(double) * (size_t)(mm - 1) * n);
          memmove(Y, Y + n, sizeof(double) * (size_t)(mm - 1) * n);
          memmove(rho, rho + 1, sizeof(double) * (mm - 1));
          np--;
        }
        memcpy(S + (size_t)np * n, dl, sizeof(double) * n);
        memcpy(Y + (size_t)np * n, t, sizeof(double) * n);
        rho[np] = 1.0 / ys;
        np++;
      }
      memcpy(R, Rn, sizeof(double) * n);
      if (!isfinite(rk)) { status = 3; break; }
      if (rk <= tol * r0) { status = 0; break; }
      if (rk > dtol * r0) { status = 1; break; }
      status = 2;
    }
    free(S);
    free(Y);
    free(rho);
  }
out:
  stats[0] = status;
  stats[1] = nit;
  stats[2] = (double)m->lit;
  stats[3] = assemblies;
  stats[4] = r0;
  stats[5] = rk;
  free(R);
  free(Rn);
  free(dl);
  free(t);
  return status;
}
