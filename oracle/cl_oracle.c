/*
 * cl_oracle.c -- plain, slow, obviously-correct CPU reference (FP64) for the
 * fermion drift of complex-Langevin QCD with staggered quarks
 * (Bloch & Schenk, arXiv:1707.08874).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path: it builds the dense Dirac matrix, factors it with a
 * textbook right-looking LU with partial pivoting, solves for columns of the
 * inverse and evaluates every formula of the method literally.
 *
 * Conventions (the paper leaves them open; the same readings are used by the
 * CUDA library and are listed with the design notes):
 *   site index   s = ((t*Ns + z)*Ns + y)*Ns + x,  direction nu = 0..3 = x,y,z,t
 *   unknown      3*s + colour
 *   links        U[s][nu][a][b]  (3x3 complex, row a, column b)
 *   D(m;mu)      D_{x,x}        = m * 1
 *                D_{x,x+nu}     = +1/2 eta_nu(x) s_nu(x) e^{+mu d_{nu,t}} U_{x,nu}
 *                D_{x+nu,x}     = -1/2 eta_nu(x) s_nu(x) e^{-mu d_{nu,t}} U_{x,nu}^{-1}
 *   eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z)
 *   s_nu(x) = -1 for the temporal hop between t = Nt-1 and t = 0 (antiperiodic
 *   fermions), +1 otherwise.
 *   Derivative (Eq. 6): left Lie derivative, d_a U = i lambda_a U and
 *   d_a U^{-1} = -i U^{-1} lambda_a.
 *
 * Parity of every function here is pinned by the CPU test-suite against the
 * free-field closed form, finite differences of log det D, exact symmetries of
 * det D, LAPACK on tiny lattices and a full-pivoting Gauss-Jordan determinant.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* geometry                                                             */
/* ------------------------------------------------------------------ */
static void coords(int Ns, int s, int c[4]) {
  c[0] = s % Ns; s /= Ns;
  c[1] = s % Ns; s /= Ns;
  c[2] = s % Ns; s /= Ns;
  c[3] = s;
}
static int site_of(int Ns, const int c[4]) {
  return ((c[3] * Ns + c[2]) * Ns + c[1]) * Ns + c[0];
}
/* neighbour of s in direction nu, dir = +1 or -1, periodic wrap */
static int neighbour(int Ns, int Nt, int s, int nu, int dir) {
  int c[4], L[4] = {Ns, Ns, Ns, Nt};
  coords(Ns, s, c);
  c[nu] = (c[nu] + dir + L[nu]) % L[nu];
  return site_of(Ns, c);
}
/* staggered phase eta_nu(x) */
static double eta(int Ns, int s, int nu) {
  int c[4], sum = 0;
  coords(Ns, s, c);
  for (int i = 0; i < nu; ++i) sum += c[i];
  return (sum & 1) ? -1.0 : 1.0;
}
/* boundary sign of the forward hop x -> x+nu (antiperiodic in time) */
static double bsign(int Ns, int Nt, int s, int nu) {
  int c[4];
  coords(Ns, s, c);
  return (nu == 3 && c[3] == Nt - 1) ? -1.0 : 1.0;
}

/* ------------------------------------------------------------------ */
/* 3x3 helpers                                                          */
/* ------------------------------------------------------------------ */
static void mul3(const cplx* A, const cplx* B, cplx* C) {
  cplx T[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cplx acc = 0;
      for (int k = 0; k < 3; ++k) acc += A[3 * i + k] * B[3 * k + j];
      T[3 * i + j] = acc;
    }
  memcpy(C, T, sizeof(T));
}
static cplx det3(const cplx* A) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}
/* inverse by the adjugate divided by the determinant (cofactor formula) */
static void inv3(const cplx* A, cplx* R) {
  cplx d = det3(A);
  cplx C[9];
  C[0] = A[4] * A[8] - A[5] * A[7];
  C[1] = A[2] * A[7] - A[1] * A[8];
  C[2] = A[1] * A[5] - A[2] * A[4];
  C[3] = A[5] * A[6] - A[3] * A[8];
  C[4] = A[0] * A[8] - A[2] * A[6];
  C[5] = A[2] * A[3] - A[0] * A[5];
  C[6] = A[3] * A[7] - A[4] * A[6];
  C[7] = A[1] * A[6] - A[0] * A[7];
  C[8] = A[0] * A[4] - A[1] * A[3];
  for (int i = 0; i < 9; ++i) R[i] = C[i] / d;
}
static cplx tr3(const cplx* A) { return A[0] + A[4] + A[8]; }

/* Gell-Mann matrices lambda_1..lambda_8 (standard order), Eq. 2 */
static void gell_mann(int a, cplx* L) {
  for (int i = 0; i < 9; ++i) L[i] = 0;
  const double r3 = 1.0 / sqrt(3.0);
  switch (a) {
    case 0: L[1] = 1; L[3] = 1; break;
    case 1: L[1] = -I; L[3] = I; break;
    case 2: L[0] = 1; L[4] = -1; break;
    case 3: L[2] = 1; L[6] = 1; break;
    case 4: L[2] = -I; L[6] = I; break;
    case 5: L[5] = 1; L[7] = 1; break;
    case 6: L[5] = -I; L[7] = I; break;
    case 7: L[0] = r3; L[4] = r3; L[8] = -2 * r3; break;
  }
}

/* exported for the pin on the Lie-algebra table: out[a][3][3] */
void or_gell_mann(cplx* out) {
  for (int a = 0; a < 8; ++a) gell_mann(a, out + 9 * a);
}

/* ------------------------------------------------------------------ */
/* Dirac operator, Eq. 1 (staggered D(m;mu), U^{-1} in place of U^dag)  */
/* ------------------------------------------------------------------ */
/* hop blocks of link (s,nu): F = D_{s,s+nu}, B = D_{s+nu,s} */
static void hop_blocks(int Ns, int Nt, const cplx* U, int s, int nu, double mu, cplx* F,
                       cplx* B) {
  const cplx* u = U + (size_t)(4 * s + nu) * 9;
  double ph = 0.5 * eta(Ns, s, nu) * bsign(Ns, Nt, s, nu);
  double ef = (nu == 3) ? exp(mu) : 1.0, eb = (nu == 3) ? exp(-mu) : 1.0;
  cplx ui[9];
  inv3(u, ui);
  for (int i = 0; i < 9; ++i) {
    F[i] = ph * ef * u[i];
    B[i] = -ph * eb * ui[i];
  }
}

void or_dirac_dense(int Ns, int Nt, const cplx* U, double m, double mu, cplx* D) {
  const int V = Ns * Ns * Ns * Nt, N = 3 * V;
  memset(D, 0, sizeof(cplx) * (size_t)N * N);
  for (int s = 0; s < V; ++s)
    for (int a = 0; a < 3; ++a) D[(size_t)(3 * s + a) * N + 3 * s + a] += m;
  for (int s = 0; s < V; ++s)
    for (int nu = 0; nu < 4; ++nu) {
      int y = neighbour(Ns, Nt, s, nu, +1);
      cplx F[9], B[9];
      hop_blocks(Ns, Nt, U, s, nu, mu, F, B);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          D[(size_t)(3 * s + a) * N + 3 * y + b] += F[3 * a + b];
          D[(size_t)(3 * y + a) * N + 3 * s + b] += B[3 * a + b];
        }
    }
}

/* ------------------------------------------------------------------ */
/* dense LU with partial (row) pivoting, right-looking, textbook form   */
/* P A = L U; L unit lower and U upper overwrite A; piv[k] = row that   */
/* was swapped with row k at step k.  Returns 0, or k+1 if the pivot    */
/* of column k is exactly zero.  Ties in |a_ik| keep the lowest row.    */
/* ------------------------------------------------------------------ */
int or_lu_steps(int N, cplx* A, int* piv, int nsteps);
int or_lu(int N, cplx* A, int* piv) { return or_lu_steps(N, A, piv, N); }

/* The first nsteps elimination steps of the same factorisation (used only to
   time a bounded sample of the dense reference). */
int or_lu_steps(int N, cplx* A, int* piv, int nsteps) {
  int info = 0;
  for (int k = 0; k < nsteps && k < N; ++k) {
    int p = k;
    double best = cabs(A[(size_t)k * N + k]);
    for (int i = k + 1; i < N; ++i) {
      double v = cabs(A[(size_t)i * N + k]);
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < N; ++j) {
        cplx t = A[(size_t)k * N + j];
        A[(size_t)k * N + j] = A[(size_t)p * N + j];
        A[(size_t)p * N + j] = t;
      }
    cplx akk = A[(size_t)k * N + k];
    if (akk == 0) { if (!info) info = k + 1; continue; }
#pragma omp parallel for schedule(static)
    for (int i = k + 1; i < N; ++i) {
      cplx* ri = A + (size_t)i * N;
      const cplx* rk = A + (size_t)k * N;
      cplx l = ri[k] / akk;
      ri[k] = l;
      for (int j = k + 1; j < N; ++j) ri[j] -= l * rk[j];
    }
  }
  return info;
}

/* Solve (P A) X = P E for the unit vectors e_{cols[c]}, i.e. X = A^{-1} E.
   X is N x ncols, row-major.  Forward then back substitution. */
void or_solve_unit_columns(int N, const cplx* LU, const int* piv, int ncols, const int* cols,
                           cplx* X) {
  memset(X, 0, sizeof(cplx) * (size_t)N * ncols);
  for (int c = 0; c < ncols; ++c) X[(size_t)cols[c] * ncols + c] = 1;
  for (int k = 0; k < N; ++k)
    if (piv[k] != k)
      for (int c = 0; c < ncols; ++c) {
        cplx t = X[(size_t)k * ncols + c];
        X[(size_t)k * ncols + c] = X[(size_t)piv[k] * ncols + c];
        X[(size_t)piv[k] * ncols + c] = t;
      }
  const int CH = 8;
  const int nch = (ncols + CH - 1) / CH;
#pragma omp parallel for schedule(dynamic)
  for (int ch = 0; ch < nch; ++ch) {
    int c0 = ch * CH, c1 = c0 + CH < ncols ? c0 + CH : ncols;
    /* L y = b (unit lower) */
    for (int i = 0; i < N; ++i) {
      const cplx* li = LU + (size_t)i * N;
      for (int j = 0; j < i; ++j) {
        cplx l = li[j];
        if (l == 0) continue;
        for (int c = c0; c < c1; ++c) X[(size_t)i * ncols + c] -= l * X[(size_t)j * ncols + c];
      }
    }
    /* U x = y */
    for (int i = N - 1; i >= 0; --i) {
      const cplx* ui = LU + (size_t)i * N;
      for (int j = i + 1; j < N; ++j) {
        cplx u = ui[j];
        if (u == 0) continue;
        for (int c = c0; c < c1; ++c) X[(size_t)i * ncols + c] -= u * X[(size_t)j * ncols + c];
      }
      for (int c = c0; c < c1; ++c) X[(size_t)i * ncols + c] /= ui[i];
    }
  }
}

/* full inverse, column by column (chunks of columns at a time) */
void or_inverse(int N, const cplx* LU, const int* piv, cplx* Ainv) {
  int* cols = (int*)malloc(sizeof(int) * N);
  for (int j = 0; j < N; ++j) cols[j] = j;
  or_solve_unit_columns(N, LU, piv, N, cols, Ainv);
  free(cols);
}

/* log det A = sum_i log u_ii + log det P (each swap contributes i*pi).
   The imaginary part is returned unwrapped (sum of arguments). */
void or_logdet(int N, const cplx* LU, const int* piv, double* re, double* im) {
  double r = 0, a = 0;
  for (int i = 0; i < N; ++i) {
    cplx u = LU[(size_t)i * N + i];
    r += log(cabs(u));
    a += carg(u);
    if (piv[i] != i) a += M_PI;
  }
  *re = r;
  *im = a;
}

/* ------------------------------------------------------------------ */
/* selected blocks of D^{-1} on the pattern of D (Sec. 3, Eq. 8)        */
/* Gdiag[s] = G_{s,s}; Gfwd[s][nu] = G_{s,s+nu}; Gbwd[s][nu] = G_{s+nu,s} */
/* ------------------------------------------------------------------ */
void or_extract_blocks(int Ns, int Nt, const cplx* Ginv, cplx* Gdiag, cplx* Gfwd, cplx* Gbwd) {
  const int V = Ns * Ns * Ns * Nt, N = 3 * V;
  for (int s = 0; s < V; ++s) {
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Gdiag[9 * s + 3 * a + b] = Ginv[(size_t)(3 * s + a) * N + 3 * s + b];
    for (int nu = 0; nu < 4; ++nu) {
      int y = neighbour(Ns, Nt, s, nu, +1);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          Gfwd[(size_t)(4 * s + nu) * 9 + 3 * a + b] = Ginv[(size_t)(3 * s + a) * N + 3 * y + b];
          Gbwd[(size_t)(4 * s + nu) * 9 + 3 * a + b] = Ginv[(size_t)(3 * y + a) * N + 3 * s + b];
        }
    }
  }
}

/* ------------------------------------------------------------------ */
/* fermion drift, Eq. 6 and Eq. 8:                                      */
/* K^f_{a,x,nu} = nf * [ Tr(P B_a) + Tr(Q F_a) ],                       */
/* P = G_{x,x+nu}, Q = G_{x+nu,x}, F_a = d_a D_{x,x+nu}, B_a = d_a D_{x+nu,x} */
/* ------------------------------------------------------------------ */
void or_fermion_drift(int Ns, int Nt, const cplx* U, const cplx* Gfwd, const cplx* Gbwd,
                      double mu, double nf, cplx* Kf) {
  const int V = Ns * Ns * Ns * Nt;
  cplx lam[8][9];
  for (int a = 0; a < 8; ++a) gell_mann(a, lam[a]);
  for (int s = 0; s < V; ++s)
    for (int nu = 0; nu < 4; ++nu) {
      const cplx* u = U + (size_t)(4 * s + nu) * 9;
      const cplx* P = Gfwd + (size_t)(4 * s + nu) * 9;
      const cplx* Q = Gbwd + (size_t)(4 * s + nu) * 9;
      double ph = 0.5 * eta(Ns, s, nu) * bsign(Ns, Nt, s, nu);
      double ef = (nu == 3) ? exp(mu) : 1.0, eb = (nu == 3) ? exp(-mu) : 1.0;
      cplx ui[9];
      inv3(u, ui);
      for (int a = 0; a < 8; ++a) {
        cplx dU[9], dUi[9], F[9], B[9], PB[9], QF[9];
        mul3(lam[a], u, dU);   /* d_a U      =  i lambda_a U      (factor i below) */
        mul3(ui, lam[a], dUi); /* d_a U^{-1} = -i U^{-1} lambda_a (factor -i below) */
        for (int i = 0; i < 9; ++i) {
          F[i] = ph * ef * (I * dU[i]);
          B[i] = -ph * eb * (-I * dUi[i]);
        }
        mul3(P, B, PB);
        mul3(Q, F, QF);
        Kf[(size_t)(4 * s + nu) * 8 + a] = nf * (tr3(PB) + tr3(QF));
      }
    }
}

/* one full drift evaluation through the dense inverse (small lattices) */
int or_drift_eval(int Ns, int Nt, const cplx* U, double m, double mu, double nf, cplx* Gdiag,
                  cplx* Gfwd, cplx* Gbwd, cplx* Kf, double* logdet_re, double* logdet_im) {
  const int V = Ns * Ns * Ns * Nt, N = 3 * V;
  cplx* D = (cplx*)malloc(sizeof(cplx) * (size_t)N * N);
  cplx* G = (cplx*)malloc(sizeof(cplx) * (size_t)N * N);
  int* piv = (int*)malloc(sizeof(int) * N);
  if (!D || !G || !piv) { free(D); free(G); free(piv); return -1; }
  or_dirac_dense(Ns, Nt, U, m, mu, D);
  int info = or_lu(N, D, piv);
  if (info == 0) {
    or_logdet(N, D, piv, logdet_re, logdet_im);
    or_inverse(N, D, piv, G);
    or_extract_blocks(Ns, Nt, G, Gdiag, Gfwd, Gbwd);
    or_fermion_drift(Ns, Nt, U, Gfwd, Gbwd, mu, nf, Kf);
  }
  free(D); free(G); free(piv);
  return info;
}

/* chiral condensate, (nf / V) sum_x Tr G_{xx} */
cplx or_condensate(int V, const cplx* Gdiag, double nf) {
  cplx acc = 0;
  for (int s = 0; s < V; ++s) acc += tr3(Gdiag + 9 * s);
  return nf * acc / V;
}
