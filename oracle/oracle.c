/*
 * Oracle: plain, slow, FP64 CPU reference for the integral-direct J/K build.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The CUDA
 * product path never links, calls or reads anything here, and this file shares
 * no code, tables or constants with it.
 *
 * What it computes (paper: Wang et al., "Extending GPU-Accelerated Gaussian
 * Integrals in the TeraChem Software Package to f Type Orbitals"):
 *   - contracted Cartesian Gaussian basis functions, Eq. contracted_basis and
 *     Eq. primtive_basis (Sec. 2.1), normalised per component;
 *   - the Boys function, Eq. boys_function, by its power series / asymptote;
 *   - electron repulsion integrals, Eq. eri_definition, by a method that is
 *     deliberately NOT the paper's McMurchie-Davidson scheme: Obara-Saika
 *     vertical recurrence with the electron-transfer term, then Head-Gordon-
 *     Pople horizontal recurrence (the paper's refs for OS and HGP);
 *   - the Cauchy-Schwarz bound Eq. cauchy_schwarz_bound and the significance
 *     test of Eq. kernel_upperbound (density factor off);
 *   - J and K by their definitions, Eq. j_definition and Eq. k_definition,
 *     either over every ordered shell quartet or over canonical quartets with
 *     the 8-fold symmetry of Eq. 8_fold_symmetry;
 *   - E_J and E_K of SI Eq. si_E_J_K and their nuclear gradient with all four
 *     centres differentiated (SI Sec. 1.4), NOT the bra-only shortcut of
 *     SI Eq. si_dE_J / si_dE_K, so that the shortcut gets checked;
 *   - one-electron overlap (Eq. overlap_definition), used to pin the ERIs and
 *     normalisation;
 *   - point-charge attraction (Eq. v1e_definition2) by the Obara-Saika
 *     three-centre recurrence, the matrix V = sum_C q_C (m|1/|r-C||n)
 *     (Eq. v1e_definition) and the gradient of sum D_mn V_mn with respect to
 *     the basis centres and the charge positions (SI Sec. 1.3);
 *   - the long-range operator erf(omega r)/r (Sec. 2.5,
 *     Eq. eri_longrange_definition) in place of 1/r in every ERI, J, K and
 *     gradient (or_set_omega), through the same recurrences with the
 *     attenuated auxiliary integrals.
 *
 * Readings where the paper is silent:
 *   - normalisation: every primitive component gets
 *     N = (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2i-1)!!(2j-1)!!(2k-1)!!), then each
 *     shell's coefficients are scaled once so the contracted (l,0,0) component
 *     has unit self-overlap;
 *   - Cartesian components in lexicographic order (xx,xy,xz,yy,yz,zz; ...);
 *   - Schwarz Q_ab = sqrt(max_{mu in a, nu in b} |(mu nu|mu nu)|) computed in
 *     FP64, rounded to float32 toward +infinity; a quartet is kept iff
 *     (double)Q_ab * (double)Q_cd >= thresh.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * (quadrature, closed forms, sum rules, invariances, finite differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_LMAX 3
#define OR_PI_L 3.141592653589793238462643383279502884L
#define OR_PI 3.141592653589793238462643383279502884

/* ------------------------------------------------------------------------ */
/* Cartesian component bookkeeping                                           */
/* ------------------------------------------------------------------------ */

static int ncart(int l) { return l < 0 ? 0 : (l + 1) * (l + 2) / 2; }
/* number of exponent triples (x,y,z) with x+y+z <= n */
static int ncart_cum(int n) { return n < 0 ? 0 : (n + 1) * (n + 2) * (n + 3) / 6; }
/* position of (x,y,z) inside its shell, lexicographic order (x desc, y desc) */
static int cart_in_shell(int x, int y, int z) {
  int r = y + z;
  (void)x;
  return r * (r + 1) / 2 + z;
}
/* position of (x,y,z) among all triples with sum <= x+y+z, grouped by sum */
static int cart_global(int x, int y, int z) {
  return ncart_cum(x + y + z - 1) + cart_in_shell(x, y, z);
}
/* the k-th component of shell l */
static void cart_comp(int l, int k, int c[3]) {
  int idx = 0;
  for (int x = l; x >= 0; --x)
    for (int y = l - x; y >= 0; --y) {
      if (idx == k) {
        c[0] = x; c[1] = y; c[2] = l - x - y;
        return;
      }
      ++idx;
    }
}
/* the k-th triple in global order */
static void cart_comp_global(int k, int c[3]) {
  int n = 0;
  while (ncart_cum(n) <= k) ++n;
  cart_comp(n, k - ncart_cum(n - 1), c);
}

static double dfact(int n) { /* n!!, with (-1)!! = 1 */
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

/* ------------------------------------------------------------------------ */
/* Boys function, Eq. boys_function: F_m(x) = int_0^1 t^(2m) exp(-x t^2) dt  */
/* x < 30 : F_m(x) = exp(-x) sum_k (2x)^k / ((2m+1)(2m+3)...(2m+2k+1))        */
/* x >= 30: F_0 = (1/2) sqrt(pi/x) erf(sqrt(x)), then                          */
/*          F_{m+1} = ((2m+1) F_m - exp(-x)) / (2x)                            */
/* ------------------------------------------------------------------------ */

void or_boys(int mmax, double x, double* F) {
  long double X = x;
  if (x < 30.0) {
    long double ex = expl(-X);
    for (int m = 0; m <= mmax; ++m) {
      long double term = 1.0L / (2 * m + 1), sum = term;
      for (int k = 1; k < 4000; ++k) {
        term *= 2.0L * X / (long double)(2 * m + 2 * k + 1);
        sum += term;
        if (term < 1e-24L * sum) break;
      }
      F[m] = (double)(ex * sum);
    }
  } else {
    long double ex = expl(-X);
    long double f = 0.5L * sqrtl(OR_PI_L / X) * erfl(sqrtl(X));
    F[0] = (double)f;
    for (int m = 0; m < mmax; ++m) {
      f = ((2 * m + 1) * f - ex) / (2.0L * X);
      F[m + 1] = (double)f;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Primitive integrals over unnormalised Cartesian Gaussians                  */
/* G(r) = (x-Ax)^i (y-Ay)^j (z-Az)^k exp(-a |r-A|^2)                          */
/* ------------------------------------------------------------------------ */

/* Obara-Saika 1-D overlap table s[i][j], i<=la, j<=lb (row stride lb+1). */
static void os_overlap_1d(int la, int lb, double a, double b, double A, double B, double* s) {
  double p = a + b, P = (a * A + b * B) / p;
  double PA = P - A, PB = P - B, o2p = 0.5 / p;
  int w = lb + 1;
  s[0] = sqrt(OR_PI / p) * exp(-a * b / p * (A - B) * (A - B));
  for (int i = 0; i <= la; ++i)
    for (int j = 0; j <= lb; ++j) {
      if (i == 0 && j == 0) continue;
      double v;
      if (i > 0) {
        v = PA * s[(i - 1) * w + j];
        if (i > 1) v += o2p * (i - 1) * s[(i - 2) * w + j];
        if (j > 0) v += o2p * j * s[(i - 1) * w + j - 1];
      } else {
        v = PB * s[i * w + j - 1];
        if (j > 1) v += o2p * (j - 1) * s[i * w + j - 2];
      }
      s[i * w + j] = v;
    }
}

/* primitive overlap block out[na][nb] */
void or_prim_overlap(int la, int lb, double a, double b, const double* A, const double* B, double* out) {
  double sx[64], sy[64], sz[64];
  os_overlap_1d(la, lb, a, b, A[0], B[0], sx);
  os_overlap_1d(la, lb, a, b, A[1], B[1], sy);
  os_overlap_1d(la, lb, a, b, A[2], B[2], sz);
  int na = ncart(la), nb = ncart(lb), w = lb + 1;
  for (int ia = 0; ia < na; ++ia) {
    int ca[3];
    cart_comp(la, ia, ca);
    for (int ib = 0; ib < nb; ++ib) {
      int cb[3];
      cart_comp(lb, ib, cb);
      out[ia * nb + ib] = sx[ca[0] * w + cb[0]] * sy[ca[1] * w + cb[1]] * sz[ca[2] * w + cb[2]];
    }
  }
}

/*
 * Head-Gordon-Pople horizontal recurrence
 *   (a, b+1_i| = (a+1_i, b| + AB_i (a, b|
 * in:  [nouter][ncart_cum(E)][ninner], indexed by global triple of a (|a|<=E)
 * out: [nouter][ncart(la)][ncart(lb)][ninner], E = la+lb
 */
static void hrr(int la, int lb, const double AB[3], int nouter, int ninner, const double* in, double* out) {
  int E = la + lb, nE = ncart_cum(E);
  int na = ncart(la), nb = ncart(lb);
  for (int o = 0; o < nouter; ++o) {
    /* cur[a_glob][b_in_level][inner] for the current |b| */
    double* cur = (double*)malloc(sizeof(double) * nE * 1 * ninner);
    memcpy(cur, in + (size_t)o * nE * ninner, sizeof(double) * nE * ninner);
    for (int nbv = 0; nbv < lb; ++nbv) {
      int nbc = ncart(nbv), nbn = ncart(nbv + 1);
      double* nxt = (double*)calloc((size_t)nE * nbn * ninner, sizeof(double));
      for (int jb = 0; jb < nbn; ++jb) {
        int b1[3];
        cart_comp(nbv + 1, jb, b1);
        int dir = b1[0] > 0 ? 0 : (b1[1] > 0 ? 1 : 2);
        int b0[3] = {b1[0], b1[1], b1[2]};
        b0[dir] -= 1;
        int ib0 = cart_in_shell(b0[0], b0[1], b0[2]);
        /* |a| runs over la .. E-(nbv+1) */
        for (int ka = ncart_cum(la - 1); ka < ncart_cum(E - nbv - 1); ++ka) {
          int a[3];
          cart_comp_global(ka, a);
          int ap[3] = {a[0], a[1], a[2]};
          ap[dir] += 1;
          int kap = cart_global(ap[0], ap[1], ap[2]);
          for (int t = 0; t < ninner; ++t)
            nxt[((size_t)ka * nbn + jb) * ninner + t] =
                cur[((size_t)kap * nbc + ib0) * ninner + t] + AB[dir] * cur[((size_t)ka * nbc + ib0) * ninner + t];
        }
      }
      free(cur);
      cur = nxt;
    }
    /* cur now [a_glob][ncart(lb)][inner]; keep |a| == la */
    for (int ia = 0; ia < na; ++ia) {
      int a[3];
      cart_comp(la, ia, a);
      int ka = cart_global(a[0], a[1], a[2]);
      for (int ib = 0; ib < nb; ++ib)
        for (int t = 0; t < ninner; ++t)
          out[(((size_t)o * na + ia) * nb + ib) * ninner + t] = cur[((size_t)ka * nb + ib) * ninner + t];
    }
    free(cur);
  }
}

/*
 * Primitive ERI block [ab|cd], out[na][nb][nc][nd], by Obara-Saika:
 *   [00|00]^(m) = 2 pi^(5/2) / (p q sqrt(p+q)) K_AB K_CD F_m(rho |PQ|^2)
 *   bra VRR  [e+1_i,0|00]^(m) = PA_i [e0|00]^(m) + WP_i [e0|00]^(m+1)
 *                               + e_i/(2p) ([e-1_i,0|00]^(m) - rho/p [e-1_i,0|00]^(m+1))
 *   ket VRR  [e0|f+1_i,0]^(m) = QC_i [e0|f0]^(m) + WQ_i [e0|f0]^(m+1)
 *                               + f_i/(2q) ([e0|f-1_i,0]^(m) - rho/q [e0|f-1_i,0]^(m+1))
 *                               + e_i/(2(p+q)) [e-1_i,0|f0]^(m+1)
 * then HRR on the bra and on the ket.  The base case is Eq. eri_base_case.
 */
static void prim_eri_op(int la, int lb, int lc, int ld, double a, double b, double c, double d, const double* A,
                        const double* B, const double* C, const double* D, double omega, double* out) {
  int E = la + lb, F = lc + ld, L = E + F;
  double p = a + b, q = c + d, rho = p * q / (p + q);
  double P[3], Q[3], W[3], PA[3], WP[3], QC[3], WQ[3], AB[3], CD[3];
  double ab2 = 0, cd2 = 0, pq2 = 0;
  for (int i = 0; i < 3; ++i) {
    P[i] = (a * A[i] + b * B[i]) / p;
    Q[i] = (c * C[i] + d * D[i]) / q;
    W[i] = (p * P[i] + q * Q[i]) / (p + q);
    PA[i] = P[i] - A[i];
    WP[i] = W[i] - P[i];
    QC[i] = Q[i] - C[i];
    WQ[i] = W[i] - Q[i];
    AB[i] = A[i] - B[i];
    CD[i] = C[i] - D[i];
    ab2 += AB[i] * AB[i];
    cd2 += CD[i] * CD[i];
    pq2 += (P[i] - Q[i]) * (P[i] - Q[i]);
  }
  double Fm[32];
  double pref = 2.0 * pow(OR_PI, 2.5) / (p * q * sqrt(p + q)) * exp(-a * b / p * ab2) * exp(-c * d / q * cd2);
  if (omega > 0.0) {
    /* erf(omega r)/r (Eq. eri_longrange_definition): writing the operator as
     * (2/sqrt(pi)) int_0^omega exp(-t^2 r^2) dt and following the Coulomb
     * derivation, the u = t/sqrt(rho + t^2) integral of the Boys function stops
     * at u_max^2 = s = omega^2/(omega^2 + rho), so the auxiliary integrals become
     *   [00|00]^(m) = pref * s^(m + 1/2) * F_m(s * rho |PQ|^2)
     * (the prefactor and argument of Eq. eri_longrange_formula); the
     * recurrences below act on the auxiliaries and do not change. */
    double sw = omega * omega / (omega * omega + rho);
    or_boys(L, sw * rho * pq2, Fm);
    pref *= sqrt(sw);
    double sm = 1.0;
    for (int m = 0; m <= L; ++m) {
      Fm[m] *= sm;
      sm *= sw;
    }
  } else {
    or_boys(L, rho * pq2, Fm);
  }

  int nE = ncart_cum(E), nF = ncart_cum(F), nm = L + 1;
  double* V = (double*)calloc((size_t)nE * nF * nm, sizeof(double));
#define VV(ie, jf, m) V[((size_t)(ie) * nF + (jf)) * nm + (m)]
  for (int m = 0; m <= L; ++m) VV(0, 0, m) = pref * Fm[m];
  /* bra VRR with f = 0 */
  for (int ie = 1; ie < nE; ++ie) {
    int e[3];
    cart_comp_global(ie, e);
    int ne = e[0] + e[1] + e[2];
    int i = e[0] > 0 ? 0 : (e[1] > 0 ? 1 : 2);
    int e1[3] = {e[0], e[1], e[2]};
    e1[i] -= 1; /* e = e1 + 1_i */
    int k1 = cart_global(e1[0], e1[1], e1[2]);
    int k2 = -1;
    if (e1[i] > 0) {
      int e2[3] = {e1[0], e1[1], e1[2]};
      e2[i] -= 1;
      k2 = cart_global(e2[0], e2[1], e2[2]);
    }
    for (int m = 0; m <= L - ne; ++m) {
      double v = PA[i] * VV(k1, 0, m) + WP[i] * VV(k1, 0, m + 1);
      if (k2 >= 0) v += e1[i] / (2.0 * p) * (VV(k2, 0, m) - rho / p * VV(k2, 0, m + 1));
      VV(ie, 0, m) = v;
    }
  }
  /* ket VRR with the electron-transfer term */
  for (int jf = 1; jf < nF; ++jf) {
    int f[3];
    cart_comp_global(jf, f);
    int nf = f[0] + f[1] + f[2];
    int i = f[0] > 0 ? 0 : (f[1] > 0 ? 1 : 2);
    int f1[3] = {f[0], f[1], f[2]};
    f1[i] -= 1;
    int j1 = cart_global(f1[0], f1[1], f1[2]);
    int j2 = -1;
    if (f1[i] > 0) {
      int f2[3] = {f1[0], f1[1], f1[2]};
      f2[i] -= 1;
      j2 = cart_global(f2[0], f2[1], f2[2]);
    }
    for (int ie = 0; ie < nE; ++ie) {
      int e[3];
      cart_comp_global(ie, e);
      int ne = e[0] + e[1] + e[2];
      int ke = -1;
      if (e[i] > 0) {
        int e1[3] = {e[0], e[1], e[2]};
        e1[i] -= 1;
        ke = cart_global(e1[0], e1[1], e1[2]);
      }
      for (int m = 0; m <= L - ne - nf; ++m) {
        double v = QC[i] * VV(ie, j1, m) + WQ[i] * VV(ie, j1, m + 1);
        if (j2 >= 0) v += f1[i] / (2.0 * q) * (VV(ie, j2, m) - rho / q * VV(ie, j2, m + 1));
        if (ke >= 0) v += e[i] / (2.0 * (p + q)) * VV(ke, j1, m + 1);
        VV(ie, jf, m) = v;
      }
    }
  }
  /* (e0|f0) at m = 0, laid out [ie][jf] */
  double* T = (double*)malloc(sizeof(double) * nE * nF);
  for (int ie = 0; ie < nE; ++ie)
    for (int jf = 0; jf < nF; ++jf) T[(size_t)ie * nF + jf] = VV(ie, jf, 0);
#undef VV
  free(V);
  int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
  /* bra HRR: [ie][jf] -> [a][b][jf] */
  double* U = (double*)malloc(sizeof(double) * na * nb * nF);
  hrr(la, lb, AB, 1, nF, T, U);
  free(T);
  /* ket HRR: [ab][jf] -> [ab][c][d] */
  hrr(lc, ld, CD, na * nb, 1, U, out);
  free(U);
}

/* Primitive Coulomb ERI [ab|cd], out[na][nb][nc][nd] (Eq. eri_definition). */
void or_prim_eri(int la, int lb, int lc, int ld, double a, double b, double c, double d, const double* A,
                 const double* B, const double* C, const double* D, double* out) {
  prim_eri_op(la, lb, lc, ld, a, b, c, d, A, B, C, D, 0.0, out);
}

/* Primitive long-range ERI [ab| erf(omega r)/r |cd] (Eq. eri_longrange_definition), omega > 0. */
void or_prim_eri_erf(int la, int lb, int lc, int ld, double a, double b, double c, double d, const double* A,
                     const double* B, const double* C, const double* D, double omega, double* out) {
  prim_eri_op(la, lb, lc, ld, a, b, c, d, A, B, C, D, omega, out);
}

/*
 * Primitive point-charge attraction (a| 1/|r-C| |b), out[na][nb], unit charge,
 * Eq. v1e_definition2, by the Obara-Saika three-centre recurrence:
 *   Theta^(m)_00 = (2 pi / p) K_AB F_m(p |PC|^2)       (Eq. v1e_base_case)
 *   Theta^(m)_{e+1_i} = PA_i Theta^(m)_e - PC_i Theta^(m+1)_e
 *                       + e_i/(2p) (Theta^(m)_{e-1_i} - Theta^(m+1)_{e-1_i})
 * then HRR.
 */
void or_prim_nuclear(int la, int lb, double a, double b, const double* A, const double* B, const double* C,
                     double* out) {
  int E = la + lb;
  double p = a + b, P[3], PA[3], PC[3], AB[3], ab2 = 0, pc2 = 0;
  for (int i = 0; i < 3; ++i) {
    P[i] = (a * A[i] + b * B[i]) / p;
    PA[i] = P[i] - A[i];
    PC[i] = P[i] - C[i];
    AB[i] = A[i] - B[i];
    ab2 += AB[i] * AB[i];
    pc2 += PC[i] * PC[i];
  }
  double Fm[32];
  or_boys(E, p * pc2, Fm);
  double pref = 2.0 * OR_PI / p * exp(-a * b / p * ab2);
  int nE = ncart_cum(E), nm = E + 1;
  double* V = (double*)calloc((size_t)nE * nm, sizeof(double));
  for (int m = 0; m <= E; ++m) V[m] = pref * Fm[m];
  for (int ie = 1; ie < nE; ++ie) {
    int e[3];
    cart_comp_global(ie, e);
    int ne = e[0] + e[1] + e[2];
    int i = e[0] > 0 ? 0 : (e[1] > 0 ? 1 : 2);
    int e1[3] = {e[0], e[1], e[2]};
    e1[i] -= 1;
    int k1 = cart_global(e1[0], e1[1], e1[2]);
    int k2 = -1;
    if (e1[i] > 0) {
      int e2[3] = {e1[0], e1[1], e1[2]};
      e2[i] -= 1;
      k2 = cart_global(e2[0], e2[1], e2[2]);
    }
    for (int m = 0; m <= E - ne; ++m) {
      double v = PA[i] * V[k1 * nm + m] - PC[i] * V[k1 * nm + m + 1];
      if (k2 >= 0) v += e1[i] / (2.0 * p) * (V[k2 * nm + m] - V[k2 * nm + m + 1]);
      V[ie * nm + m] = v;
    }
  }
  double* T = (double*)malloc(sizeof(double) * nE);
  for (int ie = 0; ie < nE; ++ie) T[ie] = V[ie * nm];
  free(V);
  hrr(la, lb, AB, 1, 1, T, out);
  free(T);
}

/* ------------------------------------------------------------------------ */
/* Basis: shells, normalisation                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
  int nshell, natom, nbf;
  int *atom, *l, *nprim, *poff, *aoff;
  double* exps;
  double* cn;     /* coefficient of the normalised (l,0,0) component, per primitive */
  double* coords; /* natom*3 */
  double omega;   /* 0: Coulomb 1/r; > 0: erf(omega r)/r (or_set_omega) */
} or_ctx;

static double norm_l00(double alpha, int l) {
  return pow(2.0 * alpha / OR_PI, 0.75) * pow(4.0 * alpha, 0.5 * l) / sqrt(dfact(2 * l - 1));
}
/* ratio between the norm of component (x,y,z) and of (l,0,0); exponent-free */
static double comp_factor(int x, int y, int z) {
  int l = x + y + z;
  return sqrt(dfact(2 * l - 1) / (dfact(2 * x - 1) * dfact(2 * y - 1) * dfact(2 * z - 1)));
}

void* or_create(int nshell, int natom, const int32_t* atom, const int32_t* l, const int32_t* nprim,
                const int32_t* poff, const double* exps, const double* coefs, const double* coords) {
  or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
  c->nshell = nshell;
  c->natom = natom;
  c->atom = (int*)malloc(sizeof(int) * nshell);
  c->l = (int*)malloc(sizeof(int) * nshell);
  c->nprim = (int*)malloc(sizeof(int) * nshell);
  c->poff = (int*)malloc(sizeof(int) * nshell);
  c->aoff = (int*)malloc(sizeof(int) * (nshell + 1));
  int ntot = 0, nbf = 0;
  for (int s = 0; s < nshell; ++s) {
    c->atom[s] = atom[s];
    c->l[s] = l[s];
    c->nprim[s] = nprim[s];
    c->poff[s] = poff[s];
    c->aoff[s] = nbf;
    nbf += ncart(l[s]);
    if (poff[s] + nprim[s] > ntot) ntot = poff[s] + nprim[s];
  }
  c->aoff[nshell] = nbf;
  c->nbf = nbf;
  c->exps = (double*)malloc(sizeof(double) * ntot);
  c->cn = (double*)malloc(sizeof(double) * ntot);
  memcpy(c->exps, exps, sizeof(double) * ntot);
  c->coords = (double*)malloc(sizeof(double) * natom * 3);
  memcpy(c->coords, coords, sizeof(double) * natom * 3);
  /* per-primitive norm, then rescale so the contracted (l,0,0) has unit norm */
  for (int s = 0; s < nshell; ++s) {
    int L = l[s], o = poff[s], np = nprim[s];
    for (int k = 0; k < np; ++k) c->cn[o + k] = coefs[o + k] * norm_l00(exps[o + k], L);
    double zero[3] = {0, 0, 0}, S = 0.0;
    double* blk = (double*)malloc(sizeof(double) * ncart(L) * ncart(L));
    for (int k1 = 0; k1 < np; ++k1)
      for (int k2 = 0; k2 < np; ++k2) {
        or_prim_overlap(L, L, exps[o + k1], exps[o + k2], zero, zero, blk);
        S += c->cn[o + k1] * c->cn[o + k2] * blk[0]; /* (l,0,0) with itself */
      }
    free(blk);
    double sc = 1.0 / sqrt(S);
    for (int k = 0; k < np; ++k) c->cn[o + k] *= sc;
  }
  return c;
}

void or_destroy(void* h) {
  or_ctx* c = (or_ctx*)h;
  if (!c) return;
  free(c->atom); free(c->l); free(c->nprim); free(c->poff); free(c->aoff);
  free(c->exps); free(c->cn); free(c->coords);
  free(c);
}

void or_set_coords(void* h, const double* coords) {
  or_ctx* c = (or_ctx*)h;
  memcpy(c->coords, coords, sizeof(double) * c->natom * 3);
}

/* Two-electron operator of every ERI, J, K and gradient below: omega = 0 is the
 * Coulomb operator 1/r, omega > 0 the long-range erf(omega r)/r of
 * Eq. eri_longrange_definition.  The Schwarz bounds (or_schwarz) stay those of
 * 1/r: erfc(omega r)/r is a positive-definite kernel too, so
 * (ab|erf|ab) <= (ab|ab) and the Coulomb Q bound the attenuated quartets. */
void or_set_omega(void* h, double omega) { ((or_ctx*)h)->omega = omega > 0.0 ? omega : 0.0; }

int or_nbf(void* h) { return ((or_ctx*)h)->nbf; }
void or_ao_offsets(void* h, int32_t* out) {
  or_ctx* c = (or_ctx*)h;
  for (int s = 0; s <= c->nshell; ++s) out[s] = c->aoff[s];
}
void or_norm_coefs(void* h, double* out) {
  or_ctx* c = (or_ctx*)h;
  for (int s = 0; s < c->nshell; ++s)
    for (int k = 0; k < c->nprim[s]; ++k) out[c->poff[s] + k] = c->cn[c->poff[s] + k];
}

static const double* ctr(const or_ctx* c, int s) { return c->coords + 3 * c->atom[s]; }

/* contracted, normalised overlap block S[na][nb] (Eq. overlap_definition) */
void or_overlap_block(void* h, int sa, int sb, double* out) {
  or_ctx* c = (or_ctx*)h;
  int la = c->l[sa], lb = c->l[sb], na = ncart(la), nb = ncart(lb);
  double* blk = (double*)malloc(sizeof(double) * na * nb);
  for (int i = 0; i < na * nb; ++i) out[i] = 0.0;
  for (int ka = 0; ka < c->nprim[sa]; ++ka)
    for (int kb = 0; kb < c->nprim[sb]; ++kb) {
      int pa = c->poff[sa] + ka, pb = c->poff[sb] + kb;
      or_prim_overlap(la, lb, c->exps[pa], c->exps[pb], ctr(c, sa), ctr(c, sb), blk);
      double w = c->cn[pa] * c->cn[pb];
      for (int i = 0; i < na * nb; ++i) out[i] += w * blk[i];
    }
  for (int ia = 0; ia < na; ++ia) {
    int ca[3];
    cart_comp(la, ia, ca);
    for (int ib = 0; ib < nb; ++ib) {
      int cb[3];
      cart_comp(lb, ib, cb);
      out[ia * nb + ib] *= comp_factor(ca[0], ca[1], ca[2]) * comp_factor(cb[0], cb[1], cb[2]);
    }
  }
  free(blk);
}

/* contracted, normalised point-charge attraction block V[na][nb], charge at C */
void or_nuclear_block(void* h, int sa, int sb, const double* C, double* out) {
  or_ctx* c = (or_ctx*)h;
  int la = c->l[sa], lb = c->l[sb], na = ncart(la), nb = ncart(lb);
  double* blk = (double*)malloc(sizeof(double) * na * nb);
  for (int i = 0; i < na * nb; ++i) out[i] = 0.0;
  for (int ka = 0; ka < c->nprim[sa]; ++ka)
    for (int kb = 0; kb < c->nprim[sb]; ++kb) {
      int pa = c->poff[sa] + ka, pb = c->poff[sb] + kb;
      or_prim_nuclear(la, lb, c->exps[pa], c->exps[pb], ctr(c, sa), ctr(c, sb), C, blk);
      double w = c->cn[pa] * c->cn[pb];
      for (int i = 0; i < na * nb; ++i) out[i] += w * blk[i];
    }
  for (int ia = 0; ia < na; ++ia) {
    int ca[3];
    cart_comp(la, ia, ca);
    for (int ib = 0; ib < nb; ++ib) {
      int cb[3];
      cart_comp(lb, ib, cb);
      out[ia * nb + ib] *= comp_factor(ca[0], ca[1], ca[2]) * comp_factor(cb[0], cb[1], cb[2]);
    }
  }
  free(blk);
}

static void apply_comp_factors(int la, int lb, int lc, int ld, double* out) {
  int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
  for (int ia = 0; ia < na; ++ia) {
    int ca[3];
    cart_comp(la, ia, ca);
    double fa = comp_factor(ca[0], ca[1], ca[2]);
    for (int ib = 0; ib < nb; ++ib) {
      int cb[3];
      cart_comp(lb, ib, cb);
      double fb = comp_factor(cb[0], cb[1], cb[2]);
      for (int ic = 0; ic < nc; ++ic) {
        int cc[3];
        cart_comp(lc, ic, cc);
        double fc = comp_factor(cc[0], cc[1], cc[2]);
        for (int id = 0; id < nd; ++id) {
          int cd[3];
          cart_comp(ld, id, cd);
          double fd = comp_factor(cd[0], cd[1], cd[2]);
          out[((ia * nb + ib) * nc + ic) * nd + id] *= fa * fb * fc * fd;
        }
      }
    }
  }
}

/* contracted, normalised ERI block (ab|cd) of the operator selected by omega */
static void eri_block_op(or_ctx* c, int sa, int sb, int sc, int sd, double omega, double* out) {
  int la = c->l[sa], lb = c->l[sb], lc = c->l[sc], ld = c->l[sd];
  int n = ncart(la) * ncart(lb) * ncart(lc) * ncart(ld);
  double* blk = (double*)malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) out[i] = 0.0;
  for (int ka = 0; ka < c->nprim[sa]; ++ka)
    for (int kb = 0; kb < c->nprim[sb]; ++kb)
      for (int kc = 0; kc < c->nprim[sc]; ++kc)
        for (int kd = 0; kd < c->nprim[sd]; ++kd) {
          int pa = c->poff[sa] + ka, pb = c->poff[sb] + kb, pc = c->poff[sc] + kc, pd = c->poff[sd] + kd;
          prim_eri_op(la, lb, lc, ld, c->exps[pa], c->exps[pb], c->exps[pc], c->exps[pd], ctr(c, sa), ctr(c, sb),
                      ctr(c, sc), ctr(c, sd), omega, blk);
          double w = c->cn[pa] * c->cn[pb] * c->cn[pc] * c->cn[pd];
          for (int i = 0; i < n; ++i) out[i] += w * blk[i];
        }
  apply_comp_factors(la, lb, lc, ld, out);
  free(blk);
}

/* contracted, normalised ERI block (ab|cd), out[na][nb][nc][nd], of the
 * context's operator (or_set_omega) */
void or_eri_block(void* h, int sa, int sb, int sc, int sd, double* out) {
  or_ctx* c = (or_ctx*)h;
  eri_block_op(c, sa, sb, sc, sd, c->omega, out);
}

/* ------------------------------------------------------------------------ */
/* Schwarz bounds and lists (Eq. cauchy_schwarz_bound, Eq. kernel_upperbound) */
/* ------------------------------------------------------------------------ */

static float round_up_f32(double x) {
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, INFINITY);
  return f;
}
static int pair_index(int a, int b) { return a >= b ? a * (a + 1) / 2 + b : b * (b + 1) / 2 + a; }
static int pair_class(int la, int lb) {
  int hi = la > lb ? la : lb, lo = la > lb ? lb : la;
  return hi * (hi + 1) / 2 + lo;
}

/* Q[pair_index(a,b)] for all a >= b, float32 rounded toward +infinity */
void or_schwarz(void* h, float* Q) {
  or_ctx* c = (or_ctx*)h;
  int ns = c->nshell;
#pragma omp parallel for schedule(dynamic)
  for (int a = 0; a < ns; ++a) {
    for (int b = 0; b <= a; ++b) {
      int na = ncart(c->l[a]), nb = ncart(c->l[b]);
      double* blk = (double*)malloc(sizeof(double) * na * nb * na * nb);
      eri_block_op(c, a, b, a, b, 0.0, blk); /* Coulomb Q, whatever the operator */
      double mx = 0.0;
      for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j) {
          double v = fabs(blk[((i * nb + j) * na + i) * nb + j]);
          if (v > mx) mx = v;
        }
      free(blk);
      Q[pair_index(a, b)] = round_up_f32(sqrt(mx));
    }
  }
}

/*
 * Lists from float32 Q: sig[pair] = 1 iff (double)Q*(double)Qmax >= thresh;
 * counts[pair*10 + cls] = number of pairs of class cls significant with it.
 */
void or_lists(void* h, double thresh, const float* Q, int32_t* sig, int32_t* counts) {
  or_ctx* c = (or_ctx*)h;
  int ns = c->nshell, np = ns * (ns + 1) / 2;
  double qmax = 0.0;
  for (int i = 0; i < np; ++i)
    if ((double)Q[i] > qmax) qmax = (double)Q[i];
  int* cls = (int*)malloc(sizeof(int) * np);
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b <= a; ++b) cls[pair_index(a, b)] = pair_class(c->l[a], c->l[b]);
  for (int i = 0; i < np; ++i) sig[i] = ((double)Q[i] * qmax >= thresh) ? 1 : 0;
  for (int i = 0; i < np; ++i) {
    for (int k = 0; k < 10; ++k) counts[i * 10 + k] = 0;
    if (!sig[i]) continue;
    for (int j = 0; j < np; ++j)
      if (sig[j] && (double)Q[i] * (double)Q[j] >= thresh) counts[i * 10 + cls[j]] += 1;
  }
  free(cls);
}

/* ------------------------------------------------------------------------ */
/* J and K (Eq. j_definition, Eq. k_definition)                               */
/* ------------------------------------------------------------------------ */

static int quartet_kept(const float* Q, double thresh, int a, int b, int cc, int d) {
  return (double)Q[pair_index(a, b)] * (double)Q[pair_index(cc, d)] >= thresh;
}

/*
 * mode 0: every ordered shell quartet, J_mn += (mn|ls) D_ls, K_ml += (mn|ls) D_ns.
 * mode 1: canonical quartets a>=b, c>=d, pair(ab)>=pair(cd), scaled by
 *         w = 1/2^[a=b] 1/2^[c=d] 1/2^[ab=cd] and scattered into all eight index
 *         permutations of Eq. 8_fold_symmetry.
 * J or K may be NULL.  Q: float32 Schwarz bounds (or_schwarz layout).
 */
void or_jk(void* h, const double* Dm, double thresh, const float* Q, int mode, double* J, double* K) {
  or_ctx* c = (or_ctx*)h;
  int ns = c->nshell, n = c->nbf;
  if (J) memset(J, 0, sizeof(double) * n * n);
  if (K) memset(K, 0, sizeof(double) * n * n);
#pragma omp parallel
  {
    double* Jt = (double*)calloc((size_t)n * n, sizeof(double));
    double* Kt = (double*)calloc((size_t)n * n, sizeof(double));
    double* X = (double*)malloc(sizeof(double) * 10000);
#pragma omp for schedule(dynamic)
    for (int a = 0; a < ns; ++a) {
      for (int b = 0; b < ns; ++b) {
        if (mode == 1 && b > a) continue;
        for (int cc = 0; cc < ns; ++cc)
          for (int d = 0; d < ns; ++d) {
            if (mode == 1 && (d > cc || pair_index(cc, d) > pair_index(a, b))) continue;
            if (!quartet_kept(Q, thresh, a, b, cc, d)) continue;
            or_eri_block(h, a, b, cc, d, X);
            int na = ncart(c->l[a]), nb = ncart(c->l[b]), nc = ncart(c->l[cc]), nd = ncart(c->l[d]);
            int oa = c->aoff[a], ob = c->aoff[b], oc = c->aoff[cc], od = c->aoff[d];
            double w = 1.0;
            if (mode == 1) {
              if (a == b) w *= 0.5;
              if (cc == d) w *= 0.5;
              if (pair_index(a, b) == pair_index(cc, d)) w *= 0.5;
            }
            for (int i = 0; i < na; ++i)
              for (int j = 0; j < nb; ++j)
                for (int k = 0; k < nc; ++k)
                  for (int l = 0; l < nd; ++l) {
                    double x = w * X[((i * nb + j) * nc + k) * nd + l];
                    int m_ = oa + i, n_ = ob + j, l_ = oc + k, s_ = od + l;
                    if (mode == 0) {
                      Jt[(size_t)m_ * n + n_] += x * Dm[(size_t)l_ * n + s_];
                      Kt[(size_t)m_ * n + l_] += x * Dm[(size_t)n_ * n + s_];
                    } else {
                      /* the eight permutations (mn|ls) (nm|ls) (mn|sl) (nm|sl)
                         (ls|mn) (sl|mn) (ls|nm) (sl|nm) */
                      Jt[(size_t)m_ * n + n_] += x * Dm[(size_t)l_ * n + s_];
                      Jt[(size_t)n_ * n + m_] += x * Dm[(size_t)l_ * n + s_];
                      Jt[(size_t)m_ * n + n_] += x * Dm[(size_t)s_ * n + l_];
                      Jt[(size_t)n_ * n + m_] += x * Dm[(size_t)s_ * n + l_];
                      Jt[(size_t)l_ * n + s_] += x * Dm[(size_t)m_ * n + n_];
                      Jt[(size_t)s_ * n + l_] += x * Dm[(size_t)m_ * n + n_];
                      Jt[(size_t)l_ * n + s_] += x * Dm[(size_t)n_ * n + m_];
                      Jt[(size_t)s_ * n + l_] += x * Dm[(size_t)n_ * n + m_];
                      Kt[(size_t)m_ * n + l_] += x * Dm[(size_t)n_ * n + s_];
                      Kt[(size_t)n_ * n + l_] += x * Dm[(size_t)m_ * n + s_];
                      Kt[(size_t)m_ * n + s_] += x * Dm[(size_t)n_ * n + l_];
                      Kt[(size_t)n_ * n + s_] += x * Dm[(size_t)m_ * n + l_];
                      Kt[(size_t)l_ * n + m_] += x * Dm[(size_t)s_ * n + n_];
                      Kt[(size_t)s_ * n + m_] += x * Dm[(size_t)l_ * n + n_];
                      Kt[(size_t)l_ * n + n_] += x * Dm[(size_t)s_ * n + m_];
                      Kt[(size_t)s_ * n + n_] += x * Dm[(size_t)l_ * n + m_];
                    }
                  }
          }
      }
    }
#pragma omp critical
    {
      for (size_t i = 0; i < (size_t)n * n; ++i) {
        if (J) J[i] += Jt[i];
        if (K) K[i] += Kt[i];
      }
    }
    free(Jt);
    free(Kt);
    free(X);
  }
}

/*
 * J and K contributions of an explicit list of canonical quartets
 * abcd[4q..4q+3] = (a, b, c, d), a>=b, c>=d, pair(ab)>=pair(cd), each scattered
 * into the eight index permutations of Eq. 8_fold_symmetry with the weight
 * w = 1/2^[a=b] 1/2^[c=d] 1/2^[ab=cd] (as mode 1 of or_jk), no screening.
 * J and K are accumulated (+=), so partial lists (one per GPU share of a split
 * build) add up to the whole.  Serial.
 */
void or_jk_quartets(void* h, const double* Dm, int nq, const int* abcd, double* J, double* K) {
  or_ctx* c = (or_ctx*)h;
  int n = c->nbf;
  double* X = (double*)malloc(sizeof(double) * 10000);
  for (int q = 0; q < nq; ++q) {
    int a = abcd[4 * q], b = abcd[4 * q + 1], cc = abcd[4 * q + 2], d = abcd[4 * q + 3];
    or_eri_block(h, a, b, cc, d, X);
    int na = ncart(c->l[a]), nb = ncart(c->l[b]), nc = ncart(c->l[cc]), nd = ncart(c->l[d]);
    int oa = c->aoff[a], ob = c->aoff[b], oc = c->aoff[cc], od = c->aoff[d];
    double w = 1.0;
    if (a == b) w *= 0.5;
    if (cc == d) w *= 0.5;
    if (pair_index(a, b) == pair_index(cc, d)) w *= 0.5;
    for (int i = 0; i < na; ++i)
      for (int j = 0; j < nb; ++j)
        for (int k = 0; k < nc; ++k)
          for (int l = 0; l < nd; ++l) {
            double x = w * X[((i * nb + j) * nc + k) * nd + l];
            int m_ = oa + i, n_ = ob + j, l_ = oc + k, s_ = od + l;
            if (J) {
              J[(size_t)m_ * n + n_] += x * (Dm[(size_t)l_ * n + s_] + Dm[(size_t)s_ * n + l_]);
              J[(size_t)n_ * n + m_] += x * (Dm[(size_t)l_ * n + s_] + Dm[(size_t)s_ * n + l_]);
              J[(size_t)l_ * n + s_] += x * (Dm[(size_t)m_ * n + n_] + Dm[(size_t)n_ * n + m_]);
              J[(size_t)s_ * n + l_] += x * (Dm[(size_t)m_ * n + n_] + Dm[(size_t)n_ * n + m_]);
            }
            if (K) {
              K[(size_t)m_ * n + l_] += x * Dm[(size_t)n_ * n + s_];
              K[(size_t)n_ * n + l_] += x * Dm[(size_t)m_ * n + s_];
              K[(size_t)m_ * n + s_] += x * Dm[(size_t)n_ * n + l_];
              K[(size_t)n_ * n + s_] += x * Dm[(size_t)m_ * n + l_];
              K[(size_t)l_ * n + m_] += x * Dm[(size_t)s_ * n + n_];
              K[(size_t)s_ * n + m_] += x * Dm[(size_t)l_ * n + n_];
              K[(size_t)l_ * n + n_] += x * Dm[(size_t)s_ * n + m_];
              K[(size_t)s_ * n + n_] += x * Dm[(size_t)l_ * n + m_];
            }
          }
  }
  free(X);
}

/* E_J = 1/2 sum D J, E_K = -1/4 sum D K (SI Eq. si_E_J_K), long double sums */
void or_energy(int n, const double* Dm, const double* J, const double* K, double* EJ, double* EK) {
  long double sj = 0.0L, sk = 0.0L;
  for (size_t i = 0; i < (size_t)n * n; ++i) {
    if (J) sj += (long double)Dm[i] * (long double)J[i];
    if (K) sk += (long double)Dm[i] * (long double)K[i];
  }
  if (EJ) *EJ = (double)(0.5L * sj);
  if (EK) *EK = (double)(-0.25L * sk);
}

/*
 * Sampled blocks for large systems.
 * J block (a,b): J_mn = sum over all ordered shells (c,d) of (ab|cd) D_cd.
 * K block (a,c): K_ml = sum over all ordered shells (b,d) of (ab|cd) D_bd.
 * Both with the quartet test on Q.
 */
void or_j_block(void* h, const double* Dm, double thresh, const float* Q, int a, int b, double* out) {
  or_ctx* c = (or_ctx*)h;
  int ns = c->nshell, n = c->nbf, na = ncart(c->l[a]), nb = ncart(c->l[b]);
  for (int i = 0; i < na * nb; ++i) out[i] = 0.0;
#pragma omp parallel
  {
    double* acc = (double*)calloc(na * nb, sizeof(double));
    double* X = (double*)malloc(sizeof(double) * 10000);
#pragma omp for schedule(dynamic)
    for (int cc = 0; cc < ns; ++cc)
      for (int d = 0; d < ns; ++d) {
        if (!quartet_kept(Q, thresh, a, b, cc, d)) continue;
        or_eri_block(h, a, b, cc, d, X);
        int nc = ncart(c->l[cc]), nd = ncart(c->l[d]), oc = c->aoff[cc], od = c->aoff[d];
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nb; ++j)
            for (int k = 0; k < nc; ++k)
              for (int l = 0; l < nd; ++l)
                acc[i * nb + j] += X[((i * nb + j) * nc + k) * nd + l] * Dm[(size_t)(oc + k) * n + od + l];
      }
#pragma omp critical
    for (int i = 0; i < na * nb; ++i) out[i] += acc[i];
    free(acc);
    free(X);
  }
}

void or_k_block(void* h, const double* Dm, double thresh, const float* Q, int a, int cc, double* out) {
  or_ctx* c = (or_ctx*)h;
  int ns = c->nshell, n = c->nbf, na = ncart(c->l[a]), nc = ncart(c->l[cc]);
  for (int i = 0; i < na * nc; ++i) out[i] = 0.0;
#pragma omp parallel
  {
    double* acc = (double*)calloc(na * nc, sizeof(double));
    double* X = (double*)malloc(sizeof(double) * 10000);
#pragma omp for schedule(dynamic)
    for (int b = 0; b < ns; ++b)
      for (int d = 0; d < ns; ++d) {
        if (!quartet_kept(Q, thresh, a, b, cc, d)) continue;
        or_eri_block(h, a, b, cc, d, X);
        int nb = ncart(c->l[b]), nd = ncart(c->l[d]), ob = c->aoff[b], od = c->aoff[d];
        for (int i = 0; i < na; ++i)
          for (int j = 0; j < nb; ++j)
            for (int k = 0; k < nc; ++k)
              for (int l = 0; l < nd; ++l)
                acc[i * nc + k] += X[((i * nb + j) * nc + k) * nd + l] * Dm[(size_t)(ob + j) * n + od + l];
      }
#pragma omp critical
    for (int i = 0; i < na * nc; ++i) out[i] += acc[i];
    free(acc);
    free(X);
  }
}

/* ------------------------------------------------------------------------ */
/* Point-charge attraction matrix and its gradient (Sec. 2.4)                 */
/* ------------------------------------------------------------------------ */

/*
 * Contracted attraction block of shells (sa, sb) with their angular momenta
 * shifted by (da, db) in {-1, 0, +1}, summed over the point charges with
 * weights q, out[ncart(la+da)][ncart(lb+db)].  `wexp` multiplies each
 * primitive term by 2 x exponent of the raised shell (0: none, 1: shell a,
 * 2: shell b) for the raising half of the derivative rule.  No component
 * factors applied (the caller applies the ones of the unshifted functions).
 */
static void nuc_block_shift(const or_ctx* c, int sa, int da, int sb, int db, int nc, const double* q,
                            const double* C, int wexp, double* out) {
  int la = c->l[sa] + da, lb = c->l[sb] + db, na = ncart(la), nb = ncart(lb);
  double* blk = (double*)malloc(sizeof(double) * na * nb);
  for (int i = 0; i < na * nb; ++i) out[i] = 0.0;
  for (int ka = 0; ka < c->nprim[sa]; ++ka)
    for (int kb = 0; kb < c->nprim[sb]; ++kb) {
      int pa = c->poff[sa] + ka, pb = c->poff[sb] + kb;
      double w = c->cn[pa] * c->cn[pb];
      if (wexp == 1) w *= 2.0 * c->exps[pa];
      if (wexp == 2) w *= 2.0 * c->exps[pb];
      for (int k = 0; k < nc; ++k) {
        or_prim_nuclear(la, lb, c->exps[pa], c->exps[pb], ctr(c, sa), ctr(c, sb), C + 3 * k, blk);
        for (int i = 0; i < na * nb; ++i) out[i] += w * q[k] * blk[i];
      }
    }
  free(blk);
}

/*
 * V_mn = sum_C q_C (m| 1/|r - C| |n) (Eq. v1e_definition, Eq. v1e_summation_over_C)
 * over every pair of shells, V nbf x nbf (row-major), charges q[nc] at C[nc*3].
 */
void or_nuclear(void* h, int nc, const double* q, const double* C, double* V) {
  or_ctx* c = (or_ctx*)h;
  int ns = c->nshell, n = c->nbf;
#pragma omp parallel for schedule(dynamic)
  for (int a = 0; a < ns; ++a) {
    double blk[100];
    for (int b = 0; b < ns; ++b) {
      int na = ncart(c->l[a]), nb = ncart(c->l[b]);
      nuc_block_shift(c, a, 0, b, 0, nc, q, C, 0, blk);
      for (int i = 0; i < na; ++i) {
        int ci[3];
        cart_comp(c->l[a], i, ci);
        for (int j = 0; j < nb; ++j) {
          int cj[3];
          cart_comp(c->l[b], j, cj);
          V[(size_t)(c->aoff[a] + i) * n + c->aoff[b] + j] =
              blk[i * nb + j] * comp_factor(ci[0], ci[1], ci[2]) * comp_factor(cj[0], cj[1], cj[2]);
        }
      }
    }
  }
}

/*
 * Gradient of E_V = sum_mn D_mn V_mn (D held fixed): gA[natom*3] with respect
 * to the basis-function centres, gC[nc*3] with respect to the charge positions.
 * Centre A of m and B of n are differentiated by the raising/lowering rule
 * d/dA_t G_i = 2a G_{i+1_t} - i_t G_{i-1_t} at primitive level (each function
 * keeps its own normalisation).  Each term (m, n, C) depends on A, B and C only
 * through their differences, so d/dC_t = -(d/dA_t + d/dB_t) term by term
 * (translational invariance); the finite-difference pins check all three.
 */
void or_nuclear_grad(void* h, const double* Dm, int nc, const double* q, const double* C, double* gA, double* gC) {
  or_ctx* c = (or_ctx*)h;
  int ns = c->nshell, n = c->nbf, nat = c->natom;
  for (int i = 0; i < 3 * nat; ++i) gA[i] = 0.0;
  for (int i = 0; i < 3 * nc; ++i) gC[i] = 0.0;
#pragma omp parallel
  {
    double* tA = (double*)calloc(3 * nat, sizeof(double));
    double* tC = (double*)calloc(3 * (nc > 0 ? nc : 1), sizeof(double));
    double up[150], dn[100];
#pragma omp for schedule(dynamic)
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < ns; ++b)
        for (int k = 0; k < nc; ++k) {
          double g[2][3] = {{0, 0, 0}, {0, 0, 0}}; /* d/dA, d/dB of sum_mn D_mn V_mnC */
          int la = c->l[a], lb = c->l[b], na = ncart(la), nb = ncart(lb);
          for (int side = 0; side < 2; ++side) {
            int lx = side == 0 ? la : lb;
            int nup_a = ncart(la + (side == 0)), nup_b = ncart(lb + (side == 1));
            nuc_block_shift(c, a, side == 0, b, side == 1, 1, q + k, C + 3 * k, side + 1, up);
            int ndn_a = 0, ndn_b = 0;
            if (lx > 0) {
              nuc_block_shift(c, a, -(side == 0), b, -(side == 1), 1, q + k, C + 3 * k, 0, dn);
              ndn_a = ncart(la - (side == 0));
              ndn_b = ncart(lb - (side == 1));
            }
            for (int i = 0; i < na; ++i) {
              int ci[3];
              cart_comp(la, i, ci);
              for (int j = 0; j < nb; ++j) {
                int cj[3];
                cart_comp(lb, j, cj);
                double dmn = Dm[(size_t)(c->aoff[a] + i) * n + c->aoff[b] + j] *
                             comp_factor(ci[0], ci[1], ci[2]) * comp_factor(cj[0], cj[1], cj[2]);
                int* cw = side == 0 ? ci : cj;
                for (int t = 0; t < 3; ++t) {
                  int cu[3] = {cw[0], cw[1], cw[2]};
                  cu[t] += 1;
                  double v;
                  if (side == 0) v = up[cart_in_shell(cu[0], cu[1], cu[2]) * nup_b + j];
                  else v = up[i * nup_b + cart_in_shell(cu[0], cu[1], cu[2])];
                  if (cw[t] > 0) {
                    int cd[3] = {cw[0], cw[1], cw[2]};
                    cd[t] -= 1;
                    if (side == 0) v -= cw[t] * dn[cart_in_shell(cd[0], cd[1], cd[2]) * ndn_b + j];
                    else v -= cw[t] * dn[i * ndn_b + cart_in_shell(cd[0], cd[1], cd[2])];
                  }
                  g[side][t] += dmn * v;
                }
              }
            }
            (void)nup_a;
            (void)ndn_a;
          }
          for (int t = 0; t < 3; ++t) {
            tA[3 * c->atom[a] + t] += g[0][t];
            tA[3 * c->atom[b] + t] += g[1][t];
            tC[3 * k + t] -= g[0][t] + g[1][t];
          }
        }
#pragma omp critical
    {
      for (int i = 0; i < 3 * nat; ++i) gA[i] += tA[i];
      for (int i = 0; i < 3 * nc; ++i) gC[i] += tC[i];
    }
    free(tA);
    free(tC);
  }
}

/* ------------------------------------------------------------------------ */
/* Nuclear gradient of E = E_J + E_K with D held fixed (SI Sec. 1.4)          */
/* ------------------------------------------------------------------------ */

/*
 * d(ab|cd)/dX_t for the centre X of shell `which` (0:a 1:b 2:c 3:d), t = x,y,z,
 * from the raising/lowering rule at primitive level
 *   d/dX_t G(i) = 2 alpha G(i + 1_t) - i_t G(i - 1_t),
 * with each function keeping its own normalisation.  out[3][na nb nc nd].
 */
static void eri_deriv_block(or_ctx* c, int s[4], int which, double* out) {
  int l[4], nn[4];
  for (int k = 0; k < 4; ++k) {
    l[k] = c->l[s[k]];
    nn[k] = ncart(l[k]);
  }
  int n = nn[0] * nn[1] * nn[2] * nn[3];
  for (int i = 0; i < 3 * n; ++i) out[i] = 0.0;
  int lup[4] = {l[0], l[1], l[2], l[3]}, ldn[4] = {l[0], l[1], l[2], l[3]};
  lup[which] += 1;
  ldn[which] -= 1;
  int nup[4], ndn[4];
  for (int k = 0; k < 4; ++k) {
    nup[k] = ncart(lup[k]);
    ndn[k] = ncart(ldn[k]);
  }
  int Nup = nup[0] * nup[1] * nup[2] * nup[3], Ndn = ldn[which] >= 0 ? ndn[0] * ndn[1] * ndn[2] * ndn[3] : 0;
  double* up = (double*)malloc(sizeof(double) * Nup);
  double* dn = (double*)malloc(sizeof(double) * (Ndn > 0 ? Ndn : 1));
  int k4[4];
  for (k4[0] = 0; k4[0] < c->nprim[s[0]]; ++k4[0])
    for (k4[1] = 0; k4[1] < c->nprim[s[1]]; ++k4[1])
      for (k4[2] = 0; k4[2] < c->nprim[s[2]]; ++k4[2])
        for (k4[3] = 0; k4[3] < c->nprim[s[3]]; ++k4[3]) {
          int pp[4];
          double ex[4];
          const double* R[4];
          double w = 1.0;
          for (int k = 0; k < 4; ++k) {
            pp[k] = c->poff[s[k]] + k4[k];
            ex[k] = c->exps[pp[k]];
            R[k] = ctr(c, s[k]);
            w *= c->cn[pp[k]];
          }
          prim_eri_op(lup[0], lup[1], lup[2], lup[3], ex[0], ex[1], ex[2], ex[3], R[0], R[1], R[2], R[3], c->omega,
                      up);
          if (Ndn > 0)
            prim_eri_op(ldn[0], ldn[1], ldn[2], ldn[3], ex[0], ex[1], ex[2], ex[3], R[0], R[1], R[2], R[3],
                        c->omega, dn);
          double alpha = ex[which];
          int idx[4];
          for (idx[0] = 0; idx[0] < nn[0]; ++idx[0])
            for (idx[1] = 0; idx[1] < nn[1]; ++idx[1])
              for (idx[2] = 0; idx[2] < nn[2]; ++idx[2])
                for (idx[3] = 0; idx[3] < nn[3]; ++idx[3]) {
                  int o = ((idx[0] * nn[1] + idx[1]) * nn[2] + idx[2]) * nn[3] + idx[3];
                  int cw[3];
                  cart_comp(l[which], idx[which], cw);
                  for (int t = 0; t < 3; ++t) {
                    int cu[3] = {cw[0], cw[1], cw[2]};
                    cu[t] += 1;
                    int iu[4] = {idx[0], idx[1], idx[2], idx[3]};
                    iu[which] = cart_in_shell(cu[0], cu[1], cu[2]);
                    double v = 2.0 * alpha * up[((iu[0] * nup[1] + iu[1]) * nup[2] + iu[2]) * nup[3] + iu[3]];
                    if (cw[t] > 0) {
                      int cdn[3] = {cw[0], cw[1], cw[2]};
                      cdn[t] -= 1;
                      int id[4] = {idx[0], idx[1], idx[2], idx[3]};
                      id[which] = cart_in_shell(cdn[0], cdn[1], cdn[2]);
                      v -= cw[t] * dn[((id[0] * ndn[1] + id[1]) * ndn[2] + id[2]) * ndn[3] + id[3]];
                    }
                    out[t * n + o] += w * v;
                  }
                }
        }
  for (int t = 0; t < 3; ++t) apply_comp_factors(l[0], l[1], l[2], l[3], out + t * n);
  free(up);
  free(dn);
}

/*
 * grad[natom*3] = dE/dR with E = 1/2 sum D_mn D_ls (mn|ls) - 1/4 sum D_ml D_ns (mn|ls),
 * i.e. sum over every ordered quartet of Gamma_mnls d(mn|ls)/dR with
 * Gamma = 1/2 D_mn D_ls - 1/4 D_ml D_ns, all four centres differentiated.
 * The quartet test uses the given (frozen) Q.  want_j / want_k select terms.
 */
void or_grad(void* h, const double* Dm, double thresh, const float* Q, int want_j, int want_k, double* grad) {
  or_ctx* c = (or_ctx*)h;
  int ns = c->nshell, n = c->nbf, nat = c->natom;
  for (int i = 0; i < nat * 3; ++i) grad[i] = 0.0;
#pragma omp parallel
  {
    double* g = (double*)calloc(nat * 3, sizeof(double));
    double* dX = (double*)malloc(sizeof(double) * 3 * 10000);
#pragma omp for schedule(dynamic)
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < ns; ++b)
        for (int cc = 0; cc < ns; ++cc)
          for (int d = 0; d < ns; ++d) {
            if (!quartet_kept(Q, thresh, a, b, cc, d)) continue;
            int s[4] = {a, b, cc, d};
            int na = ncart(c->l[a]), nb = ncart(c->l[b]), nc = ncart(c->l[cc]), nd = ncart(c->l[d]);
            int nq = na * nb * nc * nd;
            for (int which = 0; which < 4; ++which) {
              eri_deriv_block(c, s, which, dX);
              int atom = c->atom[s[which]];
              for (int i = 0; i < na; ++i)
                for (int j = 0; j < nb; ++j)
                  for (int k = 0; k < nc; ++k)
                    for (int l = 0; l < nd; ++l) {
                      int m_ = c->aoff[a] + i, n_ = c->aoff[b] + j, l_ = c->aoff[cc] + k, s_ = c->aoff[d] + l;
                      double G = 0.0;
                      if (want_j) G += 0.5 * Dm[(size_t)m_ * n + n_] * Dm[(size_t)l_ * n + s_];
                      if (want_k) G -= 0.25 * Dm[(size_t)m_ * n + l_] * Dm[(size_t)n_ * n + s_];
                      int o = ((i * nb + j) * nc + k) * nd + l;
                      for (int t = 0; t < 3; ++t) g[atom * 3 + t] += G * dX[t * nq + o];
                    }
            }
          }
#pragma omp critical
    for (int i = 0; i < nat * 3; ++i) grad[i] += g[i];
    free(g);
    free(dX);
  }
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Evaluate a list of contracted shell quartets (abcd[4*nq], user shell
 * indices) with or_eri_block, OpenMP over quartets; returns sum of |ERI| so the
 * work cannot be skipped.  Used to time the oracle on a sample of a workload.
 */
double or_quartet_batch(void* h, int nq, const int32_t* abcd) {
  double total = 0.0;
#pragma omp parallel reduction(+ : total)
  {
    double* X = (double*)malloc(sizeof(double) * 10000);
#pragma omp for schedule(dynamic, 4)
    for (int q = 0; q < nq; ++q) {
      or_ctx* c = (or_ctx*)h;
      int a = abcd[4 * q], b = abcd[4 * q + 1], cc = abcd[4 * q + 2], d = abcd[4 * q + 3];
      or_eri_block(h, a, b, cc, d, X);
      int n = ncart(c->l[a]) * ncart(c->l[b]) * ncart(c->l[cc]) * ncart(c->l[d]);
      for (int i = 0; i < n; ++i) total += fabs(X[i]);
    }
    free(X);
  }
  return total;
}

/* ======================================================================== */
/* Exchange-correlation quadrature on a molecular grid (Sec. 2.6)           */
/* ======================================================================== */
/*
 * The paper's four steps (Sec. 2.6): (1) a molecular grid, (2) the density
 * and its gradient at every grid point (Eq. xc_density_0, Eq. xc_density_1),
 * (3) the functional at every point, (4) the XC matrix as a weighted sum over
 * the points (Eq. xc_grid_sum_0, Eq. xc_grid_sum_1).  Everything below is the
 * plain definition: basis functions evaluated directly from
 * Eq. contracted_basis, full double sums over (mu, nu), no screening.
 *
 * Readings (the paper names atom-centred standard grids with Becke
 * partitioning, SI Sec. 1.5, but fixes no rule):
 *   - radial rule: Gauss-Chebyshev nodes of the second kind,
 *     x_i = cos(i pi/(n+1)), i = 1..n, mapped by Becke's r = R (1+x)/(1-x);
 *     weight (pi/(n+1)) sin(theta_i) r^2 dr/dx, with dr/dx = 2R/(1-x)^2;
 *   - angular rule: Gauss-Legendre nodes in cos(theta) (ascending) times the
 *     trapezoid rule in phi with 2 n_theta points at phi_k = 2 pi (k+1/2)/n_phi;
 *   - Becke fuzzy cells of equal size: mu_AB = (|r-A| - |r-B|)/|A-B|,
 *     p(mu) = (3 mu - mu^3)/2 applied three times, s = (1 - p)/2,
 *     P_A = prod_{B != A} s(mu_AB), w_A = P_A / sum_B P_B;
 *   - point order g = ((atom * n_rad + (i-1)) * n_theta + j) * n_phi + k;
 *   - the functional (the paper evaluates it on the CPU and names no
 *     functional): closed-shell Slater exchange, or Becke-88 exchange with
 *     beta = 0.0042; points with rho < 1e-14 contribute nothing.
 */

#define OR_XC_RHO_MIN 1e-14

/* Gauss-Legendre nodes (ascending) and weights on [-1, 1]: Newton on P_n */
static void gauss_legendre(int n, double* t, double* w) {
  for (int i = 0; i < n; ++i) {
    long double x = cosl(OR_PI_L * (i + 0.75L) / (n + 0.5L)), dp = 0.0L;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1.0L, p1 = x;
      for (int k = 2; k <= n; ++k) {
        long double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = x; p0 = 1.0L; }
      dp = n * (x * p1 - p0) / (x * x - 1.0L);
      long double dx = p1 / dp;
      x -= dx;
      if (fabsl(dx) < 1e-19L) break;
    }
    {
      long double p0 = 1.0L, p1 = x;
      for (int k = 2; k <= n; ++k) {
        long double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = x; p0 = 1.0L; }
      dp = n * (x * p1 - p0) / (x * x - 1.0L);
    }
    /* cos((i+3/4)pi/(n+1/2)) runs from +1 down: store ascending */
    t[n - 1 - i] = (double)x;
    w[n - 1 - i] = (double)(2.0L / ((1.0L - x * x) * dp * dp));
  }
}

int64_t or_xc_grid_size(void* h, int nrad, int ntheta) {
  or_ctx* c = (or_ctx*)h;
  return (int64_t)c->natom * nrad * ntheta * 2 * ntheta;
}

/* Becke partition weight of atom `own` at point r */
static double becke_weight(const or_ctx* c, int own, const double r[3]) {
  int na = c->natom;
  double sumP = 0.0, Pown = 0.0;
  for (int A = 0; A < na; ++A) {
    const double* RA = c->coords + 3 * A;
    double dA = sqrt((r[0] - RA[0]) * (r[0] - RA[0]) + (r[1] - RA[1]) * (r[1] - RA[1]) +
                     (r[2] - RA[2]) * (r[2] - RA[2]));
    double P = 1.0;
    for (int B = 0; B < na && P != 0.0; ++B) {
      if (B == A) continue;
      const double* RB = c->coords + 3 * B;
      double dB = sqrt((r[0] - RB[0]) * (r[0] - RB[0]) + (r[1] - RB[1]) * (r[1] - RB[1]) +
                       (r[2] - RB[2]) * (r[2] - RB[2]));
      double AB = sqrt((RA[0] - RB[0]) * (RA[0] - RB[0]) + (RA[1] - RB[1]) * (RA[1] - RB[1]) +
                       (RA[2] - RB[2]) * (RA[2] - RB[2]));
      double mu = (dA - dB) / AB;
      for (int it = 0; it < 3; ++it) mu = 1.5 * mu - 0.5 * mu * mu * mu;
      P *= 0.5 * (1.0 - mu);
    }
    sumP += P;
    if (A == own) Pown = P;
  }
  return sumP > 0.0 ? Pown / sumP : 0.0;
}

/* Step (1): points pts[3G] and weights w[G] of the molecular grid */
void or_xc_grid(void* h, int nrad, int ntheta, double R, double* pts, double* w) {
  or_ctx* c = (or_ctx*)h;
  int nphi = 2 * ntheta, nang = ntheta * nphi;
  double* t = (double*)malloc(sizeof(double) * ntheta);
  double* wt = (double*)malloc(sizeof(double) * ntheta);
  gauss_legendre(ntheta, t, wt);
  int64_t G = or_xc_grid_size(h, nrad, ntheta);
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < G; ++g) {
    int64_t q = g;
    int k = (int)(q % nphi); q /= nphi;
    int j = (int)(q % ntheta); q /= ntheta;
    int i = (int)(q % nrad) + 1; q /= nrad;
    int a = (int)q;
    double th = i * OR_PI / (nrad + 1), x = cos(th);
    double r = R * (1.0 + x) / (1.0 - x);
    double wr = OR_PI / (nrad + 1) * sin(th) * r * r * 2.0 * R / ((1.0 - x) * (1.0 - x));
    double ph = 2.0 * OR_PI * (k + 0.5) / nphi, st = sqrt(1.0 - t[j] * t[j]);
    double wa = wt[j] * 2.0 * OR_PI / nphi;
    const double* A = c->coords + 3 * a;
    double p[3] = {A[0] + r * st * cos(ph), A[1] + r * st * sin(ph), A[2] + r * t[j]};
    pts[3 * g] = p[0];
    pts[3 * g + 1] = p[1];
    pts[3 * g + 2] = p[2];
    w[g] = wr * wa * becke_weight(c, a, p);
  }
  (void)nang;
  free(t);
  free(wt);
}

static double ipow(double x, int n) {
  double r = 1.0;
  for (int k = 0; k < n; ++k) r *= x;
  return r;
}

/* values phi[na] (and gradients dphi[3][na] if dphi) of the components of
 * shell s at point r, Eq. contracted_basis with the component norms */
static void ao_shell(const or_ctx* c, int s, const double* r, double* phi, double* dphi) {
  int L = c->l[s], na = ncart(L);
  const double* A = ctr(c, s);
  double d[3] = {r[0] - A[0], r[1] - A[1], r[2] - A[2]};
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double e0 = 0.0, e1 = 0.0; /* sum_k c_k exp(-a r^2) and sum_k c_k a exp(-a r^2) */
  for (int k = 0; k < c->nprim[s]; ++k) {
    double a = c->exps[c->poff[s] + k], e = c->cn[c->poff[s] + k] * exp(-a * r2);
    e0 += e;
    e1 += a * e;
  }
  for (int m = 0; m < na; ++m) {
    int e[3];
    cart_comp(L, m, e);
    double cf = comp_factor(e[0], e[1], e[2]);
    double pw[3] = {ipow(d[0], e[0]), ipow(d[1], e[1]), ipow(d[2], e[2])};
    phi[m] = cf * pw[0] * pw[1] * pw[2] * e0;
    if (dphi) {
      for (int x = 0; x < 3; ++x) {
        int y = (x + 1) % 3, z = (x + 2) % 3;
        /* d/dx [d_x^i exp(-a r^2)] = i d_x^(i-1) exp - 2 a d_x^(i+1) exp */
        double lower = e[x] > 0 ? e[x] * ipow(d[x], e[x] - 1) * e0 : 0.0;
        double upper = 2.0 * ipow(d[x], e[x] + 1) * e1;
        dphi[x * na + m] = cf * (lower - upper) * pw[y] * pw[z];
      }
    }
  }
}

/* every basis function (and gradient, dphi[3][nbf]) at point r */
void or_xc_ao(void* h, const double* r, double* phi, double* dphi) {
  or_ctx* c = (or_ctx*)h;
  int n = c->nbf;
  double buf[10], dbuf[30];
  for (int s = 0; s < c->nshell; ++s) {
    int na = ncart(c->l[s]), o = c->aoff[s];
    ao_shell(c, s, r, buf, dphi ? dbuf : NULL);
    for (int m = 0; m < na; ++m) {
      phi[o + m] = buf[m];
      if (dphi)
        for (int x = 0; x < 3; ++x) dphi[x * n + o + m] = dbuf[x * na + m];
    }
  }
}

/* Step (2): rho(r_g) = sum D_mn phi_m phi_n (Eq. xc_density_0) and
 * grad rho = sum D_mn grad(phi_m phi_n) (Eq. xc_density_1), grad[3G] or NULL */
void or_xc_density(void* h, const double* Dm, int64_t G, const double* pts, double* rho, double* grad) {
  or_ctx* c = (or_ctx*)h;
  int n = c->nbf;
#pragma omp parallel
  {
    double* phi = (double*)malloc(sizeof(double) * n);
    double* dphi = (double*)malloc(sizeof(double) * 3 * n);
#pragma omp for schedule(dynamic, 16)
    for (int64_t g = 0; g < G; ++g) {
      or_xc_ao(h, pts + 3 * g, phi, dphi);
      long double r = 0.0L, gx = 0.0L, gy = 0.0L, gz = 0.0L;
      for (int m = 0; m < n; ++m)
        for (int v = 0; v < n; ++v) {
          double dmv = Dm[(size_t)m * n + v];
          r += dmv * phi[m] * phi[v];
          gx += dmv * (dphi[m] * phi[v] + phi[m] * dphi[v]);
          gy += dmv * (dphi[n + m] * phi[v] + phi[m] * dphi[n + v]);
          gz += dmv * (dphi[2 * n + m] * phi[v] + phi[m] * dphi[2 * n + v]);
        }
      rho[g] = (double)r;
      if (grad) {
        grad[3 * g] = (double)gx;
        grad[3 * g + 1] = (double)gy;
        grad[3 * g + 2] = (double)gz;
      }
    }
    free(phi);
    free(dphi);
  }
}

/* Step (3): energy density eps, v_rho = d eps/d rho and v_grad = d eps/d(grad rho)
 * (3 per point) of functional `kind`: 1 Slater exchange, 2 Becke-88 exchange.
 * Returns 0, or -1 for an unknown kind. */
int or_xc_functional(int kind, int64_t G, const double* rho, const double* grad, double* eps, double* vrho,
                     double* vgrad) {
  if (kind != 1 && kind != 2) return -1;
  const double cx = 0.75 * cbrt(3.0 / OR_PI);        /* closed-shell Slater constant */
  const double cxs = 1.5 * cbrt(3.0 / (4.0 * OR_PI)); /* per-spin Slater constant */
  const double beta = 0.0042;
  for (int64_t g = 0; g < G; ++g) {
    double r = rho[g];
    vgrad[3 * g] = vgrad[3 * g + 1] = vgrad[3 * g + 2] = 0.0;
    if (!(r >= OR_XC_RHO_MIN)) {
      eps[g] = 0.0;
      vrho[g] = 0.0;
      continue;
    }
    if (kind == 1) {
      eps[g] = -cx * pow(r, 4.0 / 3.0);
      vrho[g] = -4.0 / 3.0 * cx * cbrt(r);
      continue;
    }
    /* B88 on the spin density rho_s = rho/2, |grad rho_s| = |grad rho|/2 */
    double rs = 0.5 * r, a = pow(rs, 4.0 / 3.0);
    double gn = sqrt(grad[3 * g] * grad[3 * g] + grad[3 * g + 1] * grad[3 * g + 1] + grad[3 * g + 2] * grad[3 * g + 2]);
    double x = 0.5 * gn / a, as = asinh(x);
    double den = 1.0 + 6.0 * beta * x * as;
    double F = beta * x * x / den;
    /* F'(x)/x, regular at x = 0 */
    double Fpx = (2.0 * beta * den - beta * x * (6.0 * beta * as + 6.0 * beta * x / sqrt(1.0 + x * x))) / (den * den);
    eps[g] = -2.0 * a * (cxs + F);
    vrho[g] = -4.0 / 3.0 * cbrt(rs) * (cxs + F - x * x * Fpx);
    for (int k = 0; k < 3; ++k) vgrad[3 * g + k] = -Fpx * grad[3 * g + k] / (2.0 * a);
  }
  return 0;
}

/* E_xc = sum_g w_g eps_g (compensated) */
double or_xc_energy(int64_t G, const double* w, const double* eps) {
  long double s = 0.0L;
  for (int64_t g = 0; g < G; ++g) s += (long double)w[g] * eps[g];
  return (double)s;
}

/* Step (4): V_mn = sum_g w_g [v_rho phi_m phi_n + v_grad . grad(phi_m phi_n)]
 * (Eq. xc_grid_sum_0 + Eq. xc_grid_sum_1), V[nbf*nbf] overwritten */
void or_xc_matrix(void* h, int64_t G, const double* pts, const double* w, const double* vrho,
                  const double* vgrad, double* V) {
  or_ctx* c = (or_ctx*)h;
  int n = c->nbf;
  for (size_t i = 0; i < (size_t)n * n; ++i) V[i] = 0.0;
#pragma omp parallel
  {
    double* phi = (double*)malloc(sizeof(double) * n);
    double* dphi = (double*)malloc(sizeof(double) * 3 * n);
    double* Vt = (double*)calloc((size_t)n * n, sizeof(double));
#pragma omp for schedule(dynamic, 16)
    for (int64_t g = 0; g < G; ++g) {
      if (w[g] == 0.0) continue;
      or_xc_ao(h, pts + 3 * g, phi, dphi);
      const double* vg = vgrad + 3 * g;
      for (int m = 0; m < n; ++m)
        for (int v = 0; v < n; ++v) {
          double pp = phi[m] * phi[v];
          double gg = vg[0] * (dphi[m] * phi[v] + phi[m] * dphi[v]) +
                      vg[1] * (dphi[n + m] * phi[v] + phi[m] * dphi[n + v]) +
                      vg[2] * (dphi[2 * n + m] * phi[v] + phi[m] * dphi[2 * n + v]);
          Vt[(size_t)m * n + v] += w[g] * (vrho[g] * pp + gg);
        }
    }
#pragma omp critical
    for (size_t i = 0; i < (size_t)n * n; ++i) V[i] += Vt[i];
    free(phi);
    free(dphi);
    free(Vt);
  }
}

/* Selected elements out[e] = V_{mn[2e], mn[2e+1]} of or_xc_matrix, each summed
 * over every point (shell values of the two shells only): for large grids */
void or_xc_matrix_elements(void* h, int64_t G, const double* pts, const double* w, const double* vrho,
                           const double* vgrad, int nel, const int32_t* mn, double* out) {
  or_ctx* c = (or_ctx*)h;
  int* shell_of = (int*)malloc(sizeof(int) * c->nbf);
  for (int s = 0; s < c->nshell; ++s)
    for (int m = c->aoff[s]; m < c->aoff[s + 1]; ++m) shell_of[m] = s;
#pragma omp parallel for schedule(dynamic, 1)
  for (int e = 0; e < nel; ++e) {
    int m = mn[2 * e], v = mn[2 * e + 1], sm = shell_of[m], sv = shell_of[v];
    int im = m - c->aoff[sm], iv = v - c->aoff[sv], nm = ncart(c->l[sm]), nv = ncart(c->l[sv]);
    double pm[10], dm[30], pv[10], dv[30];
    long double acc = 0.0L;
    for (int64_t g = 0; g < G; ++g) {
      if (w[g] == 0.0) continue;
      ao_shell(c, sm, pts + 3 * g, pm, dm);
      ao_shell(c, sv, pts + 3 * g, pv, dv);
      const double* vg = vgrad + 3 * g;
      double gg = 0.0;
      for (int x = 0; x < 3; ++x) gg += vg[x] * (dm[x * nm + im] * pv[iv] + pm[im] * dv[x * nv + iv]);
      acc += (long double)w[g] * (vrho[g] * pm[im] * pv[iv] + gg);
    }
    out[e] = (double)acc;
  }
  free(shell_of);
}
