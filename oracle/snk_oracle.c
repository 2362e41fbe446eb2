/*
 * snk_oracle.c -- plain FP64 CPU oracle for the seminumerical exchange (sn-K)
 * build of arXiv 2303.14280.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path never
 * calls it and shares no code, header, table or constant with it.
 *
 * Everything is a direct transcription of a definition or of the steps of the
 * method in the paper's order, in double precision, with no blocking, fusion or
 * reordering of the sums beyond what the definitions state:
 *
 *   Boys function F_n(T)            Sec. II.B, Eq. (boys)
 *   primitive Cartesian Gaussians   Sec. II.B (definition of phi_a)
 *   3c-CP integral A_{mu lambda}(r) Sec. II.D, Eq. (3c_grid)
 *     - Obara-Saika route           App. A, Eqs. (vrr), (hrr) and the seed;
 *                                   contraction between VRR and HRR (App. A)
 *     - McMurchie-Davidson route    Sec. II.B, Eqs. (cart2herm-2), (pc), (md1)
 *   4-centre ERIs (mu lambda|nu kappa) via McMurchie-Davidson  Sec. II.B
 *   collocation Phi_{mu i}          Sec. II.C, Eq. (collocation)
 *   F = D Phi                       Sec. II.C, Eq. (fmat)
 *   G_{mu i} = sum_l w_i A F        Sec. II.D, Eq. (gmat)
 *   Ktilde = G Phi^T                Sec. II.D, Eq. (usym_k)
 *   K = (Ktilde + Ktilde^T)/2       Sec. II.D, Eq. (sn_k)
 *   exact K from ERIs               Sec. II.A, Eq. (full_k)
 *   V^xc and E_xc (GGA)             Sec. II.C, Eqs. (vxc_num), (zmat), (exc_grid),
 *                                   (den_grid), (fmat), with Slater, PBE exchange
 *                                   and PBE correlation written from their
 *                                   published definitions
 *
 * Readings where the paper is silent or garbled:
 *   - the seed of the VRR carries the standard nuclear-attraction prefactor
 *     (2 pi / zeta_p) exp(-zeta_a zeta_b |AB|^2 / zeta_p); App. A prints the
 *     Boys function alone.  The operator is +1/|r - r_i|.
 *   - each Cartesian component of a contracted shell has unit self-overlap;
 *     caller coefficients refer to x^l-normalised primitives.
 *   - Boys: power series below T = 30, erf plus upward recursion above.
 *   - no screening: every shell pair and every grid point contributes.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LMAX 2                 /* highest shell angular momentum        */
#define ORC_LA (2 * ORC_LMAX)      /* highest l_a + l_b                      */
#define ORC_LE (4 * ORC_LMAX)      /* highest total L of an ERI quartet      */
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* small helpers                                                            */
/* ------------------------------------------------------------------------ */

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* Cartesian components of angular momentum l in lexicographic order:
 * (l,0,0), (l-1,1,0), (l-1,0,1), (l-2,2,0), ... */
static void cart_list(int l, int c[][3]) {
  int k = 0;
  for (int ax = l; ax >= 0; --ax)
    for (int ay = l - ax; ay >= 0; --ay) {
      c[k][0] = ax;
      c[k][1] = ay;
      c[k][2] = l - ax - ay;
      ++k;
    }
}

/* (n)!! for odd n >= -1, with (-1)!! = 1 */
static double odd_dfact(int n) {
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

/* ------------------------------------------------------------------------ */
/* Boys function, Eq. (boys): F_n(T) = int_0^1 y^{2n} exp(-T y^2) dy        */
/* ------------------------------------------------------------------------ */

void oracle_boys(int nmax, double T, double *F) {
  if (T < 30.0) {
    /* F_n(T) = exp(-T) sum_k (2T)^k / ((2n+1)(2n+3)...(2n+2k+1)) */
    double e = exp(-T);
    for (int n = 0; n <= nmax; ++n) {
      double term = 1.0 / (2 * n + 1);
      double sum = term;
      for (int k = 0; k < 2000; ++k) {
        term *= 2.0 * T / (2 * n + 2 * k + 3);
        sum += term;
        if (term < 1e-18 * sum) break;
      }
      F[n] = e * sum;
    }
  } else {
    /* F_0 = (1/2) sqrt(pi/T) erf(sqrt T); F_{n+1} = ((2n+1) F_n - e^{-T}) / (2T) */
    double e = exp(-T);
    F[0] = 0.5 * sqrt(ORC_PI / T) * erf(sqrt(T));
    for (int n = 0; n < nmax; ++n) F[n + 1] = ((2 * n + 1) * F[n] - e) / (2.0 * T);
  }
}

/* ------------------------------------------------------------------------ */
/* basis normalisation                                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n_shells, n_func;
  const int *l, *nprim;
  const double *center;  /* 3 per shell */
  const double *exps;
  int *poff;             /* first primitive of each shell  */
  int *foff;             /* first function of each shell   */
  double *d;             /* normalised coefficient on the raw primitive x^l e^{-a r^2} */
} obasis;

/* x^l-normalised primitive: (2a/pi)^{3/4} (4a)^{l/2} / sqrt((2l-1)!!) */
static double prim_norm(double a, int l) {
  return pow(2.0 * a / ORC_PI, 0.75) * pow(4.0 * a, 0.5 * l) / sqrt(odd_dfact(2 * l - 1));
}

/* factor turning the x^l-normalised contraction into a unit-norm component */
static double comp_factor(int l, const int c[3]) {
  return sqrt(odd_dfact(2 * l - 1) /
              (odd_dfact(2 * c[0] - 1) * odd_dfact(2 * c[1] - 1) * odd_dfact(2 * c[2] - 1)));
}

static int obasis_init(obasis *b, int n_shells, const int *l, const int *nprim,
                       const double *center, const double *exps, const double *coefs) {
  b->n_shells = n_shells;
  b->l = l;
  b->nprim = nprim;
  b->center = center;
  b->exps = exps;
  b->poff = (int *)malloc(sizeof(int) * (n_shells + 1));
  b->foff = (int *)malloc(sizeof(int) * (n_shells + 1));
  int np = 0, nf = 0;
  for (int s = 0; s < n_shells; ++s) {
    if (l[s] < 0 || l[s] > ORC_LMAX) return -1;
    b->poff[s] = np;
    b->foff[s] = nf;
    np += nprim[s];
    nf += ncart(l[s]);
  }
  b->poff[n_shells] = np;
  b->foff[n_shells] = nf;
  b->n_func = nf;
  b->d = (double *)malloc(sizeof(double) * (np > 0 ? np : 1));
  for (int s = 0; s < n_shells; ++s) {
    int p0 = b->poff[s], n = nprim[s], ls = l[s];
    for (int k = 0; k < n; ++k) b->d[p0 + k] = coefs[p0 + k] * prim_norm(exps[p0 + k], ls);
    /* self-overlap of the x^l component of the contraction */
    double S = 0.0;
    for (int k = 0; k < n; ++k)
      for (int m = 0; m < n; ++m) {
        double ab = exps[p0 + k] + exps[p0 + m];
        S += b->d[p0 + k] * b->d[p0 + m] * pow(ORC_PI / ab, 1.5) * odd_dfact(2 * ls - 1) /
             pow(2.0 * ab, ls);
      }
    for (int k = 0; k < n; ++k) b->d[p0 + k] /= sqrt(S);
  }
  return 0;
}

static void obasis_free(obasis *b) {
  free(b->poff);
  free(b->foff);
  free(b->d);
}

/* normalised coefficients (per primitive) and component factors (per function) */
int oracle_normalise(int n_shells, const int *l, const int *nprim, const double *center,
                     const double *exps, const double *coefs, double *d_out, double *f_out) {
  obasis b;
  if (obasis_init(&b, n_shells, l, nprim, center, exps, coefs)) return -1;
  memcpy(d_out, b.d, sizeof(double) * b.poff[n_shells]);
  for (int s = 0; s < n_shells; ++s) {
    int c[6][3];
    cart_list(l[s], c);
    for (int i = 0; i < ncart(l[s]); ++i) f_out[b.foff[s] + i] = comp_factor(l[s], c[i]);
  }
  obasis_free(&b);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* collocation, Eq. (collocation)                                           */
/* ------------------------------------------------------------------------ */

static void collocate_point(const obasis *b, const double r[3], double *phi) {
  for (int s = 0; s < b->n_shells; ++s) {
    const double *A = b->center + 3 * s;
    double x = r[0] - A[0], y = r[1] - A[1], z = r[2] - A[2];
    double r2 = x * x + y * y + z * z;
    double rad = 0.0;
    for (int k = b->poff[s]; k < b->poff[s + 1]; ++k) rad += b->d[k] * exp(-b->exps[k] * r2);
    int c[6][3];
    cart_list(b->l[s], c);
    for (int i = 0; i < ncart(b->l[s]); ++i)
      phi[b->foff[s] + i] = comp_factor(b->l[s], c[i]) * pow(x, c[i][0]) * pow(y, c[i][1]) *
                            pow(z, c[i][2]) * rad;
  }
}

int oracle_collocation(int n_shells, const int *l, const int *nprim, const double *center,
                       const double *exps, const double *coefs, long npts, const double *xyz,
                       double *phi /* npts x n_func, row-major */) {
  obasis b;
  if (obasis_init(&b, n_shells, l, nprim, center, exps, coefs)) return -1;
  for (long i = 0; i < npts; ++i) collocate_point(&b, xyz + 3 * i, phi + i * b.n_func);
  obasis_free(&b);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* 3c-CP integrals by Obara-Saika, App. A                                   */
/* ------------------------------------------------------------------------ */

typedef double cube_t[ORC_LA + 1][ORC_LA + 1][ORC_LA + 1];

/* One primitive pair: run the VRR, Eq. (vrr), from the seed
 * Theta^n_0 = pref * F_n(zeta |P - C|^2) up to |e| = L and add the Theta^0_e
 * with lmin <= |e| <= L into acc. */
static void os_vrr_add(int L, int lmin, double zeta, const double P[3], const double Ra[3],
                       const double C[3], double pref, cube_t acc) {
  double th[ORC_LA + 1][ORC_LA + 1][ORC_LA + 1][ORC_LA + 1]; /* [n][ex][ey][ez] */
  double PA[3], PC[3], F[ORC_LA + 1];
  double pc2 = 0.0;
  for (int q = 0; q < 3; ++q) {
    PA[q] = P[q] - Ra[q];
    PC[q] = P[q] - C[q];
    pc2 += PC[q] * PC[q];
  }
  oracle_boys(L, zeta * pc2, F);
  for (int n = 0; n <= L; ++n) th[n][0][0][0] = pref * F[n];
  for (int le = 1; le <= L; ++le) {
    int c[ORC_LA * 4 + 8][3];
    int nc = ncart(le);
    cart_list(le, c);
    for (int k = 0; k < nc; ++k) {
      int e[3] = {c[k][0], c[k][1], c[k][2]};
      int q = e[0] > 0 ? 0 : (e[1] > 0 ? 1 : 2);
      int m1[3] = {e[0], e[1], e[2]};
      m1[q] -= 1; /* a = e - 1_q */
      int aq = m1[q];
      for (int n = 0; n <= L - le; ++n) {
        double v = PA[q] * th[n][m1[0]][m1[1]][m1[2]] - PC[q] * th[n + 1][m1[0]][m1[1]][m1[2]];
        if (aq > 0) {
          int m2[3] = {m1[0], m1[1], m1[2]};
          m2[q] -= 1;
          v += aq / (2.0 * zeta) * (th[n][m2[0]][m2[1]][m2[2]] - th[n + 1][m2[0]][m2[1]][m2[2]]);
        }
        th[n][e[0]][e[1]][e[2]] = v;
      }
    }
  }
  for (int le = lmin; le <= L; ++le) {
    int c[ORC_LA * 4 + 8][3];
    cart_list(le, c);
    for (int k = 0; k < ncart(le); ++k) acc[c[k][0]][c[k][1]][c[k][2]] += th[0][c[k][0]][c[k][1]][c[k][2]];
  }
}

/* HRR, Eq. (hrr): Xi_{e, f+1_q} = Xi_{e+1_q, f} + (A - B)_q Xi_{e f}, from
 * Xi_{e 0} = acc[e], then out[i][j] = Xi_{a_i b_j} for the components. */
static void os_hrr(int la, int lb, const double AB[3], cube_t acc, double *out) {
  int L = la + lb;
  /* xi[e][f] stored as xi[ex][ey][ez][fx][fy][fz] */
  enum { D = ORC_LA + 1, DB = ORC_LMAX + 1 };
  double xi[D * D * D * DB * DB * DB]; /* only entries written below are read */
#define XI(ex, ey, ez, fx, fy, fz) xi[((((((ex) * D + (ey)) * D + (ez)) * DB + (fx)) * DB + (fy)) * DB + (fz))]
  for (int le = la; le <= L; ++le) {
    int c[32][3];
    cart_list(le, c);
    for (int k = 0; k < ncart(le); ++k) XI(c[k][0], c[k][1], c[k][2], 0, 0, 0) = acc[c[k][0]][c[k][1]][c[k][2]];
  }
  for (int lf = 1; lf <= lb; ++lf) {
    int cf[8][3];
    cart_list(lf, cf);
    for (int kf = 0; kf < ncart(lf); ++kf) {
      int f[3] = {cf[kf][0], cf[kf][1], cf[kf][2]};
      int q = f[0] > 0 ? 0 : (f[1] > 0 ? 1 : 2);
      int g[3] = {f[0], f[1], f[2]};
      g[q] -= 1;
      for (int le = la; le <= L - lf; ++le) {
        int c[32][3];
        cart_list(le, c);
        for (int k = 0; k < ncart(le); ++k) {
          int e[3] = {c[k][0], c[k][1], c[k][2]};
          int e1[3] = {e[0], e[1], e[2]};
          e1[q] += 1;
          XI(e[0], e[1], e[2], f[0], f[1], f[2]) =
              XI(e1[0], e1[1], e1[2], g[0], g[1], g[2]) + AB[q] * XI(e[0], e[1], e[2], g[0], g[1], g[2]);
        }
      }
    }
  }
  int ca[6][3], cb[6][3];
  cart_list(la, ca);
  cart_list(lb, cb);
  for (int i = 0; i < ncart(la); ++i)
    for (int j = 0; j < ncart(lb); ++j)
      out[i * ncart(lb) + j] = XI(ca[i][0], ca[i][1], ca[i][2], cb[j][0], cb[j][1], cb[j][2]);
#undef XI
}

/* A for one pair of raw primitives x_A^a e^{-alpha r_A^2}, x_B^b e^{-beta r_B^2}
 * at the point C (no normalisation), out: ncart(la) x ncart(lb). */
int oracle_prim_A_os(int la, int lb, const double *A, double alpha, const double *B, double beta,
                     const double *C, double *out) {
  if (la < 0 || lb < 0 || la > ORC_LMAX || lb > ORC_LMAX) return -1;
  cube_t acc;
  memset(acc, 0, sizeof(acc));
  double zeta = alpha + beta, P[3], AB[3], ab2 = 0.0;
  for (int q = 0; q < 3; ++q) {
    P[q] = (alpha * A[q] + beta * B[q]) / zeta;
    AB[q] = A[q] - B[q];
    ab2 += AB[q] * AB[q];
  }
  double pref = 2.0 * ORC_PI / zeta * exp(-alpha * beta / zeta * ab2);
  os_vrr_add(la + lb, la, zeta, P, A, C, pref, acc);
  os_hrr(la, lb, AB, acc, out);
  return 0;
}

/* contracted, normalised shell pair (sa, sb) at the point C: primitive
 * Theta^0 are contracted between VRR and HRR (App. A). */
static void os_A_shellpair(const obasis *b, int sa, int sb, const double C[3], double *out) {
  int la = b->l[sa], lb = b->l[sb];
  const double *A = b->center + 3 * sa, *B = b->center + 3 * sb;
  cube_t acc;
  memset(acc, 0, sizeof(acc));
  double AB[3], ab2 = 0.0;
  for (int q = 0; q < 3; ++q) {
    AB[q] = A[q] - B[q];
    ab2 += AB[q] * AB[q];
  }
  for (int k = b->poff[sa]; k < b->poff[sa + 1]; ++k)
    for (int m = b->poff[sb]; m < b->poff[sb + 1]; ++m) {
      double al = b->exps[k], be = b->exps[m], zeta = al + be, P[3];
      for (int q = 0; q < 3; ++q) P[q] = (al * A[q] + be * B[q]) / zeta;
      double pref = 2.0 * ORC_PI / zeta * exp(-al * be / zeta * ab2) * b->d[k] * b->d[m];
      os_vrr_add(la + lb, la, zeta, P, A, C, pref, acc);
    }
  os_hrr(la, lb, AB, acc, out);
  int ca[6][3], cb[6][3];
  cart_list(la, ca);
  cart_list(lb, cb);
  for (int i = 0; i < ncart(la); ++i)
    for (int j = 0; j < ncart(lb); ++j) out[i * ncart(lb) + j] *= comp_factor(la, ca[i]) * comp_factor(lb, cb[j]);
}

/* ------------------------------------------------------------------------ */
/* McMurchie-Davidson route, Sec. II.B                                      */
/* ------------------------------------------------------------------------ */

/* Hermite expansion coefficients E^{ij}_t of x_A^i x_B^j exp(...) in one
 * Cartesian direction (Eq. cart2herm-2), by the MD recursion. */
static void md_E(int imax, int jmax, double a, double b, double Ax, double Bx,
                 double E[ORC_LMAX + 1][ORC_LMAX + 1][2 * ORC_LMAX + 2]) {
  double p = a + b, mu = a * b / p, Px = (a * Ax + b * Bx) / p;
  double XAB = Ax - Bx, XPA = Px - Ax, XPB = Px - Bx;
  memset(E, 0, sizeof(double) * (ORC_LMAX + 1) * (ORC_LMAX + 1) * (2 * ORC_LMAX + 2));
  E[0][0][0] = exp(-mu * XAB * XAB);
  for (int i = 0; i <= imax; ++i)
    for (int j = 0; j <= jmax; ++j) {
      if (i == 0 && j == 0) continue;
      for (int t = 0; t <= i + j; ++t) {
        double v;
        if (i > 0) {
          v = XPA * E[i - 1][j][t] + (t + 1 <= i - 1 + j ? (t + 1) * E[i - 1][j][t + 1] : 0.0);
          if (t > 0) v += E[i - 1][j][t - 1] / (2.0 * p);
        } else {
          v = XPB * E[i][j - 1][t] + (t + 1 <= i + j - 1 ? (t + 1) * E[i][j - 1][t + 1] : 0.0);
          if (t > 0) v += E[i][j - 1][t - 1] / (2.0 * p);
        }
        E[i][j][t] = v;
      }
    }
}

/* Hermite Coulomb integrals R_{tuv} = (r)^{(0)} of Eq. (md1), from
 * (0)^{(n)} = (-2 rho)^n F_n(rho |X|^2) (scaled to drop the constant), for
 * t+u+v <= L.  Rt[t][u][v] receives n = 0. */
#define RD (ORC_LE + 1)
static void md_R(int L, double rho, const double X[3], double *Rt /* RD^3 */) {
  double R[RD * RD * RD * RD]; /* only entries written below are read */
#define RR(n, t, u, v) R[(((n) * RD + (t)) * RD + (u)) * RD + (v)]
  double F[ORC_LE + 1];
  oracle_boys(L, rho * (X[0] * X[0] + X[1] * X[1] + X[2] * X[2]), F);
  double m2r = 1.0;
  for (int n = 0; n <= L; ++n) {
    RR(n, 0, 0, 0) = m2r * F[n];
    m2r *= -2.0 * rho;
  }
  for (int lt = 1; lt <= L; ++lt)
    for (int t = lt; t >= 0; --t)
      for (int u = lt - t; u >= 0; --u) {
        int v = lt - t - u;
        for (int n = 0; n <= L - lt; ++n) {
          double r;
          if (t > 0)
            r = (t > 1 ? (t - 1) * RR(n + 1, t - 2, u, v) : 0.0) + X[0] * RR(n + 1, t - 1, u, v);
          else if (u > 0)
            r = (u > 1 ? (u - 1) * RR(n + 1, t, u - 2, v) : 0.0) + X[1] * RR(n + 1, t, u - 1, v);
          else
            r = (v > 1 ? (v - 1) * RR(n + 1, t, u, v - 2) : 0.0) + X[2] * RR(n + 1, t, u, v - 1);
          RR(n, t, u, v) = r;
        }
      }
  for (int t = 0; t <= L; ++t)
    for (int u = 0; u <= L - t; ++u)
      for (int v = 0; v <= L - t - u; ++v) Rt[(t * RD + u) * RD + v] = RR(0, t, u, v);
#undef RR
}

int oracle_prim_A_md(int la, int lb, const double *A, double alpha, const double *B, double beta,
                     const double *C, double *out) {
  if (la < 0 || lb < 0 || la > ORC_LMAX || lb > ORC_LMAX) return -1;
  double p = alpha + beta, P[3], PC[3];
  for (int q = 0; q < 3; ++q) {
    P[q] = (alpha * A[q] + beta * B[q]) / p;
    PC[q] = P[q] - C[q];
  }
  double E[3][ORC_LMAX + 1][ORC_LMAX + 1][2 * ORC_LMAX + 2];
  for (int q = 0; q < 3; ++q) md_E(la, lb, alpha, beta, A[q], B[q], E[q]);
  double *R = (double *)malloc(sizeof(double) * RD * RD * RD);
  md_R(la + lb, p, PC, R);
  int ca[6][3], cb[6][3];
  cart_list(la, ca);
  cart_list(lb, cb);
  for (int i = 0; i < ncart(la); ++i)
    for (int j = 0; j < ncart(lb); ++j) {
      double s = 0.0;
      for (int t = 0; t <= ca[i][0] + cb[j][0]; ++t)
        for (int u = 0; u <= ca[i][1] + cb[j][1]; ++u)
          for (int v = 0; v <= ca[i][2] + cb[j][2]; ++v)
            s += E[0][ca[i][0]][cb[j][0]][t] * E[1][ca[i][1]][cb[j][1]][u] *
                 E[2][ca[i][2]][cb[j][2]][v] * R[(t * RD + u) * RD + v];
      out[i * ncart(lb) + j] = 2.0 * ORC_PI / p * s;
    }
  free(R);
  return 0;
}

static void md_A_shellpair(const obasis *b, int sa, int sb, const double C[3], double *out) {
  int la = b->l[sa], lb = b->l[sb], na = ncart(la), nb = ncart(lb);
  double tmp[36];
  for (int k = 0; k < na * nb; ++k) out[k] = 0.0;
  for (int k = b->poff[sa]; k < b->poff[sa + 1]; ++k)
    for (int m = b->poff[sb]; m < b->poff[sb + 1]; ++m) {
      oracle_prim_A_md(la, lb, b->center + 3 * sa, b->exps[k], b->center + 3 * sb, b->exps[m], C, tmp);
      for (int x = 0; x < na * nb; ++x) out[x] += b->d[k] * b->d[m] * tmp[x];
    }
  int ca[6][3], cb[6][3];
  cart_list(la, ca);
  cart_list(lb, cb);
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j) out[i * nb + j] *= comp_factor(la, ca[i]) * comp_factor(lb, cb[j]);
}

/* A for contracted, normalised shells sa, sb at point C; method 0 = OS, 1 = MD */
int oracle_shell_A(int n_shells, const int *l, const int *nprim, const double *center,
                   const double *exps, const double *coefs, int sa, int sb, const double *C,
                   int method, double *out) {
  obasis b;
  if (obasis_init(&b, n_shells, l, nprim, center, exps, coefs)) return -1;
  if (sa < 0 || sb < 0 || sa >= n_shells || sb >= n_shells) {
    obasis_free(&b);
    return -1;
  }
  if (method == 0)
    os_A_shellpair(&b, sa, sb, C, out);
  else
    md_A_shellpair(&b, sa, sb, C, out);
  obasis_free(&b);
  return 0;
}

/* (ab|cd) over raw primitives by MD: Eqs. (abc_to_hermite), (pc), (md1)
 * extended to a Hermite pair on each side. out: na x nb x nc x nd. */
int oracle_prim_eri_md(int la, int lb, int lc, int ld, const double *A, double alpha,
                       const double *B, double beta, const double *Cc, double gamma,
                       const double *D, double delta, double *out) {
  int Ls[4] = {la, lb, lc, ld};
  for (int k = 0; k < 4; ++k)
    if (Ls[k] < 0 || Ls[k] > ORC_LMAX) return -1;
  double p = alpha + beta, q = gamma + delta, rho = p * q / (p + q);
  double P[3], Q[3], PQ[3];
  for (int x = 0; x < 3; ++x) {
    P[x] = (alpha * A[x] + beta * B[x]) / p;
    Q[x] = (gamma * Cc[x] + delta * D[x]) / q;
    PQ[x] = P[x] - Q[x];
  }
  double Eab[3][ORC_LMAX + 1][ORC_LMAX + 1][2 * ORC_LMAX + 2];
  double Ecd[3][ORC_LMAX + 1][ORC_LMAX + 1][2 * ORC_LMAX + 2];
  for (int x = 0; x < 3; ++x) {
    md_E(la, lb, alpha, beta, A[x], B[x], Eab[x]);
    md_E(lc, ld, gamma, delta, Cc[x], D[x], Ecd[x]);
  }
  double *R = (double *)malloc(sizeof(double) * RD * RD * RD);
  md_R(la + lb + lc + ld, rho, PQ, R);
  double pref = 2.0 * pow(ORC_PI, 2.5) / (p * q * sqrt(p + q));
  int ca[6][3], cb[6][3], cc[6][3], cd[6][3];
  cart_list(la, ca);
  cart_list(lb, cb);
  cart_list(lc, cc);
  cart_list(ld, cd);
  int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j)
      for (int k = 0; k < nc; ++k)
        for (int m = 0; m < nd; ++m) {
          double s = 0.0;
          for (int t = 0; t <= ca[i][0] + cb[j][0]; ++t)
            for (int u = 0; u <= ca[i][1] + cb[j][1]; ++u)
              for (int v = 0; v <= ca[i][2] + cb[j][2]; ++v) {
                double eab = Eab[0][ca[i][0]][cb[j][0]][t] * Eab[1][ca[i][1]][cb[j][1]][u] *
                             Eab[2][ca[i][2]][cb[j][2]][v];
                for (int tt = 0; tt <= cc[k][0] + cd[m][0]; ++tt)
                  for (int uu = 0; uu <= cc[k][1] + cd[m][1]; ++uu)
                    for (int vv = 0; vv <= cc[k][2] + cd[m][2]; ++vv) {
                      double ecd = Ecd[0][cc[k][0]][cd[m][0]][tt] * Ecd[1][cc[k][1]][cd[m][1]][uu] *
                                   Ecd[2][cc[k][2]][cd[m][2]][vv];
                      double sign = ((tt + uu + vv) & 1) ? -1.0 : 1.0;
                      s += eab * sign * ecd * R[((t + tt) * RD + (u + uu)) * RD + (v + vv)];
                    }
              }
          out[((i * nb + j) * nc + k) * nd + m] = pref * s;
        }
  free(R);
  return 0;
}

/* K^exact_{mu nu} = sum_{lambda kappa} (mu lambda | nu kappa) P_{lambda kappa}, Eq. (full_k) */
int oracle_eri_K(int n_shells, const int *l, const int *nprim, const double *center,
                 const double *exps, const double *coefs, const double *Pm, double *K) {
  obasis b;
  if (obasis_init(&b, n_shells, l, nprim, center, exps, coefs)) return -1;
  int nf = b.n_func;
  for (int x = 0; x < nf * nf; ++x) K[x] = 0.0;
  double *blk = (double *)malloc(sizeof(double) * 1296);
  double *tmp = (double *)malloc(sizeof(double) * 1296);
  for (int sa = 0; sa < n_shells; ++sa)
    for (int sb = 0; sb < n_shells; ++sb)
      for (int sc = 0; sc < n_shells; ++sc)
        for (int sd = 0; sd < n_shells; ++sd) {
          int la = l[sa], lb = l[sb], lc = l[sc], ld = l[sd];
          int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
          int n = na * nb * nc * nd;
          for (int x = 0; x < n; ++x) blk[x] = 0.0;
          for (int ka = b.poff[sa]; ka < b.poff[sa + 1]; ++ka)
            for (int kb = b.poff[sb]; kb < b.poff[sb + 1]; ++kb)
              for (int kc = b.poff[sc]; kc < b.poff[sc + 1]; ++kc)
                for (int kd = b.poff[sd]; kd < b.poff[sd + 1]; ++kd) {
                  oracle_prim_eri_md(la, lb, lc, ld, center + 3 * sa, exps[ka], center + 3 * sb, exps[kb],
                                     center + 3 * sc, exps[kc], center + 3 * sd, exps[kd], tmp);
                  double dd = b.d[ka] * b.d[kb] * b.d[kc] * b.d[kd];
                  for (int x = 0; x < n; ++x) blk[x] += dd * tmp[x];
                }
          int ca[6][3], cb[6][3], cc[6][3], cd[6][3];
          cart_list(la, ca);
          cart_list(lb, cb);
          cart_list(lc, cc);
          cart_list(ld, cd);
          /* (mu lambda | nu kappa): mu in sa, lambda in sb, nu in sc, kappa in sd */
          for (int i = 0; i < na; ++i)
            for (int j = 0; j < nb; ++j)
              for (int k = 0; k < nc; ++k)
                for (int m = 0; m < nd; ++m) {
                  double v = blk[((i * nb + j) * nc + k) * nd + m] * comp_factor(la, ca[i]) *
                             comp_factor(lb, cb[j]) * comp_factor(lc, cc[k]) * comp_factor(ld, cd[m]);
                  int mu = b.foff[sa] + i, lam = b.foff[sb] + j, nu = b.foff[sc] + k, kap = b.foff[sd] + m;
                  K[mu * nf + nu] += v * Pm[lam * nf + kap];
                }
        }
  free(blk);
  free(tmp);
  obasis_free(&b);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* sn-K, Sec. II.D                                                          */
/* ------------------------------------------------------------------------ */

/* G_{mu} at one point: G_mu = w * sum_lambda A_{mu lambda}(r) F_lambda over
 * every shell pair (a, b), Eq. (gmat). Only shells with want[a] != 0 get rows. */
static void g_point(const obasis *b, const double r[3], double w, const double *F, const char *want,
                    double *G) {
  double A[36];
  for (int sa = 0; sa < b->n_shells; ++sa) {
    int na = ncart(b->l[sa]);
    for (int i = 0; i < na; ++i) G[b->foff[sa] + i] = 0.0;
    if (want && !want[sa]) continue;
    for (int sb = 0; sb < b->n_shells; ++sb) {
      int nb = ncart(b->l[sb]);
      os_A_shellpair(b, sa, sb, r, A);
      for (int i = 0; i < na; ++i) {
        double s = 0.0;
        for (int j = 0; j < nb; ++j) s += A[i * nb + j] * F[b->foff[sb] + j];
        G[b->foff[sa] + i] += w * s;
      }
    }
  }
}

static int n_threads_or_default(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/* Full sn-K build: Phi (Eq. collocation), F = P Phi (Eq. fmat), G (Eq. gmat),
 * Ktilde = G Phi^T (Eq. usym_k), K = (Ktilde + Ktilde^T)/2 (Eq. sn_k). */
int oracle_snk_K(int n_shells, const int *l, const int *nprim, const double *center,
                 const double *exps, const double *coefs, long npts, const double *xyz,
                 const double *w, const double *Pm, double *K, int nthreads) {
  obasis b;
  if (obasis_init(&b, n_shells, l, nprim, center, exps, coefs)) return -1;
  int nf = b.n_func, nt = n_threads_or_default(nthreads);
  double *Kt = (double *)calloc((size_t)nt * nf * nf, sizeof(double));
#pragma omp parallel num_threads(nt)
  {
#ifdef _OPENMP
    int tid = omp_get_thread_num();
#else
    int tid = 0;
#endif
    double *phi = (double *)malloc(sizeof(double) * nf);
    double *F = (double *)malloc(sizeof(double) * nf);
    double *G = (double *)malloc(sizeof(double) * nf);
    double *Kl = Kt + (size_t)tid * nf * nf;
#pragma omp for schedule(static)
    for (long i = 0; i < npts; ++i) {
      collocate_point(&b, xyz + 3 * i, phi);
      for (int lam = 0; lam < nf; ++lam) {
        double s = 0.0;
        for (int nu = 0; nu < nf; ++nu) s += Pm[lam * nf + nu] * phi[nu];
        F[lam] = s;
      }
      g_point(&b, xyz + 3 * i, w[i], F, NULL, G);
      for (int mu = 0; mu < nf; ++mu)
        for (int nu = 0; nu < nf; ++nu) Kl[mu * nf + nu] += G[mu] * phi[nu];
    }
    free(phi);
    free(F);
    free(G);
  }
  for (int x = 0; x < nf * nf; ++x) {
    double s = 0.0;
    for (int t = 0; t < nt; ++t) s += Kt[(size_t)t * nf * nf + x];
    Kt[x] = s;
  }
  for (int mu = 0; mu < nf; ++mu)
    for (int nu = 0; nu < nf; ++nu) K[mu * nf + nu] = 0.5 * (Kt[mu * nf + nu] + Kt[nu * nf + mu]);
  free(Kt);
  obasis_free(&b);
  return 0;
}

/* Selected entries K_{mu_k nu_k} of the same build: only the G rows of the
 * shells that hold some mu_k or nu_k are formed. */
int oracle_snk_K_entries(int n_shells, const int *l, const int *nprim, const double *center,
                         const double *exps, const double *coefs, long npts, const double *xyz,
                         const double *w, const double *Pm, int nent, const int *mu_list,
                         const int *nu_list, double *out, int nthreads) {
  obasis b;
  if (obasis_init(&b, n_shells, l, nprim, center, exps, coefs)) return -1;
  int nf = b.n_func, nt = n_threads_or_default(nthreads);
  char *want = (char *)calloc(n_shells, 1);
  for (int k = 0; k < nent; ++k) {
    if (mu_list[k] < 0 || mu_list[k] >= nf || nu_list[k] < 0 || nu_list[k] >= nf) {
      free(want);
      obasis_free(&b);
      return -1;
    }
    for (int s = 0; s < n_shells; ++s)
      if ((mu_list[k] >= b.foff[s] && mu_list[k] < b.foff[s + 1]) ||
          (nu_list[k] >= b.foff[s] && nu_list[k] < b.foff[s + 1]))
        want[s] = 1;
  }
  double *acc = (double *)calloc((size_t)nt * 2 * (nent > 0 ? nent : 1), sizeof(double));
#pragma omp parallel num_threads(nt)
  {
#ifdef _OPENMP
    int tid = omp_get_thread_num();
#else
    int tid = 0;
#endif
    double *phi = (double *)malloc(sizeof(double) * nf);
    double *F = (double *)malloc(sizeof(double) * nf);
    double *G = (double *)malloc(sizeof(double) * nf);
    double *a = acc + (size_t)tid * 2 * nent;
#pragma omp for schedule(static)
    for (long i = 0; i < npts; ++i) {
      collocate_point(&b, xyz + 3 * i, phi);
      for (int lam = 0; lam < nf; ++lam) {
        double s = 0.0;
        for (int nu = 0; nu < nf; ++nu) s += Pm[lam * nf + nu] * phi[nu];
        F[lam] = s;
      }
      g_point(&b, xyz + 3 * i, w[i], F, want, G);
      for (int k = 0; k < nent; ++k) {
        a[2 * k] += G[mu_list[k]] * phi[nu_list[k]];
        a[2 * k + 1] += G[nu_list[k]] * phi[mu_list[k]];
      }
    }
    free(phi);
    free(F);
    free(G);
  }
  for (int k = 0; k < nent; ++k) {
    double s1 = 0.0, s2 = 0.0;
    for (int t = 0; t < nt; ++t) {
      s1 += acc[(size_t)t * 2 * nent + 2 * k];
      s2 += acc[(size_t)t * 2 * nent + 2 * k + 1];
    }
    out[k] = 0.5 * (s1 + s2);
  }
  free(acc);
  free(want);
  obasis_free(&b);
  return 0;
}

/* The G rows (Eq. gmat) of the listed functions at every point of a block,
 * given the block's F (Eq. fmat: F[i][lambda], npts x nf row-major), which
 * the caller forms with a library matrix product F = Phi P.  G is written
 * npts x nfun row-major: G[i][t] = G_{fun[t]}(r_i).  Used by the blocked
 * entries mode for large grids, where streaming P once per point (the
 * per-point routines above) would dominate the oracle's time. */
int oracle_g_rows(int n_shells, const int *l, const int *nprim, const double *center, const double *exps,
                  const double *coefs, long npts, const double *xyz, const double *w, const double *F,
                  int nfun, const int *fun, double *G, int nthreads) {
  obasis b;
  if (obasis_init(&b, n_shells, l, nprim, center, exps, coefs)) return -1;
  int nf = b.n_func, nt = n_threads_or_default(nthreads);
  char *want = (char *)calloc(n_shells, 1);
  for (int t = 0; t < nfun; ++t) {
    if (fun[t] < 0 || fun[t] >= nf) {
      free(want);
      obasis_free(&b);
      return -1;
    }
    for (int s = 0; s < n_shells; ++s)
      if (fun[t] >= b.foff[s] && fun[t] < b.foff[s + 1]) want[s] = 1;
  }
#pragma omp parallel num_threads(nt)
  {
    double *Gp = (double *)malloc(sizeof(double) * nf);
#pragma omp for schedule(dynamic, 16)
    for (long i = 0; i < npts; ++i) {
      g_point(&b, xyz + 3 * i, w[i], F + (size_t)i * nf, want, Gp);
      for (int t = 0; t < nfun; ++t) G[(size_t)i * nfun + t] = Gp[fun[t]];
    }
    free(Gp);
  }
  free(want);
  obasis_free(&b);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* MLP of the learned block screen: plain FP64 forward, loss and gradient   */
/* by backpropagation, for checks of the GPU training kernels.              */
/* Weights: W1[16][64] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64] b4; */
/* ReLU hidden layers; loss = (1/n) sum c r^2, r = y - label, c = 1 if      */
/* r >= 0 else under_weight.                                                */
/* ------------------------------------------------------------------------ */

#define ORC_NIN 16
#define ORC_NH 64

static void mlp_offsets(int off[8]) {
  off[0] = 0;                          /* W1 */
  off[1] = off[0] + ORC_NIN * ORC_NH;  /* b1 */
  off[2] = off[1] + ORC_NH;            /* W2 */
  off[3] = off[2] + ORC_NH * ORC_NH;   /* b2 */
  off[4] = off[3] + ORC_NH;            /* W3 */
  off[5] = off[4] + ORC_NH * ORC_NH;   /* b3 */
  off[6] = off[5] + ORC_NH;            /* W4 */
  off[7] = off[6] + ORC_NH;            /* b4 */
}

/* one layer: out[m] = b[m] + sum_k in[k] W[k][m] */
static void mlp_dense(const double *w, int W, int B, int nin, int nout, const double *in, double *out) {
  for (int m = 0; m < nout; ++m) {
    double s = w[B + m];
    for (int k = 0; k < nin; ++k) s += in[k] * w[W + k * nout + m];
    out[m] = s;
  }
}

static double mlp_forward_store(const double *w, const double *x, double z[3][ORC_NH], double a[3][ORC_NH]) {
  int off[8];
  mlp_offsets(off);
  mlp_dense(w, off[0], off[1], ORC_NIN, ORC_NH, x, z[0]);
  for (int m = 0; m < ORC_NH; ++m) a[0][m] = z[0][m] > 0.0 ? z[0][m] : 0.0;
  mlp_dense(w, off[2], off[3], ORC_NH, ORC_NH, a[0], z[1]);
  for (int m = 0; m < ORC_NH; ++m) a[1][m] = z[1][m] > 0.0 ? z[1][m] : 0.0;
  mlp_dense(w, off[4], off[5], ORC_NH, ORC_NH, a[1], z[2]);
  for (int m = 0; m < ORC_NH; ++m) a[2][m] = z[2][m] > 0.0 ? z[2][m] : 0.0;
  double y;
  mlp_dense(w, off[6], off[7], ORC_NH, 1, a[2], &y);
  return y;
}

int oracle_mlp_forward(const double *w, const double *X, long n, double *out) {
  double z[3][ORC_NH], a[3][ORC_NH];
  for (long s = 0; s < n; ++s) out[s] = mlp_forward_store(w, X + s * ORC_NIN, z, a);
  return 0;
}

int oracle_mlp_loss_grad(const double *w, const double *X, const double *Y, long n, double under_weight,
                         double *grad, double *loss) {
  int off[8];
  mlp_offsets(off);
  const int nw = off[7] + 1;
  for (int e = 0; e < nw; ++e) grad[e] = 0.0;
  *loss = 0.0;
  double z[3][ORC_NH], a[3][ORC_NH], d[3][ORC_NH];
  for (long s = 0; s < n; ++s) {
    const double *x = X + s * ORC_NIN;
    const double y = mlp_forward_store(w, x, z, a);
    const double r = y - Y[s];
    const double c = r < 0.0 ? under_weight : 1.0;
    *loss += c * r * r / n;
    const double dy = 2.0 * c * r / n;
    /* output layer */
    grad[off[7]] += dy;
    for (int k = 0; k < ORC_NH; ++k) grad[off[6] + k] += a[2][k] * dy;
    for (int k = 0; k < ORC_NH; ++k) d[2][k] = z[2][k] > 0.0 ? w[off[6] + k] * dy : 0.0;
    /* hidden layer 3 */
    for (int m = 0; m < ORC_NH; ++m) {
      grad[off[5] + m] += d[2][m];
      for (int k = 0; k < ORC_NH; ++k) grad[off[4] + k * ORC_NH + m] += a[1][k] * d[2][m];
    }
    for (int k = 0; k < ORC_NH; ++k) {
      double t = 0.0;
      for (int m = 0; m < ORC_NH; ++m) t += w[off[4] + k * ORC_NH + m] * d[2][m];
      d[1][k] = z[1][k] > 0.0 ? t : 0.0;
    }
    /* hidden layer 2 */
    for (int m = 0; m < ORC_NH; ++m) {
      grad[off[3] + m] += d[1][m];
      for (int k = 0; k < ORC_NH; ++k) grad[off[2] + k * ORC_NH + m] += a[0][k] * d[1][m];
    }
    for (int k = 0; k < ORC_NH; ++k) {
      double t = 0.0;
      for (int m = 0; m < ORC_NH; ++m) t += w[off[2] + k * ORC_NH + m] * d[1][m];
      d[0][k] = z[0][k] > 0.0 ? t : 0.0;
    }
    /* hidden layer 1 */
    for (int m = 0; m < ORC_NH; ++m) {
      grad[off[1] + m] += d[0][m];
      for (int k = 0; k < ORC_NIN; ++k) grad[off[0] + k * ORC_NH + m] += x[k] * d[0][m];
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* exchange-correlation potential, Sec. II.C                                */
/* ------------------------------------------------------------------------ */
/*
 * Spin-restricted functionals eps(rho, sigma), sigma = |grad rho|^2, as an
 * energy per volume (E_xc = sum_i w_i eps(rho_i, sigma_i)), with the two
 * partial derivatives Eq. (exc_grid) needs.  The paper takes its functionals
 * from a library; these are written from their published definitions:
 *   1  Slater (LDA) exchange     eps = C_x rho^{4/3}, C_x = -(3/4)(3/pi)^{1/3}
 *   2  PBE exchange              eps = C_x rho^{4/3} F_x(s),
 *                                F_x = 1 + kappa - kappa / (1 + mu s^2 / kappa),
 *                                s = |grad rho| / (2 k_F rho), k_F = (3 pi^2 rho)^{1/3}
 *   3  PBE exchange + PBE correlation: rho (e_c^PW92(r_s) + H(r_s, t)),
 *                                r_s = (3 / (4 pi rho))^{1/3}, t = |grad rho| / (2 k_s rho),
 *                                k_s = sqrt(4 k_F / pi),
 *                                H = gamma ln(1 + (beta/gamma) t^2 (1 + A t^2) / (1 + A t^2 + A^2 t^4)),
 *                                A = (beta/gamma) / (exp(-e_c^PW92 / gamma) - 1)
 * PW92 (unpolarised): e_c = -2 a (1 + alpha_1 r_s) ln(1 + 1 / Q),
 *                     Q = 2 a (beta_1 r_s^{1/2} + beta_2 r_s + beta_3 r_s^{3/2} + beta_4 r_s^2).
 * Points with rho below ORC_XC_RHO_MIN contribute nothing.
 */
#define ORC_XC_RHO_MIN 1e-14
#define ORC_PBE_KAPPA 0.804
#define ORC_PBE_BETA 0.06672455060314922
#define ORC_PW92_A 0.031091
#define ORC_PW92_ALPHA1 0.21370
#define ORC_PW92_B1 7.5957
#define ORC_PW92_B2 3.5876
#define ORC_PW92_B3 1.6382
#define ORC_PW92_B4 0.49294

/* PW92 correlation energy per electron and its derivative in r_s */
static void pw92(double rs, double *ec, double *dec_drs) {
  const double a = ORC_PW92_A, srs = sqrt(rs);
  const double Q = 2.0 * a * (ORC_PW92_B1 * srs + ORC_PW92_B2 * rs + ORC_PW92_B3 * rs * srs + ORC_PW92_B4 * rs * rs);
  const double dQ = 2.0 * a * (0.5 * ORC_PW92_B1 / srs + ORC_PW92_B2 + 1.5 * ORC_PW92_B3 * srs + 2.0 * ORC_PW92_B4 * rs);
  const double lg = log(1.0 + 1.0 / Q);
  *ec = -2.0 * a * (1.0 + ORC_PW92_ALPHA1 * rs) * lg;
  *dec_drs = -2.0 * a * ORC_PW92_ALPHA1 * lg + 2.0 * a * (1.0 + ORC_PW92_ALPHA1 * rs) * dQ / (Q * (Q + 1.0));
}

/* out[0] = eps, out[1] = d eps / d rho, out[2] = d eps / d sigma */
int oracle_xc_point(int functional, double rho, double sigma, double *out) {
  out[0] = out[1] = out[2] = 0.0;
  if (functional < 1 || functional > 3) return -1;
  if (!(rho >= ORC_XC_RHO_MIN)) return 0;
  if (sigma < 0.0) sigma = 0.0;
  const double Cx = -0.75 * cbrt(3.0 / ORC_PI);
  const double r13 = cbrt(rho), r43 = rho * r13;
  if (functional == 1) {
    out[0] = Cx * r43;
    out[1] = 4.0 / 3.0 * Cx * r13;
    return 0;
  }
  /* PBE exchange */
  const double kappa = ORC_PBE_KAPPA, mu = ORC_PBE_BETA * ORC_PI * ORC_PI / 3.0;
  const double kF = cbrt(3.0 * ORC_PI * ORC_PI * rho);
  const double ds2_dsigma = 1.0 / (4.0 * kF * kF * rho * rho);   /* s^2 = sigma ds2_dsigma */
  const double s2 = sigma * ds2_dsigma;
  const double den = 1.0 + mu * s2 / kappa;
  const double Fx = 1.0 + kappa - kappa / den;
  const double dFx = mu / (den * den);                             /* dF_x / d(s^2) */
  out[0] = Cx * r43 * Fx;
  out[1] = 4.0 / 3.0 * Cx * r13 * Fx + Cx * r43 * dFx * (-8.0 / 3.0) * s2 / rho;
  out[2] = Cx * r43 * dFx * ds2_dsigma;
  if (functional == 2) return 0;
  /* PBE correlation */
  const double gam = (1.0 - log(2.0)) / (ORC_PI * ORC_PI), beta = ORC_PBE_BETA;
  const double rs = cbrt(3.0 / (4.0 * ORC_PI * rho));
  double ec, dec_drs;
  pw92(rs, &ec, &dec_drs);
  const double dec_drho = dec_drs * (-rs / (3.0 * rho));
  const double ks2 = 4.0 * kF / ORC_PI;
  const double dy_dsigma = 1.0 / (4.0 * ks2 * rho * rho);          /* y = t^2 = sigma dy_dsigma */
  const double y = sigma * dy_dsigma;
  const double E = exp(-ec / gam);
  const double A = beta / gam / (E - 1.0);
  const double N = 1.0 + A * y, D = 1.0 + A * y + A * A * y * y;
  const double R = y * N / D;
  const double arg = 1.0 + beta / gam * R;
  const double H = gam * log(arg);
  const double dH_dR = beta / arg;
  const double dR_dy = (N + A * y) / D - y * N * (A + 2.0 * A * A * y) / (D * D);
  const double dR_dA = y * y / D - y * N * (y + 2.0 * A * y * y) / (D * D);
  const double dA_dec = A * A * E / beta;
  const double dy_drho = -7.0 / 3.0 * y / rho;
  out[0] += rho * (ec + H);
  out[1] += ec + H + rho * (dec_drho * (1.0 + dH_dR * dR_dA * dA_dec) + dH_dR * dR_dy * dy_drho);
  out[2] += rho * dH_dR * dR_dy * dy_dsigma;
  return 0;
}

/* Phi and its gradient at one point: phi[nf], gphi[3 nf] (x, y, z blocks) */
static void collocate_grad_point(const obasis *b, const double r[3], double *phi, double *gphi) {
  const int nf = b->n_func;
  for (int s = 0; s < b->n_shells; ++s) {
    const double *A = b->center + 3 * s;
    double d[3] = {r[0] - A[0], r[1] - A[1], r[2] - A[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double R0 = 0.0, R1 = 0.0; /* sum_k d_k e^{-a r^2}, sum_k (-2 a_k) d_k e^{-a r^2} */
    for (int k = b->poff[s]; k < b->poff[s + 1]; ++k) {
      double e = b->d[k] * exp(-b->exps[k] * r2);
      R0 += e;
      R1 += -2.0 * b->exps[k] * e;
    }
    int c[6][3];
    cart_list(b->l[s], c);
    for (int i = 0; i < ncart(b->l[s]); ++i) {
      const int mu = b->foff[s] + i;
      const double f = comp_factor(b->l[s], c[i]);
      const double mono = pow(d[0], c[i][0]) * pow(d[1], c[i][1]) * pow(d[2], c[i][2]);
      phi[mu] = f * mono * R0;
      for (int q = 0; q < 3; ++q) {
        /* d/dq of x^a y^b z^c R(r): a_q q^{a_q - 1} (others) R + (monomial) q R1 */
        double dm = 0.0;
        if (c[i][q] > 0) {
          dm = c[i][q];
          for (int p = 0; p < 3; ++p) dm *= pow(d[p], c[i][p] - (p == q ? 1 : 0));
        }
        gphi[q * nf + mu] = f * (dm * R0 + mono * d[q] * R1);
      }
    }
  }
}

int oracle_collocation_grad(int n_shells, const int *l, const int *nprim, const double *center,
                            const double *exps, const double *coefs, long npts, const double *xyz,
                            double *phi /* npts x nf */, double *gphi /* npts x 3 x nf */) {
  obasis b;
  if (obasis_init(&b, n_shells, l, nprim, center, exps, coefs)) return -1;
  for (long i = 0; i < npts; ++i)
    collocate_grad_point(&b, xyz + 3 * i, phi + i * b.n_func, gphi + i * 3 * b.n_func);
  obasis_free(&b);
  return 0;
}

/* V^xc and E_xc for a symmetric density matrix P, point by point:
 *   Phi, grad Phi                                  Eq. (collocation)
 *   F_mu = sum_nu P_{mu nu} Phi_nu                 Eq. (fmat)
 *   rho = sum_mu F_mu Phi_mu,
 *   grad rho = 2 sum_mu F_mu grad Phi_mu           Eq. (den_grid)
 *   eps, d eps/d rho, d eps/d sigma                Eq. (exc_grid)
 *   Z_mu = w/2 (eps_rho Phi_mu + 4 eps_sigma grad rho . grad Phi_mu)   Eq. (zmat)
 *   V_{mu nu} += Phi_mu Z_nu + Z_mu Phi_nu         Eq. (vxc_num)
 *   E_xc += w eps */
int oracle_vxc(int n_shells, const int *l, const int *nprim, const double *center, const double *exps,
               const double *coefs, long npts, const double *xyz, const double *w, const double *Pm,
               int functional, double *V, double *Exc, int nthreads) {
  if (functional < 1 || functional > 3) return -2;
  obasis b;
  if (obasis_init(&b, n_shells, l, nprim, center, exps, coefs)) return -1;
  int nf = b.n_func, nt = n_threads_or_default(nthreads);
  double *Vt = (double *)calloc((size_t)nt * nf * nf, sizeof(double));
  double *Et = (double *)calloc((size_t)nt, sizeof(double));
#pragma omp parallel num_threads(nt)
  {
#ifdef _OPENMP
    int tid = omp_get_thread_num();
#else
    int tid = 0;
#endif
    double *phi = (double *)malloc(sizeof(double) * nf);
    double *gphi = (double *)malloc(sizeof(double) * 3 * nf);
    double *F = (double *)malloc(sizeof(double) * nf);
    double *Z = (double *)malloc(sizeof(double) * nf);
    double *Vl = Vt + (size_t)tid * nf * nf;
#pragma omp for schedule(static)
    for (long i = 0; i < npts; ++i) {
      collocate_grad_point(&b, xyz + 3 * i, phi, gphi);
      for (int mu = 0; mu < nf; ++mu) {
        double s = 0.0;
        for (int nu = 0; nu < nf; ++nu) s += Pm[mu * nf + nu] * phi[nu];
        F[mu] = s;
      }
      double rho = 0.0, g[3] = {0.0, 0.0, 0.0};
      for (int mu = 0; mu < nf; ++mu) {
        rho += F[mu] * phi[mu];
        for (int q = 0; q < 3; ++q) g[q] += 2.0 * F[mu] * gphi[q * nf + mu];
      }
      double e[3];
      oracle_xc_point(functional, rho, g[0] * g[0] + g[1] * g[1] + g[2] * g[2], e);
      if (!(rho >= ORC_XC_RHO_MIN)) continue;
      Et[tid] += w[i] * e[0];
      for (int mu = 0; mu < nf; ++mu) {
        double gg = g[0] * gphi[mu] + g[1] * gphi[nf + mu] + g[2] * gphi[2 * nf + mu];
        Z[mu] = 0.5 * w[i] * (e[1] * phi[mu] + 4.0 * e[2] * gg);
      }
      for (int mu = 0; mu < nf; ++mu)
        for (int nu = 0; nu < nf; ++nu) Vl[mu * nf + nu] += phi[mu] * Z[nu] + Z[mu] * phi[nu];
    }
    free(phi);
    free(gphi);
    free(F);
    free(Z);
  }
  for (int x = 0; x < nf * nf; ++x) {
    double s = 0.0;
    for (int t = 0; t < nt; ++t) s += Vt[(size_t)t * nf * nf + x];
    V[x] = s;
  }
  double es = 0.0;
  for (int t = 0; t < nt; ++t) es += Et[t];
  *Exc = es;
  free(Vt);
  free(Et);
  obasis_free(&b);
  return 0;
}

/* Selected entries V_{mu_k nu_k} and E_xc of the same computation: per point
 * the density needs F over every function, but Z only over the functions of
 * the requested entries (all of them are formed here; the saving is the
 * N_b^2 accumulation of V). */
int oracle_vxc_entries(int n_shells, const int *l, const int *nprim, const double *center, const double *exps,
                       const double *coefs, long npts, const double *xyz, const double *w, const double *Pm,
                       int functional, int n_ent, const int *mu_e, const int *nu_e, double *Ve, double *Exc,
                       int nthreads) {
  if (functional < 1 || functional > 3) return -2;
  obasis b;
  if (obasis_init(&b, n_shells, l, nprim, center, exps, coefs)) return -1;
  int nf = b.n_func, nt = n_threads_or_default(nthreads);
  for (int k = 0; k < n_ent; ++k)
    if (mu_e[k] < 0 || mu_e[k] >= nf || nu_e[k] < 0 || nu_e[k] >= nf) {
      obasis_free(&b);
      return -3;
    }
  double *Vt = (double *)calloc((size_t)nt * (n_ent > 0 ? n_ent : 1), sizeof(double));
  double *Et = (double *)calloc((size_t)nt, sizeof(double));
#pragma omp parallel num_threads(nt)
  {
#ifdef _OPENMP
    int tid = omp_get_thread_num();
#else
    int tid = 0;
#endif
    double *phi = (double *)malloc(sizeof(double) * nf);
    double *gphi = (double *)malloc(sizeof(double) * 3 * nf);
    double *F = (double *)malloc(sizeof(double) * nf);
    double *Z = (double *)malloc(sizeof(double) * nf);
    double *Vl = Vt + (size_t)tid * (n_ent > 0 ? n_ent : 1);
#pragma omp for schedule(static)
    for (long i = 0; i < npts; ++i) {
      collocate_grad_point(&b, xyz + 3 * i, phi, gphi);
      for (int mu = 0; mu < nf; ++mu) {
        double s = 0.0;
        for (int nu = 0; nu < nf; ++nu) s += Pm[mu * nf + nu] * phi[nu];
        F[mu] = s;
      }
      double rho = 0.0, g[3] = {0.0, 0.0, 0.0};
      for (int mu = 0; mu < nf; ++mu) {
        rho += F[mu] * phi[mu];
        for (int q = 0; q < 3; ++q) g[q] += 2.0 * F[mu] * gphi[q * nf + mu];
      }
      if (!(rho >= ORC_XC_RHO_MIN)) continue;
      double e[3];
      oracle_xc_point(functional, rho, g[0] * g[0] + g[1] * g[1] + g[2] * g[2], e);
      Et[tid] += w[i] * e[0];
      for (int mu = 0; mu < nf; ++mu) {
        double gg = g[0] * gphi[mu] + g[1] * gphi[nf + mu] + g[2] * gphi[2 * nf + mu];
        Z[mu] = 0.5 * w[i] * (e[1] * phi[mu] + 4.0 * e[2] * gg);
      }
      for (int k = 0; k < n_ent; ++k) Vl[k] += phi[mu_e[k]] * Z[nu_e[k]] + Z[mu_e[k]] * phi[nu_e[k]];
    }
    free(phi);
    free(gphi);
    free(F);
    free(Z);
  }
  for (int k = 0; k < n_ent; ++k) {
    double s = 0.0;
    for (int t = 0; t < nt; ++t) s += Vt[(size_t)t * n_ent + k];
    Ve[k] = s;
  }
  double es = 0.0;
  for (int t = 0; t < nt; ++t) es += Et[t];
  *Exc = es;
  free(Vt);
  free(Et);
  obasis_free(&b);
  return 0;
}
