/* Becke fuzzy-cell partition weights for the seeded grids of synth/ (input
 * generation only: no arithmetic of the sn-K method lives here).
 *
 * For a point r and atoms A_a, with d_a = |r - A_a| and R_ab = |A_a - A_b|:
 *   mu_ab = (d_a - d_b) / R_ab,  f(x) = 3x/2 - x^3/2 iterated three times,
 *   s(mu) = (1 - f3(mu)) / 2,  P_a = prod_{b != a} s(mu_ab),
 *   w(r) = P_owner / sum_a P_a
 * (three-fold iterated polynomial, no atomic-size adjustment).
 *
 * The same definition as the torch routine of synth/__init__.py, fused per
 * point so that no (points x atoms x atoms) temporary is formed.  The factors
 * of each P_a are taken nearest atom first, and the product stops once it is
 * exactly zero (it can only stay zero), which makes large clusters cheap.
 */
#include <math.h>
#include <stdlib.h>

#include <omp.h>

static double becke_s(double mu) {
  double f = mu;
  for (int k = 0; k < 3; ++k) f = 1.5 * f - 0.5 * f * f * f;
  return 0.5 * (1.0 - f);
}

typedef struct {
  double d;
  int a;
} dist_t;

static int by_distance(const void *x, const void *y) {
  const dist_t *p = (const dist_t *)x, *q = (const dist_t *)y;
  if (p->d < q->d) return -1;
  if (p->d > q->d) return 1;
  return p->a - q->a;
}

/* w_out[i] = Becke weight of point i for its own atom owner[i]. */
int synth_becke(long npts, const double *xyz, const int *owner, int nat, const double *axyz, double *w_out,
                int nthreads) {
  if (npts < 0 || nat <= 0) return 1;
  if (nat == 1) {
    for (long i = 0; i < npts; ++i) w_out[i] = 1.0;
    return 0;
  }
  double *inv = (double *)malloc(sizeof(double) * (size_t)nat * nat);
  if (!inv) return 2;
  for (int a = 0; a < nat; ++a)
    for (int b = 0; b < nat; ++b) {
      const double dx = axyz[3 * a] - axyz[3 * b], dy = axyz[3 * a + 1] - axyz[3 * b + 1],
                   dz = axyz[3 * a + 2] - axyz[3 * b + 2];
      const double R = sqrt(dx * dx + dy * dy + dz * dz);
      inv[(size_t)a * nat + b] = (a != b && R > 0.0) ? 1.0 / R : 0.0;
    }
  int bad = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
  {
    dist_t *ord = (dist_t *)malloc(sizeof(dist_t) * (size_t)nat);
    double *d = (double *)malloc(sizeof(double) * (size_t)nat);
    if (!ord || !d) {
#pragma omp atomic write
      bad = 1;
    }
#pragma omp for schedule(dynamic, 1024)
    for (long i = 0; i < npts; ++i) {
      if (!ord || !d) continue;
      for (int a = 0; a < nat; ++a) {
        const double dx = xyz[3 * i] - axyz[3 * a], dy = xyz[3 * i + 1] - axyz[3 * a + 1],
                     dz = xyz[3 * i + 2] - axyz[3 * a + 2];
        d[a] = sqrt(dx * dx + dy * dy + dz * dz);
        ord[a].d = d[a];
        ord[a].a = a;
      }
      qsort(ord, (size_t)nat, sizeof(dist_t), by_distance);
      double tot = 0.0, mine = 0.0;
      for (int a = 0; a < nat; ++a) {
        double P = 1.0;
        const double *ia = inv + (size_t)a * nat;
        for (int t = 0; t < nat && P != 0.0; ++t) {
          const int b = ord[t].a;
          if (b == a) continue;
          P *= becke_s((d[a] - d[b]) * ia[b]);
        }
        tot += P;
        if (a == owner[i]) mine = P;
      }
      w_out[i] = tot > 0.0 ? mine / tot : 0.0;
    }
    free(ord);
    free(d);
  }
  free(inv);
  return bad ? 2 : 0;
}
