// Host-side geometry setup of libsnk: validation, normalisation of the
// contracted Cartesian shells, shell pairs with primitive-pair data and
// rigorous integral bounds, octree batching of the grid (Sec. II.E), the
// basis screen B_j (Eq. basis_screen) and the Boys interpolation table.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>

#include "snk_internal.h"

namespace snk {

namespace {

constexpr double kPi = 3.14159265358979323846;

double odd_dfact(int n) {  // n!! for odd n >= -1
  double r = 1.0;
  for (int k = n; k > 1; k -= 2) r *= k;
  return r;
}

bool finite(double x) { return std::isfinite(x); }

void cart(int l, int c[][3]) {
  int k = 0;
  for (int ax = l; ax >= 0; --ax)
    for (int ay = l - ax; ay >= 0; --ay) {
      c[k][0] = ax;
      c[k][1] = ay;
      c[k][2] = l - ax - ay;
      ++k;
    }
}

// Octree partition of the points idx[lo, hi) (Sec. II.E): split the bounding
// box at its centre into octants until a leaf holds at most bmax points.
void octree(std::vector<int64_t>& idx, size_t lo, size_t hi, const double* xyz, int bmax, int depth,
            std::vector<std::pair<size_t, size_t>>& leaves) {
  size_t n = hi - lo;
  if (n == 0) return;
  if (n <= (size_t)bmax) {
    leaves.emplace_back(lo, hi);
    return;
  }
  double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
  for (size_t k = lo; k < hi; ++k)
    for (int q = 0; q < 3; ++q) {
      double v = xyz[3 * idx[k] + q];
      mn[q] = std::min(mn[q], v);
      mx[q] = std::max(mx[q], v);
    }
  bool degenerate = (mx[0] - mn[0]) + (mx[1] - mn[1]) + (mx[2] - mn[2]) <= 0.0;
  if (degenerate || depth > 48) {  // identical points: cut into consecutive leaves
    for (size_t k = lo; k < hi; k += bmax) leaves.emplace_back(k, std::min(hi, k + bmax));
    return;
  }
  double c[3] = {0.5 * (mn[0] + mx[0]), 0.5 * (mn[1] + mx[1]), 0.5 * (mn[2] + mx[2])};
  std::vector<int64_t> bucket[8];
  for (size_t k = lo; k < hi; ++k) {
    const double* p = xyz + 3 * idx[k];
    int o = (p[0] >= c[0] ? 1 : 0) | (p[1] >= c[1] ? 2 : 0) | (p[2] >= c[2] ? 4 : 0);
    bucket[o].push_back(idx[k]);
  }
  size_t pos = lo;
  size_t starts[9];
  for (int o = 0; o < 8; ++o) {
    starts[o] = pos;
    for (int64_t v : bucket[o]) idx[pos++] = v;
  }
  starts[8] = pos;
  for (int o = 0; o < 8; ++o) octree(idx, starts[o], starts[o + 1], xyz, bmax, depth + 1, leaves);
}

}  // namespace

// Boys function for the device table: for T <= 30 a power series at order 40
// followed by downward recursion F_n = (2T F_{n+1} + e^{-T}) / (2n+1); above,
// F_0 from erf and upward recursion F_{n+1} = ((2n+1) F_n - e^{-T}) / (2T).
void host_boys(int nmax, double T, double* F) {
  double e = std::exp(-T);
  if (T <= 30.0) {
    const int ntop = 40;
    double term = 1.0 / (2 * ntop + 1), sum = term;
    for (int k = 1; k < 400; ++k) {
      term *= 2.0 * T / (2 * ntop + 2 * k + 1);
      sum += term;
      if (term < 1e-20 * sum) break;
    }
    double f = e * sum;
    for (int n = ntop - 1; n >= 0; --n) {
      f = (2.0 * T * f + e) / (2 * n + 1);
      if (n <= nmax) F[n] = f;
    }
  } else {
    F[0] = 0.5 * std::sqrt(kPi / T) * std::erf(std::sqrt(T));
    for (int n = 0; n < nmax; ++n) F[n + 1] = ((2 * n + 1) * F[n] - e) / (2.0 * T);
  }
}

// Rigorous bound of max_r |A_{mu lam}(r)| for the normalised shell pair.
// |x_A^a ...| <= |r' - A|^{l_a} <= (s + |P - A|)^{l_a} with s = |r' - P|, and
// the potential of a positive, spherically symmetric charge is largest at its
// centre, so |A| <= sum |d d'| f f' K_ab 4 pi int_0^inf s (s+dA)^la (s+dB)^lb
// exp(-zeta s^2) ds, each power integrated in closed form.
// Bounds of one primitive pair (k of shell sa, m of shell sb), normalised
// coefficients and the largest component factors included:
//   *abound >= max_r |A^{km}(r)|  (the potential at the charge's centre), and
//   *qbound >= int |phi_k phi_m| d^3r (the total charge), so that at distance
//   D from the Gaussian product centre |A^{km}| <= *qbound / D.
// |x_A^a ...| <= |r' - A|^{l_a} <= (s + |P - A|)^{l_a} with s = |r' - P|; the
// potential of a positive, spherically symmetric charge is largest at its
// centre and at most Q / D outside; every power of s integrates in closed form.
void prim_pair_bounds(const Setup& s, int sa, int sb, int k, int m, double* abound, double* qbound) {
  const double fmax[3] = {1.0, 1.0, std::sqrt(3.0)};
  const int la = s.l[sa], lb = s.l[sb];
  const double* A = &s.center[3 * sa];
  const double* B = &s.center[3 * sb];
  double ab2 = 0.0;
  for (int q = 0; q < 3; ++q) ab2 += (A[q] - B[q]) * (A[q] - B[q]);
  const double al = s.exps[k], be = s.exps[m], z = al + be;
  const double K = std::exp(-al * be / z * ab2);
  double dA = 0.0, dB = 0.0;
  for (int q = 0; q < 3; ++q) {
    double P = (al * A[q] + be * B[q]) / z;
    dA += (P - A[q]) * (P - A[q]);
    dB += (P - B[q]) * (P - B[q]);
  }
  dA = std::sqrt(dA);
  dB = std::sqrt(dB);
  // polynomial (s + dA)^la (s + dB)^lb = sum_j c_j s^j
  double c[5] = {1, 0, 0, 0, 0};
  int deg = 0;
  for (int t = 0; t < la + lb; ++t) {
    double d = t < la ? dA : dB;
    for (int j = deg + 1; j >= 0; --j) c[j] = (j > 0 ? c[j - 1] : 0.0) + d * c[j];
    ++deg;
  }
  // int_0^inf s^{j+1} e^{-z s^2} ds = Gamma((j+2)/2) / (2 z^{(j+2)/2}), and
  // int_0^inf s^{j+2} e^{-z s^2} ds = Gamma((j+3)/2) / (2 z^{(j+3)/2})
  static const double g2[5] = {0.5, 0.44311346272637900682, 0.5, 0.66467019408956851023, 1.0};
  static const double g3[5] = {0.44311346272637900682, 0.5, 0.66467019408956851023, 1.0, 1.66167548522392127557};
  const double rz = 1.0 / std::sqrt(z);
  double zp = rz * rz, ia = 0.0, iq = 0.0;
  for (int j = 0; j <= deg; ++j) {
    ia += c[j] * g2[j] * zp;
    iq += c[j] * g3[j] * zp * rz;
    zp *= rz;
  }
  const double pre = std::fabs(s.d[k] * s.d[m]) * K * 4.0 * kPi * fmax[la] * fmax[lb];
  *abound = pre * ia;
  *qbound = pre * iq;
}

double pair_bound(const Setup& s, int sa, int sb) {
  double total = 0.0, a, q;
  for (int k = s.poff[sa]; k < s.poff[sa] + s.nprim[sa]; ++k)
    for (int m = s.poff[sb]; m < s.poff[sb] + s.nprim[sb]; ++m) {
      prim_pair_bounds(s, sa, sb, k, m, &a, &q);
      total += a;
    }
  return total;
}

namespace {

// Setup of one molecule (indices local to it).
int build_setup_one(const snk_basis* basis, const snk_grid* grid, const snk_options* opt, Setup* s,
                    std::string* msg) {
  if (!basis || !grid || !opt) {
    *msg = "NULL basis, grid or options";
    return SNK_ERR_INVALID_ARG;
  }
  const int ns = basis->n_shells;
  if (ns <= 0 || !basis->l || !basis->nprim || !basis->center || !basis->exps || !basis->coefs) {
    *msg = "basis: n_shells must be positive and all arrays non-NULL";
    return SNK_ERR_INVALID_ARG;
  }
  if (grid->n_points < 0 || (grid->n_points > 0 && (!grid->xyz || !grid->w || !grid->atom))) {
    *msg = "grid: n_points must be >= 0 and arrays non-NULL";
    return SNK_ERR_INVALID_ARG;
  }
  if (opt->batch_max < 1 || opt->batch_max > (1 << 20)) {
    *msg = "options: batch_max must be in [1, 2^20]";
    return SNK_ERR_INVALID_ARG;
  }
  s->ns = ns;
  s->l.assign(basis->l, basis->l + ns);
  s->nprim.assign(basis->nprim, basis->nprim + ns);
  s->atom.assign(ns, 0);
  if (basis->atom) s->atom.assign(basis->atom, basis->atom + ns);
  s->poff.resize(ns + 1);
  s->foff.resize(ns + 1);
  int np = 0, nf = 0;
  for (int a = 0; a < ns; ++a) {
    if (s->l[a] < 0 || s->l[a] > kLMax) {
      *msg = "basis: angular momentum must be 0, 1 or 2";
      return SNK_ERR_UNSUPPORTED;
    }
    if (s->nprim[a] < 1 || s->nprim[a] > 16) {
      *msg = "basis: nprim must be in [1, 16]";
      return SNK_ERR_UNSUPPORTED;
    }
    s->poff[a] = np;
    s->foff[a] = nf;
    np += s->nprim[a];
    nf += ncart(s->l[a]);
  }
  s->poff[ns] = np;
  s->foff[ns] = nf;
  s->nf = nf;
  s->nprim_total = np;
  s->center.assign(basis->center, basis->center + 3 * ns);
  s->exps.assign(basis->exps, basis->exps + np);
  for (double v : s->center)
    if (!finite(v)) {
      *msg = "basis: non-finite centre";
      return SNK_ERR_UNSUPPORTED;
    }
  for (int k = 0; k < np; ++k)
    if (!finite(basis->exps[k]) || basis->exps[k] <= 0.0 || !finite(basis->coefs[k])) {
      *msg = "basis: exponents must be finite and positive, coefficients finite";
      return SNK_ERR_UNSUPPORTED;
    }

  // normalisation: unit self-overlap of every Cartesian component
  s->d.resize(np);
  s->fcomp.resize(nf);
  s->fshell.resize(nf);
  for (int a = 0; a < ns; ++a) {
    int la = s->l[a], p0 = s->poff[a], n = s->nprim[a];
    for (int k = 0; k < n; ++k) {
      double al = s->exps[p0 + k];
      double N = std::pow(2.0 * al / kPi, 0.75) * std::pow(4.0 * al, 0.5 * la) / std::sqrt(odd_dfact(2 * la - 1));
      s->d[p0 + k] = basis->coefs[p0 + k] * N;
    }
    double S = 0.0;
    for (int k = 0; k < n; ++k)
      for (int m = 0; m < n; ++m) {
        double g = s->exps[p0 + k] + s->exps[p0 + m];
        S += s->d[p0 + k] * s->d[p0 + m] * std::pow(kPi / g, 1.5) * odd_dfact(2 * la - 1) / std::pow(2.0 * g, la);
      }
    if (!(S > 0.0) || !finite(S)) {
      *msg = "basis: contraction has non-positive norm";
      return SNK_ERR_UNSUPPORTED;
    }
    double inv = 1.0 / std::sqrt(S);
    for (int k = 0; k < n; ++k) s->d[p0 + k] *= inv;
    int c[6][3];
    cart(la, c);
    for (int i = 0; i < ncart(la); ++i) {
      s->fcomp[s->foff[a] + i] =
          std::sqrt(odd_dfact(2 * la - 1) / (odd_dfact(2 * c[i][0] - 1) * odd_dfact(2 * c[i][1] - 1) *
                                             odd_dfact(2 * c[i][2] - 1)));
      s->fshell[s->foff[a] + i] = a;
    }
  }

  // cutoff radius of each shell for the basis screen, Eq. (basis_screen)
  s->rcut.assign(ns, 1e300);
  if (opt->eps_basis > 0.0) {
    const double fmax[3] = {1.0, 1.0, std::sqrt(3.0)};
    for (int a = 0; a < ns; ++a) {
      // scan down from a radius where every primitive is far below eps_basis
      double amin = 1e300, dsum = 0.0;
      for (int k = s->poff[a]; k < s->poff[a + 1]; ++k) {
        amin = std::min(amin, s->exps[k]);
        dsum += std::fabs(s->d[k]);
      }
      double r = std::sqrt((std::log(std::max(dsum, 1.0) * 10.0 / opt->eps_basis) + 60.0) / amin) + 1.0;
      const double step = 0.01;
      for (; r > 0.0; r -= step) {
        double g = 0.0;
        for (int k = s->poff[a]; k < s->poff[a + 1]; ++k) g += std::fabs(s->d[k]) * std::exp(-s->exps[k] * r * r);
        g *= fmax[s->l[a]] * std::pow(r, s->l[a]);
        if (g >= opt->eps_basis) break;
      }
      s->rcut[a] = std::max(r, 0.0) + step;
    }
  }

  // shell pairs, class-major, with primitive-pair data and bounds
  s->pair_index.assign((size_t)ns * ns, -1);
  std::vector<std::vector<std::pair<int, int>>> bycls(kNumClasses);
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b) {
      int la = s->l[a], lb = s->l[b];
      if (la < lb || (la == lb && a < b)) continue;
      bycls[class_of(la, lb)].emplace_back(a, b);
    }
  s->pairs.clear();
  s->prims.clear();
  s->bound.clear();
  s->qbound.clear();
  s->pair_class.clear();
  for (int c = 0; c < kNumClasses; ++c) {
    s->class_begin[c] = (int)s->pairs.size();
    for (auto& ab : bycls[c]) {
      int a = ab.first, b = ab.second;
      // primitive pairs whose potential is below kPrimPairTol everywhere are
      // left out; a pair with no primitive left is dropped
      double bnd = 0.0, qb = 0.0;
      std::vector<std::pair<int, int>> keep;
      std::vector<double> kb;
      for (int k = s->poff[a]; k < s->poff[a + 1]; ++k)
        for (int m = s->poff[b]; m < s->poff[b + 1]; ++m) {
          double pa, pq;
          prim_pair_bounds(*s, a, b, k, m, &pa, &pq);
          if (pa >= kPrimPairTol) {
            keep.emplace_back(k, m);
            kb.push_back(pa);
            bnd += pa;
            qb += pq;
          }
        }
      if (keep.empty()) continue;
      // largest bound first (stable, so ties keep the input order); the FP32
      // tier takes the leading ones down to kPrimPairRelTolF32 of the largest
      std::vector<int> ord(keep.size());
      for (size_t q = 0; q < ord.size(); ++q) ord[q] = (int)q;
      std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return kb[x] > kb[y]; });
      std::vector<std::pair<int, int>> sorted_keep;
      int n32 = 0;
      for (int q : ord) {
        sorted_keep.push_back(keep[q]);
        if (kb[q] >= kPrimPairRelTolF32 * kb[ord[0]]) ++n32;
        s->prim_rel.push_back(kb[q] / bnd);  // the primitive pair's share of the pair's bound
      }
      keep.swap(sorted_keep);
      PairHdr h;
      h.sa = a;
      h.sb = b;
      h.pp_off = (int)s->prims.size();
      h.pp_n = (int)keep.size();
      const double* A = &s->center[3 * a];
      const double* B = &s->center[3 * b];
      h.ABx = A[0] - B[0];
      h.ABy = A[1] - B[1];
      h.ABz = A[2] - B[2];
      h.pp_n32 = n32;
      h.pad = 0;
      double ab2 = h.ABx * h.ABx + h.ABy * h.ABy + h.ABz * h.ABz;
      for (auto& km : keep) {
        {
          const int k = km.first, m = km.second;
          double al = s->exps[k], be = s->exps[m], z = al + be;
          PrimPair p;
          p.zeta = z;
          p.Px = (al * A[0] + be * B[0]) / z;
          p.Py = (al * A[1] + be * B[1]) / z;
          p.Pz = (al * A[2] + be * B[2]) / z;
          p.PAx = p.Px - A[0];
          p.PAy = p.Py - A[1];
          p.PAz = p.Pz - A[2];
          p.pref = 2.0 * kPi / z * std::exp(-al * be / z * ab2) * s->d[k] * s->d[m];
          p.pref_far = p.pref * 0.5 * std::sqrt(kPi);
          p.k1 = 0.5 / z;
          p.k2 = 1.0 / z;
          p.k3 = 1.5 / z;
          s->prims.push_back(p);
        }
      }
      s->pair_index[(size_t)a * ns + b] = (int)s->pairs.size();
      s->pair_index[(size_t)b * ns + a] = (int)s->pairs.size();
      s->pairs.push_back(h);
      s->bound.push_back(bnd);
      s->qbound.push_back(qb);
      s->pair_class.push_back(c);
    }
  }
  s->class_begin[kNumClasses] = (int)s->pairs.size();

  // grid: validate, then atom-centred octree batches
  const int64_t npts = grid->n_points;
  s->npts = npts;
  for (int64_t i = 0; i < npts; ++i) {
    if (!finite(grid->xyz[3 * i]) || !finite(grid->xyz[3 * i + 1]) || !finite(grid->xyz[3 * i + 2]) ||
        !finite(grid->w[i])) {
      *msg = "grid: non-finite point or weight";
      return SNK_ERR_UNSUPPORTED;
    }
    if (grid->atom[i] < 0) {
      *msg = "grid: negative atom index";
      return SNK_ERR_INVALID_ARG;
    }
  }
  std::vector<int64_t> idx(npts);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return grid->atom[x] < grid->atom[y]; });
  std::vector<std::pair<size_t, size_t>> leaves;
  size_t lo = 0;
  while (lo < (size_t)npts) {
    size_t hi = lo;
    while (hi < (size_t)npts && grid->atom[idx[hi]] == grid->atom[idx[lo]]) ++hi;
    octree(idx, lo, hi, grid->xyz, opt->batch_max, 0, leaves);
    lo = hi;
  }
  // inside each batch, the points in the order of a finer octree (leaves of at
  // most kPointTile points): the 128-point tiles of the integral kernels are
  // then spatially compact, which the per-tile screen exploits
  for (const auto& lf : leaves) {
    std::vector<std::pair<size_t, size_t>> sub;
    octree(idx, lf.first, lf.second, grid->xyz, kPointTile, 0, sub);
  }
  s->perm = idx;
  s->xyz.resize(3 * npts);
  s->w.resize(npts);
  for (int64_t k = 0; k < npts; ++k) {
    for (int q = 0; q < 3; ++q) s->xyz[3 * k + q] = grid->xyz[3 * idx[k] + q];
    s->w[k] = grid->w[idx[k]];
  }
  const int nb = (int)leaves.size();
  s->bstart.resize(nb + 1);
  s->bcenter.resize(3 * nb);
  s->bradius.resize(nb);
  for (int j = 0; j < nb; ++j) {
    s->bstart[j] = (int64_t)leaves[j].first;
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (size_t k = leaves[j].first; k < leaves[j].second; ++k)
      for (int q = 0; q < 3; ++q) {
        mn[q] = std::min(mn[q], s->xyz[3 * k + q]);
        mx[q] = std::max(mx[q], s->xyz[3 * k + q]);
      }
    double r2 = 0.0;
    for (int q = 0; q < 3; ++q) s->bcenter[3 * j + q] = 0.5 * (mn[q] + mx[q]);
    for (size_t k = leaves[j].first; k < leaves[j].second; ++k) {
      double d2 = 0.0;
      for (int q = 0; q < 3; ++q) d2 += (s->xyz[3 * k + q] - s->bcenter[3 * j + q]) * (s->xyz[3 * k + q] - s->bcenter[3 * j + q]);
      r2 = std::max(r2, d2);
    }
    s->bradius[j] = std::sqrt(r2);
  }
  s->bstart[nb] = npts;

  // basis screen B_j: shells whose cutoff sphere meets the batch's bounding sphere
  s->bshell_off.assign(nb + 1, 0);
  s->bshell.clear();
  s->bnf.assign(nb, 0);
  s->xfunc_off.assign(nb + 1, 0);
  s->xfunc.clear();
  for (int j = 0; j < nb; ++j) {
    s->bshell_off[j] = (int)s->bshell.size();
    s->xfunc_off[j] = (int)s->xfunc.size();
    for (int a = 0; a < ns; ++a) {
      double d2 = 0.0;
      for (int q = 0; q < 3; ++q) d2 += (s->center[3 * a + q] - s->bcenter[3 * j + q]) * (s->center[3 * a + q] - s->bcenter[3 * j + q]);
      if (std::sqrt(d2) - s->bradius[j] <= s->rcut[a]) {
        s->bshell.push_back(a);
        for (int i = 0; i < ncart(s->l[a]); ++i) s->xfunc.push_back(s->foff[a] + i);
        s->bnf[j] += ncart(s->l[a]);
      }
    }
  }
  s->bshell_off[nb] = (int)s->bshell.size();
  s->xfunc_off[nb] = (int)s->xfunc.size();
  return SNK_OK;
}

}  // namespace

// Boys interpolation tables of the FP64 and FP32 integral kernels.
void build_boys_tables(Setup* s) {
  // Boys table per L: F_{L+m}(T_k)/m!, exp(-T_k), T_k
  s->boys.assign((size_t)(kBoysLMax + 1) * kBoysRows * kBoysCols, 0.0);
  double F[kBoysLMax + kBoysTerms + 1];
  double invfact[kBoysTerms];
  invfact[0] = 1.0;
  for (int m = 1; m < kBoysTerms; ++m) invfact[m] = invfact[m - 1] / m;
  for (int k = 0; k < kBoysRows; ++k) {
    double T = k * kBoysH;
    host_boys(kBoysLMax + kBoysTerms, T, F);
    for (int L = 0; L <= kBoysLMax; ++L) {
      double* row = &s->boys[((size_t)L * kBoysRows + k) * kBoysCols];
      for (int m = 0; m < kBoysTerms; ++m) row[m] = F[L + m] * invfact[m];
      row[kBoysTerms] = std::exp(-T);
      row[kBoysTerms + 1] = T;
    }
  }
  // ds table of the mixed form: nodes T_k rounded to (hi, lo) float pairs and
  // the values at those nodes split the same way, so that T_k - T is exact in
  // ds arithmetic
  s->boys_ds.assign((size_t)(kBoysLMax + 1) * kBoysRows * kBoysCols * 2, 0.0f);
  for (int k = 0; k < kBoysRows; ++k) {
    const double T0 = k * kBoysH;
    const float th = (float)T0;
    const float tl = (float)(T0 - (double)th);
    const double T = (double)th + (double)tl;
    host_boys(kBoysLMax + kBoysTerms, T, F);
    for (int L = 0; L <= kBoysLMax; ++L) {
      float* row = &s->boys_ds[(((size_t)L * kBoysRows + k) * kBoysCols) * 2];
      double v[kBoysCols];
      for (int m = 0; m < kBoysTerms; ++m) v[m] = F[L + m] * invfact[m];
      v[kBoysTerms] = std::exp(-T);
      for (int m = 0; m < kBoysTerms + 1; ++m) {
        row[2 * m] = (float)v[m];
        row[2 * m + 1] = (float)(v[m] - (double)row[2 * m]);
      }
      row[2 * (kBoysTerms + 1)] = th;
      row[2 * (kBoysTerms + 1) + 1] = tl;
    }
  }
  // FP32 table of the mixed form: nodes at the float values fl32(k * 0.05f)
  // that the kernel forms itself, four Taylor coefficients per row
  s->boys_f.assign((size_t)(kBoysLMax + 1) * kBoysRowsF * kBoysColsF, 0.0f);
  for (int k = 0; k < kBoysRowsF; ++k) {
    const float tk = (float)k * kBoysHF;
    host_boys(kBoysLMax + kBoysTermsF, (double)tk, F);
    for (int L = 0; L <= kBoysLMax; ++L) {
      float* row = &s->boys_f[((size_t)L * kBoysRowsF + k) * kBoysColsF];
      for (int m = 0; m < kBoysTermsF; ++m) row[m] = (float)(F[L + m] * invfact[m]);
    }
  }
}

// Several independent molecules in one handle: each is set up on its own
// (normalisation, pairs, octree batches, basis screen), then everything is
// concatenated.  Shell, pair and batch indices become global; function
// indices inside the X / F / G column lists stay local to their molecule,
// whose P and K blocks are packed one after another (row-major, N_b,m^2 each).
int build_setup(int n_mol, const snk_basis* bases, const snk_grid* grids, const snk_options* opt, Setup* s,
                std::string* msg) {
  if (n_mol < 1 || !bases || !grids || !opt) {
    *msg = "need at least one molecule and non-NULL basis, grid and options arrays";
    return SNK_ERR_INVALID_ARG;
  }
  *s = Setup();
  s->n_mol = n_mol;
  int64_t pk = 0, pi = 0, npts = 0;
  for (int m = 0; m < n_mol; ++m) {
    Setup one;
    std::string err;
    int rc = build_setup_one(&bases[m], &grids[m], opt, &one, &err);
    if (rc != SNK_OK) {
      *msg = (n_mol > 1 ? "molecule " + std::to_string(m) + ": " : std::string()) + err;
      return rc;
    }
    Setup::Mol mol;
    mol.ms0 = s->ns;
    mol.ns = one.ns;
    mol.mf0 = s->nf;
    mol.nf = one.nf;
    mol.mb0 = (int)s->bcenter.size() / 3;
    mol.nb = (int)one.bstart.size() - 1;
    mol.pk_off = pk;
    mol.pi_off = pi;
    mol.p0 = npts;
    mol.npts = one.npts;
    const int pp0 = (int)s->prims.size(), np0 = s->nprim_total, pr0 = (int)s->pairs.size();
    for (int c = 0; c <= kNumClasses; ++c) mol.cr[c] = pr0 + one.class_begin[c];
    pk += (int64_t)one.nf * one.nf;
    pi += (int64_t)one.ns * one.ns;
    // shells and functions
    for (int a = 0; a < one.ns; ++a) {
      s->l.push_back(one.l[a]);
      s->nprim.push_back(one.nprim[a]);
      s->poff.push_back(one.poff[a] + np0);
      s->foff.push_back(one.foff[a] + s->nf);
      s->atom.push_back(one.atom[a]);
      s->rcut.push_back(one.rcut[a]);
      for (int q = 0; q < 3; ++q) s->center.push_back(one.center[3 * a + q]);
    }
    s->exps.insert(s->exps.end(), one.exps.begin(), one.exps.end());
    s->d.insert(s->d.end(), one.d.begin(), one.d.end());
    s->fcomp.insert(s->fcomp.end(), one.fcomp.begin(), one.fcomp.end());
    for (int f : one.fshell) s->fshell.push_back(f + mol.ms0);
    // pairs (class-major within the molecule)
    for (size_t p = 0; p < one.pairs.size(); ++p) {
      PairHdr h = one.pairs[p];
      h.sa += mol.ms0;
      h.sb += mol.ms0;
      h.pp_off += pp0;
      s->pairs.push_back(h);
    }
    s->prims.insert(s->prims.end(), one.prims.begin(), one.prims.end());
    s->prim_rel.insert(s->prim_rel.end(), one.prim_rel.begin(), one.prim_rel.end());
    s->bound.insert(s->bound.end(), one.bound.begin(), one.bound.end());
    s->qbound.insert(s->qbound.end(), one.qbound.begin(), one.qbound.end());
    s->pair_class.insert(s->pair_class.end(), one.pair_class.begin(), one.pair_class.end());
    for (int v : one.pair_index) s->pair_index.push_back(v < 0 ? -1 : v + pr0);
    // grid and batches
    for (int64_t v : one.perm) s->perm.push_back(v + npts);
    s->xyz.insert(s->xyz.end(), one.xyz.begin(), one.xyz.end());
    s->w.insert(s->w.end(), one.w.begin(), one.w.end());
    for (int j = 0; j < mol.nb; ++j) {
      s->bstart.push_back(one.bstart[j] + npts);
      s->bmol.push_back(m);
      s->bradius.push_back(one.bradius[j]);
      for (int q = 0; q < 3; ++q) s->bcenter.push_back(one.bcenter[3 * j + q]);
      s->bshell_off.push_back((int)s->bshell.size() + one.bshell_off[j]);
      s->xfunc_off.push_back((int)s->xfunc.size() + one.xfunc_off[j]);
      s->bnf.push_back(one.bnf[j]);
      s->cm_off.push_back(s->cm_total);
      s->phf_off.push_back(s->phf_total);
      s->cm_total += one.ns;
      s->phf_total += one.nf;
    }
    for (int a : one.bshell) s->bshell.push_back(a + mol.ms0);
    s->xfunc.insert(s->xfunc.end(), one.xfunc.begin(), one.xfunc.end());  // local function indices
    s->ns += one.ns;
    s->nf += one.nf;
    s->nprim_total += one.nprim_total;
    npts += one.npts;
    s->mols.push_back(mol);
  }
  s->poff.push_back(s->nprim_total);
  s->foff.push_back(s->nf);
  s->bstart.push_back(npts);
  s->bshell_off.push_back((int)s->bshell.size());
  s->xfunc_off.push_back((int)s->xfunc.size());
  s->npts = npts;
  s->packed = pk;
  for (int c = 0; c <= kNumClasses; ++c) s->class_begin[c] = c == kNumClasses ? (int)s->pairs.size() : 0;
  build_boys_tables(s);
  return SNK_OK;
}

}  // namespace snk
