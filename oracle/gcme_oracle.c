/*
 * gcme_oracle.c -- plain FP64 CPU oracle for the GCMe nonbonded model.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  It shares no code,
 * header, table or helper with the CUDA path and is never linked into it;
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg use it.
 *
 * Model (reduced units kT = 1, lengths in d, charges in e, Coulomb
 * prefactor e^2/(4 pi eps0 eps_r) = lB kT):
 *   u_ex(r)   = A_ij (3/(2 pi s_ij))^{3/2} exp(-3 r^2 / (2 s_ij)),
 *               s_ij = sigma_i^2 + sigma_j^2                     (Eq. u_ex)
 *   u_elec(r) = lB z_i z_j erf(beta_ij r) / r,
 *               beta_ij = sqrt(pi) / (sqrt(2) a_ij), a_ij^2 = a_i^2 + a_j^2
 *                                                               (Eq. u_elec)
 *   U_elec    = real + recip + corr + self                      (Eq. ewald)
 *     real  = sum'_{pairs,images, r<rc} lB z_i z_j [erf(beta r)-erf(kappa r)]/r
 *     recip = (2 pi lB / V) sum_{k!=0} exp(-k^2/(4 kappa^2))/k^2 |S(k)|^2
 *     corr  = -lB kappa/sqrt(pi) sum z_i^2
 *     self  = +lB sum z_i^2 / (2 a_i)     (the Born energy)
 *   with kappa = 1/(sqrt(2) G).
 *
 * Every routine works on explicit arrays: pos is (n,3) row-major FP64.
 * Compiled with -ffp-contract=off so that float expressions round exactly
 * as written (the FP32 neighbour rule below depends on it).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_2_SQRTPI 1.12837916709551257390 /* 2/sqrt(pi) */

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Periodic wrapping and the FP32 neighbour rule.                            */
/* ------------------------------------------------------------------------ */

/* Wrap one coordinate into [0, L): x - L*floor(x/L), each operation rounded
 * once; a result that rounds to L (or below 0) maps to 0. */
static double wrap1(double x, double L) {
  double s = x / L;
  double f = floor(s);
  double t = L * f;
  double w = x - t;
  if (w >= L) w = 0.0;
  if (w < 0.0) w = 0.0;
  return w;
}

void orc_wrap(int64_t n, const double *pos, const double *box, double *out) {
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) out[3 * i + a] = wrap1(pos[3 * i + a], box[a]);
}

/* In-cutoff decision for the ordered triple (i, j, image shift n), made in
 * FP32 on the wrapped positions rounded to float:
 *   d_a = fl(fl(x_j,a - x_i,a) + fl(n_a L_a)),
 *   r2  = fl(fl(fl(d_x d_x) + fl(d_y d_y)) + fl(d_z d_z)),
 *   in  iff r2 < fl(rc^2).
 * The rule is antisymmetric in (i,j,n) <-> (j,i,-n), so the set of in-cutoff
 * pairs is symmetric. */
static int in_cutoff_f32(const float *xi, const float *xj, const float *shift,
                         float rc2) {
  float d0 = xj[0] - xi[0];
  float d1 = xj[1] - xi[1];
  float d2 = xj[2] - xi[2];
  d0 = d0 + shift[0];
  d1 = d1 + shift[1];
  d2 = d2 + shift[2];
  float p0 = d0 * d0;
  float p1 = d1 * d1;
  float p2 = d2 * d2;
  float r2 = p0 + p1;
  r2 = r2 + p2;
  return r2 < rc2;
}

/* Number of periodic images to enumerate along one axis. */
static int image_range(double L, double rc) {
  int m = (int)ceil(rc / L);
  return m < 1 ? 1 : m;
}

/* Enumerate every ordered in-cutoff triple (i, j, n) by brute force over all
 * j and all image shifts n.  shift code = (nx+1) + 3 (ny+1) + 9 (nz+1) when
 * every |n_a| <= 1.  Writes up to cap triples into out (i, j, code) and
 * returns the total count. */
int64_t orc_pair_set(int64_t n, const double *pos, const double *box, double rc,
                     int64_t cap, int32_t *out) {
  double *w = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  float *f = (float *)malloc(sizeof(float) * 3 * (size_t)n);
  orc_wrap(n, pos, box, w);
  for (int64_t i = 0; i < 3 * n; ++i) f[i] = (float)w[i];
  float Lf[3] = {(float)box[0], (float)box[1], (float)box[2]};
  float rc2 = (float)(rc * rc);
  int m[3];
  for (int a = 0; a < 3; ++a) m[a] = image_range(box[a], rc);
  int64_t cnt = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j)
      for (int nz = -m[2]; nz <= m[2]; ++nz)
        for (int ny = -m[1]; ny <= m[1]; ++ny)
          for (int nx = -m[0]; nx <= m[0]; ++nx) {
            if (i == j && nx == 0 && ny == 0 && nz == 0) continue;
            float sh[3] = {(float)nx * Lf[0], (float)ny * Lf[1], (float)nz * Lf[2]};
            if (!in_cutoff_f32(f + 3 * i, f + 3 * j, sh, rc2)) continue;
            if (cnt < cap) {
              out[3 * cnt + 0] = (int32_t)i;
              out[3 * cnt + 1] = (int32_t)j;
              out[3 * cnt + 2] = (nx + 1) + 3 * (ny + 1) + 9 * (nz + 1);
            }
            ++cnt;
          }
  free(w);
  free(f);
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* Cell list (counting sort).                                                 */
/* ------------------------------------------------------------------------ */

/* Cell of every bead and the beads of each cell in (cls, index) order.
 * Cell coordinate c_a = floor(x_w,a * (nc_a / L_a)) clamped to [0, nc_a-1],
 * computed in FP64 from the wrapped position; cell id = cx + nx (cy + ny cz).
 * cell_start has ncell+1 entries. */
void orc_cell_list(int64_t n, const double *pos, const double *box,
                   const int32_t *nc, const int32_t *cls, int32_t ncls,
                   int32_t *cell_of, int32_t *cell_start, int32_t *sorted_idx) {
  int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
  double inv[3];
  for (int a = 0; a < 3; ++a) inv[a] = (double)nc[a] / box[a];
  for (int64_t i = 0; i < n; ++i) {
    int c[3];
    for (int a = 0; a < 3; ++a) {
      double w = wrap1(pos[3 * i + a], box[a]);
      double s = w * inv[a];
      int k = (int)floor(s);
      if (k > nc[a] - 1) k = nc[a] - 1;
      if (k < 0) k = 0;
      c[a] = k;
    }
    cell_of[i] = c[0] + nc[0] * (c[1] + nc[1] * c[2]);
  }
  /* counting sort on the key (cell, class), stable in the bead index */
  int64_t nkey = ncell * ncls;
  int64_t *cnt = (int64_t *)calloc((size_t)nkey + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) cnt[(int64_t)cell_of[i] * ncls + cls[i] + 1]++;
  for (int64_t k = 0; k < nkey; ++k) cnt[k + 1] += cnt[k];
  for (int64_t c = 0; c <= ncell; ++c) cell_start[c] = (int32_t)cnt[c * ncls];
  for (int64_t i = 0; i < n; ++i) {
    int64_t key = (int64_t)cell_of[i] * ncls + cls[i];
    sorted_idx[cnt[key]++] = (int32_t)i;
  }
  free(cnt);
}

/* ------------------------------------------------------------------------ */
/* Real-space pair terms: Gaussian core (Eq. u_ex) and the screened smeared  */
/* Coulomb term of Eq. ewald, summed over all images within the cutoff.      */
/* ------------------------------------------------------------------------ */

/* g(r) = [erf(b r) - erf(k r)]/r and h(r) = -g'(r)/r, so that the force on
 * bead i from j at separation vector d = r_j - r_i is -lB z_i z_j h(r) d.
 * For r -> 0 the Taylor series of erf is used (exact limit at r = 0). */
static void real_kernel(double b, double k, double r, double *g, double *h) {
  if (r < 1e-2) {
    double b2 = b * b, k2 = k * k;
    double b3 = b2 * b, k3 = k2 * k, b5 = b3 * b2, k5 = k3 * k2;
    double b7 = b5 * b2, k7 = k5 * k2;
    double r2 = r * r;
    *g = ORC_2_SQRTPI * ((b - k) - (b3 - k3) * r2 / 3.0 + (b5 - k5) * r2 * r2 / 10.0 -
                         (b7 - k7) * r2 * r2 * r2 / 42.0);
    *h = ORC_2_SQRTPI * (2.0 * (b3 - k3) / 3.0 - 2.0 * (b5 - k5) * r2 / 5.0 +
                         (b7 - k7) * r2 * r2 / 7.0);
    return;
  }
  double gg = (erf(b * r) - erf(k * r)) / r;
  double dd = ORC_2_SQRTPI * (b * exp(-b * b * r * r) - k * exp(-k * k * r * r));
  *g = gg;
  *h = (gg - dd) / (r * r);
}

/* Per-bead parameters come from a type table: A_tab[ti*nt+tj] = A_ij,
 * sig_tab[t] = sigma_t, a_tab[t] = a_t.  A type whose A row is zero has no
 * Gaussian core (image charges).
 *
 * Outputs (any may be NULL): e_out[2] = {E_gc, E_real}; f_out (n,3) forces;
 * vir_out[9] = sum over pairs of r_ij (x) F_ij (r_ij = r_i - r_j);
 * npairs_out = number of unordered in-cutoff triples; eb_out (n,2) per-bead
 * energies (half of each pair energy is given to each bead).
 *
 * Inclusion of a triple follows in_cutoff_f32; the physics is FP64 on the
 * wrapped positions.  Each bead i sums over all j and all images (both
 * orders of every pair are visited), energies are halved. */
void orc_pairs(int64_t n, const double *pos, const double *q, const int32_t *type,
               int32_t nt, const double *A_tab, const double *sig_tab,
               const double *a_tab, const double *box, double rc, double kappa,
               double lB, int32_t do_gc, int32_t do_real, double *e_out,
               double *f_out, double *vir_out, int64_t *npairs_out,
               double *eb_out) {
  double *w = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  float *f32 = (float *)malloc(sizeof(float) * 3 * (size_t)n);
  orc_wrap(n, pos, box, w);
  for (int64_t i = 0; i < 3 * n; ++i) f32[i] = (float)w[i];
  float Lf[3] = {(float)box[0], (float)box[1], (float)box[2]};
  float rc2 = (float)(rc * rc);
  int m[3];
  int minimg[3];
  for (int a = 0; a < 3; ++a) {
    m[a] = image_range(box[a], rc);
    /* With L >= 2 rc (plus a margin far above FP32 rounding) only the
     * nearest image can be inside the cutoff; the others are skipped. */
    minimg[a] = box[a] >= 2.0 * rc * (1.0 + 1e-4);
  }
  double egc = 0.0, ereal = 0.0;
  double vir[9] = {0};
  int64_t npairs2 = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : egc, ereal, npairs2) \
    reduction(+ : vir[:9])
  for (int64_t i = 0; i < n; ++i) {
    double fi[3] = {0, 0, 0};
    double ei_gc = 0.0, ei_re = 0.0;
    int ti = type[i];
    for (int64_t j = 0; j < n; ++j) {
      int tj = type[j];
      double Aij = A_tab[ti * nt + tj];
      double qq = q[i] * q[j];
      int want_gc = do_gc && Aij != 0.0;
      int want_re = do_real && qq != 0.0;
      if (!want_gc && !want_re) continue;
      int lo[3], hi[3];
      for (int a = 0; a < 3; ++a) {
        if (minimg[a]) {
          double d = w[3 * j + a] - w[3 * i + a];
          int nn = -(int)nearbyint(d / box[a]);
          lo[a] = hi[a] = nn;
        } else {
          lo[a] = -m[a];
          hi[a] = m[a];
        }
      }
      for (int nz = lo[2]; nz <= hi[2]; ++nz)
        for (int ny = lo[1]; ny <= hi[1]; ++ny)
          for (int nx = lo[0]; nx <= hi[0]; ++nx) {
            if (i == j && nx == 0 && ny == 0 && nz == 0) continue;
            float sh[3] = {(float)nx * Lf[0], (float)ny * Lf[1], (float)nz * Lf[2]};
            if (!in_cutoff_f32(f32 + 3 * i, f32 + 3 * j, sh, rc2)) continue;
            double d[3] = {w[3 * j + 0] + nx * box[0] - w[3 * i + 0],
                           w[3 * j + 1] + ny * box[1] - w[3 * i + 1],
                           w[3 * j + 2] + nz * box[2] - w[3 * i + 2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double r = sqrt(r2);
            double fs = 0.0; /* force on i = -fs * d */
            npairs2 += 1;
            if (want_gc) {
              double s = sig_tab[ti] * sig_tab[ti] + sig_tab[tj] * sig_tab[tj];
              double u = Aij * pow(3.0 / (2.0 * ORC_PI * s), 1.5) * exp(-1.5 * r2 / s);
              ei_gc += 0.5 * u;
              fs += 3.0 / s * u;
            }
            if (want_re) {
              double a2 = a_tab[ti] * a_tab[ti] + a_tab[tj] * a_tab[tj];
              double beta = sqrt(ORC_PI) / (sqrt(2.0) * sqrt(a2));
              double g, h;
              real_kernel(beta, kappa, r, &g, &h);
              ei_re += 0.5 * lB * qq * g;
              fs += lB * qq * h;
            }
            for (int a = 0; a < 3; ++a) fi[a] -= fs * d[a];
            /* r_ij (x) F_ij with r_ij = -d and F_ij = -fs d, halved because
             * both orders of the pair are visited */
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) vir[3 * a + b] += 0.5 * fs * d[a] * d[b];
          }
    }
    egc += ei_gc;
    ereal += ei_re;
    if (f_out)
      for (int a = 0; a < 3; ++a) f_out[3 * i + a] = fi[a];
    if (eb_out) {
      eb_out[2 * i + 0] = ei_gc;
      eb_out[2 * i + 1] = ei_re;
    }
  }
  if (e_out) {
    e_out[0] = egc;
    e_out[1] = ereal;
  }
  if (vir_out)
    for (int k = 0; k < 9; ++k) vir_out[k] = vir[k];
  if (npairs_out) *npairs_out = npairs2 / 2;
  free(w);
  free(f32);
}

/* ------------------------------------------------------------------------ */
/* Reciprocal-space term by direct k-sum (the standard point-charge Ewald    */
/* sum of Eq. ewald, tin-foil boundary, k = 0 excluded).                     */
/* ------------------------------------------------------------------------ */

/* E = (2 pi lB / V) sum_{k!=0} exp(-k^2/(4 kappa^2))/k^2 |S(k)|^2,
 * S(k) = sum_j z_j exp(i k.r_j), k = 2 pi (m1/L1, m2/L2, m3/L3).
 * The sum runs over |k| <= kmax with exp(-kmax^2/(4 kappa^2)) = tol.
 * Forces F_j = -dE/dr_j; virial W_ab = sum_k E_k [d_ab - 2 (1 + k^2/(4kappa^2)) k_a k_b / k^2]. */
void orc_ewald_recip(int64_t n, const double *pos, const double *q, const double *box,
                     double kappa, double lB, double tol, double *e_out, double *f_out,
                     double *vir_out) {
  double V = box[0] * box[1] * box[2];
  double kmax = 2.0 * kappa * sqrt(-log(tol));
  int mm[3];
  for (int a = 0; a < 3; ++a) mm[a] = (int)ceil(kmax * box[a] / (2.0 * ORC_PI));
  /* charged beads only */
  int64_t nq = 0;
  for (int64_t i = 0; i < n; ++i) nq += q[i] != 0.0;
  int64_t *qi = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nq > 0 ? nq : 1));
  nq = 0;
  for (int64_t i = 0; i < n; ++i)
    if (q[i] != 0.0) qi[nq++] = i;
  /* per-axis phase tables exp(i 2 pi m x / L), m in [-mm, mm] */
  double *cs[3], *sn[3];
  for (int a = 0; a < 3; ++a) {
    int W = 2 * mm[a] + 1;
    cs[a] = (double *)malloc(sizeof(double) * (size_t)W * (size_t)(nq > 0 ? nq : 1));
    sn[a] = (double *)malloc(sizeof(double) * (size_t)W * (size_t)(nq > 0 ? nq : 1));
    for (int64_t s = 0; s < nq; ++s) {
      double x = pos[3 * qi[s] + a];
      for (int mi = -mm[a]; mi <= mm[a]; ++mi) {
        double ph = 2.0 * ORC_PI * mi * x / box[a];
        cs[a][(size_t)s * W + (mi + mm[a])] = cos(ph);
        sn[a][(size_t)s * W + (mi + mm[a])] = sin(ph);
      }
    }
  }
  int W0 = 2 * mm[0] + 1, W1 = 2 * mm[1] + 1, W2 = 2 * mm[2] + 1;
  double etot = 0.0;
  double vir[9] = {0};
  int nthr = orc_num_threads();
  double *fth = NULL;
  if (f_out) fth = (double *)calloc((size_t)nthr * 3 * (size_t)(nq > 0 ? nq : 1), sizeof(double));
  int64_t nk = (int64_t)W0 * W1 * W2;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : etot) reduction(+ : vir[:9])
  for (int64_t kk = 0; kk < nk; ++kk) {
    int m0 = (int)(kk % W0) - mm[0];
    int m1 = (int)((kk / W0) % W1) - mm[1];
    int m2 = (int)(kk / ((int64_t)W0 * W1)) - mm[2];
    if (m0 == 0 && m1 == 0 && m2 == 0) continue;
    double k[3] = {2.0 * ORC_PI * m0 / box[0], 2.0 * ORC_PI * m1 / box[1],
                   2.0 * ORC_PI * m2 / box[2]};
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    if (k2 > kmax * kmax) continue;
    double coef = 2.0 * ORC_PI * lB / V * exp(-k2 / (4.0 * kappa * kappa)) / k2;
    double Sr = 0.0, Si = 0.0;
    for (int64_t s = 0; s < nq; ++s) {
      double c0 = cs[0][(size_t)s * W0 + m0 + mm[0]], s0 = sn[0][(size_t)s * W0 + m0 + mm[0]];
      double c1 = cs[1][(size_t)s * W1 + m1 + mm[1]], s1 = sn[1][(size_t)s * W1 + m1 + mm[1]];
      double c2 = cs[2][(size_t)s * W2 + m2 + mm[2]], s2 = sn[2][(size_t)s * W2 + m2 + mm[2]];
      double ar = c0 * c1 - s0 * s1, ai = c0 * s1 + s0 * c1;
      double br = ar * c2 - ai * s2, bi = ar * s2 + ai * c2;
      Sr += q[qi[s]] * br;
      Si += q[qi[s]] * bi;
    }
    double S2 = Sr * Sr + Si * Si;
    double Ek = coef * S2;
    etot += Ek;
    double fac = 2.0 * (1.0 + k2 / (4.0 * kappa * kappa)) / k2;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) vir[3 * a + b] += Ek * ((a == b) - fac * k[a] * k[b]);
    if (fth) {
#ifdef _OPENMP
      int tid = omp_get_thread_num();
#else
      int tid = 0;
#endif
      double *ft = fth + (size_t)tid * 3 * (size_t)nq;
      for (int64_t s = 0; s < nq; ++s) {
        double c0 = cs[0][(size_t)s * W0 + m0 + mm[0]], s0 = sn[0][(size_t)s * W0 + m0 + mm[0]];
        double c1 = cs[1][(size_t)s * W1 + m1 + mm[1]], s1 = sn[1][(size_t)s * W1 + m1 + mm[1]];
        double c2 = cs[2][(size_t)s * W2 + m2 + mm[2]], s2 = sn[2][(size_t)s * W2 + m2 + mm[2]];
        double ar = c0 * c1 - s0 * s1, ai = c0 * s1 + s0 * c1;
        double br = ar * c2 - ai * s2, bi = ar * s2 + ai * c2;
        /* dE/dr_j = coef * 2 Re[conj(S) i k z_j e^{ik.r_j}]
         *         = -2 coef z_j k Im[conj(S) e^{ik.r_j}] */
        double im = Sr * bi - Si * br;
        double g = 2.0 * coef * q[qi[s]] * im;
        for (int a = 0; a < 3; ++a) ft[3 * s + a] += g * k[a];
      }
    }
  }
  if (e_out) *e_out = etot;
  if (vir_out)
    for (int k = 0; k < 9; ++k) vir_out[k] = vir[k];
  if (f_out) {
    memset(f_out, 0, sizeof(double) * 3 * (size_t)n);
    for (int t = 0; t < nthr; ++t)
      for (int64_t s = 0; s < nq; ++s)
        for (int a = 0; a < 3; ++a) f_out[3 * qi[s] + a] += fth[(size_t)t * 3 * nq + 3 * s + a];
    free(fth);
  }
  for (int a = 0; a < 3; ++a) {
    free(cs[a]);
    free(sn[a]);
  }
  free(qi);
}

/* ------------------------------------------------------------------------ */
/* Smooth particle-mesh Ewald (Essmann et al. 1995) in FP64, with the 3D     */
/* discrete Fourier transform done as three separable direct 1D DFTs.        */
/* ------------------------------------------------------------------------ */

/* Cardinal B-spline M_p(u) by the recursion
 *   M_2(u) = 1 - |u - 1| on [0, 2],
 *   M_p(u) = [u M_{p-1}(u) + (p - u) M_{p-1}(u - 1)] / (p - 1). */
double orc_bspline(int p, double u) {
  if (u <= 0.0 || u >= p) return 0.0;
  if (p == 2) return 1.0 - fabs(u - 1.0);
  return (u * orc_bspline(p - 1, u) + (p - u) * orc_bspline(p - 1, u - 1.0)) / (p - 1);
}

/* dM_p/du = M_{p-1}(u) - M_{p-1}(u - 1). */
static double bspline_deriv(int p, double u) {
  return orc_bspline(p - 1, u) - orc_bspline(p - 1, u - 1.0);
}

/* |b(m)|^2 = 1 / |sum_{k=0}^{p-2} M_p(k+1) exp(2 pi i m k / K)|^2.  For odd p
 * the sum vanishes at m = K/2; that entry takes the mean of its neighbours. */
void orc_bspline_moduli(int p, int K, double *bsq) {
  for (int m = 0; m < K; ++m) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k <= p - 2; ++k) {
      double ph = 2.0 * ORC_PI * m * k / K;
      double Mk = orc_bspline(p, k + 1.0);
      re += Mk * cos(ph);
      im += Mk * sin(ph);
    }
    double den = re * re + im * im;
    bsq[m] = den > 1e-10 ? 1.0 / den : -1.0;
  }
  for (int m = 0; m < K; ++m)
    if (bsq[m] < 0.0) {
      double a = bsq[(m + K - 1) % K], b = bsq[(m + 1) % K];
      bsq[m] = 0.5 * (a + b);
    }
}

/* One direct DFT along axis `ax` of a complex grid (re, im) with sign sgn:
 * out(m) = sum_k in(k) exp(sgn 2 pi i m k / K). */
static void dft_axis(int K0, int K1, int K2, int ax, int sgn, double *re, double *im) {
  int Ks[3] = {K0, K1, K2};
  int K = Ks[ax];
  double *ct = (double *)malloc(sizeof(double) * (size_t)K * K);
  double *st = (double *)malloc(sizeof(double) * (size_t)K * K);
  for (int m = 0; m < K; ++m)
    for (int k = 0; k < K; ++k) {
      double ph = 2.0 * ORC_PI * (double)((int64_t)m * k % K) / K;
      ct[m * K + k] = cos(ph);
      st[m * K + k] = sgn * sin(ph);
    }
  int64_t stride = ax == 0 ? 1 : (ax == 1 ? K0 : (int64_t)K0 * K1);
  int64_t nlines = (int64_t)K0 * K1 * K2 / K;
#pragma omp parallel for schedule(static)
  for (int64_t l = 0; l < nlines; ++l) {
    /* base index of line l */
    int64_t base;
    if (ax == 0) base = l * K0;
    else if (ax == 1) base = (l % K0) + (l / K0) * (int64_t)K0 * K1;
    else base = l;
    double tr[1024], ti[1024];
    for (int m = 0; m < K; ++m) {
      double sr = 0.0, si = 0.0;
      for (int k = 0; k < K; ++k) {
        double xr = re[base + k * stride], xi = im[base + k * stride];
        double c = ct[m * K + k], s = st[m * K + k];
        sr += xr * c - xi * s;
        si += xr * s + xi * c;
      }
      tr[m] = sr;
      ti[m] = si;
    }
    for (int m = 0; m < K; ++m) {
      re[base + m * stride] = tr[m];
      im[base + m * stride] = ti[m];
    }
  }
  free(ct);
  free(st);
}

/* Smooth PME reciprocal energy, forces and virial (orthorhombic box).
 *   u_a = K_a x_a / L_a,
 *   Q(k) = sum_i z_i prod_a M_p(u_ia - k_a)   (periodically wrapped),
 *   E = 1/2 sum_m B(m) C(m) |F(Q)(m)|^2,
 *   B = prod_a |b_a(m_a)|^2, C = lB/(pi V) exp(-pi^2 m^2/kappa^2)/m^2, C(0)=0,
 *   F_i = -sum_k dQ(k)/dr_i (theta * Q)(k),  theta * Q = F^{-1}[B C F(Q)]
 * (unnormalised forward and backward transforms).  Grid sizes K_a <= 1024. */
void orc_spme(int64_t n, const double *pos, const double *q, const double *box,
              const int32_t *Kg, int32_t p, double kappa, double lB, double *e_out,
              double *f_out, double *vir_out) {
  int K0 = Kg[0], K1 = Kg[1], K2 = Kg[2];
  int64_t G = (int64_t)K0 * K1 * K2;
  double V = box[0] * box[1] * box[2];
  double *re = (double *)calloc((size_t)G, sizeof(double));
  double *im = (double *)calloc((size_t)G, sizeof(double));
  double *w = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  orc_wrap(n, pos, box, w);
  /* spread */
  for (int64_t i = 0; i < n; ++i) {
    if (q[i] == 0.0) continue;
    int base[3];
    double wt[3][16];
    for (int a = 0; a < 3; ++a) {
      double u = Kg[a] * w[3 * i + a] / box[a];
      int fl = (int)floor(u);
      base[a] = fl;
      for (int t = 0; t < p; ++t) wt[a][t] = orc_bspline(p, u - (fl - t));
    }
    for (int tz = 0; tz < p; ++tz)
      for (int ty = 0; ty < p; ++ty)
        for (int tx = 0; tx < p; ++tx) {
          int kx = ((base[0] - tx) % K0 + K0) % K0;
          int ky = ((base[1] - ty) % K1 + K1) % K1;
          int kz = ((base[2] - tz) % K2 + K2) % K2;
          re[kx + (int64_t)K0 * (ky + (int64_t)K1 * kz)] +=
              q[i] * wt[0][tx] * wt[1][ty] * wt[2][tz];
        }
  }
  /* forward transform */
  dft_axis(K0, K1, K2, 0, +1, re, im);
  dft_axis(K0, K1, K2, 1, +1, re, im);
  dft_axis(K0, K1, K2, 2, +1, re, im);
  double *b0 = (double *)malloc(sizeof(double) * K0);
  double *b1 = (double *)malloc(sizeof(double) * K1);
  double *b2 = (double *)malloc(sizeof(double) * K2);
  orc_bspline_moduli(p, K0, b0);
  orc_bspline_moduli(p, K1, b1);
  orc_bspline_moduli(p, K2, b2);
  double E = 0.0;
  double vir[9] = {0};
  for (int64_t kk = 0; kk < G; ++kk) {
    int i0 = (int)(kk % K0), i1 = (int)((kk / K0) % K1), i2 = (int)(kk / ((int64_t)K0 * K1));
    int mi[3] = {i0 < (K0 + 1) / 2 ? i0 : i0 - K0, i1 < (K1 + 1) / 2 ? i1 : i1 - K1,
                 i2 < (K2 + 1) / 2 ? i2 : i2 - K2};
    if (mi[0] == 0 && mi[1] == 0 && mi[2] == 0) {
      re[kk] = im[kk] = 0.0;
      continue;
    }
    double mv[3] = {mi[0] / box[0], mi[1] / box[1], mi[2] / box[2]};
    double m2 = mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2];
    double B = b0[i0] * b1[i1] * b2[i2];
    double C = lB / (ORC_PI * V) * exp(-ORC_PI * ORC_PI * m2 / (kappa * kappa)) / m2;
    double S2 = re[kk] * re[kk] + im[kk] * im[kk];
    double Em = 0.5 * B * C * S2;
    E += Em;
    double fac = 2.0 * (1.0 + ORC_PI * ORC_PI * m2 / (kappa * kappa)) / m2;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) vir[3 * a + b] += Em * ((a == b) - fac * mv[a] * mv[b]);
    re[kk] *= B * C;
    im[kk] *= B * C;
  }
  if (e_out) *e_out = E;
  if (vir_out)
    for (int k = 0; k < 9; ++k) vir_out[k] = vir[k];
  if (f_out) {
    /* backward transform gives (theta * Q)(k) in re */
    dft_axis(K0, K1, K2, 0, -1, re, im);
    dft_axis(K0, K1, K2, 1, -1, re, im);
    dft_axis(K0, K1, K2, 2, -1, re, im);
    for (int64_t i = 0; i < n; ++i) {
      f_out[3 * i + 0] = f_out[3 * i + 1] = f_out[3 * i + 2] = 0.0;
      if (q[i] == 0.0) continue;
      int base[3];
      double wt[3][16], dw[3][16];
      for (int a = 0; a < 3; ++a) {
        double u = Kg[a] * w[3 * i + a] / box[a];
        int fl = (int)floor(u);
        base[a] = fl;
        for (int t = 0; t < p; ++t) {
          wt[a][t] = orc_bspline(p, u - (fl - t));
          dw[a][t] = bspline_deriv(p, u - (fl - t)) * Kg[a] / box[a];
        }
      }
      double g[3] = {0, 0, 0};
      for (int tz = 0; tz < p; ++tz)
        for (int ty = 0; ty < p; ++ty)
          for (int tx = 0; tx < p; ++tx) {
            int kx = ((base[0] - tx) % K0 + K0) % K0;
            int ky = ((base[1] - ty) % K1 + K1) % K1;
            int kz = ((base[2] - tz) % K2 + K2) % K2;
            double c = re[kx + (int64_t)K0 * (ky + (int64_t)K1 * kz)];
            g[0] += dw[0][tx] * wt[1][ty] * wt[2][tz] * c;
            g[1] += wt[0][tx] * dw[1][ty] * wt[2][tz] * c;
            g[2] += wt[0][tx] * wt[1][ty] * dw[2][tz] * c;
          }
      for (int a = 0; a < 3; ++a) f_out[3 * i + a] = -q[i] * g[a];
    }
  }
  free(b0);
  free(b1);
  free(b2);
  free(re);
  free(im);
  free(w);
}

/* ------------------------------------------------------------------------ */
/* Constant terms of Eq. ewald.                                               */
/* ------------------------------------------------------------------------ */

/* corr = -lB kappa/sqrt(pi) sum z_i^2 ;  self = lB sum z_i^2/(2 a_i). */
void orc_ewald_constants(int64_t n, const double *q, const double *a_bead, double kappa,
                         double lB, double *corr, double *self) {
  double s2 = 0.0, sb = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    s2 += q[i] * q[i];
    if (q[i] != 0.0) sb += q[i] * q[i] / (2.0 * a_bead[i]);
  }
  *corr = -lB * kappa / sqrt(ORC_PI) * s2;
  *self = lB * sb;
}

/* ------------------------------------------------------------------------ */
/* Slab terms.                                                                */
/* ------------------------------------------------------------------------ */

/* Yeh-Berkowitz correction for a slab in a box with vacuum along z:
 * M_z = sum z_i z_pos,i,  E = 2 pi lB M_z^2 / V,  F_z,i = -4 pi lB z_i M_z / V. */
void orc_slab_yb(int64_t n, const double *pos, const double *q, const double *box,
                 double lB, double *e_out, double *fz_out) {
  double V = box[0] * box[1] * box[2];
  double M = 0.0;
  for (int64_t i = 0; i < n; ++i) M += q[i] * pos[3 * i + 2];
  *e_out = 2.0 * ORC_PI * lB * M * M / V;
  if (fz_out)
    for (int64_t i = 0; i < n; ++i) fz_out[i] = -4.0 * ORC_PI * lB * q[i] * M / V;
}

/* Continuum electrode walls at z = 0 and z = H: the Gaussian-core potential
 * integrated over a plane of areal density n_s,
 *   u_w(h) = (A n_s) (3/(2 pi s_w))^{1/2} exp(-3 h^2/(2 s_w)),
 * with h the distance to each wall (wallA = A n_s, s_w = wall_sigma2). */
void orc_walls(int64_t n, const double *pos, double H, double wallA, double s_w,
               double *e_out, double *fz_out) {
  double c = wallA * sqrt(3.0 / (2.0 * ORC_PI * s_w));
  double E = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double z0 = pos[3 * i + 2];
    double z1 = H - z0;
    double u0 = c * exp(-1.5 * z0 * z0 / s_w);
    double u1 = c * exp(-1.5 * z1 * z1 / s_w);
    E += u0 + u1;
    /* du/dz for each wall; h1 = H - z so dh1/dz = -1 */
    double dz = -3.0 * z0 / s_w * u0 + 3.0 * z1 / s_w * u1;
    if (fz_out) fz_out[i] = -dz;
  }
  *e_out = E;
}

/* ------------------------------------------------------------------------ */
/* Harmonic bonds, u = k/2 (r - r0)^2 with r the minimum-image distance.     */
/* ------------------------------------------------------------------------ */
void orc_bonds(int64_t nb, const int32_t *pairs, int64_t n, const double *pos,
               const double *box, const int32_t *periodic, double k, double r0,
               double *e_out, double *f_out, double *vir_out) {
  double E = 0.0;
  double vir[9] = {0};
  if (f_out) memset(f_out, 0, sizeof(double) * 3 * (size_t)n);
  for (int64_t b = 0; b < nb; ++b) {
    int i = pairs[2 * b], j = pairs[2 * b + 1];
    double d[3];
    for (int a = 0; a < 3; ++a) {
      d[a] = pos[3 * j + a] - pos[3 * i + a];
      if (periodic[a]) d[a] -= box[a] * nearbyint(d[a] / box[a]);
    }
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    E += 0.5 * k * (r - r0) * (r - r0);
    double fs = k * (r - r0) / r; /* force on i = +fs d */
    if (f_out)
      for (int a = 0; a < 3; ++a) {
        f_out[3 * i + a] += fs * d[a];
        f_out[3 * j + a] -= fs * d[a];
      }
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) vir[3 * a + c] += -d[a] * fs * d[c];
  }
  *e_out = E;
  if (vir_out)
    for (int a = 0; a < 9; ++a) vir_out[a] = vir[a];
}
