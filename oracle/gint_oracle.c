/*
 * gint_oracle.c -- plain FP64 CPU oracle for uniform-grid integration with
 * numerical atomic orbitals (NAOs) at the Gamma point.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the product path never calls
 * it.
 *
 * What it computes (paper Sec. 3.3.1, "Uniform Grid Integration"):
 *   orbital        phi_mu(r) = f_{I l zeta}(|r|) Y_lm(r/|r|)                 (Eq. 1)
 *   periodised     Phi_mu(r) = sum_R phi_mu(r - tau_I - R)   (Gamma point, Eq. 2 at k=0)
 *   density        rho(r_g)  = sum_{mu,nu} D_{mu nu} Phi_mu(r_g) Phi_nu(r_g)
 *                  (the density formula of Sec. 3.3.1 with rho_{mu nu}(R) summed over R)
 *   local H        H_{mu nu} = sum_g w V(r_g) Phi_mu(r_g) Phi_nu(r_g)
 *                  (the local-potential matrix element formula of Sec. 3.3.1, w = Delta V)
 *   local H(R)     H_{mu nu}(R) = sum over grid points of all space of w V phi_mu(r - tau_I)
 *                  phi_nu(r - tau_J - R) (the same formula with the lattice vector R kept apart,
 *                  Sec. 2 H(R) and its Bloch sum H(k) = sum_R e^{ik.R} H(R)); by the periodicity of
 *                  V: sum over cell points g and image pairs (I at tau_I + n_I A, J at tau_J + n_J A)
 *                  with n_J - n_I = R
 *   projector      P_{j mu}^{IJ}(A) = int beta_{I j}(r - tau_I) e^{-i A.r} Phi_{J mu}(r) dr, the
 *   overlaps       velocity-gauge nonlocal matrix element of Sec. 3.3.2 ("Spherical Grid Integration
 *                  for Nonlocal Potentials"), on an atom-centred grid around tau_I (radial nodes on
 *                  [0, rc_beta] times r^2, angular points with weights summing to 4 pi); beta_{I j} =
 *                  f(|x|) Y_lm from a projector radial table (cubic Hermite, like the orbitals), Phi the
 *                  periodised orbital (Gamma point)
 *   local Pulay    F_I = - dE/dtau_I, E = sum_g w V(r_g) rho(r_g) at fixed V, which is the
 *   force          local Pulay force formula of Sec. 3.3.1:
 *                  F_I = sum_g w V_g sum_{mu in I} grad Phi_mu(r_g) sum_nu (D_mu nu + D_nu mu) Phi_nu(r_g)
 *                  (d phi(r - tau)/d tau = - grad phi).
 *
 * Readings where the paper is silent (each is stated again in the design notes):
 *   - radial f(r) is the cubic Hermite interpolant of the tabulated (f_k, f'_k) at r_k = k dr;
 *     its derivative is the derivative of that interpolant; f = 0 for r >= rc or beyond the table;
 *   - Y_lm are orthonormal real spherical harmonics without the Condon-Shortley sign, l <= 2,
 *     m ordered 0, +1, -1, +2, -2;
 *   - at |d| < 1e-12 (grid point on an atom) phi_{l=0} = f(0) Y_00, phi_{l>0} = 0,
 *     grad phi_{l=1,m} = f'(0) sqrt(3/4pi) e_m (e = z, x, y for m = 0, +1, -1), other gradients 0;
 *   - grid point (i,j,k) is at (i/n1) a1 + (j/n2) a2 + (k/n3) a3, w = |det A| / (n1 n2 n3);
 *   - the table stores R including the r^l factor.
 *
 * An "analytic" mode replaces the table by f(r) = r^l exp(-alpha r^2) with support r < rc;
 * it exists so that grid sums can be checked against closed-form Gaussian overlaps.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC gint_oracle.c -o libgint_oracle.so -lm
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double cell[9];          /* rows a1, a2, a3 */
  int natoms;
  const double *pos;       /* [natoms][3] Cartesian */
  const int *species;      /* [natoms] */
  int nspecies;
  const int *sp_rad_begin; /* [nspecies+1]: radials of species s are [begin[s], begin[s+1]) */
  int nrad;
  const int *rad_l;        /* [nrad] */
  const int *rad_npts;     /* [nrad] */
  const double *rad_dr;    /* [nrad] */
  const double *rad_rc;    /* [nrad] */
  const long long *rad_off;/* [nrad] offset of the radial's samples in f/df */
  const double *f;         /* tabulated R(r_k) */
  const double *df;        /* tabulated R'(r_k) */
  const double *rad_alpha; /* [nrad], analytic mode only */
  int analytic;
  int n1, n2, n3;
} orc_sys;

#define PI 3.14159265358979323846

/* ---------------------------------------------------------------- geometry */

static void inverse3(const double a[9], double inv[9], double *det_out) {
  double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
               a[2] * (a[3] * a[7] - a[4] * a[6]);
  inv[0] = (a[4] * a[8] - a[5] * a[7]) / det;
  inv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  inv[3] = (a[5] * a[6] - a[3] * a[8]) / det;
  inv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  inv[6] = (a[3] * a[7] - a[4] * a[6]) / det;
  inv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
  *det_out = det;
}

double orc_weight(const orc_sys *s) {
  double inv[9], det;
  inverse3(s->cell, inv, &det);
  return fabs(det) / ((double)s->n1 * s->n2 * s->n3);
}

static void grid_point(const orc_sys *s, long long g, double r[3]) {
  long long k = g % s->n3;
  long long j = (g / s->n3) % s->n2;
  long long i = g / ((long long)s->n2 * s->n3);
  double fi = (double)i / s->n1, fj = (double)j / s->n2, fk = (double)k / s->n3;
  for (int c = 0; c < 3; ++c) r[c] = fi * s->cell[c] + fj * s->cell[3 + c] + fk * s->cell[6 + c];
}

int orc_species_norb(const orc_sys *s, int sp) {
  int n = 0;
  for (int k = s->sp_rad_begin[sp]; k < s->sp_rad_begin[sp + 1]; ++k) n += 2 * s->rad_l[k] + 1;
  return n;
}

static double species_rcut(const orc_sys *s, int sp) {
  double rc = 0;
  for (int k = s->sp_rad_begin[sp]; k < s->sp_rad_begin[sp + 1]; ++k)
    if (s->rad_rc[k] > rc) rc = s->rad_rc[k];
  return rc;
}

int orc_norb(const orc_sys *s) {
  int n = 0;
  for (int a = 0; a < s->natoms; ++a) n += orc_species_norb(s, s->species[a]);
  return n;
}

/* ---------------------------------------------------------------- radial */

/* Cubic Hermite interpolant of (f_k, f'_k) on knots k*dr and its derivative. */
static void radial_value(const orc_sys *s, int k, double r, double *f, double *df) {
  if (r >= s->rad_rc[k]) { *f = 0.0; *df = 0.0; return; }
  if (s->analytic) {
    int l = s->rad_l[k];
    double a = s->rad_alpha[k];
    double e = exp(-a * r * r);
    double rl = pow(r, l);
    *f = rl * e;
    *df = ((l > 0 ? l * pow(r, l - 1) : 0.0) - 2.0 * a * r * rl) * e;
    return;
  }
  double dr = s->rad_dr[k];
  double x = r / dr;
  long long i = (long long)floor(x);
  if (i >= s->rad_npts[k] - 1) { *f = 0.0; *df = 0.0; return; }
  double t = x - (double)i;
  const double *F = s->f + s->rad_off[k];
  const double *G = s->df + s->rad_off[k];
  double f0 = F[i], f1 = F[i + 1], g0 = G[i] * dr, g1 = G[i + 1] * dr;
  double t2 = t * t, t3 = t2 * t;
  double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t, h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
  double d00 = 6 * t2 - 6 * t, d10 = 3 * t2 - 4 * t + 1, d01 = -6 * t2 + 6 * t, d11 = 3 * t2 - 2 * t;
  *f = h00 * f0 + h10 * g0 + h01 * f1 + h11 * g1;
  *df = (d00 * f0 + d10 * g0 + d01 * f1 + d11 * g1) / dr;
}

/* ---------------------------------------------------------------- angular */

/* Real solid harmonics y_lm(x,y,z) = r^l Y_lm and their Cartesian gradients, m order 0,+1,-1,+2,-2. */
static void solid_harmonics(int l, const double d[3], double y[5], double gy[5][3]) {
  double x = d[0], yy = d[1], z = d[2];
  memset(gy, 0, sizeof(double) * 15);
  if (l == 0) {
    y[0] = 0.5 / sqrt(PI);
  } else if (l == 1) {
    double c = sqrt(3.0 / (4.0 * PI));
    y[0] = c * z;  gy[0][2] = c;
    y[1] = c * x;  gy[1][0] = c;
    y[2] = c * yy; gy[2][1] = c;
  } else { /* l == 2 */
    double c0 = sqrt(5.0 / (16.0 * PI)), c1 = sqrt(15.0 / (4.0 * PI)), c2 = sqrt(15.0 / (16.0 * PI));
    y[0] = c0 * (2 * z * z - x * x - yy * yy);
    gy[0][0] = -2 * c0 * x; gy[0][1] = -2 * c0 * yy; gy[0][2] = 4 * c0 * z;
    y[1] = c1 * x * z;  gy[1][0] = c1 * z;  gy[1][2] = c1 * x;
    y[2] = c1 * yy * z; gy[2][1] = c1 * z;  gy[2][2] = c1 * yy;
    y[3] = c2 * (x * x - yy * yy); gy[3][0] = 2 * c2 * x; gy[3][1] = -2 * c2 * yy;
    y[4] = c1 * x * yy; gy[4][0] = c1 * yy; gy[4][1] = c1 * x;
  }
}

/* phi and grad phi of all orbitals of one species at displacement d = r - tau (one image).
 * Accumulates (+=) into phi[norb] and grad[norb][3]. */
static void add_species_orbitals(const orc_sys *s, int sp, const double d[3], double *phi, double *grad) {
  double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  int col = 0;
  for (int k = s->sp_rad_begin[sp]; k < s->sp_rad_begin[sp + 1]; ++k) {
    int l = s->rad_l[k];
    int nm = 2 * l + 1;
    if (r >= s->rad_rc[k]) { col += nm; continue; }
    double f, df;
    radial_value(s, k, r, &f, &df);
    if (r < 1e-12) {
      if (l == 0) phi[col] += f * 0.5 / sqrt(PI);
      if (l == 1) {
        double c = sqrt(3.0 / (4.0 * PI));
        grad[(col + 0) * 3 + 2] += df * c; /* m=0  -> z */
        grad[(col + 1) * 3 + 0] += df * c; /* m=+1 -> x */
        grad[(col + 2) * 3 + 1] += df * c; /* m=-1 -> y */
      }
      col += nm;
      continue;
    }
    double y[5], gy[5][3];
    solid_harmonics(l, d, y, gy);
    double rl = pow(r, l);
    for (int m = 0; m < nm; ++m) {
      double Y = y[m] / rl;              /* Y_lm(d/r) */
      phi[col + m] += f * Y;
      /* grad phi = f' Y d/r + f ( grad y / r^l - l Y d / r^2 ) */
      for (int c = 0; c < 3; ++c)
        grad[(col + m) * 3 + c] += df * Y * d[c] / r + f * (gy[m][c] / rl - l * Y * d[c] / (r * r));
    }
    col += nm;
  }
}

/* Periodised orbitals of atom a at point r: sums every lattice image within the support.
 * Returns 1 if any image lies inside the support (the atom "covers" r), else 0. */
static int atom_orbitals(const orc_sys *s, const double inv[9], int a, const double r[3], double *phi, double *grad) {
  int sp = s->species[a];
  int no = orc_species_norb(s, sp);
  double rc = species_rcut(s, sp);
  memset(phi, 0, sizeof(double) * no);
  if (grad) memset(grad, 0, sizeof(double) * no * 3);
  double tmpg[64 * 3];
  double *g = grad ? grad : tmpg;
  double d0[3];
  for (int c = 0; c < 3; ++c) d0[c] = r[c] - s->pos[3 * a + c];
  /* fractional coordinates of d0: d0 = u . A  =>  u = d0 . inv(A) */
  double u[3], reach[3];
  for (int c = 0; c < 3; ++c) {
    u[c] = d0[0] * inv[0 * 3 + c] + d0[1] * inv[1 * 3 + c] + d0[2] * inv[2 * 3 + c];
    reach[c] = rc * sqrt(inv[0 * 3 + c] * inv[0 * 3 + c] + inv[1 * 3 + c] * inv[1 * 3 + c] +
                         inv[2 * 3 + c] * inv[2 * 3 + c]);
  }
  int lo[3], hi[3];
  for (int c = 0; c < 3; ++c) {
    lo[c] = (int)ceil(u[c] - reach[c]);
    hi[c] = (int)floor(u[c] + reach[c]);
  }
  int covered = 0;
  for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
    for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
      for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = d0[c] - (n0 * s->cell[c] + n1 * s->cell[3 + c] + n2 * s->cell[6 + c]);
        double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (rr >= rc) continue;
        covered = 1;
        if (grad) add_species_orbitals(s, sp, d, phi, grad);
        else {
          memset(tmpg, 0, sizeof(double) * no * 3);
          add_species_orbitals(s, sp, d, phi, tmpg);
        }
      }
  return covered;
}

/* All periodised orbitals at r.  phi[norb], grad[norb*3] (grad may be NULL), cov[natoms]. */
static void all_orbitals(const orc_sys *s, const double inv[9], const int *aoff, const double r[3], double *phi,
                         double *grad, int *cov) {
  for (int a = 0; a < s->natoms; ++a)
    cov[a] = atom_orbitals(s, inv, a, r, phi + aoff[a], grad ? grad + 3 * aoff[a] : NULL);
}

static int *atom_offsets(const orc_sys *s) {
  int *aoff = (int *)malloc(sizeof(int) * (s->natoms + 1));
  aoff[0] = 0;
  for (int a = 0; a < s->natoms; ++a) aoff[a + 1] = aoff[a] + orc_species_norb(s, s->species[a]);
  return aoff;
}

/* ---------------------------------------------------------------- public entry points */

/* Phi and grad Phi at arbitrary Cartesian points.  phi [npts][norb], grad [npts][norb][3] (may be NULL). */
int orc_phi_points(const orc_sys *s, long long npts, const double *pts, double *phi, double *grad) {
  double inv[9], det;
  inverse3(s->cell, inv, &det);
  int *aoff = atom_offsets(s);
  int norb = aoff[s->natoms];
#pragma omp parallel
  {
    int *cov = (int *)malloc(sizeof(int) * s->natoms);
#pragma omp for schedule(dynamic, 16)
    for (long long p = 0; p < npts; ++p)
      all_orbitals(s, inv, aoff, pts + 3 * p, phi + p * norb, grad ? grad + p * norb * 3 : NULL, cov);
    free(cov);
  }
  free(aoff);
  return 0;
}

/* rho at the listed grid points (idx == NULL: every point, out indexed by grid index).
 * D is dense [norb][norb] row-major. */
int orc_rho(const orc_sys *s, const double *D, long long nidx, const long long *idx, double *rho) {
  double inv[9], det;
  inverse3(s->cell, inv, &det);
  int *aoff = atom_offsets(s);
  int norb = aoff[s->natoms];
  long long ng = idx ? nidx : (long long)s->n1 * s->n2 * s->n3;
#pragma omp parallel
  {
    double *phi = (double *)malloc(sizeof(double) * norb);
    int *cov = (int *)malloc(sizeof(int) * s->natoms);
    int *list = (int *)malloc(sizeof(int) * norb);
#pragma omp for schedule(dynamic, 64)
    for (long long q = 0; q < ng; ++q) {
      long long g = idx ? idx[q] : q;
      double r[3];
      grid_point(s, g, r);
      all_orbitals(s, inv, aoff, r, phi, NULL, cov);
      int n = 0;
      for (int a = 0; a < s->natoms; ++a)
        if (cov[a])
          for (int m = aoff[a]; m < aoff[a + 1]; ++m) list[n++] = m;
      double acc = 0.0;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) acc += D[(long long)list[i] * norb + list[j]] * phi[list[i]] * phi[list[j]];
      rho[q] = acc;
    }
    free(phi); free(cov); free(list);
  }
  free(aoff);
  return 0;
}

/* Dense H[norb][norb] = sum over the listed grid points (NULL: all) of w V_g Phi Phi^T.
 * Thread-private accumulators, summed at the end. */
int orc_vlocal(const orc_sys *s, const double *V, long long nidx, const long long *idx, double *H) {
  double inv[9], det;
  inverse3(s->cell, inv, &det);
  int *aoff = atom_offsets(s);
  int norb = aoff[s->natoms];
  double w = orc_weight(s);
  long long ng = idx ? nidx : (long long)s->n1 * s->n2 * s->n3;
  memset(H, 0, sizeof(double) * (size_t)norb * norb);
#pragma omp parallel
  {
    double *phi = (double *)malloc(sizeof(double) * norb);
    double *Hp = (double *)calloc((size_t)norb * norb, sizeof(double));
    int *cov = (int *)malloc(sizeof(int) * s->natoms);
    int *list = (int *)malloc(sizeof(int) * norb);
#pragma omp for schedule(dynamic, 64)
    for (long long q = 0; q < ng; ++q) {
      long long g = idx ? idx[q] : q;
      double r[3];
      grid_point(s, g, r);
      all_orbitals(s, inv, aoff, r, phi, NULL, cov);
      int n = 0;
      for (int a = 0; a < s->natoms; ++a)
        if (cov[a])
          for (int m = aoff[a]; m < aoff[a + 1]; ++m) list[n++] = m;
      double wv = w * V[g];
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Hp[(long long)list[i] * norb + list[j]] += wv * phi[list[i]] * phi[list[j]];
    }
#pragma omp critical
    for (long long e = 0; e < (long long)norb * norb; ++e) H[e] += Hp[e];
    free(phi); free(Hp); free(cov); free(list);
  }
  free(aoff);
  return 0;
}

/* One block H_IJ [norb(I)][norb(J)] = sum over all grid points of w V_g Phi_I Phi_J^T.
 * Only atoms I and J are evaluated, so large systems can be sampled block by block. */
int orc_vlocal_block(const orc_sys *s, const double *V, int I, int J, double *out) {
  double inv[9], det;
  inverse3(s->cell, inv, &det);
  int nI = orc_species_norb(s, s->species[I]), nJ = orc_species_norb(s, s->species[J]);
  double w = orc_weight(s);
  long long ng = (long long)s->n1 * s->n2 * s->n3;
  memset(out, 0, sizeof(double) * nI * nJ);
#pragma omp parallel
  {
    double pI[64], pJ[64];
    double *acc = (double *)calloc((size_t)nI * nJ, sizeof(double));
#pragma omp for schedule(static)
    for (long long g = 0; g < ng; ++g) {
      double r[3];
      grid_point(s, g, r);
      if (!atom_orbitals(s, inv, I, r, pI, NULL)) continue;
      if (!atom_orbitals(s, inv, J, r, pJ, NULL)) continue;
      double wv = w * V[g];
      for (int i = 0; i < nI; ++i)
        for (int j = 0; j < nJ; ++j) acc[i * nJ + j] += wv * pI[i] * pJ[j];
    }
#pragma omp critical
    for (int e = 0; e < nI * nJ; ++e) out[e] += acc[e];
    free(acc);
  }
  return 0;
}

/* The lattice images of atom a whose support covers r: n_out[k] (image at tau_a + n A) and the
 * image's orbitals phi_out[k][norb(a)], k < returned count (at most ORC_MAXIMG). */
#define ORC_MAXIMG 64
static int atom_images(const orc_sys *s, const double inv[9], int a, const double r[3], int n_out[][3],
                       double *phi_out) {
  int sp = s->species[a];
  int no = orc_species_norb(s, sp);
  double rc = species_rcut(s, sp);
  double d0[3], u[3], reach[3], tmpg[64 * 3];
  for (int c = 0; c < 3; ++c) d0[c] = r[c] - s->pos[3 * a + c];
  for (int c = 0; c < 3; ++c) {
    u[c] = d0[0] * inv[0 * 3 + c] + d0[1] * inv[1 * 3 + c] + d0[2] * inv[2 * 3 + c];
    reach[c] = rc * sqrt(inv[0 * 3 + c] * inv[0 * 3 + c] + inv[1 * 3 + c] * inv[1 * 3 + c] +
                         inv[2 * 3 + c] * inv[2 * 3 + c]);
  }
  int cnt = 0;
  for (int n0 = (int)ceil(u[0] - reach[0]); n0 <= (int)floor(u[0] + reach[0]); ++n0)
    for (int n1 = (int)ceil(u[1] - reach[1]); n1 <= (int)floor(u[1] + reach[1]); ++n1)
      for (int n2 = (int)ceil(u[2] - reach[2]); n2 <= (int)floor(u[2] + reach[2]); ++n2) {
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = d0[c] - (n0 * s->cell[c] + n1 * s->cell[3 + c] + n2 * s->cell[6 + c]);
        if (sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) >= rc || cnt == ORC_MAXIMG) continue;
        double *ph = phi_out + (size_t)cnt * no;
        memset(ph, 0, sizeof(double) * no);
        memset(tmpg, 0, sizeof(tmpg));
        add_species_orbitals(s, sp, d, ph, tmpg);
        n_out[cnt][0] = n0;
        n_out[cnt][1] = n1;
        n_out[cnt][2] = n2;
        ++cnt;
      }
  return cnt;
}

/* Blocks H_IJ(R) [nR][norb(I)][norb(J)] for the listed lattice vectors R (integer triplets in units
 * of a1, a2, a3): every cell grid point, every pair of images (I at tau_I + n_I A, J at
 * tau_J + n_J A) adds w V_g phi_I phi_J^T to R = n_J - n_I.  Products that belong to an R outside
 * the list are summed in absolute value into *missed (zero when the list is complete). */
int orc_vlocal_block_R(const orc_sys *s, const double *V, int I, int J, int nR, const int *R, double *out,
                       double *missed) {
  double inv[9], det;
  inverse3(s->cell, inv, &det);
  int nI = orc_species_norb(s, s->species[I]), nJ = orc_species_norb(s, s->species[J]);
  double w = orc_weight(s);
  long long ng = (long long)s->n1 * s->n2 * s->n3;
  size_t blk = (size_t)nI * nJ;
  memset(out, 0, sizeof(double) * blk * nR);
  double miss = 0.0;
#pragma omp parallel reduction(+ : miss)
  {
    double *pI = (double *)malloc(sizeof(double) * ORC_MAXIMG * 64);
    double *pJ = (double *)malloc(sizeof(double) * ORC_MAXIMG * 64);
    int (*nIm)[3] = malloc(sizeof(int[3]) * ORC_MAXIMG), (*nJm)[3] = malloc(sizeof(int[3]) * ORC_MAXIMG);
    double *acc = (double *)calloc(blk * nR, sizeof(double));
#pragma omp for schedule(static)
    for (long long g = 0; g < ng; ++g) {
      double r[3];
      grid_point(s, g, r);
      int ci = atom_images(s, inv, I, r, nIm, pI);
      if (!ci) continue;
      int cj = atom_images(s, inv, J, r, nJm, pJ);
      if (!cj) continue;
      double wv = w * V[g];
      for (int a = 0; a < ci; ++a)
        for (int b = 0; b < cj; ++b) {
          int d0 = nJm[b][0] - nIm[a][0], d1 = nJm[b][1] - nIm[a][1], d2 = nJm[b][2] - nIm[a][2];
          int k = 0;
          while (k < nR && !(R[3 * k] == d0 && R[3 * k + 1] == d1 && R[3 * k + 2] == d2)) ++k;
          const double *fa = pI + (size_t)a * nI, *fb = pJ + (size_t)b * nJ;
          if (k == nR) {
            for (int i = 0; i < nI; ++i)
              for (int j = 0; j < nJ; ++j) miss += fabs(wv * fa[i] * fb[j]);
            continue;
          }
          double *o = acc + (size_t)k * blk;
          for (int i = 0; i < nI; ++i)
            for (int j = 0; j < nJ; ++j) o[i * nJ + j] += wv * fa[i] * fb[j];
        }
    }
#pragma omp critical
    for (size_t e = 0; e < blk * nR; ++e) out[e] += acc[e];
    free(pI); free(pJ); free(nIm); free(nJm); free(acc);
  }
  *missed = miss;
  return 0;
}

/* Projector overlaps with the velocity-gauge phase: out [nbeta(I)][norb(J)][2] (re, im) =
 * sum_{k,a} W_ka beta_{I j}(x) e^{-i A.(tau_I + x)} Phi_{J mu}(tau_I + x), x = r_k e_a, r_k = rc t_k,
 * W_ka = rc rw_k r_k^2 w_a.  `p` describes the projectors as the "orbitals" of a system with the same
 * cell and atoms (its radial tables, l and rc); rt / rw are nodes and weights on [0, 1], ang [na][4]
 * holds the angular points (x, y, z) and weights. */
int orc_psibeta(const orc_sys *s, const orc_sys *p, const double A[3], int I, int J, int nr, const double *rt,
                const double *rw, int na, const double *ang, double *out) {
  double inv[9], det;
  inverse3(s->cell, inv, &det);
  int nb = orc_species_norb(p, p->species[I]), no = orc_species_norb(s, s->species[J]);
  double rcb = species_rcut(p, p->species[I]);
  memset(out, 0, sizeof(double) * 2 * nb * no);
  double *beta = (double *)malloc(sizeof(double) * nb), *gb = (double *)malloc(sizeof(double) * nb * 3);
  double *phi = (double *)malloc(sizeof(double) * no);
  for (int k = 0; k < nr; ++k) {
    double r = rcb * rt[k], wk = rcb * rw[k] * r * r;
    for (int a = 0; a < na; ++a) {
      double x[3] = {r * ang[4 * a], r * ang[4 * a + 1], r * ang[4 * a + 2]}, pt[3];
      for (int c = 0; c < 3; ++c) pt[c] = s->pos[3 * I + c] + x[c];
      memset(beta, 0, sizeof(double) * nb);
      memset(gb, 0, sizeof(double) * nb * 3);
      add_species_orbitals(p, p->species[I], x, beta, gb);
      if (!atom_orbitals(s, inv, J, pt, phi, NULL)) continue;
      double ph = -(A[0] * pt[0] + A[1] * pt[1] + A[2] * pt[2]);
      double w = wk * ang[4 * a + 3], cr = w * cos(ph), ci = w * sin(ph);
      for (int j = 0; j < nb; ++j)
        for (int m = 0; m < no; ++m) {
          out[2 * (j * no + m)] += cr * beta[j] * phi[m];
          out[2 * (j * no + m) + 1] += ci * beta[j] * phi[m];
        }
    }
  }
  free(beta); free(gb); free(phi);
  return 0;
}

/* Forces F[natoms][3] = -dE/dtau (E = sum_g w V_g rho_g, V fixed) summed over the listed grid
 * points (NULL: all).  atom_mask (may be NULL) restricts which atoms' forces are accumulated;
 * points not covered by any selected atom are skipped before the full evaluation. */
int orc_force(const orc_sys *s, const double *D, const double *V, long long nidx, const long long *idx,
              const int *atom_mask, double *F) {
  double inv[9], det;
  inverse3(s->cell, inv, &det);
  int *aoff = atom_offsets(s);
  int norb = aoff[s->natoms];
  double w = orc_weight(s);
  long long ng = idx ? nidx : (long long)s->n1 * s->n2 * s->n3;
  memset(F, 0, sizeof(double) * s->natoms * 3);
#pragma omp parallel
  {
    double *phi = (double *)malloc(sizeof(double) * norb);
    double *grad = (double *)malloc(sizeof(double) * norb * 3);
    double *Fp = (double *)calloc((size_t)s->natoms * 3, sizeof(double));
    int *cov = (int *)malloc(sizeof(int) * s->natoms);
    int *list = (int *)malloc(sizeof(int) * norb);
    double probe[64];
#pragma omp for schedule(dynamic, 64)
    for (long long q = 0; q < ng; ++q) {
      long long g = idx ? idx[q] : q;
      double r[3];
      grid_point(s, g, r);
      if (atom_mask) {
        int any = 0;
        for (int a = 0; a < s->natoms && !any; ++a)
          if (atom_mask[a] && atom_orbitals(s, inv, a, r, probe, NULL)) any = 1;
        if (!any) continue;
      }
      all_orbitals(s, inv, aoff, r, phi, grad, cov);
      int n = 0;
      for (int a = 0; a < s->natoms; ++a)
        if (cov[a])
          for (int m = aoff[a]; m < aoff[a + 1]; ++m) list[n++] = m;
      double wv = w * V[g];
      for (int a = 0; a < s->natoms; ++a) {
        if (!cov[a] || (atom_mask && !atom_mask[a])) continue;
        for (int mu = aoff[a]; mu < aoff[a + 1]; ++mu) {
          double y = 0.0; /* sum_nu (D_mu nu + D_nu mu) Phi_nu */
          for (int j = 0; j < n; ++j) {
            int nu = list[j];
            y += (D[(long long)mu * norb + nu] + D[(long long)nu * norb + mu]) * phi[nu];
          }
          for (int c = 0; c < 3; ++c) Fp[a * 3 + c] += wv * grad[mu * 3 + c] * y;
        }
      }
    }
#pragma omp critical
    for (int e = 0; e < s->natoms * 3; ++e) F[e] += Fp[e];
    free(phi); free(grad); free(Fp); free(cov); free(list);
  }
  free(aoff);
  return 0;
}

/* Work count W = sum_g n_g^2 over the listed points (NULL: all), where n_g is the number of
 * periodised orbitals whose support covers g.  Also returns sum_g n_g in *sum_n. */
int orc_count_pairs(const orc_sys *s, long long nidx, const long long *idx, double *W, double *sum_n) {
  double inv[9], det;
  inverse3(s->cell, inv, &det);
  long long ng = idx ? nidx : (long long)s->n1 * s->n2 * s->n3;
  double tw = 0.0, tn = 0.0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : tw, tn)
  for (long long q = 0; q < ng; ++q) {
    long long g = idx ? idx[q] : q;
    double r[3];
    grid_point(s, g, r);
    double probe[64];
    long long n = 0;
    for (int a = 0; a < s->natoms; ++a)
      if (atom_orbitals(s, inv, a, r, probe, NULL)) n += orc_species_norb(s, s->species[a]);
    tw += (double)n * (double)n;
    tn += (double)n;
  }
  *W = tw;
  *sum_n = tn;
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
