// gint_internal.cuh -- device-side data structures and orbital evaluation shared by the
// libgint kernels.
//
// Orbital evaluation follows Eq. 1 of the paper (phi = f_{I l zeta}(r) Y_lm(r^)), periodised
// over lattice images at the Gamma point (Eq. 2 with k = 0).  Radials are cubic Hermite
// interpolants of tabulated (f, f') samples; Y_lm are real, orthonormal, no Condon-Shortley
// sign, l <= 2, m ordered 0, +1, -1, +2, -2.  A grid point within 1e-12 Bohr of an atom
// takes the r -> 0 limit (s: f(0) Y00; p gradient: f'(0) sqrt(3/4pi) e_m; the rest 0).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gint.h"

#define GINT_MAX_SPECIES 8
#define GINT_MAX_RADIAL 64
#define GINT_MAX_ORB_ATOM 32      // orbitals of one atom
#define GINT_MAX_ATOMS_BRICK 64   // distinct atoms covering one brick (coverage masks are 64-bit)
#define GINT_BI 4                 // brick extent along grid axis 1
#define GINT_BJ 4                 // ... axis 2
#define GINT_BK 8                 // ... axis 3 (contiguous in memory)
#define GINT_BPTS (GINT_BI * GINT_BJ * GINT_BK)  // 128 points = one tcgen05 M tile

struct GRadial {
  int l, npts, off, pad;  // off: first knot of this radial in the packed tables
  double dr, inv_dr, rc, rc2;
  float idr_hi, idr_lo, rc_f, dr_f;  // float32 images: 1/dr as hi + lo, rc, dr
};

struct GSpecies {
  int nrad, rad0, norb, porb;  // porb: orbitals padded to a multiple of 8 (tensor-core layouts)
  int shape;                   // (ns, np, nd) code 1 + ns + 8 np + 64 nd when the radials are l-sorted and
                               // share one knot grid (same npts and dr); 0 otherwise
  float rcut2f;                // rcut2 rounded to float32 (coarse support test of the float32 kernels)
  int ioff, kslot;             // shaped species: interleaved float32 table [knot][kslot] of (f, f') at
                               // float2 offset ioff, kslot = radials rounded up to even; 0 otherwise
  double rcut, rcut2;          // largest rc of the species and its square
};
#define GINT_SHAPE(ns, np, nd) (1 + (ns) + 8 * (np) + 64 * (nd))

// Geometry of one system: cell, grid and bricks.
struct GCell {
  double cell[9];   // rows a1, a2, a3
  double inv[9];    // inverse: fractional u = d . inv
  double reach[3];  // |column c of inv| (fractional extent of a unit Cartesian length)
  double w;         // grid weight
  long long ngrid, nbricks;
  int n1, n2, n3;
  int nbi, nbj, nbk;  // bricks per axis
  int natoms, pad;
};

// Species and radial-table metadata (the knot values live in a separate packed array).
// Systems whose GTabs compare equal byte for byte can share one batched launch.
struct GTabs {
  int nspecies, nrad;
  GSpecies sp[GINT_MAX_SPECIES];
  GRadial rad[GINT_MAX_RADIAL];
};

struct GGeom : GCell, GTabs {};

// Neighbour structure of the bricks (device arrays, CSR).
//   bricks  : b_at_off[b] .. b_at_off[b+1]  distinct atoms of brick b ("slots")
//   slots   : s_atom[k], s_col[k] (first column of the atom in the brick's orbital space),
//             s_ent[k] .. s_ent[k+1]  its (atom, image) entries
//   entries : e_shift[e] = tau_I + R (Cartesian, float64, 3 per entry)
//   pairs   : b_pair_off[b] .. : n_a x n_a table of global pair indices (-1: no block)
struct GNbr {
  const long long *b_at_off;
  const int *b_norb;
  const int *s_atom;
  const int *s_col;
  const long long *s_ent;
  const double *e_shift;
  const long long *b_pair_off;
  const int *b_pair;
  const long long *pair_off;  // element offset of each pair block
  const int *atom_species;
};

#define GINT_PI 3.14159265358979323846

__host__ __device__ __forceinline__ void grid_point(const GCell &g, int i, int j, int k, double r[3]) {
  double fi = (double)i / g.n1, fj = (double)j / g.n2, fk = (double)k / g.n3;
#pragma unroll
  for (int c = 0; c < 3; ++c) r[c] = fi * g.cell[c] + fj * g.cell[3 + c] + fk * g.cell[6 + c];
}

// Decode a local point index 0..127 of a brick into grid indices; returns false outside the grid.
// (brick indices fit 32 bits: gint_create refuses grids of 2^31 bricks or more, so the divisions
// are 32-bit ones, several times cheaper on the GPU than 64-bit ones)
__host__ __device__ __forceinline__ bool brick_point(const GCell &g, long long b, int p, int &i, int &j, int &k) {
  const unsigned ub = (unsigned)b, nbk = (unsigned)g.nbk, q = ub / nbk;
  const int bk = (int)(ub - q * nbk);
  const int bj = (int)(q % (unsigned)g.nbj);
  const int bi = (int)(q / (unsigned)g.nbj);
  int pk = p % GINT_BK, pj = (p / GINT_BK) % GINT_BJ, pi = p / (GINT_BK * GINT_BJ);
  i = bi * GINT_BI + pi;
  j = bj * GINT_BJ + pj;
  k = bk * GINT_BK + pk;
  return i < g.n1 && j < g.n2 && k < g.n3;
}

__host__ __device__ __forceinline__ long long grid_index(const GCell &g, int i, int j, int k) {
  return ((long long)i * g.n2 + j) * g.n3 + k;
}

// ------------------------------------------------------------------------------------------
// Radial: cubic Hermite on uniform knots. tab[k] = (f_k, f'_k).
template <typename T>
struct Tab2;
template <>
struct Tab2<double> { typedef double2 type; };
template <>
struct Tab2<float> { typedef float2 type; };

// dtab (may be NULL): f_{k+1} - f_k per knot formed in float64 (for float32 tables; see the handle)
template <typename T>
__device__ __forceinline__ void radial_eval(const typename Tab2<T>::type *__restrict__ tab, const GRadial &R, T r,
                                            T &f, T &df, const float *__restrict__ dtab = nullptr) {
  T x = r * (T)R.inv_dr;
  int i = (int)x;
  if (i >= R.npts - 1) {
    f = 0;
    df = 0;
    return;
  }
  T t = x - (T)i;
  typename Tab2<T>::type a = tab[R.off + i], b = tab[R.off + i + 1];
  T dr = (T)R.dr;
  T g0 = a.y * dr, g1 = b.y * dr;
  T t2 = t * t;
  const T dlt = dtab ? (T)dtab[R.off + i] : b.x - a.x;
  // Hermite basis in nested form: h00 = 1 - t^2 (3 - 2t), h01 = t^2 (3 - 2t),
  // h10 = t (1 - t)^2, h11 = t^2 (t - 1)
  T s = t2 * ((T)3 - (T)2 * t);
  T u = (T)1 - t;
  f = a.x + dlt * s + g0 * t * u * u + g1 * t2 * (t - (T)1);
  // derivatives: dh01 = 6 t (1 - t) = -dh00, dh10 = (1 - t)(1 - 3t), dh11 = t (3t - 2)
  df = (dlt * (T)6 * t * u + g0 * u * ((T)1 - (T)3 * t) + g1 * t * ((T)3 * t - (T)2)) * (T)R.inv_dr;
}

// ------------------------------------------------------------------------------------------
// Real solid-harmonic polynomials evaluated on the unit vector (ux,uy,uz): y[m] and grad y[m].
template <typename T>
__device__ __forceinline__ void ylm_unit(int l, T ux, T uy, T uz, T *y, T (*gy)[3]) {
  if (l == 0) {
    y[0] = (T)(0.28209479177387814347);  // 1/(2 sqrt(pi))
    gy[0][0] = gy[0][1] = gy[0][2] = 0;
  } else if (l == 1) {
    const T c = (T)(0.48860251190291992159);  // sqrt(3/(4pi))
    y[0] = c * uz; gy[0][0] = 0; gy[0][1] = 0; gy[0][2] = c;
    y[1] = c * ux; gy[1][0] = c; gy[1][1] = 0; gy[1][2] = 0;
    y[2] = c * uy; gy[2][0] = 0; gy[2][1] = c; gy[2][2] = 0;
  } else {
    const T c0 = (T)(0.31539156525252000603);  // sqrt(5/(16pi))
    const T c1 = (T)(1.09254843059207907054);  // sqrt(15/(4pi))
    const T c2 = (T)(0.54627421529603953527);  // sqrt(15/(16pi))
    y[0] = c0 * ((T)2 * uz * uz - ux * ux - uy * uy);
    gy[0][0] = -(T)2 * c0 * ux; gy[0][1] = -(T)2 * c0 * uy; gy[0][2] = (T)4 * c0 * uz;
    y[1] = c1 * ux * uz; gy[1][0] = c1 * uz; gy[1][1] = 0; gy[1][2] = c1 * ux;
    y[2] = c1 * uy * uz; gy[2][0] = 0; gy[2][1] = c1 * uz; gy[2][2] = c1 * uy;
    y[3] = c2 * (ux * ux - uy * uy); gy[3][0] = (T)2 * c2 * ux; gy[3][1] = -(T)2 * c2 * uy; gy[3][2] = 0;
    y[4] = c1 * ux * uy; gy[4][0] = c1 * uy; gy[4][1] = c1 * ux; gy[4][2] = 0;
  }
}

template <typename T>
__device__ __forceinline__ T gsqrt(T x);
template <>
__device__ __forceinline__ double gsqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float gsqrt<float>(float x) { return sqrtf(x); }

// Adds the orbitals of species `sp` at displacement d (one lattice image, |d| < rcut assumed
// by the caller) to phi[0..norb) if PHI and to grad[0..norb)[3] if GRAD.
// grad phi = u (f' Y - l f Y / r) + (f / r) grad_u y(u), with Y = y(u), u = d / r.
template <typename T, bool PHI, bool GRAD>
__device__ __forceinline__ void add_orbitals(const GTabs &g, const typename Tab2<T>::type *__restrict__ tab, int sp,
                                             T dx, T dy, T dz, T *phi, T (*grad)[3],
                                             const float *__restrict__ dtab = nullptr) {
  const GSpecies &S = g.sp[sp];
  T r2 = dx * dx + dy * dy + dz * dz;
  T r = gsqrt<T>(r2);
  bool at0 = r < (T)1e-12;
  T inv_r = at0 ? (T)0 : (T)1 / r;
  T ux = dx * inv_r, uy = dy * inv_r, uz = dz * inv_r;
  int col = 0;
  for (int k = 0; k < S.nrad; ++k) {
    const GRadial &R = g.rad[S.rad0 + k];
    const int l = R.l, nm = 2 * l + 1;
    if (r < (T)R.rc) {
      T f, df;
      radial_eval<T>(tab, R, r, f, df, dtab);
      if (at0) {
        if (PHI && l == 0) phi[col] += f * (T)0.28209479177387814347;
        if (GRAD && l == 1) {
          const T c = (T)0.48860251190291992159 * df;
          grad[col + 0][2] += c;
          grad[col + 1][0] += c;
          grad[col + 2][1] += c;
        }
      } else {
        T y[5], gy[5][3];
        ylm_unit<T>(l, ux, uy, uz, y, gy);
        T a = 0, fr = 0;
        if (GRAD) {
          fr = f * inv_r;
        }
        for (int m = 0; m < nm; ++m) {
          if (PHI) phi[col + m] += f * y[m];
          if (GRAD) {
            a = df * y[m] - (T)l * fr * y[m];
            grad[col + m][0] += a * ux + fr * gy[m][0];
            grad[col + m][1] += a * uy + fr * gy[m][1];
            grad[col + m][2] += a * uz + fr * gy[m][2];
          }
        }
      }
    }
    col += nm;
  }
}

// Device error word bits.
#define GINT_ERRBIT_CAPACITY 1u
#define GINT_ERRBIT_SKIN 2u
#define GINT_ERRBIT_INDEX 4u
#define GINT_ERRBIT_TIMEOUT 8u
