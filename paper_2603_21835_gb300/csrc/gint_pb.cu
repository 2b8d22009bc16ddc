// gint_pb.cu -- velocity-gauge nonlocal projector overlaps on atom-centred spherical grids (paper
// Sec. 3.3.2, "Spherical Grid Integration for Nonlocal Potentials"):
//   P_{j mu}^{IJ}(A) = <beta_{I j}| e^{-i A.r} |Phi_{J mu}> = int beta_{I j}(r - tau_I) e^{-i A.r} Phi_{J mu}(r) dr
// for every projector atom I and every atom J whose orbitals reach I's projectors (Phi: the orbital
// summed over the lattice images of J, Gamma point).  The integral runs on a grid centred on tau_I:
// r = tau_I + x, x = r_k e_a, with 140 Gauss-Legendre radial nodes on [0, rc_beta] (weight r^2) and an
// angular rule of degree 17.  The paper uses the 110-point Lebedev-Laikov rule; its table is not
// available here, so a product rule of the same degree stands in: 9 Gauss-Legendre nodes in
// cos(theta) times 18 equally spaced azimuths (162 points).
//
// GPU organisation (as the paper describes it): one CTA per (I, J) pair, one thread per angular
// point, each thread accumulating its ray over all radial nodes; the sums over angular points are
// warp-shuffle reductions followed by one shared-memory pass, no atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "gint_handle.cuh"

namespace {

constexpr int kPbTheta = 9, kPbPhi = 18, kPbRays = kPbTheta * kPbPhi, kPbNr = 140;
constexpr int kPbThreads = 192, kPbWarps = kPbThreads / 32;
constexpr int kPbMaxOrb = 16;  // orbitals of the neighbour atom (accumulators held in registers)
constexpr int kPbGroup = 2;    // projector radials per pass over the ray
constexpr int kPbRed = 2 * 5 * kPbMaxOrb;  // reduction slots of one projector radial (l <= 2)
constexpr double kPi = 3.14159265358979323846;
static_assert(kPbRays <= kPbThreads, "one thread per angular point");

__constant__ double c_ang[kPbRays][4];  // unit vector and weight (weights sum to 4 pi)
__constant__ double c_rad[kPbNr][2];    // node in (0, 1) and weight of the rule on [0, 1]

struct GPb {
  double A[3];
  const int *pI, *pJ;
  const long long *poff;
  const int *img_off;
  const double *img;  // image positions tau_J + R of the pair's neighbour atom
  const double *pos;
  const int *species;
  const double2 *tab, *ptab;  // orbital and projector tables, (f, f') per knot
};

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n from the three-term
// recurrence; initial guesses cos(pi (i + 3/4) / (n + 1/2))).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);  // P_n'
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Sum over the CTA of v (threads beyond the rays hold 0): warp shuffles, then lane 0 of each warp
// stores its warp's sum at red[warp][slot].
__device__ __forceinline__ void warp_sum_to(double v, double (*red)[kPbRed], int slot) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][slot] = v;
}

__global__ void __launch_bounds__(kPbThreads) k_psibeta(const __grid_constant__ GTabs orb,
                                                        const __grid_constant__ GTabs prj,
                                                        const __grid_constant__ GPb P, double *__restrict__ out) {
  __shared__ double red[kPbWarps][kPbRed];
  const int p = blockIdx.x, I = P.pI[p], J = P.pJ[p];
  const int spI = P.species[I], spJ = P.species[J];
  const GSpecies &SJ = orb.sp[spJ];
  const GSpecies &SB = prj.sp[spI];
  const int noJ = SJ.norb;
  const int a = threadIdx.x;
  const bool ray = a < kPbRays;
  const double ex = ray ? c_ang[a][0] : 0.0, ey = ray ? c_ang[a][1] : 0.0, ez = ray ? c_ang[a][2] : 0.0;
  const double wa = ray ? c_ang[a][3] : 0.0;
  const double tx = P.pos[3 * I], ty = P.pos[3 * I + 1], tz = P.pos[3 * I + 2];
  const int i0 = P.img_off[p], i1 = P.img_off[p + 1];
  const double rcb = SB.rcut;
  double *o = out + 2 * P.poff[p];
  int col = 0;  // first projector function of the group
  for (int g0 = 0; g0 < SB.nrad; g0 += kPbGroup) {
    const int ng = min(kPbGroup, SB.nrad - g0);
    double acc[kPbGroup][kPbMaxOrb][2];
#pragma unroll
    for (int g = 0; g < kPbGroup; ++g)
#pragma unroll
      for (int m = 0; m < kPbMaxOrb; ++m) acc[g][m][0] = acc[g][m][1] = 0.0;
    if (ray) {
      for (int k = 0; k < kPbNr; ++k) {
        const double r = rcb * c_rad[k][0], wk = rcb * c_rad[k][1] * r * r;
        const double px = tx + r * ex, py = ty + r * ey, pz = tz + r * ez;
        double fb[kPbGroup];
#pragma unroll
        for (int g = 0; g < kPbGroup; ++g) {
          fb[g] = 0.0;
          if (g < ng) {
            const GRadial &R = prj.rad[SB.rad0 + g0 + g];
            double df;
            if (r < R.rc) radial_eval<double>(P.ptab, R, r, fb[g], df);
          }
        }
        double phi[kPbMaxOrb];
#pragma unroll
        for (int m = 0; m < kPbMaxOrb; ++m) phi[m] = 0.0;
        for (int q = i0; q < i1; ++q) {
          const double dx = px - P.img[3 * q], dy = py - P.img[3 * q + 1], dz = pz - P.img[3 * q + 2];
          if (dx * dx + dy * dy + dz * dz < SJ.rcut2)
            add_orbitals<double, true, false>(orb, P.tab, spJ, dx, dy, dz, phi, nullptr);
        }
        double s, c;
        sincos(-(P.A[0] * px + P.A[1] * py + P.A[2] * pz), &s, &c);
#pragma unroll
        for (int g = 0; g < kPbGroup; ++g) {
          const double wr = wk * fb[g], cr = wr * c, ci = wr * s;
#pragma unroll
          for (int m = 0; m < kPbMaxOrb; ++m) {
            acc[g][m][0] += cr * phi[m];
            acc[g][m][1] += ci * phi[m];
          }
        }
      }
    }
    // angular factors w_a Y_lm(e_a) and the sums over the rays, one projector radial at a time
    // (compile-time indices into the accumulators, which stay in registers)
#pragma unroll
    for (int g = 0; g < kPbGroup; ++g) {
      if (g >= ng) break;
      const int l = prj.rad[SB.rad0 + g0 + g].l, nm = 2 * l + 1;
      double y[5], gy[5][3];
      ylm_unit<double>(l, ex, ey, ez, y, gy);
      for (int mm = 0; mm < nm; ++mm) {
        const double f = ray ? wa * y[mm] : 0.0;
#pragma unroll
        for (int m = 0; m < kPbMaxOrb; ++m)
          if (m < noJ) {
            warp_sum_to(f * acc[g][m][0], red, 2 * (mm * noJ + m));
            warp_sum_to(f * acc[g][m][1], red, 2 * (mm * noJ + m) + 1);
          }
      }
      __syncthreads();
      for (int u = threadIdx.x; u < 2 * nm * noJ; u += kPbThreads) {
        double v = 0.0;
        for (int w = 0; w < kPbWarps; ++w) v += red[w][u];
        o[2 * col * noJ + u] = v;  // (projector col + u / (2 noJ), orbital (u / 2) mod noJ, re / im)
      }
      __syncthreads();
      col += nm;
    }
  }
}

template <typename T>
void pfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
int upload(T **dst, const std::vector<T> &src) {
  if (cudaMalloc(dst, std::max<size_t>(src.size(), 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return GINT_ENOMEM;
  }
  if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return GINT_ECUDA;
  return GINT_OK;
}

}  // namespace

void gint_pb_free(gint_handle *h) {
  pfree(h->pb_tab64);
  pfree(h->pb_I);
  pfree(h->pb_J);
  pfree(h->pb_off);
  pfree(h->pb_img_off);
  pfree(h->pb_img);
  h->pb_ready = false;
  h->pb_npairs = 0;
  h->pb_nelems = 0;
  h->pb_bytes = 0;
  h->pb_pairs_host.clear();
  h->pb_off_host.clear();
}

int gint_pb_set(gint_handle *h, int nspecies, const gint_species *proj) {
  const GGeom &g = h->geom;
  if (nspecies != g.nspecies || !proj) return GINT_EINVAL;
  for (int s = 0; s < nspecies; ++s)
    if (g.sp[s].norb > kPbMaxOrb) return GINT_EUNSUPPORTED;  // neighbour orbitals held in registers
  GTabs t{};
  std::vector<double2> tab;
  int r = 0;
  t.nspecies = nspecies;
  for (int s = 0; s < nspecies; ++s) {
    const gint_species &S = proj[s];
    if (S.nradial < 0 || (S.nradial > 0 && !S.radial)) return GINT_EINVAL;
    GSpecies &GS = t.sp[s];
    GS.nrad = S.nradial;
    GS.rad0 = r;
    for (int k = 0; k < S.nradial; ++k, ++r) {
      const gint_radial &R = S.radial[k];
      if (r >= GINT_MAX_RADIAL) return GINT_EINVAL;
      if (R.l < 0 || R.l > 2 || R.npts < 2 || !(R.dr > 0) || !(R.rc > 0) || !R.f || !R.df) return GINT_EINVAL;
      if (R.rc > (R.npts - 1) * R.dr * (1 + 1e-12)) return GINT_EINVAL;
      GRadial &GR = t.rad[r];
      GR.l = R.l;
      GR.npts = R.npts;
      GR.off = (int)tab.size();
      GR.dr = R.dr;
      GR.inv_dr = 1.0 / R.dr;
      GR.rc = R.rc;
      GR.rc2 = R.rc * R.rc;
      for (int i = 0; i < R.npts; ++i) tab.push_back(make_double2(R.f[i], R.df[i]));
      GS.norb += 2 * R.l + 1;
      GS.rcut = std::max(GS.rcut, R.rc);
    }
    GS.rcut2 = GS.rcut * GS.rcut;
  }
  t.nrad = r;
  // pairs (I, J): the images of J whose orbitals reach I's projector sphere
  const int na = g.natoms;
  std::vector<int> pI, pJ, img_off(1, 0);
  std::vector<long long> poff(1, 0);
  std::vector<double> img;
  for (int I = 0; I < na; ++I) {
    const GSpecies &SB = t.sp[h->species_host[I]];
    if (SB.nrad == 0) continue;
    for (int J = 0; J < na; ++J) {
      const GSpecies &SJ = g.sp[h->species_host[J]];
      const double reach = SB.rcut + SJ.rcut;
      double d0[3], u[3];
      for (int c = 0; c < 3; ++c) d0[c] = h->pos_host[3 * J + c] - h->pos_host[3 * I + c];
      for (int c = 0; c < 3; ++c) u[c] = d0[0] * g.inv[0 * 3 + c] + d0[1] * g.inv[1 * 3 + c] + d0[2] * g.inv[2 * 3 + c];
      int lo[3], hi[3];
      for (int c = 0; c < 3; ++c) {
        lo[c] = (int)std::ceil(-u[c] - reach * g.reach[c]);
        hi[c] = (int)std::floor(-u[c] + reach * g.reach[c]);
      }
      const size_t before = img.size();
      for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
        for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
          for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
            double d[3];
            for (int c = 0; c < 3; ++c) d[c] = d0[c] + n0 * g.cell[c] + n1 * g.cell[3 + c] + n2 * g.cell[6 + c];
            if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < reach * reach)
              for (int c = 0; c < 3; ++c) img.push_back(h->pos_host[3 * I + c] + d[c]);
          }
      if (img.size() == before) continue;
      pI.push_back(I);
      pJ.push_back(J);
      img_off.push_back((int)(img.size() / 3));
      poff.push_back(poff.back() + (long long)SB.norb * SJ.norb);
    }
  }
  // quadrature: radial Gauss-Legendre on [0, 1]; angular product rule of degree 17
  std::vector<double> x, w;
  gauss_legendre(kPbNr, x, w);
  double rad[kPbNr][2];
  for (int k = 0; k < kPbNr; ++k) {
    rad[k][0] = 0.5 * (x[k] + 1.0);
    rad[k][1] = 0.5 * w[k];
  }
  gauss_legendre(kPbTheta, x, w);
  double ang[kPbRays][4];
  for (int i = 0; i < kPbTheta; ++i)
    for (int j = 0; j < kPbPhi; ++j) {
      const double ct = x[i], st = std::sqrt(1.0 - ct * ct), ph = 2.0 * kPi * j / kPbPhi;
      double *e = ang[i * kPbPhi + j];
      e[0] = st * std::cos(ph);
      e[1] = st * std::sin(ph);
      e[2] = ct;
      e[3] = w[i] * 2.0 * kPi / kPbPhi;
    }
  if (cudaMemcpyToSymbol(c_rad, rad, sizeof(rad)) != cudaSuccess ||
      cudaMemcpyToSymbol(c_ang, ang, sizeof(ang)) != cudaSuccess) {
    cudaGetLastError();
    return GINT_ECUDA;
  }
  gint_pb_free(h);
  int rc;
  if ((rc = upload(&h->pb_tab64, tab)) || (rc = upload(&h->pb_I, pI)) || (rc = upload(&h->pb_J, pJ)) ||
      (rc = upload(&h->pb_off, poff)) || (rc = upload(&h->pb_img_off, img_off)) || (rc = upload(&h->pb_img, img))) {
    gint_pb_free(h);
    return rc;
  }
  h->pb_tabs = t;
  h->pb_npairs = (int)pI.size();
  h->pb_nelems = poff.back();
  h->pb_pairs_host.resize(2 * pI.size());
  for (size_t q = 0; q < pI.size(); ++q) {
    h->pb_pairs_host[2 * q] = pI[q];
    h->pb_pairs_host[2 * q + 1] = pJ[q];
  }
  h->pb_off_host = poff;
  h->pb_bytes = (long long)(tab.size() * sizeof(double2) + (2 * pI.size() + img_off.size()) * sizeof(int) +
                            poff.size() * sizeof(long long) + img.size() * sizeof(double));
  h->pb_ready = true;
  return GINT_OK;
}

int gint_pb_run(gint_handle *h, const double A[3], double *out, cudaStream_t st) {
  if (!h->pb_ready) return GINT_EINVAL;
  if (h->pb_npairs == 0) return GINT_OK;
  GPb P{};
  for (int c = 0; c < 3; ++c) P.A[c] = A[c];
  P.pI = h->pb_I;
  P.pJ = h->pb_J;
  P.poff = h->pb_off;
  P.img_off = h->pb_img_off;
  P.img = h->pb_img;
  P.pos = h->pos_dev;
  P.species = h->species_dev;
  P.tab = h->tab64;
  P.ptab = h->pb_tab64;
  k_psibeta<<<(unsigned)h->pb_npairs, kPbThreads, 0, st>>>(h->geom, h->pb_tabs, P, out);
  return cudaGetLastError() == cudaSuccess ? GINT_OK : GINT_ECUDA;
}
