// gint_nbr.cu -- device builder of the grid-brick -> atom neighbour lists (the paper's
// BigGrid neighbour relation managed by GintInfo, Sec. 3.3.1 and Fig. 2).
//
// The grid is cut into bricks of 4 x 4 x 8 points.  An (atom, lattice image) entry belongs
// to a brick when at least one of the brick's grid points lies strictly inside the atom's
// support sphere (exact per-point test, float64).  Entries of one atom form a "slot": its
// orbitals occupy one set of columns in the brick (periodic images folded, Gamma point).  In the
// unfolded layout (the per-R twin of a folded handle) every entry is a slot of its own, in the same
// order (atom, then lattice vector (n1, n2, n3) ascending).
// Each brick also gets an n_a x n_a table of global pair indices for its slots.
#include <cuda_runtime.h>

#include "gint_handle.cuh"

namespace {

__device__ __forceinline__ void brick_box(const GGeom &g, long long b, int lo[3], int hi[3]) {
  int bk = (int)(b % g.nbk);
  int bj = (int)((b / g.nbk) % g.nbj);
  int bi = (int)(b / ((long long)g.nbk * g.nbj));
  lo[0] = bi * GINT_BI; hi[0] = min(lo[0] + GINT_BI, g.n1);
  lo[1] = bj * GINT_BJ; hi[1] = min(lo[1] + GINT_BJ, g.n2);
  lo[2] = bk * GINT_BK; hi[2] = min(lo[2] + GINT_BK, g.n3);
}

// Centre and bounding radius of a brick's point set (a parallelepiped lattice: the farthest
// point from the centre is a corner).
__device__ void brick_sphere(const GGeom &g, const int lo[3], const int hi[3], double c[3], double &rad) {
  double fc[3] = {0.5 * (lo[0] + hi[0] - 1) / g.n1, 0.5 * (lo[1] + hi[1] - 1) / g.n2,
                  0.5 * (lo[2] + hi[2] - 1) / g.n3};
  for (int d = 0; d < 3; ++d) c[d] = fc[0] * g.cell[d] + fc[1] * g.cell[3 + d] + fc[2] * g.cell[6 + d];
  double r2 = 0;
  for (int corner = 0; corner < 8; ++corner) {
    int ii = (corner & 1) ? hi[0] - 1 : lo[0];
    int jj = (corner & 2) ? hi[1] - 1 : lo[1];
    int kk = (corner & 4) ? hi[2] - 1 : lo[2];
    double p[3];
    grid_point(g, ii, jj, kk, p);
    double dd = (p[0] - c[0]) * (p[0] - c[0]) + (p[1] - c[1]) * (p[1] - c[1]) + (p[2] - c[2]) * (p[2] - c[2]);
    r2 = fmax(r2, dd);
  }
  rad = sqrt(r2) * (1.0 + 1e-12) + 1e-12;
}

// Image range of atom I around a brick sphere (centre c, radius rad); fixed arithmetic so
// that the counting and filling passes take identical decisions.
__device__ __noinline__ void image_range(const GGeom &g, const double *pos, int I, double rc, const double c[3],
                                         double rad, int nlo[3], int nhi[3]) {
  double d0[3], u[3];
  for (int d = 0; d < 3; ++d) d0[d] = c[d] - pos[3 * I + d];
  for (int d = 0; d < 3; ++d) u[d] = d0[0] * g.inv[0 * 3 + d] + d0[1] * g.inv[1 * 3 + d] + d0[2] * g.inv[2 * 3 + d];
  for (int d = 0; d < 3; ++d) {
    double reach = (rc + rad) * g.reach[d];
    nlo[d] = (int)ceil(u[d] - reach);
    nhi[d] = (int)floor(u[d] + reach);
  }
}

// The brick's grid points relative to the brick-sphere centre c as float32, four per lane (point
// q = lane + 32 k, k = 0..3, in the order kk fastest, then jj, then ii), for the warp-wide coverage
// test.  n: the number of points in the box (128 except at the grid's upper faces).
struct BrickPts {
  float x[4], y[4], z[4];
  int n;
};
__device__ __forceinline__ void point_of(const int lo[3], const int hi[3], int q, int &ii, int &jj, int &kk) {
  const int ny = hi[1] - lo[1], nz = hi[2] - lo[2];
  kk = lo[2] + q % nz;
  jj = lo[1] + (q / nz) % ny;
  ii = lo[0] + q / (nz * ny);
}
__device__ void brick_points(const GGeom &g, const int lo[3], const int hi[3], const double c[3], int lane,
                             BrickPts &P) {
  P.n = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int q = lane + 32 * k;
    P.x[k] = P.y[k] = P.z[k] = 0.f;
    if (q < P.n) {
      int ii, jj, kk;
      point_of(lo, hi, q, ii, jj, kk);
      double p[3];
      grid_point(g, ii, jj, kk, p);
      P.x[k] = (float)(p[0] - c[0]);
      P.y[k] = (float)(p[1] - c[1]);
      P.z[k] = (float)(p[2] - c[2]);
    }
  }
}

// Does the image T of an atom with support radius rc cover any grid point of the brick box (some
// point strictly inside the sphere, float64)?  All 32 lanes take part with the same T and rc, each
// testing its four points.  A float32 squared distance relative to the brick centre decides every
// point outside a shell |r^2 - rc^2| < m around the sphere; a point inside the shell is decided by
// the float64 test itself (same expression as a per-point loop), so the answer equals the float64
// one.  Bound used for m: with |p - c| <= rad and |T - c| < rc + rad (the caller's bounding-sphere
// test), each float32 difference is off by at most 2^-24 (2 rc + 4 rad) and the float32 r^2 by at
// most 2 sqrt(3) (rc + 2 rad) 2^-24 (2 rc + 4 rad) + 4 2^-24 r^2, about 1e-7 (2 rc + 4 rad)^2 +
// 2.4e-7 r^2; m is forty times the first term plus four times the second.  Warp-uniform result.
__device__ bool warp_image_hits(const GGeom &g, const BrickPts &P, const double T[3], double rc, const int lo[3],
                                const int hi[3], const double c[3], double rad, int lane) {
  const float tx = (float)(T[0] - c[0]), ty = (float)(T[1] - c[1]), tz = (float)(T[2] - c[2]);
  const double rc2 = rc * rc, ext = 2.0 * rc + 4.0 * rad;
  const double m = 4e-6 * ext * ext + 1e-6 * rc2;
  const float in2 = (float)(rc2 - m), out2 = (float)(rc2 + m);
  bool hit = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int q = lane + 32 * k;
    if (q >= P.n) continue;
    const float dx = P.x[k] - tx, dy = P.y[k] - ty, dz = P.z[k] - tz;
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (r2 < in2) {
      hit = true;
    } else if (r2 < out2) {
      int ii, jj, kk;
      point_of(lo, hi, q, ii, jj, kk);
      double p[3];
      grid_point(g, ii, jj, kk, p);
      const double e2 = (p[0] - T[0]) * (p[0] - T[0]) + (p[1] - T[1]) * (p[1] - T[1]) + (p[2] - T[2]) * (p[2] - T[2]);
      if (e2 < rc2) hit = true;
    }
  }
  return __any_sync(0xffffffffu, hit);
}

// The lattice images of the warp's atoms (lane l: atom a0 + l) near brick b, one candidate at a
// time: every image in the atom's image range whose bounding-sphere test passes (centre distance
// below rc + rad) is tested against the brick's points by the whole warp, in lane order and, within
// a lane, in the order n0, n1, n2 ascending.  visit(src, T, hit) runs in every lane with the same
// arguments (src: the lane whose atom the image belongs to).
template <typename Visit>
__device__ void warp_atom_images(const GGeom &g, const double *pos, const int *species, int a0, int lane,
                                 const int lo[3], const int hi[3], const double c[3], double rad, const BrickPts &P,
                                 Visit visit) {
  const int I = a0 + lane;
  const bool va = I < g.natoms;
  const double rc = va ? g.sp[species[I]].rcut : 0.0;
  int nlo[3] = {0, 0, 0}, nhi[3] = {-1, -1, -1};
  if (va) image_range(g, pos, I, rc, c, rad, nlo, nhi);
  const int s1 = max(0, nhi[1] - nlo[1] + 1), s2 = max(0, nhi[2] - nlo[2] + 1);
  const int nimg = max(0, nhi[0] - nlo[0] + 1) * s1 * s2;
  const double lim2 = (rc + rad) * (rc + rad);
  int k = 0;
  double T[3] = {0.0, 0.0, 0.0};
  auto next = [&]() -> bool {
    while (k < nimg) {
      const int i0 = k / (s1 * s2), r = k - i0 * s1 * s2, i1 = r / s2, i2 = r - i1 * s2;
      ++k;
      const int n0 = nlo[0] + i0, n1 = nlo[1] + i1, n2 = nlo[2] + i2;
      for (int d = 0; d < 3; ++d) T[d] = pos[3 * I + d] + n0 * g.cell[d] + n1 * g.cell[3 + d] + n2 * g.cell[6 + d];
      const double D2 = (c[0] - T[0]) * (c[0] - T[0]) + (c[1] - T[1]) * (c[1] - T[1]) + (c[2] - T[2]) * (c[2] - T[2]);
      if (!(D2 >= lim2)) return true;
    }
    return false;
  };
  bool cand = next();
  for (;;) {
    const unsigned m = __ballot_sync(0xffffffffu, cand);
    if (!m) break;
    const int src = __ffs(m) - 1;
    double Ts[3];
    for (int d = 0; d < 3; ++d) Ts[d] = __shfl_sync(0xffffffffu, T[d], src);
    const double rcs = __shfl_sync(0xffffffffu, rc, src);
    const bool hit = warp_image_hits(g, P, Ts, rcs, lo, hi, c, rad, lane);
    visit(src, Ts, hit);
    if (lane == src) cand = next();
  }
}

__device__ __forceinline__ int warp_excl_scan(int v, int lane) {
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x - v;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per brick: number of slots, entries and orbitals.
__global__ void k_brick_count(GGeom g, const double *pos, const int *species, int unfold, int *n_at, int *n_ent,
                              int *n_orb) {
  const int lane = threadIdx.x & 31;
  const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= g.nbricks) return;
  int lo[3], hi[3];
  brick_box(g, b, lo, hi);
  double c[3], rad;
  brick_sphere(g, lo, hi, c, rad);
  BrickPts P;
  brick_points(g, lo, hi, c, lane, P);
  int at = 0, ent = 0, orb = 0;
  for (int a0 = 0; a0 < g.natoms; a0 += 32) {
    const int I = a0 + lane;
    int cnt = 0;
    warp_atom_images(g, pos, species, a0, lane, lo, hi, c, rad, P, [&](int src, const double *, bool hit) {
      if (hit && lane == src) ++cnt;
    });
    const int slots = unfold ? cnt : (cnt > 0);
    at += (int)warp_sum_ll(slots);
    ent += (int)warp_sum_ll(cnt);
    orb += (int)warp_sum_ll(slots * g.sp[species[I < g.natoms ? I : 0]].norb);
  }
  if (lane == 0) {
    n_at[b] = at;
    n_ent[b] = ent;
    n_orb[b] = orb;
  }
}

// Single-CTA exclusive scans of the per-brick counts; also the totals and maxima.
//   out[0] = slots, out[1] = entries, out[2] = pair-table size, out[3] = max orbitals,
//   out[4] = max atoms, out[5] = executed pair work sum_b 128 norb_b^2, out[6] = max entries
__global__ void k_brick_scan(long long nb, const int *n_at, const int *n_ent, const int *n_orb, long long *at_off,
                             long long *ent_off, long long *pair_off, long long *out) {
  __shared__ long long s_at[1024], s_ent[1024], s_pr[1024];
  __shared__ int s_mo[1024], s_ma[1024], s_me[1024];
  __shared__ long long s_wx[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  long long chunk = (nb + nt - 1) / nt;
  long long b0 = t * chunk, b1 = min(nb, b0 + chunk);
  long long a = 0, e = 0, p = 0, wx = 0;
  int mo = 0, ma = 0, me = 0;
  for (long long b = b0; b < b1; ++b) {
    me = max(me, n_ent[b]);
    a += n_at[b];
    e += n_ent[b];
    p += (long long)n_at[b] * n_at[b];
    wx += (long long)n_orb[b] * n_orb[b];
    mo = max(mo, n_orb[b]);
    ma = max(ma, n_at[b]);
  }
  s_at[t] = a; s_ent[t] = e; s_pr[t] = p; s_mo[t] = mo; s_ma[t] = ma; s_wx[t] = wx; s_me[t] = me;
  __syncthreads();
  if (t == 0) {
    long long ra = 0, re = 0, rp = 0, rw = 0;
    int rmo = 0, rma = 0, rme = 0;
    for (int i = 0; i < nt; ++i) {
      rme = max(rme, s_me[i]);
      long long ta = s_at[i], te = s_ent[i], tp = s_pr[i];
      s_at[i] = ra; s_ent[i] = re; s_pr[i] = rp;
      ra += ta; re += te; rp += tp; rw += s_wx[i];
      rmo = max(rmo, s_mo[i]);
      rma = max(rma, s_ma[i]);
    }
    out[0] = ra; out[1] = re; out[2] = rp; out[3] = rmo; out[4] = rma; out[5] = rw * GINT_BPTS; out[6] = rme;
    at_off[nb] = ra; ent_off[nb] = re; pair_off[nb] = rp;
  }
  __syncthreads();
  a = s_at[t]; e = s_ent[t]; p = s_pr[t];
  for (long long b = b0; b < b1; ++b) {
    at_off[b] = a; ent_off[b] = e; pair_off[b] = p;
    a += n_at[b];
    e += n_ent[b];
    p += (long long)n_at[b] * n_at[b];
  }
}

// One warp per brick: writes slots (atom, column, first entry) and entries (image shifts): the
// images are visited twice in the same order, to count them (offsets of each atom's slots and
// entries) and to write them.
__global__ void k_brick_fill(GGeom g, const double *pos, const int *species, int unfold, const long long *at_off,
                             const long long *ent_off, int *s_atom, int *s_col, long long *s_ent, double *e_shift,
                             unsigned *err) {
  const int lane = threadIdx.x & 31;
  const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= g.nbricks) return;
  int lo[3], hi[3];
  brick_box(g, b, lo, hi);
  double c[3], rad;
  brick_sphere(g, lo, hi, c, rad);
  BrickPts P;
  brick_points(g, lo, hi, c, lane, P);
  long long slot = at_off[b], ent = ent_off[b];
  const long long slot_end = at_off[b + 1], ent_end = ent_off[b + 1];
  int col = 0;
  for (int a0 = 0; a0 < g.natoms; a0 += 32) {
    const int I = a0 + lane;
    int cnt = 0;
    warp_atom_images(g, pos, species, a0, lane, lo, hi, c, rad, P, [&](int src, const double *, bool hit) {
      if (hit && lane == src) ++cnt;
    });
    const int nsl = unfold ? cnt : (cnt > 0);  // slots of this atom
    const int my_slot = warp_excl_scan(nsl, lane);
    const int my_ent = warp_excl_scan(cnt, lane);
    const int no = (cnt > 0) ? g.sp[species[I]].norb : 0;
    const int my_col = warp_excl_scan(nsl * no, lane);
    if (cnt > 0) {
      const long long k = slot + my_slot;
      const long long e0 = ent + my_ent;
      for (int j = 0; j < nsl; ++j)
        if (k + j < slot_end) {
          s_atom[k + j] = I;
          s_col[k + j] = col + my_col + j * no;
          s_ent[k + j] = e0 + j;
        }
    }
    long long e = ent + my_ent;
    if (__any_sync(0xffffffffu, cnt > 0))
      warp_atom_images(g, pos, species, a0, lane, lo, hi, c, rad, P, [&](int src, const double *T, bool hit) {
        if (hit && lane == src) {
          if (e < ent_end) {
            e_shift[3 * e + 0] = T[0];
            e_shift[3 * e + 1] = T[1];
            e_shift[3 * e + 2] = T[2];
          }
          ++e;
        }
      });
    slot += warp_sum_ll(nsl);
    ent += warp_sum_ll(cnt);
    col += (int)warp_sum_ll(nsl * no);
  }
  if (lane == 0 && (slot != slot_end || ent != ent_end)) atomicOr(err, GINT_ERRBIT_INDEX);
}

// Minimum distance over lattice images between atoms I and J.
__device__ double min_image_dist(const GGeom &g, const double *pos, int I, int J, double limit) {
  double d0[3], u[3];
  for (int d = 0; d < 3; ++d) d0[d] = pos[3 * J + d] - pos[3 * I + d];
  for (int d = 0; d < 3; ++d) u[d] = d0[0] * g.inv[0 * 3 + d] + d0[1] * g.inv[1 * 3 + d] + d0[2] * g.inv[2 * 3 + d];
  double best = 1e300;
  int nlo[3], nhi[3];
  for (int d = 0; d < 3; ++d) {
    nlo[d] = (int)ceil(-u[d] - limit * g.reach[d]);
    nhi[d] = (int)floor(-u[d] + limit * g.reach[d]);
  }
  for (int n0 = nlo[0]; n0 <= nhi[0]; ++n0)
    for (int n1 = nlo[1]; n1 <= nhi[1]; ++n1)
      for (int n2 = nlo[2]; n2 <= nhi[2]; ++n2) {
        double x[3];
        for (int d = 0; d < 3; ++d) x[d] = d0[d] + n0 * g.cell[d] + n1 * g.cell[3 + d] + n2 * g.cell[6 + d];
        best = fmin(best, sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
      }
  return best;
}

// One warp per brick: pair table of its slots; flags pairs that overlap but have no block.
__global__ void k_brick_pairs(GGeom g, const double *pos, const int *species, const long long *at_off,
                              const int *s_atom, const long long *bp_off, const int *pair_row, const int *pair_col,
                              int *b_pair, unsigned *err) {
  const int lane = threadIdx.x & 31;
  const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= g.nbricks) return;
  const long long s0 = at_off[b];
  const int na = (int)(at_off[b + 1] - s0);
  for (int e = lane; e < na * na; e += 32) {
    int I = s_atom[s0 + e / na], J = s_atom[s0 + e % na];
    int lo = pair_row[I], hi = pair_row[I + 1] - 1, found = -1;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1;
      int v = pair_col[mid];
      if (v == J) { found = mid; break; }
      if (v < J) lo = mid + 1; else hi = mid - 1;
    }
    if (found < 0) {
      double lim = g.sp[species[I]].rcut + g.sp[species[J]].rcut;
      if (min_image_dist(g, pos, I, J, lim) < lim) atomicOr(err, GINT_ERRBIT_SKIN);
    }
    b_pair[bp_off[b] + e] = found;
  }
}

// Exact algorithmic work: W = sum_g n_g^2 with n_g the orbitals covering point g.  One CTA per
// brick, one thread per point.  The brick's entries and the slots' screening bounds (at most kCwE
// entries and kCwS slots; larger bricks take the plain float64 loop) are staged in shared memory,
// the entries as float32 offsets from the brick centre, and each (point, entry)
// distance is screened in float32 as in warp_image_hits, the float64 test deciding points in the
// thin shell around the sphere: the same coverage, so the same W, as the per-entry float64 loop.
constexpr int kCwE = 256, kCwS = 64;
__global__ void k_count_work(GGeom g, const long long *at_off, const int *s_atom, const long long *s_ent,
                             const double *e_shift, const int *species, double *W) {
  const long long b = blockIdx.x;
  const int p = threadIdx.x;
  __shared__ float ex[kCwE], ey[kCwE], ez[kCwE], sin2[kCwS], sout2[kCwS];
  __shared__ double sc[4];  // brick centre and bounding radius
  if (p == 0) {
    int lo[3], hi[3];
    brick_box(g, b, lo, hi);
    brick_sphere(g, lo, hi, sc, sc[3]);
  }
  __syncthreads();
  const double c[3] = {sc[0], sc[1], sc[2]}, rad = sc[3];
  const long long s0 = at_off[b], s1 = at_off[b + 1];
  const long long E0 = s1 > s0 ? s_ent[s0] : 0, E1 = s1 > s0 ? s_ent[s1] : 0;
  const bool staged = E1 - E0 <= kCwE && s1 - s0 <= kCwS;
  if (staged) {
    for (long long e = E0 + p; e < E1; e += blockDim.x) {
      ex[e - E0] = (float)(e_shift[3 * e] - c[0]);
      ey[e - E0] = (float)(e_shift[3 * e + 1] - c[1]);
      ez[e - E0] = (float)(e_shift[3 * e + 2] - c[2]);
    }
    for (long long s = s0 + p; s < s1; s += blockDim.x) {
      const GSpecies &S = g.sp[species[s_atom[s]]];
      const double ext = 2.0 * S.rcut + 4.0 * rad, m = 4e-6 * ext * ext + 1e-6 * S.rcut2;
      sin2[s - s0] = (float)(S.rcut2 - m);
      sout2[s - s0] = (float)(S.rcut2 + m);
    }
  }
  __syncthreads();
  int i, j, k;
  double acc = 0;
  if (brick_point(g, b, p, i, j, k)) {
    double r[3];
    grid_point(g, i, j, k, r);
    const float px = (float)(r[0] - c[0]), py = (float)(r[1] - c[1]), pz = (float)(r[2] - c[2]);
    int n = 0;
    for (long long s = s0; s < s1; ++s) {
      const GSpecies &S = g.sp[species[s_atom[s]]];
      const float in2 = staged ? sin2[s - s0] : 0.f, out2 = staged ? sout2[s - s0] : 0.f;
      bool cov = false;
      for (long long e = s_ent[s]; e < s_ent[s + 1] && !cov; ++e) {
        bool exact = !staged;
        if (staged) {
          const float dx = px - ex[e - E0], dy = py - ey[e - E0], dz = pz - ez[e - E0];
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < in2) cov = true;
          else exact = r2 < out2;
        }
        if (exact) {
          double dx = r[0] - e_shift[3 * e], dy = r[1] - e_shift[3 * e + 1], dz = r[2] - e_shift[3 * e + 2];
          cov = dx * dx + dy * dy + dz * dz < S.rcut2;
        }
      }
      if (cov) n += S.norb;
    }
    acc = (double)n * (double)n;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[GINT_BPTS / 32];
  if ((p & 31) == 0) red[p >> 5] = acc;
  __syncthreads();
  if (p == 0) {
    double t = 0;
    for (int w = 0; w < GINT_BPTS / 32; ++w) t += red[w];
    atomicAdd(W, t);
  }
}

}  // namespace

#define NBR_CHECK(x)                      \
  do {                                    \
    cudaError_t e_ = (x);                 \
    if (e_ != cudaSuccess) return GINT_ECUDA; \
  } while (0)

// Builds the neighbour structure for the current positions (h->pos_dev).  Synchronous.
int gint_build_neighbours(gint_handle *h, cudaStream_t st) {
  GGeom &g = h->geom;
  const long long nb = g.nbricks;
  const int wpb = 4;  // warps (bricks) per CTA
  const unsigned nblk = (unsigned)((nb + wpb - 1) / wpb);
  k_brick_count<<<nblk, 32 * wpb, 0, st>>>(g, h->pos_dev, h->species_dev, h->unfold ? 1 : 0, h->n_at, h->n_ent,
                                           h->n_orb);
  NBR_CHECK(cudaGetLastError());
  k_brick_scan<<<1, 1024, 0, st>>>(nb, h->n_at, h->n_ent, h->n_orb, h->b_at_off, h->b_ent_off, h->b_pair_off,
                                   h->scan_out);
  NBR_CHECK(cudaGetLastError());
  long long tot[7];
  NBR_CHECK(cudaMemcpyAsync(tot, h->scan_out, sizeof(tot), cudaMemcpyDeviceToHost, st));
  NBR_CHECK(cudaStreamSynchronize(st));
  h->nslots = tot[0];
  h->nent = tot[1];
  h->npairtab = tot[2];
  h->max_brick_orb = (int)tot[3];
  h->max_brick_atoms = (int)tot[4];
  h->W_exec = (double)tot[5];
  h->max_brick_ent = (int)tot[6];
  h->folded = h->nent != h->nslots;  // some slot holds several images
  if (h->max_brick_atoms > GINT_MAX_ATOMS_BRICK) return GINT_ECAPACITY;
  int rc = gint_reserve_nbr(h);
  if (rc) return rc;
  NBR_CHECK(cudaMemsetAsync(h->err_word, 0, sizeof(unsigned), st));
  k_brick_fill<<<nblk, 32 * wpb, 0, st>>>(g, h->pos_dev, h->species_dev, h->unfold ? 1 : 0, h->b_at_off,
                                          h->b_ent_off, h->s_atom, h->s_col, h->s_ent, h->e_shift, h->err_word);
  NBR_CHECK(cudaGetLastError());
  // sentinel: s_ent[nslots] = nent
  NBR_CHECK(cudaMemcpyAsync(h->s_ent + h->nslots, h->b_ent_off + nb, sizeof(long long), cudaMemcpyDeviceToDevice, st));
  k_brick_pairs<<<nblk, 32 * wpb, 0, st>>>(g, h->pos_dev, h->species_dev, h->b_at_off, h->s_atom, h->b_pair_off,
                                           h->pair_row_dev, h->pair_col_dev, h->b_pair, h->err_word);
  NBR_CHECK(cudaGetLastError());
  NBR_CHECK(cudaMemsetAsync(h->scal, 0, sizeof(double), st));
  k_count_work<<<(unsigned)nb, GINT_BPTS, 0, st>>>(g, h->b_at_off, h->s_atom, h->s_ent, h->e_shift, h->species_dev,
                                                   h->scal);
  NBR_CHECK(cudaGetLastError());
  unsigned err = 0;
  double W = 0;
  NBR_CHECK(cudaMemcpyAsync(&err, h->err_word, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  NBR_CHECK(cudaMemcpyAsync(&W, h->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  NBR_CHECK(cudaStreamSynchronize(st));
  h->W = W;
  if (err & GINT_ERRBIT_INDEX) return GINT_EDEVICE;
  if (err & GINT_ERRBIT_SKIN) return GINT_ESKIN;
  return GINT_OK;
}
