// gint_capi.cu -- the extern "C" boundary of libgint (declared in include/gint.h).
//
// Set-up mirrors the paper's GintInfo (Sec. 3.3.1, Fig. 2): geometry, the fine grid and its
// coarse blocks ("bricks"), the brick -> atom neighbour relation (built on the device), and
// the atom-pair block layout of the matrices.  Compute calls dispatch to the SIMT (FP64,
// FP32) or tensor-core (F16x3, F16x1) kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "gint_handle.cuh"

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

template <typename T>
int dalloc(T **p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  if (cudaMalloc((void **)p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return GINT_ENOMEM;
  }
  return GINT_OK;
}

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_all(gint_handle *h) {
  dfree(h->tab64); dfree(h->tab32); dfree(h->tab32i); dfree(h->dtab32); dfree(h->dtab32i);
  dfree(h->pos_dev); dfree(h->species_dev);
  dfree(h->pair_row_dev); dfree(h->pair_col_dev); dfree(h->pair_off_dev); dfree(h->pair_T_dev); dfree(h->pair_I_dev);
  dfree(h->n_at); dfree(h->n_ent); dfree(h->n_orb);
  dfree(h->b_at_off); dfree(h->b_ent_off); dfree(h->b_pair_off); dfree(h->scan_out);
  dfree(h->s_atom); dfree(h->s_col); dfree(h->s_ent); dfree(h->e_shift); dfree(h->b_pair);
  dfree(h->D32); dfree(h->work_ctr); dfree(h->red); dfree(h->scal); dfree(h->err_word);
  gint_tc_free(h);
  gint_hr_free(h);
  gint_pb_free(h);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  h->own_stream = nullptr;
  if (h->twin) {
    free_all(h->twin);
    delete h->twin;
    h->twin = nullptr;
  }
}

void inverse3(const double a[9], double inv[9], double *det) {
  double d = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
             a[2] * (a[3] * a[7] - a[4] * a[6]);
  inv[0] = (a[4] * a[8] - a[5] * a[7]) / d;
  inv[1] = (a[2] * a[7] - a[1] * a[8]) / d;
  inv[2] = (a[1] * a[5] - a[2] * a[4]) / d;
  inv[3] = (a[5] * a[6] - a[3] * a[8]) / d;
  inv[4] = (a[0] * a[8] - a[2] * a[6]) / d;
  inv[5] = (a[2] * a[3] - a[0] * a[5]) / d;
  inv[6] = (a[3] * a[7] - a[4] * a[6]) / d;
  inv[7] = (a[1] * a[6] - a[0] * a[7]) / d;
  inv[8] = (a[0] * a[4] - a[1] * a[3]) / d;
  *det = d;
}

double host_min_image(const GGeom &g, const double *pos, int I, int J, double limit) {
  double d0[3], u[3];
  for (int d = 0; d < 3; ++d) d0[d] = pos[3 * J + d] - pos[3 * I + d];
  for (int d = 0; d < 3; ++d) u[d] = d0[0] * g.inv[d] + d0[1] * g.inv[3 + d] + d0[2] * g.inv[6 + d];
  double best = 1e300;
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = (int)std::ceil(-u[d] - limit * g.reach[d]);
    hi[d] = (int)std::floor(-u[d] + limit * g.reach[d]);
  }
  for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
    for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
      for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
        double x[3];
        for (int d = 0; d < 3; ++d) x[d] = d0[d] + n0 * g.cell[d] + n1 * g.cell[3 + d] + n2 * g.cell[6 + d];
        best = std::min(best, std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
      }
  return best;
}

int validate(const gint_desc *d) {
  if (!d || d->natoms < 1 || !d->pos || !d->species || d->nspecies < 1 || d->nspecies > GINT_MAX_SPECIES || !d->sp)
    return GINT_EINVAL;
  if (d->n1 < 1 || d->n2 < 1 || d->n3 < 1 || !(d->skin >= 0)) return GINT_EINVAL;
  int nrad = 0;
  for (int s = 0; s < d->nspecies; ++s) {
    const gint_species &S = d->sp[s];
    if (S.nradial < 1 || S.nradial > 16 || !S.radial) return GINT_EINVAL;
    int norb = 0;
    for (int k = 0; k < S.nradial; ++k) {
      const gint_radial &R = S.radial[k];
      if (R.l < 0 || R.l > 2 || R.npts < 2 || !(R.dr > 0) || !(R.rc > 0) || !R.f || !R.df) return GINT_EINVAL;
      if (R.rc > (R.npts - 1) * R.dr * (1 + 1e-12)) return GINT_EINVAL;
      norb += 2 * R.l + 1;
    }
    if (norb > GINT_MAX_ORB_ATOM) return GINT_EINVAL;
    nrad += S.nradial;
  }
  if (nrad > GINT_MAX_RADIAL) return GINT_EINVAL;
  for (int a = 0; a < d->natoms; ++a) {
    if (d->species[a] < 0 || d->species[a] >= d->nspecies) return GINT_EINVAL;
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(d->pos[3 * a + c])) return GINT_EINVAL;
  }
  double inv[9], det;
  inverse3(d->cell, inv, &det);
  if (!(std::fabs(det) > 1e-12) || !std::isfinite(det)) return GINT_EINVAL;
  return GINT_OK;
}

#define TRY(x)              \
  do {                      \
    int rc_ = (x);          \
    if (rc_) {              \
      free_all(h);          \
      delete h;             \
      return rc_;           \
    }                       \
  } while (0)
#define TRYCU(x) TRY((x) == cudaSuccess ? GINT_OK : GINT_ECUDA)

}  // namespace

int gint_reserve_nbr(gint_handle *h) {
  if (h->nslots + 1 > h->cap_slots) {
    dfree(h->s_atom); dfree(h->s_col); dfree(h->s_ent);
    long long cap = h->nslots + h->nslots / 4 + 64;
    if (dalloc(&h->s_atom, cap) || dalloc(&h->s_col, cap) || dalloc(&h->s_ent, cap + 1)) return GINT_ENOMEM;
    h->cap_slots = cap;
  }
  if (h->nent > h->cap_ent) {
    dfree(h->e_shift);
    long long cap = h->nent + h->nent / 4 + 64;
    if (dalloc(&h->e_shift, 3 * cap)) return GINT_ENOMEM;
    h->cap_ent = cap;
  }
  if (h->npairtab > h->cap_pairtab) {
    dfree(h->b_pair);
    long long cap = h->npairtab + h->npairtab / 4 + 64;
    if (dalloc(&h->b_pair, cap)) return GINT_ENOMEM;
    h->cap_pairtab = cap;
  }
  return GINT_OK;
}

namespace {

// The handle's set-up; `unfold` gives every (atom, image) entry of a brick a slot of its own.
int create_impl(const gint_desc *d, bool unfold, gint_handle **out) {
  if (!out) return GINT_EINVAL;
  *out = nullptr;
  int v = validate(d);
  if (v) return v;
  gint_handle *h = new (std::nothrow) gint_handle();
  if (!h) return GINT_ENOMEM;
  h->unfold = unfold;
  std::memset(static_cast<void *>(&h->geom), 0, sizeof(GGeom));  // batched launches compare GTabs bytes
  // host copy of the descriptor's species (an unfolded twin is built from it on demand)
  {
    int nr = 0;
    for (int s = 0; s < d->nspecies; ++s) nr += d->sp[s].nradial;
    h->d_sp.assign(d->sp, d->sp + d->nspecies);
    h->d_rad.resize(nr);
    h->d_tab.resize(2 * (size_t)nr);
    h->d_skin = d->skin;
    h->d_pos0.assign(d->pos, d->pos + 3 * (size_t)d->natoms);
    int r = 0;
    for (int s = 0; s < d->nspecies; ++s) {
      h->d_sp[s].radial = h->d_rad.data() + r;
      for (int k = 0; k < d->sp[s].nradial; ++k, ++r) {
        const gint_radial &R = d->sp[s].radial[k];
        h->d_tab[2 * r].assign(R.f, R.f + R.npts);
        h->d_tab[2 * r + 1].assign(R.df, R.df + R.npts);
        h->d_rad[r] = R;
        h->d_rad[r].f = h->d_tab[2 * r].data();
        h->d_rad[r].df = h->d_tab[2 * r + 1].data();
      }
    }
  }
  TRYCU(cudaGetDevice(&h->device));
  TRYCU(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
  cudaStream_t st = h->own_stream;
  GGeom &g = h->geom;
  std::memcpy(g.cell, d->cell, sizeof(g.cell));
  double det;
  inverse3(g.cell, g.inv, &det);
  for (int c = 0; c < 3; ++c)
    g.reach[c] = std::sqrt(g.inv[c] * g.inv[c] + g.inv[3 + c] * g.inv[3 + c] + g.inv[6 + c] * g.inv[6 + c]);
  g.n1 = d->n1; g.n2 = d->n2; g.n3 = d->n3;
  g.ngrid = (long long)d->n1 * d->n2 * d->n3;
  g.w = std::fabs(det) / (double)g.ngrid;
  g.nbi = (d->n1 + GINT_BI - 1) / GINT_BI;
  g.nbj = (d->n2 + GINT_BJ - 1) / GINT_BJ;
  g.nbk = (d->n3 + GINT_BK - 1) / GINT_BK;
  g.nbricks = (long long)g.nbi * g.nbj * g.nbk;
  if (g.nbricks >= (1LL << 31)) TRY(GINT_ECAPACITY);  // brick indices are 32-bit in the kernels
  g.natoms = d->natoms;
  g.nspecies = d->nspecies;
  // radial tables
  std::vector<double2> t64;
  int r = 0;
  for (int s = 0; s < d->nspecies; ++s) {
    const gint_species &S = d->sp[s];
    GSpecies &GS = g.sp[s];
    GS.nrad = S.nradial;
    GS.rad0 = r;
    GS.norb = 0;
    GS.rcut = 0;
    for (int k = 0; k < S.nradial; ++k, ++r) {
      const gint_radial &R = S.radial[k];
      GRadial &GR = g.rad[r];
      GR.l = R.l;
      GR.npts = R.npts;
      GR.off = (int)t64.size();
      GR.dr = R.dr;
      GR.inv_dr = 1.0 / R.dr;
      GR.rc = R.rc;
      GR.rc2 = R.rc * R.rc;
      GR.idr_hi = (float)GR.inv_dr;
      GR.idr_lo = (float)(GR.inv_dr - (double)GR.idr_hi);
      GR.rc_f = (float)R.rc;
      GR.dr_f = (float)R.dr;
      for (int i = 0; i < R.npts; ++i) t64.push_back(make_double2(R.f[i], R.df[i]));
      GS.norb += 2 * R.l + 1;
      GS.rcut = std::max(GS.rcut, R.rc);
    }
    GS.rcut2 = GS.rcut * GS.rcut;
    GS.rcut2f = (float)GS.rcut2;
    GS.porb = (GS.norb + 7) / 8 * 8;
    {
      int cnt[3] = {0, 0, 0};
      bool sorted = true, same = true;
      for (int k = 0; k < S.nradial; ++k) {
        const gint_radial &R = S.radial[k];
        cnt[R.l]++;
        if (k > 0 && R.l < S.radial[k - 1].l) sorted = false;
        if (R.npts != S.radial[0].npts || R.dr != S.radial[0].dr) same = false;
      }
      GS.shape = (sorted && same && cnt[0] < 8 && cnt[1] < 8 && cnt[2] < 8) ? GINT_SHAPE(cnt[0], cnt[1], cnt[2]) : 0;
    }
    h->max_species_norb = std::max(h->max_species_norb, GS.norb);
    double fmax = 0;
    for (int k = 0; k < S.nradial; ++k)
      for (int i = 0; i < S.radial[k].npts; ++i) fmax = std::max(fmax, std::fabs(S.radial[k].f[i]));
    h->phi_bound = std::max(h->phi_bound, fmax * 1.1);
  }
  g.nrad = r;
  h->nknots = (long long)t64.size();
  std::vector<float2> t32(t64.size());
  for (size_t i = 0; i < t64.size(); ++i) t32[i] = make_float2((float)t64[i].x, (float)t64[i].y);
  std::vector<float> d32(t64.size(), 0.f);  // knot differences in float64, rounded once
  for (int k = 0; k < r; ++k)
    for (int i = 0; i + 1 < g.rad[k].npts; ++i) {
      const long long o = g.rad[k].off + i;
      d32[o] = (float)(t64[o + 1].x - t64[o].x);
    }
  // shaped species (radials on one knot grid): (f, f') of all radials at a knot side by side, so a
  // knot pair is a few 16-byte loads in the orbital kernels
  std::vector<float2> t32i;
  std::vector<float> d32i;
  for (int s = 0; s < d->nspecies; ++s) {
    GSpecies &GS = g.sp[s];
    GS.ioff = GS.kslot = 0;
    if (!GS.shape) continue;
    GS.kslot = (GS.nrad + 1) & ~1;
    if (t32i.size() & 1) {
      t32i.push_back(make_float2(0.f, 0.f));
      d32i.push_back(0.f);
    }
    GS.ioff = (int)t32i.size();
    const int npts = g.rad[GS.rad0].npts;
    for (int i = 0; i < npts; ++i)
      for (int k = 0; k < GS.kslot; ++k) {
        t32i.push_back(k < GS.nrad ? t32[g.rad[GS.rad0 + k].off + i] : make_float2(0.f, 0.f));
        d32i.push_back(k < GS.nrad ? d32[g.rad[GS.rad0 + k].off + i] : 0.f);
      }
  }
  if (t32i.empty()) {
    t32i.push_back(make_float2(0.f, 0.f));
    d32i.push_back(0.f);
  }
  h->nknots_i = (long long)t32i.size();
  TRY(dalloc(&h->tab64, t64.size()));
  TRY(dalloc(&h->tab32, t32.size()));
  TRY(dalloc(&h->tab32i, t32i.size()));
  TRYCU(cudaMemcpy(h->tab32i, t32i.data(), t32i.size() * sizeof(float2), cudaMemcpyHostToDevice));
  TRYCU(cudaMemcpy(h->tab64, t64.data(), t64.size() * sizeof(double2), cudaMemcpyHostToDevice));
  TRYCU(cudaMemcpy(h->tab32, t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice));
  TRY(dalloc(&h->dtab32, d32.size()));
  TRY(dalloc(&h->dtab32i, d32i.size()));
  TRYCU(cudaMemcpy(h->dtab32, d32.data(), d32.size() * sizeof(float), cudaMemcpyHostToDevice));
  TRYCU(cudaMemcpy(h->dtab32i, d32i.data(), d32i.size() * sizeof(float), cudaMemcpyHostToDevice));
  // atoms
  h->pos_host.assign(d->pos, d->pos + 3 * (size_t)d->natoms);
  h->species_host.assign(d->species, d->species + d->natoms);
  h->atom_norb.resize(d->natoms);
  h->atom_off.resize(d->natoms + 1);
  h->atom_off[0] = 0;
  for (int a = 0; a < d->natoms; ++a) {
    h->atom_norb[a] = g.sp[d->species[a]].norb;
    h->atom_off[a + 1] = h->atom_off[a] + h->atom_norb[a];
  }
  h->norb = h->atom_off[d->natoms];
  TRY(dalloc(&h->pos_dev, 3 * (size_t)d->natoms));
  TRY(dalloc(&h->species_dev, (size_t)d->natoms));
  TRYCU(cudaMemcpy(h->pos_dev, h->pos_host.data(), h->pos_host.size() * sizeof(double), cudaMemcpyHostToDevice));
  TRYCU(cudaMemcpy(h->species_dev, h->species_host.data(), d->natoms * sizeof(int), cudaMemcpyHostToDevice));
  // pair set: some image of J closer to I than rcut(I) + rcut(J) + skin
  h->pair_row.assign(d->natoms + 1, 0);
  h->pair_col.clear();
  h->pair_off.assign(1, 0);
  for (int I = 0; I < d->natoms; ++I) {
    for (int J = 0; J < d->natoms; ++J) {
      double lim = g.sp[d->species[I]].rcut + g.sp[d->species[J]].rcut;
      if (host_min_image(g, d->pos, I, J, lim + d->skin) < lim + d->skin) {
        h->pair_col.push_back(J);
        h->pair_off.push_back(h->pair_off.back() + (long long)h->atom_norb[I] * h->atom_norb[J]);
      }
    }
    h->pair_row[I + 1] = (int)h->pair_col.size();
  }
  h->npairs = (int)h->pair_col.size();
  h->nblock = h->pair_off.back();
  std::vector<int> pairT(h->npairs);
  for (int I = 0; I < d->natoms; ++I)
    for (int p = h->pair_row[I]; p < h->pair_row[I + 1]; ++p) {
      int J = h->pair_col[p];
      auto b = h->pair_col.begin() + h->pair_row[J], e = h->pair_col.begin() + h->pair_row[J + 1];
      auto it = std::lower_bound(b, e, I);
      pairT[p] = (it != e && *it == I) ? (int)(it - h->pair_col.begin()) : -1;
      if (pairT[p] < 0) TRY(GINT_EINVAL);  // the relation is symmetric by construction
    }
  TRY(dalloc(&h->pair_row_dev, h->pair_row.size()));
  TRY(dalloc(&h->pair_col_dev, h->pair_col.size()));
  TRY(dalloc(&h->pair_off_dev, h->pair_off.size()));
  TRY(dalloc(&h->pair_T_dev, pairT.size()));
  std::vector<int> pairI(h->npairs);
  for (int I = 0; I < d->natoms; ++I)
    for (int p = h->pair_row[I]; p < h->pair_row[I + 1]; ++p) pairI[p] = I;
  TRY(dalloc(&h->pair_I_dev, pairI.size()));
  TRYCU(cudaMemcpy(h->pair_I_dev, pairI.data(), pairI.size() * sizeof(int), cudaMemcpyHostToDevice));
  TRYCU(cudaMemcpy(h->pair_row_dev, h->pair_row.data(), h->pair_row.size() * sizeof(int), cudaMemcpyHostToDevice));
  TRYCU(cudaMemcpy(h->pair_col_dev, h->pair_col.data(), h->pair_col.size() * sizeof(int), cudaMemcpyHostToDevice));
  TRYCU(cudaMemcpy(h->pair_off_dev, h->pair_off.data(), h->pair_off.size() * sizeof(long long),
                   cudaMemcpyHostToDevice));
  TRYCU(cudaMemcpy(h->pair_T_dev, pairT.data(), pairT.size() * sizeof(int), cudaMemcpyHostToDevice));
  // neighbour structure
  const size_t nb = (size_t)g.nbricks;
  TRY(dalloc(&h->n_at, nb)); TRY(dalloc(&h->n_ent, nb)); TRY(dalloc(&h->n_orb, nb));
  TRY(dalloc(&h->b_at_off, nb + 1)); TRY(dalloc(&h->b_ent_off, nb + 1)); TRY(dalloc(&h->b_pair_off, nb + 1));
  TRY(dalloc(&h->scan_out, 8));
  TRY(dalloc(&h->red, 1024));
  TRY(dalloc(&h->scal, 16));
  TRY(dalloc(&h->err_word, 4));
  TRY(gint_build_neighbours(h, st));
  // workspace
  TRY(dalloc(&h->D32, (size_t)h->nblock));
  TRY(dalloc(&h->work_ctr, 4));
  TRYCU(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  TRYCU(cudaMemset(h->err_word, 0, sizeof(unsigned)));
  TRY(gint_tc_prepare(h));
  TRYCU(cudaStreamSynchronize(st));
  *out = h;
  return GINT_OK;
}

// The unfolded twin of h: the creation-time descriptor (so the pair set and block layout are h's),
// moved to h's current positions.
int make_twin(gint_handle *h) {
  if (h->twin) return GINT_OK;
  gint_desc d{};
  std::memcpy(d.cell, h->geom.cell, sizeof(d.cell));
  d.natoms = h->geom.natoms;
  d.pos = h->d_pos0.data();
  d.species = h->species_host.data();
  d.nspecies = h->geom.nspecies;
  d.sp = h->d_sp.data();
  d.n1 = h->geom.n1;
  d.n2 = h->geom.n2;
  d.n3 = h->geom.n3;
  d.skin = h->d_skin;
  gint_handle *t = nullptr;
  int rc = create_impl(&d, true, &t);
  if (rc) return rc;
  if (h->pos_host != h->d_pos0) {
    rc = gint_set_positions(t, h->pos_dev, h->own_stream);
    if (rc) {
      gint_destroy(t);
      return rc;
    }
  }
  if (t->nblock != h->nblock || t->npairs != h->npairs) {
    gint_destroy(t);
    return GINT_EDEVICE;
  }
  t->reduce_fp64 = h->reduce_fp64;
  h->twin = t;
  return GINT_OK;
}

// The handle whose local-H tiles give H(R), with its key tables built: h itself, or, when some
// brick of h sees two images of one atom (its tiles mix several R), h's unfolded twin.
int hr_handle(gint_handle *h, gint_handle **t) {
  *t = h;
  if (h->folded && !h->unfold) {
    const int rc = make_twin(h);
    if (rc) return rc;
    *t = h->twin;
  }
  return gint_hr_prepare(*t);
}

}  // namespace

extern "C" {

int gint_create(const gint_desc *d, gint_handle **out) { return create_impl(d, false, out); }

int gint_destroy(gint_handle *h) {
  if (!h) return GINT_OK;
  DeviceGuard guard(h->device);
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return GINT_OK;
}

int gint_layout(const gint_handle *h, int *norb, int *npairs, long long *nblock_elems) {
  if (!h) return GINT_EINVAL;
  if (norb) *norb = h->norb;
  if (npairs) *npairs = h->npairs;
  if (nblock_elems) *nblock_elems = h->nblock;
  return GINT_OK;
}

int gint_pairs(const gint_handle *h, int *pair_IJ, long long *pair_off) {
  if (!h) return GINT_EINVAL;
  if (pair_IJ) {
    for (int I = 0; I < h->geom.natoms; ++I)
      for (int p = h->pair_row[I]; p < h->pair_row[I + 1]; ++p) {
        pair_IJ[2 * p] = I;
        pair_IJ[2 * p + 1] = h->pair_col[p];
      }
  }
  if (pair_off) std::memcpy(pair_off, h->pair_off.data(), h->pair_off.size() * sizeof(long long));
  return GINT_OK;
}

int gint_stats(const gint_handle *h, double *W, double *W_exec, long long *nbricks, int *max_brick_orb,
               int *max_brick_atoms) {
  if (!h) return GINT_EINVAL;
  if (W) *W = h->W;
  if (W_exec) *W_exec = h->W_exec;
  if (nbricks) *nbricks = h->geom.nbricks;
  if (max_brick_orb) *max_brick_orb = h->max_brick_orb;
  if (max_brick_atoms) *max_brick_atoms = h->max_brick_atoms;
  return GINT_OK;
}

int gint_brick_lists(const gint_handle *h, long long *nslots, long long *nentries, long long *b_off, int *slot_atom,
                     long long *slot_ent, double *ent_pos) {
  if (!h) return GINT_EINVAL;
  long long ns = h->nslots, ne = 0;
  if (cudaMemcpy(&ne, h->s_ent + ns, sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) return GINT_ECUDA;
  if (nslots) *nslots = ns;
  if (nentries) *nentries = ne;
  const long long nb = h->geom.nbricks;
  if ((b_off && cudaMemcpy(b_off, h->b_at_off, (nb + 1) * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (slot_atom && ns && cudaMemcpy(slot_atom, h->s_atom, ns * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (slot_ent && cudaMemcpy(slot_ent, h->s_ent, (ns + 1) * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (ent_pos && ne && cudaMemcpy(ent_pos, h->e_shift, 3 * ne * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess))
    return GINT_ECUDA;
  return GINT_OK;
}

int gint_memory(const gint_handle *h, long long *device_bytes) {
  if (!h || !device_bytes) return GINT_EINVAL;
  const long long nb = h->geom.nbricks, na = h->geom.natoms, np = h->npairs, L = sizeof(long long);
  long long b = h->nknots * (long long)(sizeof(double2) + sizeof(float2) + sizeof(float)) + h->nknots_i * 12;  // tables
  b += na * (3 * (long long)sizeof(double) + 4);                                            // atoms
  b += (na + 1) * 4 + np * 4 + (np + 1) * L + 2 * np * 4;                                  // pair set
  b += nb * 3 * 4 + (nb + 1) * 3 * L + 8 * L;                                               // brick counts
  b += h->cap_slots * 8 + (h->cap_slots + 1) * L + h->cap_ent * 3 * (long long)sizeof(double) +
       h->cap_pairtab * 4;                                                                  // neighbours
  b += 1024 * (long long)sizeof(double) + 16 * (long long)sizeof(double) + 16 + h->nblock * 4 + 16;  // workspace
  long long twin = 0;
  if (h->twin) gint_memory(h->twin, &twin);
  *device_bytes = b + h->tc_bytes + h->r_bytes + h->pb_bytes + twin;
  return GINT_OK;
}

int gint_set_positions(gint_handle *h, const double *pos_dev, void *stream) {
  if (!h || !pos_dev) return GINT_EINVAL;
  DeviceGuard guard(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(h->pos_dev, pos_dev, 3 * sizeof(double) * h->geom.natoms, cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return GINT_ECUDA;
  int rc = gint_build_neighbours(h, st);
  if (rc) return rc;
  rc = gint_tc_refresh(h);
  if (rc) return rc;
  gint_hr_free(h);  // H(R) keys follow the new images (rebuilt on first use)
  if (cudaMemcpyAsync(h->pos_host.data(), h->pos_dev, 3 * sizeof(double) * h->geom.natoms, cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GINT_ECUDA;
  if (h->twin) return gint_set_positions(h->twin, pos_dev, stream);
  return GINT_OK;
}

static int check_precision(int precision) {
  return (precision == GINT_FP64 || precision == GINT_FP32 || precision == GINT_F16X3 || precision == GINT_F16X1)
             ? GINT_OK
             : GINT_EINVAL;
}

int gint_rho(gint_handle *h, int precision, const double *D_blocks, double *rho, void *stream) {
  if (!h || !D_blocks || !rho) return GINT_EINVAL;
  if (check_precision(precision)) return GINT_EINVAL;
  DeviceGuard guard(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == GINT_FP64 || precision == GINT_FP32)
    return gint_simt_rho(h, precision == GINT_FP64, D_blocks, rho, nullptr, nullptr, st);
  return gint_tc_rho(h, precision, D_blocks, rho, nullptr, nullptr, st);
}

int gint_vlocal(gint_handle *h, int precision, const double *V, double *H_blocks, void *stream) {
  if (!h || !V || !H_blocks) return GINT_EINVAL;
  if (check_precision(precision)) return GINT_EINVAL;
  DeviceGuard guard(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == GINT_FP64 || precision == GINT_FP32) {
    if (cudaMemsetAsync(H_blocks, 0, sizeof(double) * (size_t)h->nblock, st) != cudaSuccess) return GINT_ECUDA;
    return gint_simt_vlocal(h, precision == GINT_FP64, V, H_blocks, st);
  }
  return gint_tc_vlocal(h, precision, V, H_blocks, st);  // every block element is written
}

int gint_set_reduction(gint_handle *h, int mode) {
  if (!h || (mode != GINT_REDUCE_DOUBLE_FLOAT && mode != GINT_REDUCE_FP64)) return GINT_EINVAL;
  h->reduce_fp64 = mode == GINT_REDUCE_FP64;
  if (h->twin) h->twin->reduce_fp64 = h->reduce_fp64;
  return GINT_OK;
}

int gint_layout_R(gint_handle *h, int *nkeys, long long *nblock_elems, const int **keys, const long long **key_off) {
  if (!h) return GINT_EINVAL;
  DeviceGuard guard(h->device);
  gint_handle *t;
  const int rc = hr_handle(h, &t);
  if (rc) return rc;
  if (nkeys) *nkeys = t->r_nkeys;
  if (nblock_elems) *nblock_elems = t->r_nblock;
  if (keys) *keys = t->r_keys_host.data();
  if (key_off) *key_off = t->r_off_host.data();
  return GINT_OK;
}

int gint_vlocal_R(gint_handle *h, int precision, const double *V, double *H_R, void *stream) {
  if (!h || !V || !H_R) return GINT_EINVAL;
  if (check_precision(precision)) return GINT_EINVAL;
  if (precision != GINT_F16X3 && precision != GINT_F16X1) return GINT_EUNSUPPORTED;
  DeviceGuard guard(h->device);
  gint_handle *t;
  int rc = hr_handle(h, &t);
  if (rc) return rc;
  t->reduce_R = true;
  rc = gint_tc_vlocal(t, precision, V, H_R, (cudaStream_t)stream);  // every H(R) element is written
  t->reduce_R = false;
  return rc;
}

int gint_bloch(gint_handle *h, const double *H_R, int nk, const double *kfrac, double *H_k, void *stream) {
  if (!h || !H_R || !kfrac || !H_k || nk < 0) return GINT_EINVAL;
  DeviceGuard guard(h->device);
  gint_handle *t;
  const int rc = hr_handle(h, &t);
  if (rc) return rc;
  return gint_hr_bloch(t, H_R, nk, kfrac, H_k, (cudaStream_t)stream);
}

int gint_set_projectors(gint_handle *h, int nspecies, const gint_species *proj) {
  if (!h) return GINT_EINVAL;
  DeviceGuard guard(h->device);
  return gint_pb_set(h, nspecies, proj);
}

int gint_psibeta_layout(const gint_handle *h, int *npairs, long long *nelems, const int **pairs,
                        const long long **off) {
  if (!h || !h->pb_ready) return GINT_EINVAL;
  if (npairs) *npairs = h->pb_npairs;
  if (nelems) *nelems = h->pb_nelems;
  if (pairs) *pairs = h->pb_pairs_host.data();
  if (off) *off = h->pb_off_host.data();
  return GINT_OK;
}

int gint_psibeta(gint_handle *h, const double *A, double *out, void *stream) {
  if (!h || !A || !out) return GINT_EINVAL;
  DeviceGuard guard(h->device);
  return gint_pb_run(h, A, out, (cudaStream_t)stream);
}

int gint_force(gint_handle *h, int precision, const double *D_blocks, const double *V, double *F, double *rho,
               void *stream) {
  if (!h || !D_blocks || !V || !F) return GINT_EINVAL;
  if (check_precision(precision)) return GINT_EINVAL;
  DeviceGuard guard(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == GINT_FP64 || precision == GINT_FP32) {
    if (cudaMemsetAsync(F, 0, sizeof(double) * 3 * (size_t)h->geom.natoms, st) != cudaSuccess) return GINT_ECUDA;
    return gint_simt_rho(h, precision == GINT_FP64, D_blocks, rho, V, F, st);
  }
  return gint_tc_rho(h, precision, D_blocks, rho, V, F, st);  // F is zeroed by the preparation kernel
}

int gint_run_batch(const gint_task *tasks, int ntasks, int precision, void *stream) {
  return gint_run_batch_timed(tasks, ntasks, precision, stream, nullptr, nullptr);
}

int gint_run_batch_timed(const gint_task *tasks, int ntasks, int precision, void *stream, void *ev_start,
                         void *ev_stop) {
  if (ntasks < 0 || (ntasks > 0 && !tasks)) return GINT_EINVAL;
  if (check_precision(precision)) return GINT_EINVAL;
  for (int i = 0; i < ntasks; ++i) {
    const gint_task &T = tasks[i];
    if (!T.h) return GINT_EINVAL;
    if ((T.rho || T.F) && !T.D_blocks) return GINT_EINVAL;
    if ((T.H_blocks || T.F) && !T.V) return GINT_EINVAL;
  }
  if (ntasks == 0) return GINT_OK;
  DeviceGuard guard(tasks[0].h->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == GINT_F16X3 || precision == GINT_F16X1)
    return gint_tc_batch(tasks, ntasks, precision, st, (cudaEvent_t)ev_start, (cudaEvent_t)ev_stop);
  if (ev_start && cudaEventRecord((cudaEvent_t)ev_start, st) != cudaSuccess) return GINT_ECUDA;
  for (int i = 0; i < ntasks; ++i) {
    const gint_task &T = tasks[i];
    gint_handle *h = T.h;
    if (h->device != tasks[0].h->device) return GINT_EINVAL;
    for (int j = 0; j < i; ++j)
      if (tasks[j].h == h) return GINT_EINVAL;
    const bool fp64 = precision == GINT_FP64;
    int rc = GINT_OK;
    if (T.F) {
      if (cudaMemsetAsync(T.F, 0, sizeof(double) * 3 * (size_t)h->geom.natoms, st) != cudaSuccess) return GINT_ECUDA;
      rc = gint_simt_rho(h, fp64, T.D_blocks, T.rho, T.V, T.F, st);
    } else if (T.rho) {
      rc = gint_simt_rho(h, fp64, T.D_blocks, T.rho, nullptr, nullptr, st);
    }
    if (rc) return rc;
    if (T.H_blocks) {
      if (cudaMemsetAsync(T.H_blocks, 0, sizeof(double) * (size_t)h->nblock, st) != cudaSuccess) return GINT_ECUDA;
      rc = gint_simt_vlocal(h, fp64, T.V, T.H_blocks, st);
      if (rc) return rc;
    }
  }
  if (ev_stop && cudaEventRecord((cudaEvent_t)ev_stop, st) != cudaSuccess) return GINT_ECUDA;
  return GINT_OK;
}

int gint_grid_dot(gint_handle *h, const double *V, const double *rho, double *out_dev, void *stream) {
  if (!h || !rho || !out_dev) return GINT_EINVAL;
  DeviceGuard guard(h->device);
  return gint_reduce_dot(h, rho, V, h->geom.ngrid, h->geom.w, out_dev, (cudaStream_t)stream);
}

int gint_block_dot(gint_handle *h, const double *A, const double *B, double *out_dev, void *stream) {
  if (!h || !A || !B || !out_dev) return GINT_EINVAL;
  DeviceGuard guard(h->device);
  return gint_reduce_dot(h, A, B, h->nblock, 1.0, out_dev, (cudaStream_t)stream);
}

double gint_weight(const gint_handle *h) { return h ? h->geom.w : 0.0; }

int gint_sync(gint_handle *h, void *stream) {
  if (!h) return GINT_EINVAL;
  DeviceGuard guard(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned err = 0;
  if (cudaMemcpyAsync(&err, h->err_word, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GINT_ECUDA;
  if (err) {
    if (cudaMemsetAsync(h->err_word, 0, sizeof(unsigned), st) != cudaSuccess) return GINT_ECUDA;
    cudaStreamSynchronize(st);
    if (err & GINT_ERRBIT_TIMEOUT) return GINT_ETIMEDOUT;
    if (err & GINT_ERRBIT_CAPACITY) return GINT_ECAPACITY;
    return GINT_EDEVICE;
  }
  return GINT_OK;
}

const char *gint_strerror(int code) {
  switch (code) {
    case GINT_OK: return "success";
    case GINT_EINVAL: return "invalid argument";
    case GINT_ENOMEM: return "device allocation failed";
    case GINT_ECUDA: return "CUDA runtime error";
    case GINT_ETIMEDOUT: return "bounded device wait timed out";
    case GINT_EDEVICE: return "device-side consistency check failed";
    case GINT_ECAPACITY: return "brick exceeds kernel capacity";
    case GINT_ESKIN: return "atoms moved beyond the pair-set skin";
    case GINT_EUNSUPPORTED: return "unsupported precision or feature";
    case GINT_EBUSY: return "serving queue full, or the handle has a job in flight";
    default: return "unknown error";
  }
}

}  // extern "C"
