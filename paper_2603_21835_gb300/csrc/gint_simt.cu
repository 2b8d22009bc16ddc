// gint_simt.cu -- CUDA-core (SIMT) brick kernels in float64 and float32.
//
// Density (paper Sec. 3.3.1):   rho_g = sum_{a,c} Phi_a(g)^T D_ac Phi_c(g)
// Local Hamiltonian:            H_ac += sum_g w V_g Phi_a(g) Phi_c(g)^T   (float64 atomics)
// Local Pulay force:            F_I   = 2 sum_g w V_g sum_{mu in I} grad Phi_mu(g) (D Phi(g))_mu
// (F = -dE/dtau, E = sum_g w V rho, D symmetric; d phi(r - tau)/d tau = -grad phi.)
//
// One CTA (4 warps) owns a 32-point slab of a 4x4x8 brick (lane = point).  The warps first
// evaluate the periodised orbitals of the brick's atoms into shared memory (one atom per
// warp at a time), the slab's coverage set is then the atoms non-zero on any of its points,
// and the contraction loops only over covered atoms (this is where the per-point sparsity
// of the NAO supports is used).  On GB300 the float64 pipe is the bound for the FP64 mode.
#include <cuda_runtime.h>

#include "gint_handle.cuh"

namespace {

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;

struct SlabShared {
  int s_atom[GINT_MAX_ATOMS_BRICK];
  int s_col[GINT_MAX_ATOMS_BRICK];
  int s_no[GINT_MAX_ATOMS_BRICK];
  int s_sp[GINT_MAX_ATOMS_BRICK];
  long long s_e0[GINT_MAX_ATOMS_BRICK + 1];
  int covflag[GINT_MAX_ATOMS_BRICK];
  int cov[GINT_MAX_ATOMS_BRICK];
  int ncov;
};

// Loads the brick's slot metadata, evaluates Phi for the slab's 32 points into phi[lane][ld]
// (and chi = w V phi if CHI), and builds the coverage list.  Returns the number of slots.
template <typename T, bool CHI>
__device__ int slab_orbitals(const GGeom &g, const GNbr &nb, const typename Tab2<T>::type *__restrict__ tab,
                             const float *__restrict__ dtab, long long b, int lane, int warp, const double rp[3],
                             bool valid, T wv, T *phi, T *chi, int ld, SlabShared &sh) {
  const long long s0 = nb.b_at_off[b];
  const int na = (int)(nb.b_at_off[b + 1] - s0);
  for (int a = threadIdx.x; a < na; a += blockDim.x) {
    int I = nb.s_atom[s0 + a];
    int sp = nb.atom_species[I];
    sh.s_atom[a] = I;
    sh.s_col[a] = nb.s_col[s0 + a];
    sh.s_sp[a] = sp;
    sh.s_no[a] = g.sp[sp].norb;
    sh.s_e0[a] = nb.s_ent[s0 + a];
    if (a == na - 1) sh.s_e0[na] = nb.s_ent[s0 + na];
  }
  __syncthreads();
  T *myphi = phi + lane * ld;
  T *mychi = CHI ? chi + lane * ld : nullptr;
  for (int a = warp; a < na; a += kWarps) {
    const int col = sh.s_col[a], no = sh.s_no[a], sp = sh.s_sp[a];
    const double rc2 = g.sp[sp].rcut2;
    for (int i = 0; i < no; ++i) myphi[col + i] = 0;
    bool cov = false;
    if (valid) {
      for (long long e = sh.s_e0[a]; e < sh.s_e0[a + 1]; ++e) {
        double dx = rp[0] - nb.e_shift[3 * e], dy = rp[1] - nb.e_shift[3 * e + 1], dz = rp[2] - nb.e_shift[3 * e + 2];
        if (dx * dx + dy * dy + dz * dz < rc2) {
          cov = true;
          add_orbitals<T, true, false>(g, tab, sp, (T)dx, (T)dy, (T)dz, myphi + col, nullptr, dtab);
        }
      }
    }
    if (CHI)
      for (int i = 0; i < no; ++i) mychi[col + i] = wv * myphi[col + i];
    unsigned bal = __ballot_sync(0xffffffffu, cov);
    if (lane == 0) sh.covflag[a] = bal != 0u;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    for (int a = 0; a < na; ++a)
      if (sh.covflag[a]) sh.cov[n++] = a;
    sh.ncov = n;
  }
  __syncthreads();
  return na;
}

template <typename T, int MAXO, bool FORCE>
__global__ void __launch_bounds__(kThreads) k_simt_rho(GGeom g, GNbr nb, const typename Tab2<T>::type *__restrict__ tab,
                                                        const float *__restrict__ dtab, const T *__restrict__ D,
                                                        const double *__restrict__ V, double *__restrict__ rho,
                                                        double *__restrict__ F, int ld) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SlabShared sh;
  __shared__ double rpart[kWarps][32];
  T *phi = reinterpret_cast<T *>(smem);
  T(*gsc)[3] = reinterpret_cast<T(*)[3]>(phi + 32 * ld);  // [warp][lane][MAXO][3] (force only)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long b = blockIdx.x >> 2;
  const int p = (blockIdx.x & 3) * 32 + lane;
  int gi, gj, gk;
  const bool valid = brick_point(g, b, p, gi, gj, gk);
  double rp[3];
  grid_point(g, gi, gj, gk, rp);
  const long long gidx = valid ? grid_index(g, gi, gj, gk) : 0;
  const int na = slab_orbitals<T, false>(g, nb, tab, dtab, b, lane, warp, rp, valid, (T)0, phi, nullptr, ld, sh);
  const T *myphi = phi + lane * ld;
  const long long pbase = nb.b_pair_off[b];
  const double wv = (FORCE && valid) ? g.w * V[gidx] : 0.0;
  T racc = 0;
  for (int ia = warp; ia < sh.ncov; ia += kWarps) {
    const int a = sh.cov[ia];
    const int ca = sh.s_col[a], noa = sh.s_no[a];
    T y[MAXO];
#pragma unroll
    for (int i = 0; i < MAXO; ++i) y[i] = 0;
    for (int ic = FORCE ? 0 : ia; ic < sh.ncov; ++ic) {
      const int c = sh.cov[ic];
      const int pidx = nb.b_pair[pbase + a * na + c];
      if (pidx < 0) continue;
      const int cc = sh.s_col[c], noc = sh.s_no[c];
      const T *Db = D + nb.pair_off[pidx];
      const T fac = (FORCE || ic == ia) ? (T)1 : (T)2;
      for (int j = 0; j < noc; ++j) {
        const T pc = fac * myphi[cc + j];
#pragma unroll
        for (int i = 0; i < MAXO; ++i)
          if (i < noa) y[i] += Db[i * noc + j] * pc;
      }
    }
#pragma unroll
    for (int i = 0; i < MAXO; ++i)
      if (i < noa) racc += myphi[ca + i] * y[i];
    if (FORCE) {
      T(*gs)[3] = gsc + (warp * 32 + lane) * MAXO;
      for (int i = 0; i < noa; ++i) gs[i][0] = gs[i][1] = gs[i][2] = 0;
      const int sp = sh.s_sp[a];
      const double rc2 = g.sp[sp].rcut2;
      if (valid) {
        for (long long e = sh.s_e0[a]; e < sh.s_e0[a + 1]; ++e) {
          double dx = rp[0] - nb.e_shift[3 * e], dy = rp[1] - nb.e_shift[3 * e + 1], dz = rp[2] - nb.e_shift[3 * e + 2];
          if (dx * dx + dy * dy + dz * dz < rc2)
            add_orbitals<T, false, true>(g, tab, sp, (T)dx, (T)dy, (T)dz, nullptr, gs, dtab);
        }
      }
      T fx = 0, fy = 0, fz = 0;
#pragma unroll
      for (int i = 0; i < MAXO; ++i)
        if (i < noa) {
          fx += gs[i][0] * y[i];
          fy += gs[i][1] * y[i];
          fz += gs[i][2] * y[i];
        }
      double f3[3] = {2.0 * wv * (double)fx, 2.0 * wv * (double)fy, 2.0 * wv * (double)fz};
#pragma unroll
      for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) f3[d] += __shfl_xor_sync(0xffffffffu, f3[d], o);
      if (lane == 0) {
        const int I = sh.s_atom[a];
        atomicAdd(F + 3 * I + 0, f3[0]);
        atomicAdd(F + 3 * I + 1, f3[1]);
        atomicAdd(F + 3 * I + 2, f3[2]);
      }
    }
  }
  rpart[warp][lane] = (double)racc;
  __syncthreads();
  if (warp == 0 && valid && rho != nullptr)
    rho[gidx] = rpart[0][lane] + rpart[1][lane] + rpart[2][lane] + rpart[3][lane];
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_simt_vlocal(GGeom g, GNbr nb, const typename Tab2<T>::type *__restrict__ tab,
                                                           const float *__restrict__ dtab, const int *__restrict__ pair_T,
                                                           const double *__restrict__ V, double *__restrict__ H, int ld) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SlabShared sh;
  T *phi = reinterpret_cast<T *>(smem);
  T *chi = phi + 32 * ld;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long b = blockIdx.x >> 2;
  const int p = (blockIdx.x & 3) * 32 + lane;
  int gi, gj, gk;
  const bool valid = brick_point(g, b, p, gi, gj, gk);
  double rp[3];
  grid_point(g, gi, gj, gk, rp);
  const T wv = valid ? (T)(g.w * V[grid_index(g, gi, gj, gk)]) : (T)0;
  const int na = slab_orbitals<T, true>(g, nb, tab, dtab, b, lane, warp, rp, valid, wv, phi, chi, ld, sh);
  const long long pbase = nb.b_pair_off[b];
  const int nc = sh.ncov;
  int k = 0;
  for (int ia = 0; ia < nc; ++ia) {
    for (int ic = ia; ic < nc; ++ic, ++k) {
      if ((k % kWarps) != warp) continue;
      const int a = sh.cov[ia], c = sh.cov[ic];
      const int pidx = nb.b_pair[pbase + a * na + c];
      if (pidx < 0) continue;
      const int ca = sh.s_col[a], noa = sh.s_no[a], cc = sh.s_col[c], noc = sh.s_no[c];
      double *Hb = H + nb.pair_off[pidx];
      double *HbT = (ia != ic) ? H + nb.pair_off[pair_T[pidx]] : nullptr;
      for (int e = lane; e < noa * noc; e += 32) {
        const int i = e / noc, j = e - (e / noc) * noc;
        T acc = 0;
#pragma unroll 8
        for (int q = 0; q < 32; ++q) acc += chi[q * ld + ca + i] * phi[q * ld + cc + j];
        atomicAdd(Hb + i * noc + j, (double)acc);
        if (HbT) atomicAdd(HbT + j * noa + i, (double)acc);
      }
    }
  }
}

__global__ void k_to_f32(const double *__restrict__ a, float *__restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// out = scale * sum_i a_i b_i (b == NULL: sum_i a_i), float64, two-level reduction.
__global__ void k_dot_partial(const double *__restrict__ a, const double *__restrict__ b, long long n,
                              double *__restrict__ part) {
  double acc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += b ? a[i] * b[i] : a[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
  }
}

__global__ void k_dot_final(const double *__restrict__ part, int n, double scale, double *__restrict__ out) {
  double acc = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[0] = scale * t;
  }
}

inline int slab_ld(const gint_handle *h) { return h->max_brick_orb | 1; }

template <typename K>
int launch_cfg(K kern, size_t smem) {
  if (smem > 227 * 1024) return GINT_ECAPACITY;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GINT_ECUDA;
  return GINT_OK;
}

}  // namespace

#define SIMT_CHECK(x)                                   \
  do {                                                  \
    if ((x) != cudaSuccess) return GINT_ECUDA;          \
  } while (0)

int gint_convert_D32(gint_handle *h, const double *D, cudaStream_t st) {
  if (h->nblock == 0) return GINT_OK;
  k_to_f32<<<1216, 256, 0, st>>>(D, h->D32, h->nblock);
  SIMT_CHECK(cudaGetLastError());
  return GINT_OK;
}

template <typename T, int MAXO>
static int run_rho(gint_handle *h, const T *D, double *rho, const double *V, double *F, cudaStream_t st) {
  const int ld = slab_ld(h);
  const unsigned grid = (unsigned)(h->geom.nbricks * 4);
  if (F) {
    size_t smem = sizeof(T) * (32 * (size_t)ld + (size_t)kWarps * 32 * MAXO * 3);
    auto kern = k_simt_rho<T, MAXO, true>;
    int rc = launch_cfg(kern, smem);
    if (rc) return rc;
    kern<<<grid, kThreads, smem, st>>>(h->geom, h->nbr(), (const typename Tab2<T>::type *)(sizeof(T) == 8 ? (void *)h->tab64 : (void *)h->tab32),
                                       sizeof(T) == 8 ? nullptr : h->dtab32, D, V, rho, F, ld);
  } else {
    size_t smem = sizeof(T) * 32 * (size_t)ld;
    auto kern = k_simt_rho<T, MAXO, false>;
    int rc = launch_cfg(kern, smem);
    if (rc) return rc;
    kern<<<grid, kThreads, smem, st>>>(h->geom, h->nbr(), (const typename Tab2<T>::type *)(sizeof(T) == 8 ? (void *)h->tab64 : (void *)h->tab32),
                                       sizeof(T) == 8 ? nullptr : h->dtab32, D, V, rho, F, ld);
  }
  SIMT_CHECK(cudaGetLastError());
  return GINT_OK;
}

int gint_simt_rho(gint_handle *h, bool fp64, const double *D, double *rho, const double *V, double *F,
                  cudaStream_t st) {
  if (h->geom.nbricks == 0) return GINT_OK;
  const bool big = h->max_species_norb > 16;
  if (fp64) return big ? run_rho<double, 32>(h, D, rho, V, F, st) : run_rho<double, 16>(h, D, rho, V, F, st);
  int rc = gint_convert_D32(h, D, st);
  if (rc) return rc;
  return big ? run_rho<float, 32>(h, h->D32, rho, V, F, st) : run_rho<float, 16>(h, h->D32, rho, V, F, st);
}

template <typename T>
static int run_vlocal(gint_handle *h, const double *V, double *H, cudaStream_t st) {
  const int ld = slab_ld(h);
  size_t smem = sizeof(T) * 2 * 32 * (size_t)ld;
  auto kern = k_simt_vlocal<T>;
  int rc = launch_cfg(kern, smem);
  if (rc) return rc;
  kern<<<(unsigned)(h->geom.nbricks * 4), kThreads, smem, st>>>(
      h->geom, h->nbr(), (const typename Tab2<T>::type *)(sizeof(T) == 8 ? (void *)h->tab64 : (void *)h->tab32),
      sizeof(T) == 8 ? nullptr : h->dtab32, h->pair_T_dev, V, H, ld);
  SIMT_CHECK(cudaGetLastError());
  return GINT_OK;
}

int gint_simt_vlocal(gint_handle *h, bool fp64, const double *V, double *H, cudaStream_t st) {
  if (h->geom.nbricks == 0) return GINT_OK;
  return fp64 ? run_vlocal<double>(h, V, H, st) : run_vlocal<float>(h, V, H, st);
}

int gint_reduce_dot(gint_handle *h, const double *a, const double *b, long long n, double scale, double *out,
                    cudaStream_t st) {
  const int nblk = 304;
  k_dot_partial<<<nblk, 256, 0, st>>>(a, b, n, h->red);
  SIMT_CHECK(cudaGetLastError());
  k_dot_final<<<1, 256, 0, st>>>(h->red, nblk, scale, out);
  SIMT_CHECK(cudaGetLastError());
  return GINT_OK;
}
