// gint_hr.cu -- the local-potential matrix per lattice vector, H_IJ(R), and its Bloch sum
// H(k) = sum_R e^{ik.R} H(R) (paper Sec. 2, the k-space Hamiltonian; Sec. 3.3.1, the local-potential
// matrix element between phi_mu at tau_I and phi_nu at tau_J + R).
//
// The brick kernel's local-H pass writes one float32 tile per brick and pair of slots (a <= c).  A
// slot is an atom with the lattice images whose support reaches the brick; when every slot has ONE
// image, the tile of slots a, c is entirely the contribution of the image pair (tau_I + n_a A,
// tau_J + n_c A) and so belongs to H_IJ(R) with R = n_c - n_a.  These tables key the tiles by
// (I, J, R) instead of (I, J); the per-pair reduction kernel then sums them in the same fixed brick
// order into H(R) blocks.  Where some brick sees two images of one atom (a cell shorter than about
// 2 rc plus a brick) the folded tiles mix several R; such a handle computes H(R) on its unfolded
// twin, whose slots are single (atom, image) entries ordered by atom and then by lattice vector.
// There a tile of two images of one atom (slots a < c) has R = n_c - n_a > 0 in lexicographic
// order, so every tile still maps to an upper key: I < J, or I == J with R >= 0; the key (I, I, -R)
// gets the transpose.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "gint_handle.cuh"

namespace {

#define HR_CHECK(x)                   \
  do {                                \
    if ((x) != cudaSuccess) {         \
      cudaGetLastError();             \
      return GINT_ECUDA;              \
    }                                 \
  } while (0)

template <typename T>
int halloc_copy(T **dst, const std::vector<T> &src) {
  if (cudaMalloc(dst, std::max<size_t>(src.size(), 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return GINT_ENOMEM;
  }
  if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return GINT_ECUDA;
  return GINT_OK;
}

template <typename T>
void hfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// H_k (complex, interleaved re / im, Gamma-pair layout) = sum over the keys (I, J, n) of pair p of
// e^{2 pi i kf.n} H_R[key], for up to kMaxK k points at once (each H(R) element is read once for all
// of them): one CTA per pair, the phases of up to 32 keys at a time in shared memory.
constexpr int kMaxK = 8;
struct GKpts {
  int nk;
  double kf[kMaxK][3];
};
__global__ void __launch_bounds__(128) k_bloch(const long long *__restrict__ pair_off, const int *__restrict__ gk_off,
                                               const int *__restrict__ kn, const long long *__restrict__ koff,
                                               const double *__restrict__ HR, const __grid_constant__ GKpts K,
                                               long long nblock, double *__restrict__ Hk) {
  __shared__ double cs[32][kMaxK], sn[32][kMaxK];
  const int p = blockIdx.x, nk = K.nk;
  const long long o = pair_off[p], blk = pair_off[p + 1] - o;
  const int q0 = gk_off[p], q1 = gk_off[p + 1];
  for (long long e0 = 0; e0 < blk; e0 += blockDim.x) {
    const long long e = e0 + threadIdx.x;
    double re[kMaxK], im[kMaxK];
#pragma unroll
    for (int j = 0; j < kMaxK; ++j) re[j] = im[j] = 0.0;
    for (int qb = q0; qb < q1; qb += 32) {
      const int nq = min(32, q1 - qb);
      __syncthreads();
      for (int u = threadIdx.x; u < nq * nk; u += blockDim.x) {
        const int i = u / nk, j = u - i * nk, q = qb + i;
        // k.R = 2 pi (kf . n) for R = n1 a1 + n2 a2 + n3 a3 and k in reciprocal-lattice units
        sincospi(2.0 * (K.kf[j][0] * kn[3 * q] + K.kf[j][1] * kn[3 * q + 1] + K.kf[j][2] * kn[3 * q + 2]), &sn[i][j],
                 &cs[i][j]);
      }
      __syncthreads();
      if (e < blk)
        for (int i = 0; i < nq; ++i) {
          const double h = HR[koff[qb + i] + e];
#pragma unroll
          for (int j = 0; j < kMaxK; ++j)
            if (j < nk) {
              re[j] += cs[i][j] * h;
              im[j] += sn[i][j] * h;
            }
        }
    }
    if (e < blk)
#pragma unroll
      for (int j = 0; j < kMaxK; ++j)
        if (j < nk) {
          Hk[2 * (j * nblock + o + e)] = re[j];
          Hk[2 * (j * nblock + o + e) + 1] = im[j];
        }
  }
}

// The same sums for groups of kGP consecutive pairs per CTA (one or a few keys per pair, as in a cell
// where no brick sees two images of one atom): the phases of the group's keys (at most kGK) in shared
// memory, then one thread per element of the group's blocks (flattened), each H(R) element read once
// and every H(k) element written as one 16-byte store.  Small blocks no longer leave most of a CTA
// idle, and one CTA covers kGP pairs instead of one.
constexpr int kGP = 8, kGK = 64, kGT = 256;
__global__ void __launch_bounds__(kGT) k_bloch_grouped(int npairs, const long long *__restrict__ pair_off,
                                                      const int *__restrict__ gk_off, const int *__restrict__ kn,
                                                      const long long *__restrict__ koff, const double *__restrict__ HR,
                                                      const __grid_constant__ GKpts K, long long nblock,
                                                      double2 *__restrict__ Hk) {
  __shared__ double cs[kGK][kMaxK], sn[kGK][kMaxK];
  __shared__ long long poff[kGP + 1];
  __shared__ int qoff[kGP + 1];
  const int p0 = blockIdx.x * kGP, np = min(kGP, npairs - p0), nk = K.nk;
  if (threadIdx.x <= np) {
    poff[threadIdx.x] = pair_off[p0 + threadIdx.x];
    qoff[threadIdx.x] = gk_off[p0 + threadIdx.x];
  }
  __syncthreads();
  const int q0 = qoff[0], nq = qoff[np] - q0;  // the host checks nq <= kGK
  for (int u = threadIdx.x; u < nq * nk; u += kGT) {
    const int i = u / nk, j = u - i * nk, q = q0 + i;
    // k.R = 2 pi (kf . n) for R = n1 a1 + n2 a2 + n3 a3 and k in reciprocal-lattice units
    sincospi(2.0 * (K.kf[j][0] * kn[3 * q] + K.kf[j][1] * kn[3 * q + 1] + K.kf[j][2] * kn[3 * q + 2]), &sn[i][j],
             &cs[i][j]);
  }
  __syncthreads();
  const long long g0 = poff[0], g1 = poff[np];
  int pl = 0;  // pair (within the group) of the current element; elements advance monotonically
  for (long long g = g0 + threadIdx.x; g < g1; g += kGT) {
    while (g >= poff[pl + 1]) ++pl;
    const long long e = g - poff[pl];
    double re[kMaxK], im[kMaxK];
#pragma unroll
    for (int j = 0; j < kMaxK; ++j) re[j] = im[j] = 0.0;
    for (int q = qoff[pl]; q < qoff[pl + 1]; ++q) {
      const double h = HR[koff[q] + e];
      const int i = q - q0;
#pragma unroll
      for (int j = 0; j < kMaxK; ++j)
        if (j < nk) {
          re[j] += cs[i][j] * h;
          im[j] += sn[i][j] * h;
        }
    }
#pragma unroll
    for (int j = 0; j < kMaxK; ++j)
      if (j < nk) Hk[j * nblock + g] = make_double2(re[j], im[j]);
  }
}

}  // namespace

void gint_hr_free(gint_handle *h) {
  hfree(h->r_kI);
  hfree(h->r_kJ);
  hfree(h->r_kT);
  hfree(h->r_kn);
  hfree(h->r_koff);
  hfree(h->r_hu_key);
  hfree(h->r_hu_off);
  hfree(h->r_hu_src);
  hfree(h->r_gk_off);
  h->r_ready = false;
  h->r_status = GINT_OK;
  h->r_nkeys = h->r_nupper = 0;
  h->r_nblock = 0;
  h->r_keys_host.clear();
  h->r_off_host.clear();
}

// Key tables of the per-R reduction, built once per geometry on first use.
int gint_hr_prepare(gint_handle *h) {
  if (h->r_ready) return h->r_status;
  gint_hr_free(h);
  const GGeom &g = h->geom;
  const int na = g.natoms;
  const long long nb = g.nbricks, ns = h->nslots;
  std::vector<long long> at_off(nb + 1), s_ent(ns + 1), hs_off(nb + 1);
  std::vector<int> satom(std::max<long long>(ns, 1));
  std::vector<double> pos(3 * (size_t)na), ent(3 * std::max<long long>(h->nent, 1));
  HR_CHECK(cudaMemcpy(at_off.data(), h->b_at_off, (nb + 1) * sizeof(long long), cudaMemcpyDeviceToHost));
  HR_CHECK(cudaMemcpy(s_ent.data(), h->s_ent, (ns + 1) * sizeof(long long), cudaMemcpyDeviceToHost));
  if (ns) HR_CHECK(cudaMemcpy(satom.data(), h->s_atom, ns * sizeof(int), cudaMemcpyDeviceToHost));
  if (h->nent) HR_CHECK(cudaMemcpy(ent.data(), h->e_shift, 3 * h->nent * sizeof(double), cudaMemcpyDeviceToHost));
  HR_CHECK(cudaMemcpy(pos.data(), h->pos_dev, 3 * (size_t)na * sizeof(double), cudaMemcpyDeviceToHost));
  HR_CHECK(cudaMemcpy(hs_off.data(), h->hs_brick_off, (nb + 1) * sizeof(long long), cudaMemcpyDeviceToHost));
  // lattice vector n of each slot's single image: image position = tau_I + n A
  std::vector<std::array<int, 3>> sn(std::max<long long>(ns, 1));
  for (long long s = 0; s < ns; ++s) {
    if (s_ent[s + 1] - s_ent[s] != 1) {
      h->r_ready = true;
      h->r_status = GINT_EUNSUPPORTED;  // a brick sees two images of this atom: its tiles mix R
      return h->r_status;
    }
    const long long e = s_ent[s];
    double d[3], u[3];
    for (int c = 0; c < 3; ++c) d[c] = ent[3 * e + c] - pos[3 * satom[s] + c];
    for (int c = 0; c < 3; ++c) u[c] = d[0] * g.inv[0 * 3 + c] + d[1] * g.inv[1 * 3 + c] + d[2] * g.inv[2 * 3 + c];
    for (int c = 0; c < 3; ++c) {
      sn[s][c] = (int)std::lround(u[c]);
      if (std::fabs(u[c] - sn[s][c]) > 1e-6) return GINT_EDEVICE;  // not a lattice translate
    }
  }
  auto find_pair = [&](int I, int J) -> int {
    auto b = h->pair_col.begin() + h->pair_row[I], e = h->pair_col.begin() + h->pair_row[I + 1];
    auto it = std::lower_bound(b, e, J);
    return (it != e && *it == J) ? (int)(it - h->pair_col.begin()) : -1;
  };
  using Key = std::array<int, 5>;  // I, J, n1, n2, n3
  // contributions of the upper keys (I < J, or I == J with R = 0) in brick order
  std::map<Key, std::vector<long long>> contrib;
  std::vector<int> po;
  for (long long b = 0; b < nb; ++b) {
    const long long s0 = at_off[b], s1 = at_off[b + 1];
    po.assign(s1 - s0, 0);
    long long cum = 0;
    for (long long s = s0; s < s1; ++s) {
      po[s - s0] = g.sp[h->species_host[satom[s]]].norb;  // scratch tiles hold no padding
      cum += po[s - s0];
    }
    long long rowst = 0, cum_a = 0;
    for (long long a = 0; a < s1 - s0; ++a) {
      long long cum_c = cum_a;
      for (long long c = a; c < s1 - s0; ++c) {
        const int I = satom[s0 + a], J = satom[s0 + c];
        if (find_pair(I, J) >= 0) {
          const Key k{I, J, sn[s0 + c][0] - sn[s0 + a][0], sn[s0 + c][1] - sn[s0 + a][1], sn[s0 + c][2] - sn[s0 + a][2]};
          // slots are ordered by atom, then by lattice vector: an upper key by construction
          if (I > J || (I == J && std::array<int, 3>{k[2], k[3], k[4]} < std::array<int, 3>{0, 0, 0}))
            return GINT_EDEVICE;
          contrib[k].push_back(hs_off[b] + rowst + (long long)po[a] * (cum_c - cum_a));
        }
        cum_c += po[c];
      }
      rowst += (long long)po[a] * (cum - cum_a);
      cum_a += po[a];
    }
  }
  // all keys (the transposed (J, I, -R) of every upper key with I != J), sorted by (I, J, n)
  std::map<Key, int> index;
  for (const auto &kv : contrib) {
    const Key &k = kv.first;
    index[k] = 0;
    if (k[0] != k[1] || k[2] || k[3] || k[4]) index[Key{k[1], k[0], -k[2], -k[3], -k[4]}] = 0;
  }
  const int nk = (int)index.size();
  std::vector<int> kI(nk), kJ(nk), kT(nk), kn(3 * (size_t)nk), gk_off(h->npairs + 1, 0);
  std::vector<long long> koff(nk + 1, 0);
  {
    int q = 0;
    for (auto &kv : index) {
      kv.second = q;
      const Key &k = kv.first;
      kI[q] = k[0];
      kJ[q] = k[1];
      kn[3 * q] = k[2];
      kn[3 * q + 1] = k[3];
      kn[3 * q + 2] = k[4];
      koff[q + 1] = koff[q] + (long long)h->atom_norb[k[0]] * h->atom_norb[k[1]];
      const int p = find_pair(k[0], k[1]);
      if (p < 0) return GINT_EDEVICE;
      gk_off[p + 1]++;
      ++q;
    }
  }
  for (int p = 0; p < h->npairs; ++p) gk_off[p + 1] += gk_off[p];
  h->r_group_ok = true;  // the grouped Bloch kernel holds the phases of every group's keys
  for (int p0 = 0; p0 < h->npairs; p0 += kGP)
    if (gk_off[std::min(h->npairs, p0 + kGP)] - gk_off[p0] > kGK) h->r_group_ok = false;
  for (const auto &kv : index) {
    const Key &k = kv.first;
    kT[kv.second] = index.at(Key{k[1], k[0], -k[2], -k[3], -k[4]});
  }
  std::vector<int> hu_key;
  std::vector<long long> hu_off(1, 0), hu_src;
  for (const auto &kv : contrib) {
    hu_key.push_back(index.at(kv.first));
    hu_src.insert(hu_src.end(), kv.second.begin(), kv.second.end());
    hu_off.push_back((long long)hu_src.size());
  }
  int rc;
  if ((rc = halloc_copy(&h->r_kI, kI)) || (rc = halloc_copy(&h->r_kJ, kJ)) || (rc = halloc_copy(&h->r_kT, kT)) ||
      (rc = halloc_copy(&h->r_kn, kn)) || (rc = halloc_copy(&h->r_koff, koff)) ||
      (rc = halloc_copy(&h->r_hu_key, hu_key)) || (rc = halloc_copy(&h->r_hu_off, hu_off)) ||
      (rc = halloc_copy(&h->r_hu_src, hu_src)) || (rc = halloc_copy(&h->r_gk_off, gk_off))) {
    gint_hr_free(h);
    return rc;
  }
  h->r_nkeys = nk;
  h->r_nupper = (int)hu_key.size();
  h->r_nblock = koff[nk];
  h->r_keys_host.resize(5 * (size_t)nk);
  for (const auto &kv : index)
    for (int c = 0; c < 5; ++c) h->r_keys_host[5 * (size_t)kv.second + c] = kv.first[c];
  h->r_off_host = koff;
  h->r_bytes = (long long)(3 * nk + 3 * nk + h->npairs + 1 + hu_key.size()) * (long long)sizeof(int) +
               (long long)(koff.size() + hu_off.size() + hu_src.size()) * (long long)sizeof(long long);
  h->r_ready = true;
  h->r_status = GINT_OK;
  return GINT_OK;
}

int gint_hr_bloch(gint_handle *h, const double *HR, int nk, const double *kf, double *Hk, cudaStream_t st) {
  if (h->npairs == 0) return GINT_OK;
  for (int k0 = 0; k0 < nk; k0 += kMaxK) {
    GKpts K{};
    K.nk = std::min(kMaxK, nk - k0);
    for (int j = 0; j < K.nk; ++j)
      for (int c = 0; c < 3; ++c) K.kf[j][c] = kf[3 * (k0 + j) + c];
    if (h->r_group_ok)
      k_bloch_grouped<<<(unsigned)((h->npairs + kGP - 1) / kGP), kGT, 0, st>>>(
          h->npairs, h->pair_off_dev, h->r_gk_off, h->r_kn, h->r_koff, HR, K, h->nblock,
          reinterpret_cast<double2 *>(Hk) + (long long)k0 * h->nblock);
    else
      k_bloch<<<(unsigned)h->npairs, 128, 0, st>>>(h->pair_off_dev, h->r_gk_off, h->r_kn, h->r_koff, HR, K, h->nblock,
                                                   Hk + 2 * (long long)k0 * h->nblock);
    if (cudaGetLastError() != cudaSuccess) return GINT_ECUDA;
  }
  return GINT_OK;
}
