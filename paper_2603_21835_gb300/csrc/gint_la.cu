// gint_la.cu -- float64 dense linear algebra of the propagation steps around the grid passes (the
// Crank-Nicolson step and the density and energy-density matrices of paper Sec. 2): a tiled GEMM and
// the blocked L D L^T factorisation without pivoting with its triangular solves, real and complex.
//
// The GB300 runs float64 on its CUDA cores only, at about 2 fused multiply-adds per clock per SM, so
// every kernel here is bound by the float64 pipe: a 64 x 64 output tile per CTA keeps 16 independent
// accumulators per thread, far more than the pipe's latency needs, and operand traffic (a few bytes
// per thousand multiply-adds) is immaterial.  Latency-bound pieces (the 64 x 64 diagonal blocks, the
// 64-wide panel and right-hand-side substitutions) are small next to the GEMM updates.
//
// L D L^T without pivoting: the Crank-Nicolson matrix S + i dt/2 H is complex symmetric with a
// positive definite Hermitian part S, so its leading blocks are nonsingular and elimination without
// pivoting is stable for small dt (the growth stays of order 1 + dt^2 |H S^-1 H| / 4); the overlap
// S of the energy-density matrix is symmetric positive definite.  Symmetry halves the flops of a
// general LU.
#include <algorithm>

#include "gint.h"
#include "gint_la.cuh"

namespace gla {
namespace {

// scalar arithmetic for T = double and T = double2 (complex, no conjugation anywhere)
template <typename T>
struct Ar;
template <>
struct Ar<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }  // c + a b
  static __device__ __forceinline__ double fms(double a, double b, double c) { return ::fma(-a, b, c); }  // c - a b
  static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
  static __device__ __forceinline__ double scale(double a, double s) { return a * s; }
  static __device__ __forceinline__ double axpby(double a, double x, double b, double y) { return a * x + b * y; }
  static __device__ __forceinline__ double inv(double d) { return 1.0 / d; }
  static __device__ __forceinline__ bool bad_pivot(double d, bool spd) { return spd ? !(d > 0.0) : !(d != 0.0 && isfinite(d)); }
};
template <>
struct Ar<double2> {
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ double2 fma(double2 a, double2 b, double2 c) {
    return make_double2(::fma(-a.y, b.y, ::fma(a.x, b.x, c.x)), ::fma(a.y, b.x, ::fma(a.x, b.y, c.y)));
  }
  static __device__ __forceinline__ double2 fms(double2 a, double2 b, double2 c) {
    return make_double2(::fma(a.y, b.y, ::fma(-a.x, b.x, c.x)), ::fma(-a.y, b.x, ::fma(-a.x, b.y, c.y)));
  }
  static __device__ __forceinline__ double2 mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
  }
  static __device__ __forceinline__ double2 scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
  static __device__ __forceinline__ double2 axpby(double a, double2 x, double b, double2 y) {
    return make_double2(a * x.x + b * y.x, a * x.y + b * y.y);
  }
  // 1 / d = conj(d) / |d|^2
  static __device__ __forceinline__ double2 inv(double2 d) {
    const double q = 1.0 / (d.x * d.x + d.y * d.y);
    return make_double2(d.x * q, -d.y * q);
  }
  static __device__ __forceinline__ bool bad_pivot(double2 d, bool) {
    const double m = d.x * d.x + d.y * d.y;
    return !(m > 0.0 && isfinite(m));
  }
};

template <typename T>
__device__ __forceinline__ T vat(const View<T> &v, int r, int k) {
  T x = v.p[(long long)r * v.sr + (long long)(k >> 1) * v.skh + (long long)(k & 1) * v.skl];
  if (v.ks) x = Ar<T>::scale(x, v.ks[k >> 1]);
  return x;
}

// ---------------------------------------------------------------------------------------- GEMM
constexpr int kBM = 64, kGT = 256;
template <typename T>
struct GemmK {
  static constexpr int BK = 16;
};
template <>
struct GemmK<double2> {
  static constexpr int BK = 8;
};

// One CTA per 64 x 64 tile of C; thread (tx, ty) of 16 x 16 owns rows tx + 16 a and columns
// ty + 16 b (a, b < 4), so a warp reads 16 consecutive elements of each shared operand row.  The
// next K slab is loaded into registers while the current one is multiplied.
template <typename T, int MODE>
__global__ void __launch_bounds__(kGT, 2) k_gemm(int M, int N, int K, double alpha, View<T> A, View<T> B, double beta,
                                              T *__restrict__ C, long long cr, long long cc) {
  constexpr int BK = GemmK<T>::BK, NL = BK * kBM / kGT;
  const int tm = blockIdx.x, tn = blockIdx.y;
  if (MODE != 0 && tm < tn) return;
  __shared__ T As[BK][kBM], Bs[BK][kBM];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = tm * kBM, n0 = tn * kBM;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Ar<T>::zero();
  T ra[NL], rb[NL];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = tid + kGT * q, r = e & (kBM - 1), k = k0 + e / kBM;
      ra[q] = (m0 + r < M && k < K) ? vat(A, m0 + r, k) : Ar<T>::zero();
      rb[q] = (n0 + r < N && k < K) ? vat(B, n0 + r, k) : Ar<T>::zero();
    }
  };
  load(0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    __syncthreads();  // the previous slab's reads are done
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = tid + kGT * q;
      As[e / kBM][e & (kBM - 1)] = ra[q];
      Bs[e / kBM][e & (kBM - 1)] = rb[q];
    }
    __syncthreads();
    if (k0 + BK < K) load(k0 + BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[k][tx + 16 * i];
        b[i] = Bs[k][ty + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = Ar<T>::fma(a[i], b[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + tx + 16 * i, gn = n0 + ty + 16 * j;
      if (gm >= M || gn >= N || (MODE != 0 && gm < gn)) continue;
      T *c = C + (long long)gm * cr + (long long)gn * cc;
      const T v = beta == 0.0 ? Ar<T>::scale(acc[i][j], alpha) : Ar<T>::axpby(alpha, acc[i][j], beta, *c);
      *c = v;
      if (MODE == 2 && gm != gn) C[(long long)gn * cr + (long long)gm * cc] = v;
    }
}

// ------------------------------------------------------------------------ L D L^T, diagonal block
constexpr int kNB = 64;  // block width of the factorisation and of the solves

// One CTA factors the nb x nb diagonal block in shared memory (column-major, leading dimension
// nb + 1), right-looking: at step j, l_kj = a_kj / d_j, then a_ik -= a_ij l_kj for i >= k > j.
template <typename T>
__global__ void __launch_bounds__(kGT) k_ldl_diag(int nb, T *__restrict__ A, long long lda, int j0, int spd,
                                                  int *__restrict__ info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *s = reinterpret_cast<T *>(smem_raw);
  const int LS = nb + 1;
  T *lcol = s + nb * LS;
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += kGT) {
    const int i = e % nb, j = e / nb;
    if (i >= j) s[i + j * LS] = A[i + j * lda];
  }
  bool bad = false;
  for (int j = 0; j < nb; ++j) {
    __syncthreads();
    const T d = s[j + j * LS];
    if (tid == 0 && !bad && Ar<T>::bad_pivot(d, spd)) {
      bad = true;
      atomicCAS(info, 0, j0 + j + 1);
    }
    const T dinv = Ar<T>::inv(d);
    for (int k = j + 1 + tid; k < nb; k += kGT) lcol[k] = Ar<T>::mul(s[k + j * LS], dinv);
    __syncthreads();
    const int m = nb - 1 - j;
    for (int e = tid; e < m * m; e += kGT) {
      const int i = j + 1 + e % m, k = j + 1 + e / m;
      if (i >= k) s[i + k * LS] = Ar<T>::fms(s[i + j * LS], lcol[k], s[i + k * LS]);
    }
    __syncthreads();
    for (int k = j + 1 + tid; k < nb; k += kGT) s[k + j * LS] = lcol[k];
  }
  __syncthreads();
  for (int e = tid; e < nb * nb; e += kGT) {
    const int i = e % nb, j = e / nb;
    if (i >= j) A[i + j * lda] = s[i + j * LS];
  }
}

// ------------------------------------------------------------- unit-triangular multi-vector solves
// Vectors v < nv, element j < nb at X[v vs + j es]; the nb x nb block L (element (i, j) at
// L[i + j ldl]) in shared memory:
//   TRANS = false: L y = x (unit lower; forward), TRANS = true: L^T y = x (backward).
// PANEL (forward only): the panel of the factorisation, W = y (work, element (v, j) at W[v + j ldw])
// and x = y / d_j (d_j = the factor's diagonal, L[j + j ldl]).
// A CTA takes kSV vectors with one thread per (element, vector) and eliminates column by column (at
// step j, y_j is final and every later element subtracts its multiple): the float64 work of a block
// is spread over many CTAs and all four schedulers of an SM, where one thread per vector would leave
// most of the GPU's float64 units idle (a float64 warp instruction occupies a scheduler's unit for
// many cycles).
constexpr int kSV = 8;                 // vectors per CTA
constexpr int kSVT = kSV * 64;         // threads: (element < 64) x (vector < kSV)
template <typename T, bool TRANS, bool PANEL>
__global__ void __launch_bounds__(kSVT) k_trsv(int nb, const T *__restrict__ L, long long ldl, int nv, T *__restrict__ X,
                                               long long vs, long long es, T *__restrict__ W, long long ldw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Ls = reinterpret_cast<T *>(smem_raw);  // nb x nb: Ls[i + j nb] = L(i, j), or L(j, i) for TRANS
  T *xs = Ls + nb * nb;                     // [vector][element]
  const int tid = threadIdx.x, i = tid & 63, vl = tid >> 6, v = blockIdx.x * kSV + vl;
  for (int e = tid; e < nb * nb; e += kSVT) {
    const int r = e % nb, c = e / nb;
    Ls[e] = TRANS ? L[c + (long long)r * ldl] : L[r + (long long)c * ldl];
  }
  const bool act = v < nv && i < nb;
  T *x = X + (long long)(v < nv ? v : 0) * vs;
  T xi = act ? x[(long long)i * es] : Ar<T>::zero();
  xs[vl * 64 + i] = xi;
  // step j reads element j (final after the previous step's barrier) and writes elements != j only
  if (!TRANS) {
    for (int j = 0; j + 1 < nb; ++j) {
      __syncthreads();
      const T yj = xs[vl * 64 + j];
      if (i > j && i < nb) {
        xi = Ar<T>::fms(Ls[i + j * nb], yj, xi);
        xs[vl * 64 + i] = xi;
      }
    }
  } else {
    for (int j = nb - 1; j > 0; --j) {
      __syncthreads();
      const T yj = xs[vl * 64 + j];
      if (i < j) {
        xi = Ar<T>::fms(Ls[i + j * nb], yj, xi);
        xs[vl * 64 + i] = xi;
      }
    }
  }
  if (!act) return;
  if (PANEL) {
    W[v + (long long)i * ldw] = xi;
    x[(long long)i * es] = Ar<T>::mul(xi, Ar<T>::inv(Ls[i + i * nb]));
  } else {
    x[(long long)i * es] = xi;
  }
}

// B[i, c] /= d_i (the factor's diagonal)
template <typename T>
__global__ void k_dscale(int n, int nrhs, const T *__restrict__ A, long long lda, T *__restrict__ B, long long ldb) {
  const long long tot = (long long)n * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n);
    const long long c = e / n;
    B[i + c * ldb] = Ar<T>::mul(B[i + c * ldb], Ar<T>::inv(A[i + (long long)i * lda]));
  }
}

template <typename F>
int set_smem(F *f, size_t bytes) {
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess
             ? GINT_OK
             : GINT_ECUDA;
}

#define LA_CHECK()                                   \
  do {                                               \
    if (cudaGetLastError() != cudaSuccess) return GINT_ECUDA; \
  } while (0)

}  // namespace

template <typename T>
int gemm(int mode, int M, int N, int K, double alpha, View<T> A, View<T> B, double beta, T *C, long long cr,
         long long cc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return GINT_OK;
  const dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + kBM - 1) / kBM));
  if (grid.y > 65535u) return GINT_EINVAL;
  if (mode == 0)
    k_gemm<T, 0><<<grid, kGT, 0, st>>>(M, N, K, alpha, A, B, beta, C, cr, cc);
  else if (mode == 1)
    k_gemm<T, 1><<<grid, kGT, 0, st>>>(M, N, K, alpha, A, B, beta, C, cr, cc);
  else
    k_gemm<T, 2><<<grid, kGT, 0, st>>>(M, N, K, alpha, A, B, beta, C, cr, cc);
  LA_CHECK();
  return GINT_OK;
}

template <typename T>
int ldl_factor(int n, T *A, long long lda, T *work, int *info, bool spd, cudaStream_t st) {
  const size_t diag_smem = (size_t)(kNB * (kNB + 1) + kNB) * sizeof(T);
  const size_t trsv_smem = (size_t)(kNB * kNB + 64 * kSV) * sizeof(T);
  int rc;
  if ((rc = set_smem(k_ldl_diag<T>, diag_smem)) || (rc = set_smem(k_trsv<T, false, true>, trsv_smem))) return rc;
  for (int j0 = 0; j0 < n; j0 += kNB) {
    const int nb = std::min(kNB, n - j0);
    T *A11 = A + j0 + (long long)j0 * lda;
    k_ldl_diag<T><<<1, kGT, (size_t)(nb * (nb + 1) + nb) * sizeof(T), st>>>(nb, A11, lda, j0, spd ? 1 : 0, info);
    LA_CHECK();
    const int m = n - j0 - nb;
    if (m == 0) break;
    T *A21 = A11 + nb;
    // panel: W21 = A21 L11^-T, L21 = W21 D1^-1 (rows of A21 are the vectors)
    k_trsv<T, false, true><<<(unsigned)((m + kSV - 1) / kSV), kSVT, (size_t)(nb * nb + 64 * kSV) * sizeof(T), st>>>(
        nb, A11, lda, m, A21, 1, lda, work, n);
    LA_CHECK();
    // trailing update of the lower triangle: A22 -= W21 L21^T
    rc = gemm<T>(1, m, m, nb, -1.0, view<T>(work, 1, n), view<T>(A21, 1, lda), 1.0, A21 + (long long)nb * lda, 1, lda,
                 st);
    if (rc) return rc;
  }
  return GINT_OK;
}

template <typename T>
int ldl_solve(int n, int nrhs, const T *A, long long lda, T *B, long long ldb, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return GINT_OK;
  const size_t trsv_smem = (size_t)(kNB * kNB + 64 * kSV) * sizeof(T);
  int rc;
  if ((rc = set_smem(k_trsv<T, false, false>, trsv_smem)) || (rc = set_smem(k_trsv<T, true, false>, trsv_smem)))
    return rc;
  const unsigned nvb = (unsigned)((nrhs + kSV - 1) / kSV);
  // L Y = B, block by block: the diagonal block's substitution, then the rows below
  for (int k0 = 0; k0 < n; k0 += kNB) {
    const int nb = std::min(kNB, n - k0);
    const T *Lkk = A + k0 + (long long)k0 * lda;
    k_trsv<T, false, false><<<nvb, kSVT, (size_t)(nb * nb + 64 * kSV) * sizeof(T), st>>>(nb, Lkk, lda, nrhs, B + k0,
                                                                                        ldb, 1, nullptr, 0);
    LA_CHECK();
    const int m = n - k0 - nb;
    if (m > 0 &&
        (rc = gemm<T>(0, m, nrhs, nb, -1.0, view<T>(Lkk + nb, 1, lda), view<T>(B + k0, ldb, 1), 1.0, B + k0 + nb, 1, ldb,
                      st)))
      return rc;
  }
  // Y <- D^{-1} Y
  k_dscale<T><<<(unsigned)std::min<long long>(((long long)n * nrhs + 255) / 256, 4096), 256, 0, st>>>(n, nrhs, A, lda,
                                                                                                     B, ldb);
  LA_CHECK();
  // L^T X = Y, last block first, then the rows above
  for (int k0 = ((n - 1) / kNB) * kNB; k0 >= 0; k0 -= kNB) {
    const int nb = std::min(kNB, n - k0);
    const T *Lkk = A + k0 + (long long)k0 * lda;
    k_trsv<T, true, false><<<nvb, kSVT, (size_t)(nb * nb + 64 * kSV) * sizeof(T), st>>>(nb, Lkk, lda, nrhs, B + k0, ldb,
                                                                                       1, nullptr, 0);
    LA_CHECK();
    // rows i < k0: B_i -= sum_k L[k0 + k, i] X[k0 + k]
    if (k0 > 0 && (rc = gemm<T>(0, k0, nrhs, nb, -1.0, view<T>(A + k0, lda, 1), view<T>(B + k0, ldb, 1), 1.0, B, 1,
                                ldb, st)))
      return rc;
  }
  return GINT_OK;
}

template int gemm<double>(int, int, int, int, double, View<double>, View<double>, double, double *, long long,
                          long long, cudaStream_t);
template int gemm<double2>(int, int, int, int, double, View<double2>, View<double2>, double, double2 *, long long,
                           long long, cudaStream_t);
template int ldl_factor<double>(int, double *, long long, double *, int *, bool, cudaStream_t);
template int ldl_factor<double2>(int, double2 *, long long, double2 *, int *, bool, cudaStream_t);
template int ldl_solve<double>(int, int, const double *, long long, double *, long long, cudaStream_t);
template int ldl_solve<double2>(int, int, const double2 *, long long, double2 *, long long, cudaStream_t);

}  // namespace gla
