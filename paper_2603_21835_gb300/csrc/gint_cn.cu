// gint_cn.cu -- the dense steps of real-time propagation around the grid passes: the density matrix
// from coefficients and occupations, D = Re(psi diag(f) psi^dagger), one Crank-Nicolson step of the
// coefficients, (S + i dt/2 H) psi(t + dt) = (S - i dt/2 H) psi(t) (paper Sec. 2: the density matrix
// and the time propagation of the coefficients with the overlap matrix), and the energy-density
// matrix E = (S^{-1} H D + D H S^{-1}) / 2.  All in float64 on this library's own kernels
// (gint_la.cu: tiled GEMM, blocked L D L^T and its solves); the density matrix also has a
// tensor-core build (float16 three-term split, gint_dm.cu).  A context holds every buffer, so the
// compute calls allocate nothing.
//
// The step solves A X = S psi with A = S + i dt/2 H and returns 2 X - psi, which equals
// A^{-1} (S - i dt/2 H) psi since S - i dt/2 H = 2 S - A: a real-by-complex product replaces the
// complex one, and A is factored as L D L^T (A^T = A) instead of by a general LU.
#include <cuda_runtime.h>

#include <algorithm>

#include "gint.h"
#include "gint_dm.cuh"
#include "gint_la.cuh"

namespace {

// A = S + i dt/2 H (S, H real symmetric: row- and column-major alike)
__global__ void k_cn_mat(long long nn, const double *__restrict__ S, const double *__restrict__ H, double half_dt,
                         double2 *__restrict__ A) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x)
    A[e] = make_double2(S[e], half_dt * H[e]);
}

// X <- 2 X - psi
__global__ void k_cn_finish(long long m, const double2 *__restrict__ psi, double2 *__restrict__ X) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x) {
    const double2 x = X[e], p = psi[e];
    X[e] = make_double2(2.0 * x.x - p.x, 2.0 * x.y - p.y);
  }
}

// E = (X + X^T) / 2 (n x n)
__global__ void k_sym_half(int n, const double *__restrict__ X, double *__restrict__ E) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e - i * n;
    E[e] = 0.5 * (X[e] + X[j * n + i]);
  }
}

unsigned blocks_for(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 4096); }

}  // namespace

struct gint_cn {
  int n = 0, nocc = 0, device = 0;
  double2 *A = nullptr;        // n x n: the factor (complex), or two real n x n matrices (gint_edm)
  double2 *work = nullptr;     // n x 64: the factorisation's panel workspace
  int *info = nullptr;
  void *dmw = nullptr;         // tensor-core density-matrix build: packed operands and scales
  unsigned *status = nullptr;  // its device error word
};

extern "C" {

int gint_cn_destroy(gint_cn *c) {
  if (!c) return GINT_OK;
  cudaSetDevice(c->device);
  cudaFree(c->A);
  cudaFree(c->work);
  cudaFree(c->info);
  cudaFree(c->dmw);
  cudaFree(c->status);
  delete c;
  return GINT_OK;
}

int gint_cn_create(int n, int nocc, gint_cn **out) {
  if (!out || n <= 0 || nocc <= 0) return GINT_EINVAL;
  *out = nullptr;
  gint_cn *c = new gint_cn;
  c->n = n;
  c->nocc = nocc;
  cudaGetDevice(&c->device);
  const size_t nn = (size_t)n * n;
  if (cudaMalloc(&c->A, nn * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&c->work, (size_t)n * 64 * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&c->info, sizeof(int)) != cudaSuccess || cudaMalloc(&c->dmw, gint_dm_tc_bytes(n, nocc)) != cudaSuccess ||
      cudaMalloc(&c->status, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(c->info, 0, sizeof(int)) != cudaSuccess || cudaMemset(c->status, 0, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    gint_cn_destroy(c);
    return GINT_ENOMEM;
  }
  *out = c;
  return GINT_OK;
}

int gint_cn_step(gint_cn *c, const double *S, const double *H, double dt, const double *psi, double *psi_out,
                 void *stream) {
  if (!c || !S || !H || !psi || !psi_out || psi == psi_out) return GINT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = c->n, k = c->nocc;
  const long long nn = (long long)n * n;
  double2 *X = reinterpret_cast<double2 *>(psi_out);
  if (cudaMemsetAsync(c->info, 0, sizeof(int), st) != cudaSuccess) return GINT_ECUDA;
  k_cn_mat<<<blocks_for(nn), 256, 0, st>>>(nn, S, H, 0.5 * dt, c->A);
  if (cudaGetLastError() != cudaSuccess) return GINT_ECUDA;
  // X = S psi: real and imaginary parts (strided real views of the interleaved complex arrays)
  for (int part = 0; part < 2; ++part) {
    const int rc = gla::gemm<double>(0, n, k, n, 1.0, gla::view<double>(S, 1, n),
                                     gla::view<double>(psi + part, 2LL * n, 2), 0.0, psi_out + part, 2, 2LL * n, st);
    if (rc) return rc;
  }
  int rc = gla::ldl_factor<double2>(n, c->A, n, c->work, c->info, false, st);
  if (rc) return rc;
  if ((rc = gla::ldl_solve<double2>(n, k, c->A, n, X, n, st))) return rc;
  k_cn_finish<<<blocks_for((long long)n * k), 256, 0, st>>>((long long)n * k, reinterpret_cast<const double2 *>(psi), X);
  return cudaGetLastError() == cudaSuccess ? GINT_OK : GINT_ECUDA;
}

int gint_dm_build(gint_cn *c, const double *psi, const double *f, double *D, void *stream) {
  if (!c || !psi || !f || !D) return GINT_EINVAL;
  const int n = c->n;
  // D = A B^T over k = 2 s + (real, imaginary part): A_ik = f_s psi_is, B_ik = psi_is (real views);
  // the lower triangle is computed and mirrored, so D is symmetric bit for bit
  const gla::View<double> Av{psi, 2, 2LL * n, 1, f}, Bv{psi, 2, 2LL * n, 1, nullptr};
  return gla::gemm<double>(2, n, n, 2 * c->nocc, 1.0, Av, Bv, 0.0, D, 1, n, (cudaStream_t)stream);
}

int gint_dm_build_f16x3(gint_cn *c, const double *psi, const double *f, double *D, void *stream) {
  if (!c || !psi || !f || !D) return GINT_EINVAL;
  return gint_dm_tc(c->n, c->nocc, psi, f, D, c->dmw, c->status, (cudaStream_t)stream);
}

int gint_edm(gint_cn *c, const double *S, const double *H, const double *D, double *E, void *stream) {
  if (!c || !S || !H || !D || !E) return GINT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = c->n;
  // the complex n x n buffer holds two real n x n matrices: F (the factor of S) and X
  double *F = reinterpret_cast<double *>(c->A), *X = F + (size_t)n * n;
  if (cudaMemsetAsync(c->info, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemcpyAsync(F, S, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return GINT_ECUDA;
  // X = H D, then X <- S^{-1} X (S = L D L^T), E = (X + X^T) / 2
  int rc = gla::gemm<double>(0, n, n, n, 1.0, gla::view<double>(H, 1, n), gla::view<double>(D, n, 1), 0.0, X, 1, n, st);
  if (rc) return rc;
  if ((rc = gla::ldl_factor<double>(n, F, n, reinterpret_cast<double *>(c->work), c->info, true, st))) return rc;
  if ((rc = gla::ldl_solve<double>(n, n, F, n, X, n, st))) return rc;
  k_sym_half<<<blocks_for((long long)n * n), 256, 0, st>>>(n, X, E);
  return cudaGetLastError() == cudaSuccess ? GINT_OK : GINT_ECUDA;
}

int gint_cn_info(gint_cn *c, int *info) {
  if (!c || !info) return GINT_EINVAL;
  unsigned st = 0;
  if (cudaMemcpy(info, c->info, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&st, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
    return GINT_ECUDA;
  if (st != 0) {
    cudaMemset(c->status, 0, sizeof(unsigned));
    return GINT_ETIMEDOUT;
  }
  return GINT_OK;
}

}  // extern "C"
