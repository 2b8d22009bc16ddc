// gint_cn.cu -- the dense steps of real-time propagation around the grid passes: the density matrix
// from coefficients and occupations, D = Re(psi diag(f) psi^dagger), one Crank-Nicolson step of the
// coefficients, (S + i dt/2 H) psi(t + dt) = (S - i dt/2 H) psi(t), by LU factorisation (paper Sec. 2:
// the density matrix and the time propagation of the coefficients with the overlap matrix), and the
// energy-density matrix E = (S^{-1} H D + D H S^{-1}) / 2 by a Cholesky solve.  The density matrix
// also has a tensor-core build (float16 three-term split, gint_dm.cu).
//
// Both are plain library operations: complex GEMMs (cuBLAS) and an LU factorisation with partial
// pivoting and its solve (cuSOLVER).  The libraries are loaded on first use (dlopen), so the grid
// library itself keeps no link dependency on them; without them these calls return
// GINT_EUNSUPPORTED.  A context holds every buffer, so the compute calls allocate nothing.
#include <cublas_v2.h>
#include <cuComplex.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>
#include <dlfcn.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "gint.h"
#include "gint_dm.cuh"

#ifndef GINT_CUDA_LIB_DIR
#define GINT_CUDA_LIB_DIR "/usr/local/cuda/lib64"
#endif

namespace {

struct Libs {
  bool ok = false;
  cublasStatus_t (*blas_create)(cublasHandle_t *) = nullptr;
  cublasStatus_t (*blas_destroy)(cublasHandle_t) = nullptr;
  cublasStatus_t (*blas_stream)(cublasHandle_t, cudaStream_t) = nullptr;
  cublasStatus_t (*zgemm)(cublasHandle_t, cublasOperation_t, cublasOperation_t, int, int, int, const cuDoubleComplex *,
                          const cuDoubleComplex *, int, const cuDoubleComplex *, int, const cuDoubleComplex *,
                          cuDoubleComplex *, int) = nullptr;
  cusolverStatus_t (*sol_create)(cusolverDnHandle_t *) = nullptr;
  cusolverStatus_t (*sol_destroy)(cusolverDnHandle_t) = nullptr;
  cusolverStatus_t (*sol_stream)(cusolverDnHandle_t, cudaStream_t) = nullptr;
  cusolverStatus_t (*getrf_size)(cusolverDnHandle_t, int, int, cuDoubleComplex *, int, int *) = nullptr;
  cusolverStatus_t (*getrf)(cusolverDnHandle_t, int, int, cuDoubleComplex *, int, cuDoubleComplex *, int *,
                            int *) = nullptr;
  cusolverStatus_t (*getrs)(cusolverDnHandle_t, cublasOperation_t, int, int, const cuDoubleComplex *, int,
                            const int *, cuDoubleComplex *, int, int *) = nullptr;
  cublasStatus_t (*dgemm)(cublasHandle_t, cublasOperation_t, cublasOperation_t, int, int, int, const double *,
                          const double *, int, const double *, int, const double *, double *, int) = nullptr;
  cusolverStatus_t (*potrf_size)(cusolverDnHandle_t, cublasFillMode_t, int, double *, int, int *) = nullptr;
  cusolverStatus_t (*potrf)(cusolverDnHandle_t, cublasFillMode_t, int, double *, int, double *, int, int *) = nullptr;
  cusolverStatus_t (*potrs)(cusolverDnHandle_t, cublasFillMode_t, int, int, const double *, int, double *, int,
                            int *) = nullptr;
};

void *open_first(const char *const *names) {
  for (int i = 0; names[i]; ++i) {
    if (void *h = dlopen(names[i], RTLD_NOW | RTLD_GLOBAL)) return h;
    const std::string full = std::string(GINT_CUDA_LIB_DIR) + "/" + names[i];
    if (void *h = dlopen(full.c_str(), RTLD_NOW | RTLD_GLOBAL)) return h;
  }
  return nullptr;
}

const Libs &libs() {
  static Libs L;
  static std::once_flag once;
  std::call_once(once, [] {
    const char *blas_names[] = {"libcublas.so.13", "libcublas.so.12", "libcublas.so", nullptr};
    const char *sol_names[] = {"libcusolver.so.12", "libcusolver.so.11", "libcusolver.so", nullptr};
    void *hb = open_first(blas_names), *hs = open_first(sol_names);
    if (!hb || !hs) return;
    L.blas_create = (decltype(L.blas_create))dlsym(hb, "cublasCreate_v2");
    L.blas_destroy = (decltype(L.blas_destroy))dlsym(hb, "cublasDestroy_v2");
    L.blas_stream = (decltype(L.blas_stream))dlsym(hb, "cublasSetStream_v2");
    L.zgemm = (decltype(L.zgemm))dlsym(hb, "cublasZgemm_v2");
    L.sol_create = (decltype(L.sol_create))dlsym(hs, "cusolverDnCreate");
    L.sol_destroy = (decltype(L.sol_destroy))dlsym(hs, "cusolverDnDestroy");
    L.sol_stream = (decltype(L.sol_stream))dlsym(hs, "cusolverDnSetStream");
    L.getrf_size = (decltype(L.getrf_size))dlsym(hs, "cusolverDnZgetrf_bufferSize");
    L.getrf = (decltype(L.getrf))dlsym(hs, "cusolverDnZgetrf");
    L.getrs = (decltype(L.getrs))dlsym(hs, "cusolverDnZgetrs");
    L.dgemm = (decltype(L.dgemm))dlsym(hb, "cublasDgemm_v2");
    L.potrf_size = (decltype(L.potrf_size))dlsym(hs, "cusolverDnDpotrf_bufferSize");
    L.potrf = (decltype(L.potrf))dlsym(hs, "cusolverDnDpotrf");
    L.potrs = (decltype(L.potrs))dlsym(hs, "cusolverDnDpotrs");
    L.ok = L.blas_create && L.blas_destroy && L.blas_stream && L.zgemm && L.sol_create && L.sol_destroy &&
           L.sol_stream && L.getrf_size && L.getrf && L.getrs && L.dgemm && L.potrf_size && L.potrf && L.potrs;
  });
  return L;
}

// A = S + i dt/2 H, W = S - i dt/2 H (S, H real symmetric: row- and column-major alike)
__global__ void k_cn_mats(long long nn, const double *__restrict__ S, const double *__restrict__ H, double half_dt,
                          cuDoubleComplex *__restrict__ A, cuDoubleComplex *__restrict__ W) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
    const double s = S[e], h = half_dt * H[e];
    A[e] = make_cuDoubleComplex(s, h);
    W[e] = make_cuDoubleComplex(s, -h);
  }
}

// Y[:, j] = f[j] psi[:, j] (column-major n x nocc)
__global__ void k_scale_cols(int n, int nocc, const cuDoubleComplex *__restrict__ psi, const double *__restrict__ f,
                             cuDoubleComplex *__restrict__ Y) {
  const long long tot = (long long)n * nocc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const double s = f[e / n];
    Y[e] = make_cuDoubleComplex(s * cuCreal(psi[e]), s * cuCimag(psi[e]));
  }
}

__global__ void k_real_part(long long nn, const cuDoubleComplex *__restrict__ C, double *__restrict__ D) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x)
    D[e] = cuCreal(C[e]);
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
  int n = 0, nocc = 0, device = 0, lwork = 0, lwork_r = 0;
  cuDoubleComplex *A = nullptr, *W = nullptr, *Y = nullptr, *work = nullptr;
  int *ipiv = nullptr, *info = nullptr;
  void *dmw = nullptr;         // tensor-core density-matrix build: packed operands and scales
  unsigned *status = nullptr;  // its device error word
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t sol = nullptr;
};

extern "C" {

int gint_cn_destroy(gint_cn *c) {
  if (!c) return GINT_OK;
  const Libs &L = libs();
  cudaSetDevice(c->device);
  cudaFree(c->A);
  cudaFree(c->W);
  cudaFree(c->Y);
  cudaFree(c->work);
  cudaFree(c->ipiv);
  cudaFree(c->info);
  cudaFree(c->dmw);
  cudaFree(c->status);
  if (c->blas) L.blas_destroy(c->blas);
  if (c->sol) L.sol_destroy(c->sol);
  delete c;
  return GINT_OK;
}

int gint_cn_create(int n, int nocc, gint_cn **out) {
  if (!out || n <= 0 || nocc <= 0) return GINT_EINVAL;
  *out = nullptr;
  const Libs &L = libs();
  if (!L.ok) return GINT_EUNSUPPORTED;
  gint_cn *c = new gint_cn;
  c->n = n;
  c->nocc = nocc;
  cudaGetDevice(&c->device);
  const size_t nn = (size_t)n * n;
  if (cudaMalloc(&c->A, nn * sizeof(cuDoubleComplex)) != cudaSuccess ||
      cudaMalloc(&c->W, nn * sizeof(cuDoubleComplex)) != cudaSuccess ||
      cudaMalloc(&c->Y, (size_t)n * nocc * sizeof(cuDoubleComplex)) != cudaSuccess ||
      cudaMalloc(&c->ipiv, (size_t)n * sizeof(int)) != cudaSuccess || cudaMalloc(&c->info, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->dmw, gint_dm_tc_bytes(n, nocc)) != cudaSuccess ||
      cudaMalloc(&c->status, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    gint_cn_destroy(c);
    return GINT_ENOMEM;
  }
  if (L.blas_create(&c->blas) != CUBLAS_STATUS_SUCCESS || L.sol_create(&c->sol) != CUSOLVER_STATUS_SUCCESS ||
      L.getrf_size(c->sol, n, n, c->A, n, &c->lwork) != CUSOLVER_STATUS_SUCCESS ||
      L.potrf_size(c->sol, CUBLAS_FILL_MODE_LOWER, n, reinterpret_cast<double *>(c->A), n, &c->lwork_r) !=
          CUSOLVER_STATUS_SUCCESS) {
    gint_cn_destroy(c);
    return GINT_ECUDA;
  }
  // one workspace for both factorisations (complex elements; the real one needs lwork_r doubles)
  c->lwork = std::max(c->lwork, (c->lwork_r + 1) / 2);
  if (cudaMalloc(&c->work, (size_t)std::max(c->lwork, 1) * sizeof(cuDoubleComplex)) != cudaSuccess ||
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
  const Libs &L = libs();
  cudaStream_t st = (cudaStream_t)stream;
  const long long nn = (long long)c->n * c->n;
  k_cn_mats<<<blocks_for(nn), 256, 0, st>>>(nn, S, H, 0.5 * dt, c->A, c->W);
  if (cudaGetLastError() != cudaSuccess) return GINT_ECUDA;
  if (L.blas_stream(c->blas, st) != CUBLAS_STATUS_SUCCESS || L.sol_stream(c->sol, st) != CUSOLVER_STATUS_SUCCESS)
    return GINT_ECUDA;
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  cuDoubleComplex *B = reinterpret_cast<cuDoubleComplex *>(psi_out);
  // B = (S - i dt/2 H) psi, then B <- A^{-1} B with A = LU (partial pivoting)
  if (L.zgemm(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, c->n, c->nocc, c->n, &one, c->W, c->n,
              reinterpret_cast<const cuDoubleComplex *>(psi), c->n, &zero, B, c->n) != CUBLAS_STATUS_SUCCESS)
    return GINT_ECUDA;
  if (L.getrf(c->sol, c->n, c->n, c->A, c->n, c->work, c->ipiv, c->info) != CUSOLVER_STATUS_SUCCESS) return GINT_ECUDA;
  if (L.getrs(c->sol, CUBLAS_OP_N, c->n, c->nocc, c->A, c->n, c->ipiv, B, c->n, c->info) != CUSOLVER_STATUS_SUCCESS)
    return GINT_ECUDA;
  return GINT_OK;
}

int gint_dm_build(gint_cn *c, const double *psi, const double *f, double *D, void *stream) {
  if (!c || !psi || !f || !D) return GINT_EINVAL;
  const Libs &L = libs();
  cudaStream_t st = (cudaStream_t)stream;
  const long long nn = (long long)c->n * c->n;
  const cuDoubleComplex *P = reinterpret_cast<const cuDoubleComplex *>(psi);
  k_scale_cols<<<blocks_for((long long)c->n * c->nocc), 256, 0, st>>>(c->n, c->nocc, P, f, c->Y);
  if (cudaGetLastError() != cudaSuccess) return GINT_ECUDA;
  if (L.blas_stream(c->blas, st) != CUBLAS_STATUS_SUCCESS) return GINT_ECUDA;
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0);
  // W = (psi diag f) psi^dagger, D = Re W
  if (L.zgemm(c->blas, CUBLAS_OP_N, CUBLAS_OP_C, c->n, c->n, c->nocc, &one, c->Y, c->n, P, c->n, &zero, c->W, c->n) !=
      CUBLAS_STATUS_SUCCESS)
    return GINT_ECUDA;
  k_real_part<<<blocks_for(nn), 256, 0, st>>>(nn, c->W, D);
  return cudaGetLastError() == cudaSuccess ? GINT_OK : GINT_ECUDA;
}

int gint_dm_build_f16x3(gint_cn *c, const double *psi, const double *f, double *D, void *stream) {
  if (!c || !psi || !f || !D) return GINT_EINVAL;
  return gint_dm_tc(c->n, c->nocc, psi, f, D, c->dmw, c->status, (cudaStream_t)stream);
}

int gint_edm(gint_cn *c, const double *S, const double *H, const double *D, double *E, void *stream) {
  if (!c || !S || !H || !D || !E) return GINT_EINVAL;
  const Libs &L = libs();
  cudaStream_t st = (cudaStream_t)stream;
  const int n = c->n;
  // the n x n complex buffers hold two real n x n matrices each: A -> Cholesky factor of S, W -> X
  double *F = reinterpret_cast<double *>(c->A), *X = reinterpret_cast<double *>(c->W);
  if (cudaMemcpyAsync(F, S, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return GINT_ECUDA;
  if (L.blas_stream(c->blas, st) != CUBLAS_STATUS_SUCCESS || L.sol_stream(c->sol, st) != CUSOLVER_STATUS_SUCCESS)
    return GINT_ECUDA;
  const double one = 1.0, zero = 0.0;
  // X = H D, then X <- S^{-1} X (S = L L^T), E = (X + X^T) / 2
  if (L.dgemm(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, n, n, &one, H, n, D, n, &zero, X, n) != CUBLAS_STATUS_SUCCESS)
    return GINT_ECUDA;
  if (L.potrf(c->sol, CUBLAS_FILL_MODE_LOWER, n, F, n, reinterpret_cast<double *>(c->work), 2 * c->lwork, c->info) !=
      CUSOLVER_STATUS_SUCCESS)
    return GINT_ECUDA;
  if (L.potrs(c->sol, CUBLAS_FILL_MODE_LOWER, n, n, F, n, X, n, c->info) != CUSOLVER_STATUS_SUCCESS) return GINT_ECUDA;
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
