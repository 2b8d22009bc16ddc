// gint_la.cuh -- float64 dense linear algebra of the propagation steps (gint_la.cu): a tiled GEMM
// on strided operand views, and the blocked L D L^T factorisation (no pivoting) with its solve, for
// real symmetric and complex symmetric (A^T = A, no conjugation) matrices.
#pragma once
#include <cuda_runtime.h>

namespace gla {

// Operand view of a GEMM: element (r, k) -- r the output row (A) or column (B) index, k the
// contraction index -- is p[r sr + (k >> 1) skh + (k & 1) skl], times ks[k >> 1] when ks is not
// null.  An ordinary strided matrix has skh = 2 sk, skl = sk; the real view of interleaved complex
// data (k = 2 s + real / imaginary part) has skh = the complex stride in doubles, skl = 1.
template <typename T>
struct View {
  const T *p;
  long long sr, skh, skl;
  const double *ks;
};
template <typename T>
inline View<T> view(const T *p, long long sr, long long sk, const double *ks = nullptr) {
  return View<T>{p, sr, 2 * sk, sk, ks};
}

// C (element (i, j) at C[i cr + j cc]) = alpha A B + beta C, M x N, contraction K; T = double or
// double2 (complex).  mode 0: every element; mode 1: lower triangle only (i >= j; tiles above the
// diagonal are skipped); mode 2: the lower triangle, each value also written to (j, i) (C symmetric
// bit for bit).  beta = 0 does not read C.
template <typename T>
int gemm(int mode, int M, int N, int K, double alpha, View<T> A, View<T> B, double beta, T *C, long long cr,
         long long cc, cudaStream_t st);

// In-place A = L D L^T of the n x n matrix A (column-major, leading dimension lda; only the lower
// triangle is read): L unit lower (strictly lower part of A), D on the diagonal.  work: n x 64
// elements.  *info (device) = first j + 1 whose pivot d_j is zero or not finite (spd: not positive),
// else unchanged (the caller zeroes it).
template <typename T>
int ldl_factor(int n, T *A, long long lda, T *work, int *info, bool spd, cudaStream_t st);

// B <- (L D L^T)^{-1} B for the factor of ldl_factor; B n x nrhs column-major (leading dimension ldb).
template <typename T>
int ldl_solve(int n, int nrhs, const T *A, long long lda, T *B, long long ldb, cudaStream_t st);

}  // namespace gla
