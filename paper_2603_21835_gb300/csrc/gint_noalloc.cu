// gint_noalloc.cu -- float64 dot-product reduction that allocates no device memory.
//
// Some callers cannot let a library allocate device memory: applications whose device memory
// is owned entirely by their own pool allocator (a cudaMalloc from elsewhere fails or fragments
// the pool), and latency-critical loops where the implicit synchronisation of cudaMalloc and
// cudaFree is not acceptable.  gint_grid_dot_noalloc serves them: it takes the caller's input
// and output pointers and keeps its only scratch (one float64 partial sum per chunk of
// GINT_NOALLOC_CHUNK elements) in the file-scope array below, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "gint.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// Scratch of the no-allocation reduction: one partial per chunk.  Shared by every call.
static __device__ __align__(256) double g_noalloc_partials[GINT_NOALLOC_MAX_CHUNKS];

// Device address of g_noalloc_partials per device (host code cannot use the symbol's name as
// a device pointer: in host code it names a host-side stand-in).
std::atomic<double *> g_partials_addr[kMaxDevices];
std::mutex g_setup_mutex;

// Partial sums of a[i] * b[i] (b == NULL: a[i]) over fixed chunks of GINT_NOALLOC_CHUNK
// elements, one CTA per chunk, so the summation order does not depend on the GPU.
__global__ void k_chunk_dot(const double *__restrict__ a, const double *__restrict__ b, long long n,
                            double *__restrict__ partials) {
  const long long c0 = (long long)blockIdx.x * GINT_NOALLOC_CHUNK;
  const long long c1 = c0 + GINT_NOALLOC_CHUNK < n ? c0 + GINT_NOALLOC_CHUNK : n;
  double acc = 0.0;
  for (long long i = c0 + threadIdx.x; i < c1; i += kThreads) acc += b ? a[i] * b[i] : a[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

__global__ void k_partials_sum(const double *__restrict__ partials, int nchunks, double scale,
                               double *__restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nchunks; i += kThreads) acc += partials[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    out[0] = scale * t;
  }
}

// Once per device, with that device current: the device address of the scratch array.
int partials_address(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GINT_ECUDA;
  double *p = g_partials_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    p = g_partials_addr[dev].load(std::memory_order_relaxed);
    if (!p) {
      if (cudaGetSymbolAddress((void **)&p, g_noalloc_partials) != cudaSuccess || !p) {
        cudaGetLastError();
        return GINT_ECUDA;
      }
      g_partials_addr[dev].store(p, std::memory_order_release);
    }
  }
  *out = p;
  return GINT_OK;
}

}  // namespace

extern "C" int gint_grid_dot_noalloc(const double *a, const double *b, long long n, double scale, double *out_dev,
                                     void *stream) {
  if (!a || !out_dev || n < 0) return GINT_EINVAL;
  if (n > (long long)GINT_NOALLOC_MAX_CHUNKS * GINT_NOALLOC_CHUNK) return GINT_ECAPACITY;
  double *partials = nullptr;
  int rc = partials_address(&partials);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int nchunks = (int)((n + GINT_NOALLOC_CHUNK - 1) / GINT_NOALLOC_CHUNK);
  if (nchunks > 0) {
    k_chunk_dot<<<nchunks, kThreads, 0, st>>>(a, b, n, partials);
    if (cudaGetLastError() != cudaSuccess) return GINT_ECUDA;
  }
  k_partials_sum<<<1, kThreads, 0, st>>>(partials, nchunks, scale, out_dev);
  if (cudaGetLastError() != cudaSuccess) return GINT_ECUDA;
  return GINT_OK;
}
