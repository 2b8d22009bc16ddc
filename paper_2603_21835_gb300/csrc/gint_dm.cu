// gint_dm.cu -- the density matrix D = Re(psi diag(f) psi^dagger) (paper Sec. 2: rho_{mu nu} =
// sum_n f_n c_{mu n} c*_{nu n}, real part at the Gamma point) on the tcgen05 tensor cores.
//
// With k = 2 s + (0: real part, 1: imaginary part) the build is one real product D = A B^T,
// A_ik = f_s psi_is and B_ik = psi_is (parts), K = 2 nocc.  Each operand is scaled by one power of
// two (its largest magnitude lands in [2^14, 2^15)) and split into float16 hi + lo, and
//   A B^T ~ Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T
// runs as kind::f16 MMAs with float32 accumulators in tensor memory (lo lo, ~2^-22 of a product,
// is dropped).  The tensor core's float32 accumulation does not round to nearest, so its error grows
// with the number of MMAs added into one accumulator: the hi hi products of each K chunk of 64 (four
// MMAs) go to a fresh accumulator of a 3-deep ring, which drain warps add into float32 Kahan sums in
// registers; the cross products, 2^-11 smaller, stay in one accumulator for the whole K range.
//
// k_dm_absmax: the two scales' maxima (bit patterns of |x|, integer compares, atomicMax).
// k_dm_pack: operands -> hi/lo core-matrix blocks: block (row tile t, chunk q) is 32 KB,
//   [hi 16 KB | lo 16 KB], each 128 rows x 64 k float16, core matrix (row group g, k group h) at
//   byte (g * 8 + h) * 128 (K-major, no swizzle: LBO 128, SBO 1024).  Rows >= n, k >= 2 nocc: 0.
// k_dm_mma: one CTA of 16 warps per tile pair I <= J of D (128 x 128).  Lane 0 of warp 0 streams
//   the A (tile I) and B (tile J) blocks of each chunk by two bulk copies into a 3-stage ring and
//   issues 12 MMAs per chunk (4 K steps x 3 products); all 16 warps drain the hi hi accumulators
//   (row = TMEM lane, 32 columns a warp) and write D[i, j] and D[j, i] from one value, so D is
//   symmetric bit for bit.  (Sixteen warps keep the register cap at 128 for the Kahan sums.)
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "gint.h"
#include "gint_dm.cuh"
#include "gint_ptx.cuh"

namespace {
using namespace gptx;

constexpr int kTile = 128;                        // rows (and columns) of a D tile: M = N = 128
constexpr int kKC = 64;                           // k values per chunk: 4 MMA K steps of 16
constexpr int kStages = 3;                        // chunks in flight
constexpr int kHH = 3;                            // ring of hi hi accumulators (128 TMEM columns each)
constexpr uint32_t kCrossCol = kHH * 128;         // the hi lo + lo hi accumulator
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kHalfBytes = kTile * kKC * 2;  // one float16 part of a block: 16 KB
constexpr uint32_t kBlockBytes = 2 * kHalfBytes;  // hi then lo
constexpr uint32_t kStageBytes = 2 * kBlockBytes;  // A block then B block
constexpr uint32_t kSmemBytes = kStages * kStageBytes;
constexpr int kDrainWarps = 16;                   // four per TMEM lane quarter, 32 columns each
constexpr int kDrainCols = kTile / (kDrainWarps / 4);
constexpr int kDmThreads = 32 * kDrainWarps;
static_assert(kCrossCol + 128 <= kTmemCols, "tensor memory columns");
constexpr long long kWaitNs = 2000000000LL;  // bounded waits: 2 s
constexpr unsigned kErrTimeout = 1u;
// the final completion wait gave up too: MMAs issued by the CTA may still have been running when it
// released its tensor memory (the call's result and later tensor-core results are unreliable)
constexpr unsigned kErrInflight = 2u;

// Scale exponent of an operand: 2^sigma * max lands in [2^14, 2^15) (float16 max 65504).
__device__ __forceinline__ int dm_sigma(unsigned long long bits) {
  const double m = __longlong_as_double((long long)bits);
  return m > 0.0 ? 14 - ilogb(m) : 0;
}

// Bit pattern of |x|: for non-negative doubles it orders like the value.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// m[0] = max |f_s psi_is| and m[1] = max |psi_is| over real and imaginary parts, as the bit
// patterns of non-negative doubles.  Blocks along y take states, along x orbitals (coalesced); the
// maxima over psi are integer compares, one multiply by |f_s| per thread and state.
__global__ void __launch_bounds__(256) k_dm_absmax(int n, int nocc, const double2 *__restrict__ psi,
                                                   const double *__restrict__ f, unsigned long long *m) {
  unsigned long long a = 0, b = 0;
  for (int s = blockIdx.y; s < nocc; s += gridDim.y) {
    const double2 *row = psi + (long long)s * n;
    unsigned long long x = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const double2 p = row[i];
      x = max(x, max(abs_bits(p.x), abs_bits(p.y)));
    }
    b = max(b, x);
    a = max(a, abs_bits(f[s] * __longlong_as_double((long long)x)));
  }
  __shared__ unsigned long long ra[8], rb[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    ra[warp] = a;
    rb[warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      a = max(a, ra[w]);
      b = max(b, rb[w]);
    }
    atomicMax(&m[0], a);
    atomicMax(&m[1], b);
  }
}

__device__ __forceinline__ void split_f16(float x, __half &hi, __half &lo) {
  hi = __float2half_rn(x);
  lo = __float2half_rn(x - __half2float(hi));
}

// Block (x, y): rows i = 128 x + t of the operands, groups of 8 k (4 states) kg = y, y + gridDim.y,
// ...; each thread reads psi[s][i] (coalesced over i) and writes one 16-byte core-matrix row of hi
// and of lo, for A and for B.  B = 2^sigmaB psi is scaled in float64 (exact) and rounded to float32
// once; A = B (f_s 2^(sigmaA - sigmaB)) is formed in float32 (relative error 2^-24, below the
// split's 2^-23); the hi / lo split is float32 arithmetic.
__global__ void __launch_bounds__(kTile) k_dm_pack(int n, int nocc, int nq, const double2 *__restrict__ psi,
                                                   const double *__restrict__ f, const unsigned long long *__restrict__ m,
                                                   unsigned char *__restrict__ PA, unsigned char *__restrict__ PB) {
  const int sa = dm_sigma(m[0]), sb = dm_sigma(m[1]);
  const double scb = ldexp(1.0, sb), rab = ldexp(1.0, sa - sb);
  const int t = blockIdx.x, r = threadIdx.x, i = t * kTile + r;
  for (int kg = blockIdx.y; kg < nq * (kKC / 8); kg += gridDim.y) {
    __align__(16) __half ah[8], al[8], bh[8], bl[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int s = kg * 4 + j;
      float bx = 0.f, by = 0.f, fa = 0.f;
      if (i < n && s < nocc) {
        const double2 p = psi[(long long)s * n + i];
        bx = (float)(p.x * scb);
        by = (float)(p.y * scb);
        fa = (float)(f[s] * rab);
      }
      split_f16(bx * fa, ah[2 * j], al[2 * j]);
      split_f16(by * fa, ah[2 * j + 1], al[2 * j + 1]);
      split_f16(bx, bh[2 * j], bl[2 * j]);
      split_f16(by, bh[2 * j + 1], bl[2 * j + 1]);
    }
    const int q = kg / (kKC / 8), h = kg % (kKC / 8);
    const size_t off = ((size_t)t * nq + q) * kBlockBytes + (size_t)((r >> 3) * 8 + h) * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4 *>(PA + off) = *reinterpret_cast<const uint4 *>(ah);
    *reinterpret_cast<uint4 *>(PA + off + kHalfBytes) = *reinterpret_cast<const uint4 *>(al);
    *reinterpret_cast<uint4 *>(PB + off) = *reinterpret_cast<const uint4 *>(bh);
    *reinterpret_cast<uint4 *>(PB + off + kHalfBytes) = *reinterpret_cast<const uint4 *>(bl);
  }
}

// Kahan step: (s, c) += x, the running sum s and its lost low part c (true sum ~ s - c).
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

struct DmShared {
  uint64_t full[kStages], empty[kStages], hfull[kHH], hfree[kHH], done;
  uint32_t tmem;
};

// Copies of chunk c (A tile I, B tile J) into its stage.
__device__ __forceinline__ void dm_load(DmShared &sh, unsigned char *smem, const unsigned char *PA,
                                        const unsigned char *PB, int I, int J, int nq, int c) {
  const int s = c % kStages;
  mbar_arrive_tx(&sh.full[s], kStageBytes);
  bulk_g2s(smem + s * kStageBytes, PA + ((size_t)I * nq + c) * kBlockBytes, kBlockBytes, &sh.full[s]);
  bulk_g2s(smem + s * kStageBytes + kBlockBytes, PB + ((size_t)J * nq + c) * kBlockBytes, kBlockBytes, &sh.full[s]);
}

// One warp adds its 32 rows x kDrainCols columns of the hi hi accumulator of chunk c into the
// Kahan sums and releases the accumulator; false if the wait gave up.
__device__ __forceinline__ bool dm_drain(DmShared &sh, uint32_t lane_base, int c, float *sum, float *cmp,
                                         unsigned *status) {
  const int a = c % kHH;
  const bool ok = __all_sync(0xffffffffu, mbar_wait(&sh.hfull[a], (uint32_t)(c / kHH) & 1u, status, kErrTimeout,
                                                     kWaitNs));
  if (!ok) return false;
  tc_fence_after();
#pragma unroll
  for (int g = 0; g < kDrainCols / 16; ++g) {
    float y[16];
    tmem_ld16(lane_base + (uint32_t)a * 128u + (uint32_t)g * 16u, y);
#pragma unroll
    for (int j = 0; j < 16; ++j) kahan_add(sum[g * 16 + j], cmp[g * 16 + j], y[j]);
  }
  tc_fence_before();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(&sh.hfree[a]);
  return true;
}

__global__ void __launch_bounds__(kDmThreads, 1)
    k_dm_mma(int n, int nq, const unsigned char *__restrict__ PA, const unsigned char *__restrict__ PB,
             const unsigned long long *__restrict__ m, double *__restrict__ D, unsigned *status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ DmShared sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tile pair p -> (I, J), I <= J, p = J (J + 1) / 2 + I
  const long long p = blockIdx.x;
  int J = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
  while ((long long)J * (J + 1) / 2 > p) --J;
  while ((long long)(J + 1) * (J + 2) / 2 <= p) ++J;
  const int I = (int)(p - (long long)J * (J + 1) / 2);

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sh.full[s], 1);
      mbar_init(&sh.empty[s], 1);
    }
    for (int a = 0; a < kHH; ++a) {
      mbar_init(&sh.hfull[a], 1);
      mbar_init(&sh.hfree[a], kDrainWarps);
    }
    mbar_init(&sh.done, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&sh.tmem, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;

  // warp w reads TMEM lanes 32 (w mod 4) .. + 31 (its rows) and kDrainCols columns from kDrainCols (w / 4)
  const int r = (warp & 3) * 32 + lane, c0 = (warp >> 2) * kDrainCols;
  const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
  float sum[kDrainCols], cmp[kDrainCols];
#pragma unroll
  for (int j = 0; j < kDrainCols; ++j) sum[j] = cmp[j] = 0.f;
  bool ok = true;

  if (warp == 0) {
    // the warp runs the issue loop together (warp-uniform descriptor arithmetic; one elected lane
    // issues, which keeps the tensor pipe fed better than a loop confined to one lane): chunk c's
    // MMAs (hi hi into ring slot c mod kHH, hi lo + lo hi into the cross slot), then the refill of
    // chunk c - 1's stage once its MMAs are done (lane 0 issues the copies); the warp drains chunk
    // c - 2 (the slot the MMAs of chunk c + 1 will take).  Wait results are lane 0's, broadcast.
    const uint32_t idesc = idesc_f16(kTile, kTile), sbase = smem_u32(smem), dx = tmem + kCrossCol;
    int issued = 0, consumed = 0;
    for (; issued < min(kStages, nq); ++issued)
      if (lane == 0) dm_load(sh, smem, PA, PB, I, J, nq, issued);
    for (int c = 0; c < nq && ok; ++c) {
      const int s = c % kStages, a = c % kHH;
      bool lok = mbar_wait(&sh.full[s], (uint32_t)(c / kStages) & 1u, status, kErrTimeout, kWaitNs);
      lok = __shfl_sync(0xffffffffu, lok, 0);
      if (lok) consumed = c + 1;
      if (lok && c >= kHH)
        lok = __shfl_sync(0xffffffffu,
                          mbar_wait(&sh.hfree[a], (uint32_t)((c / kHH) - 1) & 1u, status, kErrTimeout, kWaitNs), 0);
      if (lok) {
        tc_fence_after();
        const uint32_t sa = sbase + s * kStageBytes, sb = sa + kBlockBytes;
        const uint32_t dh = tmem + (uint32_t)a * 128u;
        if (elect_one()) {
#pragma unroll
          for (int ks = 0; ks < kKC / 16; ++ks) {
            const uint32_t o = ks * 256;  // two core matrices along K per step
            const uint64_t ah = sdesc(sa + o, 128, 1024), al = sdesc(sa + kHalfBytes + o, 128, 1024);
            const uint64_t bh = sdesc(sb + o, 128, 1024), bl = sdesc(sb + kHalfBytes + o, 128, 1024);
            mma_f16(dh, ah, bh, idesc, ks > 0 ? 1u : 0u);
            mma_f16(dx, ah, bl, idesc, (c > 0 || ks > 0) ? 1u : 0u);
            mma_f16(dx, al, bh, idesc, 1u);
          }
          mma_commit(&sh.empty[s]);
          mma_commit(&sh.hfull[a]);
        }
        __syncwarp();
        if (c >= 1 && issued < nq) {
          lok = __shfl_sync(0xffffffffu,
                            mbar_wait(&sh.empty[(c - 1) % kStages], (uint32_t)((c - 1) / kStages) & 1u, status,
                                      kErrTimeout, kWaitNs),
                            0);
          if (lok) {
            if (lane == 0) dm_load(sh, smem, PA, PB, I, J, nq, issued);
            ++issued;
          }
        }
      }
      ok = lok;
      if (ok && c >= 2) ok = dm_drain(sh, lane_base, c - 2, sum, cmp, status);
    }
    if (elect_one()) mma_commit(&sh.done);  // the lane that issued the MMAs
    __syncwarp();
    if (lane == 0) {
      // no copy may still be landing in shared memory when the CTA exits
      for (int c = consumed; c < issued; ++c)
        mbar_wait(&sh.full[c % kStages], (uint32_t)(c / kStages) & 1u, status, kErrTimeout, kWaitNs);
    }
    for (int c = max(0, nq - 2); c < nq && ok; ++c) ok = dm_drain(sh, lane_base, c, sum, cmp, status);
  } else {
    for (int c = 0; c < nq && ok; ++c) ok = dm_drain(sh, lane_base, c, sum, cmp, status);
  }

  ok = __all_sync(0xffffffffu, ok && mbar_wait(&sh.done, 0u, status, kErrTimeout, kWaitNs));
  tc_fence_after();
  if (ok) {
    const double scale = ldexp(1.0, -(dm_sigma(m[0]) + dm_sigma(m[1])));
    const long long i = (long long)I * kTile + r;
#pragma unroll
    for (int g = 0; g < kDrainCols / 16; ++g) {
      float x[16];
      tmem_ld16(lane_base + kCrossCol + (uint32_t)g * 16u, x);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const long long jj = (long long)J * kTile + c0 + g * 16 + j;
        if (i < n && jj < n && (I != J || jj >= i)) {
          const double v = (((double)sum[g * 16 + j] - (double)cmp[g * 16 + j]) + (double)x[j]) * scale;
          D[i * n + jj] = v;
          D[jj * n + i] = v;
        }
      }
    }
  }
  if (!ok && warp == 0 && lane == 0) {
    // before the tensor memory is released: once more (bounded) for the MMAs issued so far, which
    // complete by themselves; if they still have not, say so
    if (!mbar_wait(&sh.done, 0u, status, kErrTimeout, 4 * kWaitNs)) atomicOr(status, kErrInflight);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

size_t gint_dm_tc_bytes(int n, int nocc) {
  const long long T = (n + kTile - 1) / kTile, nq = (2LL * nocc + kKC - 1) / kKC;
  return (size_t)(2 * T * nq) * kBlockBytes + 2 * sizeof(unsigned long long);
}

int gint_dm_tc(int n, int nocc, const double *psi, const double *f, double *D, void *work, unsigned *status,
               cudaStream_t st) {
  // set on every call: the attribute is per device and the call is cheap next to the build
  if (cudaFuncSetAttribute(k_dm_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess)
    return GINT_ECUDA;
  const int T = (n + kTile - 1) / kTile, nq = (2 * nocc + kKC - 1) / kKC;
  unsigned char *PA = static_cast<unsigned char *>(work), *PB = PA + (size_t)T * nq * kBlockBytes;
  unsigned long long *m = reinterpret_cast<unsigned long long *>(PB + (size_t)T * nq * kBlockBytes);
  if (cudaMemsetAsync(m, 0, 2 * sizeof(unsigned long long), st) != cudaSuccess) return GINT_ECUDA;
  const double2 *P = reinterpret_cast<const double2 *>(psi);
  const dim3 ga((unsigned)std::max(1, std::min((n + 1023) / 1024, 64)), (unsigned)std::min(nocc, 256));
  k_dm_absmax<<<ga, 256, 0, st>>>(n, nocc, P, f, m);
  const dim3 gp((unsigned)T, (unsigned)std::min(nq * (kKC / 8), 256));
  k_dm_pack<<<gp, kTile, 0, st>>>(n, nocc, nq, P, f, m, PA, PB);
  k_dm_mma<<<(unsigned)((long long)T * (T + 1) / 2), kDmThreads, kSmemBytes, st>>>(n, nq, PA, PB, m, D, status);
  return cudaGetLastError() == cudaSuccess ? GINT_OK : GINT_ECUDA;
}
