// gint_tc.cu -- tensor-core (tcgen05, sm_103a) brick kernels for the density, force and
// local-Hamiltonian passes of uniform-grid integration (paper Sec. 3.3.1: orbitals packed into
// dense tiles per grid block, then batched tile contractions).
//
// Arithmetic: float32 orbital evaluation with compensated (double-float) distance and knot
// parameter; operands split x = hi + lo into two float16 values (22 significant bits, with
// power-of-two scales that keep every value inside the float16 range); products
// hi*hi + hi*lo + lo*hi on kind::f16 tensor cores with float32 accumulation in tensor memory;
// float64 for every cross-brick reduction.
//
// Layout: the orbitals of each atom occupy porb = roundup(norb, 8) columns of the brick's
// orbital space (zero padded), no atom crosses a multiple of 128 columns, NP = padded total.
// D is pre-tiled per atom pair into float16 (hi, lo) 128-byte core matrices, stored
// column-atom-major with the hi and lo 8 x 8 blocks interleaved, so the B operand of a chunk that is
// one 16-column atom arrives in a few bulk (TMA) copies: one per run of row atoms that are adjacent
// in the brick and in the tile store.
//
// Density (D symmetric): columns are streamed in chunks of 16.  With the chunk's own
// diagonal block halved, rho = 2 sum_k P_k Y_k where Y_k accumulates P_j D_jk over the chunks
// j <= chunk(k) only, so chunk c's columns are final right after chunk c's MMA: the epilogue of
// chunk c overlaps the MMA of chunk c+1 and the MMA work is halved.  Seven prefetch warps issue
// the chunks' bulk copies, chunk k by warp k mod 7 (the first stages during the orbital evaluation,
// each later chunk as soon as its stage is freed), one MMA thread issues, and eight epilogue warps
// drain finished chunks, all decoupled by mbarriers.
// Force: full Y = P D (all chunks, all columns), then per atom 2 w V grad(phi) . Y.
// Local H from the same orbital tile P: H = (W P)^T P with K = grid points (blocks of 16-32),
// M = N = orbitals (128-row tiles, upper block triangle); both operands are MN-major views of
// [point][orbital] buffers, W P built per block in the freed chunk stages.  Each brick writes its
// float32 slot-pair tiles to a scratch area and a per-pair float64 reduction (fixed order, no
// atomics) produces both H(I,J) and H(J,I).  One work item per brick runs every requested pass,
// so the orbitals are evaluated once per brick.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "gint_handle.cuh"
#include "gint_ptx.cuh"

namespace {
using namespace gptx;

constexpr int kT = 512;          // threads of the brick kernels (16 warps)
constexpr int kNPMAX = 320;      // padded orbitals of a brick (density / force)
constexpr int kNPMAXH = 288;     // padded orbitals of a brick (local H: tensor-memory limit)
constexpr int kMAXA = 40;        // atoms of a brick
constexpr int kMAXE = 160;       // (atom, image) entries of a brick
constexpr int kRC = 16;          // density chunk width (one f16 K step)
constexpr long long kWaitNs = 2000000000LL;  // bounded mbarrier waits: 2 s
constexpr unsigned char kNoSlot = 255;
constexpr int kMmaWarp = 5;  // the warp that runs the density MMA loop (one elected lane issues)
constexpr float kFxScaleD = 1.f / 16.f;  // fixed-point D scale relative to the floating split's
constexpr uint32_t kHTail = 2048;  // >= 15 core matrices of 128 bytes read above the last local-H operand rows
// density phase B roles: epilogue groups of four warps (warps 0-3, 6-9), the MMA warp (5), and the
// prefetch warps (10-15, 4) that issue the bulk copies of the D chunks.  Orbital slots go to four
// slices of warps (warps 4q .. 4q+3 take slots q, q+4, ...), so the last slices have the fewest: the
// prefetch warps are taken from those.  Chunk k goes to the warp of prefetch index k mod 7 (the
// first chunks during the orbital evaluation, the others once their stage is free).
constexpr int kEpiGroups = 2, kEpiWarps = 4 * kEpiGroups;
__device__ __forceinline__ int prefetch_index(int warp) {  // -1: no prefetch chunk
  return warp >= 10 ? warp - 10 : warp == 4 ? 6 : -1;
}
__device__ __forceinline__ int epi_group(int warp) {  // -1: not an epilogue warp
  return warp < 4 ? 0 : (warp >= 6 && warp < 6 + 4 * (kEpiGroups - 1)) ? 1 + ((warp - 6) >> 2) : -1;
}

// ------------------------------------------------------------------------------ PTX wrappers
// (gint_ptx.cuh) with this file's bounded-wait limit and error bit
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned *err) {
  return gptx::mbar_wait(bar, parity, err, GINT_ERRBIT_TIMEOUT, kWaitNs);
}
// Named barrier 1 over the density epilogue warps (barrier 0 is __syncthreads).
__device__ __forceinline__ void epi_barrier() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory"); }

// x = hi + lo with both parts float16 (hi = round(x), lo = round(x - hi)), two values at once
// (packed float32x2 -> float16x2 round-to-nearest conversions): hw, lw hold the hi and lo halves
// of a (low 16 bits) and b (high 16 bits).
__device__ __forceinline__ void split_h2(float a, float b, uint32_t &hw, uint32_t &lw) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
  hw = *reinterpret_cast<const uint32_t *>(&h);
  lw = *reinterpret_cast<const uint32_t *>(&l);
}

// Fixed-point split (force pass): hi = the nearest integer (|x| <= 2048, exact in float16), lo =
// round(x - hi), |lo| <= 1/2.  Every hi * hi product is then an integer, so as long as the partial
// sums stay below 2^24 the tensor core's float32 accumulation of the hi * hi products is exact (no
// bits fall below the accumulator's last place, whatever its rounding).  The lo parts carry the rest
// to float16 precision; all three products with a lo factor go to a separate accumulator whose
// values are about 2^-10 of the main one, where rounding is negligible.
__device__ __forceinline__ void split_fx2(float a, float b, uint32_t &hw, uint32_t &lw) {
  const float ha = rintf(a), hb = rintf(b);
  const __half2 h = __floats2half2_rn(ha, hb);
  const __half2 l = __floats2half2_rn(a - ha, b - hb);
  hw = *reinterpret_cast<const uint32_t *>(&h);
  lw = *reinterpret_cast<const uint32_t *>(&l);
}

// ------------------------------------------------------------------------------ orbital evaluation
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// r = |dh + dl| as a double-float (rh, rl) and 1/rh; at0 when the point is on the atom.
__device__ __forceinline__ void dist_df(const float dh[3], const float dl[3], float &rh, float &rl, float &ir,
                                        bool &at0) {
  const float px = dh[0] * dh[0], py = dh[1] * dh[1], pz = dh[2] * dh[2];
  const float ex = fmaf(dh[0], dh[0], -px), ey = fmaf(dh[1], dh[1], -py), ez = fmaf(dh[2], dh[2], -pz);
  float s1, e1, s2, e2;
  two_sum(px, py, s1, e1);
  two_sum(s1, pz, s2, e2);
  float r2l = (ex + ey + ez) + (e1 + e2) + 2.f * (dh[0] * dl[0] + dh[1] * dl[1] + dh[2] * dl[2]);
  const float r2h = s2 + r2l;
  r2l = r2l - (r2h - s2);
  at0 = r2h < 1e-24f;
  rh = at0 ? 0.f : sqrtf(r2h);
  ir = at0 ? 0.f : 1.f / rh;
  rl = at0 ? 0.f : (fmaf(-rh, rh, r2h) + r2l) * (0.5f * ir);
}

// Knot index i and parameter t in [0,1) of r = rh + rl on a grid of spacing 1/idr (exact index,
// t accurate to float32 rounding).  Returns false beyond the table.
__device__ __forceinline__ bool knot_df(const GRadial &R, float rh, float rl, int &i, float &t) {
  const float xh = rh * R.idr_hi;
  const float xl = fmaf(rh, R.idr_hi, -xh) + (rl * R.idr_hi + rh * R.idr_lo);
  i = (int)floorf(xh);
  t = (xh - (float)i) + xl;
  if (t < 0.f) {
    i -= 1;
    t += 1.f;
  } else if (t >= 1.f) {
    i += 1;
    t -= 1.f;
  }
  if (i < 0) {
    i = 0;
    t = 0.f;
  }
  return i < R.npts - 1;
}

// Cubic Hermite basis in t: value weights (s = h01, c0 = h10, c1 = h11; h00 = 1 - s) and derivative
// weights (ds = dh01/dt, d0 = dh10/dt, d1 = dh11/dt).
struct Basis {
  float s, c0, c1, ds, d0, d1;
};
__device__ __forceinline__ Basis hermite_basis(float t) {
  Basis B;
  const float t2 = t * t, u = 1.f - t;
  B.s = t2 * (3.f - 2.f * t);
  B.c0 = t * u * u;
  B.c1 = t2 * (t - 1.f);
  B.ds = 6.f * t * u;
  B.d0 = u * (1.f - 3.f * t);
  B.d1 = t * (3.f * t - 2.f);
  return B;
}
// dtab (may be NULL): knot differences formed in float64 (accurate derivatives; see the handle)
__device__ __forceinline__ void radial_at(const float2 *__restrict__ tab, const float *__restrict__ dtab,
                                          const GRadial &R, int i, const Basis &B, float &f, float &df) {
  const float2 a = tab[R.off + i], b = tab[R.off + i + 1];
  const float dlt = dtab ? dtab[R.off + i] : b.x - a.x;
  f = a.x + dlt * B.s + R.dr_f * (a.y * B.c0 + b.y * B.c1);
  df = (dlt * B.ds + R.dr_f * (a.y * B.d0 + b.y * B.d1)) * R.idr_hi;
}

// Generic path (any radial order or knot grids): adds one image to v[col] (+ gv[3 col + c]).
template <bool GRAD>
__device__ void add_image_generic(const GTabs &g, const float2 *__restrict__ tab, const float *__restrict__ dtab,
                                  const GSpecies &S, const float dh[3], const float dl[3], float *v, float *gv) {
  float r, rl, ir;
  bool at0;
  dist_df(dh, dl, r, rl, ir, at0);
  const float ux = dh[0] * ir, uy = dh[1] * ir, uz = dh[2] * ir;
  int col = 0;
  for (int k = 0; k < S.nrad; ++k) {
    const GRadial &R = g.rad[S.rad0 + k];
    const int l = R.l, nm = 2 * l + 1;
    int i;
    float t;
    if (r < R.rc_f && knot_df(R, r, rl, i, t)) {
      float f, df;
      radial_at(tab, GRAD ? dtab : nullptr, R, i, hermite_basis(t), f, df);
      if (at0) {
        if (l == 0) v[col] += f * 0.28209479177387814347f;
        if (GRAD && l == 1) {
          const float c = 0.48860251190291992159f * df;
          gv[3 * (col + 0) + 2] += c;
          gv[3 * (col + 1) + 0] += c;
          gv[3 * (col + 2) + 1] += c;
        }
      } else {
        float y[5], gy[5][3];
        ylm_unit<float>(l, ux, uy, uz, y, gy);
        const float fr = f * ir;
        for (int m = 0; m < nm; ++m) {
          v[col + m] += f * y[m];
          if (GRAD) {
            const float a = df * y[m] - (float)l * fr * y[m];
            gv[3 * (col + m) + 0] += a * ux + fr * gy[m][0];
            gv[3 * (col + m) + 1] += a * uy + fr * gy[m][1];
            gv[3 * (col + m) + 2] += a * uz + fr * gy[m][2];
          }
        }
      }
    }
    col += nm;
  }
}

// Fast path for l-sorted species (NS s, NP p, ND d radials) on one knot grid: one knot/basis
// computation per image, the knot pair of every radial from the interleaved table (tabi: a few
// 16-byte loads), all column indices static (register arrays).
template <int NS, int NPR, int ND, bool GRAD>
__device__ __forceinline__ void add_image_fast(const GTabs &g, const float2 *__restrict__ tabi,
                                               const float *__restrict__ dtabi, const GSpecies &S, const float dh[3],
                                               const float dl[3], float *v, float *gv) {
  constexpr int NR = NS + NPR + ND, KS = (NR + 1) & ~1;
  float r, rl, ir;
  bool at0;
  dist_df(dh, dl, r, rl, ir, at0);
  const GRadial &R0 = g.rad[S.rad0];
  int i;
  float t;
  if (!knot_df(R0, r, rl, i, t)) return;
  const Basis B = hermite_basis(t);
  // (f, f') at knots i and i + 1: preloaded for values only; with gradients (more live registers)
  // each radial's pair is loaded where it is used
  const float2 *q2 = tabi + S.ioff + (long long)i * KS;
  float2 ka[GRAD ? 1 : KS], kb[GRAD ? 1 : KS];
  if (!GRAD) {
    const float4 *q = reinterpret_cast<const float4 *>(q2);
#pragma unroll
    for (int h = 0; h < KS / 2; ++h) {
      const float4 x = __ldg(q + h), y = __ldg(q + KS / 2 + h);
      ka[2 * h] = make_float2(x.x, x.y);
      ka[2 * h + 1] = make_float2(x.z, x.w);
      kb[2 * h] = make_float2(y.x, y.y);
      kb[2 * h + 1] = make_float2(y.z, y.w);
    }
  }
  const float drf = R0.dr_f, idr = R0.idr_hi;  // shared knot grid
  // with gradients the knot difference comes from the float64-formed table (values alone: the
  // difference of the two float32 knot values is accurate enough)
  const float *qd = GRAD ? dtabi + S.ioff + (long long)i * KS : nullptr;
  auto radial_k = [&](int k, float &f, float &df) {
    const float2 a = GRAD ? __ldg(q2 + k) : ka[GRAD ? 0 : k], b = GRAD ? __ldg(q2 + KS + k) : kb[GRAD ? 0 : k];
    const float dlt = GRAD ? __ldg(qd + k) : b.x - a.x;
    f = a.x + dlt * B.s + drf * (a.y * B.c0 + b.y * B.c1);
    df = (dlt * B.ds + drf * (a.y * B.d0 + b.y * B.d1)) * idr;
  };
  const float ux = dh[0] * ir, uy = dh[1] * ir, uz = dh[2] * ir;
  const float Y0 = 0.28209479177387814347f;
  float y1[3], gy1[3][3], y2[5], gy2[5][3];
  if (NPR > 0) ylm_unit<float>(1, ux, uy, uz, y1, gy1);
  if (ND > 0) ylm_unit<float>(2, ux, uy, uz, y2, gy2);
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const GRadial &R = g.rad[S.rad0 + k];
    if (r < R.rc_f) {
      float f, df;
      radial_k(k, f, df);
      v[k] += f * Y0;
      if (GRAD && !at0) {
        const float a = df * Y0;
        gv[3 * k + 0] += a * ux;
        gv[3 * k + 1] += a * uy;
        gv[3 * k + 2] += a * uz;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NPR; ++k) {
    const GRadial &R = g.rad[S.rad0 + NS + k];
    const int col = NS + 3 * k;
    if (r < R.rc_f) {
      float f, df;
      radial_k(NS + k, f, df);
      if (at0) {
        if (GRAD) {
          const float c = 0.48860251190291992159f * df;
          gv[3 * (col + 0) + 2] += c;
          gv[3 * (col + 1) + 0] += c;
          gv[3 * (col + 2) + 1] += c;
        }
      } else {
        const float fr = f * ir;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          v[col + m] += f * y1[m];
          if (GRAD) {
            const float a = df * y1[m] - fr * y1[m];
            gv[3 * (col + m) + 0] += a * ux + fr * gy1[m][0];
            gv[3 * (col + m) + 1] += a * uy + fr * gy1[m][1];
            gv[3 * (col + m) + 2] += a * uz + fr * gy1[m][2];
          }
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    const GRadial &R = g.rad[S.rad0 + NS + NPR + k];
    const int col = NS + 3 * NPR + 5 * k;
    if (r < R.rc_f && !at0) {
      float f, df;
      radial_k(NS + NPR + k, f, df);
      const float fr = f * ir;
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        v[col + m] += f * y2[m];
        if (GRAD) {
          const float a = df * y2[m] - 2.f * fr * y2[m];
          gv[3 * (col + m) + 0] += a * ux + fr * gy2[m][0];
          gv[3 * (col + m) + 1] += a * uy + fr * gy2[m][1];
          gv[3 * (col + m) + 2] += a * uz + fr * gy2[m][2];
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------ brick metadata
constexpr int kMaxStages = 6;
constexpr int kPrefetchWarps = 7;  // warps 10-15 and 4
static_assert(kMaxStages <= kPrefetchWarps, "one prefetch warp per prefetched stage");
constexpr int kMaxChunks = kNPMAX / kRC;
constexpr int kPlanWords = 1536;  // prefetch buffer of a brick plan record (6 KB); larger records take the slow path
struct BrickSh {
  uint64_t full[kMaxStages];  // density: B stage loaded (bulk-copy transactions)
  uint64_t done[kMaxChunks];  // density: MMAs of chunk c complete (one use per brick)
  uint64_t hdone[2];          // local H: MMAs of a stage complete
  uint64_t hbuilt[2];         // local H: W P block of a stage written (one arrival per builder warp)
  uint32_t tmem;
  int item, na, np, nent, abort;
  int s_atom[kMAXA], s_no[kMAXA], s_po[kMAXA], s_sp[kMAXA], s_pcol[kMAXA], s_e0[kMAXA + 1];
  int s_cumno[kMAXA + 1];       // prefix of norb over slots (local-H scratch layout)
  int s_rowst[kMAXA + 1];       // local-H scratch: first element of slot a's row of tiles; [na]: the total
  int s_tile[kMAXA * kMAXA];    // D tile element offset of (row slot b, K slot a), -1 if none
  float e_hi[kMAXE][3], e_lo[kMAXE][3];  // entry positions relative to the brick origin
  float pt_hi[128][3], pt_lo[128][3];    // grid point positions relative to the brick origin
  unsigned char col2slot[kNPMAX];
  double fpart[kMAXA][3];
  union alignas(8) {
    float rpart[4][128];  // density / force epilogues, fixed-point rows: per-slice partials of a point
    // local-H epilogue (after those): per 8-column group h of the padded columns, (dense index of
    // its first column among the brick's orbitals) << 4 | (its real columns), or -1 for padding
    int hcol[kNPMAX / 8];
  };
  union {
    float rpartl[4][128];  // density epilogue: compensation terms of the groups' partial sums
    double vd[128];        // V at the brick's points, copied asynchronously (formed into wv after the
                           // orbitals, before the density epilogue uses rpartl)
  };
  float wv[128];   // w V at the brick's points (local H, force)
  float rsc[128];  // force launches: power-of-two scale of each row of P (fixed-point split)
  double ob[3];    // brick origin (Cartesian)
  float sc[4];     // scales
  uint64_t plan_bar;  // the next item's plan record has landed in planbuf
  int plan_pref;      // 1 if planbuf is being filled for the next item
  alignas(16) uint32_t planbuf[kPlanWords];
};

__device__ __forceinline__ void split2(double v, float &hi, float &lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

__device__ void init_points(const GCell &g, BrickSh &sh) {
  for (int p = threadIdx.x; p < 128; p += blockDim.x) {
    const int pi = p >> 5, pj = (p >> 3) & 3, pk = p & 7;
    for (int c = 0; c < 3; ++c) {
      const double v =
          (double)pi / g.n1 * g.cell[c] + (double)pj / g.n2 * g.cell[3 + c] + (double)pk / g.n3 * g.cell[6 + c];
      split2(v, sh.pt_hi[p][c], sh.pt_lo[p][c]);
    }
  }
}

// Padded column layout of the brick's slots: 8-aligned, never crossing a multiple of 128.
// Shared by the device kernels and the host preparation (identical integer arithmetic).
__host__ __device__ __forceinline__ int place_slot(int cur, int po) {
  int pc = (cur + 7) & ~7;
  if ((pc & 127) + po > 128) pc = (pc + 127) & ~127;
  return pc;
}

// Loads slots, entries, padded layout, tile table, local-H tile offsets.
__device__ void load_brick(const GCell &g, const GTabs &tb, const GNbr &nb, const long long *__restrict__ tile_off,
                           long long b, BrickSh &sh) {
  const int t = threadIdx.x;
  if (t == 0) {  // brick origin, once per brick (float64 division is slow on this GPU)
    const int bk = (int)(b % g.nbk), bj = (int)((b / g.nbk) % g.nbj), bi = (int)(b / ((long long)g.nbk * g.nbj));
    grid_point(g, bi * GINT_BI, bj * GINT_BJ, bk * GINT_BK, sh.ob);
  }
  const long long s0 = nb.b_at_off[b];
  const int na = (int)(nb.b_at_off[b + 1] - s0);
  const long long e_begin = nb.s_ent[s0], e_end = nb.s_ent[s0 + na];
  const int nent = (int)(e_end - e_begin);
  for (int a = t; a < na; a += blockDim.x) {
    const int I = nb.s_atom[s0 + a], sp = nb.atom_species[I];
    sh.s_atom[a] = I;
    sh.s_sp[a] = sp;
    sh.s_no[a] = tb.sp[sp].norb;
    sh.s_po[a] = tb.sp[sp].porb;
    sh.s_e0[a] = (int)(nb.s_ent[s0 + a] - e_begin);
    sh.fpart[a][0] = sh.fpart[a][1] = sh.fpart[a][2] = 0.0;
  }
  for (int k = t; k < kNPMAX; k += blockDim.x) sh.col2slot[k] = kNoSlot;
  __syncthreads();
  // entry positions relative to the brick origin (one (entry, axis) per thread; thread 0 is busy below)
  for (int u = t - 1; u >= 0 && u < 3 * nent; u += blockDim.x - 1) {
    const int e = u / 3, c = u - 3 * (u / 3);
    split2(nb.e_shift[3 * (e_begin + e) + c] - sh.ob[c], sh.e_hi[e][c], sh.e_lo[e][c]);
  }
  if (t == 0) {
    sh.na = na;
    sh.nent = nent;
    sh.s_e0[na] = nent;
    int cur = 0, cum = 0;
    for (int a = 0; a < na; ++a) {
      const int pc = place_slot(cur, sh.s_po[a]);
      sh.s_pcol[a] = pc;
      cur = pc + sh.s_po[a];
      sh.s_cumno[a] = cum;
      cum += sh.s_no[a];
    }
    sh.s_cumno[na] = cum;
    sh.np = (cur + 15) & ~15;
    int rs = 0;
    for (int a = 0; a < na; ++a) {
      sh.s_rowst[a] = rs;
      rs += sh.s_no[a] * (cum - sh.s_cumno[a]);
    }
    sh.s_rowst[na] = rs;
  }
  __syncthreads();
  const long long pbase = nb.b_pair_off[b];
  for (int e = t; e < na * na; e += blockDim.x) {
    const int p = nb.b_pair[pbase + e];  // row slot e / na, column slot e % na
    sh.s_tile[e] = p < 0 ? -1 : (int)tile_off[p];
  }
  for (int a = t; a < na; a += blockDim.x)
    for (int i = 0; i < sh.s_po[a]; ++i) sh.col2slot[sh.s_pcol[a] + i] = (unsigned char)a;
  __syncthreads();
}

// Plan record of a brick (built once per geometry from load_brick's result, 32-bit words):
//   [0] na  [1] nent  [2] np  [3] cumulative norb of all slots
//   [4 + 8a + k], k = 0..7: atom, species, norb, porb, pcol, first entry, cumno, rowst of slot a
//   [4 + 8 na + 6 e + c]: entry e, c < 3: hi part of axis c, c >= 3: lo part (float bits)
//   then na * na tile offsets, then np bytes of the column -> slot map; padded to 16 bytes.
__host__ __device__ __forceinline__ long long plan_words(int na, int nent, int np) {
  const long long w = 4 + 8LL * na + 6LL * nent + (long long)na * na + (np + 3) / 4;
  return (w + 3) & ~3LL;
}

// Unpacks the record in sh.planbuf into the brick metadata (all threads; ends with a barrier).
// wait_store: thread 0 also waits, before the closing barrier, until the previous item's bulk store
// of local-H tiles has read shared memory (overlapping that store with the unpack).
__device__ void unpack_plan(BrickSh &sh, bool wait_store = false) {
  const int t = threadIdx.x, nt = blockDim.x;
  const uint32_t *w = sh.planbuf;
  const int na = (int)w[0], nent = (int)w[1], np = (int)w[2];
  for (int a = t; a < na; a += nt) {
    const uint32_t *q = w + 4 + 8 * a;
    sh.s_atom[a] = (int)q[0];
    sh.s_sp[a] = (int)q[1];
    sh.s_no[a] = (int)q[2];
    sh.s_po[a] = (int)q[3];
    sh.s_pcol[a] = (int)q[4];
    sh.s_e0[a] = (int)q[5];
    sh.s_cumno[a] = (int)q[6];
    sh.s_rowst[a] = (int)q[7];
    sh.fpart[a][0] = sh.fpart[a][1] = sh.fpart[a][2] = 0.0;
  }
  if (t == 0) {
    sh.na = na;
    sh.nent = nent;
    sh.np = np;
    sh.s_e0[na] = nent;
    sh.s_cumno[na] = (int)w[3];
    sh.s_rowst[na] = na > 0 ? (int)w[4 + 8 * (na - 1) + 7] + (int)w[4 + 8 * (na - 1) + 2] * ((int)w[3] - (int)w[4 + 8 * (na - 1) + 6]) : 0;
  }
  const int eb = 4 + 8 * na;
  for (int u = t; u < 6 * nent; u += nt) {
    const int e = u / 6, c = u - 6 * e;
    const float v = __uint_as_float(w[eb + u]);
    if (c < 3)
      sh.e_hi[e][c] = v;
    else
      sh.e_lo[e][c - 3] = v;
  }
  const int tb = eb + 6 * nent;
  for (int i = t; i < na * na; i += nt) sh.s_tile[i] = (int)w[tb + i];
  const unsigned char *cb = reinterpret_cast<const unsigned char *>(w + tb + na * na);
  for (int k = t; k < kNPMAX; k += nt) sh.col2slot[k] = k < np ? cb[k] : kNoSlot;
  if (wait_store && t == 0) bulk_wait_read();
  __syncthreads();
}

// Grid point position relative to the brick origin as a double-float (held in registers).
struct PointDF {
  float h[3], l[3];
};
__device__ __forceinline__ PointDF point_df(const BrickSh &sh, int p) {
  PointDF P;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    P.h[c] = sh.pt_hi[p][c];
    P.l[c] = sh.pt_lo[p][c];
  }
  return P;
}
__device__ __forceinline__ void rel_disp_df(const BrickSh &sh, const PointDF &P, int e, float dh[3], float dl[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float s, err;
    two_sum(P.h[c], -sh.e_hi[e][c], s, err);
    const float lo = err + (P.l[c] - sh.e_lo[e][c]);
    dh[c] = s + lo;
    dl[c] = lo - (dh[c] - s);
  }
}

// Periodised orbitals (all images) of slot a at local point p: v[PO] (+ gv[3 PO]), zero based.
template <int NS, int NPR, int ND, bool GRAD>
__device__ __forceinline__ void slot_values(const GTabs &g, const float2 *__restrict__ tab,
                                            const float *__restrict__ dtab, const BrickSh &sh, int a,
                                            const PointDF &P, bool valid, float *v, float *gv) {
  constexpr int PO = (NS + 3 * NPR + 5 * ND + 7) / 8 * 8;
#pragma unroll
  for (int i = 0; i < PO; ++i) {
    v[i] = 0.f;
    if (GRAD) gv[3 * i] = gv[3 * i + 1] = gv[3 * i + 2] = 0.f;
  }
  if (!valid) return;
  const GSpecies &S = g.sp[sh.s_sp[a]];
  const float rc2 = S.rcut2f;
  for (int e = sh.s_e0[a]; e < sh.s_e0[a + 1]; ++e) {
    float dh[3], dl[3];
    rel_disp_df(sh, P, e, dh, dl);
    if (dh[0] * dh[0] + dh[1] * dh[1] + dh[2] * dh[2] < rc2) {
      if (NS + NPR + ND > 0)
        add_image_fast<NS, NPR, ND, GRAD>(g, tab, dtab, S, dh, dl, v, gv);
      else
        add_image_generic<GRAD>(g, tab, dtab, S, dh, dl, v, gv);
    }
  }
}

// Species shapes with a static fast path; others use the generic evaluator (NS=NPR=ND=0).
#define GINT_FOR_SHAPES(X) X(2, 2, 1) X(2, 1, 0) X(1, 1, 1) X(1, 1, 0) X(1, 0, 0) X(3, 3, 2)

// --- per-atom jobs ---
// Density phase A: scaled orbitals of slot a at point p -> P row p, columns [pcol, pcol + PO).
template <int PO>
__device__ __forceinline__ void store_P(const float *v, int pc, int p, float Sphi, unsigned char *Ph,
                                        unsigned char *Pl, uint32_t sboP) {
#pragma unroll
  for (int k = 0; k < PO; k += 8) {
    uint32_t wh[4], wl[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      split_h2(v[k + 2 * e] * Sphi, v[k + 2 * e + 1] * Sphi, wh[e], wl[e]);
    }
    const uint32_t off = (p >> 3) * sboP + ((pc + k) >> 3) * 128 + (p & 7) * 16;
    *reinterpret_cast<uint4 *>(Ph + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    *reinterpret_cast<uint4 *>(Pl + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
  }
}
// Two atoms of the same shape at once (two independent evaluation chains per thread).
template <int NS, int NPR, int ND, int PO>
__device__ __forceinline__ void job_P2(const GTabs &g, const float2 *__restrict__ tab, const BrickSh &sh, int a0,
                                       int a1, const PointDF &P, int p, bool valid, float Sphi, unsigned char *Ph,
                                       unsigned char *Pl, uint32_t sboP) {
  float v0[PO], v1[PO];
  slot_values<NS, NPR, ND, false>(g, tab, nullptr, sh, a0, P, valid, v0, nullptr);
  slot_values<NS, NPR, ND, false>(g, tab, nullptr, sh, a1, P, valid, v1, nullptr);
  store_P<PO>(v0, sh.s_pcol[a0], p, Sphi, Ph, Pl, sboP);
  store_P<PO>(v1, sh.s_pcol[a1], p, Sphi, Ph, Pl, sboP);
}
template <int NS, int NPR, int ND, int PO>
__device__ __forceinline__ void job_P(const GTabs &g, const float2 *__restrict__ tab, const BrickSh &sh, int a,
                                      const PointDF &P, int p, bool valid, float Sphi, unsigned char *Ph,
                                      unsigned char *Pl, uint32_t sboP) {
  float v[PO];
  slot_values<NS, NPR, ND, false>(g, tab, nullptr, sh, a, P, valid, v, nullptr);
  store_P<PO>(v, sh.s_pcol[a], p, Sphi, Ph, Pl, sboP);
}

// Force epilogue: y[PO] (true Y values of slot a's columns) -> rho part and force components.
template <int NS, int NPR, int ND, int PO>
__device__ __forceinline__ void job_F(const GTabs &g, const float2 *__restrict__ tab, const float *__restrict__ dtab,
                                      const BrickSh &sh, int a, int p, bool valid, const float *y, float &rp, float &fx,
                                      float &fy, float &fz) {
  float v[PO], gv[3 * PO];
  slot_values<NS, NPR, ND, true>(g, tab, dtab, sh, a, point_df(sh, p), valid, v, gv);
#pragma unroll
  for (int i = 0; i < PO; ++i) {
    rp += v[i] * y[i];
    fx += gv[3 * i] * y[i];
    fy += gv[3 * i + 1] * y[i];
    fz += gv[3 * i + 2] * y[i];
  }
}

// Generic-shape jobs (any species up to GINT_MAX_ORB_ATOM orbitals).
__device__ __noinline__ void job_P_generic(const GTabs &g, const float2 *__restrict__ tab, const BrickSh &sh, int a,
                                           int p, bool valid, float Sphi, unsigned char *Ph,
                                           unsigned char *Pl, uint32_t sboP) {
  float v[GINT_MAX_ORB_ATOM];
  const int po = sh.s_po[a], pc = sh.s_pcol[a];
  for (int i = 0; i < po; ++i) v[i] = 0.f;
  if (valid) {
    const GSpecies &S = g.sp[sh.s_sp[a]];
    for (int e = sh.s_e0[a]; e < sh.s_e0[a + 1]; ++e) {
      float dh[3], dl[3];
      rel_disp_df(sh, point_df(sh, p), e, dh, dl);
      if (dh[0] * dh[0] + dh[1] * dh[1] + dh[2] * dh[2] < S.rcut2f)
        add_image_generic<false>(g, tab, nullptr, S, dh, dl, v, nullptr);
    }
  }
  for (int k = 0; k < po; k += 8) {
    uint32_t wh[4], wl[4];
    for (int e = 0; e < 4; ++e) {
      split_h2(v[k + 2 * e] * Sphi, v[k + 2 * e + 1] * Sphi, wh[e], wl[e]);
    }
    const uint32_t off = (p >> 3) * sboP + ((pc + k) >> 3) * 128 + (p & 7) * 16;
    *reinterpret_cast<uint4 *>(Ph + off) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    *reinterpret_cast<uint4 *>(Pl + off) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
  }
}
__device__ __noinline__ void job_F_generic(const GTabs &g, const float2 *__restrict__ tab,
                                           const float *__restrict__ dtab, const BrickSh &sh, int a, int p, bool valid,
                                           const float *y, float &rp, float &fx, float &fy, float &fz) {
  float v[GINT_MAX_ORB_ATOM], gv[3 * GINT_MAX_ORB_ATOM];
  const int no = sh.s_no[a];
  for (int i = 0; i < no; ++i) v[i] = gv[3 * i] = gv[3 * i + 1] = gv[3 * i + 2] = 0.f;
  if (valid) {
    const GSpecies &S = g.sp[sh.s_sp[a]];
    for (int e = sh.s_e0[a]; e < sh.s_e0[a + 1]; ++e) {
      float dh[3], dl[3];
      rel_disp_df(sh, point_df(sh, p), e, dh, dl);
      if (dh[0] * dh[0] + dh[1] * dh[1] + dh[2] * dh[2] < S.rcut2f)
        add_image_generic<true>(g, tab, dtab, S, dh, dl, v, gv);
    }
  }
  for (int i = 0; i < no; ++i) {
    rp += v[i] * y[i];
    fx += gv[3 * i] * y[i];
    fy += gv[3 * i + 1] * y[i];
    fz += gv[3 * i + 2] * y[i];
  }
}

// Zero fill of the padding gap in front of slot a (density P rows / local-H operand rows).
__device__ __forceinline__ int gap_begin(const BrickSh &sh, int a) {
  return a == 0 ? 0 : sh.s_pcol[a - 1] + sh.s_po[a - 1];
}

// ------------------------------------------------------------------------------ batch descriptors
// Several systems share one persistent launch.  They must have identical species/radial
// metadata (GTabs, a kernel parameter); everything else is per system.  Work items are the bricks
// of system 0, then those of system 1, ...; an item runs every pass its system asks for.
constexpr int kMaxBatch = 32;

struct GSys {
  GCell c;
  GNbr nb;
  const float2 *tab;                         // float32 knot table of this system's handle
  const float2 *tabi;                        // its interleaved copy (shaped species)
  const float *dtab, *dtabi;                 // knot differences formed in float64 (gradients)
  const __half *Dhl, *Dhl2;                 // D tiles, hi and lo 8 x 8 blocks interleaved (and halved)
  const long long *tile_off;
  const float *scales;                       // [0] S_phi, [1] S_D, [2] S_Q
  const double *V;                           // NULL: no local-H items, zero force weight
  double *rho, *F;                           // NULL: not written
  const long long *hs_brick_off;
  float *hs;                                 // local-H scratch tiles
  unsigned *err;                             // device error word of the handle
  const uint4 *plan;                         // brick plan records (NULL: metadata built per item)
  const long long *plan_off;                 // [nbricks + 1] record offsets in 16-byte units
  int do_rho, do_h;                          // passes of this system's brick items
};

struct GBatch {
  int nsys, np_max, split3;
  int dsmem;                       // dynamic shared memory of the launch (bytes)
  long long start[kMaxBatch + 1];  // first item of each system; start[nsys] = total
  GSys sys[kMaxBatch];
};

// System owning item `it` (largest s with start[s] <= it; systems without items are skipped).
__device__ __forceinline__ int batch_sys(const GBatch &B, long long it) {
  int lo = 0, hi = B.nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.start[mid] <= it)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------------------ brick kernel
// One persistent CTA per SM walks the batch's items.  Dynamic shared memory, laid out per item for
// the item's padded width NP:
//   density: P (hi, lo) [128 x NP] | nst x B stage [NP x 16] (hi and lo interleaved), nst = as many as
//     fit, up to kMaxStages
//     P element (p, k): (p/8)*16*NP + (k/8)*128 + (p%8)*16 + (k%8)*2
//     B element (r, j) of part h (0 hi, 1 lo): (r/8)*512 + (j/8)*256 + h*128 + (r%8)*16 + (j%8)*2
//     (the layout of a row group of a 16-column tile in the interleaved tile store)
//   local H: two blocks of W P (hi, lo), hkb points x NP each, in the stage region, with the P layout;
//     the last 128-row A tile reads up to kHTail bytes above them (rows above NP, whose outputs are
//     ignored); afterwards the whole region stages the brick's scratch tiles for one bulk store.
// FORCE: density items produce rho and forces (full Y); a system without F only gets rho.
// One brick item of the persistent kernels (its metadata already unpacked into sh, the per-point
// potential in sh.wv): orbitals, the density / force chunk stream and the local-H pass.  Dynamic
// shared memory, laid out for the item's padded width NP: P (hi, lo), then as many density stages
// (hi and lo of an NP x 16 panel each) as fit, up to kMaxStages (narrower bricks get more chunks in
// flight), then at least kHTail bytes.  cx carries the CTA's barrier phases across items.
struct ItemCtx {
  uint32_t fpar;  // bit s: phase parity of the next use of stage s (full[s])
  uint32_t dpar;  // bit c: phase parity of done[c] (used once per density brick that has a chunk c)
  uint32_t GH;    // local-H stages issued by this CTA
  bool ok;        // no bounded wait has given up
  bool vpend;     // V of the brick's points is wanted in sh.vd: orbital slice 3 (the last four warps)
                  // copies one value per thread asynchronously during the orbital phase
};
template <bool FORCE>
__device__ __forceinline__ void brick_body(const GTabs &g, const GSys &S, long long b, bool do_rho, bool do_h,
                                           int split3, int dsmem, const __half *__restrict__ zero, uint32_t tmem,
                                           BrickSh &sh, unsigned char *smem, ItemCtx &cx) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  uint32_t &fpar = cx.fpar, &dpar = cx.dpar, &GH = cx.GH;
  bool &ok = cx.ok;
  const int na = sh.na, NP = sh.np;
  // force launches with the three-term split use a fixed-point split of P and D (exact hi * hi
  // accumulation, four products): D at 2^-4 of the floating split's scale (|hi| < 2048), and each
  // row of P (grid point) rescaled by its own power of two s_p so that its largest |value| lies in
  // [512, 1024)
  const bool fixp = FORCE && split3;
  const float Sphi = sh.sc[0];
  {
    // ================================================================ orbitals, density / force
    const float SD = fixp ? sh.sc[1] * kFxScaleD : sh.sc[1];
    const int p = t & 127, q = t >> 7;  // grid point, slot slice (0..3)
    const uint32_t lane_base = (uint32_t)((p >> 5) * 32) << 16;
    int gi, gj, gk;
    const bool valid = brick_point(S.c, b, p, gi, gj, gk);
    const long long gidx = valid ? grid_index(S.c, gi, gj, gk) : 0;
    if (na == 0) {
      if (cx.vpend && q == 3) cp_async_wait_all();  // no copy into sh.vd outlives the item
      if (do_rho && q == 0 && valid && S.rho) S.rho[gidx] = 0.0;
      return;
    }
    if (cx.vpend && q == 3) {  // V of this thread's point (slice 3 has the fewest atoms)
      if (valid)
        cp_async8(&sh.vd[p], S.V + gidx);
      else
        sh.vd[p] = 0.0;
    }
    const int nch = NP / kRC;
    const uint32_t sboP = 16u * (uint32_t)NP;  // P row-group stride
    unsigned char *const Ph = smem, *const Pl = smem + 128u * (uint32_t)NP * 2u;
    unsigned char *const B0 = smem + 128u * (uint32_t)NP * 4u;
    const uint32_t bop = (uint32_t)NP * kRC * 2u;  // one B operand (hi or lo) of one stage
    const int nst = min(kMaxStages, (int)(((uint32_t)dsmem - 128u * (uint32_t)NP * 4u - kHTail) / (2u * bop)));
  // bulk copies of chunk c's B tile (rows [rowbase, NP) x columns [16c, 16c+16)) into stage s
  auto issue_copies = [&](const GSys &S, int c, int s, int NP, int na) {
    const int rowbase = FORCE ? 0 : c * kRC;
    const int ngroups = (NP - rowbase) >> 3;
    if (lane == 0) mbar_arrive_tx(&sh.full[s], (uint32_t)ngroups * 512);  // the stage's one arrival
    __syncwarp();
    unsigned char *Bs = B0 + s * 2 * bop;
    const int ca = sh.col2slot[c * kRC];
    if (ca != kNoSlot && sh.s_po[ca] == 16 && sh.s_pcol[ca] == c * kRC) {
      // the chunk is one 16-column atom: a row group of the stage (512 bytes: segment-major pairs of
      // hi and lo 8 x 8 blocks) is laid out like a row group of a 16-column tile in the interleaved
      // store, so whole tiles copy as they are (hi and lo in one copy),
      // and slots that are adjacent in the brick's rows and in the column-atom-major tile store
      // form one copy.  Gap rows and absent tiles are zero-filled per row group.
      // one lane per slot (windows of 32 slots): a slot continues the previous slot's run if
      // both have present, non-diagonal tiles that are adjacent in rows and in the tile store
      auto zero_rows = [&](int r0, int r1) {
        for (int r = r0; r < r1; r += 8) bulk_g2s(Bs + (r - rowbase) * 64, zero, 512, &sh.full[s]);
      };
      for (int base = 0; base < na; base += 32) {
        const int bs = base + lane;
        const bool in = bs < na && sh.s_pcol[bs] >= rowbase;
        const int pc = in ? sh.s_pcol[bs] : 0, po = in ? sh.s_po[bs] : 0;
        const int tile = in ? sh.s_tile[bs * na + ca] : -1;
        const bool diag = !FORCE && bs == ca;
        const bool pin = in && bs > 0 && sh.s_pcol[bs - 1] >= rowbase;  // previous slot in the chunk rows
        const int ppc = pin ? sh.s_pcol[bs - 1] : 0, ppo = pin ? sh.s_po[bs - 1] : 0;
        const int ptile = pin ? sh.s_tile[(bs - 1) * na + ca] : -1;
        const bool pdiag = !FORCE && bs - 1 == ca;
        const bool run_ok = in && tile >= 0 && !diag;
        const bool cont = run_ok && lane > 0 && pin && ptile >= 0 && !pdiag && ppc + ppo == pc &&
                          (long long)ptile + (long long)ppo * 16 == (long long)tile;
        const unsigned brk = __ballot_sync(0xffffffffu, !cont);  // run boundaries (and non-slots)
        const int endrow = pc + po;
        if (in) {
          const int gap0 = pin ? ppc + ppo : rowbase;  // rows of no slot in front of this one
          if (pc > gap0) zero_rows(gap0, pc);
          if (bs == na - 1 && endrow < NP) zero_rows(endrow, NP);  // tail rows
          if (tile < 0) {
            zero_rows(pc, endrow);
          } else if (diag) {  // the chunk's own block: halved tiles
            bulk_g2s(Bs + (pc - rowbase) * 64, S.Dhl2 + 2 * (long long)tile, (uint32_t)po * 64, &sh.full[s]);
          }
        }
        // the last slot of a run ends where the next boundary starts
        const unsigned later = lane < 31 ? (brk >> (lane + 1)) : 0u;
        const int last = later ? lane + __ffs(later) - 1 : 31;
        const int run_end = __shfl_sync(0xffffffffu, endrow, last);
        if (run_ok && !cont) {
          bulk_g2s(Bs + (pc - rowbase) * 64, S.Dhl + 2 * (long long)tile, (uint32_t)(run_end - pc) * 64, &sh.full[s]);
        }
      }
      __syncwarp();
      return;
    }
    // general chunk (8-column atoms): one copy (hi and lo block) per row group and column segment
    for (int u = lane; u < ngroups * 2; u += 32) {
      const int gr = u >> 1, sg = u & 1;
      const int k0 = rowbase + 8 * gr, j0 = c * kRC + 8 * sg;
      const int bs = sh.col2slot[k0], as = sh.col2slot[j0];
      long long src = -1;
      if (bs != kNoSlot && as != kNoSlot) {
        const int tile = sh.s_tile[bs * na + as];
        const int kl0 = k0 - sh.s_pcol[bs];
        if (tile >= 0)
          src = (long long)tile + (long long)((kl0 >> 3) * (sh.s_po[as] >> 3) + ((j0 - sh.s_pcol[as]) >> 3)) * 64;
      }
      const bool diag = !FORCE && gr < 2;
      bulk_g2s(Bs + gr * 512 + sg * 256, src < 0 ? zero : (diag ? S.Dhl2 : S.Dhl) + 2 * src, 256u, &sh.full[s]);
    }
  };
    // chunk c uses stage c mod nst; its phase parity is that stage's next parity, flipped once per
    // earlier use of the stage in this item
    // the previous item's MMAs are complete: every stage is free, prefetch the first density chunks
    // (one chunk per prefetch warp: a warp issuing a chunk's bulk copies spends a sizeable part of
    // the orbital evaluation on it)
    if (do_rho) {
      const int li = prefetch_index(warp);
      if (li >= 0 && li < nch && li < nst) issue_copies(S, li, li, NP, na);
    }
    // ---- phase A: scaled orbitals of all atoms at every point -> P (hi, lo), zero padding
    for (int a = q; a < na; a += 4) {
      const int gap0 = gap_begin(sh, a), pc = sh.s_pcol[a];
      for (int k = gap0; k < pc; k += 8) {
        const uint32_t off = (p >> 3) * sboP + (k >> 3) * 128 + (p & 7) * 16;
        *reinterpret_cast<uint4 *>(Ph + off) = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(Pl + off) = make_uint4(0u, 0u, 0u, 0u);
      }
      if (a == na - 1)
        for (int k = pc + sh.s_po[a]; k < NP; k += 8) {
          const uint32_t off = (p >> 3) * sboP + (k >> 3) * 128 + (p & 7) * 16;
          *reinterpret_cast<uint4 *>(Ph + off) = make_uint4(0u, 0u, 0u, 0u);
          *reinterpret_cast<uint4 *>(Pl + off) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    {
      const float2 *tab = S.tab, *tabi = S.tabi;
      const PointDF P = point_df(sh, p);
      for (int a = q; a < na; a += 8) {
        const int a1 = a + 4;
        const int shp = g.sp[sh.s_sp[a]].shape;
        const bool pair = a1 < na && g.sp[sh.s_sp[a1]].shape == shp;
        switch (shp) {
#define CASE_P(ns, np_, nd)                                                                                      \
case GINT_SHAPE(ns, np_, nd):                                                                                \
  if (pair)                                                                                                  \
    job_P2<ns, np_, nd, (ns + 3 * np_ + 5 * nd + 7) / 8 * 8>(g, tabi, sh, a, a1, P, p, valid, Sphi, Ph, Pl, sboP); \
  else                                                                                                       \
    job_P<ns, np_, nd, (ns + 3 * np_ + 5 * nd + 7) / 8 * 8>(g, tabi, sh, a, P, p, valid, Sphi, Ph, Pl, sboP);    \
  break;
          GINT_FOR_SHAPES(CASE_P)
#undef CASE_P
          default:
            job_P_generic(g, tab, sh, a, p, valid, Sphi, Ph, Pl, sboP);
        }
        if (a1 < na && !(pair && shp != 0)) {
          switch (g.sp[sh.s_sp[a1]].shape) {
#define CASE_P1(ns, np_, nd)                                                                                      \
case GINT_SHAPE(ns, np_, nd):                                                                                 \
  job_P<ns, np_, nd, (ns + 3 * np_ + 5 * nd + 7) / 8 * 8>(g, tabi, sh, a1, P, p, valid, Sphi, Ph, Pl, sboP);    \
  break;
            GINT_FOR_SHAPES(CASE_P1)
#undef CASE_P1
            default:
              job_P_generic(g, tab, sh, a1, p, valid, Sphi, Ph, Pl, sboP);
          }
        }
      }
    }
    if (fixp) {
      // ---- fixed-point rows: s_p from the row's largest |value| (the four slices' maxima), then
      // every element x = (hi + lo) s_p re-split as hi = rint(x), lo = x - hi (float16)
      float m = 0.f;
      for (int a = q; a < na; a += 4)
        for (int k = sh.s_pcol[a]; k < sh.s_pcol[a] + sh.s_po[a]; k += 8) {
          const uint32_t off = (p >> 3) * sboP + (k >> 3) * 128 + (p & 7) * 16;
          const uint4 wh = *reinterpret_cast<const uint4 *>(Ph + off), wl = *reinterpret_cast<const uint4 *>(Pl + off);
          const uint32_t hw[4] = {wh.x, wh.y, wh.z, wh.w}, lw[4] = {wl.x, wl.y, wl.z, wl.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 hf = __half22float2(*reinterpret_cast<const __half2 *>(&hw[e]));
            const float2 lf = __half22float2(*reinterpret_cast<const __half2 *>(&lw[e]));
            m = fmaxf(m, fmaxf(fabsf(hf.x + lf.x), fabsf(hf.y + lf.y)));
          }
        }
      sh.rpart[q][p] = m;
      __syncthreads();
      const float rm = fmaxf(fmaxf(sh.rpart[0][p], sh.rpart[1][p]), fmaxf(sh.rpart[2][p], sh.rpart[3][p]));
      int ex = 0;
      frexpf(rm, &ex);  // rm = f 2^ex, f in [0.5, 1)
      const float sp = rm > 0.f ? ldexpf(1.f, 10 - ex) : 1.f;
      if (q == 0) sh.rsc[p] = sp;
      for (int a = q; a < na; a += 4)
        for (int k = sh.s_pcol[a]; k < sh.s_pcol[a] + sh.s_po[a]; k += 8) {
          const uint32_t off = (p >> 3) * sboP + (k >> 3) * 128 + (p & 7) * 16;
          const uint4 wh = *reinterpret_cast<const uint4 *>(Ph + off), wl = *reinterpret_cast<const uint4 *>(Pl + off);
          const uint32_t hw[4] = {wh.x, wh.y, wh.z, wh.w}, lw[4] = {wl.x, wl.y, wl.z, wl.w};
          uint32_t oh[4], ol[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 hf = __half22float2(*reinterpret_cast<const __half2 *>(&hw[e]));
            const float2 lf = __half22float2(*reinterpret_cast<const __half2 *>(&lw[e]));
            split_fx2((hf.x + lf.x) * sp, (hf.y + lf.y) * sp, oh[e], ol[e]);
          }
          *reinterpret_cast<uint4 *>(Ph + off) = make_uint4(oh[0], oh[1], oh[2], oh[3]);
          *reinterpret_cast<uint4 *>(Pl + off) = make_uint4(ol[0], ol[1], ol[2], ol[3]);
        }
    }
    if (cx.vpend && q == 3) {  // the copy has had the orbital phase to land
      cp_async_wait_all();
      sh.wv[p] = (float)(S.c.w * sh.vd[p]);
    }
    fence_async_smem();
    __syncthreads();
    if (do_rho) {
    // ---- phase B: chunks of 16 columns, prefetch warps / MMA thread / epilogue warps
    const uint32_t corr_base = (NP <= 256) ? 256u : 0u;  // separate correction accumulator if it fits
    if (warp == kMmaWarp) {
      if (NP <= 256 && split3 && corr_base) {
        // common case, straight-line issue (branches and descriptor rebuilds in this loop cost more
        // issue time than the MMAs take to run): the whole warp runs the loop and one elected lane
        // issues, the descriptors' start-address field (bytes / 16) advancing by constants, 256
        // bytes of P per chunk and 2 bop per stage.  The stage barrier orders the copies before the
        // MMAs; the epilogue's tensor-memory reads touch finished columns only, so one tcgen05
        // fence per item suffices.
        unsigned *errp = S.err;
        uint32_t s = 0, wrap = 0;
        const uint64_t dah0 = sdesc(smem_u32(Ph), 128, sboP), dal0 = sdesc(smem_u32(Pl), 128, sboP);
        const uint64_t dbh0 = sdesc(smem_u32(B0), 256, 512);
        const uint32_t sstep = (2 * bop) >> 4, lstep = 128 >> 4;
        tc_fence_after();  // after the barrier that ended the previous item's tensor-memory reads
        for (int c = 0; c < nch; ++c) {
          if (!mbar_wait(&sh.full[s], ((fpar >> s) & 1u) ^ wrap, errp)) ok = false;
          const uint32_t rowbase = FORCE ? 0u : (uint32_t)c * kRC;
          const uint32_t id = idesc_f16(128, NP - (int)rowbase), acc = c > 0 ? 1u : 0u;
          const uint64_t dah = dah0 + (uint64_t)(16 * c), dal = dal0 + (uint64_t)(16 * c);
          const uint64_t dbh = dbh0 + (uint64_t)(s * sstep), dbl = dbh + lstep;
          if (elect_one()) {
            mma_f16(tmem + rowbase, dah, dbh, id, acc);
            mma_f16(tmem + 256u + rowbase, dah, dbl, id, acc);
            mma_f16(tmem + 256u + rowbase, dal, dbh, id, 1u);
            if (FORCE) mma_f16(tmem + 256u + rowbase, dal, dbl, id, 1u);  // fixed-point split: lo * lo too
            mma_commit(&sh.done[c]);
          }
          __syncwarp();
          if (++s == (uint32_t)nst) {
            s = 0;
            wrap ^= 1u;
          }
        }
      } else if (lane == 0) {
        unsigned *errp = S.err;
        uint32_t s = 0, wrap = 0;  // stage of chunk c, and 1 once the stages have wrapped an odd number of times
        for (int c = 0; c < nch; ++c) {
          if (!mbar_wait(&sh.full[s], ((fpar >> s) & 1u) ^ wrap, errp)) ok = false;
          tc_fence_after();
          unsigned char *Bh = B0 + s * 2 * bop, *Bl = Bh + 128;
          const int rowbase = FORCE ? 0 : c * kRC;
          const int N = NP - rowbase;
          const uint64_t dah = sdesc(smem_u32(Ph) + (c * kRC / 8) * 128, 128, sboP);
          const uint64_t dal = sdesc(smem_u32(Pl) + (c * kRC / 8) * 128, 128, sboP);
          for (int n0 = 0; n0 < N; n0 += 256) {
            const int nn = min(256, N - n0);
            const uint32_t id = idesc_f16(128, nn);
            const uint64_t dbh = sdesc(smem_u32(Bh) + (n0 >> 3) * 512, 256, 512);
            const uint64_t dbl = sdesc(smem_u32(Bl) + (n0 >> 3) * 512, 256, 512);
            const uint32_t dm = tmem + rowbase + n0, dc = tmem + corr_base + rowbase + n0;
            mma_f16(dm, dah, dbh, id, c > 0 ? 1u : 0u);
            if (split3) {
              mma_f16(dc, dah, dbl, id, (c > 0 || corr_base == 0) ? 1u : 0u);
              mma_f16(dc, dal, dbh, id, 1u);
              if (fixp) mma_f16(dc, dal, dbl, id, 1u);
            }
          }
          mma_commit(&sh.done[c]);
          if (++s == (uint32_t)nst) {
            s = 0;
            wrap ^= 1u;
          }
        }
      }
      __syncwarp();
    } else if (prefetch_index(warp) >= 0) {
      // prefetch warps, later chunks: chunk k (k mod kPrefetchWarps = the warp's prefetch index),
      // its bulk copies issued once chunk k - nst's MMAs are done (the stage is free)
      unsigned *errp = S.err;
      const int li = prefetch_index(warp);
      for (int k = nst + ((li - nst) % kPrefetchWarps + kPrefetchWarps) % kPrefetchWarps; k < nch;
           k += kPrefetchWarps) {
        if (!mbar_wait(&sh.done[k - nst], (dpar >> (k - nst)) & 1u, errp)) ok = false;
        issue_copies(S, k, k % nst, NP, na);
      }
    } else if (!FORCE) {
      // density epilogue groups (each covers the 128 lanes) drain finished chunks round robin
      // (compensated float32 sums per point and group)
      const int grp = epi_group(warp);
      float rhi = 0.f, rlo = 0.f;
      for (int c = grp; c < nch; c += kEpiGroups) {
        if (!mbar_wait(&sh.done[c], (dpar >> c) & 1u, S.err)) ok = false;
        tc_fence_after();
        // chunk c's columns are final: rho += P_k Y_k
        const int k0 = c * kRC;
        float y[16], yc[16];
        if (split3 && corr_base) {
          tmem_ld16x2(tmem + lane_base + k0, tmem + lane_base + corr_base + k0, y, yc);
#pragma unroll
          for (int i = 0; i < 16; ++i) y[i] += yc[i];
        } else {
          tmem_ld16(tmem + lane_base + k0, y);
        }
        float part = 0.f;
#pragma unroll
        for (int hseg = 0; hseg < 2; ++hseg) {
          const uint32_t off = (p >> 3) * sboP + ((k0 >> 3) + hseg) * 128 + (p & 7) * 16;
          const uint4 wh = *reinterpret_cast<const uint4 *>(Ph + off), wl = *reinterpret_cast<const uint4 *>(Pl + off);
          const uint32_t hw[4] = {wh.x, wh.y, wh.z, wh.w}, lw[4] = {wl.x, wl.y, wl.z, wl.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 hf = __half22float2(*reinterpret_cast<const __half2 *>(&hw[e]));
            const float2 lf = __half22float2(*reinterpret_cast<const __half2 *>(&lw[e]));
            part += (hf.x + lf.x) * y[hseg * 8 + 2 * e] + (hf.y + lf.y) * y[hseg * 8 + 2 * e + 1];
          }
        }
        float sum, err;
        two_sum(rhi, part, sum, err);
        rhi = sum;
        rlo += err;
      }
      if (grp > 0) {
        sh.rpart[grp][p] = rhi;
        sh.rpartl[grp][p] = rlo;
      }
      epi_barrier();
      if (grp == 0) {
        for (int g2 = 1; g2 < kEpiGroups; ++g2) {
          float sum, err;
          two_sum(rhi, sh.rpart[g2][p], sum, err);
          rhi = sum;
          rlo += err + sh.rpartl[g2][p];
        }
        if (valid && S.rho)
          S.rho[gidx] = ((double)rhi + (double)rlo) * (2.0 / ((double)Sphi * (double)Sphi * (double)SD));
      }
    }
    // all MMAs of the brick are complete once the last chunk's barrier has flipped (in order)
    if (!mbar_wait(&sh.done[nch - 1], (dpar >> (nch - 1)) & 1u, S.err)) ok = false;
    tc_fence_after();
    for (int st = 0; st < nst && st < nch; ++st)  // stage st served chunks st, st + nst, ...
      if ((((nch - 1 - st) / nst) & 1) == 0) fpar ^= 1u << st;
    dpar ^= (nch >= 32) ? 0xffffffffu : ((1u << nch) - 1u);
    if (FORCE) {
      // full Y: per atom, rho and force from recomputed phi and grad phi (unscaled float32)
      const float2 *tab = S.tab, *tabi = S.tabi;
      const float inv = 1.f / (Sphi * SD * (fixp ? sh.rsc[p] : 1.f));
      const float wv = (valid && S.V) ? sh.wv[p] : 0.f;
      float rp = 0.f;
      for (int a = q; a < na; a += 4) {
        const int pc = sh.s_pcol[a], po = sh.s_po[a];
        // the atom's own columns only (an 8-column atom may end the accumulator: a 16-column
        // load there would reach past the tensor-memory allocation)
        float y[GINT_MAX_ORB_ATOM], yc[16];
        for (int h = 0; h < po; h += 16) {
          if (po - h >= 16) {
            if (split3 && corr_base) {
              tmem_ld16x2(tmem + lane_base + pc + h, tmem + lane_base + corr_base + pc + h, y + h, yc);
#pragma unroll
              for (int i = 0; i < 16; ++i) y[h + i] += yc[i];
            } else {
              tmem_ld16(tmem + lane_base + pc + h, y + h);
            }
          } else {
            tmem_ld8(tmem + lane_base + pc + h, y + h);
            if (split3 && corr_base) {
              tmem_ld8(tmem + lane_base + corr_base + pc + h, yc);
#pragma unroll
              for (int i = 0; i < 8; ++i) y[h + i] += yc[i];
            }
          }
        }
        for (int i = 0; i < po; ++i) y[i] *= inv;
        float fx = 0.f, fy = 0.f, fz = 0.f;
        switch (g.sp[sh.s_sp[a]].shape) {
#define CASE_F(ns, np_, nd)                                                                          \
case GINT_SHAPE(ns, np_, nd):                                                                    \
  job_F<ns, np_, nd, (ns + 3 * np_ + 5 * nd + 7) / 8 * 8>(g, tabi, S.dtabi, sh, a, p, valid, y, rp, fx, fy, fz); \
  break;
          GINT_FOR_SHAPES(CASE_F)
#undef CASE_F
          default:
            job_F_generic(g, tab, S.dtab, sh, a, p, valid, y, rp, fx, fy, fz);
        }
        fx *= 2.f * wv;
        fy *= 2.f * wv;
        fz *= 2.f * wv;
        for (int o = 16; o > 0; o >>= 1) {
          fx += __shfl_xor_sync(0xffffffffu, fx, o);
          fy += __shfl_xor_sync(0xffffffffu, fy, o);
          fz += __shfl_xor_sync(0xffffffffu, fz, o);
        }
        if (lane == 0) {
          atomicAdd(&sh.fpart[a][0], (double)fx);
          atomicAdd(&sh.fpart[a][1], (double)fy);
          atomicAdd(&sh.fpart[a][2], (double)fz);
        }
      }
      sh.rpart[q][p] = rp;
      __syncthreads();
      if (q == 0 && valid && S.rho)
        S.rho[gidx] =
            (double)sh.rpart[0][p] + (double)sh.rpart[1][p] + (double)sh.rpart[2][p] + (double)sh.rpart[3][p];
      if (S.F)
        for (int a = t; a < na; a += kT) {
          const int I = sh.s_atom[a];
          atomicAdd(S.F + 3 * I + 0, sh.fpart[a][0]);
          atomicAdd(S.F + 3 * I + 1, sh.fpart[a][1]);
          atomicAdd(S.F + 3 * I + 2, sh.fpart[a][2]);
        }
    }
    }  // do_rho
    if (do_h) {
      // ================================================================ local H from P
      // H_mu,nu = sum_g (w V_g P_g,mu) P_g,nu: K = grid points in blocks of hkb, both operands
      // MN-major views of [point][orbital] buffers (P itself, and W P built per block in one of
      // two halves of the stage region, ping-pong with the MMAs of the previous block).  Warps
      // 1-15 build the blocks and warp 0 issues their MMAs, the two sides paced by mbarriers only
      // (hbuilt: a half has been written; hdone: its MMAs are complete and it may be rewritten), so
      // the builders run one block ahead of the MMAs without a CTA-wide barrier per block.
      tc_fence_before();  // the density part's tensor-memory reads are finished
      __syncthreads();
      tc_fence_after();
      for (int h8 = t; h8 < NP / 8; h8 += kT) {  // the epilogue's column table (read after the barriers below)
        const int cs = sh.col2slot[8 * h8];
        int v = -1;
        if (cs != kNoSlot) {
          const int j0 = 8 * h8 - sh.s_pcol[cs];
          if (j0 < sh.s_no[cs]) v = ((sh.s_cumno[cs] + j0) << 4) | min(8, sh.s_no[cs] - j0);
        }
        sh.hcol[h8] = v;
      }
      const float SA = sh.sc[2];
      const float out_scale = 1.f / (Sphi * SA);
      const float wscale = SA / Sphi;
      const int hkb = nst >= 4 ? 32 : 16, ng = NP >> 3;  // two halves of hkb x NP (hi, lo) fit the stages
      const uint32_t whalf = (uint32_t)hkb * 4u * (uint32_t)NP;  // hi and lo of one block
      const int ntile = (NP + 127) / 128;
      int tb[3] = {0, 0, 0}, T = 0;
      for (int m = 0; m < ntile; ++m) {
        tb[m] = T;
        T += NP - 128 * m;
      }
      const uint32_t corr_base = (2 * T <= 512) ? (uint32_t)T : 0u;
      for (int j = 0; j < 128 / hkb; ++j, ++GH) {
        const int hh = GH & 1;
        unsigned char *Wh = B0 + hh * whalf, *Wl = Wh + whalf / 2;
        const int p0 = j * hkb;
        if (warp != 0) {
        // the MMAs that last read this half (two blocks ago) are complete
        if (GH >= 2 && !mbar_wait(&sh.hdone[hh], ((GH - 2) >> 1) & 1, S.err)) ok = false;
        // warps 1-15 build the block while warp 0 may still be issuing the previous block's MMAs.
        // Unit u = (point octet, orbital group, point in octet) with the point fastest: eight
        // consecutive threads touch one 128-byte core-matrix row block (no bank conflicts).
        for (int u = t - 32; u < hkb * ng; u += kT - 32) {
          const int v8 = u >> 3, po8 = v8 / ng, gg = v8 - po8 * ng;
          const int pl = po8 * 8 + (u & 7), pt = p0 + pl;
          const uint32_t so = (pt >> 3) * sboP + gg * 128 + (pt & 7) * 16;
          const uint32_t dso = (pl >> 3) * sboP + gg * 128 + (pl & 7) * 16;
          const float f = fixp ? sh.wv[pt] * wscale / (sh.rsc[pt] * sh.rsc[pt]) : sh.wv[pt] * wscale;
          const uint4 wh = *reinterpret_cast<const uint4 *>(Ph + so), wl = *reinterpret_cast<const uint4 *>(Pl + so);
          const uint32_t hw[4] = {wh.x, wh.y, wh.z, wh.w}, lw[4] = {wl.x, wl.y, wl.z, wl.w};
          uint32_t oh[4], ol[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 hf = __half22float2(*reinterpret_cast<const __half2 *>(&hw[e]));
            const float2 lf = __half22float2(*reinterpret_cast<const __half2 *>(&lw[e]));
            split_h2((hf.x + lf.x) * f, (hf.y + lf.y) * f, oh[e], ol[e]);
          }
          *reinterpret_cast<uint4 *>(Wh + dso) = make_uint4(oh[0], oh[1], oh[2], oh[3]);
          *reinterpret_cast<uint4 *>(Wl + dso) = make_uint4(ol[0], ol[1], ol[2], ol[3]);
        }
        fence_async_smem();  // this thread's writes before the MMAs' (async-proxy) reads
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.hbuilt[hh]);
        } else {
        // warp 0: the block's W P is complete (every builder warp has arrived)
        if (!mbar_wait(&sh.hbuilt[hh], (GH >> 1) & 1, S.err)) ok = false;
        if (NP <= 256 && split3) {
          // common case, straight-line issue by an elected lane of warp 0 (which builds no block):
          // at most two 128-row tiles of one N <= 256 each; the descriptors' start-address field
          // advances by 2 sboP / 16 per K step of 16 points, and by 2048 / 16 from the first to the
          // second tile (orbitals 128-255, rows of A and columns of B)
          tc_fence_after();
          const uint64_t wh0 = sdesc(smem_u32(Wh), sboP, 128), wl0 = sdesc(smem_u32(Wl), sboP, 128);
          const uint32_t pofs = (uint32_t)(p0 >> 3) * sboP;
          const uint64_t ph0 = sdesc(smem_u32(Ph) + pofs, sboP, 128), pl0 = sdesc(smem_u32(Pl) + pofs, sboP, 128);
          const uint32_t kstep = (2u * sboP) >> 4;
          const uint32_t id0 = idesc_f16_mn(128, NP), id1 = idesc_f16_mn(128, NP > 128 ? NP - 128 : 16);
          const uint32_t m0 = tmem + (uint32_t)tb[0], m1 = tmem + (uint32_t)tb[1];
          const uint32_t c0 = m0 + corr_base, c1 = m1 + corr_base;
          if (elect_one()) {
            for (int ks = 0; ks < hkb / 16; ++ks) {
              const uint64_t ko = (uint64_t)ks * kstep;
              const bool first = (j == 0 && ks == 0);
              const uint32_t am = first ? 0u : 1u, ac = (first && corr_base) ? 0u : 1u;
              mma_f16(m0, wh0 + ko, ph0 + ko, id0, am);
              mma_f16(c0, wh0 + ko, pl0 + ko, id0, ac);
              mma_f16(c0, wl0 + ko, ph0 + ko, id0, 1u);
              if (NP > 128) {
                mma_f16(m1, wh0 + ko + 128u, ph0 + ko + 128u, id1, am);
                mma_f16(c1, wh0 + ko + 128u, pl0 + ko + 128u, id1, ac);
                mma_f16(c1, wl0 + ko + 128u, ph0 + ko + 128u, id1, 1u);
              }
            }
            mma_commit(&sh.hdone[hh]);
          }
          __syncwarp();
        } else if (lane == 0) {
          tc_fence_after();
          for (int ks = 0; ks < hkb / 16; ++ks) {
            const uint32_t kw = (uint32_t)(2 * ks) * sboP, kp = (uint32_t)((p0 >> 3) + 2 * ks) * sboP;
            for (int m = 0; m < ntile; ++m) {
              const uint64_t dah = sdesc(smem_u32(Wh) + kw + m * 16 * 128, sboP, 128);
              const uint64_t dal = sdesc(smem_u32(Wl) + kw + m * 16 * 128, sboP, 128);
              const int N = NP - 128 * m;
              for (int n0 = 0; n0 < N; n0 += 256) {
                const int nn = min(256, N - n0);
                const uint32_t id = idesc_f16_mn(128, nn);
                const uint32_t col = (uint32_t)(128 * m + n0);
                const uint64_t dbh = sdesc(smem_u32(Ph) + kp + (col >> 3) * 128, sboP, 128);
                const uint64_t dbl = sdesc(smem_u32(Pl) + kp + (col >> 3) * 128, sboP, 128);
                const uint32_t dm = tmem + tb[m] + n0, dc = tmem + corr_base + tb[m] + n0;
                const bool first = (j == 0 && ks == 0);
                mma_f16(dm, dah, dbh, id, first ? 0u : 1u);
                if (split3) {
                  mma_f16(dc, dah, dbl, id, (first && corr_base) ? 0u : 1u);
                  mma_f16(dc, dal, dbh, id, 1u);
                }
              }
            }
          }
          mma_commit(&sh.hdone[hh]);
        }
        __syncwarp();
        }
      }
      {
        const uint32_t Gp = GH - 1;
        if (!mbar_wait(&sh.hdone[Gp & 1], (Gp >> 1) & 1, S.err)) ok = false;
        tc_fence_after();
      }
      __syncthreads();  // every block built and its MMAs complete; the column table is visible
    // epilogue: upper slot-pair tiles -> scratch (float32, unscaled), column-major: tile (a, c),
    // a <= c, holds norb(c) columns of norb(a) rows at rowst(a) + norb(a) (cumno(c) - cumno(a));
    // element (i, j) at j norb(a) + i (the row-major norb(c) x norb(a) block (c, a) of the
    // symmetric brick H).  Only the orbitals themselves are stored (no padding rows or columns),
    // so the brick's tiles are one dense range of rowst(na) values (padded to 16 bytes).  The range
    // is assembled in shared memory (the orbital tile and the stage region are free once the MMAs
    // are done: consecutive rows of a column land in consecutive words, no bank conflicts) and
    // leaves in one bulk copy that overlaps the next item's set-up; a range larger than the
    // dynamic shared memory is stored directly.
    {
      const int ln = t & 127, qq = t >> 7;
      const uint32_t lane_base = (uint32_t)((ln >> 5) * 32) << 16;
      const long long base = S.hs_brick_off[b];
      const int total = sh.s_rowst[na], padded = (total + 3) & ~3;
      const bool staged = padded * 4 <= dsmem;
      float *const stg = staged ? reinterpret_cast<float *>(smem) : S.hs + base;
      for (int m = 0; m < ntile; ++m) {
        const int mu = 128 * m + ln;
        const int as = mu < NP ? sh.col2slot[mu] : kNoSlot;
        const int il = as != kNoSlot ? mu - sh.s_pcol[as] : 0;
        const int no_a = as != kNoSlot ? sh.s_no[as] : 0;
        const bool rowok = as != kNoSlot && il < no_a;
        const int cum_a = rowok ? sh.s_cumno[as] : 0;
        float *rowp = stg + (rowok ? sh.s_rowst[as] : 0) + il;
        const int N = NP - 128 * m;
        for (int gcol = qq; gcol < N / 16; gcol += 4) {
          const int2 hc = *reinterpret_cast<const int2 *>(&sh.hcol[16 * m + 2 * gcol]);
          float y[16], yc[16];
          if (split3 && corr_base) {
            tmem_ld16x2(tmem + lane_base + tb[m] + gcol * 16, tmem + lane_base + corr_base + tb[m] + gcol * 16, y,
                        yc);
#pragma unroll
            for (int i = 0; i < 16; ++i) y[i] += yc[i];
          } else {
            tmem_ld16(tmem + lane_base + tb[m] + gcol * 16, y);
          }
          if (!rowok) continue;
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int v = hh ? hc.y : hc.x;
            const int cc = (v >> 4) - cum_a;  // < 0: a column slot before the row slot (lower triangle)
            if (v < 0 || cc < 0) continue;
            const int nj = v & 15;
            float *dst = rowp + no_a * cc;
#pragma unroll
            for (int i = 0; i < 8; ++i)
              if (i < nj) dst[i * no_a] = y[8 * hh + i] * out_scale;
          }
        }
      }
      for (int k = total + t; k < padded; k += kT) stg[k] = 0.f;
      if (staged) {
        fence_async_smem();  // the generic writes above before the bulk copy reads them
        __syncthreads();
        if (t == 0 && padded > 0) bulk_s2g(S.hs + base, stg, (uint32_t)padded * 4u);
      }
    }
    }  // do_h
  }
}

template <bool FORCE>
__global__ void __launch_bounds__(kT, 1)
    k_tc_fused(const __grid_constant__ GTabs g, const __grid_constant__ GBatch B, const __half *__restrict__ zero,
               int *work) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ BrickSh sh;
  const int t = threadIdx.x, warp = t >> 5;
  const int split3 = B.split3;
  const long long total = B.start[B.nsys];
  // publishes the next item (nx, claimed from the work counter) and starts the bulk copy of its plan
  // record into planbuf (the buffer is free: the current item's record was unpacked before the last
  // barrier).  Inside the item loop lane 0 of the last warp does this (kNextT): its orbital slice
  // has the fewest atoms whenever the atom count is not a multiple of four, so the claim's round
  // trip and the plan offsets' loads do not delay the slowest slice (thread 0's)
  constexpr int kNextT = kT - 32;
  auto next_item = [&](long long nx) {
    sh.item = (int)nx;
    sh.plan_pref = 0;
    if (nx >= total) return;
    const int s2 = batch_sys(B, nx);
    const GSys &S2 = B.sys[s2];
    if (!S2.plan) return;
    const long long b2 = nx - B.start[s2];
    const long long o0 = S2.plan_off[b2], o1 = S2.plan_off[b2 + 1];
    const uint32_t bytes = (uint32_t)((o1 - o0) * 16);
    if (bytes > 4u * kPlanWords) return;
    fence_async_smem();  // earlier generic reads of planbuf before the asynchronous write
    mbar_arrive_tx(&sh.plan_bar, bytes);
    bulk_g2s(sh.planbuf, S2.plan + o0, bytes, &sh.plan_bar);
    sh.plan_pref = 1;
  };
  if (t == 0) {
    for (int s = 0; s < kMaxStages; ++s) mbar_init(&sh.full[s], 1);
    for (int c = 0; c < kMaxChunks; ++c) mbar_init(&sh.done[c], 1);
    mbar_init(&sh.hdone[0], 1);
    mbar_init(&sh.hdone[1], 1);
    mbar_init(&sh.hbuilt[0], kT / 32 - 1);
    mbar_init(&sh.hbuilt[1], kT / 32 - 1);
    mbar_init(&sh.plan_bar, 1);
    fence_mbar_init();
    sh.abort = 0;
    next_item(atomicAdd(work, 1));
  }
  if (warp == 0) {
    tmem_alloc(&sh.tmem, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;
  uint32_t pphase = 0;  // plan records consumed by this CTA (phase parity of plan_bar)
  uint32_t fpar = 0;  // bit s: phase parity of the next use of stage s (full[s])
  uint32_t dpar = 0;  // bit c: phase parity of done[c] (used once per density brick that has a chunk c)
  uint32_t GH = 0;    // local-H stages issued by this CTA
  int cur = -1;       // system whose points and scales are in shared memory
  bool ok = true;
  for (;;) {
    __syncthreads();
    const long long it = sh.item;
    const int pref = sh.plan_pref;
    if (it >= total || sh.abort) {
      if (pref) mbar_wait(&sh.plan_bar, pphase & 1u, B.sys[0].err);  // no copy may be in flight at exit
      break;
    }
    // the next item is claimed now and published after the unpack: the atomic's round trip overlaps
    // the set-up
    long long nclaim = 0;
    if (t == kNextT) nclaim = atomicAdd(work, 1);
    const int sidx = batch_sys(B, it);
    const GSys &S = B.sys[sidx];
    const long long b = it - B.start[sidx];
    const bool do_rho = S.do_rho != 0, do_h = S.do_h != 0;
    if (sidx != cur) {  // the previous item is finished (barrier above): replace points and scales
      init_points(S.c, sh);
      if (t == 0) {
        sh.sc[0] = S.scales[0];
        sh.sc[1] = S.scales[1];
        sh.sc[2] = S.scales[2];
      }
      cur = sidx;
    }
    // w V at the brick's points: V is copied asynchronously at the start of the orbital phase by the
    // last four warps (its DRAM latency would stall the set-up) and w V formed after the orbitals;
    // the local-H pass and the force epilogue read it later
    const bool vpend = S.V && (do_h || FORCE);
    // the previous item's local-H tiles have left shared memory (its bulk store has read them)
    // before this item writes any dynamic shared memory: thread 0 waits for that store before the
    // closing barrier of the unpack (the unpack itself writes static shared memory only)
    if (pref) {  // prefetched plan record (the common case)
      if (!mbar_wait(&sh.plan_bar, pphase & 1u, S.err)) ok = false;
      ++pphase;
      unpack_plan(sh, true);  // ends with a barrier
    } else {
      if (t == 0) bulk_wait_read();
      load_brick(S.c, g, S.nb, S.tile_off, b, sh);  // ends with a barrier
    }
    if (t == kNextT) next_item(nclaim);  // every thread has read sh.item and sh.plan_pref
    ItemCtx cx{fpar, dpar, GH, ok, vpend};
    brick_body<FORCE>(g, S, b, do_rho, do_h, split3, B.dsmem, zero, tmem, sh, smem, cx);
    fpar = cx.fpar;
    dpar = cx.dpar;
    GH = cx.GH;
    ok = cx.ok;
    tc_fence_before();
    if (!ok) sh.abort = 1;
  }
  if (t == 0) bulk_wait_all();  // the last item's bulk store is complete
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------------------ batched reduction
struct GRedSys {
  const int *hu_pair;
  const long long *hu_off, *hu_src;
  const float *hs;
  const int *pair_I, *pair_J, *pair_T;
  const long long *pair_off;
  const int *species;
  double *H;
  int fp64;  // 1: every tile value added in float64 (gint_set_reduction), 0: double-float pairs
};
struct GRed {
  int nsys;
  long long start[kMaxBatch + 1];  // first upper pair of each system
  GRedSys sys[kMaxBatch];
};

// One CTA per upper pair (I <= J) of any system: H_IJ = sum over the bricks containing both (their
// scratch tiles are column-major, norb(J) columns of norb(I) rows, element e = j norb(I) + i), summed
// as double-float pairs (two-sum: error-free additions into a hi + lo pair of float32, relative error
// about n^2 2^-48 for n bricks, far below the float32 rounding of the tiles themselves) and combined
// in float64; H_JI = H_IJ^T (per R: H_JI(-R) = H_IJ(R)^T, also for I == J, R != 0).  A thread
// sums kRedE elements of the block (stride kRedLanes) over one of kRedGroups contiguous parts of
// the pair's brick list, kRedB bricks' loads in flight; the parts'
// sums are then combined in part order (the result does not depend on scheduling).  A float64 sum
// of every tile value would cost more than the brick pass itself on this GPU (float64 runs at about
// 1/64 of the float32 rate), so the float64 step is the final combination only.
constexpr int kRedLanes = 64, kRedGroups = 4, kRedThreads = kRedLanes * kRedGroups, kRedE = 3, kRedB = 8;
__device__ __forceinline__ void bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// Upper pair u of system S by NG groups of kRedLanes threads (tid in [0, NG kRedLanes)); part_hi and
// part_lo hold (NG - 1) kRedE kRedLanes floats each; the groups synchronise on barrier `bar`.
// F64: every tile value converted and added in float64 (a part's float64 sum travels between the
// groups as the two 32-bit halves of its bits in part_lo / part_hi), the same parts and order.
template <int NG, bool F64, bool PF>
__device__ __forceinline__ void reduce_pair_t(const GTabs &g, const GRedSys &S, int u, int tid, float *part_hi,
                                              float *part_lo, int bar) {
  const int p = S.hu_pair[u];
  const int I = S.pair_I[p], J = S.pair_J[p];
  const int nI = g.sp[S.species[I]].norb, nJ = g.sp[S.species[J]].norb;
  const int ln = tid % kRedLanes, grp = tid / kRedLanes;
  const long long kk0 = S.hu_off[u], kk1 = S.hu_off[u + 1];
  const long long per = (kk1 - kk0 + NG - 1) / NG;
  const long long k0 = min(kk1, kk0 + grp * per), k1 = min(kk1, k0 + per);
  const float *__restrict__ hs = S.hs;
  const long long *__restrict__ src = S.hu_src;
  const int ne = nI * nJ;
  for (int base = 0; base < ne; base += kRedLanes * kRedE) {  // uniform trip count within the groups
    int e[kRedE];
    bool act[kRedE];
    float ah[kRedE], al[kRedE];
    double ad[kRedE];
#pragma unroll
    for (int q = 0; q < kRedE; ++q) {
      e[q] = base + q * kRedLanes + ln;
      act[q] = e[q] < ne;
      if (!act[q]) e[q] = 0;  // a valid address; its loads are discarded
      ah[q] = al[q] = 0.f;
      ad[q] = 0.0;
    }
    auto add = [&](int q, float x) {
      if (F64) {
        ad[q] += (double)x;
      } else {
        float sum, err;
        two_sum(ah[q], x, sum, err);
        ah[q] = sum;
        al[q] += err;
      }
    };
    long long k = k0;
    // PF: the next batch's tile offsets are loaded while the current batch's values are summed, so
    // the offset and value loads of a batch are not two round trips in a row (the standalone
    // reduction; the resident kernel keeps the lighter loop, its registers being spoken for)
    long long o[kRedB];
    if (PF && k + kRedB <= k1) {
#pragma unroll
      for (int jj = 0; jj < kRedB; ++jj) o[jj] = __ldg(src + k + jj);
    }
    for (; k + kRedB <= k1; k += kRedB) {
      if (!PF) {
#pragma unroll
        for (int jj = 0; jj < kRedB; ++jj) o[jj] = __ldg(src + k + jj);
      }
      float v[kRedB][kRedE];
#pragma unroll
      for (int jj = 0; jj < kRedB; ++jj)
#pragma unroll
        for (int q = 0; q < kRedE; ++q) v[jj][q] = __ldcg(hs + o[jj] + e[q]);  // written by this or another launch
      if (PF && k + 2 * kRedB <= k1) {
#pragma unroll
        for (int jj = 0; jj < kRedB; ++jj) o[jj] = __ldg(src + k + kRedB + jj);
      }
#pragma unroll
      for (int jj = 0; jj < kRedB; ++jj)
#pragma unroll
        for (int q = 0; q < kRedE; ++q) add(q, v[jj][q]);
    }
    for (; k < k1; ++k) {
      const long long o = __ldg(src + k);
#pragma unroll
      for (int q = 0; q < kRedE; ++q) add(q, __ldcg(hs + o + e[q]));
    }
    if (grp > 0) {
#pragma unroll
      for (int q = 0; q < kRedE; ++q) {
        const int w = ((grp - 1) * kRedE + q) * kRedLanes + ln;
        if (F64) {
          part_hi[w] = __int_as_float(__double2hiint(ad[q]));
          part_lo[w] = __int_as_float(__double2loint(ad[q]));
        } else {
          part_hi[w] = ah[q];
          part_lo[w] = al[q];
        }
      }
    }
    bar_sync(bar, NG * kRedLanes);
    if (grp == 0) {
#pragma unroll
      for (int q = 0; q < kRedE; ++q) {
        if (!act[q]) continue;
        double acc = F64 ? ad[q] : (double)ah[q] + (double)al[q];
        for (int g2 = 0; g2 < NG - 1; ++g2) {
          const int w = (g2 * kRedE + q) * kRedLanes + ln;
          acc += F64 ? __hiloint2double(__float_as_int(part_hi[w]), __float_as_int(part_lo[w]))
                     : (double)part_hi[w] + (double)part_lo[w];
        }
        const int j = e[q] / nI, i = e[q] - j * nI;
        S.H[S.pair_off[p] + (long long)i * nJ + j] = acc;
        if (S.pair_T[p] != p) S.H[S.pair_off[S.pair_T[p]] + (long long)j * nI + i] = acc;  // (J, I, -R)
      }
    }
    bar_sync(bar, NG * kRedLanes);
  }
}

template <int NG, bool PF = false>
__device__ __forceinline__ void reduce_pair(const GTabs &g, const GRedSys &S, int u, int tid, float *part_hi,
                                            float *part_lo, int bar) {
  if (S.fp64)
    reduce_pair_t<NG, true, PF>(g, S, u, tid, part_hi, part_lo, bar);
  else
    reduce_pair_t<NG, false, PF>(g, S, u, tid, part_hi, part_lo, bar);
}

__global__ void __launch_bounds__(kRedThreads, 4) k_h_reduce(const __grid_constant__ GTabs g, const __grid_constant__ GRed R) {
  __shared__ float part_hi[(kRedGroups - 1) * kRedE * kRedLanes], part_lo[(kRedGroups - 1) * kRedE * kRedLanes];
  const long long gu = blockIdx.x;
  int lo = 0, hi = R.nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (R.start[mid] <= gu)
      lo = mid;
    else
      hi = mid - 1;
  }
  reduce_pair<kRedGroups, true>(g, R.sys[lo], (int)(gu - R.start[lo]), threadIdx.x, part_hi, part_lo, 0);
}

// ------------------------------------------------------------------------------ batched preparation
struct GPrepSys {
  const double *D;  // NULL: no density / force items
  long long nblock;
  const double *V;  // NULL: no local-H / force items
  long long ngrid;
  double *F;        // zeroed here (the brick kernel accumulates into it)
  long long natoms;
  unsigned *mx;     // [0] bits of max |D|, [1] bits of max |V| (atomicMax on non-negative floats)
  float *scales;
  double phi_bound, w;
};
struct GPrep {
  int nsys;
  int *work;
  GPrepSys sys[kMaxBatch];
};

// Elements [i0, i1) of the system's D blocks, grid and force arrays, by nt threads (this one t):
// max |D| and max |V| (float32, rounded; atomicMax into S.mx), F zeroed.
__device__ __forceinline__ void prep_range(const GPrepSys &S, long long i0, long long i1, long long t, long long nt) {
  // |x| of a float64 orders like its bit pattern without the sign, so the maxima are integer maxima
  // (no float64 arithmetic, which runs at a small fraction of the integer rate on this GPU); the
  // largest one is rounded to float32 once (rounding is monotonic: the same value as the largest
  // rounded element).  Inputs are read through L2 (__ldcg): a resident launch may see them
  // rewritten between its jobs.
  unsigned long long bD = 0, bV = 0;
  const unsigned long long mag = 0x7fffffffffffffffull;
  // eight loads in flight per thread
  auto absmax = [&](const double *x, long long n) {
    unsigned long long b = 0;
    const long long e = min(i1, n);
    long long i = i0 + t;
    for (; i + 7 * nt < e; i += 8 * nt) {
      long long v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = __double_as_longlong(__ldcg(x + i + k * nt));
#pragma unroll
      for (int k = 0; k < 8; ++k) b = max(b, (unsigned long long)v[k] & mag);
    }
    for (; i < e; i += nt) b = max(b, (unsigned long long)__double_as_longlong(__ldcg(x + i)) & mag);
    return b;
  };
  if (S.D) bD = absmax(S.D, S.nblock);
  if (S.V) bV = absmax(S.V, S.ngrid);
  if (S.F)
    for (long long i = i0 + t; i < min(i1, 3 * S.natoms); i += nt) S.F[i] = 0.0;
  for (int o = 16; o > 0; o >>= 1) {
    bD = max(bD, __shfl_xor_sync(0xffffffffu, bD, o));
    bV = max(bV, __shfl_xor_sync(0xffffffffu, bV, o));
  }
  const float mD = (float)__longlong_as_double((long long)bD), mV = (float)__longlong_as_double((long long)bV);
  if ((threadIdx.x & 31) == 0) {
    if (mD > 0.f) atomicMax(S.mx, __float_as_uint(mD));
    if (mV > 0.f) atomicMax(S.mx + 1, __float_as_uint(mV));
  }
}

// blockIdx.y = system: prep_range over the whole arrays; also resets the work counter.
__global__ void k_prep(const __grid_constant__ GPrep P) {
  prep_range(P.sys[blockIdx.y], 0, 0x7fffffffffffffffLL, blockIdx.x * (long long)blockDim.x + threadIdx.x,
             (long long)gridDim.x * blockDim.x);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *P.work = 0;
}

__device__ double pow2_scale(double lim, double m) {
  if (!(m > 0)) return 1048576.0;
  return exp2(floor(log2(lim / m)));
}

// Power-of-two scales of a system ([0] orbitals, [1] D, [2] w V orbitals), with the largest scaled
// magnitudes below 2^15 (float16 max 65504; a zero input gets 2^20); then clears the maxima for the
// next call.  One thread.
__device__ __forceinline__ void prep_scales(const GPrepSys &S) {
  const double pb = 4.0 * S.phi_bound;
  S.scales[0] = (float)pow2_scale(30000.0, pb);
  S.scales[1] = (float)pow2_scale(30000.0, (double)__uint_as_float(S.mx[0]));
  S.scales[2] = (float)pow2_scale(30000.0, pb * S.w * (double)__uint_as_float(S.mx[1]));
  S.mx[0] = 0u;
  S.mx[1] = 0u;
}

// Thread s: the scales of system s.
__global__ void k_prep_scales(const __grid_constant__ GPrep P) {
  if (threadIdx.x < P.nsys) prep_scales(P.sys[threadIdx.x]);
}

struct GTileSys {
  const double *D;
  const int *pair_I, *pair_J;
  const long long *pair_off, *tile_off;
  const int *species;
  const float *scales;
  __half *Dhl, *Dhl2;  // interleaved: 8 x 8 block b of the tile has hi at 128 b, lo at 128 b + 64
};
struct GTile {
  int nsys;
  int fixed;  // 1: fixed-point split at 2^-4 of the floating split's scale (force launches)
  long long start[kMaxBatch + 1];  // first pair of each system
  GTileSys sys[kMaxBatch];
};

// Pair p of a system: D block (float64, row-major norb(I) x norb(J)) -> scaled float16 (hi, lo)
// tile of roundup(norb(I), 8) x porb(J) in core-matrix order [row group][K group][8][8], plus the
// same tile halved (floating split), or the fixed-point split (hi the nearest integer, exact in
// float16 for |x| < 2048, lo the float16 remainder).
// One warp builds the tile: a lane takes one row of an 8 x 8 block at a time (8 elements, one
// 16-byte store per array).  The floating split is formed in float32: the scale is a power of two,
// so the scaled value is D rounded once to float32 (2^-24 relative, below the split's 2^-22), and
// hi, x - hi, x / 2 and x / 2 - hi2 are exact in float32.  The fixed-point split (force launches)
// keeps the remainder x - rint(x) in float64, since it is the lo term of an exact hi * hi sum.
__device__ __forceinline__ void build_tile_warp(const GTabs &g, const GTileSys &S, int p, bool fixed, int lane) {
  const int I = S.pair_I[p], J = S.pair_J[p];
  const int nI = g.sp[S.species[I]].norb, nJ = g.sp[S.species[J]].norb, pJ = g.sp[S.species[J]].porb;
  const int rI = (nI + 7) & ~7, sJ = pJ >> 3;
  const float scf = __ldcg(S.scales + 1) * (fixed ? kFxScaleD : 1.f);
  const long long o = S.pair_off[p], to = S.tile_off[p];
  const double *__restrict__ Dp = S.D + o;
  for (int u = lane; u < rI * sJ; u += 32) {  // units: (block, row of the block)
    const int cm = u >> 3, r8 = u & 7;
    const int i = (cm / sJ) * 8 + r8, j0 = (cm % sJ) * 8;
    uint32_t wh[4], wl[4], w2h[4], w2l[4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      float hv[2], lv[2], h2v[2], l2v[2];
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int j = j0 + k + m;
        const bool in = i < nI && j < nJ;
        const double d = in ? __ldcg(Dp + (long long)i * nJ + j) : 0.0;
        if (fixed) {
          const double x = d * (double)scf, hx = rint(x);
          hv[m] = (float)hx;
          lv[m] = (float)(x - hx);
          h2v[m] = l2v[m] = 0.f;  // the halved tiles are unused in force launches
        } else {
          const float x = (float)d * scf;
          hv[m] = __half2float(__float2half_rn(x));
          lv[m] = x - hv[m];
          h2v[m] = __half2float(__float2half_rn(0.5f * x));
          l2v[m] = 0.5f * x - h2v[m];
        }
      }
      const __half2 a = __floats2half2_rn(hv[0], hv[1]), b = __floats2half2_rn(lv[0], lv[1]);
      const __half2 c = __floats2half2_rn(h2v[0], h2v[1]), e = __floats2half2_rn(l2v[0], l2v[1]);
      wh[k >> 1] = *reinterpret_cast<const uint32_t *>(&a);
      wl[k >> 1] = *reinterpret_cast<const uint32_t *>(&b);
      w2h[k >> 1] = *reinterpret_cast<const uint32_t *>(&c);
      w2l[k >> 1] = *reinterpret_cast<const uint32_t *>(&e);
    }
    const long long q = 2 * to + (long long)cm * 128 + r8 * 8;  // hi of the row; lo 64 halves later
    *reinterpret_cast<uint4 *>(S.Dhl + q) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
    *reinterpret_cast<uint4 *>(S.Dhl + q + 64) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    *reinterpret_cast<uint4 *>(S.Dhl2 + q) = make_uint4(w2h[0], w2h[1], w2h[2], w2h[3]);
    *reinterpret_cast<uint4 *>(S.Dhl2 + q + 64) = make_uint4(w2l[0], w2l[1], w2l[2], w2l[3]);
  }
}

// One warp per pair of any system, eight pairs per CTA.
constexpr int kTileWarps = 8;
__global__ void __launch_bounds__(32 * kTileWarps) k_build_tiles(const __grid_constant__ GTabs g,
                                                                 const __grid_constant__ GTile TB) {
  const long long gp = (long long)blockIdx.x * kTileWarps + (threadIdx.x >> 5);
  if (gp >= TB.start[TB.nsys]) return;
  int lo = 0, hi = TB.nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (TB.start[mid] <= gp)
      lo = mid;
    else
      hi = mid - 1;
  }
  build_tile_warp(g, TB.sys[lo], (int)(gp - TB.start[lo]), TB.fixed != 0, threadIdx.x & 31);
}

// One CTA per brick: the brick's metadata exactly as the brick kernel's slow path builds it,
// serialised into its plan record (see plan_words).  Record capacity mismatch: index error bit.
__global__ void __launch_bounds__(128) k_build_plans(const __grid_constant__ GTabs g, GCell c, GNbr nb,
                                                     const long long *__restrict__ tile_off,
                                                     const long long *__restrict__ plan_off, uint32_t *plan,
                                                     unsigned *err) {
  __shared__ BrickSh sh;
  const long long b = blockIdx.x;
  const int t = threadIdx.x;
  load_brick(c, g, nb, tile_off, b, sh);
  const int na = sh.na, nent = sh.nent, np = sh.np;
  const long long cap = (plan_off[b + 1] - plan_off[b]) * 4;
  if (plan_words(na, nent, np) > cap) {
    if (t == 0) atomicOr(err, GINT_ERRBIT_INDEX);
    return;
  }
  uint32_t *w = plan + plan_off[b] * 4;
  if (t == 0) {
    w[0] = (uint32_t)na;
    w[1] = (uint32_t)nent;
    w[2] = (uint32_t)np;
    w[3] = (uint32_t)sh.s_cumno[na];
  }
  for (int a = t; a < na; a += blockDim.x) {
    uint32_t *q = w + 4 + 8 * a;
    q[0] = (uint32_t)sh.s_atom[a];
    q[1] = (uint32_t)sh.s_sp[a];
    q[2] = (uint32_t)sh.s_no[a];
    q[3] = (uint32_t)sh.s_po[a];
    q[4] = (uint32_t)sh.s_pcol[a];
    q[5] = (uint32_t)sh.s_e0[a];
    q[6] = (uint32_t)sh.s_cumno[a];
    q[7] = (uint32_t)sh.s_rowst[a];
  }
  const int eb = 4 + 8 * na;
  for (int u = t; u < 6 * nent; u += blockDim.x) {
    const int e = u / 6, k = u - 6 * e;
    w[eb + u] = __float_as_uint(k < 3 ? sh.e_hi[e][k] : sh.e_lo[e][k - 3]);
  }
  const int tb = eb + 6 * nent;
  for (int i = t; i < na * na; i += blockDim.x) w[tb + i] = (uint32_t)sh.s_tile[i];
  // column -> slot bytes, packed four per word, zero padded to the record end
  const long long cw0 = tb + (long long)na * na;
  for (long long i = cw0 + t; i < cap; i += blockDim.x) {
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k) {
      const long long col = 4 * (i - cw0) + k;
      if (col < np) v |= (uint32_t)sh.col2slot[col] << (8 * k);
    }
    w[i] = v;
  }
}

// ------------------------------------------------------------------------------ resident serving kernel
// Continuous batching: one resident launch drains a device work queue to which the host appends jobs
// (one task: the density / force and local-H passes of one system) while it runs.  A job's items, in
// the global item order: kServePrep max-reduction chunks, one scales item, tile items (kServeTilePairs
// pairs each), one item per brick, reduction items (kServeRedPairs upper pairs each).  A CTA claims
// ranges of a published job's items, in order, by a fetch-and-add on that job's claim counter (a
// count past the job's end sends the CTA to the next job); an item waits (bounded) for the items of
// its job it depends on (scales after the
// chunks, tiles after the scales, bricks after the tiles, reductions after the bricks), which were
// all claimed earlier, so the wait always ends.  The last item of a job to complete writes the job's
// completion word into host-mapped memory.  A CTA with nothing to claim for idle_ns (or on the stop
// flag, or when a wait gave up anywhere) leaves; the host relaunches when it has unclaimed work.
constexpr int kServeRing = 64;                  // jobs in flight at most (descriptor ring)
constexpr long long kServePrep = 1LL << 16;     // elements per max-reduction item
constexpr int kServeRange = 16;                 // most items one claim takes
constexpr int kServeTilePairs = 32;             // pairs per tile item (four at a time, 128 threads each)
constexpr int kServeRedPairs = 2;               // upper pairs per reduction item (256 threads each)
constexpr long long kServeMaxJobs = 1LL << 20;  // jobs over a server's lifetime (completion-order table)

struct GJob {
  GSys sys;
  GPrepSys prep;
  GTileSys tile;
  GRedSys red;
  int npairs, nupper, fixed, pad;
  long long nbricks;
  long long n_prep, n_tile, n_red;  // items of each kind (plus one scales item)
  long long item0, nitems;          // first item and item count of the job
  unsigned long long seq;
};
struct GJobState {  // completed items of the job per kind, in total, and claimed (zeroed at publication)
  int prep, scales, tiles, bricks, red, all, claim, pad;
};
struct GServeCtl {
  unsigned long long head;       // unused (claims count per job)
  unsigned long long tail;       // published items (written by the host)
  unsigned long long first_seq;  // claims never go to jobs before this one (cursor start, host hint)
  int stop;                      // host: leave as soon as idle
  unsigned err;                  // GINT_ERRBIT_* of any item; every CTA leaves
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ long long ld_acquire_s64(const long long *p) {
  long long v;
  asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_s32(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Bounded wait (thread 0) until *cnt >= target; false after kWaitNs (timeout bit in *err).
__device__ __forceinline__ bool wait_count(const int *cnt, long long target, unsigned *err) {
  if (ld_acquire_s32(cnt) >= target) return true;
  const long long t0 = globaltimer();
  while (ld_acquire_s32(cnt) < target) {
    if (globaltimer() - t0 > kWaitNs) {
      atomicOr(err, GINT_ERRBIT_TIMEOUT);
      return false;
    }
    __nanosleep(256);
  }
  return true;
}

template <bool FORCE>
__global__ void __launch_bounds__(kT, 1)
    k_serve(const __grid_constant__ GTabs g, GServeCtl *ctl, const GJob *__restrict__ jobs, GJobState *st,
            const long long *__restrict__ job_end, volatile unsigned long long *done, const __half *__restrict__ zero,
            int split3, int dsmem, long long idle_ns) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ BrickSh sh;
  __shared__ GJob sj;    // the item's job (copied through L2 for every item: a ring slot is rewritten
                         // by the host for later jobs while this launch runs)
  __shared__ long long s_item, s_seq, s_plan_next;  // s_plan_next: the item whose plan record is in flight
  // thread 0's bookkeeping, kept in shared memory (not registers) so that it does not add to the
  // register pressure of the brick items: the claim still to run, the job cursor, the current job,
  // and completed items not yet counted (one job and kind; counted before this CTA waits for
  // anything, a dependency or a new claim, and when the job or kind changes)
  struct ServeState {
    unsigned long long range_next, range_end, cursor, cur_sys, cur_job, pseq;
    int *pc;
    GJobState *pjs;
    int pn, pitems;
    unsigned long long bseq;           // the job whose stage bounds follow (claims)
    long long b_i0, b_bb, b_rr, b_ee;  // its first item, first brick, first reduction, end
    unsigned long long tiles_seq;      // a job whose tile stage this CTA has seen complete (+1)
    int bad;                           // this item's dependency wait gave up (every thread skips it)
  };
  __shared__ ServeState ss;
  const int t = threadIdx.x, warp = t >> 5;
  if (t == 0) {
    for (int s2 = 0; s2 < kMaxStages; ++s2) mbar_init(&sh.full[s2], 1);
    for (int c = 0; c < kMaxChunks; ++c) mbar_init(&sh.done[c], 1);
    mbar_init(&sh.hdone[0], 1);
    mbar_init(&sh.hdone[1], 1);
    mbar_init(&sh.hbuilt[0], kT / 32 - 1);
    mbar_init(&sh.hbuilt[1], kT / 32 - 1);
    mbar_init(&sh.plan_bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&sh.tmem, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;
  ItemCtx cx{0u, 0u, 0u, true};
  uint32_t pphase = 0;
  auto flush = [&]() {  // thread 0
    if (!ss.pn) return;
    __threadfence();  // the items' results before their counts
    atomicAdd(ss.pc, ss.pn);
    if (atomicAdd(&ss.pjs->all, ss.pn) + ss.pn == ss.pitems) {
      __threadfence_system();
      done[ss.pseq % kServeRing] = ss.pseq + 1;  // the job's results are in device memory
    }
    ss.pn = 0;
  };
  if (t == 0) {
    ss.cursor = ld_acquire_u64(&ctl->first_seq);
    ss.range_next = ss.range_end = 0;
    ss.cur_sys = ss.cur_job = ~0ull;
    ss.pc = nullptr;
    ss.pjs = nullptr;
    ss.pn = ss.pitems = 0;
    ss.pseq = 0;
    ss.bseq = ~0ull;
    ss.tiles_seq = 0;
    s_plan_next = -1;
  }
  for (;;) {
    if (t == 0) {
      // the next item of the current claim, or a new claim of up to kServeRange published items
      // (fewer as the published work runs low: a few items per CTA at most), or leave
      long long item = -1;
      if (ss.range_next < ss.range_end) {
        item = (long long)ss.range_next++;
      } else {
        flush();
        const long long t0 = globaltimer();
        for (;;) {
          if (*(volatile unsigned *)&ctl->err) break;
          // the job at this CTA's cursor, if published (the host writes a job's end before the tail
          // that covers it); its items are claimed with a fetch-and-add on the job's own counter, so
          // no claim waits for another and an over-claim is only a count past the job's end
          const unsigned long long tl = ld_acquire_u64(&ctl->tail);
          const unsigned long long c = ss.cursor;
          const long long e = ld_acquire_s64(job_end + c);
          if (e > 0 && (unsigned long long)e <= tl) {
            if (ss.bseq != c) {
              const GJob *jc = jobs + c % kServeRing;
              ss.b_i0 = __ldcg(&jc->item0);
              ss.b_bb = ss.b_i0 + __ldcg(&jc->n_prep) + 1 + __ldcg(&jc->n_tile);
              ss.b_rr = ss.b_bb + __ldcg(&jc->nbricks);
              ss.b_ee = ss.b_i0 + __ldcg(&jc->nitems);
              ss.bseq = c;
            }
            int *claim = &st[c % kServeRing].claim;
            const long long n = ss.b_ee - ss.b_i0, cl = *(volatile int *)claim;
            if (cl < n) {
              // the claim's size from the stage of the next item: up to kServeRange bricks or
              // kServeRange / 2 reduction items, fewer as the job's items run low; the short
              // preparation and tile stages one item at a time so that every CTA helps with them
              const long long hi = ss.b_i0 + cl;
              const long long lim = hi < ss.b_bb ? 1
                                    : hi < ss.b_rr ? min((long long)kServeRange, ss.b_rr - hi)
                                                   : min((long long)kServeRange / 2, ss.b_ee - hi);
              const int r = (int)max(1LL, min(lim, (n - cl) / (2LL * gridDim.x)));
              const long long got = atomicAdd(claim, r);
              if (got < n) {
                item = ss.b_i0 + got;
                ss.range_next = (unsigned long long)(item + 1);
                ss.range_end = (unsigned long long)(ss.b_i0 + min(got + r, n));
                break;
              }
            }
            ss.cursor = c + 1;  // every item of job c is claimed
            continue;
          }
          if (*(volatile int *)&ctl->stop || globaltimer() - t0 > idle_ns) break;
          __nanosleep(1000);
        }
      }

      s_item = item;
      s_seq = (long long)ss.cursor;
      bulk_wait_read();  // a previous brick item's tiles have left shared memory
    }
    __syncthreads();
    const long long item = s_item;
    if (item < 0) break;
    const unsigned long long seq = (unsigned long long)s_seq;
    if (seq != ss.cur_job) {  // a job's descriptor does not change while it is in flight
      const int *src = reinterpret_cast<const int *>(jobs + seq % kServeRing);
      int *dst = reinterpret_cast<int *>(&sj);
      for (int k = t; k < (int)(sizeof(GJob) / sizeof(int)); k += kT) dst[k] = __ldcg(src + k);
      __syncthreads();
      if (t == 0) ss.cur_job = seq;
    }
    const GJob &J = sj;
    GJobState &JS = st[seq % kServeRing];
    unsigned *err = &ctl->err;
    const long long li = item - J.item0;
    const long long b0 = J.n_prep + 1 + J.n_tile, r0 = b0 + J.nbricks;
    if (li < J.n_prep) {  // max-reduction chunk
      prep_range(J.prep, li * kServePrep, (li + 1) * kServePrep, t, kT);
    } else if (li == J.n_prep) {  // scales
      if (t == 0) {
        flush();
        if (wait_count(&JS.prep, J.n_prep, err)) prep_scales(J.prep);
      }
    } else if (li < b0) {  // D tiles
      bool go = true;
      if (t == 0) {
        flush();
        go = wait_count(&JS.scales, 1, err);
      }
      __syncthreads();
      if (go && !*(volatile unsigned *)err) {
        const long long p0 = (li - J.n_prep - 1) * kServeTilePairs;
        for (long long p = p0 + (t >> 5); p < min((long long)J.npairs, p0 + kServeTilePairs); p += kT / 32)
          build_tile_warp(g, J.tile, (int)p, J.fixed != 0, t & 31);
      }
    } else if (li < r0) {  // a brick
      const long long b = li - b0;
      cx.ok = true;
      // the job's tiles: awaited once per job and CTA (errors of other CTAs are seen at the next claim)
      if (t == 0) {
        ss.bad = 0;
        if (ss.tiles_seq != seq + 1) {
          if (ld_acquire_s32(&JS.tiles) < J.n_tile) {
            flush();
            if (!wait_count(&JS.tiles, J.n_tile, err)) ss.bad = 1;
          }
          if (!ss.bad) ss.tiles_seq = seq + 1;
        }
      }
      // V at the brick's points: loaded now, stored after the unpack (the load overlaps it); the
      // L1-bypassing load sees V rewritten for a later job.  brick_body reads wv only after its
      // own barriers.
      const GSys &S0 = sj.sys;
      float wvv = 0.f;
      if (t < 128 && S0.V && (S0.do_h || FORCE)) {
        int gi, gj, gk;
        if (brick_point(S0.c, b, t, gi, gj, gk)) wvv = (float)(S0.c.w * __ldcg(S0.V + grid_index(S0.c, gi, gj, gk)));
      }
      __syncthreads();
      if (!ss.bad) {  // the same decision in every thread (read after the barrier)
        const GSys &S = sj.sys;
        if (seq != ss.cur_sys) {  // a new job: points and scales into shared memory
          init_points(S.c, sh);
          __syncthreads();  // every thread has read ss.cur_sys
          if (t == 0) {
            sh.sc[0] = __ldcg(S.scales + 0);
            sh.sc[1] = __ldcg(S.scales + 1);
            sh.sc[2] = __ldcg(S.scales + 2);
            ss.cur_sys = seq;
          }
        }
        const bool do_rho = S.do_rho != 0, do_h = S.do_h != 0;
        const long long o0 = S.plan_off[b], o1 = S.plan_off[b + 1];
        const uint32_t bytes = (uint32_t)((o1 - o0) * 16);
        if (S.plan && bytes <= 4u * kPlanWords) {
          if (s_plan_next != item && t == 0) {  // not prefetched by the previous item
            fence_async_smem();
            mbar_arrive_tx(&sh.plan_bar, bytes);
            bulk_g2s(sh.planbuf, S.plan + o0, bytes, &sh.plan_bar);
          }
          if (!mbar_wait(&sh.plan_bar, pphase & 1u, err)) cx.ok = false;
          ++pphase;
          unpack_plan(sh);  // ends with a barrier
        } else {
          load_brick(S.c, g, S.nb, S.tile_off, b, sh);  // ends with a barrier
        }
        if (t == 0) {
          // the plan record of the next item of this claim, if it is a brick of this job, while this
          // one runs (the buffer is free: unpacked before the barrier above)
          s_plan_next = -1;
          const long long li2 = (long long)ss.range_next - J.item0;
          if (ss.range_next < ss.range_end && li2 >= b0 && li2 < r0 && S.plan) {
            const long long p0 = S.plan_off[li2 - b0], p1 = S.plan_off[li2 - b0 + 1];
            const uint32_t nb2 = (uint32_t)((p1 - p0) * 16);
            if (nb2 <= 4u * kPlanWords) {
              fence_async_smem();
              mbar_arrive_tx(&sh.plan_bar, nb2);
              bulk_g2s(sh.planbuf, S.plan + p0, nb2, &sh.plan_bar);
              s_plan_next = (long long)ss.range_next;
            }
          }
        }
        if (t < 128) sh.wv[t] = wvv;  // read by brick_body after its barriers
        brick_body<FORCE>(g, S, b, do_rho, do_h, split3, dsmem, zero, tmem, sh, smem, cx);
        tc_fence_before();
      }
    } else {  // H reduction: two upper pairs, one per 256 threads (named barriers 2, 3), split into parts
      // exactly as k_h_reduce splits them, so the blocks equal those of the batched call bit for bit
      bool go = true;
      if (t == 0 && ld_acquire_s32(&JS.bricks) < J.nbricks) {
        flush();
        go = wait_count(&JS.bricks, J.nbricks, err);
      }
      __syncthreads();
      if (go && !*(volatile unsigned *)err) {
        const int sg = t / kRedThreads, u = (int)((li - r0) * kServeRedPairs) + sg;
        float *part = reinterpret_cast<float *>(smem) + sg * 2 * (kRedGroups - 1) * kRedE * kRedLanes;
        if (u < J.nupper)
          reduce_pair<kRedGroups>(g, J.red, u, t % kRedThreads, part, part + (kRedGroups - 1) * kRedE * kRedLanes,
                                  2 + sg);
      }
    }
    if (!cx.ok) atomicOr(err, GINT_ERRBIT_TIMEOUT);  // the next claim sees it: every CTA leaves
    __syncthreads();
    if (t == 0) {  // everything from shared memory: nothing of the item stays live in registers
      const unsigned long long sq = (unsigned long long)s_seq;
      GJobState *js = st + sq % kServeRing;
      const long long l2 = s_item - sj.item0, bb = sj.n_prep + 1 + sj.n_tile, rr = bb + sj.nbricks;
      int *counter = l2 < sj.n_prep ? &js->prep
                   : l2 == sj.n_prep ? &js->scales
                   : l2 < bb ? &js->tiles
                   : l2 < rr ? &js->bricks
                             : &js->red;
      if (ss.pn && (ss.pc != counter || ss.pjs != js)) flush();
      ss.pc = counter;
      ss.pjs = js;
      ss.pitems = (int)sj.nitems;
      ss.pseq = sq;
      ++ss.pn;
    }
  }
  if (t == 0) {
    flush();
    // a plan record still in flight (the claim ended on an error): wait for it, bounded
    if (s_plan_next >= 0) mbar_wait(&sh.plan_bar, pphase & 1u, &ctl->err);
    bulk_wait_all();
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------------------ orbital diagnostic
// One thread per (point, atom): the periodised orbitals of the atom and their gradients at an
// arbitrary point, summed over the lattice images whose support covers it, by the brick kernels'
// own evaluators: float64 (the CUDA-core path's add_orbitals) or float32 (the tensor-core path's
// double-float distance, knot and Hermite evaluation, difference tables for the derivatives).
__global__ void k_orbitals(const __grid_constant__ GGeom g, const double2 *__restrict__ tab64,
                           const float2 *__restrict__ tab, const float2 *__restrict__ tabi,
                           const float *__restrict__ dtab, const float *__restrict__ dtabi, const double *__restrict__ pos,
                           const int *__restrict__ species, const int *__restrict__ aoff, long long npts, int norb,
                           const double *__restrict__ pts, int fp64, double *__restrict__ phi, double *__restrict__ grad) {
  const long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= npts * g.natoms) return;
  const long long q = u / g.natoms;
  const int I = (int)(u - q * g.natoms), sp = species[I];
  const GSpecies &S = g.sp[sp];
  const int no = S.norb, o = aoff[I];
  double v64[GINT_MAX_ORB_ATOM], gv64[GINT_MAX_ORB_ATOM][3];
  float v32[GINT_MAX_ORB_ATOM], gv32[3 * GINT_MAX_ORB_ATOM];
  for (int i = 0; i < no; ++i) {
    v64[i] = gv64[i][0] = gv64[i][1] = gv64[i][2] = 0.0;
    v32[i] = gv32[3 * i] = gv32[3 * i + 1] = gv32[3 * i + 2] = 0.f;
  }
  double d0[3], uf[3];
  for (int d = 0; d < 3; ++d) d0[d] = pts[3 * q + d] - pos[3 * I + d];
  for (int d = 0; d < 3; ++d) uf[d] = d0[0] * g.inv[0 * 3 + d] + d0[1] * g.inv[1 * 3 + d] + d0[2] * g.inv[2 * 3 + d];
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = (int)ceil(uf[d] - S.rcut * g.reach[d]);
    hi[d] = (int)floor(uf[d] + S.rcut * g.reach[d]);
  }
  for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
    for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
      for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
        double dd[3];
        for (int d = 0; d < 3; ++d) dd[d] = d0[d] - (n0 * g.cell[d] + n1 * g.cell[3 + d] + n2 * g.cell[6 + d]);
        if (dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2] >= S.rcut2) continue;
        if (fp64) {
          add_orbitals<double, true, true>(g, tab64, sp, dd[0], dd[1], dd[2], v64, gv64);
        } else {
          float dh[3], dl[3];
          for (int d = 0; d < 3; ++d) split2(dd[d], dh[d], dl[d]);
          if (dh[0] * dh[0] + dh[1] * dh[1] + dh[2] * dh[2] >= S.rcut2f) continue;  // the brick kernels' test
          switch (S.shape) {
#define CASE_O(ns, np_, nd) \
  case GINT_SHAPE(ns, np_, nd): add_image_fast<ns, np_, nd, true>(g, tabi, dtabi, S, dh, dl, v32, gv32); break;
            GINT_FOR_SHAPES(CASE_O)
#undef CASE_O
            default:
              add_image_generic<true>(g, tab, dtab, S, dh, dl, v32, gv32);
          }
        }
      }
  for (int i = 0; i < no; ++i) {
    phi[q * norb + o + i] = fp64 ? v64[i] : (double)v32[i];
    if (grad)
      for (int d = 0; d < 3; ++d) grad[(q * norb + o + i) * 3 + d] = fp64 ? gv64[i][d] : (double)gv32[3 * i + d];
  }
}

// ------------------------------------------------------------------------------ self-test
// One f16 MMA per operand layout the brick kernels use, on integer data; err_out[0] = max |D - exact|.
//   layout 0, 1: K-major, LBO 128 (K), SBO 256 / 512 (8-row groups) -- density P and B stages
//   layout 2: both operands MN-major, LBO = K-direction stride, SBO = 128 -- local H from P
__global__ void __launch_bounds__(128, 1) k_tc_selftest(int N, float *err_out, unsigned *status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_s;
  const int t = threadIdx.x, warp = t >> 5;
  if (t == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&tmem_s, 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_s;
  float maxerr = 0.f;
  for (int layout = 0; layout < 3; ++layout) {
    const bool mn = layout == 2;
    const uint32_t sbo = layout == 0 ? 256u : 512u;
    unsigned char *A = smem, *B = smem + 8192;
    const uint32_t ksa = 16 * 128, ksb = (uint32_t)(N / 8) * 128;  // MN-major K strides
    for (int e = t; e < 128 * 16; e += 128) {
      const int i = e >> 4, k = e & 15;
      const uint32_t off = mn ? (k >> 3) * ksa + (i >> 3) * 128 + (k & 7) * 16 + (i & 7) * 2
                              : (i >> 3) * sbo + (k >> 3) * 128 + (i & 7) * 16 + (k & 7) * 2;
      *reinterpret_cast<__half *>(A + off) = __float2half((float)(((i * 7 + k * 3) % 9) - 4));
    }
    for (int e = t; e < N * 16; e += 128) {
      const int n = e >> 4, k = e & 15;
      const uint32_t off = mn ? (k >> 3) * ksb + (n >> 3) * 128 + (k & 7) * 16 + (n & 7) * 2
                              : (n >> 3) * sbo + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
      *reinterpret_cast<__half *>(B + off) = __float2half((float)(((n * 5 + k * 11) % 9) - 4));
    }
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      if (mn)
        mma_f16(tmem, sdesc(smem_u32(A), ksa, 128), sdesc(smem_u32(B), ksb, 128), idesc_f16_mn(128, N), 0u);
      else
        mma_f16(tmem, sdesc(smem_u32(A), 128, sbo), sdesc(smem_u32(B), 128, sbo), idesc_f16(128, N), 0u);
      mma_commit(&bar);
    }
    if (!mbar_wait(&bar, (uint32_t)layout & 1, status)) break;
    tc_fence_after();
    for (int cg = 0; cg < N / 16; ++cg) {
      float y[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cg * 16, y);
      for (int i = 0; i < 16; ++i) {
        const int n = cg * 16 + i;
        float ex = 0.f;
        for (int k = 0; k < 16; ++k) ex += (float)(((t * 7 + k * 3) % 9) - 4) * (float)(((n * 5 + k * 11) % 9) - 4);
        maxerr = fmaxf(maxerr, fabsf(y[i] - ex));
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  atomicMax(reinterpret_cast<int *>(err_out), __float_as_int(maxerr));
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

inline uint32_t rho_smem_bytes(int np, int nstages) { return 128u * np * 4 + (uint32_t)nstages * np * kRC * 4; }

// The dynamic shared memory a kernel can have next to its static shared memory (the static part
// rounded up to the 1024-byte alignment of the dynamic region), in whole KB.
template <typename K>
uint32_t dyn_smem_limit(K kern) {
  cudaFuncAttributes fa{};
  int dev = 0, optin = 227 * 1024;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const size_t stat = (fa.sharedSizeBytes + 1023) & ~(size_t)1023;
  return stat >= (size_t)optin ? 0u : (uint32_t)(((size_t)optin - stat) & ~(size_t)1023);
}

template <typename K>
int set_smem(K kern, uint32_t bytes) {
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
    return GINT_ECUDA;
  return GINT_OK;
}

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

}  // namespace

#define TC_CHECK(x)                            \
  do {                                         \
    if ((x) != cudaSuccess) return GINT_ECUDA; \
  } while (0)

void gint_tc_free(gint_handle *h) {
  h->tc_bytes = 0;
  dfree(h->plan);
  dfree(h->plan_off_dev);
  dfree(h->Dt_hl);
  dfree(h->Dt_hl2);
  dfree(h->zero_dev);
  dfree(h->tile_off_dev);
  dfree(h->scales);
  dfree(h->hs_brick_off);
  dfree(h->hs);
  dfree(h->hu_pair);
  dfree(h->hu_off);
  dfree(h->hu_src);
}

// Layouts of the tensor-core path for the current neighbour lists: D tile offsets, the padded
// brick width, the local-H scratch offsets and the per-pair contribution lists (host, fixed
// brick order so that the float64 reduction order is deterministic).
int gint_tc_prepare(gint_handle *h) {
  gint_tc_free(h);
  h->tc_at_off.clear();  // set again once every layout below is built
  h->tc_ent_off.clear();
  h->tc_satom.clear();
  const GGeom &g = h->geom;
  const int na_tot = g.natoms;
  // D tiles: roundup(norb(I), 8) x porb(J) per pair
  // D tiles: porb(I) x porb(J) per pair, stored column-atom-major (for each J its row atoms I in
  // ascending order), so that a brick's consecutive row atoms of one chunk are one copy
  auto find_pair = [&](int I, int J) -> int {
    auto b = h->pair_col.begin() + h->pair_row[I], e = h->pair_col.begin() + h->pair_row[I + 1];
    auto it = std::lower_bound(b, e, J);
    return (it != e && *it == J) ? (int)(it - h->pair_col.begin()) : -1;
  };
  h->tile_off.assign(h->npairs + 1, 0);
  {
    long long off = 0;
    for (int J = 0; J < na_tot; ++J)
      for (int q = h->pair_row[J]; q < h->pair_row[J + 1]; ++q) {
        const int I = h->pair_col[q];  // pair (J, I) exists, so (I, J) does too
        const int p = find_pair(I, J);
        if (p < 0) return GINT_EINVAL;
        h->tile_off[p] = off;
        off += (long long)g.sp[h->species_host[I]].porb * g.sp[h->species_host[J]].porb;
      }
    h->tile_off[h->npairs] = off;
  }
  h->ntile_elems = h->tile_off[h->npairs];
  const size_t tbytes = std::max<long long>(h->ntile_elems, 64) * sizeof(__half);
  if (cudaMalloc(&h->Dt_hl, 2 * tbytes) != cudaSuccess || cudaMalloc(&h->Dt_hl2, 2 * tbytes) != cudaSuccess ||
      cudaMalloc(&h->zero_dev, 512) != cudaSuccess ||
      cudaMalloc(&h->tile_off_dev, (h->npairs + 1) * sizeof(long long)) != cudaSuccess ||
      cudaMalloc(&h->scales, 8 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return GINT_ENOMEM;
  }
  TC_CHECK(cudaMemset(h->zero_dev, 0, 512));
  TC_CHECK(cudaMemset(h->scales, 0, 8 * sizeof(float)));
  TC_CHECK(cudaMemcpy(h->tile_off_dev, h->tile_off.data(), (h->npairs + 1) * sizeof(long long),
                      cudaMemcpyHostToDevice));
  // brick slot lists on the host
  const long long nb = g.nbricks;
  std::vector<long long> at_off(nb + 1);
  std::vector<int> satom(std::max<long long>(h->nslots, 1));
  TC_CHECK(cudaMemcpy(at_off.data(), h->b_at_off, (nb + 1) * sizeof(long long), cudaMemcpyDeviceToHost));
  if (h->nslots) TC_CHECK(cudaMemcpy(satom.data(), h->s_atom, h->nslots * sizeof(int), cudaMemcpyDeviceToHost));
  std::vector<long long> hs_off(nb + 1, 0);
  std::vector<long long> cnt(h->npairs + 1, 0);
  int npmax = 0;
  std::vector<long long> ent_off(nb + 1);
  TC_CHECK(cudaMemcpy(ent_off.data(), h->b_ent_off, (nb + 1) * sizeof(long long), cudaMemcpyDeviceToHost));
  std::vector<long long> plan_off(nb + 1, 0);  // plan records, 16-byte units
  // the bricks' slot-pair tables (global pair index or -1, row slot major), from the neighbour build
  std::vector<long long> bp_off(nb + 1);
  std::vector<int> bpair(std::max<long long>(h->npairtab, 1));
  TC_CHECK(cudaMemcpy(bp_off.data(), h->b_pair_off, (nb + 1) * sizeof(long long), cudaMemcpyDeviceToHost));
  if (h->npairtab) TC_CHECK(cudaMemcpy(bpair.data(), h->b_pair, h->npairtab * sizeof(int), cudaMemcpyDeviceToHost));
  // pass 1: sizes and counts, the bricks split into nthr contiguous ranges on host threads; each
  // range counts its own contributions per pair (tcnt), so that pass 2 can place them in brick
  // order without a shared cursor
  const int nthr = (int)std::max<long long>(1, std::min<long long>({16, (long long)std::thread::hardware_concurrency(),
                                                                      (nb + 1023) / 1024}));
  std::vector<long long> bstart(nthr + 1);
  for (int k = 0; k <= nthr; ++k) bstart[k] = nb * k / nthr;
  std::vector<std::vector<long long>> tcnt(nthr, std::vector<long long>(h->npairs, 0));
  std::vector<long long> hs_sz(nb), plan_sz(nb);
  std::vector<int> np_thr(nthr, 0);
  auto pass1 = [&](int k) {
    std::vector<int> nol;
    long long *tc = tcnt[k].data();
    for (long long b = bstart[k]; b < bstart[k + 1]; ++b) {
      const long long s0 = at_off[b], s1 = at_off[b + 1];
      int cur = 0;
      long long cum = 0;
      nol.assign(s1 - s0, 0);
      for (long long s = s0; s < s1; ++s) {
        const GSpecies &S = g.sp[h->species_host[satom[s]]];
        cur = place_slot(cur, S.porb) + S.porb;
        nol[s - s0] = S.norb;
        cum += S.norb;
      }
      np_thr[k] = std::max(np_thr[k], (cur + 15) & ~15);
      plan_sz[b] = plan_words((int)(s1 - s0), (int)(ent_off[b + 1] - ent_off[b]), (cur + 15) & ~15) / 4;
      long long tot = 0, rest = cum;
      for (long long a = 0; a < s1 - s0; ++a) {
        tot += (long long)nol[a] * rest;
        rest -= nol[a];
      }
      hs_sz[b] = (tot + 3) & ~3LL;  // 16-byte aligned ranges (one bulk copy each)
      const long long nab = s1 - s0;
      const int *bpb = bpair.data() + bp_off[b];
      for (long long a = 0; a < nab; ++a)
        for (long long c = a; c < nab; ++c) {
          const int p = bpb[a * nab + c];
          if (p >= 0) tc[p]++;
        }
    }
  };
  auto run_threads = [&](auto &&fn) {  // ranges 1.. on new threads (serially if none can start), 0 here
    std::vector<std::thread> th;
    int k = 1;
    try {
      for (; k < nthr; ++k) th.emplace_back(fn, k);
    } catch (...) {
    }
    for (int r = k; r < nthr; ++r) fn(r);
    fn(0);
    for (auto &t : th) t.join();
  };
  run_threads(pass1);
  for (long long b = 0; b < nb; ++b) {
    plan_off[b + 1] = plan_off[b] + plan_sz[b];
    hs_off[b + 1] = hs_off[b] + hs_sz[b];
  }
  for (int k = 0; k < nthr; ++k) {
    npmax = std::max(npmax, np_thr[k]);
    for (long long p = 0; p < h->npairs; ++p) cnt[p + 1] += tcnt[k][p];
  }
  h->max_brick_porb = npmax;
  h->hs_elems = hs_off[nb];
  // upper pairs (I <= J) and their contribution lists (CSR, brick order)
  std::vector<int> upair;
  std::vector<long long> uoff(1, 0);
  std::vector<long long> pstart(h->npairs, -1);
  for (int I = 0; I < na_tot; ++I)
    for (int p = h->pair_row[I]; p < h->pair_row[I + 1]; ++p)
      if (h->pair_col[p] >= I) {
        pstart[p] = uoff.back();
        upair.push_back(p);
        uoff.push_back(uoff.back() + cnt[p + 1]);
      }
  std::vector<long long> src(std::max<long long>(uoff.back(), 1));
  // each range's first place in every pair's list: the pair's start plus the earlier ranges' counts
  for (long long p = 0; p < h->npairs; ++p) {
    long long at = pstart[p];
    for (int k = 0; k < nthr; ++k) {
      const long long n = tcnt[k][p];
      tcnt[k][p] = at;
      at += n;
    }
  }
  auto pass2 = [&](int k) {
    std::vector<int> nol;
    long long *cur = tcnt[k].data();
    for (long long b = bstart[k]; b < bstart[k + 1]; ++b) {
      const long long s0 = at_off[b], s1 = at_off[b + 1];
      nol.assign(s1 - s0, 0);
      long long cum = 0;
      for (long long s = s0; s < s1; ++s) {
        nol[s - s0] = g.sp[h->species_host[satom[s]]].norb;
        cum += nol[s - s0];
      }
      long long rowst = 0, cumno_a = 0;
      const long long nab = s1 - s0;
      const int *bpb = bpair.data() + bp_off[b];
      for (long long a = 0; a < nab; ++a) {
        long long cumno_c = cumno_a;
        for (long long c = a; c < nab; ++c) {
          const int p = bpb[a * nab + c];
          if (p >= 0) src[cur[p]++] = hs_off[b] + rowst + (long long)nol[a] * (cumno_c - cumno_a);
          cumno_c += nol[c];
        }
        rowst += (long long)nol[a] * (cum - cumno_a);
        cumno_a += nol[a];
      }
    }
  };
  run_threads(pass2);
  h->nupper = (int)upair.size();
  if (cudaMalloc(&h->hs_brick_off, (nb + 1) * sizeof(long long)) != cudaSuccess ||
      cudaMalloc(&h->hs, std::max<long long>(h->hs_elems, 1) * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&h->hu_pair, std::max<size_t>(upair.size(), 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->hu_off, uoff.size() * sizeof(long long)) != cudaSuccess ||
      cudaMalloc(&h->hu_src, src.size() * sizeof(long long)) != cudaSuccess) {
    cudaGetLastError();
    return GINT_ENOMEM;
  }
  h->tc_bytes = 4 * (long long)tbytes + 512 + (h->npairs + 1) * (long long)sizeof(long long) + 8 * sizeof(float) +
                (nb + 1) * (long long)sizeof(long long) + std::max<long long>(h->hs_elems, 1) * (long long)sizeof(float) +
                (long long)std::max<size_t>(upair.size(), 1) * (long long)sizeof(int) +
                (long long)(uoff.size() + src.size()) * (long long)sizeof(long long);
  TC_CHECK(cudaMemcpy(h->hs_brick_off, hs_off.data(), (nb + 1) * sizeof(long long), cudaMemcpyHostToDevice));
  if (!upair.empty())
    TC_CHECK(cudaMemcpy(h->hu_pair, upair.data(), upair.size() * sizeof(int), cudaMemcpyHostToDevice));
  TC_CHECK(cudaMemcpy(h->hu_off, uoff.data(), uoff.size() * sizeof(long long), cudaMemcpyHostToDevice));
  TC_CHECK(cudaMemcpy(h->hu_src, src.data(), src.size() * sizeof(long long), cudaMemcpyHostToDevice));
  // brick plan records, built on the device by the slow-path metadata code itself
  if (cudaMalloc(&h->plan_off_dev, (nb + 1) * sizeof(long long)) != cudaSuccess ||
      cudaMalloc(&h->plan, std::max<long long>(plan_off[nb], 1) * 16) != cudaSuccess) {
    cudaGetLastError();
    return GINT_ENOMEM;
  }
  h->tc_bytes += (nb + 1) * (long long)sizeof(long long) + std::max<long long>(plan_off[nb], 1) * 16;
  TC_CHECK(cudaMemcpy(h->plan_off_dev, plan_off.data(), (nb + 1) * sizeof(long long), cudaMemcpyHostToDevice));
  // (bricks beyond the kernels' capacity get no records: compute calls report GINT_ECAPACITY)
  if (nb > 0 && h->max_brick_atoms <= kMAXA && h->max_brick_ent <= kMAXE && h->max_brick_porb <= kNPMAX) {
    TC_CHECK(cudaMemset(h->err_word, 0, sizeof(unsigned)));
    k_build_plans<<<(unsigned)nb, 128>>>(h->geom, static_cast<const GCell &>(h->geom), h->nbr(), h->tile_off_dev,
                                         h->plan_off_dev, reinterpret_cast<uint32_t *>(h->plan), h->err_word);
    TC_CHECK(cudaGetLastError());
    TC_CHECK(cudaDeviceSynchronize());
    unsigned err = 0;
    TC_CHECK(cudaMemcpy(&err, h->err_word, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (err) return GINT_EDEVICE;
  }
  satom.resize(h->nslots);
  h->tc_at_off.swap(at_off);
  h->tc_ent_off.swap(ent_off);
  h->tc_satom.swap(satom);
  return GINT_OK;
}

// New positions, neighbour lists rebuilt: when every brick keeps its slots (the same atoms in the
// same order) and its entry count, the D tile layout, the scratch ranges and the per-pair
// contribution lists stay valid and only the plan records (entry positions relative to the brick)
// change, so only k_build_plans runs again; otherwise the layouts are rebuilt (gint_tc_prepare).
int gint_tc_refresh(gint_handle *h) {
  const long long nb = h->geom.nbricks;
  if (!h->Dt_hl || !h->plan || (long long)h->tc_at_off.size() != nb + 1 ||
      (long long)h->tc_ent_off.size() != nb + 1 || (long long)h->tc_satom.size() != h->nslots)
    return gint_tc_prepare(h);
  std::vector<long long> at_off(nb + 1), ent_off(nb + 1);
  std::vector<int> satom(std::max<long long>(h->nslots, 1));
  TC_CHECK(cudaMemcpy(at_off.data(), h->b_at_off, (nb + 1) * sizeof(long long), cudaMemcpyDeviceToHost));
  TC_CHECK(cudaMemcpy(ent_off.data(), h->b_ent_off, (nb + 1) * sizeof(long long), cudaMemcpyDeviceToHost));
  if (h->nslots) TC_CHECK(cudaMemcpy(satom.data(), h->s_atom, h->nslots * sizeof(int), cudaMemcpyDeviceToHost));
  satom.resize(h->nslots);
  if (at_off != h->tc_at_off || ent_off != h->tc_ent_off || satom != h->tc_satom) return gint_tc_prepare(h);
  if (nb > 0 && h->max_brick_atoms <= kMAXA && h->max_brick_ent <= kMAXE && h->max_brick_porb <= kNPMAX) {
    TC_CHECK(cudaMemset(h->err_word, 0, sizeof(unsigned)));
    k_build_plans<<<(unsigned)nb, 128>>>(h->geom, static_cast<const GCell &>(h->geom), h->nbr(), h->tile_off_dev,
                                         h->plan_off_dev, reinterpret_cast<uint32_t *>(h->plan), h->err_word);
    TC_CHECK(cudaGetLastError());
    TC_CHECK(cudaDeviceSynchronize());
    unsigned err = 0;
    TC_CHECK(cudaMemcpy(&err, h->err_word, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (err) return GINT_EDEVICE;
  }
  return GINT_OK;
}

int gint_tc_check_capacity(const gint_handle *h) {
  if (h->max_brick_porb > kNPMAX || h->max_brick_atoms > kMAXA || h->max_brick_ent > kMAXE ||
      h->max_species_norb > GINT_MAX_ORB_ATOM || h->ntile_elems > 0x7fffffffLL || !h->Dt_hl)
    return GINT_ECAPACITY;
  return GINT_OK;
}

static_assert(sizeof(GTabs) + sizeof(GBatch) + 64 <= 32764, "brick kernel parameters exceed the launch limit");
static_assert(sizeof(GTabs) + sizeof(GTile) <= 32764 && sizeof(GTabs) + sizeof(GRed) <= 32764 &&
                  sizeof(GPrep) <= 32764,
              "batch kernel parameters exceed the launch limit");

// One launch group (at most kMaxBatch tasks, validated by the caller).  ev0 / ev1 (may be NULL)
// are recorded on the stream right before / after the brick kernel.
// Per-system descriptors of one task (density / force bricks need D, local H needs V).
static void fill_prep(GPrepSys &ps, const gint_task &T) {
  gint_handle *h = T.h;
  const bool dens = T.rho || T.F, loc = T.H_blocks != nullptr;
  ps.D = dens ? T.D_blocks : nullptr;
  ps.nblock = h->nblock;
  ps.V = (loc || T.F) ? T.V : nullptr;
  ps.ngrid = h->geom.ngrid;
  ps.F = T.F;
  ps.natoms = h->geom.natoms;
  ps.mx = reinterpret_cast<unsigned *>(h->scales + 4);
  ps.scales = h->scales;
  ps.phi_bound = h->phi_bound;
  ps.w = h->geom.w;
}
static void fill_tile(GTileSys &ts, const gint_task &T) {
  gint_handle *h = T.h;
  ts.D = T.D_blocks;
  ts.pair_I = h->pair_I_dev;
  ts.pair_J = h->pair_col_dev;
  ts.pair_off = h->pair_off_dev;
  ts.tile_off = h->tile_off_dev;
  ts.species = h->species_dev;
  ts.scales = h->scales;
  ts.Dhl = h->Dt_hl;
  ts.Dhl2 = h->Dt_hl2;
}
static void fill_sys(GSys &S, const gint_task &T) {
  gint_handle *h = T.h;
  const bool dens = T.rho || T.F, loc = T.H_blocks != nullptr;
  S.c = static_cast<const GCell &>(h->geom);
  S.nb = h->nbr();
  S.tab = h->tab32;
  S.tabi = h->tab32i;
  S.dtab = h->dtab32;
  S.dtabi = h->dtab32i;
  S.Dhl = h->Dt_hl;
  S.Dhl2 = h->Dt_hl2;
  S.tile_off = h->tile_off_dev;
  S.scales = h->scales;
  S.V = T.V;
  S.rho = T.rho;
  S.F = T.F;
  S.hs_brick_off = h->hs_brick_off;
  S.hs = h->hs;
  S.err = h->err_word;
  S.plan = h->plan;
  S.plan_off = h->plan_off_dev;
  S.do_rho = dens ? 1 : 0;
  S.do_h = loc ? 1 : 0;
}
static void fill_red_gamma(GRedSys &rs, const gint_task &T) {
  gint_handle *h = T.h;
  rs.hs = h->hs;
  rs.species = h->species_dev;
  rs.H = T.H_blocks;
  rs.hu_pair = h->hu_pair;
  rs.hu_off = h->hu_off;
  rs.hu_src = h->hu_src;
  rs.pair_I = h->pair_I_dev;
  rs.pair_J = h->pair_col_dev;
  rs.pair_T = h->pair_T_dev;
  rs.pair_off = h->pair_off_dev;
  rs.fp64 = h->reduce_fp64 ? 1 : 0;
}

static int run_group(const gint_task *tk, int n, int split3, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1) {
  gint_handle *h0 = tk[0].h;
  const GTabs &tabs = h0->geom;
  GPrep P{};
  GTile TB{};
  GBatch B{};
  GRed R{};
  P.nsys = n;
  P.work = h0->work_ctr;
  bool force = false;
  int np = kRC;
  long long items = 0, pairs = 0, uppers = 0;
  int nt = 0, nr = 0;
  for (int i = 0; i < n; ++i) {
    const gint_task &T = tk[i];
    gint_handle *h = T.h;
    const bool dens = T.rho || T.F, loc = T.H_blocks != nullptr;
    force |= T.F != nullptr;
    fill_prep(P.sys[i], T);
    if (dens && h->npairs > 0) {
      TB.start[nt] = pairs;
      fill_tile(TB.sys[nt++], T);
      pairs += h->npairs;
    }
    fill_sys(B.sys[i], T);
    B.start[i] = items;
    items += (dens || loc) ? h->geom.nbricks : 0;
    if (dens || loc) np = std::max(np, h->max_brick_porb);
    if (loc && (h->reduce_R ? h->r_nupper : h->nupper) > 0) {
      R.start[nr] = uppers;
      GRedSys &rs = R.sys[nr++];
      rs.hs = h->hs;
      rs.species = h->species_dev;
      rs.H = T.H_blocks;
      rs.fp64 = h->reduce_fp64 ? 1 : 0;
      if (h->reduce_R) {  // the same tiles keyed by (I, J, R): H(R) blocks
        rs.hu_pair = h->r_hu_key;
        rs.hu_off = h->r_hu_off;
        rs.hu_src = h->r_hu_src;
        rs.pair_I = h->r_kI;
        rs.pair_J = h->r_kJ;
        rs.pair_T = h->r_kT;
        rs.pair_off = h->r_koff;
        uppers += h->r_nupper;
      } else {
        rs.hu_pair = h->hu_pair;
        rs.hu_off = h->hu_off;
        rs.hu_src = h->hu_src;
        rs.pair_I = h->pair_I_dev;
        rs.pair_J = h->pair_col_dev;
        rs.pair_T = h->pair_T_dev;
        rs.pair_off = h->pair_off_dev;
        uppers += h->nupper;
      }
    }
  }
  B.nsys = n;
  B.start[n] = items;
  TB.nsys = nt;
  TB.start[nt] = pairs;
  TB.fixed = (force && split3) ? 1 : 0;
  R.nsys = nr;
  R.start[nr] = uppers;
  np = (np + 15) & ~15;
  // dynamic shared memory: P (hi, lo) | stage region (density chunk stages; afterwards the two W P
  // halves of the local-H pass) | tail pad read by the last 128-row A tile above NP
  // all the shared memory a CTA may have: items lay out P and as many stages as fit for their own
  // width (at least two stages at the widest brick of the launch)
  static const uint32_t smem = std::min(dyn_smem_limit(k_tc_fused<false>), dyn_smem_limit(k_tc_fused<true>));
  if (rho_smem_bytes(np, 2) + kHTail > smem) return GINT_ECAPACITY;
  B.np_max = np;
  B.split3 = split3;
  B.dsmem = (int)smem;
  const int bx = std::max(8, 2 * h0->num_sms / n);
  k_prep<<<dim3(bx, n), 256, 0, st>>>(P);
  k_prep_scales<<<1, kMaxBatch, 0, st>>>(P);
  TC_CHECK(cudaGetLastError());
  if (pairs > 0) {
    k_build_tiles<<<(unsigned)((pairs + kTileWarps - 1) / kTileWarps), 32 * kTileWarps, 0, st>>>(tabs, TB);
    TC_CHECK(cudaGetLastError());
  }
  if (items > 0) {
    const unsigned grid = (unsigned)std::min<long long>(h0->num_sms, items);
    auto kern = force ? k_tc_fused<true> : k_tc_fused<false>;
    int rc = set_smem(kern, smem);
    if (rc) return rc;
    if (ev0) TC_CHECK(cudaEventRecord(ev0, st));
    kern<<<grid, kT, smem, st>>>(tabs, B, h0->zero_dev, h0->work_ctr);
    TC_CHECK(cudaGetLastError());
    if (ev1) TC_CHECK(cudaEventRecord(ev1, st));
  }
  if (uppers > 0) {
    k_h_reduce<<<(unsigned)uppers, kRedThreads, 0, st>>>(tabs, R);
    TC_CHECK(cudaGetLastError());
  }
  return GINT_OK;
}

int gint_tc_batch(const gint_task *tasks, int n, int precision, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1) {
  if (n <= 0) return GINT_OK;
  const gint_handle *h0 = tasks[0].h;
  for (int i = 0; i < n; ++i) {
    const gint_task &T = tasks[i];
    const gint_handle *h = T.h;
    int rc = gint_tc_check_capacity(h);
    if (rc) return rc;
    if (T.H_blocks && h->max_brick_porb > kNPMAXH) return GINT_ECAPACITY;
    if (h->device != h0->device) return GINT_EINVAL;
    if (std::memcmp(static_cast<const GTabs *>(&h->geom), static_cast<const GTabs *>(&h0->geom), sizeof(GTabs)))
      return GINT_EINVAL;
    for (int j = 0; j < i; ++j)
      if (tasks[j].h == h) return GINT_EINVAL;
  }
  const int split3 = precision == GINT_F16X3 ? 1 : 0;
  for (int i0 = 0; i0 < n; i0 += kMaxBatch) {
    const bool first = i0 == 0, last = i0 + kMaxBatch >= n;
    int rc = run_group(tasks + i0, std::min(kMaxBatch, n - i0), split3, st, first ? ev0 : nullptr,
                       last ? ev1 : nullptr);
    if (rc) return rc;
  }
  return GINT_OK;
}

int gint_tc_rho(gint_handle *h, int precision, const double *D, double *rho, const double *V, double *F,
                cudaStream_t st) {
  const gint_task t{h, D, V, rho, nullptr, F};
  return gint_tc_batch(&t, 1, precision, st, nullptr, nullptr);
}

int gint_tc_vlocal(gint_handle *h, int precision, const double *V, double *H, cudaStream_t st) {
  const gint_task t{h, nullptr, V, nullptr, H, nullptr};
  return gint_tc_batch(&t, 1, precision, st, nullptr, nullptr);
}


// ------------------------------------------------------------------------------ serving API (host)
struct gint_server {
  int device = 0, forces = 1, split3 = 1, num_sms = 0, dsmem = 0;
  long long idle_ns = 0;
  GTabs tabs{};
  bool have_tabs = false, launched = false;
  GServeCtl *ctl = nullptr;
  GJob *jobs = nullptr;
  GJobState *st = nullptr;
  long long *job_end = nullptr;
  unsigned long long *done_h = nullptr, *done_d = nullptr;  // host-mapped completion words
  GJob *stage = nullptr;                                     // pinned staging, one per ring slot
  long long *stage_end = nullptr;
  unsigned long long *stage_tail = nullptr, *stage_misc = nullptr;
  __half *zero = nullptr;
  cudaStream_t kstream = nullptr, cstream = nullptr;
  cudaEvent_t kdone = nullptr, ev_in = nullptr;
  unsigned long long next_seq = 0, next_item = 0;
  gint_handle *slot_h[kServeRing] = {};
  long long launches = 0;
};

static int server_free(gint_server *v) {
  if (!v) return GINT_OK;
  if (v->ctl) cudaFree(v->ctl);
  if (v->jobs) cudaFree(v->jobs);
  if (v->st) cudaFree(v->st);
  if (v->job_end) cudaFree(v->job_end);
  if (v->zero) cudaFree(v->zero);
  if (v->done_h) cudaFreeHost(v->done_h);
  if (v->stage) cudaFreeHost(v->stage);
  if (v->stage_end) cudaFreeHost(v->stage_end);
  if (v->stage_tail) cudaFreeHost(v->stage_tail);
  if (v->stage_misc) cudaFreeHost(v->stage_misc);
  if (v->kstream) cudaStreamDestroy(v->kstream);
  if (v->cstream) cudaStreamDestroy(v->cstream);
  if (v->kdone) cudaEventDestroy(v->kdone);
  if (v->ev_in) cudaEventDestroy(v->ev_in);
  delete v;
  return GINT_OK;
}

static bool slot_done(const gint_server *v, unsigned long long seq) {
  return *(volatile unsigned long long *)&v->done_h[seq % kServeRing] == seq + 1;
}

// (Re)launches the resident kernel if it is not running; claims start at the oldest unfinished job.
static int server_launch(gint_server *v) {
  if (v->launched && cudaEventQuery(v->kdone) == cudaErrorNotReady) return GINT_OK;
  cudaGetLastError();
  unsigned long long first = v->next_seq;
  for (unsigned long long q = v->next_seq > kServeRing ? v->next_seq - kServeRing : 0; q < v->next_seq; ++q)
    if (!slot_done(v, q)) {
      first = q;
      break;
    }
  v->stage_misc[0] = first;
  if (cudaMemcpyAsync(&v->ctl->first_seq, v->stage_misc, sizeof(unsigned long long), cudaMemcpyHostToDevice,
                      v->kstream) != cudaSuccess)
    return GINT_ECUDA;
  auto kern = v->forces ? k_serve<true> : k_serve<false>;
  kern<<<v->num_sms, kT, v->dsmem, v->kstream>>>(v->tabs, v->ctl, v->jobs, v->st, v->job_end, v->done_d, v->zero,
                                                  v->split3, v->dsmem, v->idle_ns);
  if (cudaGetLastError() != cudaSuccess || cudaEventRecord(v->kdone, v->kstream) != cudaSuccess) return GINT_ECUDA;
  v->launched = true;
  ++v->launches;
  return GINT_OK;
}

extern "C" int gint_server_create(int precision, int forces, double idle_s, gint_server **out) {
  if (!out) return GINT_EINVAL;
  *out = nullptr;
  if (precision != GINT_F16X3 && precision != GINT_F16X1) return GINT_EUNSUPPORTED;
  if (!(idle_s > 0) || idle_s > 10.0) return GINT_EINVAL;
  gint_server *v = new gint_server();
  v->forces = forces ? 1 : 0;
  v->split3 = precision == GINT_F16X3 ? 1 : 0;
  v->idle_ns = (long long)(idle_s * 1e9);
  if (cudaGetDevice(&v->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&v->num_sms, cudaDevAttrMultiProcessorCount, v->device) != cudaSuccess) {
    server_free(v);
    return GINT_ECUDA;
  }
  v->dsmem = (int)std::min(dyn_smem_limit(k_serve<false>), dyn_smem_limit(k_serve<true>));
  bool okm = cudaMalloc(&v->ctl, sizeof(GServeCtl)) == cudaSuccess &&
             cudaMalloc(&v->jobs, kServeRing * sizeof(GJob)) == cudaSuccess &&
             cudaMalloc(&v->st, kServeRing * sizeof(GJobState)) == cudaSuccess &&
             cudaMalloc(&v->job_end, kServeMaxJobs * sizeof(long long)) == cudaSuccess &&
             cudaMalloc(&v->zero, 512) == cudaSuccess &&
             cudaHostAlloc(&v->done_h, kServeRing * sizeof(unsigned long long), cudaHostAllocMapped) == cudaSuccess &&
             cudaHostAlloc(&v->stage, kServeRing * sizeof(GJob), cudaHostAllocDefault) == cudaSuccess &&
             cudaHostAlloc(&v->stage_end, kServeRing * sizeof(long long), cudaHostAllocDefault) == cudaSuccess &&
             cudaHostAlloc(&v->stage_tail, kServeRing * sizeof(unsigned long long), cudaHostAllocDefault) == cudaSuccess &&
             cudaHostAlloc(&v->stage_misc, 8 * sizeof(unsigned long long), cudaHostAllocDefault) == cudaSuccess;
  if (!okm) {
    cudaGetLastError();
    server_free(v);
    return GINT_ENOMEM;
  }
  std::memset(v->done_h, 0, kServeRing * sizeof(unsigned long long));
  if (cudaHostGetDevicePointer((void **)&v->done_d, v->done_h, 0) != cudaSuccess ||
      cudaMemset(v->ctl, 0, sizeof(GServeCtl)) != cudaSuccess || cudaMemset(v->zero, 0, 512) != cudaSuccess ||
      cudaMemset(v->st, 0, kServeRing * sizeof(GJobState)) != cudaSuccess ||
      cudaMemset(v->job_end, 0, kServeMaxJobs * sizeof(long long)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&v->kstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&v->cstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&v->kdone, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&v->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      set_smem(k_serve<true>, (uint32_t)v->dsmem) != GINT_OK || set_smem(k_serve<false>, (uint32_t)v->dsmem) != GINT_OK) {
    cudaGetLastError();
    server_free(v);
    return GINT_ECUDA;
  }
  *out = v;
  return GINT_OK;
}

extern "C" int gint_server_submit(gint_server *v, const gint_task *T, void *stream, long long *ticket) {
  if (!v || !T || !T->h || !ticket) return GINT_EINVAL;
  gint_handle *h = T->h;
  const bool dens = T->rho || T->F, loc = T->H_blocks != nullptr;
  if ((!dens && !loc) || (dens && !T->D_blocks) || ((loc || T->F) && !T->V)) return GINT_EINVAL;
  if (T->F && !v->forces) return GINT_EINVAL;
  if (h->device != v->device) return GINT_EINVAL;
  int rc = gint_tc_check_capacity(h);
  if (rc) return rc;
  if (loc && h->max_brick_porb > kNPMAXH) return GINT_ECAPACITY;
  if (h->max_brick_porb + 0 > kNPMAX || rho_smem_bytes(std::max(h->max_brick_porb, kRC), 2) + kHTail > (uint32_t)v->dsmem)
    return GINT_ECAPACITY;
  if (!v->have_tabs) {
    v->tabs = h->geom;
    v->have_tabs = true;
  } else if (std::memcmp(static_cast<const GTabs *>(&h->geom), &v->tabs, sizeof(GTabs))) {
    return GINT_EINVAL;
  }
  if (v->next_seq >= (unsigned long long)kServeMaxJobs) return GINT_ECAPACITY;
  const unsigned long long seq = v->next_seq;
  const int slot = (int)(seq % kServeRing);
  if (seq >= (unsigned long long)kServeRing && !slot_done(v, seq - kServeRing)) return GINT_EBUSY;
  for (unsigned long long q = seq > kServeRing ? seq - kServeRing : 0; q < seq; ++q)
    if (v->slot_h[q % kServeRing] == h && !slot_done(v, q)) return GINT_EBUSY;  // one job per handle
  GJob &J = v->stage[slot];
  std::memset(&J, 0, sizeof(GJob));
  fill_sys(J.sys, *T);
  fill_prep(J.prep, *T);
  if (dens && h->npairs > 0) fill_tile(J.tile, *T);
  if (loc) fill_red_gamma(J.red, *T);
  J.npairs = dens ? h->npairs : 0;
  J.nupper = loc ? h->nupper : 0;
  J.fixed = (v->forces && v->split3) ? 1 : 0;
  J.nbricks = h->geom.nbricks;
  const long long span = std::max(std::max(h->nblock, h->geom.ngrid), 3LL * h->geom.natoms);
  J.n_prep = std::max(1LL, (span + kServePrep - 1) / kServePrep);
  J.n_tile = (J.npairs + kServeTilePairs - 1) / kServeTilePairs;
  J.n_red = (J.nupper + kServeRedPairs - 1) / kServeRedPairs;
  J.item0 = (long long)v->next_item;
  J.nitems = J.n_prep + 1 + J.n_tile + J.nbricks + J.n_red;
  J.seq = seq;
  cudaStream_t cs = (cudaStream_t)stream;
  v->done_h[slot] = 0;
  v->stage_end[slot] = J.item0 + J.nitems;
  v->stage_tail[slot] = (unsigned long long)(J.item0 + J.nitems);
  // inputs copied on the caller's stream first; then descriptor, counters, job end and the new tail
  if (cudaEventRecord(v->ev_in, cs) != cudaSuccess || cudaStreamWaitEvent(v->cstream, v->ev_in, 0) != cudaSuccess ||
      cudaMemcpyAsync(v->jobs + slot, &J, sizeof(GJob), cudaMemcpyHostToDevice, v->cstream) != cudaSuccess ||
      cudaMemsetAsync(v->st + slot, 0, sizeof(GJobState), v->cstream) != cudaSuccess ||
      cudaMemcpyAsync(v->job_end + seq, v->stage_end + slot, sizeof(long long), cudaMemcpyHostToDevice, v->cstream) !=
          cudaSuccess ||
      cudaMemcpyAsync(&v->ctl->tail, v->stage_tail + slot, sizeof(unsigned long long), cudaMemcpyHostToDevice,
                      v->cstream) != cudaSuccess)
    return GINT_ECUDA;
  v->slot_h[slot] = h;
  v->next_item += (unsigned long long)J.nitems;
  v->next_seq = seq + 1;
  *ticket = (long long)seq;
  return server_launch(v);
}

extern "C" int gint_server_test(gint_server *v, long long ticket, int *done) {
  if (!v || !done || ticket < 0 || (unsigned long long)ticket >= v->next_seq) return GINT_EINVAL;
  if ((unsigned long long)ticket + kServeRing < v->next_seq) {
    *done = 1;  // its slot has been reused: it completed
    return GINT_OK;
  }
  *done = slot_done(v, (unsigned long long)ticket) ? 1 : 0;
  if (*done) return GINT_OK;
  if (v->launched && cudaEventQuery(v->kdone) == cudaErrorNotReady) return GINT_OK;  // still resident
  cudaGetLastError();
  // the kernel has left: an error, or it went idle while this job's copies were still on their way
  GServeCtl c;
  if (cudaStreamSynchronize(v->cstream) != cudaSuccess ||
      cudaMemcpy(&c, v->ctl, sizeof(GServeCtl), cudaMemcpyDeviceToHost) != cudaSuccess)
    return GINT_ECUDA;
  if (c.err) return (c.err & GINT_ERRBIT_TIMEOUT) ? GINT_ETIMEDOUT : GINT_EDEVICE;
  *done = slot_done(v, (unsigned long long)ticket) ? 1 : 0;
  if (*done) return GINT_OK;
  return server_launch(v);  // its items are not all claimed: the kernel went idle before it was published
}

extern "C" int gint_server_stats(const gint_server *v, long long *launches, long long *jobs) {
  if (!v) return GINT_EINVAL;
  if (launches) *launches = v->launches;
  if (jobs) *jobs = (long long)v->next_seq;
  return GINT_OK;
}

extern "C" int gint_server_stop(gint_server *v) {
  if (!v) return GINT_EINVAL;
  if (!v->launched) return GINT_OK;
  v->stage_misc[1] = 1;
  if (cudaMemcpyAsync(&v->ctl->stop, v->stage_misc + 1, sizeof(int), cudaMemcpyHostToDevice, v->cstream) !=
          cudaSuccess ||
      cudaStreamSynchronize(v->cstream) != cudaSuccess || cudaEventSynchronize(v->kdone) != cudaSuccess)
    return GINT_ECUDA;
  v->stage_misc[1] = 0;
  if (cudaMemcpy(&v->ctl->stop, v->stage_misc + 1, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return GINT_ECUDA;
  v->launched = false;
  return GINT_OK;
}

extern "C" int gint_server_destroy(gint_server *v) {
  if (!v) return GINT_OK;
  const int rc = gint_server_stop(v);
  server_free(v);
  return rc;
}

extern "C" int gint_orbitals(gint_handle *h, int precision, long long npts, const double *pts, double *phi,
                             double *grad) {
  if (!h || npts < 0 || (npts > 0 && (!pts || !phi))) return GINT_EINVAL;
  if (precision != GINT_FP64 && precision != GINT_F16X3) return GINT_EUNSUPPORTED;
  if (h->max_species_norb > GINT_MAX_ORB_ATOM) return GINT_ECAPACITY;
  if (npts == 0) return GINT_OK;
  const int norb = h->norb, na = h->geom.natoms;
  double *dp = nullptr, *dphi = nullptr, *dgrad = nullptr;
  int *daoff = nullptr;
  int rc = GINT_OK;
  if (cudaMalloc(&dp, 3 * npts * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dphi, npts * norb * sizeof(double)) != cudaSuccess ||
      (grad && cudaMalloc(&dgrad, 3 * npts * norb * sizeof(double)) != cudaSuccess) ||
      cudaMalloc(&daoff, (na + 1) * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    rc = GINT_ENOMEM;
  }
  if (!rc && (cudaMemcpy(dp, pts, 3 * npts * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
              cudaMemcpy(daoff, h->atom_off.data(), (na + 1) * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess))
    rc = GINT_ECUDA;
  if (!rc) {
    const long long nt = npts * na;
    k_orbitals<<<(unsigned)((nt + 127) / 128), 128>>>(h->geom, h->tab64, h->tab32, h->tab32i, h->dtab32, h->dtab32i,
                                                      h->pos_dev, h->species_dev, daoff, npts, norb, dp,
                                                      precision == GINT_FP64 ? 1 : 0, dphi, dgrad);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = GINT_ECUDA;
  }
  if (!rc && (cudaMemcpy(phi, dphi, npts * norb * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
              (grad && cudaMemcpy(grad, dgrad, 3 * npts * norb * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)))
    rc = GINT_ECUDA;
  cudaFree(dp);
  cudaFree(dphi);
  cudaFree(dgrad);
  cudaFree(daoff);
  return rc;
}

extern "C" int gint_tc_selftest(int n, double *max_err) {
  if (n < 16 || n > 256 || (n % 16) || !max_err) return GINT_EINVAL;
  float *d_err = nullptr;
  unsigned *d_status = nullptr;
  if (cudaMalloc(&d_err, sizeof(float)) != cudaSuccess) return GINT_ENOMEM;
  if (cudaMalloc(&d_status, sizeof(unsigned)) != cudaSuccess) {
    cudaFree(d_err);
    return GINT_ENOMEM;
  }
  int rc = GINT_OK;
  cudaMemset(d_err, 0, sizeof(float));
  cudaMemset(d_status, 0, sizeof(unsigned));
  const uint32_t smem = 24 * 1024;  // A in [0, 8 KB), B in [8 KB, 24 KB) for every layout
  if (set_smem(k_tc_selftest, smem) != GINT_OK) rc = GINT_ECUDA;
  if (!rc) {
    k_tc_selftest<<<1, 128, smem>>>(n, d_err, d_status);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = GINT_ECUDA;
  }
  float e = -1.f;
  unsigned status = 0;
  if (!rc) {
    cudaMemcpy(&e, d_err, sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(&status, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (status) rc = GINT_ETIMEDOUT;
  }
  *max_err = (double)e;
  cudaFree(d_err);
  cudaFree(d_status);
  return rc;
}
