// Mixed-precision Gram and Rayleigh-Ritz contractions on 5th-generation tensor cores (tcgen05).
//
// S = Y Y^T and A = Y (HY)^T per fragment (K = fragment points, n <= 64 orbitals), the
// orthonormalisation and diagonalisation inputs of Sec. 2.2 (Eq. 1).  Every FP32 value is split
// into three BF16 words, y = h + m + l (exact up to the last bit), and the products that carry
// FP32 accuracy are accumulated in FP32 in tensor memory:
//   S = hh + hm + mh + hl + lh + mm            (lh = (hl)^T by symmetry)
//   A = h.zh + h.zm + m.zh + h.zl + l.zh + m.zm (z = HY split the same way)
// Persistent CTAs (one per SM, 16 warps) walk the (fragment, 4096-point item) list as a warp-
// specialised pipeline.  Seven converter warps bring 64-point K-tiles of Y and HY into a ring of
// raw FP32 tiles in shared memory (by TMA when the fragments share one shape, else by cp.async),
// split them into BF16 rows of a ring of shared-memory stages (K-major, no-swizzle canonical layout,
// rows [zh | h | m | l | zm | zl], nb each, then zero rows) and arrive on the stage's `full` barrier;
// one thread of warp 15 waits on it and issues three MMAs per 16-point K-step, the A operand being the
// 128 rows from h ([h; m] and the first l rows) or from l:
//   [A_h | S_h] = [h; m] [zh | h]^T                        (the large terms, N = 2 nb)
//   [S_r | A_r] = [h; m] [m | l | zm | zl]^T               (N = 4 nb)
//   L           = [l; ...] zh^T                            (N = nb, only the l rows are read)
// and commits them to the stage's `empty` barrier, which frees it for the converters.  (Five MMAs per
// K-step, one per block, re-read the 128-row A operand five times: on Si512 the MMA issue took ~1,360
// of a ~2,800-cycle tile period.)  The FP32
// accumulators in tensor memory are drained into FP32 sums kept in the registers of warps 7-14 (two
// warps per tensor-memory lane group, half the columns each): the large set every 256 points (the
// rounding of a tensor-memory sum grows with its length) from two alternating buffers, so that its
// drain runs while the MMAs fill the other buffer; the small set, ~2^-8 of the large one, every 1024
// points, when the MMA thread waits for it.  The register sums go to shared memory once per item.
// Each item leaves as one FP64 partial of S and A that the FP64 subspace kernel adds in a fixed
// order.  Every wait is bounded; after a timeout every later wait returns at once, the kernel sets
// DC_FLAG_TIMEOUT, waits (bounded) for its committed MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "dc_internal.h"

namespace {

constexpr int TKT = 64;   // points per K-tile
constexpr int TNT = 512;  // threads per CTA
// K-tiles per tensor-memory drain (256 points).  Longer FP32 accumulations were measured on Si512 (mixed
// vs FP64 energy difference after 43 steps, Gram time): 256 points 4.5e-7 Ha/atom, 1.09 ms; 512 points
// 9.2e-7, 0.92 ms; 1024 points 2.1e-6, 0.90 ms.  The 1e-6 Ha/atom budget keeps 256.
constexpr int TDR = 4;
// Large-set drain groups per small-set drain (1024 points).
constexpr int TSR = 4;
constexpr int TMEM_COLS = 512;

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle): start >> 4, leading byte offset (between core
// matrices adjacent in K) >> 4, stride byte offset (between core matrices adjacent in M/N) >> 4,
// descriptor version 1 at bit 46.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t kstride, uint32_t mnstride) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(kstride >> 4) << 16) | ((uint64_t)(mnstride >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, N, M.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

// Bounded wait; gives up at once when another thread of the CTA has already timed out.
__device__ __forceinline__ bool mbar_wait_or(uint64_t *bar, uint32_t phase, volatile int *timed_out) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < DC_SPIN_LIMIT; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(phase)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255 && *timed_out) return false;
  }
  *timed_out = 1;
  return false;
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < DC_SPIN_LIMIT; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(phase));
    if (done) return true;
  }
  return false;
}

// Three 32-lane x 8-column tensor-memory loads and one wait for all of them.  The wait names the 24
// destination registers as in/out operands, so nothing reads them before the loads have completed.
__device__ __forceinline__ void tmem_ld8x3(uint32_t t0, uint32_t t1, uint32_t t2, float *v0, float *v1, float *v2) {
  uint32_t r[24];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(t0));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(t1));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
                 "=r"(r[23])
               : "r"(t2));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v0[k] = __uint_as_float(r[k]);
    v1[k] = __uint_as_float(r[8 + k]);
    v2[k] = __uint_as_float(r[16 + k]);
  }
}

__device__ __forceinline__ void tmem_ld8x2(uint32_t t0, uint32_t t1, float *v0, float *v1) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(t0));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(t1));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v0[k] = __uint_as_float(r[k]);
    v1[k] = __uint_as_float(r[8 + k]);
  }
}

// byte offset of element (r, k) in a K-tile with `rows` rows (K-major, no swizzle)
__device__ __forceinline__ int toff(int r, int k, int kstride) {
  return (k >> 3) * kstride + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Three-word BF16 split of two values at once: y = h + m + l per lane.  Each residual is one paired
// FMA, y - h = fma(h, -1, y), exact like the scalar subtraction it replaces.
__device__ __forceinline__ float2 bf2_to_f2(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

__device__ __forceinline__ void split3x2(float y0, float y1, uint32_t &h, uint32_t &m, uint32_t &l) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 y = make_float2(y0, y1);
  const __nv_bfloat162 hb = __floats2bfloat162_rn(y0, y1);
  h = *reinterpret_cast<const uint32_t *>(&hb);
  const float2 r = __ffma2_rn(bf2_to_f2(h), m1, y);
  const __nv_bfloat162 mb = __floats2bfloat162_rn(r.x, r.y);
  m = *reinterpret_cast<const uint32_t *>(&mb);
  const float2 s = __ffma2_rn(bf2_to_f2(m), m1, r);
  const __nv_bfloat162 lb = __floats2bfloat162_rn(s.x, s.y);
  l = *reinterpret_cast<const uint32_t *>(&lb);
}

// Loads of one K-tile: rows i < n, points pb..pb+63, as 16 float4 per row (slots idx = tid + j*TNT).
__device__ __forceinline__ float4 ld4g(const float *row, long long p, long long p1, bool vec) {
  if (vec && p + 3 < p1) return *reinterpret_cast<const float4 *>(row + p);
  float4 v;
  v.x = p < p1 ? row[p] : 0.f;
  v.y = p + 1 < p1 ? row[p + 1] : 0.f;
  v.z = p + 2 < p1 ? row[p + 2] : 0.f;
  v.w = p + 3 < p1 ? row[p + 3] : 0.f;
  return v;
}

constexpr int TCV = 224;  // converter threads (warps 0-6); warps 7-14 drain, warp 15 issues the MMAs
constexpr int TSL = 5;    // float4 slots per converter thread per array: 64 rows x 16 float4 / 224

// Slot idx of a K-tile -> (row i, 4-point quad kq): a warp covers 8 rows x 4 quads, so its 8-byte
// shared-memory stores fill all 32 banks twice (16 rows apart in the canonical layout) instead of
// piling 16 lanes onto one core-matrix column.  Rows below n use slots idx < ((n + 7) / 8) * 128.
__device__ __forceinline__ void tile_slot(int idx, int &i, int &kq) {
  i = ((idx >> 7) << 3) | (idx & 7);
  kq = (idx >> 3) & 15;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(dst)), "l"(src) : "memory");
}

// Copy this thread's slots of the K-tile starting at point pb into one raw ring slot (raw[2][nslots]
// float4: Y then HY).  Aligned whole chunks go by cp.async; ragged or unaligned ones by plain loads,
// zero past p1.  Closes one copy group.
__device__ __forceinline__ void fetch_tile(float4 *raw, int nslots, const float *Yf, const float *Zf, long long P,
                                           int n, long long pb, long long p1, bool vec) {
#pragma unroll
  for (int j = 0; j < TSL; ++j) {
    const int idx = threadIdx.x + j * TCV;
    int i, kq;
    tile_slot(idx, i, kq);
    if (idx < 1024 && i < n) {
      const long long p = pb + 4 * kq;
      const float *yr = Yf + (long long)i * P, *zr = Zf + (long long)i * P;
      if (vec && p + 3 < p1) {
        cp_async16(&raw[idx], yr + p);
        cp_async16(&raw[nslots + idx], zr + p);
      } else {
        raw[idx] = ld4g(yr, p, p1, vec);
        raw[nslots + idx] = ld4g(zr, p, p1, vec);
      }
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Wait until at most `pending` of this thread's copy groups are still in flight.
__device__ __forceinline__ void cp_async_wait(int pending) {
  if (pending <= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
  else if (pending == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
  else asm volatile("cp.async.wait_group 2;" ::: "memory");
}

// Stage rows: [zh | h | m | l | zm | zl] (nb each), then zero rows up to the 128 that an A operand
// starting at l reads.
__host__ __device__ constexpr int stage_rows(int nb) { return 6 * nb > 3 * nb + 128 ? 6 * nb : 3 * nb + 128; }

// Split 4 consecutive-point values of one orbital into its three BF16 words, stored in rows rh, rm, rl.
__device__ __forceinline__ void store_split(unsigned char *st, int rh, int rm, int rl, int k, int ks, float4 v) {
  uint32_t h0, m0, l0, h1, m1, l1;
  split3x2(v.x, v.y, h0, m0, l0);
  split3x2(v.z, v.w, h1, m1, l1);
  *reinterpret_cast<uint2 *>(st + toff(rh, k, ks)) = make_uint2(h0, h1);
  *reinterpret_cast<uint2 *>(st + toff(rm, k, ks)) = make_uint2(m0, m1);
  *reinterpret_cast<uint2 *>(st + toff(rl, k, ks)) = make_uint2(l0, l1);
}

// Orbital i's value of Y into rows h, m, l and of HY into rows zh, zm, zl.
__device__ __forceinline__ void store_pair(unsigned char *st, int i, int k, int ks, int nb, float4 y, float4 z) {
  store_split(st, nb + i, 2 * nb + i, 3 * nb + i, k, ks, y);
  store_split(st, i, 4 * nb + i, 5 * nb + i, k, ks, z);
}

// Tensor maps over Y and HY as rows of P points, boxes of 32 points x 8 (k + 1) rows: a tile's boxes are
// the fragment's orbital count rounded up to 8 rows (a box of the largest count would also carry the next
// fragment's rows).
struct GramMaps {
  CUtensorMap y[8], z[8];
};

// TMA form of the raw ring: each array's K-tile arrives as two 32-point boxes (of up to nbmax rows, at
// nbmax-row spacing) with the 128-byte swizzle (16-byte chunk c of row i stored at chunk c ^ (i % 8)), so that the converters' reads
// (one warp: 8 rows x 4 quads) hit eight different chunks of a 128-byte line.
__device__ __forceinline__ float4 raw_tma(const unsigned char *slot, int nbmax, int a, int i, int kq) {
  return *reinterpret_cast<const float4 *>(slot + ((a * 2 + (kq >> 3)) * nbmax + i) * 128 + (((kq & 7) ^ (i & 7)) << 4));
}

__device__ __forceinline__ void convert_tile_tma(const unsigned char *slot, int nbmax, unsigned char *st, int n,
                                                 int nb, int ks) {
#pragma unroll
  for (int j = 0; j < TSL; ++j) {
    const int idx = threadIdx.x + j * TCV;
    int i, kq;
    tile_slot(idx, i, kq);
    if (idx < 1024 && i < n)
      store_pair(st, i, 4 * kq, ks, nb, raw_tma(slot, nbmax, 0, i, kq), raw_tma(slot, nbmax, 1, i, kq));
  }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(su32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void convert_tile(const float4 *raw, int nslots, unsigned char *st, int n, int nb,
                                             int ks) {
#pragma unroll
  for (int j = 0; j < TSL; ++j) {
    const int idx = threadIdx.x + j * TCV;
    int i, kq;
    tile_slot(idx, i, kq);
    if (idx < 1024 && i < n) store_pair(st, i, 4 * kq, ks, nb, raw[idx], raw[nslots + idx]);
  }
}

// Drain warps 7-14: warp w reads tensor-memory lanes 32 (w % 4) .. +31 (its rows r) and the
// 8-column groups 2 j + h (h = (w - 7) / 4, j < NG).  Rows r < n (h rows) keep P1S = hh + hm + hl,
// HL = hl, P1A = h.zh + h.zm + h.zl + l.zh; rows nb <= r < nb + n (m rows) keep P2S = mh + mm and
// P2A = m.zh + m.zm; columns past n and other rows add nothing.
//
// The accumulators come in two sets.  The large terms (the h-column blocks: hh and mh of S, h.zh and
// m.zh of A) are summed in FP32 in tensor memory over 256 points, the length the accuracy budget
// allows; they alternate between two buffers, so that the drain of one overlaps the MMAs into the
// other.  The remaining blocks (hm, hl, mm; h.zm, h.zl, m.zm; l.zh) are ~2^-8 of the large terms, so
// their FP32 rounding over 1024 points stays ~2^-6 below that of the large terms over 256: they are
// drained every 1024 points, and only then does the MMA thread wait for a drain.
template <int NG>
struct DrainRegs {
  float a0[8 * NG], a1[8 * NG], a2[8 * NG];
};

// The large set: S_h = [h; m] h^T and A_h = [h; m] zh^T.
template <int NG>
__device__ __forceinline__ void drain_big(DrainRegs<NG> &R, uint32_t tSh, uint32_t tAh, int n, int nb) {
  const int warp = threadIdx.x >> 5;
  const int half = (warp - 7) >> 2;
  const int r = 32 * (warp & 3) + (threadIdx.x & 31);
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const bool own = r < n, mrow = (r >= nb && r < nb + n);
#pragma unroll
  for (int j = 0; j < NG; ++j) {
    const int cg = 8 * (2 * j + half);
    if (cg >= nb) continue;  // warp-uniform
    float x0[8], y0[8];
    tmem_ld8x2(tSh + lane_base + cg, tAh + lane_base + cg, x0, y0);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (own) {
        R.a0[8 * j + e] += x0[e];
        R.a2[8 * j + e] += y0[e];
      } else if (mrow) {
        R.a0[8 * j + e] += x0[e];
        R.a1[8 * j + e] += y0[e];
      }
    }
  }
}

// The small set: S_r = [h; m] [m | l]^T, A_r = [h; m] [zm | zl]^T and L = [l; 0] zh^T.
template <int NG>
__device__ __forceinline__ void drain_small(DrainRegs<NG> &R, uint32_t tSr, uint32_t tAr, uint32_t tL, int n,
                                            int nb) {
  const int warp = threadIdx.x >> 5;
  const int half = (warp - 7) >> 2;
  const int r = 32 * (warp & 3) + (threadIdx.x & 31);
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const bool own = r < n, mrow = (r >= nb && r < nb + n);
#pragma unroll
  for (int j = 0; j < NG; ++j) {
    const int cg = 8 * (2 * j + half);
    if (cg >= nb) continue;  // warp-uniform
    float x1[8], x2[8], y3[8];
    tmem_ld8x3(tSr + lane_base + cg, tSr + lane_base + nb + cg, tL + lane_base + cg, x1, x2, y3);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (own) {
        R.a0[8 * j + e] += x1[e] + x2[e];
        R.a1[8 * j + e] += x2[e];
        R.a2[8 * j + e] += y3[e];
      } else if (mrow) {
        R.a0[8 * j + e] += x1[e];
      }
    }
    float y1[8], y2[8];
    tmem_ld8x2(tAr + lane_base + cg, tAr + lane_base + nb + cg, y1, y2);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (own) R.a2[8 * j + e] += y1[e] + y2[e];
      else if (mrow) R.a1[8 * j + e] += y1[e];
    }
  }
}

// The item's register sums to shared memory (row stride n + 1), each element by its one owner.
template <int NG>
__device__ __forceinline__ void drain_store(const DrainRegs<NG> &R, int n, int nb, float *acc) {
  const int ld = n + 1;
  float *P1S = acc, *HL = acc + n * ld, *P1A = HL + n * ld, *P2S = P1A + n * ld, *P2A = P2S + n * ld;
  const int warp = threadIdx.x >> 5;
  const int half = (warp - 7) >> 2;
  const int r = 32 * (warp & 3) + (threadIdx.x & 31);
  const bool own = r < n, mrow = (r >= nb && r < nb + n);
  const int i = own ? r : r - nb;
#pragma unroll
  for (int j = 0; j < NG; ++j) {
    const int cg = 8 * (2 * j + half);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int c = cg + e;
      if (c >= n) continue;
      if (own) {
        P1S[i * ld + c] = R.a0[8 * j + e];
        HL[i * ld + c] = R.a1[8 * j + e];
        P1A[i * ld + c] = R.a2[8 * j + e];
      } else if (mrow) {
        P2S[i * ld + c] = R.a0[8 * j + e];
        P2A[i * ld + c] = R.a1[8 * j + e];
      }
    }
  }
}

constexpr int TDW = 256;  // drain threads (warps 7-14)

template <int NG, bool TMA>
__global__ void __launch_bounds__(TNT, 1) k_gram_tc(const FragDesc *desc, const int2 *gitems, int n_items,
                                                    const long long *goff, int chunk, int nmax, int nstages,
                                                    int nraw, const float *Y, const float *HY, double *out,
                                                    unsigned *flags, const __grid_constant__ GramMaps tm) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t full[3], empty[3], dready_b[2], ddone_b[2], dready_s, ddone_s, rfull[3],
      rempty[3];
  __shared__ int timed_out;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const bool mma_warp = warp == TNT / 32 - 1;
  const int nbmax = (nmax + 15) & ~15;
  const int stage_max = stage_rows(nbmax) * TKT * 2;
  const int nslots = ((nmax + 7) / 8) * 128;                          // raw float4 slots per array
  float4 *rawring = reinterpret_cast<float4 *>(sm + nstages * stage_max);  // [nraw][2][nslots]
  // [5][n][n + 1] FP32 item sums.  They share the raw ring's space: the drains write them only after
  // the item's last tile has been converted (every copy into the ring has landed and been read), and
  // the next item's first copies start after the barrier that follows their read-out.
  float *acc = reinterpret_cast<float *>(rawring);

  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    timed_out = 0;
    for (int k = 0; k < 3; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&full[k])), "r"(TCV));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&empty[k])), "r"(1));
    }
    for (int k = 0; k < 2; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&dready_b[k])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&ddone_b[k])), "r"(TDW));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&dready_s)), "r"(1));
    for (int k = 0; k < 3; ++k) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&rfull[k])), "r"(4));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&rempty[k])), "r"(TCV));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&ddone_s)), "r"(TDW));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tslot;
  int gt = 0;     // K-tiles this CTA has passed through the ring (stage gt % nstages, use gt / nstages)
  int gr = 0;     // K-tiles loaded through the TMA raw ring (slot gr % nraw, its use gr / nraw)
  const int rslot = 4 * nbmax * 128;  // TMA raw slot: two arrays x two 32-point boxes of nbmax rows
  int gb = 0;     // large-set drain groups of this CTA (buffer gb % nbuf, its use gb / nbuf)
  int gs = 0;     // small-set drains of this CTA
  // tensor-memory columns (blocks sized for the largest orbital count): nbuf large-set buffers of
  // [A_h | S_h] (2 nbmax columns each), then [S_r | A_r] (4 nbmax) and L (nbmax)
  const int nbuf = 9 * nbmax <= TMEM_COLS ? 2 : 1;
  int prev_n = -1;
  int commits = 0;  // MMA groups committed by the MMA thread (tracked for the final wait)

  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int2 it = gitems[item];
    const int f = it.x, ch = it.y;
    const FragDesc D = desc[f];
    const int n = D.norb;
    const int nb = (n + 15) & ~15;
    const long long P = (long long)D.E[0] * D.E[1] * D.E[2];
    const long long p0 = (long long)ch * chunk;
    const long long p1 = min(P, p0 + chunk);
    const int ks = (stage_rows(nb) / 8) * 128;  // bytes per 8-point K column of a stage
    const int stage_bytes = stage_rows(nb) * TKT * 2;
    const float *Yf = Y + D.psi_off;
    const float *Zf = HY + D.psi_off;
    const bool vec = ((P | D.psi_off) & 3) == 0;
    const uint32_t tSr = tbase + 2 * nbuf * nbmax, tAr = tSr + 2 * nb, tL = tSr + 4 * nbmax;
    const uint32_t iN1 = idesc_bf16(128, nb), iN2 = idesc_bf16(128, 2 * nb), iN4 = idesc_bf16(128, 4 * nb);
    const int ntiles = (int)((p1 - p0 + TKT - 1) / TKT);

    // item start (the whole CTA is here, no MMA in flight): stage padding rows zero for this orbital
    // count, FP32 sums zero
    if (n != prev_n) {
      for (int t = tid; t < nstages * stage_bytes / 16; t += TNT)
        reinterpret_cast<uint4 *>(sm)[t] = make_uint4(0, 0, 0, 0);
      prev_n = n;
    }
    // ordinary stores into memory that the async proxy touches next (zeroed stages, which the MMAs
    // read; the item sums, whose space the next TMA tiles overwrite) are ordered before it here
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (timed_out) break;

    if (TMA && tid < TCV) {
      // ---- converters.  Each raw slot holds four 32-point boxes (Y and HY, two halves); box k of every
      // tile is issued by converter thread 64 k (warps 0, 2, 4, 6), once every converter has arrived on
      // the slot's `rempty` barrier after converting the tile that used it ----
      const int row0 = (int)(D.psi_off / P);
      unsigned char *rbase = reinterpret_cast<unsigned char *>(rawring);
      const int box = (tid & 63) == 0 ? tid >> 6 : -1;  // 0..3 on the issuing threads
      const int h8 = (n + 7) >> 3;                       // box height in units of 8 rows
      auto issue = [&](int t) {
        const int r = (gr + t) % nraw;
        unsigned char *dst = rbase + (size_t)r * rslot + box * nbmax * 128;
        // the slot was last accessed through ordinary loads and stores (tiles, item sums)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&rfull[r])),
                     "r"(8 * h8 * 128)
                     : "memory");
        tma_load_2d(dst, box < 2 ? &tm.y[h8 - 1] : &tm.z[h8 - 1], (int)(p0 + (long long)t * TKT) + 32 * (box & 1),
                    row0, &rfull[r]);
      };
      if (box >= 0)
        for (int t = 0; t < nraw && t < ntiles; ++t) issue(t);
      for (int t = 0; t < ntiles; ++t, ++gt) {
        const int s = gt % nstages;
        const uint32_t use = (uint32_t)(gt / nstages);
        const int r = (gr + t) % nraw;
        const uint32_t ruse = (uint32_t)((gr + t) / nraw);
        if (!mbar_wait_or(&rfull[r], ruse & 1u, &timed_out)) break;
        if (!mbar_wait_or(&empty[s], (use & 1u) ^ 1u, &timed_out)) break;
        convert_tile_tma(rbase + (size_t)r * rslot, nbmax, sm + s * stage_bytes, n, nb, ks);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&full[s]);
        mbar_arrive(&rempty[r]);
        if (box >= 0 && t + nraw < ntiles) {
          if (!mbar_wait_or(&rempty[r], ruse & 1u, &timed_out)) break;
          issue(t + nraw);
        }
      }
      gr += ntiles;
    } else if (tid < TCV) {
      // ---- converters: tile t's raw copy was issued nraw tiles earlier into ring slot t % nraw ----
      for (int r = 0; r < nraw; ++r) {
        if (r < ntiles) fetch_tile(rawring + (size_t)r * 2 * nslots, nslots, Yf, Zf, P, n, p0 + (long long)r * TKT,
                                   p1, vec);
        else asm volatile("cp.async.commit_group;" ::: "memory");
      }
      for (int t = 0; t < ntiles; ++t, ++gt) {
        const int s = gt % nstages;
        const uint32_t use = (uint32_t)(gt / nstages);
        float4 *raw = rawring + (size_t)(t % nraw) * 2 * nslots;
        cp_async_wait(nraw - 1);  // this thread's chunks of tile t have landed
        if (!mbar_wait_or(&empty[s], (use & 1u) ^ 1u, &timed_out)) break;
        convert_tile(raw, nslots, sm + s * stage_bytes, n, nb, ks);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&full[s]);
        // the slot's values are in the stage now: refill it with tile t + nraw
        if (t + nraw < ntiles)
          fetch_tile(raw, nslots, Yf, Zf, P, n, p0 + (long long)(t + nraw) * TKT, p1, vec);
        else
          asm volatile("cp.async.commit_group;" ::: "memory");
      }
      cp_async_wait(0);
    } else if (!mma_warp) {
      // ---- drain warps ----
      DrainRegs<NG> R;
#pragma unroll
      for (int k = 0; k < 8 * NG; ++k) R.a0[k] = R.a1[k] = R.a2[k] = 0.f;
      const int ngroups = (ntiles + TDR - 1) / TDR;
      for (int g = 0; g < ngroups; ++g) {
        const int bb = gb % nbuf, bu = gb / nbuf;
        if (!mbar_wait_or(&dready_b[bb], (uint32_t)(bu & 1), &timed_out)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        drain_big<NG>(R, tbase + 2 * bb * nbmax + nb, tbase + 2 * bb * nbmax, n, nb);  // S_h, A_h
        asm volatile("tcgen05.fence::before_thread_sync;");
        mbar_arrive(&ddone_b[bb]);
        ++gb;
        if (g % TSR == TSR - 1 || g == ngroups - 1) {
          if (!mbar_wait_or(&dready_s, (uint32_t)(gs & 1), &timed_out)) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          drain_small<NG>(R, tSr, tAr, tL, n, nb);
          asm volatile("tcgen05.fence::before_thread_sync;");
          mbar_arrive(&ddone_s);
          ++gs;
        }
      }
      drain_store<NG>(R, n, nb, acc);
    } else if ((tid & 31) == 0) {
      // ---- MMA issuer ----
      for (int t = 0; t < ntiles; ++t, ++gt) {
        const int s = gt % nstages;
        const uint32_t use = (uint32_t)(gt / nstages);
        const bool gstart = t % TDR == 0, wstart = t % (TDR * TSR) == 0;
        const int bb = gb % nbuf, bu = gb / nbuf;
        // a large-set buffer is overwritten only after its previous group has been drained (with two
        // buffers, the drain of the other one may still be running); the small set after its last drain
        if (gstart && bu > 0 && !mbar_wait_or(&ddone_b[bb], (uint32_t)((bu - 1) & 1), &timed_out)) break;
        if (wstart && gs > 0 && !mbar_wait_or(&ddone_s, (uint32_t)((gs - 1) & 1), &timed_out)) break;
        if (!mbar_wait_or(&full[s], use & 1u, &timed_out)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t sa = su32(sm + s * stage_bytes);
        const uint32_t tAh = tbase + 2 * bb * nbmax;  // [A_h | S_h]
        // the four operand descriptors of K-step 0; a K-step of 16 points advances each start address by
        // two core-matrix columns (the start field counts 16-byte units)
        const uint64_t dA = sdesc(sa + (nb / 8) * 128, ks, 128);      // A: 128 rows from h
        const uint64_t dAL = sdesc(sa + (3 * nb / 8) * 128, ks, 128); // A: 128 rows from l
        const uint64_t dB1 = sdesc(sa, ks, 128);                      // B: zh, h (N = nb or 2 nb)
        const uint64_t dB2 = sdesc(sa + (2 * nb / 8) * 128, ks, 128); // B: m, l, zm, zl
        const uint64_t stp = (uint64_t)((2 * ks) >> 4);
#pragma unroll
        for (int kk = 0; kk < TKT / 16; ++kk) {
          const uint32_t accB = (!gstart || kk > 0) ? 1u : 0u;
          const uint32_t accS = (!wstart || kk > 0) ? 1u : 0u;
          const uint64_t a = dA + kk * stp, b1 = dB1 + kk * stp;
          mma_bf16(tAh, a, b1, iN2, accB);                      // [h; m] [zh | h]^T
          mma_bf16(tSr, a, dB2 + kk * stp, iN4, accS);          // [h; m] [m | l | zm | zl]^T
          mma_bf16(tL, dAL + kk * stp, b1, iN1, accS);          // [l; ...] zh^T
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(&empty[s])));
        ++commits;
        if (t % TDR == TDR - 1 || t == ntiles - 1) {
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              su32(&dready_b[bb])));
          ++gb;
        }
        if (t % (TDR * TSR) == TDR * TSR - 1 || t == ntiles - 1) {
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              su32(&dready_s)));
          ++gs;
        }
      }
    } else {
      // lanes 1-31 of the MMA warp: no role
    }
    // every role counted the same tiles and drains
    __syncthreads();
    if (timed_out) break;
    // the item's partial sums, each element once: S = P1S + P2S + HL^T, A = P1A + P2A
    const int ld = n + 1;
    const float *P1S = acc, *HL = acc + n * ld, *P1A = HL + n * ld, *P2S = P1A + n * ld, *P2A = P2S + n * ld;
    double *o = out + goff[f] + (long long)ch * 2 * n * n;
    for (int t = tid; t < n * n; t += TNT) {
      const int a = t / n, b = t - a * n;
      const int u = a * ld + b;
      o[t] = (double)P1S[u] + (double)P2S[u] + (double)HL[b * ld + a];
      o[n * n + t] = (double)P1A[u] + (double)P2A[u];
    }
    __syncthreads();
  }
  if (timed_out && tid == 0) atomicOr(flags, DC_FLAG_TIMEOUT);
  // the MMA thread waits (bounded) for everything it committed before the tensor memory is freed
  if (mma_warp && (tid & 31) == 0 && commits > 0) {
    const int s = (gt - 1) % nstages;
    const uint32_t use = (uint32_t)((gt - 1) / nstages);
    if (!mbar_wait(&empty[s], use & 1u)) atomicOr(flags, DC_FLAG_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS));
}

}  // namespace

namespace dck {

int launch_gram_tc(dc_ctx *c, const float *Y, const float *HY, cudaStream_t s) {
  const int nmax = c->layout.max_norb;
  const int nb = (nmax + 15) & ~15;
  if (nb > 64) {
    dc_set_error("mixed-precision Gram needs n <= 64 orbitals per fragment");
    return DC_ERR_ARG;
  }
  // raw tiles by TMA when every fragment has the same point count P (a multiple of 4): the blocks are then
  // rows of P points, and a tile is two 32-point boxes per array of the fragment's orbital count rounded up
  // to 8 rows
  GramMaps maps{};
  bool tma = c->h_desc.size() > 0;
  const long long P0 = tma ? (long long)c->h_desc[0].E[0] * c->h_desc[0].E[1] * c->h_desc[0].E[2] : 0;
  for (const auto &D : c->h_desc)
    if ((long long)D.E[0] * D.E[1] * D.E[2] != P0) tma = false;
  tma = tma && (P0 & 3) == 0 && c->gram_chunk % TKT == 0;
  if (tma) {
    const long long rows = c->layout.psi_elems / P0;
    for (int k = 0; k < nb / 8 && tma; ++k)
      tma = tensor_map_rows(&maps.y[k], Y, P0, rows, 32, 8 * (k + 1), true) &&
            tensor_map_rows(&maps.z[k], HY, P0, rows, 32, 8 * (k + 1), true);
  }
  const size_t stage = (size_t)stage_rows(nb) * TKT * 2;
  const size_t rawslot = tma ? 4 * (size_t)nb * 128 : 2 * (size_t)((nmax + 7) / 8) * 128 * sizeof(float4);
  const size_t accb = 5 * (size_t)nmax * (nmax + 1) * sizeof(float);
  // deepest (BF16 stages, raw tiles) pair that fits: three stages let the conversion run two tiles
  // ahead of the MMA (which pauses for each drain), the raw ring keeps up to three tiles of loads in
  // flight; the FP32 item sums share the raw ring's space
  int nstages = 0, nraw = 0;
  for (int ns : {3, 2, 1}) {
    for (int nr : {3, 2, 1})
      if (ns * stage + std::max(nr * rawslot, accb) + 1024 <= 227 * 1024) {
        nstages = ns;
        nraw = nr;
        break;
      }
    if (nstages) break;
  }
  if (!nstages) {
    dc_set_error("mixed-precision Gram: tiles exceed shared memory");
    return DC_ERR_ARG;
  }
  const size_t sm = nstages * stage + std::max(nraw * rawslot, accb);
  const int grid = std::min(c->n_gram_items, c->sm_count);
  // column groups per drain warp: nb / 8 groups split over two warps per lane group
  const int ng = (nb / 8 + 1) / 2;
  auto run = [&](auto kern) -> int {
    DC_CUDA(dc_set_smem((const void *)kern, sm));
    kern<<<grid, TNT, sm, s>>>(c->d_desc, c->d_gram_items, c->n_gram_items, c->d_gram_off, c->gram_chunk, nmax,
                               nstages, nraw, Y, HY, c->d_gram, c->d_flags, maps);
    DC_CUDA(cudaGetLastError());
    return DC_OK;
  };
  if (tma) {
    switch (ng) {
      case 1: return run(k_gram_tc<1, true>);
      case 2: return run(k_gram_tc<2, true>);
      case 3: return run(k_gram_tc<3, true>);
      default: return run(k_gram_tc<4, true>);
    }
  }
  switch (ng) {
    case 1: return run(k_gram_tc<1, false>);
    case 2: return run(k_gram_tc<2, false>);
    case 3: return run(k_gram_tc<3, false>);
    default: return run(k_gram_tc<4, false>);
  }
}

}  // namespace dck
