// Subspace rotation Psi = Y C of the FP32 state block on 5th-generation tensor cores (tcgen05), the
// last step of the Rayleigh-Ritz update of Sec. 2.2 (Eq. 1): psi_i(p) = sum_j y_j(p) C_ji per fragment.
//
// One 128-point tile of a fragment is one MMA problem D[128 points x nb] = A[128 x nb] B[nb x nb]^T with
// A(p, j) = y_j(p) and B(i, j) = C_ji (nb = the orbital count rounded up to 16).  Both operands are split
// into three BF16 words (y = h + m + l, exact to the last bit of FP32) and the six products that carry
// FP32 accuracy, hh hm hl mh mm lh, accumulate in FP32 in tensor memory over the nb-long contraction.
// Both operands use the K-major no-swizzle canonical layout (8-row core matrices of 16 bytes).
//
// Persistent CTAs (one per SM) run contiguous blocks of (fragment, tile) items as a warp-specialised
// pipeline:
//  - one thread loads each tile's [orbital][point] FP32 rows with one 2-D TMA copy (a tensor map over
//    the block as rows of P points, whose box is the fragment's orbital count rounded up to 8 rows, one
//    map per height; points past P arrive as zeros) into a ring of three raw tiles;
//  - eight converter warps transpose and split a raw tile into a BF16 stage (a thread takes one point
//    and eight orbitals: eight conflict-free shared loads, three 16-byte stores), two stages;
//  - one thread issues the tile's 6 x nb/16 MMAs into one of two tensor-memory accumulators;
//  - eight drain warps (two per tensor-memory lane group of 32 points, alternate column groups) store
//    Psi while the next tile's MMAs run into the other accumulator.
// The roles hand off through mbarriers; every wait is bounded (a timeout sets DC_FLAG_TIMEOUT and an
// abort word that ends every role's loop; the converters leave together after their own barrier).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "dc_internal.h"

namespace {

constexpr int RTM = 128;                   // points per tile (MMA M)
constexpr int RT_CONV = 256;               // converter threads (warps 0-7)
constexpr int RT_MMAW = 16;                // MMA warp (warps 8-15 drain: lane groups 0-3, two per group)
constexpr int RTNT = 32 * (RT_MMAW + 1);   // threads per CTA
constexpr int RT_NRAW = 3;                 // raw tiles in flight
constexpr int RT_NST = 2;                  // BF16 stages
constexpr int RT_ACC = 192;                // tensor-memory columns per accumulator: three blocks of up to 64
constexpr int RT_TMEM_COLS = 512;          // two accumulators
constexpr int RT_TP = 36;                  // drain transpose buffer row pitch (floats; 16-byte rows)
constexpr int RT_DRAIN_SM = 8 * 8 * RT_TP * 4;  // eight drain warps x [8 orbitals][32 points]

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle): start >> 4, leading byte offset (between core matrices
// adjacent in K) >> 4, stride byte offset (between core matrices adjacent in M/N) >> 4, version 1.
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

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)));
}

// Bounded wait for phase `parity`; gives up at once when another thread has set the abort word.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < DC_SPIN_LIMIT; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255 && *abort) return false;
  }
  *abort = 1;
  return false;
}

// One 32-lane x 8-column tensor-memory load (completed by a later wait).
__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(addr));
}

// Wait for every earlier tensor-memory load of the thread; the 24 registers named as in/out operands are
// not read before it.
__device__ __forceinline__ void tmem_wait24(uint32_t (&a)[8], uint32_t (&b)[8], uint32_t (&c)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                 "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]),
                 "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3]), "+r"(c[4]), "+r"(c[5]), "+r"(c[6]), "+r"(c[7]));
}

// 2-D TMA load of box (x = first point, y = first row) into shared memory, completion on `bar`.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(su32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

// byte offset of element (r, k) in a K-major tile with core-matrix column stride ks
__device__ __forceinline__ int toff(int r, int k, int ks) {
  return (k >> 3) * ks + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ float2 bf2_to_f2(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// Three-word BF16 split of two values: y = h + m + l per lane, each residual one paired FMA (exact).
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

__device__ __forceinline__ void split8(const float *v, uint4 &h, uint4 &m, uint4 &l) {
  split3x2(v[0], v[1], h.x, m.x, l.x);
  split3x2(v[2], v[3], h.y, m.y, l.y);
  split3x2(v[4], v[5], h.z, m.z, l.z);
  split3x2(v[6], v[7], h.w, m.w, l.w);
}

// Tensor maps over the block as rows of P points, box 128 points x 8 (k + 1) rows.  A box of the
// largest orbital count would also load the next fragment's rows: on the water cell (orbital counts
// 15-53) that doubled the rotation's reads of Y.
struct RotMaps {
  CUtensorMap m[8];
};

struct RotArgs {
  const FragDesc *desc;
  const int2 *items;  // (fragment, 128-point tile)
  const float *C;     // FP32 C per fragment (n x n at sub_off)
  float *out;         // Psi block
  unsigned *flags;
  int n_items;
  int nmax;
  long long P;        // points per fragment (the same for every fragment)
};

__global__ void __launch_bounds__(RTNT, 1) k_rotate_tc(const __grid_constant__ RotArgs a,
                                                       const __grid_constant__ RotMaps tmY) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t rfull[RT_NRAW], afull[RT_NST], aempty[RT_NST], dfull[2], dempty[2];
  __shared__ int abort_w;
  volatile int *abort = &abort_w;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nbm = (a.nmax + 15) & ~15;
  const int ksA = (RTM / 8) * 128, ksB = (3 * nbm / 8) * 128;  // B: rows [B_h | B_m | B_l], nb each
  const int abytes = RTM * nbm * 2, bbytes = nbm * nbm * 2;
  const int rawbytes = nbm * RTM * 4;  // one raw slot (the largest box: nbm rows of 128 points)
  // raw tiles [NRAW] (1024-aligned), BF16 stages [NST][3 words], B words [3]
  const int rawpitch = (rawbytes + 1023) & ~1023;
  float *raw0 = reinterpret_cast<float *>(sm);
  unsigned char *Aw = sm + RT_NRAW * rawpitch;
  unsigned char *Bw = Aw + RT_NST * 3 * abytes;
  float *tbuf = reinterpret_cast<float *>(Bw + 3 * bbytes);  // drain transposes
  const long long P = a.P;
  const int it0 = (int)(((long long)blockIdx.x * a.n_items) / gridDim.x);
  const int it1 = (int)(((long long)(blockIdx.x + 1) * a.n_items) / gridDim.x);
  const int nt = it1 - it0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)),
                 "r"(RT_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int k = 0; k < RT_NRAW; ++k) mbar_init(&rfull[k], 1);
    for (int k = 0; k < RT_NST; ++k) {
      mbar_init(&afull[k], RT_CONV);
      mbar_init(&aempty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&dfull[k], 1);
      mbar_init(&dempty[k], 256);
    }
    abort_w = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // operand padding (orbitals past n) stays zero: the stages and B are cleared once
  for (int t = tid; t < (RT_NST * 3 * abytes + 3 * bbytes) / 16; t += RTNT)
    reinterpret_cast<uint4 *>(Aw)[t] = make_uint4(0, 0, 0, 0);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tslot;
  int tcommit = 0;  // tiles whose MMAs the MMA thread has committed

  if (warp < RT_CONV / 32) {
    // ---- converters (thread 0 also issues the TMA loads) ----
    auto issue = [&](int t) {
      const int2 fi = a.items[it0 + t];
      const FragDesc &D = a.desc[fi.x];
      const int r = t % RT_NRAW;
      const int hb = (D.norb + 7) >> 3;  // box height in units of 8 rows
      mbar_expect_tx(&rfull[r], (uint32_t)(8 * hb * RTM * 4));
      tma_load_2d(reinterpret_cast<unsigned char *>(raw0) + r * rawpitch, &tmY.m[hb - 1], fi.y * RTM,
                  (int)(D.psi_off / P), &rfull[r]);
    };
    if (tid == 0)
      for (int t = 0; t < RT_NRAW && t < nt; ++t) issue(t);
    int cur_f = -1;
    for (int t = 0; t < nt; ++t) {
      const int2 fi = a.items[it0 + t];
      const FragDesc &D = a.desc[fi.x];
      const int n = D.norb, nb = (n + 15) & ~15;
      const int s = t % RT_NST, r = t % RT_NRAW;
      mbar_wait(&rfull[r], (uint32_t)((t / RT_NRAW) & 1), abort);
      mbar_wait(&aempty[s], (uint32_t)(((t / RT_NST) & 1) ^ 1), abort);
      if (fi.x != cur_f) {
        // a new fragment's B(i, j) = C_ji: every MMA of the previous tiles has completed (their commit
        // to aempty of tile t - 1 has fired) before B is overwritten
        if (t > 0) mbar_wait(&aempty[(t - 1) % RT_NST], (uint32_t)(((t - 1) / RT_NST) & 1), abort);
        // (the MMAs read rows i < nb and orbitals j < nb of it)
        const float *Cf = a.C + D.sub_off;
        for (int u = tid; u < nb * (nb / 8); u += RT_CONV) {
          const int i = u / (nb / 8), q = u - i * (nb / 8);
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int j = 8 * q + e;
            v[e] = (i < n && j < n) ? Cf[(long long)j * n + i] : 0.f;
          }
          uint4 h, m, l;
          split8(v, h, m, l);
          *reinterpret_cast<uint4 *>(Bw + toff(i, 8 * q, ksB)) = h;
          *reinterpret_cast<uint4 *>(Bw + toff(nb + i, 8 * q, ksB)) = m;
          *reinterpret_cast<uint4 *>(Bw + toff(2 * nb + i, 8 * q, ksB)) = l;
        }
        cur_f = fi.x;
      }
      // transpose-split: A(p, j) for eight orbitals j = 8q .. 8q + 7 of point p, j < nb (orbitals >= n are
      // zero; the MMAs read no orbital past nb, so the work follows the fragment's own count)
      const float *raw = reinterpret_cast<const float *>(reinterpret_cast<const unsigned char *>(raw0) + r * rawpitch);
      unsigned char *As = Aw + s * 3 * abytes;
      for (int u = tid; u < RTM * (nb / 8); u += RT_CONV) {
        const int q = u / RTM, p = u - q * RTM;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int j = 8 * q + e;
          v[e] = j < n ? raw[j * RTM + p] : 0.f;
        }
        uint4 h, m, l;
        split8(v, h, m, l);
        const int o = toff(p, 8 * q, ksA);
        *reinterpret_cast<uint4 *>(As + o) = h;
        *reinterpret_cast<uint4 *>(As + abytes + o) = m;
        *reinterpret_cast<uint4 *>(As + 2 * abytes + o) = l;
      }
      // the stage was written through ordinary stores; the MMAs read it through the async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&afull[s]);
      // every converter is done with raw tile r: refill it.  The barrier also ORs the converters' view of
      // the abort word, so that they all leave together.
      int any;
      asm volatile(
          "{\n.reg .pred pa, pr;\nsetp.ne.u32 pa, %1, 0;\nbar.red.or.pred pr, 1, %2, pa;\nselp.u32 %0, 1, 0, pr;\n}\n"
          : "=r"(any)
          : "r"((unsigned)*abort), "n"(RT_CONV)
          : "memory");
      if (any) break;
      if (tid == 0 && t + RT_NRAW < nt) issue(t + RT_NRAW);
    }
  } else if (warp < RT_MMAW) {
    // ---- drain warps: lanes 32 (warp % 4) .. + 31 of the accumulator = points, column groups of 8
    // alternating between the two warps of a lane group ----
    const int q4 = warp & 3, lane = tid & 31, gh = (warp - RT_CONV / 32) >> 2;
    for (int t = 0; t < nt; ++t) {
      const int b = t & 1;
      if (!mbar_wait(&dfull[b], (uint32_t)((t >> 1) & 1), abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int2 fi = a.items[it0 + t];
      const FragDesc &D = a.desc[fi.x];
      const int n = D.norb, nb = (n + 15) & ~15;
      float *of = a.out + D.psi_off;
      const uint32_t tl = tbase + (uint32_t)(b * RT_ACC) + ((uint32_t)(32 * q4) << 16);
      // this warp's column groups (up to four), two per wait: the three blocks of each group summed small to
      // large, then stored through a per-warp [8 orbitals][32 points] shared buffer, so that a lane writes 4
      // consecutive points of one orbital
      float *tb = tbuf + (warp - RT_CONV / 32) * 8 * RT_TP;
      const long long p0 = (long long)fi.y * RTM + 32 * q4;  // the warp's first point
#pragma unroll
      for (int jb = 0; jb < 4; jb += 2) {
        if (gh + 2 * jb >= nb / 8) break;  // warp-uniform
        uint32_t w[2][3][8];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int g = gh + 2 * (jb + u);
          if (g < nb / 8) {  // warp-uniform
            tmem_ld8(tl + 8 * g, w[u][0]);
            tmem_ld8(tl + nb + 8 * g, w[u][1]);
            tmem_ld8(tl + 2 * nb + 8 * g, w[u][2]);
          }
        }
        tmem_wait24(w[0][0], w[0][1], w[0][2]);
        tmem_wait24(w[1][0], w[1][1], w[1][2]);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int g = gh + 2 * (jb + u);
          if (g >= nb / 8) break;  // warp-uniform
          __syncwarp();  // the previous group's reads of the buffer are done
#pragma unroll
          for (int e = 0; e < 8; ++e)
            tb[e * RT_TP + lane] =
                __uint_as_float(w[u][0][e]) + (__uint_as_float(w[u][1][e]) + __uint_as_float(w[u][2][e]));
          __syncwarp();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int i = lane + 32 * h, e = i >> 3, q = i & 7;
            const long long pq = p0 + 4 * q;
            if (8 * g + e < n && pq < P)  // P is a multiple of 4: a quad lies wholly inside or outside
              *reinterpret_cast<float4 *>(of + (long long)(8 * g + e) * P + pq) =
                  *reinterpret_cast<const float4 *>(tb + e * RT_TP + 4 * q);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      mbar_arrive(&dempty[b]);
    }
  } else if (tid == 32 * RT_MMAW) {
    // ---- MMA issuer ----
    for (int t = 0; t < nt; ++t) {
      const int s = t % RT_NST, b = t & 1;
      if (!mbar_wait(&afull[s], (uint32_t)((t / RT_NST) & 1), abort)) break;
      if (!mbar_wait(&dempty[b], (uint32_t)(((t >> 1) & 1) ^ 1), abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int2 fi = a.items[it0 + t];
      const int nb = (a.desc[fi.x].norb + 15) & ~15;
      const uint32_t id3 = idesc_bf16(RTM, 3 * nb), id2 = idesc_bf16(RTM, 2 * nb), id1 = idesc_bf16(RTM, nb);
      const uint32_t a0 = su32(Aw + s * 3 * abytes), b0 = su32(Bw);
      const uint32_t td = tbase + (uint32_t)(b * RT_ACC);
      // blocks [hh + mh + lh | hm + mm | hl]: A_h [B_h | B_m | B_l]^T, A_m [B_h | B_m]^T, A_l B_h^T
      for (int kk = 0; kk < nb / 16; ++kk) {
        const uint64_t db = sdesc(b0 + kk * 2 * ksB, ksB, 128);
        mma_bf16(td, sdesc(a0 + kk * 2 * ksA, ksA, 128), db, id3, kk > 0 ? 1u : 0u);
        mma_bf16(td, sdesc(a0 + abytes + kk * 2 * ksA, ksA, 128), db, id2, 1u);
        mma_bf16(td, sdesc(a0 + 2 * abytes + kk * 2 * ksA, ksA, 128), db, id1, 1u);
      }
      mma_commit(&aempty[s]);
      mma_commit(&dfull[b]);
      ++tcommit;
    }
  }
  __syncthreads();
  if (*abort && tid == 0) atomicOr(a.flags, DC_FLAG_TIMEOUT);
  // every issued MMA has completed: the drains waited for each tile's commit.  After an abort the MMA
  // thread waits (bounded) for its last commit before the tensor memory is freed.
  if (*abort && tid == 32 * RT_MMAW && tcommit > 0) {
    const int t = tcommit - 1;
    uint32_t done = 0;
    for (uint32_t it = 0; it < DC_SPIN_LIMIT && !done; ++it)
      asm volatile(
          "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(su32(&aempty[t % RT_NST])), "r"((uint32_t)((t / RT_NST) & 1))
          : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(RT_TMEM_COLS));
}

}  // namespace

namespace dck {

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}
}  // namespace

bool tensor_map_rows(CUtensorMap *map, const float *base, long long inner, long long rows, int box_inner,
                     int box_rows, bool swizzle128) {
  const EncodeTiled enc = encode_fn();
  if (!enc || (inner & 3) || ((uintptr_t)base & 15)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)inner * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Psi = Y C on the tensor cores when the context qualifies (every fragment has the same point count P,
// a multiple of 4; at most 64 orbitals; 16-byte aligned blocks); DC_ERR_ARG otherwise, so that the
// caller can take the SIMT kernel.
int launch_rotate_tc(dc_ctx *c, const float *Y, float *out, cudaStream_t s) {
  const int nmax = c->layout.max_norb;
  const int nbm = (nmax + 15) & ~15;
  if (nbm > 64 || nmax <= 0 || c->n_rot_items <= 0) return DC_ERR_ARG;
  const FragDesc &D0 = c->h_desc[0];
  const long long P = (long long)D0.E[0] * D0.E[1] * D0.E[2];
  if (P & 3) return DC_ERR_ARG;
  for (const auto &D : c->h_desc)
    if ((long long)D.E[0] * D.E[1] * D.E[2] != P) return DC_ERR_ARG;
  if ((((uintptr_t)Y) | ((uintptr_t)out)) & 15) return DC_ERR_ARG;
  // the block as rows of P points, boxes of 128 points and 8, 16, .. nbm rows
  RotMaps maps{};
  for (int k = 0; k < nbm / 8; ++k)
    if (!tensor_map_rows(&maps.m[k], Y, P, c->layout.psi_elems / P, RTM, 8 * (k + 1), false)) return DC_ERR_ARG;
  RotArgs a;
  a.desc = c->d_desc;
  a.items = c->d_rot_items;
  a.C = c->d_C32;
  a.out = out;
  a.flags = c->d_flags;
  a.n_items = c->n_rot_items;
  a.nmax = nmax;
  a.P = P;
  const size_t rawpitch = ((size_t)nbm * RTM * 4 + 1023) & ~(size_t)1023;
  const size_t sm = RT_NRAW * rawpitch + (size_t)RT_NST * 3 * RTM * nbm * 2 + 3 * (size_t)nbm * nbm * 2 + RT_DRAIN_SM;
  DC_CUDA(dc_set_smem((const void *)k_rotate_tc, sm));
  const int grid = std::min(c->n_rot_items, c->sm_count);
  k_rotate_tc<<<(unsigned)grid, RTNT, sm, s>>>(a, maps);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

}  // namespace dck
