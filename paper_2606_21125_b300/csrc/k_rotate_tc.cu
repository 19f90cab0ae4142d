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
constexpr int RT_TMEM_COLS = 128;          // two accumulators of up to 64 columns
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
  const int ksA = (RTM / 8) * 128, ksB = (nbm / 8) * 128;
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
          const int o = toff(i, 8 * q, ksB);
          *reinterpret_cast<uint4 *>(Bw + o) = h;
          *reinterpret_cast<uint4 *>(Bw + bbytes + o) = m;
          *reinterpret_cast<uint4 *>(Bw + 2 * bbytes + o) = l;
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
      const uint32_t tl = tbase + (uint32_t)(b * 64) + ((uint32_t)(32 * q4) << 16);
      // all of this warp's column groups (up to four) with one wait, then each group through a per-warp
      // [8 orbitals][32 points] shared buffer, so that a lane stores 4 consecutive points of one orbital
      uint32_t v[4][8];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int g = gh + 2 * j;
        if (g < nb / 8)  // warp-uniform
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                       : "=r"(v[j][0]), "=r"(v[j][1]), "=r"(v[j][2]), "=r"(v[j][3]), "=r"(v[j][4]), "=r"(v[j][5]),
                         "=r"(v[j][6]), "=r"(v[j][7])
                       : "r"(tl + 8 * g));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;"
                   : "+r"(v[0][0]), "+r"(v[0][1]), "+r"(v[0][2]), "+r"(v[0][3]), "+r"(v[0][4]), "+r"(v[0][5]),
                     "+r"(v[0][6]), "+r"(v[0][7]), "+r"(v[1][0]), "+r"(v[1][1]), "+r"(v[1][2]), "+r"(v[1][3]),
                     "+r"(v[1][4]), "+r"(v[1][5]), "+r"(v[1][6]), "+r"(v[1][7]), "+r"(v[2][0]), "+r"(v[2][1]),
                     "+r"(v[2][2]), "+r"(v[2][3]), "+r"(v[2][4]), "+r"(v[2][5]), "+r"(v[2][6]), "+r"(v[2][7]),
                     "+r"(v[3][0]), "+r"(v[3][1]), "+r"(v[3][2]), "+r"(v[3][3]), "+r"(v[3][4]), "+r"(v[3][5]),
                     "+r"(v[3][6]), "+r"(v[3][7]));
      float *tb = tbuf + (warp - RT_CONV / 32) * 8 * RT_TP;
      const long long p0 = (long long)fi.y * RTM + 32 * q4;  // the warp's first point
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int g = gh + 2 * j;
        if (g >= nb / 8) break;  // warp-uniform
        __syncwarp();  // the previous group's reads of the buffer are done
#pragma unroll
        for (int e = 0; e < 8; ++e) tb[e * RT_TP + lane] = __uint_as_float(v[j][e]);
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
      const uint32_t id = idesc_bf16(RTM, nb);
      const uint32_t a0 = su32(Aw + s * 3 * abytes), b0 = su32(Bw);
      const uint32_t td = tbase + (uint32_t)(b * 64);
      // terms (A word, B word): hh hm hl mh mm lh
      for (int kk = 0; kk < nb / 16; ++kk) {
#pragma unroll
        for (int u = 0; u < 6; ++u) {
          const int wa = u < 3 ? 0 : (u < 5 ? 1 : 2);
          const int wb = u < 3 ? u : (u < 5 ? u - 3 : 0);
          const uint64_t da = sdesc(a0 + wa * abytes + kk * 2 * ksA, ksA, 128);
          const uint64_t db = sdesc(b0 + wb * bbytes + kk * 2 * ksB, ksB, 128);
          mma_bf16(td, da, db, id, (kk > 0 || u > 0) ? 1u : 0u);
        }
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
