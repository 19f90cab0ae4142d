// Mixed-precision Gram and Rayleigh-Ritz contractions on 5th-generation tensor cores (tcgen05).
//
// S = Y Y^T and A = Y (HY)^T per fragment (K = fragment points, n <= 64 orbitals), the
// orthonormalisation and diagonalisation inputs of Sec. 2.2 (Eq. 1).  Every FP32 value is split
// into three BF16 words, y = h + m + l (exact up to the last bit), and the products that carry
// FP32 accuracy are accumulated in FP32 in tensor memory:
//   S = hh + hm + mh + hl + lh + mm            (lh = (hl)^T by symmetry)
//   A = h.zh + h.zm + m.zh + h.zl + l.zh + m.zm (z = HY split the same way)
// Persistent CTAs (one per SM, 16 warps) walk the (fragment, 2048-point item) list.  Per 64-point
// K-tile the CTA splits Y and HY into BF16 rows in shared memory (K-major, no-swizzle canonical
// layout), and one thread issues three MMAs per 16-point K-step:
//   D_S[128 x 3nb] = [Yh;Ym;Yl..] x [Yh|Ym|Yl]^T,  D_A[128 x 3nb] = [Yh;Ym;..] x [Zh|Zm|Zl]^T,
//   D_L[128 x nb]  = [Yl;0] x [Zh]^T                                   (nb = n rounded up to 16)
// with two K-tile stages in flight (mbarrier per stage) and the FP32 tiles of the next two K-tiles
// already loading into registers (16-byte loads).  The FP32 accumulators in tensor memory are
// drained every 256 points into FP32 sums in shared memory (the rounding of a tensor-memory sum
// grows with its length), and each item leaves as one FP64 partial of S and A that the FP64
// subspace kernel adds in a fixed order.  Every wait is bounded; on a timeout the kernel sets
// DC_FLAG_TIMEOUT, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "dc_internal.h"

namespace {

constexpr int TKT = 64;   // points per K-tile
constexpr int TNT = 512;  // threads per CTA
constexpr int TDR = 4;    // K-tiles per tensor-memory drain (256 points)
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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

// byte offset of element (r, k) in a K-tile with `rows` rows (K-major, no swizzle)
__device__ __forceinline__ int toff(int r, int k, int kstride) {
  return (k >> 3) * kstride + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Three-word BF16 split of two values at once: y = h + m + l per lane (paired conversions).
__device__ __forceinline__ void split3x2(float y0, float y1, uint32_t &h, uint32_t &m, uint32_t &l) {
  const __nv_bfloat162 hb = __floats2bfloat162_rn(y0, y1);
  const float r0 = y0 - __low2float(hb), r1 = y1 - __high2float(hb);
  const __nv_bfloat162 mb = __floats2bfloat162_rn(r0, r1);
  const float s0 = r0 - __low2float(mb), s1 = r1 - __high2float(mb);
  const __nv_bfloat162 lb = __floats2bfloat162_rn(s0, s1);
  h = *reinterpret_cast<const uint32_t *>(&hb);
  m = *reinterpret_cast<const uint32_t *>(&mb);
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

constexpr int TSL = 2;  // float4 slots per thread per array: 64 rows x 16 float4 / 512 threads

struct TileRegs {
  float4 y[TSL], z[TSL];
};

// Slot idx of a K-tile -> (row i, 4-point quad kq): a warp covers 8 rows x 4 quads, so its 8-byte
// shared-memory stores fill all 32 banks twice (16 rows apart in the canonical layout) instead of
// piling 16 lanes onto one core-matrix column.
__device__ __forceinline__ void tile_slot(int idx, int &i, int &kq) {
  i = ((idx >> 7) << 3) | (idx & 7);
  kq = (idx >> 3) & 15;
}

__device__ __forceinline__ void load_tile(TileRegs &r, const float *Yf, const float *Zf, long long P, int n,
                                          long long pb, long long p1, bool vec) {
#pragma unroll
  for (int j = 0; j < TSL; ++j) {
    const int idx = threadIdx.x + j * TNT;
    int i, kq;
    tile_slot(idx, i, kq);
    if (i < n) {
      const long long p = pb + 4 * kq;
      r.y[j] = ld4g(Yf + (long long)i * P, p, p1, vec);
      r.z[j] = ld4g(Zf + (long long)i * P, p, p1, vec);
    }
  }
}

// Split 4 consecutive-point values of row i into h/m/l rows (base row offsets 0, nb, 2 nb).
__device__ __forceinline__ void store_split(unsigned char *st, int i, int k, int ks, int nb, float4 v) {
  uint32_t h0, m0, l0, h1, m1, l1;
  split3x2(v.x, v.y, h0, m0, l0);
  split3x2(v.z, v.w, h1, m1, l1);
  *reinterpret_cast<uint2 *>(st + toff(i, k, ks)) = make_uint2(h0, h1);
  *reinterpret_cast<uint2 *>(st + toff(nb + i, k, ks)) = make_uint2(m0, m1);
  *reinterpret_cast<uint2 *>(st + toff(2 * nb + i, k, ks)) = make_uint2(l0, l1);
}

__device__ __forceinline__ void convert_tile(const TileRegs &r, unsigned char *ys, unsigned char *zs, int n, int nb,
                                             int ksY, int ksZ) {
#pragma unroll
  for (int j = 0; j < TSL; ++j) {
    const int idx = threadIdx.x + j * TNT;
    int i, kq;
    tile_slot(idx, i, kq);
    if (i < n) {
      const int k = 4 * kq;
      store_split(ys, i, k, ksY, nb, r.y[j]);
      store_split(zs, i, k, ksZ, nb, r.z[j]);
    }
  }
}

struct GramPipe {
  uint32_t phase[2];
  int commits[2], waits[2];
};

// Wait until every committed MMA group has completed.
__device__ __forceinline__ bool wait_all(GramPipe &g, uint64_t *mbar) {
  bool ok = true;
  for (int s = 0; s < 2; ++s) {
    while (g.commits[s] > g.waits[s]) {
      if (!mbar_wait(&mbar[s], g.phase[s])) ok = false;
      g.phase[s] ^= 1u;
      ++g.waits[s];
    }
  }
  return ok;
}

// Adds the tensor-memory accumulators into the FP32 sums: rows r < n (h rows) give
// P1S += hh + hm + hl, HL += hl, P1A += h.zh + h.zm + h.zl + l.zh; rows nb <= r < nb + n (m rows)
// give P2S += mh + mm, P2A += m.zh + m.zm.  Warp w reads lanes 32 (w % 4) .. +31 and the 8-column
// groups g with g % 4 == w / 4.
__device__ __forceinline__ void drain(uint32_t tS, uint32_t tA, uint32_t tL, int n, int nb, float *acc) {
  const int ld = n + 1;  // odd row stride: the 32 lanes (rows) of a warp hit 32 different banks
  float *P1S = acc, *HL = acc + n * ld, *P1A = HL + n * ld, *P2S = P1A + n * ld, *P2A = P2S + n * ld;
  const int warp = threadIdx.x >> 5;
  const int r = 32 * (warp & 3) + (threadIdx.x & 31);
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const bool own = r < n, mrow = (r >= nb && r < nb + n);
  const int i = own ? r : r - nb;
  for (int cg = 8 * (warp >> 2); cg < nb; cg += 32) {
    float sh[8], sm_[8], sl[8], ah[8], am[8], al[8], ll[8];
    tmem_ld8(tS + lane_base + cg, sh);
    tmem_ld8(tS + lane_base + nb + cg, sm_);
    tmem_ld8(tS + lane_base + 2 * nb + cg, sl);
    tmem_ld8(tA + lane_base + cg, ah);
    tmem_ld8(tA + lane_base + nb + cg, am);
    tmem_ld8(tA + lane_base + 2 * nb + cg, al);
    tmem_ld8(tL + lane_base + cg, ll);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = cg + e;
      if (j < n) {
        if (own) {
          P1S[i * ld + j] += sh[e] + sm_[e] + sl[e];
          HL[i * ld + j] += sl[e];
          P1A[i * ld + j] += ah[e] + am[e] + al[e] + ll[e];
        } else if (mrow) {
          P2S[i * ld + j] += sh[e] + sm_[e];
          P2A[i * ld + j] += ah[e] + am[e];
        }
      }
    }
  }
}

__global__ void __launch_bounds__(TNT, 1) k_gram_tc(const FragDesc *desc, const int2 *gitems, int n_items,
                                                    const long long *goff, int chunk, int nmax, const float *Y,
                                                    const float *HY, double *out, unsigned *flags) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int timed_out;
  const int tid = threadIdx.x;
  const int nbmax = (nmax + 15) & ~15;
  const int stage_max = (2 * nbmax + 128) * TKT * 2 + 3 * nbmax * TKT * 2;
  float *acc = reinterpret_cast<float *>(sm + 2 * stage_max);  // [5][n][n + 1]

  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    timed_out = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tslot;
  GramPipe g{{0u, 0u}, {0, 0}, {0, 0}};
  int gt = 0;         // K-tiles issued by this CTA (selects the stage)
  int prev_n = -1;

  for (int item = blockIdx.x; item < n_items && !timed_out; item += gridDim.x) {
    const int2 it = gitems[item];
    const int f = it.x, ch = it.y;
    const FragDesc D = desc[f];
    const int n = D.norb;
    const int nb = (n + 15) & ~15;
    const long long P = (long long)D.E[0] * D.E[1] * D.E[2];
    const long long p0 = (long long)ch * chunk;
    const long long p1 = min(P, p0 + chunk);
    const int Ry = 2 * nb + 128, Rz = 3 * nb;
    const int ksY = (Ry / 8) * 128, ksZ = (Rz / 8) * 128;
    const int ybytes = Ry * TKT * 2, zbytes = Rz * TKT * 2;
    const int stage_bytes = ybytes + zbytes;
    const float *Yf = Y + D.psi_off;
    const float *Zf = HY + D.psi_off;
    const bool vec = ((P | D.psi_off) & 3) == 0;
    const uint32_t tS = tbase, tA = tbase + 3 * nb, tL = tbase + 6 * nb;
    const uint32_t iS = idesc_bf16(128, 3 * nb), iL = idesc_bf16(128, nb);

    // stage padding rows must be zero for this orbital count (no MMA is in flight here)
    if (n != prev_n) {
      for (int t = tid; t < 2 * stage_bytes / 16; t += TNT) reinterpret_cast<uint4 *>(sm)[t] = make_uint4(0, 0, 0, 0);
      prev_n = n;
    }
    for (int t = tid; t < 5 * n * (n + 1); t += TNT) acc[t] = 0.f;
    const int ntiles = (int)((p1 - p0 + TKT - 1) / TKT);
    TileRegs ra, rb;
    load_tile(ra, Yf, Zf, P, n, p0, p1, vec);
    if (ntiles > 1) load_tile(rb, Yf, Zf, P, n, p0 + TKT, p1, vec);
    __syncthreads();

    for (int t = 0; t < ntiles; ++t) {
      const int s = gt & 1;
      if (g.commits[s] > g.waits[s]) {
        if (!mbar_wait(&mbar[s], g.phase[s])) timed_out = 1;
        g.phase[s] ^= 1u;
        ++g.waits[s];
      }
      __syncthreads();
      if (timed_out) break;
      unsigned char *ys = sm + s * stage_bytes;
      unsigned char *zs = ys + ybytes;
      // the registers of tile t hold ra (even t) or rb (odd t); refill them with tile t + 2
      if ((t & 1) == 0) {
        convert_tile(ra, ys, zs, n, nb, ksY, ksZ);
        if (t + 2 < ntiles) load_tile(ra, Yf, Zf, P, n, p0 + (long long)(t + 2) * TKT, p1, vec);
      } else {
        convert_tile(rb, ys, zs, n, nb, ksY, ksZ);
        if (t + 2 < ntiles) load_tile(rb, Yf, Zf, P, n, p0 + (long long)(t + 2) * TKT, p1, vec);
      }
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) {
        const uint32_t ya = su32(ys), za = su32(zs);
#pragma unroll
        for (int kk = 0; kk < TKT / 16; ++kk) {
          const uint32_t accum = (t % TDR != 0 || kk > 0) ? 1u : 0u;
          const uint64_t aY = sdesc(ya + kk * 2 * ksY, ksY, 128);
          const uint64_t aL = sdesc(ya + kk * 2 * ksY + (2 * nb / 8) * 128, ksY, 128);
          const uint64_t bZ = sdesc(za + kk * 2 * ksZ, ksZ, 128);
          mma_bf16(tS, aY, aY, iS, accum);
          mma_bf16(tA, aY, bZ, iS, accum);
          mma_bf16(tL, aL, bZ, iL, accum);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(&mbar[s])));
      }
      ++g.commits[s];
      ++gt;
      if (t % TDR == TDR - 1 || t == ntiles - 1) {
        if (!wait_all(g, mbar)) timed_out = 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (timed_out) break;
        drain(tS, tA, tL, n, nb, acc);
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
      }
    }
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
  // every committed MMA group has completed (or timed out) before the tensor memory is freed
  if (!wait_all(g, mbar) && tid == 0) atomicOr(flags, DC_FLAG_TIMEOUT);
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
  const size_t stage = (size_t)(2 * nb + 128) * TKT * 2 + (size_t)(3 * nb) * TKT * 2;
  const size_t sm = 2 * stage + 5 * (size_t)nmax * (nmax + 1) * sizeof(float);
  DC_CUDA(dc_set_smem((const void *)k_gram_tc, sm));
  const int grid = std::min(c->n_gram_items, c->sm_count);
  k_gram_tc<<<grid, TNT, sm, s>>>(c->d_desc, c->d_gram_items, c->n_gram_items, c->d_gram_off, c->gram_chunk, nmax,
                                  Y, HY, c->d_gram, c->d_flags);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

}  // namespace dck
