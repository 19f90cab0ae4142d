// Mixed-precision Gram and Rayleigh-Ritz contractions on 5th-generation tensor cores (tcgen05).
//
// S = Y Y^T and A = Y (HY)^T per fragment (K = fragment points, n <= 64 orbitals), the
// orthonormalisation and diagonalisation inputs of Sec. 2.2 (Eq. 1).  Every FP32 value is split
// into three BF16 words, y = h + m + l (exact up to the last bit), and the products that carry
// FP32 accuracy are accumulated in FP32 in tensor memory:
//   S = hh + hm + mh + hl + lh + mm            (lh = (hl)^T by symmetry)
//   A = h.zh + h.zm + m.zh + h.zl + l.zh + m.zm (z = HY split the same way)
// One CTA (4 warps) handles one (fragment, 2048-point chunk).  Per 64-point K-tile the CTA splits
// Y and HY into BF16 rows in shared memory (K-major, no-swizzle canonical layout), and one thread
// issues three MMAs per 16-point K-step:
//   D_S[128 x 3nb] = [Yh;Ym;Yl..] x [Yh|Ym|Yl]^T,  D_A[128 x 3nb] = [Yh;Ym;..] x [Zh|Zm|Zl]^T,
//   D_L[128 x nb]  = [Yl;0] x [Zh]^T                                   (nb = n rounded up to 16)
// with two K-tile stages in flight (mbarrier per stage).  The chunk's partial S and A leave in FP64
// and the FP64 subspace kernel adds the chunks in a fixed order.  Every wait is bounded; on a
// timeout the kernel sets DC_FLAG_TIMEOUT, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "dc_internal.h"

namespace {

constexpr int TKT = 64;   // points per K-tile
constexpr int TNT = 128;  // threads per CTA
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

__device__ __forceinline__ void split3(float y, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
  h = __float2bfloat16_rn(y);
  const float r1 = y - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(m);
  l = __float2bfloat16_rn(r2);
}

__global__ void __launch_bounds__(TNT) k_gram_tc(const FragDesc *desc, const int2 *gitems, const long long *goff,
                                                 int chunk, const float *Y, const float *HY, double *out,
                                                 unsigned *flags) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ int timed_out;
  const int tid = threadIdx.x;
  const int2 it = gitems[blockIdx.x];
  const int f = it.x, ch = it.y;
  const FragDesc D = desc[f];
  const int n = D.norb;
  const int nb = (n + 15) & ~15;
  const long long P = (long long)D.E[0] * D.E[1] * D.E[2];
  const long long p0 = (long long)ch * chunk;
  const long long p1 = min(P, p0 + chunk);
  const int Ry = 2 * nb + 128, Rz = 3 * nb;
  const int ksY = (Ry / 8) * 128, ksZ = (Rz / 8) * 128;  // K-direction strides (8 K-columns apart)
  const int ybytes = Ry * TKT * 2, zbytes = Rz * TKT * 2;
  const int stage_bytes = ybytes + zbytes;
  const float *Yf = Y + D.psi_off;
  const float *Zf = HY + D.psi_off;

  // zero both stages: padding rows stay zero for the whole kernel
  for (int t = tid; t < 2 * stage_bytes / 16; t += TNT) reinterpret_cast<uint4 *>(sm)[t] = make_uint4(0, 0, 0, 0);
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
  const uint32_t tS = tbase, tA = tbase + 3 * nb, tL = tbase + 6 * nb;
  const uint32_t iS = idesc_bf16(128, 3 * nb), iL = idesc_bf16(128, nb);

  const int ntiles = (int)((p1 - p0 + TKT - 1) / TKT);
  uint32_t phase[2] = {0u, 0u};
  int commits[2] = {0, 0}, waits[2] = {0, 0};
  for (int t = 0; t < ntiles; ++t) {
    const int s = t & 1;
    if (commits[s] > waits[s]) {
      if (!mbar_wait(&mbar[s], phase[s])) timed_out = 1;
      phase[s] ^= 1u;
      ++waits[s];
    }
    __syncthreads();
    if (timed_out) break;
    unsigned char *ys = sm + s * stage_bytes;
    unsigned char *zs = ys + ybytes;
    const long long pb = p0 + (long long)t * TKT;
    for (int idx = tid; idx < n * (TKT / 2); idx += TNT) {
      const int i = idx / (TKT / 2);
      const int k = 2 * (idx - i * (TKT / 2));
      const long long p = pb + k;
      const float y0 = p < p1 ? Yf[(long long)i * P + p] : 0.f;
      const float y1 = p + 1 < p1 ? Yf[(long long)i * P + p + 1] : 0.f;
      const float z0 = p < p1 ? Zf[(long long)i * P + p] : 0.f;
      const float z1 = p + 1 < p1 ? Zf[(long long)i * P + p + 1] : 0.f;
      __nv_bfloat16 h0, m0, l0, h1, m1, l1;
      split3(y0, h0, m0, l0);
      split3(y1, h1, m1, l1);
      *reinterpret_cast<__nv_bfloat162 *>(ys + toff(i, k, ksY)) = __halves2bfloat162(h0, h1);
      *reinterpret_cast<__nv_bfloat162 *>(ys + toff(nb + i, k, ksY)) = __halves2bfloat162(m0, m1);
      *reinterpret_cast<__nv_bfloat162 *>(ys + toff(2 * nb + i, k, ksY)) = __halves2bfloat162(l0, l1);
      split3(z0, h0, m0, l0);
      split3(z1, h1, m1, l1);
      *reinterpret_cast<__nv_bfloat162 *>(zs + toff(i, k, ksZ)) = __halves2bfloat162(h0, h1);
      *reinterpret_cast<__nv_bfloat162 *>(zs + toff(nb + i, k, ksZ)) = __halves2bfloat162(m0, m1);
      *reinterpret_cast<__nv_bfloat162 *>(zs + toff(2 * nb + i, k, ksZ)) = __halves2bfloat162(l0, l1);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      const uint32_t ya = su32(ys), za = su32(zs);
#pragma unroll
      for (int kk = 0; kk < TKT / 16; ++kk) {
        const uint32_t acc = (t > 0 || kk > 0) ? 1u : 0u;
        const uint64_t aY = sdesc(ya + kk * 2 * ksY, ksY, 128);
        const uint64_t aL = sdesc(ya + kk * 2 * ksY + (2 * nb / 8) * 128, ksY, 128);
        const uint64_t bZ = sdesc(za + kk * 2 * ksZ, ksZ, 128);
        mma_bf16(tS, aY, aY, iS, acc);
        mma_bf16(tA, aY, bZ, iS, acc);
        mma_bf16(tL, aL, bZ, iL, acc);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(&mbar[s])));
    }
    ++commits[s];
  }
  // drain
  for (int s = 0; s < 2; ++s) {
    while (commits[s] > waits[s]) {
      if (!mbar_wait(&mbar[s], phase[s])) timed_out = 1;
      phase[s] ^= 1u;
      ++waits[s];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!timed_out) {
    // partial sums from each thread's own accumulator row (row = tid)
    float *P1S = reinterpret_cast<float *>(sm);  // [n][n] hh + hm + hl
    float *HL = P1S + n * n;                     // [n][n] hl
    float *P1A = HL + n * n;                     // [n][n] h.zh + h.zm + h.zl + l.zh
    float *P2S = P1A + n * n;                    // [n][n] mh + mm
    float *P2A = P2S + n * n;                    // [n][n] m.zh + m.zm
    const int warp = tid >> 5;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const int r = tid;
    const bool own = r < n, mrow = (r >= nb && r < nb + n);
    const int i = own ? r : r - nb;
    for (int cg = 0; cg < nb; cg += 8) {
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
        if (j >= n) break;
        if (own) {
          P1S[i * n + j] = sh[e] + sm_[e] + sl[e];
          HL[i * n + j] = sl[e];
          P1A[i * n + j] = ah[e] + am[e] + al[e] + ll[e];
        } else if (mrow) {
          P2S[i * n + j] = sh[e] + sm_[e];
          P2A[i * n + j] = ah[e] + am[e];
        }
      }
    }
    __syncthreads();
    double *o = out + goff[f] + (long long)ch * 2 * n * n;
    for (int t = tid; t < n * n; t += TNT) {
      const int a = t / n, b = t - a * n;
      o[t] = (double)P1S[t] + (double)P2S[t] + (double)HL[b * n + a];
      o[n * n + t] = (double)P1A[t] + (double)P2A[t];
    }
  } else if (tid == 0) {
    atomicOr(flags, DC_FLAG_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS));
}

}  // namespace

namespace dck {

int launch_gram_tc(dc_ctx *c, const float *Y, const float *HY, cudaStream_t s) {
  const int nb = (c->layout.max_norb + 15) & ~15;
  if (nb > 64) {
    dc_set_error("mixed-precision Gram needs n <= 64 orbitals per fragment");
    return DC_ERR_ARG;
  }
  const size_t stage = (size_t)(2 * nb + 128) * TKT * 2 + (size_t)(3 * nb) * TKT * 2;
  const size_t sm = 2 * stage;
  DC_CUDA(dc_set_smem((const void *)k_gram_tc, sm));
  k_gram_tc<<<c->n_gram_items, TNT, sm, s>>>(c->d_desc, c->d_gram_items, c->d_gram_off, c->gram_chunk, Y, HY,
                                            c->d_gram, c->d_flags);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

}  // namespace dck
