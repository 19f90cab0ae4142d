// Specialised FP32 Chebyshev-step / H-apply kernel for cells whose fragments are all E^3 cubes with
// the zero (buffer-edge) boundary and equal grid spacing on the three axes (Eq. 5 model Hamiltonian:
// -1/2 L8 + V_f + sum_a D_a p_a <p_a|.>, 8th-order 25-point Laplacian).
//
// Same work decomposition as the general orbital-pair kernel: one CTA per (fragment, orbital pair),
// a float2 holds (y_i, y_i+1) at one grid point, each thread owns the x-adjacent points (x, x+1) of
// one row of the plane and streams z with its 9-deep column in registers; the haloed plane z sits in
// shared memory (its 4-point zero halo is written once) and the x and y taps are 16-byte shared
// loads covering both points.  What differs is that everything the general kernel decides at run
// time is fixed here at compile time: the extent E (so every shared-memory offset is an immediate
// and the (x, y) of a thread is a division by a constant), the boundary (no wrap-around stores),
// the isotropic stencil coefficients, the presence of Y_{k-1} and of output projections (template
// flags), and even extents (every point pair and every orbital row is 8-byte aligned, so each global
// access is one 8-byte load or store, without predicates).
//
// Data movement: the kernel is bound by memory latency unless several planes are in flight, and
// register prefetch holds at most one.  So one thread streams, for every plane z, the planes
// y_in(z + 4), y_prev(z) and V(z) with 1-D bulk asynchronous copies (cp.async.bulk, whole contiguous
// planes of the orbital-major layout, completion counted in bytes on an mbarrier) into a ring of
// RING slots in shared memory, RING - 1 planes ahead of their use; the other threads read their points
// from the ring.  Every wait on a slot is bounded: a thread that gives up sets the error flag and an
// abort word that every thread reads after the next barrier; the CTA then waits (bounded) for the
// copies still in flight and returns.
//
// Nonlocal term: the fragment's row lists (one entry per (row, projector slot) with gz gy != 0,
// host-built) are staged in shared memory once per CTA; each plane turns its entries into records
// (u_i gz gy, u_i+1 gz gy, the slot's x-factor offset, gz gy), u = D C <p|y>, in a three-slot ring;
// a point adds u gx[x] over its row's records.  The projections of the output, needed by the next
// Chebyshev step, are formed one plane behind by one task per record: gz gy sum_x gx[x] out(x, y)
// into a dense [row][slot] accumulator (one writer per element and plane), rows summed at the end.
// One barrier per plane.
#include <stdint.h>

#include <type_traits>

#include "dc_internal.h"

namespace {

struct ChebArgs {
  const FragDesc *desc;
  const int2 *items;      // (fragment, first orbital) per CTA
  const ProjSlot *slots;  // per (fragment, slot)
  const float *tab;       // FP32 projector factors
  const int *row_beg;     // per (fragment, z, y) start into row_ent
  const int2 *row_ent;    // (slot | y << 16, FP32 bits of gz gy)
  const double *Datom;
  const float *vf;        // V per fragment point (FP32)
  unsigned *flags;        // device error flags (DC_FLAG_TIMEOUT)
  const float *yin;
  const float *yprev;
  float *yout;
  const float *cin;       // projections <p|y_in> (n_f x A_f per fragment)
  float *cout;            // projections <p|y_out> (PROJ)
  const double *bounds;   // per fragment: a, b_up, aL, shift, 2m step coefficients
  int bstride;
  int step;
  int cheb;               // 0: out = H y; 1: out = alpha (H - shift) y + beta y_prev
  int maxent;             // max entries of one plane
  int amax, nentmax;      // max projector slots and row-list entries of one fragment (shared-memory carve)
  int n_items;            // work items (the CTAs are persistent: CTA b takes a contiguous block of items)
  float dV;
  float k1, k2, k3, k4, kc;  // -1/2 c_n / h^2 (n = 1..4) and the centre term -2 (k3 + k4) * 3 axes
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Projection tasks per record.  Splitting each record's x-support into two tasks with two accumulator
// planes spreads a plane's tasks over every warp, but the second accumulator plane took the shared
// memory of the second CTA per SM (Si, 22^3 fragments): 269 -> 394 us per launch on the 64-atom cell.
constexpr int kPSplit = 1;
// Task t runs on thread t, so a plane's ~110 tasks fill the first warps.  Spreading them one lane per
// warp per round (all warps then run the task loop) was slower: 270 -> 295 us per launch on the
// 64-atom cell (more issue slots outweighed the shorter barrier waits).

template <int E>
struct Geo {
  static constexpr int NPX = E / 2;                  // point pairs per row
  static constexpr int NP = NPX * E;                 // point pairs per plane
  static constexpr int NT = (NP + 31) / 32 * 32;     // threads per CTA
  static constexpr int PITCH = E + 16;               // haloed row pitch (float2), conflict-free
  static constexpr int HROWS = E + 8;
  static constexpr int PPLANE = PITCH * HROWS;       // one haloed plane (float2)
  static constexpr int PLANE = E * E;
  // Two 256-thread CTAs per SM.  Three (80 registers, two ring slots, the row-list entries read from
  // global memory to fit the shared memory) ran 311 us per launch on the 64-atom cell against 271.
  static constexpr int MINB = NT <= 256 ? 2 : 1;
  static constexpr int RING = 4;                     // plane slots in flight
};

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completion counted
// on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}

// Bounded wait for phase `parity` of `bar`; false when the poll limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < DC_SPIN_LIMIT; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Shared-memory carve (float2 units first, 16-byte aligned blocks).
template <int E>
struct ChebSmem {
  float2 *pin;   // [2][PPLANE]   haloed planes of y_in
  float2 *pout;  // [2][E*E]      output planes (projections)
  float2 *gx2;   // [A][E]        x factors, splatted (g, g)
  float2 *pacc;  // [kPSplit][E][A] projection accumulators
  float2 *sk2;   // [A]           D C <p|y> of the pair
  float4 *rec;   // [3][maxent]   per-plane records (a plane's records are read by its own stencil and, one
                 //               plane later, by its projection tasks, so three slots keep the writer of
                 //               plane z + 1 clear of both)
  int2 *sent;    // [nent]        the fragment's row-list entries
  int2 *box;     // [A]           even-aligned x support
  int *rb;       // [E*E + 1]     row starts (relative to the fragment's first entry)
  float *ring;   // [RING][NSUB][E*E] y_in(z + 4) (2 orbitals), [y_prev(z) (2 orbitals)], V(z)
  uint64_t *full;  // [RING] slot barriers
  volatile int *abort;  // set by a thread whose bounded wait ran out
  int *issued;          // [RING] uses of each slot so far (producer thread only)
  struct Hdr {
    const float *yin, *yprev, *vf;  // the pair's rows (orbital i; i + 1 at + E^3) and V of the fragment
    int nvalid;                     // 1 or 2 orbitals
    float2 ksh, al2, be2;           // kc - shift, alpha, beta (splatted)
  } *hdr;
};

// Planes per ring slot: y_in of the pair, y_prev of the pair (with PREV), V.
template <bool PREV>
__host__ __device__ constexpr int ring_sub() {
  return PREV ? 5 : 3;
}

template <int E, bool PREV>
__host__ __device__ inline size_t cheb_smem_bytes(int A, int maxent, int nent) {
  using G = Geo<E>;
  size_t b = (size_t)G::RING * ring_sub<PREV>() * G::PLANE * sizeof(float) + 256;  // ring, barriers, header
  size_t n2 = 2 * (size_t)G::PPLANE + 2 * (size_t)G::PLANE + (size_t)A * E + (size_t)kPSplit * E * A + A;
  b += (n2 * sizeof(float2) + 15) & ~(size_t)15;
  b += 3 * (size_t)maxent * sizeof(float4);
  b += (size_t)nent * sizeof(int2) + (size_t)A * sizeof(int2) + (size_t)(G::PLANE + 1) * sizeof(int);
  return b + 64;
}

template <int E, bool PREV>
__device__ __forceinline__ ChebSmem<E> cheb_carve(unsigned char *raw, int A, int maxent, int nent) {
  using G = Geo<E>;
  ChebSmem<E> m;
  m.ring = reinterpret_cast<float *>(raw);  // 16-byte aligned slots (E^2 floats are multiples of 16 bytes)
  unsigned char *after = raw + (size_t)G::RING * ring_sub<PREV>() * G::PLANE * sizeof(float);
  m.full = reinterpret_cast<uint64_t *>(after);
  m.abort = reinterpret_cast<volatile int *>(m.full + G::RING);
  m.issued = reinterpret_cast<int *>(m.full + G::RING) + 1;
  m.hdr = reinterpret_cast<typename ChebSmem<E>::Hdr *>(after + 64);
  after += 64 + 128;
  raw = after + 64;
  m.pin = reinterpret_cast<float2 *>(raw);
  m.pout = m.pin + 2 * G::PPLANE;
  m.gx2 = m.pout + 2 * G::PLANE;
  m.pacc = m.gx2 + A * E;
  m.sk2 = m.pacc + kPSplit * E * A;
  size_t off = (size_t)(reinterpret_cast<unsigned char *>(m.sk2 + A) - raw);
  off = (off + 15) & ~(size_t)15;
  m.rec = reinterpret_cast<float4 *>(raw + off);
  m.sent = reinterpret_cast<int2 *>(m.rec + 3 * maxent);
  m.box = m.sent + nent;
  m.rb = reinterpret_cast<int *>(m.box + A);
  return m;
}

// Per-thread state that the unrolled plane function reads.
struct ChebT {
  int px, py;      // owned points (px, py), (px + 1, py)
  bool active;     // owns a point pair
  int t0;          // py E + px
};

// Issue the bulk copies of plane z of the current item (y_in(z + 4), y_prev(z), V(z)) into ring slot
// gz % RING, gz = the CTA's running plane count (slots and their barrier phases continue from item to item).
template <int E, bool PREV>
__device__ __forceinline__ void ring_issue(const ChebSmem<E> &m, int z, int gz) {
  const typename ChebSmem<E>::Hdr &F = *m.hdr;
  using G = Geo<E>;
  constexpr uint32_t PB = G::PLANE * sizeof(float);
  constexpr long long P = (long long)G::PLANE * E;
  const int s = gz % G::RING;
  float *slot = m.ring + (size_t)s * ring_sub<PREV>() * G::PLANE;
  uint64_t *bar = m.full + s;
  const bool has_y = z + 4 < E;
  uint32_t bytes = PB;  // V
  if (has_y) bytes += F.nvalid * PB;
  if (PREV) bytes += F.nvalid * PB;
  // the slot was last read through ordinary shared loads (ordered before this by the CTA barrier); the
  // bulk copies write it through the async proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  m.issued[s] += 1;
  mbar_expect_tx(bar, bytes);
  if (has_y) {
    const float *src = F.yin + (long long)(z + 4) * G::PLANE;
    bulk_g2s(slot, src, PB, bar);
    if (F.nvalid > 1) bulk_g2s(slot + G::PLANE, src + P, PB, bar);
  }
  if (PREV) {
    const float *src = F.yprev + (long long)z * G::PLANE;
    bulk_g2s(slot + 2 * G::PLANE, src, PB, bar);
    if (F.nvalid > 1) bulk_g2s(slot + 3 * G::PLANE, src + P, PB, bar);
  }
  bulk_g2s(slot + (ring_sub<PREV>() - 1) * G::PLANE, F.vf + (long long)z * G::PLANE, PB, bar);
}

// Plane z.  The column registers q[k] hold plane z - 4 + k (q[8], plane z + 4, arrives from the ring
// during this plane) and are moved down by one plane at the end.  A loop over z with these moves runs
// faster than a body unrolled nine times that renames the registers instead: the unrolled kernel's
// instruction footprint stalled the warps on instruction fetch.  Returns false when the CTA aborts.
template <int E, bool PREV, bool PROJ>
__device__ __forceinline__ bool cheb_plane(const ChebArgs &a, const ChebSmem<E> &m, const ChebT &T, float4 (&q)[9],
                                           int z, int gbase, int A, float *yout) {
  using G = Geo<E>;
  const int slot = z & 1;
  float2 *P0 = m.pin + slot * G::PPLANE;
  const int c = (T.py + 4) * G::PITCH + T.px + 4;
  if (T.active) *reinterpret_cast<float4 *>(P0 + c) = q[4];
  // this plane's records from its row-list entries
  {
    const int e0 = m.rb[z * E], n = m.rb[(z + 1) * E] - e0;
    float4 *rc = m.rec + (z % 3) * a.maxent;
    for (int t = threadIdx.x; t < n; t += G::NT) {
      const int2 en = m.sent[e0 + t];
      const float w = __int_as_float(en.y);
      const int k = en.x & 0xffff;
      const float2 u = m.sk2[k];
      rc[t] = make_float4(u.x * w, u.y * w, __int_as_float(k * G::NPX), w);
    }
  }
  __syncthreads();
  if (*m.abort) return false;
  // refill the slot that plane z - 1 has finished with, for plane z - 1 + RING
  if (threadIdx.x == 0 && z >= 1 && z - 1 + G::RING < E) ring_issue<E, PREV>(m, z - 1 + G::RING, gbase + z - 1 + G::RING);
  // projections of the previous output plane
  if (PROJ && z > 0) {
    const int zp = z - 1, ps = zp & 1;
    const int e0 = m.rb[zp * E], n = m.rb[z * E] - e0;
    const float4 *rc = m.rec + ((z + 2) % 3) * a.maxent;
    const float4 *o4 = reinterpret_cast<const float4 *>(m.pout + ps * G::PLANE);
    const float4 *g4 = reinterpret_cast<const float4 *>(m.gx2);
    for (int t = threadIdx.x; t < kPSplit * n; t += G::NT) {
      const int e = t / kPSplit, part = t - e * kPSplit;
      const int kb = m.sent[e0 + e].x;
      const int k = kb & 0xffff, y = kb >> 16;
      const int2 bx = m.box[k];
      const int len = bx.y - bx.x;
      const int xa = bx.x + (part * len) / kPSplit, xb = bx.x + ((part + 1) * len) / kPSplit;
      const float4 *orow = o4 + y * G::NPX;
      const float4 *grow = g4 + k * G::NPX;
      float2 s0 = f2(0.f, 0.f), s1 = f2(0.f, 0.f);
      for (int x2 = xa; x2 < xb; ++x2) {
        const float4 o = orow[x2];
        const float4 g = grow[x2];
        s0 = fma2(lo2(o), lo2(g), s0);
        s1 = fma2(hi2(o), hi2(g), s1);
      }
      const float w = rc[e].w;
      float2 &pa = m.pacc[(part * E + y) * A + k];
      pa = fma2(f2(w, w), add2(s0, s1), pa);
    }
  }
  if (!T.active) return true;
  // this plane's ring slot: y_in(z + 4) completes the column; y_prev(z) and V(z)
  const int gz = gbase + z;
  if (!mbar_wait(m.full + gz % G::RING, (uint32_t)((gz / G::RING) & 1))) {
    atomicOr(a.flags, DC_FLAG_TIMEOUT);
    *m.abort = 1;
    return true;
  }
  const float *rs = m.ring + (size_t)(gz % G::RING) * ring_sub<PREV>() * G::PLANE + T.t0;
  const int nvalid = m.hdr->nvalid;
  {
    float4 nxt = make_float4(0.f, 0.f, 0.f, 0.f);
    if (z + 4 < E) {
      const float2 u0 = *reinterpret_cast<const float2 *>(rs);
      const float2 u1 = nvalid > 1 ? *reinterpret_cast<const float2 *>(rs + G::PLANE) : f2(0.f, 0.f);
      nxt = make_float4(u0.x, u1.x, u0.y, u1.y);
    }
    q[8] = nxt;  // plane z + 4
  }
  // Laplacian in difference form: taps 1, 2 as (y+n - y) + (y-n - y), taps 3, 4 as y+n + y-n with the
  // centre term added once; tap by tap, so each tap's loads die before the next are needed.
  // x neighbours of point 0 (x = px) and point 1 (px + 1): X0 = (px-4, px-3), X1 = (px-2, px-1),
  // centre (px, px+1), X3 = (px+2, px+3), X4 = (px+4, px+5), each float2 = the orbital pair
  const float2 *co = P0 + c;
  const float4 C = q[4];
  const float2 c0 = lo2(C), c1 = hi2(C);
  const float4 X1 = *reinterpret_cast<const float4 *>(co - 2);
  const float4 X3 = *reinterpret_cast<const float4 *>(co + 2);
  // H y without alpha: the taps, (kc - shift + V) y, then the nonlocal term
  float2 h0, h1;
  float2 t0, t1;
#define DC_YZ_TAPS(N, DIFF)                                                                                  \
  {                                                                                                        \
    const float4 U = *reinterpret_cast<const float4 *>(co + N * G::PITCH);                                 \
    const float4 Dn = *reinterpret_cast<const float4 *>(co - N * G::PITCH);                                \
    const float4 ZU = q[4 + N];                                                                 \
    const float4 ZD = q[4 - N];                                                                 \
    if (DIFF) {                                                                                            \
      t0 = add2(t0, add2(add2(sub2(lo2(U), c0), sub2(lo2(Dn), c0)), add2(sub2(lo2(ZU), c0), sub2(lo2(ZD), c0)))); \
      t1 = add2(t1, add2(add2(sub2(hi2(U), c1), sub2(hi2(Dn), c1)), add2(sub2(hi2(ZU), c1), sub2(hi2(ZD), c1)))); \
    } else {                                                                                               \
      t0 = add2(t0, add2(add2(lo2(U), lo2(Dn)), add2(lo2(ZU), lo2(ZD))));                                  \
      t1 = add2(t1, add2(add2(hi2(U), hi2(Dn)), add2(hi2(ZU), hi2(ZD))));                                  \
    }                                                                                                      \
  }
  // tap 1
  t0 = add2(sub2(c1, c0), sub2(hi2(X1), c0));
  t1 = add2(sub2(lo2(X3), c1), sub2(c0, c1));
  DC_YZ_TAPS(1, true)
  h0 = mul2(f2(a.k1, a.k1), t0);
  h1 = mul2(f2(a.k1, a.k1), t1);
  // tap 2
  t0 = add2(sub2(lo2(X3), c0), sub2(lo2(X1), c0));
  t1 = add2(sub2(hi2(X3), c1), sub2(hi2(X1), c1));
  DC_YZ_TAPS(2, true)
  h0 = fma2(f2(a.k2, a.k2), t0, h0);
  h1 = fma2(f2(a.k2, a.k2), t1, h1);
  // taps 3 and 4
  const float4 X0 = *reinterpret_cast<const float4 *>(co - 4);
  const float4 X4 = *reinterpret_cast<const float4 *>(co + 4);
  t0 = add2(hi2(X3), hi2(X0));
  t1 = add2(lo2(X4), lo2(X1));
  DC_YZ_TAPS(3, false)
  h0 = fma2(f2(a.k3, a.k3), t0, h0);
  h1 = fma2(f2(a.k3, a.k3), t1, h1);
  t0 = add2(lo2(X4), lo2(X0));
  t1 = add2(hi2(X4), hi2(X0));
  DC_YZ_TAPS(4, false)
  h0 = fma2(f2(a.k4, a.k4), t0, h0);
  h1 = fma2(f2(a.k4, a.k4), t1, h1);
#undef DC_YZ_TAPS
  {
    const float2 ksh = m.hdr->ksh;
    const float2 vr = *reinterpret_cast<const float2 *>(rs + (ring_sub<PREV>() - 1) * G::PLANE);
    h0 = fma2(ksh, c0, fma2(f2(vr.x, vr.x), c0, h0));
    h1 = fma2(ksh, c1, fma2(f2(vr.y, vr.y), c1, h1));
  }
  // nonlocal term over the row's records
  {
    const int rz = z * E + T.py;
    const int eb = m.rb[rz] - m.rb[z * E], ee = m.rb[rz + 1] - m.rb[z * E];
    const float4 *rc = m.rec + (z % 3) * a.maxent;
    const float4 *g4 = reinterpret_cast<const float4 *>(m.gx2) + (T.px >> 1);
    int e = eb;
    for (; e + 1 < ee; e += 2) {
      const float4 ra = rc[e], rb = rc[e + 1];
      const float4 ga = g4[__float_as_int(ra.z)], gb = g4[__float_as_int(rb.z)];
      h0 = fma2(lo2(ra), lo2(ga), h0);
      h1 = fma2(lo2(ra), hi2(ga), h1);
      h0 = fma2(lo2(rb), lo2(gb), h0);
      h1 = fma2(lo2(rb), hi2(gb), h1);
    }
    if (e < ee) {
      const float4 ra = rc[e];
      const float4 ga = g4[__float_as_int(ra.z)];
      h0 = fma2(lo2(ra), lo2(ga), h0);
      h1 = fma2(lo2(ra), hi2(ga), h1);
    }
  }
  float2 o0, o1;
  const float2 al2 = m.hdr->al2;
  if (PREV) {
    const float2 be2 = m.hdr->be2;
    const float2 u0 = *reinterpret_cast<const float2 *>(rs + 2 * G::PLANE);
    const float2 u1 = nvalid > 1 ? *reinterpret_cast<const float2 *>(rs + 3 * G::PLANE) : f2(0.f, 0.f);
    o0 = fma2(al2, h0, mul2(be2, f2(u0.x, u1.x)));
    o1 = fma2(al2, h1, mul2(be2, f2(u0.y, u1.y)));
  } else {
    o0 = mul2(al2, h0);
    o1 = mul2(al2, h1);
  }
  {
    float *po = yout + z * G::PLANE + T.t0;
    *reinterpret_cast<float2 *>(po) = f2(o0.x, o1.x);
    if (nvalid > 1) *reinterpret_cast<float2 *>(po + E * G::PLANE) = f2(o0.y, o1.y);
  }
  if (PROJ)
    *reinterpret_cast<float4 *>(m.pout + slot * G::PLANE + T.t0) =
        make_float4(o0.x, nvalid > 1 ? o0.y : 0.f, o1.x, nvalid > 1 ? o1.y : 0.f);
#pragma unroll
  for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
  return true;
}

// Persistent CTAs: CTA b runs the contiguous block of work items [b n / G, (b + 1) n / G) (all items cost
// the same: one orbital pair of an E^3 fragment).  Consecutive items are mostly the same fragment, whose
// tables (x factors, supports, row lists) stay in shared memory; only the pair's projections are read
// again.  The ring's slots and barrier phases run on across items.
template <int E, bool PREV, bool PROJ>
__global__ void __launch_bounds__(Geo<E>::NT, Geo<E>::MINB) k_cheb(const __grid_constant__ ChebArgs a) {
  using G = Geo<E>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ChebSmem<E> m = cheb_carve<E, PREV>(smem_raw, a.amax, a.maxent, a.nentmax);
  constexpr long long P = (long long)G::PLANE * E;
  const int it0 = (int)(((long long)blockIdx.x * a.n_items) / gridDim.x);
  const int it1 = (int)(((long long)(blockIdx.x + 1) * a.n_items) / gridDim.x);

  ChebT T;
  const int tid = threadIdx.x;
  T.active = tid < G::NP;
  T.py = T.active ? tid / G::NPX : 0;
  T.px = T.active ? 2 * (tid - T.py * G::NPX) : 0;
  T.t0 = T.py * E + T.px;

  if (tid == 0) {
    for (int k = 0; k < G::RING; ++k) {
      mbar_init(m.full + k, 1);
      m.issued[k] = 0;
    }
    *m.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int t = tid; t < 2 * G::PPLANE; t += G::NT) m.pin[t] = f2(0.f, 0.f);  // the halo stays zero

  int prev_f = -1;
  int gbase = 0;  // running plane count of this CTA
  for (int item = it0; item < it1; ++item) {
    const int2 fi = a.items[item];
    const int f = fi.x, i0 = fi.y;
    const FragDesc &D = a.desc[f];
    const int A = D.natom;
    const long long base = D.psi_off + (long long)i0 * P;
    const int nvalid = min(2, D.norb - i0);
    float *yout = a.yout + base;
    __syncthreads();  // the previous item no longer reads the header, tables or ring
    if (tid == 0) {
      float alpha = 1.f, beta = 0.f, shift = 0.f;
      if (a.cheb) {
        const double *bd = a.bounds + (long long)f * a.bstride;
        shift = float(bd[3]);
        alpha = float(bd[4 + 2 * a.step]);
        beta = float(bd[5 + 2 * a.step]);
      }
      typename ChebSmem<E>::Hdr &F = *m.hdr;
      F.yin = a.yin + base;
      F.yprev = PREV ? a.yprev + base : nullptr;
      F.vf = a.vf + D.pt_off;
      F.nvalid = nvalid;
      F.ksh = f2(a.kc - shift, a.kc - shift);
      F.al2 = f2(alpha, alpha);
      F.be2 = f2(beta, beta);
      for (int z = 0; z < G::RING && z < E; ++z) ring_issue<E, PREV>(m, z, gbase + z);
    }
    if (f != prev_f) {
      // the fragment's tables: x factors (splatted), supports, row starts and entries
      const int tabw = tab_width(D);
      const int r0 = a.row_beg[D.row_off];
      const int nent = a.row_beg[D.row_off + G::PLANE] - r0;
      for (int t = tid; t < A * E; t += G::NT) {
        const int k = t / E, x = t - k * E;
        const float g = a.tab[D.tab_off + (long long)k * tabw + x];
        m.gx2[t] = f2(g, g);
      }
      for (int k = tid; k < A; k += G::NT) {
        const ProjSlot S = a.slots[D.at_off + k];
        m.box[k] = make_int2(S.lo[0] >> 1, min((S.hi[0] + 1) >> 1, G::NPX));
      }
      for (int t = tid; t <= G::PLANE; t += G::NT) m.rb[t] = a.row_beg[D.row_off + t] - r0;
      for (int t = tid; t < nent; t += G::NT) m.sent[t] = a.row_ent[r0 + t];
      prev_f = f;
    }
    // the pair's D C <p|y>, zeroed accumulators
    for (int k = tid; k < A; k += G::NT) {
      const ProjSlot S = a.slots[D.at_off + k];
      const float ds = float(a.Datom[S.atom] * S.coef);
      const float *ci = a.cin + D.c_off + (long long)i0 * A + k;
      m.sk2[k] = f2(ds * ci[0], nvalid > 1 ? ds * ci[A] : 0.f);
    }
    for (int t = tid; t < kPSplit * E * A; t += G::NT) m.pacc[t] = f2(0.f, 0.f);

    // z column q[k] = plane k - 4: planes -4..-1 are zero, planes 0..3 read directly; plane 4 arrives
    // with plane 0's ring slot
    float4 q[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      q[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (T.active && k >= 4 && k < 8 && k - 4 < E) {
        const float *p = a.yin + base + (k - 4) * G::PLANE + T.t0;
        const float2 u0 = *reinterpret_cast<const float2 *>(p);
        const float2 u1 = nvalid > 1 ? *reinterpret_cast<const float2 *>(p + P) : f2(0.f, 0.f);
        q[k] = make_float4(u0.x, u1.x, u0.y, u1.y);
      }
    }
    __syncthreads();

    bool ok = true;
#pragma unroll 1
    for (int z = 0; z < E && ok; ++z) ok = cheb_plane<E, PREV, PROJ>(a, m, T, q, z, gbase, A, yout);
    __syncthreads();
    if (*m.abort) break;
    gbase += E;
    if (PROJ) {
      // the last plane's projection tasks
      {
        const int zp = E - 1, ps = zp & 1;
        const int e0 = m.rb[zp * E], n = m.rb[E * E] - e0;
        const float4 *rc = m.rec + (zp % 3) * a.maxent;
        const float4 *o4 = reinterpret_cast<const float4 *>(m.pout + ps * G::PLANE);
        const float4 *g4 = reinterpret_cast<const float4 *>(m.gx2);
        for (int t = tid; t < kPSplit * n; t += G::NT) {
          const int e = t / kPSplit, part = t - e * kPSplit;
          const int kb = m.sent[e0 + e].x;
          const int k = kb & 0xffff, y = kb >> 16;
          const int2 bx = m.box[k];
          const int len = bx.y - bx.x;
          const int xa = bx.x + (part * len) / kPSplit, xb = bx.x + ((part + 1) * len) / kPSplit;
          float2 s0 = f2(0.f, 0.f), s1 = f2(0.f, 0.f);
          for (int x2 = xa; x2 < xb; ++x2) {
            const float4 o = o4[y * G::NPX + x2];
            const float4 g = g4[k * G::NPX + x2];
            s0 = fma2(lo2(o), lo2(g), s0);
            s1 = fma2(hi2(o), hi2(g), s1);
          }
          const float w = rc[e].w;
          float2 &pa = m.pacc[(part * E + y) * A + k];
          pa = fma2(f2(w, w), add2(s0, s1), pa);
        }
      }
      __syncthreads();
      for (int t = tid; t < nvalid * A; t += G::NT) {
        const int o = t / A, k = t - o * A;
        float s = 0.f;
        for (int y = 0; y < kPSplit * E; ++y) {
          const float2 v = m.pacc[y * A + k];
          s += o == 0 ? v.x : v.y;
        }
        const ProjSlot S = a.slots[D.at_off + k];
        a.cout[D.c_off + (long long)(i0 + o) * A + k] = float(S.coef * a.dV) * s;
      }
    }
  }
  if (*m.abort) {
    // a bounded wait ran out: let the copies still in flight land (bounded) before the CTA's shared
    // memory is released, then return
    if (tid == 0)
      for (int k = 0; k < G::RING; ++k)
        if (m.issued[k] > 0) mbar_wait(m.full + k, (uint32_t)((m.issued[k] - 1) & 1));  // its last use
  }
}

template <int E>
bool cheb_fits(const dc_ctx *c) {
  return cheb_smem_bytes<E, true>(c->max_atoms, std::max(1, c->max_plane_ent), std::max(1, c->max_frag_ent)) <=
         227 * 1024;
}

template <int E, bool PREV, bool PROJ>
int run_cheb(const dc_ctx *c, const ChebArgs &a, cudaStream_t s) {
  using G = Geo<E>;
  const size_t sm = cheb_smem_bytes<E, PREV>(a.amax, a.maxent, a.nentmax);
  DC_CUDA(dc_set_smem((const void *)k_cheb<E, PREV, PROJ>, sm));
  int per_sm = 0;
  DC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cheb<E, PREV, PROJ>, G::NT, sm));
  const int grid = std::min(c->n_items2, std::max(1, per_sm) * c->sm_count);
  if (grid > 0) k_cheb<E, PREV, PROJ><<<(unsigned)grid, G::NT, sm, s>>>(a);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

template <int E>
int run_cheb_e(const dc_ctx *c, const ChebArgs &a, bool prev, bool proj, cudaStream_t s) {
  if (prev && proj) return run_cheb<E, true, true>(c, a, s);
  if (proj) return run_cheb<E, false, true>(c, a, s);
  if (prev) return run_cheb<E, true, false>(c, a, s);
  return run_cheb<E, false, false>(c, a, s);
}

}  // namespace

namespace dck {

// The extents this kernel is compiled for; 0 if the context's fragments do not qualify (cubic E^3 of one
// compiled size, zero boundary, equal spacing on the three axes, tables within shared memory).
int cheb_extent(const dc_ctx *c) {
  if (c->frag_cfg.bc != DC_BC_ZERO) return 0;
  if (c->h[0] != c->h[1] || c->h[0] != c->h[2]) return 0;
  const int E = c->max_E[0];
  for (const auto &D : c->h_desc)
    if (D.E[0] != E || D.E[1] != E || D.E[2] != E) return 0;
  switch (E) {
    case 18: return cheb_fits<18>(c) ? 18 : 0;
    case 20: return cheb_fits<20>(c) ? 20 : 0;
    case 22: return cheb_fits<22>(c) ? 22 : 0;
    case 32: return cheb_fits<32>(c) ? 32 : 0;
    default: return 0;
  }
}

int launch_cheb(dc_ctx *c, int mode, int step, const float *yin, const float *yprev, float *yout, const float *cin,
                float *cout, cudaStream_t s) {
  const int E = cheb_extent(c);
  if (!E || (mode != HSTEP_CHEB && mode != HSTEP_HPSI) || !cin || !yout) {
    dc_set_error("hpsi: the specialised FP32 kernel does not apply here");
    return DC_ERR_ARG;
  }
  ChebArgs a{};
  a.desc = c->d_desc;
  a.items = c->d_items2;
  a.slots = c->d_slots;
  a.tab = c->d_tab32;
  a.row_beg = c->d_row_beg;
  a.row_ent = c->d_row_ent;
  a.Datom = c->d_atom_D;
  a.vf = c->d_vf32;
  a.flags = c->d_flags;
  a.yin = yin;
  a.yprev = yprev;
  a.yout = yout;
  a.cin = cin;
  a.cout = cout;
  a.bounds = c->d_bounds;
  a.bstride = 4 + 2 * c->params.cheb_degree;
  a.step = step;
  a.cheb = mode == HSTEP_CHEB ? 1 : 0;
  a.maxent = std::max(1, c->max_plane_ent);
  a.amax = std::max(1, c->max_atoms);
  a.nentmax = std::max(1, c->max_frag_ent);
  a.n_items = c->n_items2;
  a.dV = (float)c->dV;
  const double fd[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
  const double h2 = c->h[0] * c->h[0];
  float kn[5];
  for (int n = 1; n < 5; ++n) kn[n] = float(-0.5 * fd[n] / h2);
  a.k1 = kn[1];
  a.k2 = kn[2];
  a.k3 = kn[3];
  a.k4 = kn[4];
  a.kc = -2.f * 3.f * (kn[3] + kn[4]);
  const bool prev = mode == HSTEP_CHEB && step > 0 && yprev != nullptr;
  const bool proj = cout != nullptr;
  switch (E) {
    case 18: return run_cheb_e<18>(c, a, prev, proj, s);
    case 20: return run_cheb_e<20>(c, a, prev, proj, s);
    case 22: return run_cheb_e<22>(c, a, prev, proj, s);
    default: return run_cheb_e<32>(c, a, prev, proj, s);
  }
}

}  // namespace dck
