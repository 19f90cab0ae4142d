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
// What bounds it: shared memory.  Per plane and warp the x and y taps, the ring reads, the nonlocal term
// and the projection tasks issue ~140 shared-memory wavefronts, and the shared-memory data pipe runs at
// ~60% of its peak over a launch (more under load peaks); the design choices below are the ones that
// cut wavefronts per point-orbital without adding resident state (the 9-deep column in registers and
// ~100 KB of shared memory per CTA leave two 256-thread CTAs per SM).
//
// Data movement: the kernel needs several planes in flight, and register prefetch holds at most one.  So
// the last lanes of the last warp (idle for E < 32: E^2 / 2 point pairs leave that warp partly empty)
// stream, for every plane z, the planes y_in(z + 4), y_prev(z) and V(z) with 1-D bulk asynchronous copies
// (cp.async.bulk, whole contiguous planes of the orbital-major layout, completion counted in bytes on an
// mbarrier) into a ring of RING slots in shared memory, RING - 1 planes ahead of their use, one copy per
// lane; the other threads read their points from the ring.  The CTAs are persistent and the ring runs on
// across a CTA's items.  Every wait on a slot is bounded: a thread that gives up sets the error flag and
// an abort word that every thread reads after the next barrier; the CTA then waits (bounded) for the
// copies still in flight and returns.
//
// Nonlocal term: the fragment's row lists (one entry per (row, projector slot) with gz gy != 0,
// host-built) and its x factors (one float2 per point pair) are staged in shared memory once per
// fragment; a point adds (u gz gy) gx[x] over its row's entries, u = D C <p|y> of the pair.  The
// projections of the output, needed by the next Chebyshev step, are formed one plane behind by one task
// per entry: gz gy sum_x gx[x] out(x, y) into a dense [row][slot] accumulator (one writer per element
// and plane), rows summed at the end of the item.  One barrier per plane.
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
  const int *row_split;   // per row: left-only entries | (left-only + both) << 16
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
  int amax, nentmax;      // max projector slots and row-list entries of one fragment (shared-memory carve)
  int n_items;            // work items (the CTAs are persistent: CTA b takes a contiguous block of items)
  int ipc;                // most items of one CTA (item-table size)
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

// Projection tasks.  Earlier forms, measured on the 64-atom cell (Si, 22^3 fragments): one task per record
// on thread t (the first warps carry all of them and the others wait at the plane's barrier), 270 us per
// launch; the same tasks spread one lane per warp per round, 295 us (every warp then runs the full task
// loop); two x-halves with a second accumulator plane, 394 us (its shared memory cost the second CTA per
// SM).  The halves combined by a shuffle on adjacent lanes (below) need no second plane.

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
  // Row pitches of the output planes (float4 = point pair x orbital pair) and of the x factors (float2 =
  // point pair), padded so that the projection tasks' loads (one record per lane, rows and supports
  // scattered) meet fewer bank conflicts: on the Si row lists the padding takes ~11% off their shared
  // memory wavefronts.
  static constexpr int OP = NPX + 1;
  static constexpr int GP = NPX + 2;
  static constexpr bool HALF_ROWS = E <= 22;  // point walks only its half-row's entries
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

// Per-item constants of one CTA's work items, built once at kernel start (32 bytes each).
struct ItemInfo {
  long long base;  // element offset of the pair's first orbital in the orbital blocks
  int vf;          // offset of the fragment's points (V); equal offsets = the same fragment
  int coff;        // offset of the pair's projections (orbital i; i + 1 at + A)
  int nva;         // nvalid (1 or 2) | A << 2
  float ksh;       // kc - shift
  float al, be;    // alpha, beta of this Chebyshev step
};

// Shared-memory carve (byte offsets; the same function sizes the launch on the host).
template <int E, bool PREV>
struct ChebLayout {
  size_t ring, full, itab, pin, pout, gxp, pacc, sk2, dsk, cdv, sent, box, rb, rsp, end;
  static __host__ __device__ size_t up(size_t o, size_t a) { return (o + a - 1) / a * a; }
  __host__ __device__ ChebLayout(int A, int nent, int ipc) {
    using G = Geo<E>;
    size_t o = 0;
    ring = o;  // 16-byte aligned slots (E^2 floats are multiples of 16 bytes for even E)
    o += (size_t)G::RING * (PREV ? 5 : 3) * G::PLANE * sizeof(float);
    full = o = up(o, 16);
    o += G::RING * sizeof(uint64_t) + 16 + G::RING * sizeof(int);  // barriers, abort word, issue counts
    itab = o = up(o, 16);
    o += (size_t)ipc * sizeof(ItemInfo);
    pin = o = up(o, 16);
    o += 2 * (size_t)G::PPLANE * sizeof(float2);
    pout = o;
    o += 2 * (size_t)E * G::OP * sizeof(float4);
    gxp = o;
    o += (size_t)A * G::GP * sizeof(float2);
    pacc = o;
    o += (size_t)E * A * sizeof(float2);
    sk2 = o;
    o += 2 * (size_t)A * sizeof(float2);
    dsk = o;
    o += (size_t)A * sizeof(float);
    cdv = o;
    o += (size_t)A * sizeof(float);
    sent = o = up(o, 8);
    o += (size_t)nent * sizeof(int2);
    box = o;
    o += (size_t)A * sizeof(int2);
    rb = o;
    o += (size_t)(G::PLANE + 1) * sizeof(int);
    rsp = o;
    o += (size_t)G::PLANE * sizeof(int);
    end = up(o, 16);
  }
};

template <int E>
struct ChebSmem {
  float *ring;          // [RING][NSUB][E*E] y_in(z + 4) (2 orbitals), [y_prev(z) (2 orbitals)], V(z)
  uint64_t *full;       // [RING] slot barriers
  volatile int *abort;  // set by a thread whose bounded wait ran out
  int *issued;          // [RING] uses of each slot so far (producer thread only)
  ItemInfo *itab;       // [ipc] the CTA's items
  float2 *pin;          // [2][PPLANE]   haloed planes of y_in
  float2 *pout;         // [2][E][OP]    output planes (float4 per point pair; projections)
  float2 *gxp;          // [A][GP]       x factors of each point pair (g(2 x2), g(2 x2 + 1))
  float2 *pacc;         // [E][A]        projection accumulators
  float2 *sk2;          // [2][A]        D C <p|y> of the pair (two items: current, next)
  float *dsk;           // [A]           D_atom coef per slot
  float *cdv;           // [A]           coef dV per slot
  int2 *sent;           // [nent]        the fragment's row-list entries
  int2 *box;            // [A]           even-aligned x support
  int *rb;              // [E*E + 1]     row starts (relative to the fragment's first entry)
  int *rsp;             // [E*E]         row splits: left-only entries | (left-only + both) << 16
};

// Planes per ring slot: y_in of the pair, y_prev of the pair (with PREV), V.
template <bool PREV>
__host__ __device__ constexpr int ring_sub() {
  return PREV ? 5 : 3;
}

template <int E, bool PREV>
__device__ __forceinline__ ChebSmem<E> cheb_carve(unsigned char *raw, int A, int nent, int ipc) {
  const ChebLayout<E, PREV> L(A, nent, ipc);
  ChebSmem<E> m;
  m.ring = reinterpret_cast<float *>(raw + L.ring);
  m.full = reinterpret_cast<uint64_t *>(raw + L.full);
  m.abort = reinterpret_cast<volatile int *>(m.full + Geo<E>::RING);
  m.issued = reinterpret_cast<int *>(raw + L.full + Geo<E>::RING * sizeof(uint64_t) + 16);
  m.itab = reinterpret_cast<ItemInfo *>(raw + L.itab);
  m.pin = reinterpret_cast<float2 *>(raw + L.pin);
  m.pout = reinterpret_cast<float2 *>(raw + L.pout);
  m.gxp = reinterpret_cast<float2 *>(raw + L.gxp);
  m.pacc = reinterpret_cast<float2 *>(raw + L.pacc);
  m.sk2 = reinterpret_cast<float2 *>(raw + L.sk2);
  m.dsk = reinterpret_cast<float *>(raw + L.dsk);
  m.cdv = reinterpret_cast<float *>(raw + L.cdv);
  m.sent = reinterpret_cast<int2 *>(raw + L.sent);
  m.box = reinterpret_cast<int2 *>(raw + L.box);
  m.rb = reinterpret_cast<int *>(raw + L.rb);
  m.rsp = reinterpret_cast<int *>(raw + L.rsp);
  return m;
}

// Per-thread state that the plane function reads.
struct ChebT {
  int px, py;      // owned points (px, py), (px + 1, py)
  bool active;     // owns a point pair
  int t0;          // py E + px
};

// The ring's producer lanes: the last COPIES lanes of the last warp.  For E < 32 they own no point pair
// (E^2 / 2 point pairs leave the last warp partly idle), so issuing the copies, which holds the issuing
// warp for ~100+ cycles per copy, does not delay the warps whose stencil and projection work set the
// plane's length.
constexpr int kCopies = 5;

// Issue the bulk copies of the CTA's running plane g (item g / E, plane z = g % E): y_in(z + 4), y_prev(z)
// and V(z) into ring slot g % RING.  Run by the kCopies producer lanes together; lane NT - 1 counts the
// bytes on the slot's barrier first, then each lane issues at most one copy.
template <int E, bool PREV>
__device__ __forceinline__ void ring_issue(const ChebArgs &a, const ChebSmem<E> &m, int g) {
  using G = Geo<E>;
  constexpr uint32_t PB = G::PLANE * sizeof(float);
  constexpr long long P = (long long)G::PLANE * E;
  const int lg = g / E, z = g - lg * E;
  const ItemInfo &I = m.itab[lg];
  const int nvalid = I.nva & 3;
  const int s = g % G::RING;
  float *slot = m.ring + (size_t)s * ring_sub<PREV>() * G::PLANE;
  uint64_t *bar = m.full + s;
  const bool has_y = z + 4 < E;
  const int j = G::NT - 1 - (int)threadIdx.x;  // 0 .. kCopies - 1
  if (j == 0) {
    uint32_t bytes = PB;  // V
    if (has_y) bytes += nvalid * PB;
    if (PREV) bytes += nvalid * PB;
    // the slot was last read through ordinary shared loads (ordered before this by the CTA barrier); the
    // bulk copies write it through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    m.issued[s] += 1;
    mbar_expect_tx(bar, bytes);
  }
  __syncwarp(((1u << kCopies) - 1) << (32 - kCopies));
  for (int cp = j; cp < 5; cp += kCopies) {
    if (cp == 0) {
      bulk_g2s(slot + (ring_sub<PREV>() - 1) * G::PLANE, a.vf + I.vf + (long long)z * G::PLANE, PB, bar);
    } else if (cp <= 2) {
      if (has_y && cp <= nvalid)
        bulk_g2s(slot + (cp - 1) * G::PLANE, a.yin + I.base + (cp - 1) * P + (long long)(z + 4) * G::PLANE, PB, bar);
    } else if (PREV) {
      if (cp - 2 <= nvalid)
        bulk_g2s(slot + (cp - 1) * G::PLANE, a.yprev + I.base + (cp - 3) * P + (long long)z * G::PLANE, PB, bar);
    }
  }
}

// Projection tasks of output plane zp: one per record, gz gy sum_x gx[x] out(x, y) into the dense [row][slot]
// accumulator (one writer per element and plane).
template <int E>
__device__ __forceinline__ void proj_plane(const ChebSmem<E> &m, int zp, int A) {
  using G = Geo<E>;
  const int e0 = m.rb[zp * E], n = m.rb[(zp + 1) * E] - e0;
  const float4 *o4 = reinterpret_cast<const float4 *>(m.pout) + (zp & 1) * E * G::OP;
  for (int t = threadIdx.x; t < n; t += G::NT) {
    const int kb = m.sent[e0 + t].x;
    const int k = kb & 0xffff, y = kb >> 16;
    const int2 bx = m.box[k];
    const float4 *orow = o4 + y * G::OP;
    const float2 *grow = m.gxp + k * G::GP;
    float2 s0 = f2(0.f, 0.f), s1 = f2(0.f, 0.f);
    for (int x2 = bx.x; x2 < bx.y; ++x2) {
      const float4 o = orow[x2];
      const float2 g = grow[x2];
      s0 = fma2(lo2(o), f2(g.x, g.x), s0);
      s1 = fma2(hi2(o), f2(g.y, g.y), s1);
    }
    const float w = __int_as_float(m.sent[e0 + t].y);
    float2 &pa = m.pacc[y * A + k];
    pa = fma2(f2(w, w), add2(s0, s1), pa);
  }
}

// Plane z of the current item (CTA running plane gz = gbase + z).  The column registers q[k] hold plane
// z - 4 + k (q[8], plane z + 4, arrives from the ring at this plane) and are moved down by one plane at
// the end.  A loop over z with these moves runs faster than a body unrolled nine times that renames the
// registers instead: the unrolled kernel's instruction footprint stalled the warps on instruction fetch.
// Returns false when the CTA aborts.
template <int E, bool PREV, bool PROJ, bool NL>
__device__ __forceinline__ bool cheb_plane(const ChebArgs &a, const ChebSmem<E> &m, const ChebT &T, float4 (&q)[9],
                                           int z, int gbase, int ntot, const ItemInfo &I, const float2 *sk2,
                                           float *yout) {
  using G = Geo<E>;
  const int A = I.nva >> 2, nvalid = I.nva & 3;
  const int slot = z & 1;
  float2 *P0 = m.pin + slot * G::PPLANE;
  const int c = (T.py + 4) * G::PITCH + T.px + 4;
  if (T.active) *reinterpret_cast<float4 *>(P0 + c) = q[4];
  // the item's projection accumulators start at zero (read from plane 1's tasks on)
  if (PROJ && z == 0)
    for (int t = threadIdx.x; t < E * A; t += G::NT) m.pacc[t] = f2(0.f, 0.f);
  // this plane's ring slot (y_in(z + 4) completes the column; y_prev(z) and V(z) are read below); the
  // wait sits before the barrier so that its latency overlaps the other warps' work
  const int gz = gbase + z;
  const float *rs = m.ring + (size_t)(gz % G::RING) * ring_sub<PREV>() * G::PLANE + T.t0;
  __syncthreads();
  if (*m.abort) return false;
  // refill the slot that plane gz - 1 has finished with, for running plane gz - 1 + RING
  if ((int)threadIdx.x >= G::NT - kCopies && gz >= 1 && gz - 1 + G::RING < ntot)
    ring_issue<E, PREV>(a, m, gz - 1 + G::RING);
  // projections of the previous output plane
  if (PROJ && z > 0) proj_plane<E>(m, z - 1, A);
  if (!T.active) return true;
  if (!mbar_wait(m.full + gz % G::RING, (uint32_t)((gz / G::RING) & 1))) {
    atomicOr(a.flags, DC_FLAG_TIMEOUT);
    *m.abort = 1;
    return true;
  }
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
    const float4 ZU = q[4 + N];                                                                            \
    const float4 ZD = q[4 - N];                                                                            \
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
    const float2 ksh = f2(I.ksh, I.ksh);
    const float2 vr = *reinterpret_cast<const float2 *>(rs + (ring_sub<PREV>() - 1) * G::PLANE);
    h0 = fma2(ksh, c0, fma2(f2(vr.x, vr.x), c0, h0));
    h1 = fma2(ksh, c1, fma2(f2(vr.y, vr.y), c1, h1));
  }
  // nonlocal term over the row's records (NL = false: the local part of H only)
  if (NL) {
    const int rz = z * E + T.py;
    // entries that can reach this point's half of the row: [left-only | both] or [both | right-only].
    // Measured per extent: 22^3 fragments 1.650 -> 1.639 ms per Si512 launch with the halves; on 32^3
    // (a warp spans both halves of two rows, so only the divergence grows) the water cell's stencil
    // stage 108.0 -> 109.5 ms, so there the whole row is walked.
    const int r0 = m.rb[rz];
    int eb, ee;
    if (G::HALF_ROWS) {
      const int sp = m.rsp[rz];
      const bool left = (T.px >> 1) < (G::NPX + 1) / 2;
      eb = left ? r0 : r0 + (sp & 0xffff);
      ee = left ? r0 + (sp >> 16) : m.rb[rz + 1];
    } else {
      eb = r0;
      ee = m.rb[rz + 1];
    }
    const float2 *gp = m.gxp + (T.px >> 1);
    int e = eb;
    for (; e + 1 < ee; e += 2) {
      const int2 na = m.sent[e], nb = m.sent[e + 1];
      const int ka = na.x & 0xffff, kb = nb.x & 0xffff;
      const float wa = __int_as_float(na.y), wb = __int_as_float(nb.y);
      const float2 ua = sk2[ka], ub = sk2[kb];
      const float2 ga = gp[ka * G::GP], gb = gp[kb * G::GP];
      const float2 ra = mul2(ua, f2(wa, wa)), rb = mul2(ub, f2(wb, wb));
      h0 = fma2(ra, f2(ga.x, ga.x), h0);
      h1 = fma2(ra, f2(ga.y, ga.y), h1);
      h0 = fma2(rb, f2(gb.x, gb.x), h0);
      h1 = fma2(rb, f2(gb.y, gb.y), h1);
    }
    if (e < ee) {
      const int2 na = m.sent[e];
      const int ka = na.x & 0xffff;
      const float wa = __int_as_float(na.y);
      const float2 ra = mul2(sk2[ka], f2(wa, wa));
      const float2 ga = gp[ka * G::GP];
      h0 = fma2(ra, f2(ga.x, ga.x), h0);
      h1 = fma2(ra, f2(ga.y, ga.y), h1);
    }
  }
  float2 o0, o1;
  const float2 al2 = f2(I.al, I.al);
  if (PREV) {
    const float2 be2 = f2(I.be, I.be);
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
    reinterpret_cast<float4 *>(m.pout)[(slot * E + T.py) * G::OP + (T.px >> 1)] =
        make_float4(o0.x, nvalid > 1 ? o0.y : 0.f, o1.x, nvalid > 1 ? o1.y : 0.f);
#pragma unroll
  for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
  return true;
}

// The column of a new item: planes -4..-1 are zero, planes 0..3 read directly (plane 4 arrives with plane
// 0's ring slot).
template <int E>
__device__ __forceinline__ void column_start(const ChebArgs &a, const ChebT &T, const ItemInfo &I, float4 (&q)[9]) {
  using G = Geo<E>;
  constexpr long long P = (long long)G::PLANE * E;
  const int nvalid = I.nva & 3;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    q[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (T.active && k >= 4 && k < 8 && k - 4 < E) {
      const float *p = a.yin + I.base + (k - 4) * G::PLANE + T.t0;
      const float2 u0 = *reinterpret_cast<const float2 *>(p);
      const float2 u1 = nvalid > 1 ? *reinterpret_cast<const float2 *>(p + P) : f2(0.f, 0.f);
      q[k] = make_float4(u0.x, u1.x, u0.y, u1.y);
    }
  }
}

// Global -> shared copy of n int2 with four loads in flight per thread.
template <int NT>
__device__ __forceinline__ void copy_int2(int2 *dst, const int2 *src, int n) {
  for (int t = threadIdx.x; t < n; t += 4 * NT) {
    int2 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (t + j * NT < n) v[j] = src[t + j * NT];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (t + j * NT < n) dst[t + j * NT] = v[j];
  }
}

// Persistent CTAs: CTA b runs the contiguous block of work items [b n / G, (b + 1) n / G) (all items cost
// the same: one orbital pair of an E^3 fragment).  Item constants for the whole block are built once.
// Consecutive items are mostly the same fragment, whose tables (x factors, supports, row lists, D coef,
// coef dV) stay in shared memory.  The ring runs on across items (the next item's first planes are in
// flight while the current item ends), and the next item's first column planes and, for the same
// fragment, its D C <p|y> are fetched during the current item's tail.
template <int E, bool PREV, bool PROJ, bool NL>
__global__ void __launch_bounds__(Geo<E>::NT, Geo<E>::MINB) k_cheb(const __grid_constant__ ChebArgs a) {
  using G = Geo<E>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ChebSmem<E> m = cheb_carve<E, PREV>(smem_raw, a.amax, a.nentmax, a.ipc);
  constexpr long long P = (long long)G::PLANE * E;
  const int it0 = (int)(((long long)blockIdx.x * a.n_items) / gridDim.x);
  const int it1 = (int)(((long long)(blockIdx.x + 1) * a.n_items) / gridDim.x);
  const int nit = it1 - it0;  // <= a.ipc
  const int ntot = nit * E;   // running planes of this CTA

  ChebT T;
  const int tid = threadIdx.x;
  T.active = tid < G::NP;
  T.py = T.active ? tid / G::NPX : 0;
  T.px = T.active ? 2 * (tid - T.py * G::NPX) : 0;
  T.t0 = T.py * E + T.px;

  if (tid == G::NT - 1) {
    for (int k = 0; k < G::RING; ++k) {
      mbar_init(m.full + k, 1);
      m.issued[k] = 0;
    }
    *m.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int t = tid; t < 2 * G::PPLANE; t += G::NT) m.pin[t] = f2(0.f, 0.f);  // the halo stays zero
  for (int t = tid; t < nit; t += G::NT) {
    const int2 fi = a.items[it0 + t];
    const FragDesc &D = a.desc[fi.x];
    ItemInfo I;
    I.base = D.psi_off + (long long)fi.y * P;
    I.vf = (int)D.pt_off;
    I.coff = (int)(D.c_off + (long long)fi.y * D.natom);
    I.nva = min(2, D.norb - fi.y) | (D.natom << 2);
    float alpha = 1.f, beta = 0.f, shift = 0.f;
    if (a.cheb) {
      const double *bd = a.bounds + (long long)fi.x * a.bstride;
      shift = float(bd[3]);
      alpha = float(bd[4 + 2 * a.step]);
      beta = float(bd[5 + 2 * a.step]);
    }
    I.ksh = a.kc - shift;
    I.al = alpha;
    I.be = beta;
    m.itab[t] = I;
  }
  __syncthreads();  // item table, barriers
  if (tid >= G::NT - kCopies)
    for (int g = 0; g < G::RING && g < ntot; ++g) {
      ring_issue<E, PREV>(a, m, g);
      __syncwarp(((1u << kCopies) - 1) << (32 - kCopies));
    }

  float4 q[9];
  if (nit > 0) column_start<E>(a, T, m.itab[0], q);
  int cur_vf = -1;
  for (int lj = 0; lj < nit; ++lj) {
    const ItemInfo &I = m.itab[lj];
    const int A = I.nva >> 2, nvalid = I.nva & 3;
    float2 *sk2 = m.sk2 + (lj & 1) * a.amax;
    if ((NL || PROJ) && I.vf != cur_vf) {
      // a new fragment: its tables, and the pair's D C <p|y> (the tables' previous readers finished
      // before the barrier that ended the last item)
      const int f = a.items[it0 + lj].x;
      const FragDesc &D = a.desc[f];
      const int tabw = tab_width(D);
      const int r0 = a.row_beg[D.row_off];
      const int nent = a.row_beg[D.row_off + G::PLANE] - r0;
      for (int t = tid; t < A * G::NPX; t += G::NT) {
        const int k = t / G::NPX, x2 = t - k * G::NPX;
        const float *g = a.tab + D.tab_off + (long long)k * tabw + 2 * x2;
        m.gxp[k * G::GP + x2] = f2(g[0], g[1]);
      }
      for (int k = tid; k < A; k += G::NT) {
        const ProjSlot S = a.slots[D.at_off + k];
        m.box[k] = make_int2(S.lo[0] >> 1, min((S.hi[0] + 1) >> 1, G::NPX));
        const float ds = float(a.Datom[S.atom] * S.coef);
        m.dsk[k] = ds;
        m.cdv[k] = float(S.coef * a.dV);
        const float *ci = a.cin + I.coff + k;
        sk2[k] = f2(ds * ci[0], nvalid > 1 ? ds * ci[A] : 0.f);
      }
      for (int t = tid; t <= G::PLANE; t += G::NT) m.rb[t] = a.row_beg[D.row_off + t] - r0;
      for (int t = tid; t < G::PLANE; t += G::NT) m.rsp[t] = a.row_split[D.row_off + t];
      copy_int2<G::NT>(m.sent, a.row_ent + r0, nent);
      cur_vf = I.vf;
      __syncthreads();
    }
    float *yout = a.yout + I.base;
    bool ok = true;
#pragma unroll 1
    for (int z = 0; z < E && ok; ++z) ok = cheb_plane<E, PREV, PROJ, NL>(a, m, T, q, z, lj * E, ntot, I, sk2, yout);
    __syncthreads();
    if (*m.abort) break;
    // the next item: its first column planes (the loads are in flight during this item's tail) and, for
    // the same fragment, its D C <p|y>
    if (lj + 1 < nit) {
      const ItemInfo &In = m.itab[lj + 1];
      column_start<E>(a, T, In, q);
      if (NL && In.vf == I.vf && tid >= G::NT - 32) {
        float2 *skn = m.sk2 + ((lj + 1) & 1) * a.amax;
        const int nvn = In.nva & 3;
        for (int k = tid - (G::NT - 32); k < A; k += 32) {
          const float ds = m.dsk[k];
          const float *ci = a.cin + In.coff + k;
          skn[k] = f2(ds * ci[0], nvn > 1 ? ds * ci[A] : 0.f);
        }
      }
    }
    if (PROJ) {
      proj_plane<E>(m, E - 1, A);  // the last plane's projection tasks
      __syncthreads();
      for (int t = tid; t < nvalid * A; t += G::NT) {
        const int o = t / A, k = t - o * A;
        float s = 0.f;
#pragma unroll
        for (int y = 0; y < E; ++y) {
          const float2 v = m.pacc[y * A + k];
          s += o == 0 ? v.x : v.y;
        }
        a.cout[I.coff + (long long)o * A + k] = m.cdv[k] * s;
      }
    }
    __syncthreads();  // pacc, sk2 and the tables are free for the next item
  }
  if (*m.abort) {
    // a bounded wait ran out: let the copies still in flight land (bounded) before the CTA's shared
    // memory is released, then return
    if (tid == G::NT - 1)
      for (int k = 0; k < G::RING; ++k)
        if (m.issued[k] > 0) mbar_wait(m.full + k, (uint32_t)((m.issued[k] - 1) & 1));  // its last use
  }
}

// Work items per CTA of the persistent grid (the largest block of [b n / G, (b + 1) n / G)).
inline int cheb_ipc(int n_items, int grid) { return grid > 0 ? (n_items + grid - 1) / grid : 0; }

template <int E>
bool cheb_fits(const dc_ctx *c) {
  // the worst case: one CTA per SM, so the most items per CTA
  const ChebLayout<E, true> L(std::max(1, c->max_atoms), std::max(1, c->max_frag_ent),
                              cheb_ipc(c->n_items2, c->sm_count));
  return L.end <= 227 * 1024;
}

template <int E, bool PREV, bool PROJ, bool NL>
int run_cheb(const dc_ctx *c, ChebArgs a, cudaStream_t s) {
  using G = Geo<E>;
  const int n = c->n_items2;
  if (n <= 0) return DC_OK;
  // the largest CTAs-per-SM count (up to the launch bound) whose shared memory, item table included,
  // still allows it
  int grid = 0;
  size_t sm = 0;
  for (int per = G::MINB; per >= 1 && !grid; --per) {
    const int g = std::min(n, per * c->sm_count);
    const int ipc = cheb_ipc(n, g);
    sm = ChebLayout<E, PREV>(a.amax, a.nentmax, ipc).end;
    DC_CUDA(dc_set_smem((const void *)k_cheb<E, PREV, PROJ, NL>, sm));
    int occ = 0;
    DC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cheb<E, PREV, PROJ, NL>, G::NT, sm));
    if (occ >= per) {
      grid = g;
      a.ipc = ipc;
    }
  }
  if (!grid) {
    dc_set_error("hpsi: the specialised FP32 kernel's shared memory does not fit");
    return DC_ERR_ARG;
  }
  k_cheb<E, PREV, PROJ, NL><<<(unsigned)grid, G::NT, sm, s>>>(a);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

template <int E>
int run_cheb_e(const dc_ctx *c, const ChebArgs &a, bool prev, bool proj, bool nl, cudaStream_t s) {
  if (!nl) return run_cheb<E, false, false, false>(c, a, s);  // the local part of H (no y_prev, no projections)
  if (prev && proj) return run_cheb<E, true, true, true>(c, a, s);
  if (proj) return run_cheb<E, false, true, true>(c, a, s);
  if (prev) return run_cheb<E, true, false, true>(c, a, s);
  return run_cheb<E, false, false, true>(c, a, s);
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
  if (!E || (mode != HSTEP_CHEB && mode != HSTEP_HPSI && mode != HSTEP_HLOC) || !cin || !yout) {
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
  a.row_split = c->d_row_split;
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
  const bool nl = mode != HSTEP_HLOC;
  if (!nl && (prev || proj)) {
    dc_set_error("hpsi: the local part of H is applied without y_prev or output projections");
    return DC_ERR_ARG;
  }
  switch (E) {
    case 18: return run_cheb_e<18>(c, a, prev, proj, nl, s);
    case 20: return run_cheb_e<20>(c, a, prev, proj, nl, s);
    case 22: return run_cheb_e<22>(c, a, prev, proj, nl, s);
    default: return run_cheb_e<32>(c, a, prev, proj, nl, s);
  }
}

}  // namespace dck
