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
// access is one 8-byte load or store, without predicates).  The potential is read pre-splatted,
// (V, V) per point, so no lane copies are needed to multiply an orbital pair.
//
// Nonlocal term: the fragment's row lists (one entry per (row, projector slot) with gz gy != 0,
// host-built) are staged in shared memory once per CTA; each plane turns its entries into records
// (u_i gz gy, u_i+1 gz gy, the slot's x-factor offset, gz gy), u = D C <p|y>, in a three-slot ring;
// a point adds u gx[x] over its row's records.  The projections of the output, needed by the next
// Chebyshev step, are formed one plane behind by one task per record: gz gy sum_x gx[x] out(x, y)
// into a dense [row][slot] accumulator (one writer per element and plane), rows summed at the end.
// One barrier per plane.
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
  const float2 *vf2;      // (V, V) per fragment point
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

template <int E>
struct Geo {
  static constexpr int NPX = E / 2;                  // point pairs per row
  static constexpr int NP = NPX * E;                 // point pairs per plane
  static constexpr int NT = (NP + 31) / 32 * 32;     // threads per CTA
  static constexpr int PITCH = E + 16;               // haloed row pitch (float2), conflict-free
  static constexpr int HROWS = E + 8;
  static constexpr int PPLANE = PITCH * HROWS;       // one haloed plane (float2)
  static constexpr int PLANE = E * E;
  static constexpr int MINB = NT <= 256 ? 2 : 1;
};

// Shared-memory carve (float2 units first, 16-byte aligned blocks).
template <int E>
struct ChebSmem {
  float2 *pin;   // [2][PPLANE]   haloed planes of y_in
  float2 *pout;  // [2][E*E]      output planes (projections)
  float2 *gx2;   // [A][E]        x factors, splatted (g, g)
  float2 *pacc;  // [E][A]        projection accumulators
  float2 *sk2;   // [A]           D C <p|y> of the pair
  float4 *rec;   // [3][maxent]   per-plane records (a plane's records are read by its own stencil and, one
                 //               plane later, by its projection tasks, so three slots keep the writer of
                 //               plane z + 1 clear of both)
  int2 *sent;    // [nent]        the fragment's row-list entries
  int2 *box;     // [A]           even-aligned x support
  int *rb;       // [E*E + 1]     row starts (relative to the fragment's first entry)
};

template <int E>
__host__ __device__ inline size_t cheb_smem_bytes(int A, int maxent, int nent) {
  using G = Geo<E>;
  size_t n2 = 2 * (size_t)G::PPLANE + 2 * (size_t)G::PLANE + (size_t)A * E + (size_t)E * A + A;
  size_t b = (n2 * sizeof(float2) + 15) & ~(size_t)15;
  b += 3 * (size_t)maxent * sizeof(float4);
  b += (size_t)nent * sizeof(int2) + (size_t)A * sizeof(int2) + (size_t)(G::PLANE + 1) * sizeof(int);
  return b + 64;
}

template <int E>
__device__ __forceinline__ ChebSmem<E> cheb_carve(unsigned char *raw, int A, int maxent, int nent) {
  using G = Geo<E>;
  ChebSmem<E> m;
  m.pin = reinterpret_cast<float2 *>(raw);
  m.pout = m.pin + 2 * G::PPLANE;
  m.gx2 = m.pout + 2 * G::PLANE;
  m.pacc = m.gx2 + A * E;
  m.sk2 = m.pacc + E * A;
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
  float2 ksh;      // centre coefficient minus the filter shift, splatted
  float2 al2, be2; // alpha, beta splatted
};

// Plane z.  ZI = z mod 9 names the column registers: q[(ZI + k) % 9] holds plane z - 4 + k.
template <int E, bool PREV, bool PROJ, int ZI>
__device__ __forceinline__ void cheb_plane(const ChebArgs &a, const ChebSmem<E> &m, const ChebT &T, float4 (&q)[9],
                                           float4 &vv, float4 &pv, int z, int A, int nvalid, const float *yin,
                                           const float *yprev, float *yout, const float2 *vf2) {
  using G = Geo<E>;
  const int slot = z & 1;
  float2 *P0 = m.pin + slot * G::PPLANE;
  const int c = (T.py + 4) * G::PITCH + T.px + 4;
  if (T.active) *reinterpret_cast<float4 *>(P0 + c) = q[(ZI + 4) % 9];
  // this plane's records from its row-list entries
  {
    const int e0 = m.rb[z * E], n = m.rb[(z + 1) * E] - e0;
    float4 *rc = m.rec + (ZI % 3) * a.maxent;
    for (int t = threadIdx.x; t < n; t += G::NT) {
      const int2 en = m.sent[e0 + t];
      const float w = __int_as_float(en.y);
      const int k = en.x & 0xffff;
      const float2 u = m.sk2[k];
      rc[t] = make_float4(u.x * w, u.y * w, __int_as_float(k * G::NPX), w);
    }
  }
  __syncthreads();
  // projections of the previous output plane
  if (PROJ && z > 0) {
    const int zp = z - 1, ps = zp & 1;
    const int e0 = m.rb[zp * E], n = m.rb[z * E] - e0;
    const float4 *rc = m.rec + ((ZI + 2) % 3) * a.maxent;
    const float4 *o4 = reinterpret_cast<const float4 *>(m.pout + ps * G::PLANE);
    const float4 *g4 = reinterpret_cast<const float4 *>(m.gx2);
    for (int t = threadIdx.x; t < n; t += G::NT) {
      const int kb = m.sent[e0 + t].x;
      const int k = kb & 0xffff, y = kb >> 16;
      const int2 bx = m.box[k];
      const float4 *orow = o4 + y * G::NPX;
      const float4 *grow = g4 + k * G::NPX;
      float2 s0 = f2(0.f, 0.f), s1 = f2(0.f, 0.f);
      for (int x2 = bx.x; x2 < bx.y; ++x2) {
        const float4 o = orow[x2];
        const float4 g = grow[x2];
        s0 = fma2(lo2(o), lo2(g), s0);
        s1 = fma2(hi2(o), hi2(g), s1);
      }
      const float w = rc[t].w;
      float2 &pa = m.pacc[y * A + k];
      pa = fma2(f2(w, w), add2(s0, s1), pa);
    }
  }
  if (!T.active) return;
  const float4 V = vv;
  const float4 Y1 = pv;
  // Laplacian in difference form: taps 1, 2 as (y+n - y) + (y-n - y), taps 3, 4 as y+n + y-n with the
  // centre term added once; tap by tap, so each tap's loads die before the next are needed.
  // x neighbours of point 0 (x = px) and point 1 (px + 1): X0 = (px-4, px-3), X1 = (px-2, px-1),
  // centre (px, px+1), X3 = (px+2, px+3), X4 = (px+4, px+5), each float2 = the orbital pair
  const float2 *co = P0 + c;
  const float4 C = q[(ZI + 4) % 9];
  const float2 c0 = lo2(C), c1 = hi2(C);
  const float4 X1 = *reinterpret_cast<const float4 *>(co - 2);
  const float4 X3 = *reinterpret_cast<const float4 *>(co + 2);
  // H y without alpha: (kc - shift + V) y, the taps, then the nonlocal term
  float2 h0 = fma2(T.ksh, c0, mul2(lo2(V), c0));
  float2 h1 = fma2(T.ksh, c1, mul2(hi2(V), c1));
  float2 t0, t1;
#define DC_YZ_TAPS(N, DIFF)                                                                                  \
  {                                                                                                        \
    const float4 U = *reinterpret_cast<const float4 *>(co + N * G::PITCH);                                 \
    const float4 Dn = *reinterpret_cast<const float4 *>(co - N * G::PITCH);                                \
    const float4 ZU = q[(ZI + 4 + N) % 9];                                                                 \
    const float4 ZD = q[(ZI + 4 - N) % 9];                                                                 \
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
  h0 = fma2(f2(a.k1, a.k1), t0, h0);
  h1 = fma2(f2(a.k1, a.k1), t1, h1);
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
  // nonlocal term over the row's records
  {
    const int rz = z * E + T.py;
    const int eb = m.rb[rz] - m.rb[z * E], ee = m.rb[rz + 1] - m.rb[z * E];
    const float4 *rc = m.rec + (ZI % 3) * a.maxent;
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
  if (PREV) {
    o0 = fma2(T.al2, h0, mul2(T.be2, lo2(Y1)));
    o1 = fma2(T.al2, h1, mul2(T.be2, hi2(Y1)));
  } else {
    o0 = mul2(T.al2, h0);
    o1 = mul2(T.al2, h1);
  }
  {
    float *po = yout + z * G::PLANE + T.t0;
    *reinterpret_cast<float2 *>(po) = f2(o0.x, o1.x);
    if (nvalid > 1) *reinterpret_cast<float2 *>(po + E * G::PLANE) = f2(o0.y, o1.y);
  }
  if (PROJ)
    *reinterpret_cast<float4 *>(m.pout + slot * G::PLANE + T.t0) =
        make_float4(o0.x, nvalid > 1 ? o0.y : 0.f, o1.x, nvalid > 1 ? o1.y : 0.f);
  // loads for later planes, issued once this plane's stencil no longer needs registers: y_in of plane
  // z + 5 into the column slot of plane z - 4, V and y_prev of plane z + 1
  {
    const int zn = z + 5;
    float4 nxt = make_float4(0.f, 0.f, 0.f, 0.f);
    if (zn < E) {
      const float *p = yin + zn * G::PLANE + T.t0;
      const float2 u0 = *reinterpret_cast<const float2 *>(p);
      const float2 u1 = nvalid > 1 ? *reinterpret_cast<const float2 *>(p + E * G::PLANE) : f2(0.f, 0.f);
      nxt = make_float4(u0.x, u1.x, u0.y, u1.y);
    }
    q[ZI % 9] = nxt;
    if (z + 1 < E) {
      const int t1 = (z + 1) * G::PLANE + T.t0;
      vv = *reinterpret_cast<const float4 *>(vf2 + t1);
      if (PREV) {
        const float2 u0 = *reinterpret_cast<const float2 *>(yprev + t1);
        const float2 u1 = nvalid > 1 ? *reinterpret_cast<const float2 *>(yprev + t1 + E * G::PLANE) : f2(0.f, 0.f);
        pv = make_float4(u0.x, u1.x, u0.y, u1.y);
      }
    }
  }
}

template <int E, bool PREV, bool PROJ>
__global__ void __launch_bounds__(Geo<E>::NT, Geo<E>::MINB) k_cheb(const __grid_constant__ ChebArgs a) {
  using G = Geo<E>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 fi = a.items[blockIdx.x];
  const int f = fi.x, i0 = fi.y;
  const FragDesc &D = a.desc[f];
  const int A = D.natom;
  const int nvalid = min(2, D.norb - i0);
  const int r0 = a.row_beg[D.row_off];
  const int nent = a.row_beg[D.row_off + G::PLANE] - r0;
  const ChebSmem<E> m = cheb_carve<E>(smem_raw, A, a.maxent, nent);
  const int tabw = tab_width(D);

  float alpha = 1.f, beta = 0.f, shift = 0.f;
  if (a.cheb) {
    const double *bd = a.bounds + (long long)f * a.bstride;
    shift = float(bd[3]);
    alpha = float(bd[4 + 2 * a.step]);
    beta = float(bd[5 + 2 * a.step]);
  }
  // tables: x factors (splatted), supports, D C <p|y>, row starts, entries; zero halo and accumulators
  for (int t = threadIdx.x; t < A * E; t += G::NT) {
    const int k = t / E, x = t - k * E;
    const float g = a.tab[D.tab_off + (long long)k * tabw + x];
    m.gx2[t] = f2(g, g);
  }
  for (int k = threadIdx.x; k < A; k += G::NT) {
    const ProjSlot S = a.slots[D.at_off + k];
    m.box[k] = make_int2(S.lo[0] >> 1, min((S.hi[0] + 1) >> 1, G::NPX));
    const float ds = float(a.Datom[S.atom] * S.coef);
    const float *ci = a.cin + D.c_off + (long long)i0 * A + k;
    m.sk2[k] = f2(ds * ci[0], nvalid > 1 ? ds * ci[A] : 0.f);
  }
  for (int t = threadIdx.x; t <= G::PLANE; t += G::NT) m.rb[t] = a.row_beg[D.row_off + t] - r0;
  for (int t = threadIdx.x; t < nent; t += G::NT) m.sent[t] = a.row_ent[r0 + t];
  for (int t = threadIdx.x; t < E * A; t += G::NT) m.pacc[t] = f2(0.f, 0.f);
  for (int t = threadIdx.x; t < 2 * G::PPLANE; t += G::NT) m.pin[t] = f2(0.f, 0.f);

  ChebT T;
  const int tid = threadIdx.x;
  T.active = tid < G::NP;
  T.py = T.active ? tid / G::NPX : 0;
  T.px = T.active ? 2 * (tid - T.py * G::NPX) : 0;
  T.t0 = T.py * E + T.px;
  T.ksh = f2(a.kc - shift, a.kc - shift);
  T.al2 = f2(alpha, alpha);
  T.be2 = f2(beta, beta);

  const long long P = (long long)G::PLANE * E;
  const long long base = D.psi_off + (long long)i0 * P;
  const float *yin = a.yin + base;
  const float *yprev = PREV ? a.yprev + base : nullptr;
  float *yout = a.yout + base;
  const float2 *vf2 = a.vf2 + D.pt_off;
  // z column of planes -4..4 (zero outside the fragment), V and y_prev of plane 0
  float4 q[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    q[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (T.active && k >= 4 && k - 4 < E) {
      const float *p = yin + (k - 4) * G::PLANE + T.t0;
      const float2 u0 = *reinterpret_cast<const float2 *>(p);
      const float2 u1 = nvalid > 1 ? *reinterpret_cast<const float2 *>(p + P) : f2(0.f, 0.f);
      q[k] = make_float4(u0.x, u1.x, u0.y, u1.y);
    }
  }
  float4 vv = make_float4(0.f, 0.f, 0.f, 0.f), pv = make_float4(0.f, 0.f, 0.f, 0.f);
  if (T.active) {
    vv = *reinterpret_cast<const float4 *>(vf2 + T.t0);
    if (PREV) {
      const float2 u0 = *reinterpret_cast<const float2 *>(yprev + T.t0);
      const float2 u1 = nvalid > 1 ? *reinterpret_cast<const float2 *>(yprev + T.t0 + P) : f2(0.f, 0.f);
      pv = make_float4(u0.x, u1.x, u0.y, u1.y);
    }
  }
  __syncthreads();

#define DC_CHEB_PLANE(ZI)                                                                                  \
  if (z0 + ZI < E)                                                                                         \
    cheb_plane<E, PREV, PROJ, ZI>(a, m, T, q, vv, pv, z0 + ZI, A, nvalid, yin, yprev, yout, vf2);
  for (int z0 = 0; z0 < E; z0 += 9) {
    DC_CHEB_PLANE(0)
    DC_CHEB_PLANE(1)
    DC_CHEB_PLANE(2)
    DC_CHEB_PLANE(3)
    DC_CHEB_PLANE(4)
    DC_CHEB_PLANE(5)
    DC_CHEB_PLANE(6)
    DC_CHEB_PLANE(7)
    DC_CHEB_PLANE(8)
  }
#undef DC_CHEB_PLANE
  if (PROJ) {
    __syncthreads();
    // the last plane's projection tasks
    {
      const int zp = E - 1, ps = zp & 1;
      const int e0 = m.rb[zp * E], n = m.rb[E * E] - e0;
      const float4 *rc = m.rec + (zp % 3) * a.maxent;
      const float4 *o4 = reinterpret_cast<const float4 *>(m.pout + ps * G::PLANE);
      const float4 *g4 = reinterpret_cast<const float4 *>(m.gx2);
      for (int t = threadIdx.x; t < n; t += G::NT) {
        const int kb = m.sent[e0 + t].x;
        const int k = kb & 0xffff, y = kb >> 16;
        const int2 bx = m.box[k];
        float2 s0 = f2(0.f, 0.f), s1 = f2(0.f, 0.f);
        for (int x2 = bx.x; x2 < bx.y; ++x2) {
          const float4 o = o4[y * G::NPX + x2];
          const float4 g = g4[k * G::NPX + x2];
          s0 = fma2(lo2(o), lo2(g), s0);
          s1 = fma2(hi2(o), hi2(g), s1);
        }
        const float w = rc[t].w;
        float2 &pa = m.pacc[y * A + k];
        pa = fma2(f2(w, w), add2(s0, s1), pa);
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nvalid * A; t += G::NT) {
      const int o = t / A, k = t - o * A;
      float s = 0.f;
      for (int y = 0; y < E; ++y) {
        const float2 v = m.pacc[y * A + k];
        s += o == 0 ? v.x : v.y;
      }
      const ProjSlot S = a.slots[D.at_off + k];
      a.cout[D.c_off + (long long)(i0 + o) * A + k] = float(S.coef * a.dV) * s;
    }
  }
}

template <int E>
bool cheb_fits(const dc_ctx *c) {
  return cheb_smem_bytes<E>(c->max_atoms, std::max(1, c->max_plane_ent), std::max(1, c->max_frag_ent)) <=
         227 * 1024;
}

template <int E, bool PREV, bool PROJ>
int run_cheb(const dc_ctx *c, const ChebArgs &a, cudaStream_t s) {
  using G = Geo<E>;
  const size_t sm = cheb_smem_bytes<E>(c->max_atoms, a.maxent, std::max(1, c->max_frag_ent));
  DC_CUDA(dc_set_smem((const void *)k_cheb<E, PREV, PROJ>, sm));
  if (c->n_items2 > 0) k_cheb<E, PREV, PROJ><<<(unsigned)c->n_items2, G::NT, sm, s>>>(a);
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
  a.vf2 = c->d_vf2;
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
