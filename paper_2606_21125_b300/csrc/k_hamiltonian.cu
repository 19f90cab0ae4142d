// Fragment Hamiltonian kernels (Eq. 5, model Hamiltonian) for sm_103a.
//
// H_f y = -1/2 L8 y + V_f y + sum_a D_a p_a <p_a|y>, <u|v> = dV sum u v, with the 8th-order
// 25-point Laplacian and ghost points that are zero (buffer edge) or wrap within the fragment.
// The projectors are separable, p_a(j) = C_a gx_a[jx] gy_a[jy] gz_a[jz].
//
// One CTA handles NO orbitals of one fragment (NO = 2 in FP32) and streams the fragment along z.
// Each thread owns pairs of x-adjacent points of the xy-plane, for every one of the CTA's
// orbitals, and keeps their 9-deep z columns in registers; the current planes sit in shared memory
// with a 4-point halo (zeros, or wrapped values for the periodic boundary), so the x and y taps
// are unconditional vector loads, and each pair is updated with paired FP32 instructions
// (FFMA2/FADD2).  Addressing, the per-plane atom lists and all loop control are shared by the
// orbitals of a thread, which is where most of the instructions of this kernel go.
//
// The Laplacian is evaluated in difference form, sum_n k_n [(y_{+n} - y) + (y_{-n} - y)], which
// equals the textbook form because c_0 = -2 sum_n c_n; the differences of neighbouring values are
// exact in floating point for smooth orbitals, so the large centre and neighbour terms never cancel
// in rounded arithmetic (100x smaller FP32 error at the same data movement).
//
// Nonlocal term: for each plane, warps compact, per row y, the atoms whose projector touches (y, z)
// into records (slot, D_a C_a <p_a|psi_o> gz_a[z] gy_a[y] for each orbital o); a point adds
// u_o * gx_a[x] over its row's records only.  The projections of the output, which the next
// Chebyshev step needs, are accumulated one plane behind: one task per (row, atom of that row)
// forms sum_x gx_a[x] out_o(x, y) and adds it into a dense [orbital][row][atom] array (each slot has
// one writer per plane, so the order is fixed and the result deterministic); rows are summed last.
#include <algorithm>
#include <type_traits>

#include "dc_internal.h"

namespace {

template <typename T>
struct HArgs {
  const FragDesc *desc;
  const int2 *items;
  const ProjSlot *slots;
  const T *tab;
  const int *zl_beg;
  const int *zl_items;
  const int *row_beg;
  const int2 *row_ent;
  int maxent;
  const T *vf;
  const T *yin;
  const T *yprev;
  T *yout;
  const T *cin;
  T *cout;
  const double *Datom;
  const double *occ;
  double *dots;
  const double *bounds;
  int bstride;
  int step;
  int mode;
  int periodic;
  double dV;
  T kx[5], ky[5], kz[5];  // -1/2 c_n / h_d^2
};

// Arithmetic on the two points of a pair: paired FP32 instructions, scalar pairs for FP64.
template <typename T>
struct P2;
template <>
struct P2<float> {
  using V = float2;
  static __device__ __forceinline__ V mk(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ V splat(float a) { return make_float2(a, a); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
  static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
};
template <>
struct P2<double> {
  using V = double2;
  static __device__ __forceinline__ V mk(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ V splat(double a) { return make_double2(a, a); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y)); }
  static __device__ __forceinline__ V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ V sub(V a, V b) { return make_double2(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ V mul(V a, V b) { return make_double2(a.x * b.x, a.y * b.y); }
};

// Per-row record coefficients of the NO orbitals, each splatted over the two points of a pair.
template <typename T, int NO>
struct RU {
  typename P2<T>::V u[NO];
};

template <typename T>
__device__ __forceinline__ typename P2<T>::V ld2(const T *p) {
  return *reinterpret_cast<const typename P2<T>::V *>(p);
}

template <typename T, int NT>
__device__ __forceinline__ T block_sum(T v, T *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NT / 32; ++i) s += red[i];
  }
  return s;  // valid in thread 0
}

// Per-row atom lists of plane z: for every row y, the slots k of the plane's z-list whose y factor
// is non-zero there.  One warp per row, compaction by ballot.  With ru != nullptr the records also
// get u_o = sk[o][k] gz_k[z] gy_k[y] for the NO orbitals.
template <typename T, int NT, int NO>
__device__ __forceinline__ void build_rows(int z, int Ex, int Ey, int A, const T *stab, int tabw, const int *zl_b,
                                           const int *zl_i, const T *sk, RU<T, NO> *ru, int *rk, int *rn) {
  using Op = P2<T>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int zbeg = zl_b[z], zend = zl_b[z + 1];
  for (int y = warp; y < Ey; y += NT / 32) {
    int cnt = 0;
    for (int e0 = zbeg; e0 < zend; e0 += 32) {
      const int e = e0 + lane;
      int k = 0;
      T gzy = T(0);
      if (e < zend) {
        k = zl_i[e];
        const T *g = stab + k * tabw;
        gzy = g[Ex + Ey + z] * g[Ex + y];
      }
      const bool in = gzy != T(0);
      const unsigned m = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int pos = cnt + __popc(m & ((1u << lane) - 1u));
        rk[y * A + pos] = k;
        if (ru) {
          RU<T, NO> r;
#pragma unroll
          for (int o = 0; o < NO; ++o) r.u[o] = Op::splat(sk[o * A + k] * gzy);
          ru[y * A + pos] = r;
        }
      }
      cnt += __popc(m);
    }
    if (lane == 0) rn[y] = cnt;
  }
}

// Projection tasks of one plane (values pl[o][y][x], plane stride `ps`, row pitch Ex): for each
// row y and listed slot k, pacc[o][y][k] += gz_k[z] gy_k[y] sum_x gx_k[x] pl[o][y][x].  Slot (o, y, k)
// has one writer per plane.
template <typename T, int NT, int NO>
__device__ __forceinline__ void project_rows(const T *pl, int ps, int z, int Ex, int Ey, int A, const T *stab,
                                             int tabw, const int4 *box, const int *rk, const int *rn, T *pacc,
                                             int nvalid) {
  const int nslot = Ey * A;
  for (int s = threadIdx.x; s < nslot; s += NT) {
    const int y = s % Ey, e = s / Ey;
    if (e >= rn[y]) continue;
    const int k = rk[y * A + e];
    const T *g = stab + k * tabw;
    const int4 bx = box[k];
    const T gzy = g[Ex + Ey + z] * g[Ex + y];
    T w[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) w[o] = T(0);
    for (int x = bx.x; x < bx.y; ++x) {
      const T gv = g[x];
#pragma unroll
      for (int o = 0; o < NO; ++o) w[o] += gv * pl[o * ps + y * Ex + x];
    }
#pragma unroll
    for (int o = 0; o < NO; ++o)
      if (o < nvalid) pacc[(o * Ey + y) * A + k] += gzy * w[o];
  }
}

template <typename T, int NT, int PP, int NO>
__global__ void __launch_bounds__(NT, NT <= 256 ? (NO == 2 ? 2 : 3) : 1) k_hstep(HArgs<T> a) {
  using Op = P2<T>;
  using V = typename Op::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int item = blockIdx.x;
  const int2 fi = a.items[item];
  const int f = fi.x, i0 = fi.y;
  const FragDesc D = a.desc[f];
  const int nvalid = min(NO, D.norb - i0);  // orbitals i0 .. i0+nvalid-1 of fragment f
  const int Ex = D.E[0], Ey = D.E[1], Ez = D.E[2];
  const int plane = Ex * Ey;
  const int nxp = (Ex + 1) >> 1;
  const int npairs = nxp * Ey;
  const int pitch = (Ex + 9) & ~1;  // >= Ex + 8, even
  const int pplane = pitch * (Ey + 8);
  const long long P = (long long)plane * Ez;
  const int A = D.natom;
  const int tabw = tab_width(D);
  const bool proj = a.cout != nullptr;

  // shared memory: element arrays (vector-read ones first, at even offsets), then 16-byte aligned
  // records and integers
  T *pin = reinterpret_cast<T *>(smem_raw);  // [2 buf][NO][pplane]
  T *stab = pin + 2 * NO * pplane;           // [A][tabw]
  T *pout = stab + A * tabw;                 // [2 buf][NO][plane]
  T *pacc = pout + 2 * NO * plane;           // [NO][Ey][A]
  T *sk = pacc + NO * Ey * A;                // [NO][A]
  T *red = sk + NO * A;                      // [NT/32]
  size_t off = (size_t)(2 * NO * pplane + A * tabw + 2 * NO * plane + NO * Ey * A + NO * A + NT / 32) * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  int4 *box = reinterpret_cast<int4 *>(smem_raw + off);         // [A]
  RU<T, NO> *ru = reinterpret_cast<RU<T, NO> *>(box + A);       // [2 buf][Ey][A]
  int *rk = reinterpret_cast<int *>(ru + 2 * Ey * A);           // [2 buf][Ey][A]
  int *rn = rk + 2 * Ey * A;                                    // [2 buf][Ey]
  int *zl_b = rn + 2 * Ey;                                      // [Ez+1]
  int *zl_i = zl_b + Ez + 1;                                    // [list]

  const int zb0 = a.zl_beg[D.zl_off];
  const int nzl = a.zl_beg[D.zl_off + Ez] - zb0;
  for (int t = threadIdx.x; t < A * tabw; t += NT) stab[t] = a.tab[D.tab_off + t];
  for (int t = threadIdx.x; t <= Ez; t += NT) zl_b[t] = a.zl_beg[D.zl_off + t] - zb0;
  for (int t = threadIdx.x; t < nzl; t += NT) zl_i[t] = a.zl_items[zb0 + t];
  for (int k = threadIdx.x; k < A; k += NT) {
    const ProjSlot S = a.slots[D.at_off + k];
    box[k] = make_int4(S.lo[0], S.hi[0], S.lo[1], S.hi[1]);
    const T ds = T(a.Datom[S.atom] * S.coef);
#pragma unroll
    for (int o = 0; o < NO; ++o)
      sk[o * A + k] = (a.cin && o < nvalid) ? ds * a.cin[D.c_off + (long long)(i0 + o) * A + k] : T(0);
  }
  for (int t = threadIdx.x; t < NO * Ey * A; t += NT) pacc[t] = T(0);
  for (int t = threadIdx.x; t < 2 * NO * pplane; t += NT) pin[t] = T(0);

  T alpha = T(1), beta = T(0), shift = T(0);
  if (a.mode == HSTEP_CHEB) {
    const double *bd = a.bounds + (long long)f * a.bstride;
    shift = T(bd[3]);
    alpha = T(bd[4 + 2 * a.step]);
    beta = T(bd[5 + 2 * a.step]);
  }
  const bool use_prev = (a.mode == HSTEP_CHEB) && a.yprev != nullptr && a.step > 0;
  // orbital o of the item lives at element offset base + o * P (invalid orbitals read orbital 0)
  const long long base = D.psi_off + (long long)i0 * P;
  const long long ostride = P;
  const T *vf = a.vf + D.pt_off;
  T occ2[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o)
    occ2[o] = (a.mode == HSTEP_ADJ && o < nvalid) ? T(2.0 * a.occ[D.st_off + i0 + o] * a.dV) : T(0);

  int px[PP], py[PP];
  bool valid[PP], v1[PP];
  V q[PP][NO][9];
#pragma unroll
  for (int r = 0; r < PP; ++r) {
    const int p = threadIdx.x + r * NT;
    valid[r] = p < npairs;
    py[r] = valid[r] ? p / nxp : 0;
    px[r] = valid[r] ? 2 * (p - py[r] * nxp) : 0;
    v1[r] = valid[r] && (px[r] + 1 < Ex);
    const int t0 = px[r] + py[r] * Ex;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const T *col = a.yin + base + (o < nvalid ? o : 0) * ostride + t0;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        int zz = k - 4;
        bool in = zz >= 0 && zz < Ez;
        if (!in && a.periodic) {
          zz = zz < 0 ? zz + Ez : zz - Ez;
          in = true;
        }
        const T *pz = col + (long long)zz * plane;
        q[r][o][k] = Op::mk((in && valid[r]) ? pz[0] : T(0), (in && v1[r]) ? pz[1] : T(0));
      }
    }
  }
  __syncthreads();

  T dot[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) dot[o] = T(0);
  for (int z = 0; z < Ez; ++z) {
    const int buf = z & 1;
    T *P0 = pin + buf * NO * pplane;
#pragma unroll
    for (int r = 0; r < PP; ++r) {
      if (!valid[r]) continue;
      const int x = px[r], y = py[r];
      const int c = (y + 4) * pitch + x + 4;
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        T *Po = P0 + o * pplane;
        const V v = q[r][o][4];
        Po[c] = v.x;
        if (v1[r]) Po[c + 1] = v.y;
        if (a.periodic) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (h == 1 && !v1[r]) continue;
            const int xx = x + h;
            const T vv = h == 0 ? v.x : v.y;
            if (xx < 4) Po[c + h + Ex] = vv;
            if (xx >= Ex - 4) Po[c + h - Ex] = vv;
            if (y < 4) Po[c + h + Ey * pitch] = vv;
            if (y >= Ey - 4) Po[c + h - Ey * pitch] = vv;
          }
        }
      }
    }
    RU<T, NO> *RUb = ru + buf * Ey * A;
    int *RK = rk + buf * Ey * A;
    int *RN = rn + buf * Ey;
    build_rows<T, NT, NO>(z, Ex, Ey, A, stab, tabw, zl_b, zl_i, sk, RUb, RK, RN);
    __syncthreads();
    if (proj && z > 0) {
      const int pb = (z - 1) & 1;
      project_rows<T, NT, NO>(pout + pb * NO * plane, plane, z - 1, Ex, Ey, A, stab, tabw, box, rk + pb * Ey * A,
                              rn + pb * Ey, pacc, nvalid);
    }

    // next planes' global values: issue the loads early
    int zn = z + 5;
    bool zin = zn < Ez;
    if (!zin && a.periodic) {
      zn -= Ez;
      zin = true;
    }
    const long long zoff = (long long)zn * plane;
    const long long o_here = (long long)z * plane;
#pragma unroll
    for (int r = 0; r < PP; ++r) {
      if (!valid[r]) continue;
      const int x = px[r], y = py[r];
      const int t0 = y * Ex + x;
      const T *c0 = P0 + (y + 4) * pitch + x + 4;
      V nxt[NO];
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        const T *pz = a.yin + base + (o < nvalid ? o : 0) * ostride + zoff + t0;
        nxt[o] = Op::mk(zin ? pz[0] : T(0), (zin && v1[r]) ? pz[1] : T(0));
      }
      const V vv = Op::mk(vf[o_here + t0], v1[r] ? vf[o_here + t0 + 1] : T(0));
      V hxy[NO], hz[NO], hn[NO];
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        const T *co = c0 + o * pplane;
        const V cv = q[r][o][4];
        T xv[10];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          const V v = ld2(co - 4 + 2 * j);
          xv[2 * j] = v.x;
          xv[2 * j + 1] = v.y;
        }
        if constexpr (std::is_same<T, double>::value) {
          // FP64: direct form, sum_n k_n (y+n + y-n) per axis plus (V + k_0) y at the centre (k_0 summed over
          // the axes): ~35 FP64 operations per point against ~60 for the difference form, whose rounding
          // advantage matters only in FP32.  On this part FP64 runs at 1/64 of the FP32 rate, so the
          // operation count is the kernel's cost.
          V h = Op::mul(Op::add(vv, Op::splat(a.kx[0] + a.ky[0] + a.kz[0])), cv);
#pragma unroll
          for (int n = 1; n <= 4; ++n) {
            const V sx = Op::add(Op::mk(xv[4 + n], xv[5 + n]), Op::mk(xv[4 - n], xv[5 - n]));
            const V sy = Op::add(ld2(co + n * pitch), ld2(co - n * pitch));
            const V sz = Op::add(q[r][o][4 + n], q[r][o][4 - n]);
            h = Op::fma(Op::splat(a.kx[n]), sx, Op::fma(Op::splat(a.ky[n]), sy, Op::fma(Op::splat(a.kz[n]), sz, h)));
          }
          hxy[o] = h;
        } else {
          // FP32: difference form (each tap as (y+n - y) + (y-n - y)), which keeps the cancellation against
          // the centre out of the rounding
          V h1 = Op::splat(T(0)), h2 = Op::splat(T(0));
#pragma unroll
          for (int n = 1; n <= 4; ++n) {
            const V pa = Op::mk(xv[4 + n], xv[5 + n]);
            const V pb = Op::mk(xv[4 - n], xv[5 - n]);
            h1 = Op::fma(Op::splat(a.kx[n]), Op::add(Op::sub(pa, cv), Op::sub(pb, cv)), h1);
            const V up = ld2(co + n * pitch);
            const V dn = ld2(co - n * pitch);
            h2 = Op::fma(Op::splat(a.ky[n]), Op::add(Op::sub(up, cv), Op::sub(dn, cv)), h2);
          }
          V h3 = Op::mul(vv, cv);
#pragma unroll
          for (int n = 1; n <= 4; ++n)
            h3 = Op::fma(Op::splat(a.kz[n]), Op::add(Op::sub(q[r][o][4 + n], cv), Op::sub(q[r][o][4 - n], cv)), h3);
          hxy[o] = Op::add(h1, h2);
          hz[o] = h3;
        }
        hn[o] = Op::splat(T(0));
      }
      const int cnt = RN[y];
      const RU<T, NO> *ry = RUb + y * A;
      const int *rky = RK + y * A;
      for (int e = 0; e < cnt; ++e) {
        const V g = ld2(stab + rky[e] * tabw + x);
        const RU<T, NO> rec = ry[e];
#pragma unroll
        for (int o = 0; o < NO; ++o) hn[o] = Op::fma(rec.u[o], g, hn[o]);
      }
      const long long o0 = o_here + t0;
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        if (o >= nvalid) continue;
        const V cv = q[r][o][4];
        V hv;
        if constexpr (std::is_same<T, double>::value)
          hv = Op::add(hxy[o], hn[o]);
        else
          hv = Op::add(Op::add(hxy[o], hz[o]), hn[o]);
        V out;
        if (a.mode == HSTEP_CHEB) {
          out = Op::mul(Op::splat(alpha), Op::fma(Op::splat(-shift), cv, hv));
          if (use_prev) {
            const T *pv = a.yprev + base + o * ostride + o0;
            out = Op::fma(Op::splat(beta), Op::mk(pv[0], v1[r] ? pv[1] : T(0)), out);
          }
        } else if (a.mode == HSTEP_ADJ) {
          dot[o] += cv.x * hv.x + (v1[r] ? cv.y * hv.y : T(0));
          out = Op::mul(Op::splat(occ2[o]), hv);
        } else {
          out = hv;
        }
        if (a.yout) {
          T *po = a.yout + base + o * ostride + o0;
          po[0] = out.x;
          if (v1[r]) po[1] = out.y;
        }
        if (proj) {
          T *pp = pout + (buf * NO + o) * plane + t0;
          pp[0] = out.x;
          if (v1[r]) pp[1] = out.y;
        }
      }
      // advance the z columns
#pragma unroll
      for (int o = 0; o < NO; ++o) {
#pragma unroll
        for (int k = 0; k < 8; ++k) q[r][o][k] = q[r][o][k + 1];
        q[r][o][8] = nxt[o];
      }
    }
  }
  if (proj) {
    __syncthreads();
    const int pb = (Ez - 1) & 1;
    project_rows<T, NT, NO>(pout + pb * NO * plane, plane, Ez - 1, Ex, Ey, A, stab, tabw, box, rk + pb * Ey * A,
                            rn + pb * Ey, pacc, nvalid);
    __syncthreads();
    for (int t = threadIdx.x; t < nvalid * A; t += NT) {
      const int o = t / A, k = t - o * A;
      T s = T(0);
      for (int y = 0; y < Ey; ++y) s += pacc[(o * Ey + y) * A + k];
      const ProjSlot S = a.slots[D.at_off + k];
      a.cout[D.c_off + (long long)(i0 + o) * A + k] = T(S.coef * a.dV) * s;
    }
  }
  if (a.mode == HSTEP_ADJ) {
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const T s = block_sum<T, NT>(dot[o], red);
      if (threadIdx.x == 0 && o < nvalid) a.dots[D.st_off + i0 + o] = a.occ[D.st_off + i0 + o] * a.dV * (double)s;
    }
  }
}

// Projections c[k] = C_k dV sum_j p_k(j) y(j) of one orbital block (no stencil), with the same
// row-list tasks as the H-apply epilogue.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_project(HArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int item = blockIdx.x;
  const int2 fi = a.items[item];
  const int f = fi.x, i = fi.y;
  const FragDesc D = a.desc[f];
  const int Ex = D.E[0], Ey = D.E[1], Ez = D.E[2];
  const int plane = Ex * Ey;
  const long long P = (long long)plane * Ez;
  const int A = D.natom;
  const int tabw = tab_width(D);
  T *pl = reinterpret_cast<T *>(smem_raw);  // [2][plane]
  T *stab = pl + 2 * plane;                 // [A][tabw]
  T *pacc = stab + A * tabw;                // [Ey][A]
  size_t off = (size_t)(2 * plane + A * tabw + Ey * A) * sizeof(T);
  off = (off + 15) & ~(size_t)15;
  int4 *box = reinterpret_cast<int4 *>(smem_raw + off);  // [A]
  int *kl = reinterpret_cast<int *>(box + A);            // [2][Ey][A]
  int *rn = kl + 2 * Ey * A;                             // [2][Ey]
  int *zl_b = rn + 2 * Ey;                               // [Ez+1]
  int *zl_i = zl_b + Ez + 1;                             // [list]
  const int zb0 = a.zl_beg[D.zl_off];
  const int nzl = a.zl_beg[D.zl_off + Ez] - zb0;
  for (int t = threadIdx.x; t < A * tabw; t += NT) stab[t] = a.tab[D.tab_off + t];
  for (int t = threadIdx.x; t <= Ez; t += NT) zl_b[t] = a.zl_beg[D.zl_off + t] - zb0;
  for (int t = threadIdx.x; t < nzl; t += NT) zl_i[t] = a.zl_items[zb0 + t];
  for (int k = threadIdx.x; k < A; k += NT) {
    const ProjSlot S = a.slots[D.at_off + k];
    box[k] = make_int4(S.lo[0], S.hi[0], S.lo[1], S.hi[1]);
  }
  for (int t = threadIdx.x; t < Ey * A; t += NT) pacc[t] = T(0);
  __syncthreads();
  const T *yin = a.yin + D.psi_off + (long long)i * P;
  for (int z = 0; z < Ez; ++z) {
    const int buf = z & 1;
    T *cur = pl + buf * plane;
    for (int t = threadIdx.x; t < plane; t += NT) cur[t] = yin[(long long)z * plane + t];
    build_rows<T, NT, 1>(z, Ex, Ey, A, stab, tabw, zl_b, zl_i, nullptr, nullptr, kl + buf * Ey * A, rn + buf * Ey);
    __syncthreads();
    project_rows<T, NT, 1>(cur, plane, z, Ex, Ey, A, stab, tabw, box, kl + buf * Ey * A, rn + buf * Ey, pacc, 1);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < A; k += NT) {
    T s = T(0);
    for (int y = 0; y < Ey; ++y) s += pacc[y * A + k];
    const ProjSlot S = a.slots[D.at_off + k];
    a.cout[D.c_off + (long long)i * A + k] = T(S.coef * a.dV) * s;
  }
}

// ---- orbital-pair kernel (FP32) -----------------------------------------------------------------
// Two orbitals of one fragment are interleaved at every point: a float2 holds (y_i, y_i+1) at one
// grid point, so each tap, the potential product and each nonlocal update of both orbitals is one
// paired instruction on operands that need no lane rearrangement, and every stencil read is an
// aligned 16-byte shared load covering two x-adjacent points.  A thread owns PP such point pairs of
// the plane and keeps their 9-deep z columns in registers (float4 = 2 points x 2 orbitals).
// The taps n = 1, 2 are taken in difference form, (y+n - y) + (y-n - y), the small outer taps
// n = 3, 4 as sums y+n + y-n with the centre term -2 (k3 + k4) y added once: their coefficients are
// 60x below k1, so their rounding stays under that of the V y product.  The Chebyshev scaling is
// folded into the coefficients: out = alpha L y + alpha (V - shift) y + alpha NL + beta y_prev.
// The per-row projector lists come precomputed from the host (one entry per (row, slot), in z-list
// order); each plane's entries are turned into records (u_i, u_i+1, slot|row, gz gy) once per CTA.
// One barrier per plane: point planes and output planes are double-buffered, records triple-buffered.

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Stencil coefficients, splatted over the orbital pair.  ISO: one set for all three axes.
template <bool ISO>
struct PairK {
  float2 k1[ISO ? 1 : 3], k2[ISO ? 1 : 3], k3[ISO ? 1 : 3], k4[ISO ? 1 : 3];
  float2 kc;  // -2 sum over axes of (k3 + k4)
};

// alpha (-1/2 L8) y at one point (centre c) from its 24 neighbours, plus h.
template <bool ISO>
__device__ __forceinline__ float2 lap_pair(const PairK<ISO> &K, float2 c, const float2 (&xm)[4],
                                           const float2 (&xp)[4], const float2 (&ym)[4], const float2 (&yp)[4],
                                           const float2 (&zm)[4], const float2 (&zp)[4], float2 h) {
  if (ISO) {
#pragma unroll
    for (int n = 0; n < 2; ++n) {
      float2 d = add2(sub2(xp[n], c), sub2(xm[n], c));
      d = add2(d, add2(sub2(yp[n], c), sub2(ym[n], c)));
      d = add2(d, add2(sub2(zp[n], c), sub2(zm[n], c)));
      h = fma2(n == 0 ? K.k1[0] : K.k2[0], d, h);
    }
#pragma unroll
    for (int n = 2; n < 4; ++n) {
      const float2 t = add2(add2(add2(xp[n], xm[n]), add2(yp[n], ym[n])), add2(zp[n], zm[n]));
      h = fma2(n == 2 ? K.k3[0] : K.k4[0], t, h);
    }
  } else {
#pragma unroll
    for (int n = 0; n < 2; ++n) {
      const float2 *kk = n == 0 ? K.k1 : K.k2;
      h = fma2(kk[0], add2(sub2(xp[n], c), sub2(xm[n], c)), h);
      h = fma2(kk[1], add2(sub2(yp[n], c), sub2(ym[n], c)), h);
      h = fma2(kk[2], add2(sub2(zp[n], c), sub2(zm[n], c)), h);
    }
#pragma unroll
    for (int n = 2; n < 4; ++n) {
      const float2 *kk = n == 2 ? K.k3 : K.k4;
      h = fma2(kk[0], add2(xp[n], xm[n]), h);
      h = fma2(kk[1], add2(yp[n], ym[n]), h);
      h = fma2(kk[2], add2(zp[n], zm[n]), h);
    }
  }
  return fma2(K.kc, c, h);
}

// Shared-memory carve of the orbital-pair kernels (sizes in the fragment's own extents).
struct PairSmem {
  float2 *pin, *pout, *gx2, *pacc, *sk2;
  float4 *rec;  // [nrec][maxent] (u_i, u_i+1, float4 index of the slot's x factors, gz gy)
  int *recky;   // [nrec][maxent] slot | row << 16
  int2 *box;
  int *rb;
  float *red;  // [2][NT / 32] (at most 2 x 32 floats)
};

// Row pitch (in float2) of the haloed plane of the pair kernels: at least Ex + 8, and congruent modulo
// 16 to the 2 ceil(Ex/2) float2 that one row of threads covers, so that the 16-byte loads of a warp whose
// threads run over several rows still fall on consecutive banks (no shared-memory bank conflicts).
__host__ __device__ __forceinline__ int pair_pitch(int Ex) { return 2 * ((Ex + 1) >> 1) + 16; }

__device__ __forceinline__ PairSmem pair_carve(unsigned char *raw, int Ex, int Ey, int Ez, int A, int maxent,
                                               int nrec, bool halo) {
  const int pitch = pair_pitch(Ex), pitch2 = (Ex + 1) & ~1;
  PairSmem m;
  m.pin = reinterpret_cast<float2 *>(raw);
  m.pout = m.pin + (halo ? 2 * (Ey + 8) * pitch : 0);
  m.gx2 = m.pout + 2 * Ey * pitch2;
  m.pacc = m.gx2 + A * pitch2;
  m.sk2 = m.pacc + Ey * A;
  size_t off = (size_t)(reinterpret_cast<unsigned char *>(m.sk2 + A) - raw);
  off = (off + 15) & ~(size_t)15;
  m.rec = reinterpret_cast<float4 *>(raw + off);
  m.recky = reinterpret_cast<int *>(m.rec + nrec * maxent);
  m.box = reinterpret_cast<int2 *>(m.recky + ((nrec * maxent + 1) & ~1));
  m.rb = reinterpret_cast<int *>(m.box + A);
  m.red = reinterpret_cast<float *>(m.rb + Ez * Ey + 1);
  return m;
}

size_t pair_smem_bytes(int Ex, int Ey, int Ez, int A, int maxent, int nrec, bool halo, int NT, int PP = 0) {
  const int pitch = pair_pitch(Ex), pitch2 = (Ex + 1) & ~1;
  size_t n2 = (halo ? 2 * (size_t)(Ey + 8) * pitch : 0) + 2 * (size_t)Ey * pitch2 + (size_t)A * pitch2 +
              (size_t)Ey * A + A;
  size_t b = (n2 * sizeof(float2) + 15) & ~(size_t)15;
  b += (size_t)nrec * maxent * sizeof(float4) + (size_t)((nrec * maxent + 1) & ~1) * sizeof(int) +
       (size_t)A * sizeof(int2) + (size_t)(Ez * Ey + 1) * sizeof(int) + 2 * 32 * sizeof(float);
  (void)PP;
  return b + 64;
}

// Common CTA setup: x factors splatted over the pair (zero on the padded column), x supports rounded
// out to even bounds, row starts relative to the fragment's first entry, zeroed accumulators.
template <int NT>
__device__ __forceinline__ void pair_setup(const HArgs<float> &a, const FragDesc &D, const PairSmem &m, int i0,
                                           int nvalid, float alpha) {
  const int Ex = D.E[0], Ey = D.E[1], Ez = D.E[2], A = D.natom, tabw = tab_width(D);
  const int pitch2 = (Ex + 1) & ~1;
  for (int t = threadIdx.x; t < A * pitch2; t += NT) {
    const int k = t / pitch2, x = t - k * pitch2;
    const float g = x < Ex ? a.tab[D.tab_off + (long long)k * tabw + x] : 0.f;
    m.gx2[t] = f2(g, g);
  }
  for (int k = threadIdx.x; k < A; k += NT) {
    const ProjSlot S = a.slots[D.at_off + k];
    m.box[k] = make_int2(S.lo[0] & ~1, min((S.hi[0] + 1) & ~1, pitch2));
    const float ds = alpha * float(a.Datom[S.atom] * S.coef);
    float u0 = 0.f, u1 = 0.f;
    if (a.cin) {
      u0 = ds * a.cin[D.c_off + (long long)i0 * A + k];
      if (nvalid > 1) u1 = ds * a.cin[D.c_off + (long long)(i0 + 1) * A + k];
    }
    m.sk2[k] = f2(u0, u1);
  }
  const int r0 = a.row_beg[D.row_off];
  for (int t = threadIdx.x; t <= Ez * Ey; t += NT) m.rb[t] = a.row_beg[D.row_off + t] - r0;
  for (int t = threadIdx.x; t < Ey * A; t += NT) m.pacc[t] = f2(0.f, 0.f);
  for (int t = threadIdx.x; t < 2 * Ey * pitch2; t += NT) m.pout[t] = f2(0.f, 0.f);
}

// Projection tasks of one plane: one task per row-list entry (row y, slot k) forms
// gz gy sum_x gx_k[x] out(x, y) for both orbitals and adds it to pacc[y][k] (one writer per plane).
template <int NT>
__device__ __forceinline__ void pair_project(const float2 *pl, const float4 *rc, const int *rky, int ne,
                                             const PairSmem &m, int pitch2, int A) {
  for (int t = threadIdx.x; t < ne; t += NT) {
    const int kb = rky[t];
    const float w = rc[t].w;
    const int k = kb & 0xffff, y = kb >> 16;
    const int2 bx = m.box[k];
    const float4 *o4 = reinterpret_cast<const float4 *>(pl + y * pitch2);
    const float4 *g4 = reinterpret_cast<const float4 *>(m.gx2 + k * pitch2);
    float2 s0 = f2(0.f, 0.f), s1 = f2(0.f, 0.f);
    for (int x = bx.x; x < bx.y; x += 2) {
      const float4 o = o4[x >> 1];
      const float4 g = g4[x >> 1];
      s0 = fma2(lo2(o), lo2(g), s0);
      s1 = fma2(hi2(o), hi2(g), s1);
    }
    float2 &pa = m.pacc[y * A + k];
    pa = fma2(f2(w, w), add2(s0, s1), pa);
  }
}

// Final projections c[i][k] = C_k dV sum_y pacc[y][k] of the pair.
template <int NT>
__device__ __forceinline__ void pair_finish(const HArgs<float> &a, const FragDesc &D, const PairSmem &m, int i0,
                                            int nvalid) {
  const int Ey = D.E[1], A = D.natom;
  for (int t = threadIdx.x; t < nvalid * A; t += NT) {
    const int o = t / A, k = t - o * A;
    float s = 0.f;
    for (int y = 0; y < Ey; ++y) {
      const float2 v = m.pacc[y * A + k];
      s += o == 0 ? v.x : v.y;
    }
    const ProjSlot S = a.slots[D.at_off + k];
    a.cout[D.c_off + (long long)(i0 + o) * A + k] = float(S.coef * a.dV) * s;
  }
}

// Records of plane z from its row-list entries: (u_i, u_i+1, float4 index k pitch2/2 of the slot's
// x factors, gz gy) and slot|row, with u = alpha D C <p|y> gz gy.  The first 2 NT entries come from
// registers (loaded one plane ahead), any further ones straight from global memory.
__device__ __forceinline__ void pair_record(int t, int2 e, const float2 *sk2, int pitch2, float4 *rc, int *rky) {
  const float w = __int_as_float(e.y);
  const int k = e.x & 0xffff;
  const float2 u = sk2[k];
  rc[t] = make_float4(u.x * w, u.y * w, __int_as_float(k * (pitch2 >> 1)), w);
  rky[t] = e.x;
}

template <int NT>
__device__ __forceinline__ void pair_records(const int2 *ent, int ne, const int2 (&pre)[2], const float2 *sk2,
                                             int pitch2, float4 *rc, int *rky) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int t = threadIdx.x + j * NT;
    if (t < ne) pair_record(t, pre[j], sk2, pitch2, rc, rky);
  }
  for (int t = threadIdx.x + 2 * NT; t < ne; t += NT) pair_record(t, ent[t], sk2, pitch2, rc, rky);
}

template <int NT>
__device__ __forceinline__ void pair_prefetch(const int2 *ent, int ne, int2 (&pre)[2]) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int t = threadIdx.x + j * NT;
    pre[j] = t < ne ? ent[t] : make_int2(0, 0);
  }
}

// Per-CTA constants of k_hpair.
template <int PP>
struct HPair {
  int Ex, Ey, Ez, plane, pitch, pitch2, pplane, A, P, nvalid, o1off;
  bool proj, use_prev, periodic;
  int mode;
  float vsh, alpha;
  float2 bb, occ2;
  const float *yin, *yprev, *vf;
  float *yout;
  const int2 *ent;
  int t0[PP];  // point offset y Ex + x of each owned pair (x even)
  int px[PP], py[PP];
  bool valid[PP], v1[PP];
};

// One plane z of k_hpair.  ZI = z mod 9 names the register slots: q[r][(ZI + k) % 9] holds plane
// z - 4 + k, so the column advances without moving registers (the kernel unrolls z by 9).
// vv/pvv hold this plane's V (2 points) and Y_{k-1} (2 points x 2 orbitals) per pair, loaded one
// plane earlier; the plane refills them for plane z + 1 right after reading them.
// ALLREC: the records of every plane were built once at CTA start (m.rec / m.recky indexed by the
// fragment's entry number); otherwise plane z builds its own into ring slot b3.
template <int NT, int PP, bool ISO, bool ALLREC, int ZI>
__device__ __forceinline__ void hpair_plane(const HPair<PP> &H, const PairK<ISO> &K, const PairSmem &m, int maxent,
                                            float4 (&q)[PP][9], float2 (&vv)[PP], float4 (&pvv)[PP],
                                            int2 (&pre)[2], float2 &dot, int z, int b3) {
  float2 *P0 = m.pin + (z & 1) * H.pplane;
  // centre values of plane z (and the periodic halo)
#pragma unroll
  for (int r = 0; r < PP; ++r) {
    if (!H.valid[r]) continue;
    const float4 cv = q[r][(ZI + 4) % 9];
    const int x = H.px[r], y = H.py[r];
    const int c = (y + 4) * H.pitch + x + 4;
    if (H.v1[r]) *reinterpret_cast<float4 *>(P0 + c) = cv;
    else P0[c] = lo2(cv);
    if (H.periodic) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !H.v1[r]) continue;
        const int xx = x + h;
        const float2 vv = h == 0 ? lo2(cv) : hi2(cv);
        if (xx < 4) P0[c + h + H.Ex] = vv;
        if (xx >= H.Ex - 4) P0[c + h - H.Ex] = vv;
        if (y < 4) P0[c + h + H.Ey * H.pitch] = vv;
        if (y >= H.Ey - 4) P0[c + h - H.Ey * H.pitch] = vv;
      }
    }
  }
  const int rz = z * H.Ey;
  const int e0 = m.rb[rz];
  const float4 *RC;
  if (ALLREC) {
    RC = m.rec + e0;
  } else {
    const int nez = m.rb[rz + H.Ey] - e0;
    float4 *rc = m.rec + b3 * maxent;
    pair_records<NT>(H.ent + e0, nez, pre, m.sk2, H.pitch2, rc, m.recky + b3 * maxent);
    if (z + 1 < H.Ez) pair_prefetch<NT>(H.ent + m.rb[rz + H.Ey], m.rb[rz + 2 * H.Ey] - m.rb[rz + H.Ey], pre);
    RC = rc;
  }
  __syncthreads();
  if (H.proj && z > 0) {
    const int zb = m.rb[rz - H.Ey];
    if (ALLREC) {
      pair_project<NT>(m.pout + ((z - 1) & 1) * H.Ey * H.pitch2, m.rec + zb, m.recky + zb, e0 - zb, m, H.pitch2,
                       H.A);
    } else {
      const int bp = b3 == 0 ? 2 : b3 - 1;
      pair_project<NT>(m.pout + ((z - 1) & 1) * H.Ey * H.pitch2, m.rec + bp * maxent, m.recky + bp * maxent,
                       e0 - zb, m, H.pitch2, H.A);
    }
  }

  int zn = z + 5;
  bool zin = zn < H.Ez;
  if (!zin && H.periodic) {
    zn -= H.Ez;
    zin = true;
  }
  const int zoff = zn * H.plane;
  const int oh = z * H.plane;
#pragma unroll
  for (int r = 0; r < PP; ++r) {
    if (!H.valid[r]) continue;
    const int x = H.px[r], y = H.py[r];
    const bool v1 = H.v1[r];
    const int t0 = H.t0[r];
    const float *pn = H.yin + zoff + t0;
    const float4 nxt = make_float4(zin ? pn[0] : 0.f, zin ? pn[H.o1off] : 0.f, (zin && v1) ? pn[1] : 0.f,
                                   (zin && v1) ? pn[H.o1off + 1] : 0.f);
    const float va = fmaf(H.alpha, vv[r].x, H.vsh);
    const float vb = v1 ? fmaf(H.alpha, vv[r].y, H.vsh) : 0.f;
    const float4 pv = pvv[r];
    if (z + 1 < H.Ez) {
      const int t1 = oh + H.plane + t0;
      vv[r] = make_float2(H.vf[t1], v1 ? H.vf[t1 + 1] : 0.f);
      if (H.use_prev) {
        const float *pp = H.yprev + t1;
        pvv[r] = make_float4(pp[0], pp[H.o1off], v1 ? pp[1] : 0.f, v1 ? pp[H.o1off + 1] : 0.f);
      }
    }
    const float2 *co = P0 + (y + 4) * H.pitch + x + 4;
    float2 row[10];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const float4 X = *reinterpret_cast<const float4 *>(co - 4 + 2 * j);
      row[2 * j] = lo2(X);
      row[2 * j + 1] = hi2(X);
    }
    float2 ym0[4], yp0[4], ym1[4], yp1[4], zm0[4], zp0[4], zm1[4], zp1[4], xm0[4], xp0[4], xm1[4], xp1[4];
#pragma unroll
    for (int n = 1; n <= 4; ++n) {
      const float4 u = *reinterpret_cast<const float4 *>(co + n * H.pitch);
      const float4 d = *reinterpret_cast<const float4 *>(co - n * H.pitch);
      yp0[n - 1] = lo2(u);
      yp1[n - 1] = hi2(u);
      ym0[n - 1] = lo2(d);
      ym1[n - 1] = hi2(d);
      zp0[n - 1] = lo2(q[r][(ZI + 4 + n) % 9]);
      zp1[n - 1] = hi2(q[r][(ZI + 4 + n) % 9]);
      zm0[n - 1] = lo2(q[r][(ZI + 4 - n) % 9]);
      zm1[n - 1] = hi2(q[r][(ZI + 4 - n) % 9]);
      xp0[n - 1] = row[4 + n];
      xm0[n - 1] = row[4 - n];
      xp1[n - 1] = row[5 + n];
      xm1[n - 1] = row[5 - n];
    }
    const float2 c0 = lo2(q[r][(ZI + 4) % 9]), c1 = hi2(q[r][(ZI + 4) % 9]);
    float2 h0 = fma2(f2(va, va), c0, mul2(H.bb, lo2(pv)));
    float2 h1 = fma2(f2(vb, vb), c1, mul2(H.bb, hi2(pv)));
    h0 = lap_pair<ISO>(K, c0, xm0, xp0, ym0, yp0, zm0, zp0, h0);
    h1 = lap_pair<ISO>(K, c1, xm1, xp1, ym1, yp1, zm1, zp1, h1);
    // nonlocal term over the row's records
    {
      const int eb = m.rb[rz + y] - e0, ee = m.rb[rz + y + 1] - e0;
      const float4 *g4 = reinterpret_cast<const float4 *>(m.gx2 + x);
      int e = eb;
      for (; e + 1 < ee; e += 2) {
        const float4 ra = RC[e], rb = RC[e + 1];
        const float4 ga = g4[__float_as_int(ra.z)], gb = g4[__float_as_int(rb.z)];
        h0 = fma2(lo2(ra), lo2(ga), h0);
        h1 = fma2(lo2(ra), hi2(ga), h1);
        h0 = fma2(lo2(rb), lo2(gb), h0);
        h1 = fma2(lo2(rb), hi2(gb), h1);
      }
      if (e < ee) {
        const float4 rr = RC[e];
        const float4 g = g4[__float_as_int(rr.z)];
        h0 = fma2(lo2(rr), lo2(g), h0);
        h1 = fma2(lo2(rr), hi2(g), h1);
      }
    }
    float2 out0 = h0, out1 = h1;
    if (H.mode == HSTEP_ADJ) {
      dot = fma2(c0, h0, dot);
      if (v1) dot = fma2(c1, h1, dot);
      out0 = mul2(H.occ2, h0);
      out1 = mul2(H.occ2, h1);
    }
    if (H.yout) {
      float *po = H.yout + oh + t0;
      po[0] = out0.x;
      if (v1) po[1] = out1.x;
      if (H.nvalid > 1) {
        po[H.P] = out0.y;
        if (v1) po[H.P + 1] = out1.y;
      }
    }
    if (H.proj) {
      float2 *pp = m.pout + (z & 1) * H.Ey * H.pitch2 + y * H.pitch2 + x;
      *reinterpret_cast<float4 *>(pp) = make_float4(out0.x, out0.y, v1 ? out1.x : 0.f, v1 ? out1.y : 0.f);
    }
    q[r][ZI % 9] = nxt;  // plane z + 5 replaces plane z - 4
  }
}

template <int NT, int PP, bool ISO, int MINB, bool ALLREC>
__global__ void __launch_bounds__(NT, MINB) k_hpair(HArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 fi = a.items[blockIdx.x];
  const int f = fi.x, i0 = fi.y;
  const FragDesc D = a.desc[f];
  HPair<PP> H;
  H.nvalid = min(2, D.norb - i0);
  H.Ex = D.E[0];
  H.Ey = D.E[1];
  H.Ez = D.E[2];
  H.plane = H.Ex * H.Ey;
  H.pitch = pair_pitch(H.Ex);
  H.pitch2 = (H.Ex + 1) & ~1;
  H.pplane = H.pitch * (H.Ey + 8);
  H.A = D.natom;
  H.P = H.plane * H.Ez;
  H.o1off = H.nvalid > 1 ? H.P : 0;
  H.proj = a.cout != nullptr;
  H.periodic = a.periodic != 0;
  H.mode = a.mode;
  const PairSmem m = pair_carve(smem_raw, H.Ex, H.Ey, H.Ez, H.A, a.maxent, ALLREC ? 1 : 3, true);

  float alpha = 1.f, beta = 0.f, shift = 0.f;
  if (a.mode == HSTEP_CHEB) {
    const double *bd = a.bounds + (long long)f * a.bstride;
    shift = float(bd[3]);
    alpha = float(bd[4 + 2 * a.step]);
    beta = float(bd[5 + 2 * a.step]);
  }
  H.use_prev = (a.mode == HSTEP_CHEB) && a.yprev != nullptr && a.step > 0;
  H.alpha = alpha;
  H.vsh = -alpha * shift;
  H.bb = f2(beta, beta);
  H.occ2 = f2(0.f, 0.f);
  if (a.mode == HSTEP_ADJ) {
    H.occ2.x = float(2.0 * a.occ[D.st_off + i0] * a.dV);
    if (H.nvalid > 1) H.occ2.y = float(2.0 * a.occ[D.st_off + i0 + 1] * a.dV);
  }
  // orbital i0 at element offset base, i0+1 at base + P (an invalid second orbital reads the first)
  const long long base = D.psi_off + (long long)i0 * H.P;
  H.yin = a.yin + base;
  H.yprev = H.use_prev ? a.yprev + base : nullptr;
  H.yout = a.yout ? a.yout + base : nullptr;
  H.vf = a.vf + D.pt_off;
  H.ent = a.row_ent + a.row_beg[D.row_off];
  pair_setup<NT>(a, D, m, i0, H.nvalid, alpha);
  for (int t = threadIdx.x; t < 2 * H.pplane; t += NT) m.pin[t] = f2(0.f, 0.f);

  PairK<ISO> K;
  {
    float s34 = 0.f;
#pragma unroll
    for (int d = 0; d < (ISO ? 1 : 3); ++d) {
      float kd[5];
#pragma unroll
      for (int n = 1; n < 5; ++n) kd[n] = alpha * (d == 0 ? a.kx[n] : (d == 1 ? a.ky[n] : a.kz[n]));
      K.k1[d] = f2(kd[1], kd[1]);
      K.k2[d] = f2(kd[2], kd[2]);
      K.k3[d] = f2(kd[3], kd[3]);
      K.k4[d] = f2(kd[4], kd[4]);
      s34 += (ISO ? 3.f : 1.f) * (kd[3] + kd[4]);
    }
    K.kc = f2(-2.f * s34, -2.f * s34);
  }

  const int nxp = (H.Ex + 1) >> 1;
  const int npairs = nxp * H.Ey;
  float4 q[PP][9];
#pragma unroll
  for (int r = 0; r < PP; ++r) {
    const int p = threadIdx.x + r * NT;
    H.valid[r] = p < npairs;
    H.py[r] = H.valid[r] ? p / nxp : 0;
    H.px[r] = H.valid[r] ? 2 * (p - H.py[r] * nxp) : 0;
    H.v1[r] = H.valid[r] && (H.px[r] + 1 < H.Ex);
    H.t0[r] = H.px[r] + H.py[r] * H.Ex;
    const float *col = H.yin + H.t0[r];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      int zz = k - 4;
      bool in = zz >= 0 && zz < H.Ez;
      if (!in && H.periodic) {
        zz = zz < 0 ? zz + H.Ez : zz - H.Ez;
        in = true;
      }
      const float *pz = col + zz * H.plane;
      const bool i0k = in && H.valid[r], i1k = in && H.v1[r];
      q[r][k] = make_float4(i0k ? pz[0] : 0.f, i0k ? pz[H.o1off] : 0.f, i1k ? pz[1] : 0.f,
                            i1k ? pz[H.o1off + 1] : 0.f);
    }
  }
  float2 vv[PP];
  float4 pvv[PP];
#pragma unroll
  for (int r = 0; r < PP; ++r) {
    vv[r] = make_float2(0.f, 0.f);
    pvv[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!H.valid[r]) continue;
    const int t0 = H.t0[r];
    vv[r] = make_float2(H.vf[t0], H.v1[r] ? H.vf[t0 + 1] : 0.f);
    if (H.use_prev) {
      const float *pp = H.yprev + t0;
      pvv[r] = make_float4(pp[0], pp[H.o1off], H.v1[r] ? pp[1] : 0.f, H.v1[r] ? pp[H.o1off + 1] : 0.f);
    }
  }
  __syncthreads();
  int2 pre[2];
  if (ALLREC) {
    // every plane's records at once (sk2 is set): entry t of the fragment -> slot t
    const int ne = m.rb[H.Ez * H.Ey];
    for (int t = threadIdx.x; t < ne; t += NT) pair_record(t, H.ent[t], m.sk2, H.pitch2, m.rec, m.recky);
    pre[0] = pre[1] = make_int2(0, 0);
    __syncthreads();
  } else {
    pair_prefetch<NT>(H.ent, m.rb[H.Ey], pre);
  }

  float2 dot = f2(0.f, 0.f);
  const int maxent = a.maxent;
  for (int z0 = 0; z0 < H.Ez; z0 += 9) {
    hpair_plane<NT, PP, ISO, ALLREC, 0>(H, K, m, maxent, q, vv, pvv, pre, dot, z0, 0);
    if (z0 + 1 >= H.Ez) break;
    hpair_plane<NT, PP, ISO, ALLREC, 1>(H, K, m, maxent, q, vv, pvv, pre, dot, z0 + 1, 1);
    if (z0 + 2 >= H.Ez) break;
    hpair_plane<NT, PP, ISO, ALLREC, 2>(H, K, m, maxent, q, vv, pvv, pre, dot, z0 + 2, 2);
    if (z0 + 3 >= H.Ez) break;
    hpair_plane<NT, PP, ISO, ALLREC, 3>(H, K, m, maxent, q, vv, pvv, pre, dot, z0 + 3, 0);
    if (z0 + 4 >= H.Ez) break;
    hpair_plane<NT, PP, ISO, ALLREC, 4>(H, K, m, maxent, q, vv, pvv, pre, dot, z0 + 4, 1);
    if (z0 + 5 >= H.Ez) break;
    hpair_plane<NT, PP, ISO, ALLREC, 5>(H, K, m, maxent, q, vv, pvv, pre, dot, z0 + 5, 2);
    if (z0 + 6 >= H.Ez) break;
    hpair_plane<NT, PP, ISO, ALLREC, 6>(H, K, m, maxent, q, vv, pvv, pre, dot, z0 + 6, 0);
    if (z0 + 7 >= H.Ez) break;
    hpair_plane<NT, PP, ISO, ALLREC, 7>(H, K, m, maxent, q, vv, pvv, pre, dot, z0 + 7, 1);
    if (z0 + 8 >= H.Ez) break;
    hpair_plane<NT, PP, ISO, ALLREC, 8>(H, K, m, maxent, q, vv, pvv, pre, dot, z0 + 8, 2);
  }
  if (H.proj) {
    __syncthreads();
    const int zp = H.Ez - 1;
    const int zb = m.rb[zp * H.Ey];
    if (ALLREC) {
      pair_project<NT>(m.pout + (zp & 1) * H.Ey * H.pitch2, m.rec + zb, m.recky + zb, m.rb[(zp + 1) * H.Ey] - zb, m,
                       H.pitch2, H.A);
    } else {
      const int bp = zp % 3;
      pair_project<NT>(m.pout + (zp & 1) * H.Ey * H.pitch2, m.rec + bp * maxent, m.recky + bp * maxent,
                       m.rb[(zp + 1) * H.Ey] - zb, m, H.pitch2, H.A);
    }
    __syncthreads();
    pair_finish<NT>(a, D, m, i0, H.nvalid);
  }
  if (a.mode == HSTEP_ADJ) {
    for (int o = 16; o > 0; o >>= 1) {
      dot.x += __shfl_xor_sync(0xffffffffu, dot.x, o);
      dot.y += __shfl_xor_sync(0xffffffffu, dot.y, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
      m.red[w] = dot.x;
      m.red[NT / 32 + w] = dot.y;
    }
    __syncthreads();
    if (threadIdx.x < H.nvalid) {
      float sum = 0.f;
      for (int i = 0; i < NT / 32; ++i) sum += m.red[threadIdx.x * (NT / 32) + i];
      const int st = D.st_off + i0 + threadIdx.x;
      a.dots[st] = a.occ[st] * a.dV * (double)sum;
    }
  }
}

// Projections of an orbital block (no stencil), orbital pairs interleaved like k_hpair: plane z of
// both orbitals is staged in shared memory while the row-list tasks of plane z-1 run.
template <int NT>
__global__ void __launch_bounds__(NT) k_project_pair(HArgs<float> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 fi = a.items[blockIdx.x];
  const int f = fi.x, i0 = fi.y;
  const FragDesc D = a.desc[f];
  const int nvalid = min(2, D.norb - i0);
  const int Ex = D.E[0], Ey = D.E[1], Ez = D.E[2];
  const int plane = Ex * Ey;
  const int pitch2 = (Ex + 1) & ~1;
  const int A = D.natom;
  const long long P = (long long)plane * Ez;
  const PairSmem m = pair_carve(smem_raw, Ex, Ey, Ez, A, a.maxent, 2, false);
  pair_setup<NT>(a, D, m, i0, nvalid, 1.f);
  const long long base = D.psi_off + (long long)i0 * P;
  const long long o1off = nvalid > 1 ? P : 0;
  const int2 *ent = a.row_ent + a.row_beg[D.row_off];
  const float *y0 = a.yin + base;
  // sk2 is zero here (no input projections): only the (slot|row, weight) part of a record is used
  __syncthreads();
  int2 pre[2];
  pair_prefetch<NT>(ent, m.rb[Ey], pre);
  for (int z = 0; z < Ez; ++z) {
    float2 *pl = m.pout + (z & 1) * Ey * pitch2;
    for (int t = threadIdx.x; t < plane; t += NT) {
      const int y = t / Ex, x = t - y * Ex;
      const float *p = y0 + (long long)z * plane + t;
      pl[y * pitch2 + x] = f2(p[0], p[o1off]);
    }
    const int e0 = m.rb[z * Ey];
    pair_records<NT>(ent + e0, m.rb[(z + 1) * Ey] - e0, pre, m.sk2, pitch2, m.rec + (z & 1) * a.maxent,
                     m.recky + (z & 1) * a.maxent);
    if (z + 1 < Ez) pair_prefetch<NT>(ent + m.rb[(z + 1) * Ey], m.rb[(z + 2) * Ey] - m.rb[(z + 1) * Ey], pre);
    __syncthreads();
    pair_project<NT>(pl, m.rec + (z & 1) * a.maxent, m.recky + (z & 1) * a.maxent, m.rb[(z + 1) * Ey] - e0, m,
                     pitch2, A);
  }
  __syncthreads();
  pair_finish<NT>(a, D, m, i0, nvalid);
}

template <typename T>
const T *tab_of(dc_ctx *c);
template <>
const double *tab_of<double>(dc_ctx *c) { return c->d_tab64; }
template <>
const float *tab_of<float>(dc_ctx *c) { return c->d_tab32; }
template <typename T>
const T *vf_of(dc_ctx *c);
template <>
const double *vf_of<double>(dc_ctx *c) { return c->d_vf64; }
template <>
const float *vf_of<float>(dc_ctx *c) { return c->d_vf32; }

template <typename T>
HArgs<T> make_args(dc_ctx *c) {
  HArgs<T> a{};
  a.desc = c->d_desc;
  a.items = c->d_items + c->st_lo;  // the states of the context's fragment shard
  a.slots = c->d_slots;
  a.tab = tab_of<T>(c);
  a.zl_beg = c->d_zl_beg;
  a.zl_items = c->d_zl_items;
  a.row_beg = c->d_row_beg;
  a.row_ent = c->d_row_ent;
  a.maxent = c->max_plane_ent;
  a.vf = vf_of<T>(c);
  a.Datom = c->d_atom_D;
  a.bounds = c->d_bounds;
  a.bstride = 4 + 2 * c->params.cheb_degree;
  a.periodic = c->frag_cfg.bc == DC_BC_PERIODIC;
  a.dV = c->dV;
  // 8th-order central second-derivative weights (exact rationals), scaled by -1/2 h^-2
  const double fd[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
  for (int n = 0; n < 5; ++n) {
    a.kx[n] = T(-0.5 * fd[n] / (c->h[0] * c->h[0]));
    a.ky[n] = T(-0.5 * fd[n] / (c->h[1] * c->h[1]));
    a.kz[n] = T(-0.5 * fd[n] / (c->h[2] * c->h[2]));
  }
  return a;
}

int max_tabw(const dc_ctx *c) {
  int w = 0;
  for (const auto &D : c->h_desc) w = w > tab_width(D) ? w : tab_width(D);
  return w;
}

size_t hstep_smem(dc_ctx *c, size_t esz, int NT, int NO) {
  const int Ex = c->max_E[0], Ey = c->max_E[1], Ez = c->max_E[2];
  const int A = c->max_atoms;
  const int pitch = (Ex + 9) & ~1;
  size_t n = 2 * (size_t)NO * pitch * (Ey + 8) + (size_t)A * max_tabw(c) + 2 * (size_t)NO * Ex * Ey +
             (size_t)NO * Ey * A + (size_t)NO * A + NT / 32;
  size_t bytes = (n * esz + 15) & ~(size_t)15;
  const size_t rue = 2 * esz * NO;  // one record: NO splatted pairs
  bytes += sizeof(int4) * (size_t)A + rue * 2 * (size_t)Ey * A + sizeof(int) * 2 * (size_t)Ey * A +
           sizeof(int) * 2 * (size_t)Ey + sizeof(int) * (size_t)(Ez + 1) + sizeof(int) * (size_t)c->max_zlist;
  return bytes + 64;
}

size_t project_smem(dc_ctx *c, size_t esz) {
  const int Ex = c->max_E[0], Ey = c->max_E[1], Ez = c->max_E[2];
  const int A = c->max_atoms;
  size_t n = 2 * (size_t)Ex * Ey + (size_t)A * max_tabw(c) + (size_t)Ey * A;
  size_t bytes = ((n * esz) + 15) & ~(size_t)15;
  bytes += sizeof(int4) * (size_t)A + sizeof(int) * 2 * (size_t)Ey * A + sizeof(int) * 2 * (size_t)Ey +
           sizeof(int) * (size_t)(Ez + 1) + sizeof(int) * (size_t)c->max_zlist;
  return bytes + 64;
}

template <typename T, int NT, int PP, int NO>
int run_hstep(dc_ctx *c, HArgs<T> a, cudaStream_t s) {
  const size_t sm = hstep_smem(c, sizeof(T), NT, NO);
  if (sm > 227 * 1024) {
    dc_set_error("hpsi: fragment tables exceed shared memory");
    return DC_ERR_ARG;
  }
  DC_CUDA(dc_set_smem((const void *)k_hstep<T, NT, PP, NO>, sm));
  if (NO == 2) a.items = c->d_items2;
  const unsigned grid = NO == 2 ? (unsigned)c->n_items2 : (unsigned)(c->st_hi - c->st_lo);
  if (grid == 0) return DC_OK;
  k_hstep<T, NT, PP, NO><<<grid, NT, sm, s>>>(a);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

// Launch shapes of the stencil kernels: kind 0 = x-adjacent point pairs of one orbital (NO orbitals
// per CTA), kind 1 = orbital-pair kernel (FP32 only), kind 2 = the orbital-pair kernel with its
// registers capped for three 256-thread CTAs per SM, kind 3 = the orbital-pair kernel with every
// plane's projector records built once per CTA (when a fragment's records fit in shared memory);
// threads per CTA; point pairs per thread.
struct Shape {
  int kind, nt, pp;
};
constexpr Shape kShapes[] = {{0, 128, 1}, {0, 128, 2}, {0, 256, 1}, {0, 256, 2}, {0, 512, 1},
                             {0, 512, 2}, {0, 512, 4}, {1, 128, 1}, {1, 256, 1}, {1, 512, 1},
                             {1, 1024, 1}, {1, 256, 2}, {1, 512, 2}, {2, 128, 1}, {2, 256, 1}, {3, 256, 1},
                             {4, 256, 1}, {4, 512, 1}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);
static_assert(kNumShapes <= DC_TUNE_SLOTS, "tuning slots");

size_t hpair_smem(const dc_ctx *c, int NT, int PP, bool allrec = false) {
  if (allrec)
    return pair_smem_bytes(c->max_E[0], c->max_E[1], c->max_E[2], c->max_atoms, std::max(1, c->max_frag_ent), 1,
                           true, NT, PP);
  return pair_smem_bytes(c->max_E[0], c->max_E[1], c->max_E[2], c->max_atoms, std::max(1, c->max_plane_ent), 3,
                         true, NT, PP);
}
size_t project_pair_smem(const dc_ctx *c) {
  return pair_smem_bytes(c->max_E[0], c->max_E[1], c->max_E[2], c->max_atoms, std::max(1, c->max_plane_ent), 2,
                         false, 256);
}

// The three axes share one set of coefficients when their FP32 values agree (cubic spacing).
bool iso_coeffs(const HArgs<float> &a) {
  for (int n = 1; n < 5; ++n)
    if (a.kx[n] != a.ky[n] || a.kx[n] != a.kz[n]) return false;
  return true;
}

// MINB: CTAs per SM the register budget is cut for (launch bounds); the default keeps two
// 256-thread CTAs per SM, the register-capped variant three.
template <int NT, int PP, int MINB = ((PP == 1 && NT <= 256) ? 512 / NT : 1), bool ALLREC = false>
int run_hpair(dc_ctx *c, HArgs<float> a, cudaStream_t s) {
  const size_t sm = hpair_smem(c, NT, PP, ALLREC);
  if (sm > 227 * 1024) {
    dc_set_error("hpsi: fragment tables exceed shared memory (orbital-pair kernel)");
    return DC_ERR_ARG;
  }
  a.items = c->d_items2;
  a.maxent = std::max(1, ALLREC ? c->max_frag_ent : c->max_plane_ent);
  if (iso_coeffs(a)) {
    DC_CUDA(dc_set_smem((const void *)k_hpair<NT, PP, true, MINB, ALLREC>, sm));
    k_hpair<NT, PP, true, MINB, ALLREC><<<(unsigned)c->n_items2, NT, sm, s>>>(a);
  } else {
    DC_CUDA(dc_set_smem((const void *)k_hpair<NT, PP, false, MINB, ALLREC>, sm));
    k_hpair<NT, PP, false, MINB, ALLREC><<<(unsigned)c->n_items2, NT, sm, s>>>(a);
  }
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

// FP32 row-pair kernels run two orbitals per CTA; FP64 one (its pairs of doubles would not fit in
// registers twice).  The orbital-pair kernel exists for FP32 only.
template <typename T>
int run_shape(dc_ctx *c, int shape, HArgs<T> a, cudaStream_t s);
template <>
int run_shape<double>(dc_ctx *c, int shape, HArgs<double> a, cudaStream_t s) {
  switch (shape) {
    case 0: return run_hstep<double, 128, 1, 1>(c, a, s);
    case 1: return run_hstep<double, 128, 2, 1>(c, a, s);
    case 2: return run_hstep<double, 256, 1, 1>(c, a, s);
    case 3: return run_hstep<double, 256, 2, 1>(c, a, s);
    case 4: return run_hstep<double, 512, 1, 1>(c, a, s);
    case 5: return run_hstep<double, 512, 2, 1>(c, a, s);
    case 6: return run_hstep<double, 512, 4, 1>(c, a, s);
    default: dc_set_error("hpsi: no such FP64 launch shape"); return DC_ERR_ARG;
  }
}
template <>
int run_shape<float>(dc_ctx *c, int shape, HArgs<float> a, cudaStream_t s) {
  switch (shape) {
    case 0: return run_hstep<float, 128, 1, 2>(c, a, s);
    case 1: return run_hstep<float, 128, 2, 2>(c, a, s);
    case 2: return run_hstep<float, 256, 1, 2>(c, a, s);
    case 3: return run_hstep<float, 256, 2, 2>(c, a, s);
    case 4: return run_hstep<float, 512, 1, 2>(c, a, s);
    case 5: return run_hstep<float, 512, 2, 2>(c, a, s);
    case 6: return run_hstep<float, 512, 4, 2>(c, a, s);
    case 7: return run_hpair<128, 1>(c, a, s);
    case 8: return run_hpair<256, 1>(c, a, s);
    case 9: return run_hpair<512, 1>(c, a, s);
    case 10: return run_hpair<1024, 1>(c, a, s);
    case 11: return run_hpair<256, 2>(c, a, s);
    case 12: return run_hpair<512, 2>(c, a, s);
    case 13: return run_hpair<128, 1, 6>(c, a, s);
    case 14: return run_hpair<256, 1, 3>(c, a, s);
    case 15: return run_hpair<256, 1, 2, true>(c, a, s);
    default:
      return dck::launch_cheb(c, a.mode, a.step, a.yin, a.yprev, a.yout, a.cin, a.cout, s);
  }
}

// A shape is valid when one CTA covers every x-pair of the largest plane and its shared memory
// fits, and useful when it does not leave more than three quarters of its threads idle.
bool shape_ok(const dc_ctx *c, int shape, size_t esz) {
  if (shape < 0 || shape >= kNumShapes) return false;
  const Shape S = kShapes[shape];
  if (S.kind == 4) {
    // the specialised kernel: one CTA of 256 threads for extents up to 22, 512 for 32
    const int E = esz == sizeof(float) ? dck::cheb_extent(c) : 0;
    return E > 0 && S.nt == (E <= 22 ? 256 : 512);
  }
  if (S.kind >= 1 && (esz != sizeof(float) || hpair_smem(c, S.nt, S.pp, S.kind == 3) > 227 * 1024)) return false;
  const int pairs = ((c->max_E[0] + 1) / 2) * c->max_E[1];
  const int cover = S.nt * S.pp;
  return cover >= pairs && (cover <= 4 * pairs || S.nt == 128);
}

int default_shape(const dc_ctx *c, size_t esz) {
  if (esz == sizeof(float))
    for (int k : {7, 8, 11, 9, 12, 10})
      if (shape_ok(c, k, esz)) return k;
  for (int k : {0, 2, 3, 5, 6})
    if (shape_ok(c, k, esz)) return k;
  return 6;
}

}  // namespace

namespace dck {

template <typename T>
int launch_hstep(dc_ctx *c, int mode, int step, const T *yin, const T *yprev, T *yout, const T *cin, T *cout,
                 const double *Datom, const double *occ, double *dots, const T *vf, cudaStream_t s) {
  HArgs<T> a = make_args<T>(c);
  if (vf) a.vf = vf;
  a.mode = mode;
  a.step = step;
  a.yin = yin;
  a.yprev = yprev;
  a.yout = yout;
  a.cin = cin;
  a.cout = cout;
  if (Datom) a.Datom = Datom;
  a.occ = occ;
  a.dots = dots;
  int shape = c->hstep_shape[sizeof(T) == 8 ? 1 : 0];
  if (!shape_ok(c, shape, sizeof(T))) shape = default_shape(c, sizeof(T));
  // the specialised kernel takes Chebyshev steps and plain H-applies with input projections; the
  // adjoint (and any call without projections) runs the general kernel's default shape
  if (kShapes[shape].kind == 4 && ((mode != HSTEP_CHEB && mode != HSTEP_HPSI && mode != HSTEP_HLOC) || !cin || !yout))
    shape = default_shape(c, sizeof(T));
  if (mode == HSTEP_HLOC && kShapes[shape].kind != 4) {
    dc_set_error("hpsi: the local part of H alone runs only in the specialised kernel");
    return DC_ERR_ARG;
  }
  return run_shape<T>(c, shape, a, s);
}

bool hstep_specialised(const dc_ctx *c) {
  int shape = c->hstep_shape[0];
  if (!shape_ok(c, shape, sizeof(float))) shape = default_shape(c, sizeof(float));
  return kShapes[shape].kind == 4;
}

// Time every useful launch shape on the context's fragments (H applied to `y`, written to `out`,
// projections in `cbuf`), best of three repetitions each, and keep the fastest for this element type.
template <typename T>
int tune_hstep(dc_ctx *c, const T *y, T *out, T *cbuf, cudaStream_t s) {
  HArgs<T> a = make_args<T>(c);
  a.mode = HSTEP_HPSI;
  a.yin = y;
  a.yout = out;
  a.cin = cbuf;
  cudaEvent_t e0, e1;
  DC_CUDA(cudaEventCreate(&e0));
  DC_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_shape = default_shape(c, sizeof(T));
  int st = DC_OK;
  for (int k = 0; k < kNumShapes && st == DC_OK; ++k) {
    if (!shape_ok(c, k, sizeof(T))) continue;
    st = run_shape<T>(c, k, a, s);  // warm-up and attribute set
    float tk = 1e30f;
    for (int r = 0; r < 3 && st == DC_OK; ++r) {
      cudaEventRecord(e0, s);
      st = run_shape<T>(c, k, a, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = DC_ERR_CUDA;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      tk = t < tk ? t : tk;
    }
    c->tune_ms[sizeof(T) == 8 ? 1 : 0][k] = tk;
    if (st == DC_OK && tk < best) {
      best = tk;
      best_shape = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DC_OK) return st;
  c->hstep_shape[sizeof(T) == 8 ? 1 : 0] = best_shape;
  return DC_OK;
}

int hstep_shape_find(const dc_ctx *c, size_t esz, int kind, int threads, int pairs) {
  for (int k = 0; k < kNumShapes; ++k)
    if (kShapes[k].kind == kind && kShapes[k].nt == threads && kShapes[k].pp == pairs)
      return shape_ok(c, k, esz) ? k : -1;
  return -1;
}

int hstep_shape_info(int shape, int *kind, int *threads, int *pairs) {
  if (shape < 0 || shape >= kNumShapes) return DC_ERR_ARG;
  *kind = kShapes[shape].kind;
  *threads = kShapes[shape].nt;
  *pairs = kShapes[shape].pp;
  return DC_OK;
}

template <typename T>
int launch_project(dc_ctx *c, const T *psi, T *cout, cudaStream_t s) {
  HArgs<T> a = make_args<T>(c);
  a.yin = psi;
  a.cout = cout;
  if constexpr (std::is_same<T, float>::value) {
    if (project_pair_smem(c) <= 227 * 1024) {
      a.items = c->d_items2;
      a.maxent = std::max(1, c->max_plane_ent);
      const size_t sm = project_pair_smem(c);
      DC_CUDA(dc_set_smem((const void *)k_project_pair<256>, sm));
      k_project_pair<256><<<(unsigned)c->n_items2, 256, sm, s>>>(a);
      DC_CUDA(cudaGetLastError());
      return DC_OK;
    }
  }
  const size_t sm = project_smem(c, sizeof(T));
  DC_CUDA(dc_set_smem((const void *)k_project<T, 256>, sm));
  if (c->st_hi <= c->st_lo) return DC_OK;
  k_project<T, 256><<<(unsigned)(c->st_hi - c->st_lo), 256, sm, s>>>(a);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

template int tune_hstep<double>(dc_ctx *, const double *, double *, double *, cudaStream_t);
template int tune_hstep<float>(dc_ctx *, const float *, float *, float *, cudaStream_t);
template int launch_hstep<double>(dc_ctx *, int, int, const double *, const double *, double *, const double *,
                                  double *, const double *, const double *, double *, const double *, cudaStream_t);
template int launch_hstep<float>(dc_ctx *, int, int, const float *, const float *, float *, const float *, float *,
                                 const double *, const double *, double *, const float *, cudaStream_t);
template int launch_project<double>(dc_ctx *, const double *, double *, cudaStream_t);
template int launch_project<float>(dc_ctx *, const float *, float *, cudaStream_t);

}  // namespace dck
