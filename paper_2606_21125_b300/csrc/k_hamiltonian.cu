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
        V h1 = Op::splat(T(0)), h2 = Op::splat(T(0));
        T xv[10];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          const V v = ld2(co - 4 + 2 * j);
          xv[2 * j] = v.x;
          xv[2 * j + 1] = v.y;
        }
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
        const V hv = Op::add(Op::add(hxy[o], hz[o]), hn[o]);
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
  a.items = c->d_items;
  a.slots = c->d_slots;
  a.tab = tab_of<T>(c);
  a.zl_beg = c->d_zl_beg;
  a.zl_items = c->d_zl_items;
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
  const unsigned grid = NO == 2 ? (unsigned)c->n_items2 : (unsigned)c->layout.nstates;
  k_hstep<T, NT, PP, NO><<<grid, NT, sm, s>>>(a);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

// Launch shapes of the stencil kernel: (threads per CTA, x-pairs per thread).
constexpr int kShapes[][2] = {{128, 1}, {128, 2}, {256, 1}, {256, 2}, {512, 1}, {512, 2}, {512, 4}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

// FP32 runs two orbitals per thread; FP64 one (its pairs of doubles would not fit in registers twice)
template <typename T>
int run_shape(dc_ctx *c, int shape, HArgs<T> a, cudaStream_t s) {
  constexpr int NO = sizeof(T) == 4 ? 2 : 1;
  switch (shape) {
    case 0: return run_hstep<T, 128, 1, NO>(c, a, s);
    case 1: return run_hstep<T, 128, 2, NO>(c, a, s);
    case 2: return run_hstep<T, 256, 1, NO>(c, a, s);
    case 3: return run_hstep<T, 256, 2, NO>(c, a, s);
    case 4: return run_hstep<T, 512, 1, NO>(c, a, s);
    case 5: return run_hstep<T, 512, 2, NO>(c, a, s);
    default: return run_hstep<T, 512, 4, NO>(c, a, s);
  }
}

// A shape is valid when one CTA covers every x-pair of the largest plane, and useful when it does
// not leave more than three quarters of its threads idle.
bool shape_ok(const dc_ctx *c, int shape) {
  const int pairs = ((c->max_E[0] + 1) / 2) * c->max_E[1];
  const int cover = kShapes[shape][0] * kShapes[shape][1];
  return cover >= pairs && (cover <= 4 * pairs || kShapes[shape][0] == 128);
}

int default_shape(const dc_ctx *c) {
  for (int k : {0, 2, 3, 5, 6})
    if (shape_ok(c, k)) return k;
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
  if (shape < 0 || !shape_ok(c, shape)) shape = default_shape(c);
  return run_shape<T>(c, shape, a, s);
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
  int best_shape = default_shape(c);
  int st = DC_OK;
  for (int k = 0; k < kNumShapes && st == DC_OK; ++k) {
    if (!shape_ok(c, k)) continue;
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

int hstep_shape_info(int shape, int *threads, int *pairs) {
  if (shape < 0 || shape >= kNumShapes) return DC_ERR_ARG;
  *threads = kShapes[shape][0];
  *pairs = kShapes[shape][1];
  return DC_OK;
}

template <typename T>
int launch_project(dc_ctx *c, const T *psi, T *cout, cudaStream_t s) {
  HArgs<T> a = make_args<T>(c);
  a.yin = psi;
  a.cout = cout;
  const size_t sm = project_smem(c, sizeof(T));
  DC_CUDA(dc_set_smem((const void *)k_project<T, 256>, sm));
  k_project<T, 256><<<(unsigned)c->layout.nstates, 256, sm, s>>>(a);
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
