// Fragment Hamiltonian kernels (Eq. 5, model Hamiltonian) for sm_103a.
//
// H_f y = -1/2 L8 y + V_f y + sum_a D_a p_a <p_a|y>, <u|v> = dV sum u v, with the 8th-order
// 25-point Laplacian and ghost points that are zero (buffer edge) or wrap within the fragment.
// The projectors are separable, p_a(j) = C_a gx_a[jx] gy_a[jy] gz_a[jz].
//
// One CTA handles one (fragment, orbital) item and streams the fragment along z: every thread
// owns PPT points of the xy-plane and keeps their 9-deep z column in registers; the current plane
// sits in shared memory with a 4-point halo (zeros, or wrapped values for the periodic boundary)
// so the x and y taps need no bounds tests.  The nonlocal term uses the projections of the input
// (computed beforehand) and per-plane coefficients; the projections of the output, which the next
// Chebyshev step needs, are accumulated plane by plane in the epilogue by one warp per atom, in a
// fixed order (deterministic).
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
  T k0;      // -1/2 c0 sum_d 1/h_d^2
  T kx[5], ky[5], kz[5];  // -1/2 c_n / h_d^2
};

template <typename T>
__device__ __forceinline__ T ldz(const T *base, int zz, int Ez, int plane, int t, bool valid, int periodic) {
  if (!valid) return T(0);
  if (zz < 0 || zz >= Ez) {
    if (!periodic) return T(0);
    zz = zz < 0 ? zz + Ez : zz - Ez;
  }
  return base[(long long)zz * plane + t];
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

// Projection of one plane (values in `pl`, row pitch Ex) onto every atom of the plane's list;
// accumulates gz[k][z] * sum_y gy[k][y] sum_x gx[k][x] pl[y][x] into acc[k].  Atom slot k is
// always handled by warp k % nwarps, so the summation order is fixed.
template <typename T, int NT>
__device__ __forceinline__ void project_plane(const T *pl, int z, int Ex, int Ey, const T *stab, int tabw,
                                              const int *zl_b, const int *zl_i, const int4 *box, T *acc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int beg = zl_b[z], end = zl_b[z + 1];
  for (int e = beg; e < end; ++e) {
    const int k = zl_i[e];
    if ((k % (NT / 32)) != warp) continue;
    const T *gx = stab + k * tabw;
    const T *gy = gx + Ex;
    const T *gz = gy + Ey;
    const int4 bx = box[k];  // x lo, x hi, y lo, y hi
    T s = T(0);
    for (int y = bx.z + lane; y < bx.w; y += 32) {
      T r = T(0);
      const T *row = pl + y * Ex;
      for (int x = bx.x; x < bx.y; ++x) r += gx[x] * row[x];
      s += gy[y] * r;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) acc[k] += gz[z] * s;
  }
}

template <typename T, int NT, int PPT>
__global__ void __launch_bounds__(NT) k_hstep(HArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int item = blockIdx.x;
  const int2 fi = a.items[item];
  const int f = fi.x, i = fi.y;
  const FragDesc D = a.desc[f];
  const int Ex = D.E[0], Ey = D.E[1], Ez = D.E[2];
  const int plane = Ex * Ey;
  const int pitch = Ex + 8;
  const int pplane = pitch * (Ey + 8);
  const long long P = (long long)plane * Ez;
  const int A = D.natom;
  const int tabw = Ex + Ey + Ez;

  // shared memory carve-up
  T *sp = reinterpret_cast<T *>(smem_raw);
  T *pin = sp;                      // [2][pplane]
  T *pout = pin + 2 * pplane;       // [2][plane]
  T *stab = pout + 2 * plane;       // [A][tabw]
  T *sk = stab + A * tabw;          // [A] apply strengths
  T *acc = sk + A;                  // [A] output projections
  T *tz = acc + A;                  // [2][A] per-plane coefficients
  T *red = tz + 2 * A;              // [NT/32]
  size_t ioff = (size_t)(2 * pplane + 2 * plane + A * tabw + 4 * A + NT / 32) * sizeof(T);
  ioff = (ioff + 15) & ~(size_t)15;
  int *zl_b = reinterpret_cast<int *>(smem_raw + ioff);  // [Ez+1], 16-byte aligned
  int4 *box = reinterpret_cast<int4 *>(zl_b + ((Ez + 1 + 3) & ~3));  // [A]
  int *zl_i = reinterpret_cast<int *>(box + A);        // [list]

  const int zb0 = a.zl_beg[D.zl_off];
  const int nzl = a.zl_beg[D.zl_off + Ez] - zb0;
  for (int t = threadIdx.x; t < A * tabw; t += NT) stab[t] = a.tab[D.tab_off + t];
  for (int t = threadIdx.x; t <= Ez; t += NT) zl_b[t] = a.zl_beg[D.zl_off + t] - zb0;
  for (int t = threadIdx.x; t < nzl; t += NT) zl_i[t] = a.zl_items[zb0 + t];
  for (int k = threadIdx.x; k < A; k += NT) {
    const ProjSlot S = a.slots[D.at_off + k];
    box[k] = make_int4(S.lo[0], S.hi[0], S.lo[1], S.hi[1]);
    sk[k] = a.cin ? T(a.Datom[S.atom] * S.coef) * a.cin[D.c_off + (long long)i * A + k] : T(0);
    acc[k] = T(0);
  }
  for (int t = threadIdx.x; t < 2 * pplane; t += NT) pin[t] = T(0);

  T alpha = T(1), beta = T(0), shift = T(0);
  if (a.mode == HSTEP_CHEB) {
    const double *bd = a.bounds + (long long)f * a.bstride;
    shift = T(bd[3]);
    alpha = T(bd[4 + 2 * a.step]);
    beta = T(bd[5 + 2 * a.step]);
  }
  const bool use_prev = (a.mode == HSTEP_CHEB) && a.yprev != nullptr && a.step > 0;
  const T *yin = a.yin + D.psi_off + (long long)i * P;
  const T *ypv = use_prev ? a.yprev + D.psi_off + (long long)i * P : nullptr;
  T *yout = a.yout ? a.yout + D.psi_off + (long long)i * P : nullptr;
  const T *vf = a.vf + D.pt_off;

  int px[PPT], py[PPT];
  bool valid[PPT];
  T q[PPT][9];
#pragma unroll
  for (int r = 0; r < PPT; ++r) {
    const int t = threadIdx.x + r * NT;
    valid[r] = t < plane;
    py[r] = valid[r] ? t / Ex : 0;
    px[r] = valid[r] ? t - py[r] * Ex : 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) q[r][k] = ldz(yin, k - 4, Ez, plane, t, valid[r], a.periodic);
  }
  __syncthreads();

  T dot = T(0);
  for (int z = 0; z < Ez; ++z) {
    const int buf = z & 1;
    T *P0 = pin + buf * pplane;
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
      if (!valid[r]) continue;
      const int x = px[r], y = py[r];
      const T v = q[r][4];
      P0[(y + 4) * pitch + x + 4] = v;
      if (a.periodic) {
        if (x < 4) P0[(y + 4) * pitch + x + Ex + 4] = v;
        if (x >= Ex - 4) P0[(y + 4) * pitch + x - Ex + 4] = v;
        if (y < 4) P0[(y + Ey + 4) * pitch + x + 4] = v;
        if (y >= Ey - 4) P0[(y - Ey + 4) * pitch + x + 4] = v;
      }
    }
    const int zbeg = zl_b[z], zend = zl_b[z + 1];
    T *tzb = tz + buf * A;
    for (int e = zbeg + threadIdx.x; e < zend; e += NT) {
      const int k = zl_i[e];
      tzb[e - zbeg] = sk[k] * stab[k * tabw + Ex + Ey + z];
    }
    __syncthreads();
    if (a.cout && z > 0)
      project_plane<T, NT>(pout + ((z - 1) & 1) * plane, z - 1, Ex, Ey, stab, tabw, zl_b, zl_i, box, acc);

#pragma unroll
    for (int r = 0; r < PPT; ++r) {
      if (!valid[r]) continue;
      const int x = px[r], y = py[r];
      const int t = x + y * Ex;
      const T *c0 = P0 + (y + 4) * pitch + x + 4;
      const T cv = q[r][4];
      T hy = a.k0 * cv;
#pragma unroll
      for (int n = 1; n <= 4; ++n) {
        hy += a.kz[n] * (q[r][4 + n] + q[r][4 - n]);
        hy += a.ky[n] * (c0[n * pitch] + c0[-n * pitch]);
        hy += a.kx[n] * (c0[n] + c0[-n]);
      }
      hy += vf[(long long)z * plane + t] * cv;
      T nl = T(0);
      for (int e = zbeg; e < zend; ++e) {
        const int k = zl_i[e];
        const T *g = stab + k * tabw;
        nl += tzb[e - zbeg] * (g[Ex + y] * g[x]);
      }
      hy += nl;
      T out;
      if (a.mode == HSTEP_CHEB) {
        out = alpha * (hy - shift * cv);
        if (use_prev) out += beta * ypv[(long long)z * plane + t];
      } else if (a.mode == HSTEP_ADJ) {
        dot += cv * hy;
        out = T(2.0 * a.occ[D.st_off + i] * a.dV) * hy;
      } else {
        out = hy;
      }
      if (yout) yout[(long long)z * plane + t] = out;
      if (a.cout) pout[buf * plane + t] = out;
    }
    // advance the z column
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
#pragma unroll
      for (int k = 0; k < 8; ++k) q[r][k] = q[r][k + 1];
      q[r][8] = ldz(yin, z + 5, Ez, plane, threadIdx.x + r * NT, valid[r], a.periodic);
    }
  }
  if (a.cout) {
    __syncthreads();
    project_plane<T, NT>(pout + ((Ez - 1) & 1) * plane, Ez - 1, Ex, Ey, stab, tabw, zl_b, zl_i, box, acc);
    __syncthreads();
    for (int k = threadIdx.x; k < A; k += NT) {
      const ProjSlot S = a.slots[D.at_off + k];
      a.cout[D.c_off + (long long)i * A + k] = T(S.coef * a.dV) * acc[k];
    }
  }
  if (a.mode == HSTEP_ADJ) {
    const T s = block_sum<T, NT>(dot, red);
    if (threadIdx.x == 0) a.dots[item] = a.occ[D.st_off + i] * a.dV * (double)s;
  }
}

// Projections c[k] = C_k dV sum_j p_k(j) y(j) of one orbital block (no stencil).
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
  const int tabw = Ex + Ey + Ez;
  T *sp = reinterpret_cast<T *>(smem_raw);
  T *pl = sp;                 // [2][plane]
  T *stab = pl + 2 * plane;   // [A][tabw]
  T *acc = stab + A * tabw;   // [A]
  size_t ioff = (size_t)(2 * plane + A * tabw + A) * sizeof(T);
  ioff = (ioff + 15) & ~(size_t)15;
  int *zl_b = reinterpret_cast<int *>(smem_raw + ioff);
  int4 *box = reinterpret_cast<int4 *>(zl_b + ((Ez + 1 + 3) & ~3));
  int *zl_i = reinterpret_cast<int *>(box + A);
  const int zb0 = a.zl_beg[D.zl_off];
  const int nzl = a.zl_beg[D.zl_off + Ez] - zb0;
  for (int t = threadIdx.x; t < A * tabw; t += NT) stab[t] = a.tab[D.tab_off + t];
  for (int t = threadIdx.x; t <= Ez; t += NT) zl_b[t] = a.zl_beg[D.zl_off + t] - zb0;
  for (int t = threadIdx.x; t < nzl; t += NT) zl_i[t] = a.zl_items[zb0 + t];
  for (int k = threadIdx.x; k < A; k += NT) {
    const ProjSlot S = a.slots[D.at_off + k];
    box[k] = make_int4(S.lo[0], S.hi[0], S.lo[1], S.hi[1]);
    acc[k] = T(0);
  }
  const T *yin = a.yin + D.psi_off + (long long)i * P;
  for (int z = 0; z < Ez; ++z) {
    T *cur = pl + (z & 1) * plane;
    for (int t = threadIdx.x; t < plane; t += NT) cur[t] = yin[(long long)z * plane + t];
    __syncthreads();
    project_plane<T, NT>(cur, z, Ex, Ey, stab, tabw, zl_b, zl_i, box, acc);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < A; k += NT) {
    const ProjSlot S = a.slots[D.at_off + k];
    a.cout[D.c_off + (long long)i * A + k] = T(S.coef * a.dV) * acc[k];
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
  double w[3];
  for (int d = 0; d < 3; ++d) w[d] = 1.0 / (c->h[d] * c->h[d]);
  a.k0 = T(-0.5 * fd[0] * (w[0] + w[1] + w[2]));
  for (int n = 0; n < 5; ++n) {
    a.kx[n] = T(-0.5 * fd[n] * w[0]);
    a.ky[n] = T(-0.5 * fd[n] * w[1]);
    a.kz[n] = T(-0.5 * fd[n] * w[2]);
  }
  return a;
}

size_t hstep_smem(dc_ctx *c, size_t esz, int NT) {
  const int Ex = c->max_E[0], Ey = c->max_E[1], Ez = c->max_E[2];
  const int A = c->max_atoms;
  size_t n = 2 * (size_t)(Ex + 8) * (Ey + 8) + 2 * (size_t)Ex * Ey + (size_t)A * (Ex + Ey + Ez) + 4 * (size_t)A + NT / 32;
  size_t bytes = n * esz;
  bytes = (bytes + 15) & ~(size_t)15;
  bytes += sizeof(int) * (size_t)((Ez + 1 + 3) & ~3) + sizeof(int4) * (size_t)A + sizeof(int) * (size_t)c->max_zlist;
  return bytes + 64;
}

size_t project_smem(dc_ctx *c, size_t esz) {
  const int Ex = c->max_E[0], Ey = c->max_E[1], Ez = c->max_E[2];
  const int A = c->max_atoms;
  size_t n = 2 * (size_t)Ex * Ey + (size_t)A * (Ex + Ey + Ez) + (size_t)A;
  size_t bytes = ((n * esz) + 15) & ~(size_t)15;
  bytes += sizeof(int) * (size_t)((Ez + 1 + 3) & ~3) + sizeof(int4) * (size_t)A + sizeof(int) * (size_t)c->max_zlist;
  return bytes + 64;
}

template <typename T, int NT, int PPT>
int run_hstep(dc_ctx *c, HArgs<T> a, cudaStream_t s) {
  const size_t sm = hstep_smem(c, sizeof(T), NT);
  if (sm > 227 * 1024) {
    dc_set_error("hpsi: fragment tables exceed shared memory");
    return DC_ERR_ARG;
  }
  DC_CUDA(cudaFuncSetAttribute(k_hstep<T, NT, PPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_hstep<T, NT, PPT><<<(unsigned)c->layout.nstates, NT, sm, s>>>(a);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
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
  const int plane = c->max_E[0] * c->max_E[1];
  if (plane <= 256) return run_hstep<T, 128, 2>(c, a, s);
  if (plane <= 512) return run_hstep<T, 256, 2>(c, a, s);
  if (plane <= 1024) return run_hstep<T, 512, 2>(c, a, s);
  return run_hstep<T, 512, 8>(c, a, s);
}

template <typename T>
int launch_project(dc_ctx *c, const T *psi, T *cout, cudaStream_t s) {
  HArgs<T> a = make_args<T>(c);
  a.yin = psi;
  a.cout = cout;
  const size_t sm = project_smem(c, sizeof(T));
  DC_CUDA(cudaFuncSetAttribute(k_project<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_project<T, 256><<<(unsigned)c->layout.nstates, 256, sm, s>>>(a);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

template int launch_hstep<double>(dc_ctx *, int, int, const double *, const double *, double *, const double *,
                                  double *, const double *, const double *, double *, const double *, cudaStream_t);
template int launch_hstep<float>(dc_ctx *, int, int, const float *, const float *, float *, const float *, float *,
                                 const double *, const double *, double *, const float *, cudaStream_t);
template int launch_project<double>(dc_ctx *, const double *, double *, cudaStream_t);
template int launch_project<float>(dc_ctx *, const float *, float *, cudaStream_t);

}  // namespace dck
