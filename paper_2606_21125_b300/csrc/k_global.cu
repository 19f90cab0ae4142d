// Global-grid stages: ionic potential, Poisson + exchange (Eq. 5), potential gather with the
// fragments' spectral bounds, energies, mixing, starting orbitals and deterministic reductions.
#include <cuda_runtime.h>

#include "dc_internal.h"

namespace {

__device__ __forceinline__ int fft_freq(int g, int N) { return g < (N + 1) / 2 ? g : g - N; }

// G of grid index idx in a layout whose rows hold nxl x-entries: nxl = nx (full grid) or nx/2 + 1 (the
// half grid of a real-to-complex transform, x = 0 .. nx/2)
__device__ __forceinline__ double gsq(long long idx, int nxl, int nx, int ny, int nz, double Lx, double Ly, double Lz,
                                      double *gx, double *gy, double *gz) {
  const int x = (int)(idx % nxl);
  const int y = (int)((idx / nxl) % ny);
  const int z = (int)(idx / ((long long)nxl * ny));
  *gx = 2.0 * M_PI * fft_freq(x, nx) / Lx;
  *gy = 2.0 * M_PI * fft_freq(y, ny) / Ly;
  *gz = 2.0 * M_PI * fft_freq(z, nz) / Lz;
  return (*gx) * (*gx) + (*gy) * (*gy) + (*gz) * (*gz);
}

// rho_ion(G) = (1/Omega) sum_a Z_a exp(-G^2 sigma_a^2/2) exp(-i G.R_a)  (Gaussian ion charges)
__global__ void k_rho_ion_G(long long npts, int nxl, int nx, int ny, int nz, double Lx, double Ly, double Lz,
                            int natom, const double *pos, const int *species, const double *spec, int nspecies,
                            double volume, double2 *out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npts) return;
  double gx, gy, gz;
  const double g2 = gsq(idx, nxl, nx, ny, nz, Lx, Ly, Lz, &gx, &gy, &gz);
  double re = 0.0, im = 0.0;
  for (int a = 0; a < natom; ++a) {
    const int s = species[a];
    const double Z = spec[s], sig = spec[nspecies + s];
    const double amp = Z * exp(-0.5 * g2 * sig * sig);
    const double ph = gx * pos[3 * a] + gy * pos[3 * a + 1] + gz * pos[3 * a + 2];
    double sn, cs;
    sincos(ph, &sn, &cs);
    re += amp * cs;
    im -= amp * sn;
  }
  out[idx] = make_double2(re / volume, im / volume);
}

// The G-dependent factors of the per-step reciprocal-space stages on the half grid, fixed for a context:
// 1/G^2 (0 at G = 0) and the Kerker weight alpha G^2/(G^2 + q0^2), divided by N (the full grid's point
// count) for the unnormalised inverse transform.
__global__ void k_gtables(long long nh, int nx, int ny, int nz, double Lx, double Ly, double Lz, double alpha,
                          double q0sq, long long npts, double *ig2, double *kw) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nh) return;
  double gx, gy, gz;
  const double g2 = gsq(idx, nx / 2 + 1, nx, ny, nz, Lx, Ly, Lz, &gx, &gy, &gz);
  ig2[idx] = g2 > 0.0 ? 1.0 / g2 : 0.0;
  kw[idx] = alpha * g2 / (g2 + q0sq) / (double)npts;
}

// V_loc(G) = -4 pi rho_ion(G) / G^2 (0 at G = 0) on the full grid
__global__ void k_vloc_G(long long npts, int nx, int ny, int nz, double Lx, double Ly, double Lz, const double2 *in,
                         double2 *out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npts) return;
  double gx, gy, gz;
  const double g2 = gsq(idx, nx, nx, ny, nz, Lx, Ly, Lz, &gx, &gy, &gz);
  const double sc = g2 > 0.0 ? -4.0 * M_PI / g2 : 0.0;
  const double2 v = in[idx];
  out[idx] = make_double2(sc * v.x, sc * v.y);
}

__global__ void k_poisson_scale(long long npts, const double *ig2, const double2 *in, double factor, double2 *out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npts) return;
  const double2 v = in[idx];
  const double s = factor * ig2[idx];
  out[idx] = make_double2(s * v.x, s * v.y);
}

__global__ void k_cplx_real(long long n, const double2 *in, double scale, double *out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i].x * scale;
}

__global__ void k_clamp_pos(long long n, double *x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = fmax(x[i], 0.0);
}

__global__ void k_scale(long long n, double *x, const double *num, double den_scale) {
  // x *= num[0]... helper: x[i] *= ne / (dV * sum) with sum in num[0]
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= den_scale / num[0];
}

// V_eff = V_loc + V_H + v_x[rho]  (vh holds the unnormalised inverse transform, scaled by 1/N); with
// with_x = 0 the exchange is left to the per-fragment gather (Eq. 5, V_xc[rho_alpha])
__global__ void k_veff(long long n, const double *vion, const double *vh, double inv_n, const double *rho, int hxc,
                       int with_x, double *veff) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = vion[i];
  if (hxc == DC_HXC_HARTREE_X) {
    v += vh[i] * inv_n;
    if (with_x) v -= cbrt(3.0 * fmax(rho[i], 0.0) / M_PI);
  }
  veff[i] = v;
}

// Per-fragment potential gather and rigorous spectral upper bound of H_f:
//   b_up = max symbol of -1/2 L8 + max_j V_f(j) + sum_k max(D_k, 0) <p_k|p_k>.
// With rhof != nullptr (per-fragment exchange, Eq. 5): V_f(j) = V(g) + v_x(rho_alpha(j)) [+ (rho_alpha(j) -
// rho_in(g)) / xi for xi > 0], rho_alpha = 2 rhof (rhof holds sum_i f_i psi_i^2 over every fragment point).
__global__ void k_gather(const FragDesc *desc, const int32_t *idx_map, const double *veff, double *vf64, float *vf32,
                         const double *nl_bound, double kin_max, double *bounds, int bstride, const double *rhof,
                         const double *rho_in, double inv_xi) {
  __shared__ double red[8];
  const int f = blockIdx.x;
  const FragDesc D = desc[f];
  const long long P = (long long)D.E[0] * D.E[1] * D.E[2];
  double vmax = -1e300;
  for (long long j = threadIdx.x; j < P; j += blockDim.x) {
    const int32_t g = idx_map[D.pt_off + j];
    double v = veff[g];
    if (rhof) {
      const double ra = 2.0 * rhof[D.pt_off + j];
      v -= cbrt(3.0 * fmax(ra, 0.0) / M_PI);
      if (inv_xi > 0.0) v += (ra - rho_in[g]) * inv_xi;
    }
    vf64[D.pt_off + j] = v;
    if (vf32) vf32[D.pt_off + j] = (float)v;
    vmax = fmax(vmax, v);
  }
  for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    bounds[(long long)f * bstride + 1] = kin_max + m + nl_bound[f];
  }
}

__global__ void k_vcore(long long npts, const FragDesc *desc, const int32_t *owner, const int32_t *core_local,
                        const double *vf64, double *vcore) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npts) return;
  vcore[g] = vf64[desc[owner[g]].pt_off + core_local[g]];
}

__global__ void k_gather_plain(long long total, const int32_t *idx_map, const double *V, double *vf64, float *vf32) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const double v = V[idx_map[t]];
  if (vf64) vf64[t] = v;
  if (vf32) vf32[t] = (float)v;
}

// Starting orbitals: SplitMix64 of key = seed ^ ((f << 20 | i) << 32) ^ j, mapped to [-1, 1).
__global__ void k_init_psi(const FragDesc *desc, const int2 *items, unsigned long long seed, double *psi) {
  const int2 it = items[blockIdx.x];
  const FragDesc D = desc[it.x];
  const long long P = (long long)D.E[0] * D.E[1] * D.E[2];
  double *y = psi + D.psi_off + (long long)it.y * P;
  const unsigned long long hi = ((((unsigned long long)it.x) << 20) | (unsigned long long)it.y) << 32;
  for (long long j = threadIdx.x; j < P; j += blockDim.x) {
    unsigned long long z = (seed ^ hi ^ (unsigned long long)j) + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    y[j] = (double)(z >> 11) * 0x1.0p-52 - 1.0;
  }
}

__global__ void k_d2f(long long n, const double *a, float *b) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_f2d(long long n, const float *a, double *b) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

// ---- deterministic reductions: fixed partition into RB blocks, then one block in fixed order ----
constexpr int RB = 512;
constexpr int RNT = 256;

template <class Fn>
__global__ void __launch_bounds__(RNT) k_reduce(Fn fn, long long n, double *partials) {
  __shared__ double red[RNT / 32];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * RNT + threadIdx.x; i < n; i += (long long)gridDim.x * RNT) s += fn(i);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < RNT / 32; ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

__global__ void k_reduce_final(const double *partials, int np, double scale, double *out) {
  __shared__ double red[RNT / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += RNT) s += partials[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < RNT / 32; ++w) t += red[w];
    out[0] = t * scale;
  }
}

template <class Fn>
int reduce(Fn fn, long long n, double scale, double *out, double *partials, cudaStream_t s) {
  long long nb = (n + RNT - 1) / RNT;
  if (nb > RB) nb = RB;
  if (nb < 1) nb = 1;
  k_reduce<Fn><<<(unsigned)nb, RNT, 0, s>>>(fn, n, partials);
  k_reduce_final<<<1, RNT, 0, s>>>(partials, (int)nb, scale, out);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

struct FnSum {
  const double *x;
  __device__ double operator()(long long i) const { return x[i]; }
};
struct FnDot {
  const double *a, *b;
  __device__ double operator()(long long i) const { return a[i] * b[i]; }
};
struct FnAbsDiff {
  const double *a, *b;
  __device__ double operator()(long long i) const { return fabs(a[i] - b[i]); }
};
struct FnEx {
  const double *r;
  __device__ double operator()(long long i) const {
    const double v = fmax(r[i], 0.0);
    return v * cbrt(v);
  }
};
struct FnBand {
  const double *occ, *eps, *q;
  __device__ double operator()(long long i) const { return 2.0 * occ[i] * eps[i] * q[i]; }
};
struct FnEntropy {
  const double *occ, *q;
  __device__ double operator()(long long i) const {
    const double f = occ[i];
    double t = 0.0;
    if (f > 0.0) t += f * log(f);
    if (f < 1.0) t += (1.0 - f) * log1p(-f);
    return -2.0 * q[i] * t;
  }
};
// 4 pi |rho(G)/N - rho_ion(G)|^2 / G^2 for G != 0 (ig2 = 1/G^2, 0 at G = 0), summed over the full grid from
// the half spectrum rG of the real field rho: an entry with 0 < x < nx/2 also stands for its partner
// -G = (nx - x, -y, -z), where rho(-G) = conj rho(G).  The analytic ion spectrum iG (full grid) is not
// conjugate-paired on the y and z Nyquist planes, so the partner's rho_ion is read, not inferred.
struct FnEs {
  const double2 *rG, *iG;
  const double *ig2;
  double inv_n;
  int nx, ny, nz;
  __device__ double operator()(long long i) const {
    const int nxh = nx / 2 + 1;
    const int x = (int)(i % nxh);
    const long long yz = i / nxh;
    const int y = (int)(yz % ny), z = (int)(yz / ny);
    const double2 r = rG[i];
    const double2 a = iG[((long long)z * ny + y) * nx + x];
    const double ar = r.x * inv_n - a.x, ai = r.y * inv_n - a.y;
    double t = ar * ar + ai * ai;
    if (x != 0 && 2 * x != nx) {
      const int yp = y == 0 ? 0 : ny - y, zp = z == 0 ? 0 : nz - z;
      const double2 b = iG[((long long)zp * ny + yp) * nx + (nx - x)];
      const double br = r.x * inv_n - b.x, bi = -r.y * inv_n - b.y;
      t += br * br + bi * bi;
    }
    return 4.0 * M_PI * t * ig2[i];
  }
};

__global__ void k_energy_combine(double *sc, int hxc, double kT) {
  // slots: 0 mu, 1 eband, 2 int V rho_out, 3 E_es, 4 E_x, 5 drho, 6 ne_out, 7 entropy, 8 E, 9 F
  double E = sc[1];
  if (hxc == DC_HXC_HARTREE_X) E = sc[1] - sc[2] + sc[3] + sc[4];
  sc[8] = E;
  sc[9] = E - kT * sc[7];
}

__global__ void k_mix(long long n, double *rho_in, const double *rho_out, double alpha) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rho_in[i] = rho_in[i] + alpha * (rho_out[i] - rho_in[i]);
}

__global__ void k_residual(long long n, const double *rho_out, const double *rho_in, double *out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = rho_out[i] - rho_in[i];
}

// Kerker weight (tabulated: alpha G^2/(G^2+q0^2)/N for the unnormalised inverse transform)
__global__ void k_kerker(long long npts, const double *kw, double2 *c) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npts) return;
  const double w = kw[idx];
  const double2 v = c[idx];
  c[idx] = make_double2(w * v.x, w * v.y);
}

__global__ void k_sub_cplx(long long n, const double2 *b, double2 *a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

__global__ void k_add_real(long long n, double *rho_in, const double *d) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rho_in[i] += d[i];
}

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

int fft(dc_ctx *c, double2 *data, int dir) {
  const cufftResult r = cufftExecZ2Z(c->plan_z2z, reinterpret_cast<cufftDoubleComplex *>(data),
                                     reinterpret_cast<cufftDoubleComplex *>(data), dir);
  if (r != CUFFT_SUCCESS) {
    dc_set_error("cufftExecZ2Z failed");
    return DC_ERR_CUDA;
  }
  return DC_OK;
}

// Real field (N) -> its half spectrum (out of place; the input is left as it is)
int fft_r2c(dc_ctx *c, const double *in, double2 *out) {
  if (cufftExecD2Z(c->plan_d2z, const_cast<double *>(in), reinterpret_cast<cufftDoubleComplex *>(out)) !=
      CUFFT_SUCCESS) {
    dc_set_error("cufftExecD2Z failed");
    return DC_ERR_CUDA;
  }
  return DC_OK;
}

// Half spectrum -> real field (unnormalised; out of place, the spectrum is overwritten)
int fft_c2r(dc_ctx *c, double2 *in, double *out) {
  if (cufftExecZ2D(c->plan_z2d, reinterpret_cast<cufftDoubleComplex *>(in), out) != CUFFT_SUCCESS) {
    dc_set_error("cufftExecZ2D failed");
    return DC_ERR_CUDA;
  }
  return DC_OK;
}

int fft_streams(dc_ctx *c, cudaStream_t s) {
  const bool ok = cufftSetStream(c->plan_z2z, s) == CUFFT_SUCCESS && cufftSetStream(c->plan_d2z, s) == CUFFT_SUCCESS &&
                  cufftSetStream(c->plan_z2d, s) == CUFFT_SUCCESS;
  if (!ok) {
    dc_set_error("cufftSetStream failed");
    return DC_ERR_CUDA;
  }
  return DC_OK;
}

}  // namespace

namespace dck {

int launch_vion(dc_ctx *c, cudaStream_t s) {
  const long long N = c->npts;
  const int *n = c->grid.n;
  const double *L = c->grid.L;
  const long long NH = c->nh;
  DC_TRY(fft_streams(c, s));
  k_gtables<<<nblk(NH), 256, 0, s>>>(NH, n[0], n[1], n[2], L[0], L[1], L[2], c->params.mix_alpha,
                                     c->params.kerker_q0 * c->params.kerker_q0, N, c->d_ig2, c->d_kerkw);
  k_rho_ion_G<<<nblk(N), 256, 0, s>>>(N, n[0], n[0], n[1], n[2], L[0], L[1], L[2], c->natom, c->d_atom_pos,
                                      c->d_atom_species, c->d_species, c->nspecies, c->volume, c->d_rhoiG);
  DC_CUDA(cudaGetLastError());
  // V_loc(G) = -4 pi rho_ion(G)/G^2 ; V_loc(r) = Re sum_G V(G) e^{iG.r}.  The analytic spectrum's
  // Nyquist planes are not conjugate-paired, so this once-per-context stage keeps the full transform.
  k_vloc_G<<<nblk(N), 256, 0, s>>>(N, n[0], n[1], n[2], L[0], L[1], L[2], c->d_rhoiG, c->d_cplx);
  DC_TRY(fft(c, c->d_cplx, CUFFT_INVERSE));
  k_cplx_real<<<nblk(N), 256, 0, s>>>(N, c->d_cplx, 1.0, c->d_vion);
  // starting density: max(Re sum_G rho_ion(G) e^{iG.r}, 0) scaled to N_e
  DC_CUDA(cudaMemcpyAsync(c->d_cplx, c->d_rhoiG, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
  DC_TRY(fft(c, c->d_cplx, CUFFT_INVERSE));
  k_cplx_real<<<nblk(N), 256, 0, s>>>(N, c->d_cplx, 1.0, c->d_rho0);
  k_clamp_pos<<<nblk(N), 256, 0, s>>>(N, c->d_rho0);
  DC_TRY(reduce(FnSum{c->d_rho0}, N, c->dV, c->d_scalar + 15, c->d_partials, s));
  k_scale<<<nblk(N), 256, 0, s>>>(N, c->d_rho0, c->d_scalar + 15, c->ne);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

int launch_potential(dc_ctx *c, const double *rho, cudaStream_t s, double2 *save_rhoG, bool with_fragment_xc) {
  const long long N = c->npts;
  if (c->params.hxc == DC_HXC_HARTREE_X) {
    const long long NH = c->nh;
    DC_TRY(fft_streams(c, s));
    // rho(G) on the half grid, kept in save_rhoG when the mixing stage wants it
    double2 *spec = save_rhoG ? save_rhoG : c->d_cplxh;
    DC_TRY(fft_r2c(c, rho, spec));
    k_poisson_scale<<<nblk(NH), 256, 0, s>>>(NH, c->d_ig2, spec, 4.0 * M_PI, c->d_cplxh);
    DC_TRY(fft_c2r(c, c->d_cplxh, c->d_fftr));
  }
  const int with_x = c->params.xc_fragment && with_fragment_xc ? 0 : 1;
  k_veff<<<nblk(N), 256, 0, s>>>(N, c->d_vion, c->d_fftr, 1.0 / (double)N, rho, c->params.hxc, with_x, c->d_veff);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

int launch_gather(dc_ctx *c, cudaStream_t s, const double *rho_in) {
  const double fd[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
  const double sym = fd[0] + 2.0 * (-fd[1] + fd[2] - fd[3] + fd[4]);
  double kin = 0.0;
  for (int d = 0; d < 3; ++d) kin += -sym / (2.0 * c->h[d] * c->h[d]);
  const int bstride = 4 + 2 * c->params.cheb_degree;
  const int nf = c->f_hi - c->f_lo;  // the context's fragment shard (all fragments on one rank)
  if (nf <= 0) return DC_OK;
  const bool frag_xc = rho_in != nullptr;
  k_gather<<<nf, 256, 0, s>>>(c->d_desc + c->f_lo, c->d_idx_map, c->d_veff, c->d_vf64, c->d_vf32,
                              c->d_nl_bound + c->f_lo, kin, c->d_bounds + (long long)c->f_lo * bstride, bstride,
                              frag_xc ? c->d_rhof : nullptr, rho_in, c->params.xi > 0.0 ? 1.0 / c->params.xi : 0.0);
  if (frag_xc) {
    // the potential each core point feels (its owner fragment's), for the energy's double counting
    k_vcore<<<nblk(c->npts), 256, 0, s>>>(c->npts, c->d_desc, c->d_owner, c->d_core_local, c->d_vf64, c->d_vcore);
  }
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

int launch_gather_plain(dc_ctx *c, const double *V, double *vf64, float *vf32, cudaStream_t s) {
  const long long n = c->layout.frag_points;
  k_gather_plain<<<nblk(n), 256, 0, s>>>(n, c->d_idx_map, V, vf64, vf32);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

int launch_energy(dc_ctx *c, const double *rho_in, cudaStream_t s) {
  const long long N = c->npts;
  const int *n = c->grid.n;
  double *sc = c->d_scalar;
  const long long ns = c->layout.nstates;
  DC_TRY(reduce(FnBand{c->d_occ, c->d_eps, c->d_q}, ns, 1.0, sc + 1, c->d_partials, s));
  DC_TRY(reduce(FnEntropy{c->d_occ, c->d_q}, ns, 1.0, sc + 7, c->d_partials, s));
  DC_TRY(reduce(FnDot{c->params.xc_fragment ? c->d_vcore : c->d_veff, c->d_rho_out}, N, c->dV, sc + 2,
                 c->d_partials, s));
  DC_TRY(reduce(FnEx{c->d_rho_out}, N, -0.75 * cbrt(3.0 / M_PI) * c->dV, sc + 4, c->d_partials, s));
  DC_TRY(reduce(FnAbsDiff{c->d_rho_out, rho_in}, N, c->dV / c->ne, sc + 5, c->d_partials, s));
  DC_TRY(reduce(FnSum{c->d_rho_out}, N, c->dV, sc + 6, c->d_partials, s));
  if (c->params.hxc == DC_HXC_HARTREE_X) {
    DC_TRY(fft_streams(c, s));
    DC_TRY(fft_r2c(c, c->d_rho_out, c->d_cplxh));
    FnEs fe{c->d_cplxh, c->d_rhoiG, c->d_ig2, 1.0 / (double)N, n[0], n[1], n[2]};
    DC_TRY(reduce(fe, c->nh, 0.5 * c->volume, sc + 3, c->d_partials, s));
  }
  k_energy_combine<<<1, 1, 0, s>>>(sc, c->params.hxc, c->params.kT);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

// rho_in_G: the half spectrum of rho_in from this step's potential stage, with c->d_cplxh still holding the
// energy stage's spectrum of rho_out; the residual's spectrum is then their difference (linearity of
// the transform) and its forward transform is skipped.  nullptr: transform the residual.
int launch_mix(dc_ctx *c, double *rho_in, cudaStream_t s, const double2 *rho_in_G) {
  const long long N = c->npts;
  const double q0 = c->params.kerker_q0;
  if (!(q0 > 0.0)) {
    k_mix<<<nblk(N), 256, 0, s>>>(N, rho_in, c->d_rho_out, c->params.mix_alpha);
    DC_CUDA(cudaGetLastError());
    return DC_OK;
  }
  const long long NH = c->nh;
  DC_TRY(fft_streams(c, s));
  if (rho_in_G) {
    k_sub_cplx<<<nblk(NH), 256, 0, s>>>(NH, rho_in_G, c->d_cplxh);
  } else {
    k_residual<<<nblk(N), 256, 0, s>>>(N, c->d_rho_out, rho_in, c->d_fftr);
    DC_TRY(fft_r2c(c, c->d_fftr, c->d_cplxh));
  }
  k_kerker<<<nblk(NH), 256, 0, s>>>(NH, c->d_kerkw, c->d_cplxh);
  DC_TRY(fft_c2r(c, c->d_cplxh, c->d_fftr));
  k_add_real<<<nblk(N), 256, 0, s>>>(N, rho_in, c->d_fftr);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

int launch_init_psi(dc_ctx *c, double *psi64, cudaStream_t s) {
  k_init_psi<<<(unsigned)c->layout.nstates, 256, 0, s>>>(c->d_desc, c->d_items, c->params.seed, psi64);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

int launch_convert(const double *src, float *dst, long long n, cudaStream_t s) {
  k_d2f<<<nblk(n), 256, 0, s>>>(n, src, dst);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}
int launch_convert(const float *src, double *dst, long long n, cudaStream_t s) {
  k_f2d<<<nblk(n), 256, 0, s>>>(n, src, dst);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

int launch_sum(const double *x, long long n, double *out, double *partials, int, cudaStream_t s) {
  return reduce(FnSum{x}, n, 1.0, out, partials, s);
}

}  // namespace dck
