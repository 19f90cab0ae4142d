// Density stage (Sec. 2.2, Eqs. 2-4): core weights, global chemical potential, occupations and the
// core-projected density rho_tot(g) = sum_i 2 f_i^f psi_i^f(j)^2 with f = owner(g).
#include <climits>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "dc_internal.h"

namespace {

constexpr int QNT = 256;

template <typename T>
__global__ void __launch_bounds__(QNT) k_core_weights(const FragDesc *desc, const int2 *items, const T *psi,
                                                     double dV, double *q) {
  __shared__ double red[QNT / 32];
  const int2 it = items[blockIdx.x];
  const FragDesc D = desc[it.x];
  const int Ex = D.E[0], Ey = D.E[1];
  const long long P = (long long)Ex * Ey * D.E[2];
  const T *y = psi + D.psi_off + (long long)it.y * P;
  const int cx = D.c[0], cy = D.c[1], cz = D.c[2];
  const int ncore = cx * cy * cz;
  double s = 0.0;
  for (int t = threadIdx.x; t < ncore; t += QNT) {
    const int x = t % cx, yz = t / cx, yy = yz % cy, z = yz / cy;
    const long long j = (x + D.b[0]) + (long long)Ex * ((yy + D.b[1]) + (long long)Ey * (z + D.b[2]));
    const double v = (double)y[j];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < QNT / 32; ++w) tot += red[w];
    q[D.st_off + it.y] = dV * tot;
  }
}

// Grid-wide barrier for a cooperative launch.  The wait is bounded: after DC_SPIN_LIMIT polls the
// block sets DC_FLAG_TIMEOUT and returns false, and the kernel then stops.
__device__ bool grid_sync(unsigned *count, unsigned *gen, unsigned nblocks, unsigned *flags) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = *((volatile unsigned *)gen);
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u) + 1u;
    if (arrived == nblocks) {
      *((volatile unsigned *)count) = 0u;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned it = 0;
      while (*((volatile unsigned *)gen) == g) {
        if (++it > DC_SPIN_LIMIT) {
          atomicOr(flags, DC_FLAG_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Failure-detection self-test: every block arrives at a grid barrier that expects one arrival more
// than the launch has, so no block can pass; each gives up after its bounded poll count, sets
// DC_FLAG_TIMEOUT and returns.  Nothing after the barrier runs.
__global__ void k_wait_selftest(unsigned *bar, unsigned *flags, unsigned nexpect) {
  if (!grid_sync(bar, bar + 1, nexpect, flags)) return;
}

__device__ __forceinline__ double fermi_occ(double e, double mu, double kT) {
  return 0.5 * (1.0 - tanh(0.5 * (e - mu) / kT));
}

// FP64 bisection for mu (the bracket and stopping rule of the FP64 oracle), all blocks in step:
// every block evaluates its share of sum 2 f q, the partial sums meet at a grid barrier and each
// block adds them in the same fixed order, so all blocks take identical decisions.
__global__ void __launch_bounds__(QNT) k_fermi(const double *eps, const double *q, int nst, double ne, double kT,
                                              double *partials, unsigned *bar, unsigned *flags, double *mu_out,
                                              double *occ) {
  __shared__ double red[QNT / 32];
  __shared__ double red2[QNT / 32];
  const int nb = gridDim.x;
  const int stride = nb * QNT;
  const int base = blockIdx.x * QNT + threadIdx.x;
  // global min / max of eps
  double lo = 1e300, hi = -1e300;
  for (int p = base; p < nst; p += stride) {
    lo = fmin(lo, eps[p]);
    hi = fmax(hi, eps[p]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = lo;
    red2[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = red[0], b = red2[0];
    for (int w = 1; w < QNT / 32; ++w) {
      a = fmin(a, red[w]);
      b = fmax(b, red2[w]);
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
  if (!grid_sync(bar, bar + 1, nb, flags)) return;
  // partial sums written by other blocks are read with L2-coherent loads (no stale L1 lines)
  lo = __ldcg(&partials[0]);
  hi = __ldcg(&partials[1]);
  for (int b = 1; b < nb; ++b) {
    lo = fmin(lo, __ldcg(&partials[2 * b]));
    hi = fmax(hi, __ldcg(&partials[2 * b + 1]));
  }
  lo -= 40.0 * kT;
  hi += 40.0 * kT;
  // Safeguarded Newton: every iteration evaluates N(mu) and dN/dmu in one pass, shrinks the bracket
  // by the sign of N - N_e, and takes the Newton step when it stays inside the bracket (bisection
  // otherwise).  Starts from the previous mu when that lies in the bracket.  Converged when the
  // Newton correction is below 1e-14 Ha, the bracket below 1e-13 Ha, or the correction has reached the
  // rounding floor of the FP64 electron count (~1e-13 Ha for 1e4-1e5 states): below 1e-10 Ha and no
  // longer at least ten times smaller than the one before (quadratic convergence shrinks it by orders
  // of magnitude until then).  Every block reads the same sums, so every block takes the same exit.
  double *pacc = partials + 2 * nb;  // [2][2 nb]
  const double guess = __ldcg(mu_out);
  double mu = (guess > lo && guess < hi) ? guess : 0.5 * (lo + hi);
  double prev = 1e300;  // |Newton correction| of the previous iteration
  for (int itn = 0; itn < 200; ++itn) {
    double s = 0.0, ds = 0.0;
    for (int p = base; p < nst; p += stride) {
      const double fo = fermi_occ(eps[p], mu, kT);
      s += 2.0 * fo * q[p];
      ds += 2.0 * q[p] * fo * (1.0 - fo) / kT;
    }
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, o);
      ds += __shfl_xor_sync(0xffffffffu, ds, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5] = s;
      red2[threadIdx.x >> 5] = ds;
    }
    __syncthreads();
    double *pa = pacc + (itn & 1) * 2 * nb;
    if (threadIdx.x == 0) {
      double t = 0.0, dt = 0.0;
      for (int w = 0; w < QNT / 32; ++w) {
        t += red[w];
        dt += red2[w];
      }
      pa[2 * blockIdx.x] = t;
      pa[2 * blockIdx.x + 1] = dt;
    }
    if (!grid_sync(bar, bar + 1, nb, flags)) return;
    // every block adds the block partials in the same fixed order: warp 0's lanes stride over the
    // blocks (independent loads), then a shuffle tree; lane 0's result is shared through red
    if (threadIdx.x < 32) {
      double t = 0.0, dt = 0.0;
      for (int b = threadIdx.x; b < nb; b += 32) {
        t += __ldcg(&pa[2 * b]);
        dt += __ldcg(&pa[2 * b + 1]);
      }
      for (int o = 16; o > 0; o >>= 1) {
        t += __shfl_xor_sync(0xffffffffu, t, o);
        dt += __shfl_xor_sync(0xffffffffu, dt, o);
      }
      if (threadIdx.x == 0) {
        red[0] = t;
        red2[0] = dt;
      }
    }
    __syncthreads();
    const double tot = red[0], dtot = red2[0];
    const double r = tot - ne;
    if (r < 0.0) lo = mu;
    else hi = mu;
    const double step = dtot > 0.0 ? r / dtot : 0.0;
    double nm = mu - step;
    const bool newton_ok = dtot > 0.0 && nm > lo && nm < hi;
    const bool floor = dtot > 0.0 && fabs(step) < 1e-10 && fabs(step) > 0.1 * prev;
    if (r == 0.0 || (newton_ok && fabs(step) < 1e-14) || hi - lo < 1e-13 || floor) {
      if (newton_ok) mu = nm;
      break;
    }
    prev = dtot > 0.0 ? fabs(step) : 1e300;
    mu = newton_ok ? nm : 0.5 * (lo + hi);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    mu_out[0] = mu;
    if (!isfinite(mu)) atomicOr(flags, DC_FLAG_NONFINITE);
  }
  for (int p = base; p < nst; p += stride) occ[p] = fermi_occ(eps[p], mu, kT);
}

// Points whose owner lies outside the fragment range [f_lo, f_hi) get 0 (a rank's share of rho).
template <typename T>
__global__ void k_density(const FragDesc *desc, const int32_t *owner, const int32_t *core_local, long long npts,
                          const T *psi, const double *occ, double *rho, int f_lo, int f_hi) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npts) return;
  const int f = owner[g];
  if (f < f_lo || f >= f_hi) {
    rho[g] = 0.0;
    return;
  }
  const FragDesc D = desc[f];
  const long long P = (long long)D.E[0] * D.E[1] * D.E[2];
  const T *y = psi + D.psi_off + core_local[g];
  const double *o = occ + D.st_off;
  double s = 0.0;
  for (int i = 0; i < D.norb; ++i) {
    const double v = (double)y[(long long)i * P];
    s += 2.0 * o[i] * v * v;
  }
  rho[g] = s;
}

// ---- FP32 orbital blocks: FP32 products with double-word FP32 accumulation ---------------------
// The FP64 pipe of this part runs at ~1/64 of FP32, so summing FP32 orbitals in FP64 made these
// kernels FP64-bound.  Here every square is formed exactly as an unevaluated FP32 pair (product and
// its FMA residual) and the sums are kept as (hi, lo) FP32 pairs (TwoSum), which carries ~2^-44
// relative accuracy; the pair is converted to FP64 once per result.
__device__ __forceinline__ void dw_add(float &hi, float &lo, float a) {
  const float s = hi + a;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (a - bp);
  hi = s;
  lo += e;
}

// Scalar forms of the two kernels below, for cells whose core rows do not split into point pairs.
// q_i = dV sum_core psi_i^2: CTA = (fragment, 8 orbitals), one warp per orbital.
__global__ void __launch_bounds__(256) k_core_weights32s(const FragDesc *desc, const float *psi, double dV,
                                                        double *q) {
  const FragDesc D = desc[blockIdx.x];
  const int i = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (i >= D.norb) return;
  const int lane = threadIdx.x & 31;
  const int Ex = D.E[0], Ey = D.E[1];
  const long long P = (long long)Ex * Ey * D.E[2];
  const float *y = psi + D.psi_off + (long long)i * P;
  const int cx = D.c[0], cy = D.c[1];
  const int ncore = cx * cy * D.c[2];
  float hi = 0.f, lo = 0.f;
  for (int t = lane; t < ncore; t += 32) {
    const int x = t % cx, yz = t / cx, yy = yz % cy, z = yz / cy;
    const float v = y[(x + D.b[0]) + Ex * ((yy + D.b[1]) + Ey * (z + D.b[2]))];
    const float p = __fmul_rn(v, v);  // not contracted into the TwoSum below
    dw_add(hi, lo, p);
    lo += fmaf(v, v, -p);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    dw_add(hi, lo, h2);
    lo += l2;
  }
  if (lane == 0) q[D.st_off + i] = dV * ((double)hi + (double)lo);
}

// rho(g) = sum_i 2 f_i psi_i(j)^2 over the core points of one fragment (CTA = fragment): each core
// point is owned by exactly one fragment, so every global point is written once.  The occupations
// are carried as FP32 pairs (2 f = oh + ol) and every term is formed with exact products, so the
// density integrates to sum 2 f q = N_e to ~1e-12 (an FP32-rounded 2 f would break that at 1e-8).
__global__ void __launch_bounds__(256) k_density32s(const FragDesc *desc, const float *psi, const double *occ, int Nx,
                                                   int Ny, double *rho) {
  __shared__ float occh[DC_MAX_NORB], occl[DC_MAX_NORB];
  const FragDesc D = desc[blockIdx.x];
  const int n = D.norb;
  for (int i = threadIdx.x; i < n; i += 256) {
    const double o2 = 2.0 * occ[D.st_off + i];
    const float h = (float)o2;
    occh[i] = h;
    occl[i] = (float)(o2 - (double)h);
  }
  __syncthreads();
  const int Ex = D.E[0], Ey = D.E[1];
  const long long P = (long long)Ex * Ey * D.E[2];
  const float *y0 = psi + D.psi_off;
  const int cx = D.c[0], cy = D.c[1];
  const int ncore = cx * cy * D.c[2];
  const int gx0 = D.org[0] + D.b[0], gy0 = D.org[1] + D.b[1], gz0 = D.org[2] + D.b[2];
  for (int t = threadIdx.x; t < ncore; t += 256) {
    const int x = t % cx, yz = t / cx, yy = yz % cy, z = yz / cy;
    const float *y = y0 + (x + D.b[0]) + Ex * ((yy + D.b[1]) + Ey * (z + D.b[2]));
    float hi = 0.f, lo = 0.f;
#pragma unroll 4
    for (int i = 0; i < n; ++i) {
      const float v = y[(long long)i * P];
      const float p = __fmul_rn(v, v), pe = fmaf(v, v, -p);  // v^2 = p + pe exactly
      const float oh = occh[i];
      const float th = __fmul_rn(oh, p), te = fmaf(oh, p, -th);  // oh p = th + te exactly
      dw_add(hi, lo, th);
      lo += te + fmaf(oh, pe, occl[i] * p);
    }
    rho[(gx0 + x) + (long long)Nx * ((gy0 + yy) + (long long)Ny * (gz0 + z))] = (double)hi + (double)lo;
  }
}

// Core points are read as x-adjacent pairs (one 8-byte load) when every fragment's core rows start at an
// even x and have an even length and its rows an even length (dc_ctx::core_pairs).  A core row is
// c_x of the fragment's E_x points, so the sectors a warp touches carry buffer points too; the loads
// are unrolled so that several are in flight per thread.

// q_i = dV sum_core psi_i^2: CTA = (fragment, 8 orbitals), one warp per orbital.
__global__ void __launch_bounds__(256) k_core_weights32(const FragDesc *desc, const float *psi, double dV,
                                                        double *q) {
  const FragDesc D = desc[blockIdx.x];
  const int i = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (i >= D.norb) return;
  const int lane = threadIdx.x & 31;
  const int Ex = D.E[0], Ey = D.E[1];
  const long long P = (long long)Ex * Ey * D.E[2];
  const float *y = psi + D.psi_off + (long long)i * P + D.b[0] + (long long)Ex * (D.b[1] + (long long)Ey * D.b[2]);
  const int cx2 = D.c[0] >> 1, cy = D.c[1];
  const int nu = cx2 * cy * D.c[2];  // core point pairs
  float hi = 0.f, lo = 0.f;
  constexpr int U = 4;
  for (int t0 = lane; t0 < nu; t0 += 32 * U) {
    float2 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = t0 + 32 * u;
      v[u] = make_float2(0.f, 0.f);
      if (t < nu) {
        const int x2 = t % cx2, yz = t / cx2, yy = yz % cy, z = yz / cy;
        v[u] = *reinterpret_cast<const float2 *>(y + 2 * x2 + Ex * (yy + (long long)Ey * z));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const float p0 = __fmul_rn(v[u].x, v[u].x);  // not contracted into the TwoSum below
      dw_add(hi, lo, p0);
      lo += fmaf(v[u].x, v[u].x, -p0);
      const float p1 = __fmul_rn(v[u].y, v[u].y);
      dw_add(hi, lo, p1);
      lo += fmaf(v[u].y, v[u].y, -p1);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    dw_add(hi, lo, h2);
    lo += l2;
  }
  if (lane == 0) q[D.st_off + i] = dV * ((double)hi + (double)lo);
}

// rho(g) = sum_i 2 f_i psi_i(j)^2 over the core points of one fragment (CTA = fragment): each core
// point is owned by exactly one fragment, so every global point is written once.  The occupations
// are carried as FP32 pairs (2 f = oh + ol) and every term is formed with exact products, so the
// density integrates to sum 2 f q = N_e to ~1e-12 (an FP32-rounded 2 f would break that at 1e-8).
// A thread takes one core point pair and walks the orbitals eight loads at a time.
__global__ void __launch_bounds__(256) k_density32(const FragDesc *desc, const float *psi, const double *occ, int Nx,
                                                   int Ny, double *rho) {
  __shared__ float occh[DC_MAX_NORB], occl[DC_MAX_NORB];
  const FragDesc D = desc[blockIdx.x];
  const int n = D.norb;
  for (int i = threadIdx.x; i < n; i += 256) {
    const double o2 = 2.0 * occ[D.st_off + i];
    const float h = (float)o2;
    occh[i] = h;
    occl[i] = (float)(o2 - (double)h);
  }
  __syncthreads();
  const int Ex = D.E[0], Ey = D.E[1];
  const long long P = (long long)Ex * Ey * D.E[2];
  const float *y0 = psi + D.psi_off + D.b[0] + (long long)Ex * (D.b[1] + (long long)Ey * D.b[2]);
  const int cx2 = D.c[0] >> 1, cy = D.c[1];
  const int nu = cx2 * cy * D.c[2];
  const int gx0 = D.org[0] + D.b[0], gy0 = D.org[1] + D.b[1], gz0 = D.org[2] + D.b[2];
  for (int t = threadIdx.x; t < nu; t += 256) {
    const int x2 = t % cx2, yz = t / cx2, yy = yz % cy, z = yz / cy;
    const float *y = y0 + 2 * x2 + Ex * (yy + (long long)Ey * z);
    float hi0 = 0.f, lo0 = 0.f, hi1 = 0.f, lo1 = 0.f;
    constexpr int U = 8;
    for (int i0 = 0; i0 < n; i0 += U) {
      float2 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = i0 + u < n ? *reinterpret_cast<const float2 *>(y + (long long)(i0 + u) * P)
                                                   : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (i0 + u >= n) break;
        const float oh = occh[i0 + u], ol = occl[i0 + u];
        {
          const float p = __fmul_rn(v[u].x, v[u].x), pe = fmaf(v[u].x, v[u].x, -p);  // v^2 = p + pe exactly
          const float th = __fmul_rn(oh, p), te = fmaf(oh, p, -th);                  // oh p = th + te exactly
          dw_add(hi0, lo0, th);
          lo0 += te + fmaf(oh, pe, ol * p);
        }
        {
          const float p = __fmul_rn(v[u].y, v[u].y), pe = fmaf(v[u].y, v[u].y, -p);
          const float th = __fmul_rn(oh, p), te = fmaf(oh, p, -th);
          dw_add(hi1, lo1, th);
          lo1 += te + fmaf(oh, pe, ol * p);
        }
      }
    }
    double *r = rho + (gx0 + 2 * x2) + (long long)Nx * ((gy0 + yy) + (long long)Ny * (gz0 + z));
    r[0] = (double)hi0 + (double)lo0;
    r[1] = (double)hi1 + (double)lo1;
  }
}

}  // namespace

namespace dck {

template <typename T>
int launch_core_weights(dc_ctx *c, const T *psi, double *q, cudaStream_t s) {
  const int nf = c->f_hi - c->f_lo;
  if (nf <= 0) return DC_OK;
  if constexpr (std::is_same<T, float>::value) {
    const dim3 grid((unsigned)nf, (unsigned)((c->layout.max_norb + 7) / 8));
    if (c->core_pairs)
      k_core_weights32<<<grid, 256, 0, s>>>(c->d_desc + c->f_lo, psi, c->dV, q);
    else
      k_core_weights32s<<<grid, 256, 0, s>>>(c->d_desc + c->f_lo, psi, c->dV, q);
  } else {
    k_core_weights<T><<<(unsigned)(c->st_hi - c->st_lo), QNT, 0, s>>>(c->d_desc, c->d_items + c->st_lo, psi, c->dV, q);
  }
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

int launch_fermi(dc_ctx *c, const double *eps_in, const double *q_in, double *mu_io, double *occ_out, cudaStream_t s) {
  int nb = 0;
  DC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fermi, QNT, 0));
  if (nb < 1) {
    dc_set_error("fermi: kernel cannot be resident");
    return DC_ERR_CUDA;
  }
  int grid = c->sm_count;  // one block per SM, all co-resident (cooperative launch checks it)
  const int need = (int)((c->layout.nstates + QNT - 1) / QNT);
  if (grid > need) grid = need > 0 ? need : 1;
  DC_CUDA(cudaMemsetAsync(c->d_flags + 1, 0, 2 * sizeof(unsigned), s));
  const double *eps = eps_in;
  const double *q = q_in;
  int nst = (int)c->layout.nstates;
  double ne = c->ne, kT = c->params.kT;
  double *partials = c->d_partials;
  unsigned *bar = c->d_flags + 1;
  unsigned *flags = c->d_flags;
  double *mu = mu_io;
  double *occ = occ_out;
  void *args[] = {&eps, &q, &nst, &ne, &kT, &partials, &bar, &flags, &mu, &occ};
  DC_CUDA(cudaLaunchCooperativeKernel((const void *)k_fermi, dim3(grid), dim3(QNT), args, 0, s));
  return DC_OK;
}

int launch_wait_selftest(dc_ctx *c, cudaStream_t s) {
  DC_CUDA(cudaMemsetAsync(c->d_flags + 1, 0, 2 * sizeof(unsigned), s));
  k_wait_selftest<<<2, 32, 0, s>>>(c->d_flags + 1, c->d_flags, 3u);  // two blocks, three expected
  DC_CUDA(cudaGetLastError());
  DC_CUDA(cudaMemsetAsync(c->d_flags + 1, 0, 2 * sizeof(unsigned), s));
  return DC_OK;
}

template <typename T>
int launch_density(dc_ctx *c, const T *psi, const double *occ, double *rho, cudaStream_t s) {
  const int nf = c->f_hi - c->f_lo;
  if constexpr (std::is_same<T, float>::value) {
    // one CTA per owned core writes exactly that core's points; on a shard the rest of rho is zero
    if (nf < c->nfrag) DC_CUDA(cudaMemsetAsync(rho, 0, sizeof(double) * (size_t)c->npts, s));
    if (nf > 0)
      if (c->core_pairs)
        k_density32<<<(unsigned)nf, 256, 0, s>>>(c->d_desc + c->f_lo, psi, occ, c->grid.n[0], c->grid.n[1], rho);
      else
        k_density32s<<<(unsigned)nf, 256, 0, s>>>(c->d_desc + c->f_lo, psi, occ, c->grid.n[0], c->grid.n[1], rho);
  } else {
    const unsigned nb = (unsigned)((c->npts + 255) / 256);
    k_density<T><<<nb, 256, 0, s>>>(c->d_desc, c->d_owner, c->d_core_local, c->npts, psi, occ, rho, c->f_lo,
                                    c->f_hi);
  }
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

template int launch_core_weights<double>(dc_ctx *, const double *, double *, cudaStream_t);
template int launch_core_weights<float>(dc_ctx *, const float *, double *, cudaStream_t);
template int launch_density<double>(dc_ctx *, const double *, const double *, double *, cudaStream_t);
template int launch_density<float>(dc_ctx *, const float *, const double *, double *, cudaStream_t);

}  // namespace dck

// ---- allocation-free Fermi level ---------------------------------------------------------------
// dc_fermi_level_noalloc runs the k_fermi solve above without a context: its scratch is a fixed
// array in this module's static device memory instead of context buffers.  It exists for callers
// that may not allocate device memory at the point where they need mu: code working inside a
// caller-owned memory pool or arena that holds the whole device (no cudaMalloc can succeed
// there), and code interleaved with work on other streams, where a cudaFree would synchronise
// the device.  Layout of the array: bytes [0, 64) are unsigned words (0: error flags,
// 1: barrier arrival count, 2: barrier generation), zeroed on the stream before every launch;
// from byte 64 on, 6 FP64 partials per block (a min/max pair, then two double-buffered pairs of
// sums), written before they are read inside each launch, so they need no clearing.
constexpr int kFermiNoallocBlocks = 256;
constexpr size_t kFermiNoallocHeader = 64;
constexpr size_t kFermiNoallocBytes = kFermiNoallocHeader + 6 * sizeof(double) * kFermiNoallocBlocks;  // 12,352

static __device__ __align__(256) unsigned char g_fermi_scratch[kFermiNoallocBytes];

namespace {

constexpr int kFermiNoallocMaxDevices = 64;

struct FermiNoallocDevice {
  bool ready = false;
  unsigned char *scratch = nullptr;  // device address of g_fermi_scratch on this device
  int sm_count = 0;
};

std::mutex g_fermi_noalloc_mutex;
FermiNoallocDevice g_fermi_noalloc_dev[kFermiNoallocMaxDevices];

// Looks up the scratch address, the SM count and the co-residency of k_fermi once per device.
int fermi_noalloc_setup(FermiNoallocDevice **out) {
  int dev = -1;
  DC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kFermiNoallocMaxDevices) {
    dc_set_error("dc_fermi_level_noalloc: device ordinal above 63");
    return DC_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_fermi_noalloc_mutex);
  FermiNoallocDevice &d = g_fermi_noalloc_dev[dev];
  if (!d.ready) {
    void *addr = nullptr;
    DC_CUDA(cudaGetSymbolAddress(&addr, g_fermi_scratch));
    int sms = 0, resident = 0;
    DC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_fermi, QNT, 0));
    if (sms < 1 || resident < 1) {
      dc_set_error("dc_fermi_level_noalloc: k_fermi cannot be resident on this device");
      return DC_ERR_CUDA;
    }
    d.scratch = static_cast<unsigned char *>(addr);
    d.sm_count = sms;
    d.ready = true;
  }
  *out = &d;
  return DC_OK;
}

}  // namespace

extern "C" int dc_fermi_level_noalloc(const double *d_eps, const double *d_q, int64_t nstates, double n_elec,
                                      double kT, double *d_mu, double *d_occ, void *stream) {
  if (nstates < 0 || nstates > (int64_t)INT_MAX) {
    dc_set_error("dc_fermi_level_noalloc: nstates outside [0, 2^31 - 1] (the kernel indexes states with int)");
    return DC_ERR_ARG;
  }
  FermiNoallocDevice *dev = nullptr;
  DC_TRY(fermi_noalloc_setup(&dev));
  if (nstates == 0) return DC_OK;  // setup only
  if (!d_eps || !d_q || !d_mu || !d_occ) {
    dc_set_error("dc_fermi_level_noalloc: NULL device pointer");
    return DC_ERR_ARG;
  }
  if (!(kT > 0.0) || !std::isfinite(kT) || !(n_elec >= 0.0) || !std::isfinite(n_elec)) {
    dc_set_error("dc_fermi_level_noalloc: kT must be finite and > 0, n_elec finite and >= 0");
    return DC_ERR_ARG;
  }
  // one block per SM (all co-resident), no more blocks than states need or the scratch holds
  int grid = dev->sm_count;
  const int need = (int)((nstates + QNT - 1) / QNT);
  if (grid > need) grid = need;
  if (grid > kFermiNoallocBlocks) grid = kFermiNoallocBlocks;
  if (kFermiNoallocHeader + 6 * sizeof(double) * (size_t)grid > kFermiNoallocBytes) {
    dc_set_error("dc_fermi_level_noalloc: partials exceed the 12,352-byte static scratch");
    return DC_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned *words = reinterpret_cast<unsigned *>(dev->scratch);
  if (cudaMemsetAsync(words, 0, kFermiNoallocHeader, s) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    std::lock_guard<std::mutex> lock(g_fermi_noalloc_mutex);
    dev->ready = false;
    return dc_cuda_status(e, "dc_fermi_level_noalloc: clearing the scratch header");
  }
  const double *eps = d_eps;
  const double *q = d_q;
  int nst = (int)nstates;
  double ne = n_elec, t = kT;
  double *partials = reinterpret_cast<double *>(dev->scratch + kFermiNoallocHeader);
  unsigned *bar = words + 1;
  unsigned *flags = words;
  double *mu = d_mu;
  double *occ = d_occ;
  void *args[] = {&eps, &q, &nst, &ne, &t, &partials, &bar, &flags, &mu, &occ};
  unsigned fl = 0;
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_fermi, dim3(grid), dim3(QNT), args, 0, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&fl, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    // a device reset or a torn-down primary context leaves the cached scratch address stale: the next
    // call looks it up again
    std::lock_guard<std::mutex> lock(g_fermi_noalloc_mutex);
    dev->ready = false;
    return dc_cuda_status(e, "dc_fermi_level_noalloc");
  }
  if (fl & DC_FLAG_TIMEOUT) {
    dc_set_error("dc_fermi_level_noalloc: a bounded device wait ran out (grid barrier)");
    return DC_ERR_TIMEOUT;
  }
  if (fl & DC_FLAG_NONFINITE) {
    dc_set_error("dc_fermi_level_noalloc: non-finite chemical potential");
    return DC_ERR_NONFINITE;
  }
  return DC_OK;
}
