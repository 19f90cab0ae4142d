// Subspace kernels of the fragment eigensolver (Eq. 1): filter bounds, Gram and Rayleigh-Ritz
// contractions, FP64 Cholesky orthonormalisation and symmetric eigensolve, rotation.
//
// The paper's inner solver is "the same procedure as conventional DFT" (Sec. 2.2) and the
// dominant costs are diagonalisation and orthonormalisation.  Here one pass is a scaled
// Chebyshev filter (Zhou, Saad, Tiago & Chelikowsky, J. Comput. Phys. 219 (2006) 172) followed by
// S = <Y|Y> = L L^T, Hs = L^-1 <Y|HY> L^-T = Q diag(eps) Q^T and Psi = Y L^-T Q.
#include <type_traits>

#include "dc_internal.h"

namespace {

// ---------------------------------------------------------------------------------------------
// Filter bounds and per-step coefficients (one thread per fragment)
//   bounds[f] = {a, b_up, aL, c, alpha_0, beta_0, ..., alpha_{m-1}, beta_{m-1}}
// b_up is written by the potential gather; a and aL come from the fragment's Ritz values.
// ---------------------------------------------------------------------------------------------
__global__ void k_bounds(const FragDesc *desc, int f_lo, int f_hi, const double *eps, double *bounds, int m,
                         int stride) {
  const int f = f_lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= f_hi) return;
  const FragDesc D = desc[f];
  double lo = eps[D.st_off], hi = eps[D.st_off];
  for (int i = 1; i < D.norb; ++i) {
    lo = fmin(lo, eps[D.st_off + i]);
    hi = fmax(hi, eps[D.st_off + i]);
  }
  double *bd = bounds + (long long)f * stride;
  const double a = hi, aL = lo, b = bd[1];
  const double e = (b - a) / 2.0;
  const double c = (b + a) / 2.0;
  double sigma = e / (aL - c);
  const double tau = 2.0 / sigma;
  bd[0] = a;
  bd[2] = aL;
  bd[3] = c;
  bd[4] = sigma / e;
  bd[5] = 0.0;
  for (int k = 1; k < m; ++k) {
    const double sn = 1.0 / (tau - sigma);
    bd[4 + 2 * k] = 2.0 * sn / e;
    bd[5 + 2 * k] = -sigma * sn;
    sigma = sn;
  }
}

// ---------------------------------------------------------------------------------------------
// Gram / Rayleigh-Ritz partial sums over a chunk of points: S_p = Y_c Y_c^T and A_p = Y_c (HY)_c^T
// (no dV factor).  One CTA per (fragment, chunk); each of 256 threads owns a 4x4 tile of the
// (padded) 64x64 outputs.  FP32 inputs: products of 32-point sub-tiles summed in FP32, then
// accumulated as an unevaluated (hi, lo) FP32 pair (TwoSum); FP64 inputs: plain FP64.
// ---------------------------------------------------------------------------------------------
constexpr int GKT = 32;   // points per sub-tile
constexpr int GPAD = 68;  // padded orbital stride in shared memory

template <typename T>
struct Vec4 {
  T v[4];
};
__device__ __forceinline__ Vec4<float> ld4(const float *p) {
  const float4 t = *reinterpret_cast<const float4 *>(p);
  return {{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ Vec4<double> ld4(const double *p) {
  const double2 a = *reinterpret_cast<const double2 *>(p);
  const double2 b = *reinterpret_cast<const double2 *>(p + 2);
  return {{a.x, a.y, b.x, b.y}};
}

__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}

// Gram partials S = Y^T Y and A = Y^T HY of one (fragment, point chunk) item.  Tiles of 4 x 4 elements,
// one per thread.  When the fragment's tiles fit one per thread (n <= 48: T(T+1)/2 upper-triangle tiles
// of S and T^2 tiles of A, T = ceil(n / 4)), only those are computed and S is mirrored (a_i a_j and
// a_j a_i are the same products in the same order, so the mirror is exact); otherwise a fixed 16 x 16
// grid of tile pairs covers n <= 64.  The FP32 form accumulates each 32-point chunk in FP32 and the
// chunks with a compensated (two-sum) FP32 pair; the FP64 form in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_gram(const FragDesc *desc, const int2 *gitems, const long long *goff,
                                              int chunk, const T *Y, const T *HY, double *out) {
  __shared__ __align__(16) T sY[GKT][GPAD];
  __shared__ __align__(16) T sH[GKT][GPAD];
  const int2 it = gitems[blockIdx.x];
  const int f = it.x, ch = it.y;
  const FragDesc D = desc[f];
  const int n = D.norb;
  const long long P = (long long)D.E[0] * D.E[1] * D.E[2];
  const long long p0 = (long long)ch * chunk;
  const long long p1 = min(P, p0 + chunk);
  const T *Yf = Y + D.psi_off;
  const T *Hf = HY ? HY + D.psi_off : nullptr;
  // tile assignment
  const int TT = (n + 3) >> 2;
  const int nS = TT * (TT + 1) / 2;
  const bool tiled = nS + TT * TT <= 256;
  int ti, tj;
  bool isA = false, act = true;
  if (tiled) {
    int t = threadIdx.x;
    act = t < nS + TT * TT;
    if (t < nS) {  // upper triangle, row by row: row ti holds tiles ti .. TT - 1
      ti = 0;
      while (t >= TT - ti) {
        t -= TT - ti;
        ++ti;
      }
      tj = ti + t;
    } else if (act) {
      t -= nS;
      isA = true;
      ti = t / TT;
      tj = t - ti * TT;
    } else {
      ti = tj = 0;
    }
  } else {
    ti = threadIdx.x >> 4;
    tj = threadIdx.x & 15;
  }
  for (int t = threadIdx.x; t < GKT * GPAD; t += 256) {
    (&sY[0][0])[t] = T(0);
    (&sH[0][0])[t] = T(0);
  }
  float shi[16], slo[16], ahi[16], alo[16];
  double sd[16], ad[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    shi[e] = slo[e] = ahi[e] = alo[e] = 0.f;
    sd[e] = ad[e] = 0.0;
  }
  __syncthreads();
  for (long long pb = p0; pb < p1; pb += GKT) {
    for (int t = threadIdx.x; t < GKT * n; t += 256) {
      const int r = t / GKT, p = t - r * GKT;
      const long long pp = pb + p;
      sY[p][r] = pp < p1 ? Yf[(long long)r * P + pp] : T(0);
      if (Hf) sH[p][r] = pp < p1 ? Hf[(long long)r * P + pp] : T(0);
    }
    __syncthreads();
    T ps[16], pa[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) ps[e] = pa[e] = T(0);
    if (tiled) {
      if (act) {
        const T(*sB)[GPAD] = isA ? sH : sY;
#pragma unroll 4
        for (int p = 0; p < GKT; ++p) {
          const Vec4<T> a = ld4(&sY[p][4 * ti]);
          const Vec4<T> b = ld4(&sB[p][4 * tj]);
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) ps[4 * r + cc] += a.v[r] * b.v[cc];
        }
      }
    } else {
#pragma unroll 4
      for (int p = 0; p < GKT; ++p) {
        const Vec4<T> a = ld4(&sY[p][4 * ti]);
        const Vec4<T> b = ld4(&sY[p][4 * tj]);
        const Vec4<T> h = ld4(&sH[p][4 * tj]);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            ps[4 * r + cc] += a.v[r] * b.v[cc];
            pa[4 * r + cc] += a.v[r] * h.v[cc];
          }
      }
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      if (sizeof(T) == 4) {
        two_sum_acc(shi[e], slo[e], (float)ps[e]);
        if (!tiled) two_sum_acc(ahi[e], alo[e], (float)pa[e]);
      } else {
        sd[e] += (double)ps[e];
        if (!tiled) ad[e] += (double)pa[e];
      }
    }
    __syncthreads();
  }
  double *o = out + goff[f] + (long long)ch * 2 * n * n;
  if (!act) return;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int i = 4 * ti + r, j = 4 * tj + cc;
      if (i < n && j < n) {
        const int e = 4 * r + cc;
        const double sv = sizeof(T) == 4 ? (double)shi[e] + (double)slo[e] : sd[e];
        if (tiled) {
          if (isA) {
            o[n * n + i * n + j] = sv;
          } else {
            o[i * n + j] = sv;
            o[j * n + i] = sv;
          }
        } else {
          const double av = sizeof(T) == 4 ? (double)ahi[e] + (double)alo[e] : ad[e];
          o[i * n + j] = sv;
          o[n * n + i * n + j] = av;
        }
      }
    }
}

// ---------------------------------------------------------------------------------------------
// Subspace solve, one CTA per fragment (FP64 results): S = L L^T, Hs = L^-1 A L^-T, eigenpairs of
// Hs, C = L^-T Q sorted by eigenvalue.  The eigensolve is cyclic Jacobi (round-robin ordering, n/2
// disjoint rotations per round) in two precisions: FP32 sweeps take Hs to the FP32 rounding floor
// (off-diagonal ~1e-7 |Hs|) at 1/64 of the FP64 instruction cost on this part, one FP64
// Newton-Schulz step makes their rotation Q32 orthonormal to FP64 rounding, and FP64 sweeps on
// Q^T Hs Q (quadratically convergent from there, 1-3 sweeps) finish the solve.  FP64 contexts sweep
// to full convergence.  FP32/mixed contexts take the diagonal of the FP64 Q^T Hs Q as it stands:
// with off-diagonals ~1e-7 |Hs| these Rayleigh quotients are within ~1e-14/gap Ha of the
// eigenvalues, and the vectors' ~1e-7 mixing is below the FP32 rounding of the rotation that
// applies them.
// ---------------------------------------------------------------------------------------------
constexpr int SNT = 512;

template <typename T>
__device__ __forceinline__ T block_sum_t(T v, T *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T s = T(0);
  for (int i = 0; i < SNT / 32; ++i) s += red[i];
  __syncthreads();
  return s;  // all threads
}

// Cyclic Jacobi on the symmetric np x np matrix M (leading dimension ld), V <- V J, all arithmetic
// in T.  Before each sweep the off-diagonal and diagonal sums of squares are formed; the solve
// stops when off <= rel (dia + off), when off is already below stall (dia + off) and the last sweep
// failed to cut it fourfold (the rounding floor: quadratic convergence would cut it by orders of
// magnitude), or after max_sweeps sweeps.  A rotation is skipped when
// |a_pq| <= skip sqrt|a_pp a_qq|.  rc, rs, red: shared scratch of T.
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

template <typename T>
__device__ void jacobi_sweeps(T *M, T *V, int np, int ld, int max_sweeps, T rel, T stall, T skip, T *red, T *rc,
                              T *rs, int *rp, int *rq) {
  const int tid = threadIdx.x;
  const int half = np / 2;
  T prev = T(-1);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    T off = T(0), dia = T(0);
    for (int t = tid; t < np * np; t += SNT) {
      const int i = t / np, j = t - i * np;
      const T v = M[i * ld + j];
      if (i == j) dia += v * v;
      else off += v * v;
    }
    off = block_sum_t<T>(off, red);
    dia = block_sum_t<T>(dia, red);
    if (!(off > rel * (dia + off))) break;
    if (prev >= T(0) && off <= stall * (dia + off) && off > T(0.25) * prev) break;
    prev = off;
    for (int r = 0; r < np - 1; ++r) {
      if (tid < half) {
        int p, q;
        if (tid == 0) {
          p = r;
          q = np - 1;
        } else {
          p = (r + tid) % (np - 1);
          q = (r - tid + (np - 1)) % (np - 1);
        }
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        const T app = M[p * ld + p], aqq = M[q * ld + q], apq = M[q * ld + p];
        T c = T(1), sn = T(0);
        if (apq != T(0) && fabs(apq) > skip * sqrt(fabs(app * aqq))) {
          // one division per rotation: sqrt(1 + tau^2) = (1 + tau^2) rsqrt(1 + tau^2), c = rsqrt(1 + t^2)
          const T tau = (aqq - app) / (T(2) * apq);
          const T w = T(1) + tau * tau;
          const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + w * rsqrt_t(w));
          c = rsqrt_t(T(1) + t * t);
          sn = t * c;
        }
        rp[tid] = p;
        rq[tid] = q;
        rc[tid] = c;
        rs[tid] = sn;
      }
      __syncthreads();
      // A <- J^T A J: the round's rotations act on disjoint index pairs, so each 2 x 2 block (row
      // pair k, column pair l) takes its row rotation and then its column rotation in one pass;
      // V <- V J on the same pass (V is not read by the block updates)
      for (int t = tid; t < half * half; t += SNT) {
        const int k = t / half, l = t - k * half;
        const T sk = rs[k], sl = rs[l];
        if (sk == T(0) && sl == T(0)) continue;
        const int pk = rp[k], qk = rq[k], pl = rp[l], ql = rq[l];
        const T ck = rc[k], cl = rc[l];
        const T a = M[pk * ld + pl], b = M[pk * ld + ql], c = M[qk * ld + pl], d = M[qk * ld + ql];
        const T a1 = ck * a - sk * c, b1 = ck * b - sk * d;
        const T c1 = sk * a + ck * c, d1 = sk * b + ck * d;
        M[pk * ld + pl] = cl * a1 - sl * b1;
        M[pk * ld + ql] = sl * a1 + cl * b1;
        M[qk * ld + pl] = cl * c1 - sl * d1;
        M[qk * ld + ql] = sl * c1 + cl * d1;
      }
      for (int t = tid; t < half * np; t += SNT) {
        const int k = t / np, i = t - k * np;
        const T sn = rs[k];
        if (sn == T(0)) continue;
        const int p = rp[k], q = rq[k];
        const T c = rc[k];
        const T vp = V[i * ld + p], vq = V[i * ld + q];
        V[i * ld + p] = c * vp - sn * vq;
        V[i * ld + q] = sn * vp + c * vq;
      }
      __syncthreads();
    }
  }
}

// Upper-triangle index t in [0, np (np + 1) / 2) -> (i, j) with i <= j, row-major.  Threads walk the
// triangle itself: masked lanes would still occupy the FP64 pipe.
__device__ __forceinline__ void tri_ij(int t, int np, int &i, int &j) {
  const float b = 2.f * np + 1.f;
  int r = (int)((b - sqrtf(b * b - 8.f * (float)t)) * 0.5f);
  r = max(0, min(r, np - 1));
  while (r > 0 && r * (2 * np - r + 1) / 2 > t) --r;
  while ((r + 1) * (2 * np - r) / 2 <= t) ++r;
  i = r;
  j = t - r * (2 * np - r + 1) / 2 + r;
}

__global__ void __launch_bounds__(SNT) k_subspace(const FragDesc *desc, const long long *goff, const int *gnchunk,
                                                  const double *gram, double dV, double *eps, double *C64,
                                                  float *C32, unsigned *flags, int fp64_sweeps,
                                                  const int *order, const float *cnl, const ProjSlot *slots,
                                                  const double *Datom) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int f = order[blockIdx.x];
  const FragDesc D = desc[f];
  const int n = D.norb;
  const int np = n + (n & 1);  // even size for the round-robin pairing (index n is a dummy)
  const int ld = np + 1;
  double *M0 = reinterpret_cast<double *>(smem_raw);  // S -> L; FP32 Jacobi arrays; V
  double *M1 = M0 + np * ld;                          // L^-1
  double *M2 = M1 + np * ld;                          // A -> Hs -> Q^T Hs Q -> diag
  double *M3 = M2 + np * ld;                          // X; Q32 promoted; Hs Q
  double *M4 = M3 + np * ld;                          // Newton-Schulz factor; Q^T Hs Q unsymmetrised
  __shared__ double red[SNT / 32];
  __shared__ double rc[32], rs[32];
  __shared__ float redf[SNT / 32], rcf[32], rsf[32];
  __shared__ int rp[32], rq[32];
  __shared__ int failed;
  __shared__ double pinv, dinv[DC_MAX_NORB];
  const int tid = threadIdx.x;
  if (tid == 0) failed = 0;

  // 1. reduce the chunk partials in a fixed order
  const double *g = gram + goff[f];
  const int nch = gnchunk[f];
  for (int t = tid; t < np * np; t += SNT) {
    const int i = t / np, j = t - i * np;
    double s = 0.0, a = 0.0;
    if (i < n && j < n) {
      for (int ch = 0; ch < nch; ++ch) {
        s += g[(long long)ch * 2 * n * n + i * n + j];
        a += g[(long long)ch * 2 * n * n + n * n + i * n + j];
      }
      s *= dV;
      a *= dV;
    }
    M0[i * ld + j] = s;
    M2[i * ld + j] = a;
  }
  __syncthreads();

  // 1b. H Y held only the local part of H: A += sum_a D_a <p_a|y_i> <p_a|y_j> from the block's projections
  // (orbital-major n x A per fragment), staged with an odd row pitch in the space of M3 and M4, which step 4
  // fills (read from global memory instead when n + 1 rows of A do not fit there); FP32 products and sums,
  // like the contraction of the rest of A
  if (cnl) {
    const int A = D.natom, ap = A | 1;
    const float *cf = cnl + D.c_off;
    float *cs = reinterpret_cast<float *>(M3);
    const bool staged = (size_t)(n + 1) * ap <= (size_t)4 * np * ld;
    if (staged) {
      for (int t = tid; t < n * A; t += SNT) {
        const int i = t / A, k = t - i * A;
        cs[i * ap + k] = cf[t];
      }
      for (int k = tid; k < A; k += SNT) cs[n * ap + k] = float(Datom[slots[D.at_off + k].atom]);
      __syncthreads();
    }
    for (int t = tid; t < n * n; t += SNT) {
      const int i = t / n, j = t - i * n;
      float acc = 0.f;
      for (int k = 0; k < A; ++k) {
        const float dk = staged ? cs[n * ap + k] : float(Datom[slots[D.at_off + k].atom]);
        const float ci = staged ? cs[i * ap + k] : cf[i * A + k], cj = staged ? cs[j * ap + k] : cf[j * A + k];
        acc = fmaf(dk * ci, cj, acc);
      }
      M2[i * ld + j] += (double)acc;
    }
    __syncthreads();
  }

  // 2. Cholesky S = L L^T (lower, in M0)
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const double d = M0[k * ld + k];
      if (!(d > 0.0) || !isfinite(d)) {
        failed = 1;
        M0[k * ld + k] = 1.0;
        pinv = 1.0;
      } else {
        const double r = rsqrt(d);  // one reciprocal square root: L_kk = d r, the column scales by r
        M0[k * ld + k] = d * r;
        pinv = r;
      }
    }
    __syncthreads();
    const double rp = pinv;
    for (int i = k + 1 + tid; i < n; i += SNT) M0[i * ld + k] *= rp;
    __syncthreads();
    const int m = n - k - 1;
    for (int t = tid; t < m * m; t += SNT) {
      const int i = k + 1 + t / m, j = k + 1 + t % m;
      if (j <= i) M0[i * ld + j] -= M0[i * ld + k] * M0[j * ld + k];
    }
    __syncthreads();
  }
  if (failed) {
    if (tid == 0) atomicOr(flags, DC_FLAG_NOTSPD);
    return;
  }

  // 3. L^-1 (lower) by forward substitution, one column per thread; the diagonal's reciprocals once,
  // each dot product in four independent FP64 chains
  for (int i = tid; i < n; i += SNT) dinv[i] = 1.0 / M0[i * ld + i];
  __syncthreads();
  for (int j = tid; j < np; j += SNT) {
    for (int i = 0; i < np; ++i) M1[i * ld + j] = 0.0;
    if (j < n) {
      for (int i = j; i < n; ++i) {
        const double *Li = M0 + i * ld;
        double s0 = (i == j) ? 1.0 : 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int k = j;
        for (; k + 3 < i; k += 4) {
          s0 = fma(-Li[k], M1[k * ld + j], s0);
          s1 = fma(-Li[k + 1], M1[(k + 1) * ld + j], s1);
          s2 = fma(-Li[k + 2], M1[(k + 2) * ld + j], s2);
          s3 = fma(-Li[k + 3], M1[(k + 3) * ld + j], s3);
        }
        for (; k < i; ++k) s0 = fma(-Li[k], M1[k * ld + j], s0);
        M1[i * ld + j] = ((s0 + s1) + (s2 + s3)) * dinv[i];
      }
    }
  }
  __syncthreads();
  // 4. X = L^-1 A (M3), Hs = X L^-T (M2), symmetrised
  for (int t = tid; t < n * n; t += SNT) {
    const int i = t / n, j = t - i * n;
    double s = 0.0;
    for (int k = 0; k <= i; ++k) s += M1[i * ld + k] * M2[k * ld + j];
    M3[i * ld + j] = s;
  }
  __syncthreads();
  for (int t = tid; t < n * n; t += SNT) {
    const int i = t / n, j = t - i * n;
    double s = 0.0;
    for (int k = 0; k <= j; ++k) s += M3[i * ld + k] * M1[j * ld + k];
    M4[i * ld + j] = s;
  }
  __syncthreads();
  // symmetrised Hs in M2 (FP64) and its FP32 copy plus Q32 = I in M0's space
  float *Mf = reinterpret_cast<float *>(M0);
  float *Vf = Mf + np * ld;
  for (int t = tid; t < np * np; t += SNT) {
    const int i = t / np, j = t - i * np;
    double v = 0.0;
    if (i < n && j < n) v = 0.5 * (M4[i * ld + j] + M4[j * ld + i]);
    M2[i * ld + j] = v;
    Mf[i * ld + j] = (float)v;
    Vf[i * ld + j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();

  // 5a. FP32 Jacobi to the FP32 rounding floor
  jacobi_sweeps<float>(Mf, Vf, np, ld, 30, 1e-12f, 0.f, 1e-9f, redf, rcf, rsf, rp, rq);
  // 5b. Q = Q32 (3 I - Q32^T Q32) / 2 in FP64 (orthonormal to FP64 rounding; Q32^T Q32 = I + O(1e-7))
  for (int t = tid; t < np * np; t += SNT) {
    const int i = t / np, j = t - i * np;
    M3[i * ld + j] = (double)Vf[i * ld + j];
  }
  __syncthreads();
  const int ntri = np * (np + 1) / 2;
  for (int t = tid; t < ntri; t += SNT) {
    int i, j;
    tri_ij(t, np, i, j);
    double s = 0.0;
    for (int k = 0; k < np; ++k) s += M3[k * ld + i] * M3[k * ld + j];
    const double v = 0.5 * ((i == j ? 3.0 : 0.0) - s);
    M4[i * ld + j] = v;
    M4[j * ld + i] = v;
  }
  __syncthreads();
  for (int t = tid; t < np * np; t += SNT) {
    const int i = t / np, j = t - i * np;
    double s = 0.0;
    for (int k = 0; k < np; ++k) s += M3[i * ld + k] * M4[k * ld + j];
    M0[i * ld + j] = s;  // Q
  }
  __syncthreads();
  // 5c. Q^T Hs Q (FP64), symmetrised
  for (int t = tid; t < np * np; t += SNT) {
    const int i = t / np, j = t - i * np;
    double s = 0.0;
    for (int k = 0; k < np; ++k) s += M2[i * ld + k] * M0[k * ld + j];
    M3[i * ld + j] = s;
  }
  __syncthreads();
  // Q^T (Hs Q) is symmetric up to rounding: form the upper triangle and mirror it
  for (int t = tid; t < ntri; t += SNT) {
    int i, j;
    tri_ij(t, np, i, j);
    double s = 0.0;
    for (int k = 0; k < np; ++k) s += M0[k * ld + i] * M3[k * ld + j];
    M2[i * ld + j] = s;
    M2[j * ld + i] = s;
  }
  __syncthreads();
  // 5d. FP64 Jacobi from there
  jacobi_sweeps<double>(M2, M0, np, ld, fp64_sweeps, 1e-30, 1e-20, 1e-18, red, rc, rs, rp, rq);

  // 6. sort ascending (rank by value, ties by index) and C = L^-T V
  __shared__ int rank[DC_MAX_NORB];
  for (int i = tid; i < n; i += SNT) {
    const double li = M2[i * ld + i];
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = M2[j * ld + j];
      rk += (lj < li) || (lj == li && j < i);
    }
    rank[i] = rk;
    eps[D.st_off + rk] = li;
    if (!isfinite(li)) atomicOr(flags, DC_FLAG_NONFINITE);
  }
  __syncthreads();
  for (int t = tid; t < n * n; t += SNT) {
    const int k = t / n, i = t - k * n;  // C[k][rank[i]] = sum_{m>=k} Linv[m][k] V[m][i]
    double s = 0.0;
    for (int m = k; m < n; ++m) s += M1[m * ld + k] * M0[m * ld + i];
    const long long o = D.sub_off + (long long)k * n + rank[i];
    C64[o] = s;
    if (C32) C32[o] = (float)s;
  }
}

// ---------------------------------------------------------------------------------------------
// Rotation out[i][p] = sum_k C[k][i] Y[k][p].  One CTA per (fragment, 128-point chunk); thread
// (pq, og) owns points 4pq..4pq+3 and orbitals 8og..8og+7.
// ---------------------------------------------------------------------------------------------
constexpr int RCH = 128;
constexpr int RPAD = RCH + 4;

template <typename T>
__global__ void __launch_bounds__(256) k_rotate(const FragDesc *desc, const int2 *ritems, const T *C, const T *Y,
                                                T *out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 it = ritems[blockIdx.x];
  const int f = it.x, ch = it.y;
  const FragDesc D = desc[f];
  const int n = D.norb;
  const long long P = (long long)D.E[0] * D.E[1] * D.E[2];
  const long long p0 = (long long)ch * RCH;
  T *sY = reinterpret_cast<T *>(smem_raw);  // [n][RPAD]
  T *sC = sY + DC_MAX_NORB * RPAD;          // [n][64]
  const T *Cf = C + D.sub_off;
  for (int t = threadIdx.x; t < n * DC_MAX_NORB; t += 256) {
    const int k = t / DC_MAX_NORB, i = t - k * DC_MAX_NORB;
    sC[t] = i < n ? Cf[k * n + i] : T(0);
  }
  const T *Yf = Y + D.psi_off;
  for (int t = threadIdx.x; t < n * RCH; t += 256) {
    const int k = t / RCH, p = t - k * RCH;
    const long long pp = p0 + p;
    sY[k * RPAD + p] = pp < P ? Yf[(long long)k * P + pp] : T(0);
  }
  __syncthreads();
  const int pq = threadIdx.x & 31, og = threadIdx.x >> 5;
  if (8 * og >= n) return;
  T acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int k = 0; k < n; ++k) {
    const Vec4<T> y = ld4(&sY[k * RPAD + 4 * pq]);
    const Vec4<T> c0 = ld4(&sC[k * DC_MAX_NORB + 8 * og]);
    const Vec4<T> c1 = ld4(&sC[k * DC_MAX_NORB + 8 * og + 4]);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        acc[a][b] += c0.v[a] * y.v[b];
        acc[a + 4][b] += c1.v[a] * y.v[b];
      }
    }
  }
  T *of = out + D.psi_off;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int i = 8 * og + a;
    if (i >= n) break;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const long long pp = p0 + 4 * pq + b;
      if (pp < P) of[(long long)i * P + pp] = acc[a][b];
    }
  }
}

// FP32 rotation out[i][p] = sum_k C[k][i] Y[k][p] with paired FP32 FMAs.  One CTA per (fragment,
// 256-point chunk); warp w owns output orbitals [w OPT, (w + 1) OPT) (OPT = ceil(max n / 8)), lane l
// the points 4l..4l+3 and 128+4l..128+4l+3 (two conflict-free 16-byte shared loads per k); C is
// splatted over point pairs in shared memory and read as a warp broadcast.
constexpr int R2CH = 256;
constexpr int R2PAD = R2CH + 4;

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <int OPT>
__global__ void __launch_bounds__(256) k_rotate32(const FragDesc *desc, const int2 *ritems, const float *C,
                                                  const float *Y, float *out, int nmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 it = ritems[blockIdx.x];
  const int f = it.x, ch = it.y;
  const FragDesc D = desc[f];
  const int n = D.norb;
  const long long P = (long long)D.E[0] * D.E[1] * D.E[2];
  const long long p0 = (long long)ch * R2CH;
  constexpr int NC = 8 * OPT;                                     // padded orbital count
  float *sY = reinterpret_cast<float *>(smem_raw);               // [n][R2PAD]
  float2 *sC = reinterpret_cast<float2 *>(sY + nmax * R2PAD);  // [n][NC] splatted
  const float *Cf = C + D.sub_off;
  const float *Yf = Y + D.psi_off;
  const bool vec = ((P | D.psi_off) & 3) == 0;
  if (vec) {
    // Every 16-byte copy of the Y tile in flight at once; a quad past the fragment's end is zero-filled
    // (P is a multiple of 4, so a quad is either wholly inside or wholly outside).
    for (int t = threadIdx.x; t < n * (R2CH / 4); t += 256) {
      const int k = t / (R2CH / 4), q = t - k * (R2CH / 4);
      const long long pp = p0 + 4 * q;
      const float *src = Yf + (long long)k * P + (pp < P ? pp : 0);
      const unsigned dst = (unsigned)__cvta_generic_to_shared(sY + k * R2PAD + 4 * q);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(pp < P ? 16 : 0)
                   : "memory");
    }
  } else {
    for (int t = threadIdx.x; t < n * (R2CH / 4); t += 256) {
      const int k = t / (R2CH / 4), q = t - k * (R2CH / 4);
      const long long pp = p0 + 4 * q;
      const float *row = Yf + (long long)k * P;
      float4 v;
      v.x = pp < P ? row[pp] : 0.f;
      v.y = pp + 1 < P ? row[pp + 1] : 0.f;
      v.z = pp + 2 < P ? row[pp + 2] : 0.f;
      v.w = pp + 3 < P ? row[pp + 3] : 0.f;
      *reinterpret_cast<float4 *>(sY + k * R2PAD + 4 * q) = v;
    }
  }
  // C splatted to (c, c) pairs: the loads of one thread are independent and issued together.
  constexpr int CPT = (8 * OPT * 8 * OPT + 255) / 256;
  float cv[CPT];
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    const int t = threadIdx.x + 256 * j, k = t / NC, i = t - k * NC;
    cv[j] = (k < n && i < n) ? Cf[k * n + i] : 0.f;
  }
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    const int t = threadIdx.x + 256 * j;
    if (t < n * NC) sC[t] = make_float2(cv[j], cv[j]);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i0 = w * OPT;
  if (i0 >= n) return;
  float2 acc[OPT][4];
#pragma unroll
  for (int o = 0; o < OPT; ++o)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[o][b] = make_float2(0.f, 0.f);
  for (int k = 0; k < n; ++k) {
    const float4 ya = *reinterpret_cast<const float4 *>(sY + k * R2PAD + 4 * lane);
    const float4 yb = *reinterpret_cast<const float4 *>(sY + k * R2PAD + 128 + 4 * lane);
    const float2 y0 = make_float2(ya.x, ya.y), y1 = make_float2(ya.z, ya.w);
    const float2 y2 = make_float2(yb.x, yb.y), y3 = make_float2(yb.z, yb.w);
    const float2 *cr = sC + k * NC + i0;
#pragma unroll
    for (int o = 0; o < OPT; ++o) {
      const float2 c = cr[o];
      acc[o][0] = ffma2(c, y0, acc[o][0]);
      acc[o][1] = ffma2(c, y1, acc[o][1]);
      acc[o][2] = ffma2(c, y2, acc[o][2]);
      acc[o][3] = ffma2(c, y3, acc[o][3]);
    }
  }
  float *of = out + D.psi_off;
#pragma unroll
  for (int o = 0; o < OPT; ++o) {
    const int i = i0 + o;
    if (i >= n) break;
    float *row = of + (long long)i * P;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long pp = p0 + 128 * h + 4 * lane;
      const float4 v = make_float4(acc[o][2 * h].x, acc[o][2 * h].y, acc[o][2 * h + 1].x, acc[o][2 * h + 1].y);
      if (vec && pp + 3 < P) {
        *reinterpret_cast<float4 *>(row + pp) = v;
      } else {
        if (pp < P) row[pp] = v.x;
        if (pp + 1 < P) row[pp + 1] = v.y;
        if (pp + 2 < P) row[pp + 2] = v.z;
        if (pp + 3 < P) row[pp + 3] = v.w;
      }
    }
  }
}

// Projections of the rotated block, per fragment: cout[i][k] = sum_j C[j][i] cin[j][k].  C maps the
// filtered block to Psi = Y C, so <p_k|Psi_i> = sum_j C[j][i] <p_k|Y_j>.
template <typename T>
__global__ void __launch_bounds__(256) k_rotate_proj(const FragDesc *desc, const T *C, const T *cin, T *cout) {
  const FragDesc D = desc[blockIdx.x];
  const int n = D.norb, A = D.natom;
  const T *Cf = C + D.sub_off;
  const T *ci = cin + D.c_off;
  T *co = cout + D.c_off;
  for (int t = threadIdx.x; t < n * A; t += 256) {
    const int i = t / A, k = t - i * A;
    T s = T(0);
    for (int j = 0; j < n; ++j) s += Cf[j * n + i] * ci[j * A + k];
    co[t] = s;
  }
}


// ---------------------------------------------------------------------------------------------
// DC-LCFO basis (Sec. 2.3, Eqs. 6-7).  One CTA per fragment: orbitals with eps_i < eps_cut (in
// orbital order) are projected onto the core, their overlap S_ij = dV sum_core phi_i phi_j is
// accumulated in FP64 over 64-point core tiles (each thread keeps its upper-triangle entries in
// registers), S is diagonalised by the FP64 Jacobi above, eigenvalues are ranked in descending order
// (ties by index), the directions with s > lambda_cut are kept, and the basis
// lambda_k = sum_i phibar_i U_ik / sqrt(s_k) is written on the core points (x fastest).
// ---------------------------------------------------------------------------------------------
constexpr int LCH = 64;                               // core points per tile
constexpr int LTS = LCH + 1;                          // tile row stride (rows of a warp on different banks)
constexpr int LTRI = (DC_MAX_NORB * (DC_MAX_NORB + 1) / 2 + SNT - 1) / SNT;  // triangle entries per thread

__device__ __forceinline__ long long core_point(const FragDesc &D, long long cp) {
  const long long cxy = (long long)D.c[0] * D.c[1];
  const int cz = (int)(cp / cxy);
  const long long r = cp - cz * cxy;
  const int cy = (int)(r / D.c[0]), cx = (int)(r - (long long)cy * D.c[0]);
  return (long long)(D.b[0] + cx) + (long long)D.E[0] * ((D.b[1] + cy) + (long long)D.E[1] * (D.b[2] + cz));
}

template <typename T>
__device__ __forceinline__ void lcfo_tile(const FragDesc &D, const T *psi, long long P, const int *sel, int nsel,
                                          long long ncore, long long cp0, double *tile) {
  for (int t = threadIdx.x; t < nsel * LCH; t += SNT) {
    const int i = t / LCH, p = t - i * LCH;
    const long long cp = cp0 + p;
    tile[i * LTS + p] = cp < ncore ? (double)psi[D.psi_off + (long long)sel[i] * P + core_point(D, cp)] : 0.0;
  }
}

template <typename T>
__global__ void __launch_bounds__(SNT) k_lcfo(const FragDesc *desc, const T *psi, const double *eps, double eps_cut,
                                              double lambda_cut, double dV, double *basis, int *nbasis,
                                              double *s_out, int f_lo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int LD = DC_MAX_NORB + 1;
  double *S = reinterpret_cast<double *>(smem_raw);  // [np][LD] overlap -> eigenvalues; then W
  double *V = S + DC_MAX_NORB * LD;                   // [np][LD] eigenvectors
  double *tile = V + DC_MAX_NORB * LD;                // [nsel][LTS]
  __shared__ double red[SNT / 32], rc[32], rs[32], sv[DC_MAX_NORB], vn[DC_MAX_NORB];
  __shared__ float redf[SNT / 32], rcf[32], rsf[32];
  __shared__ long long redl[SNT / 32];
  __shared__ int rp[32], rq[32], sel[DC_MAX_NORB], perm[DC_MAX_NORB], nsel_s;
  const int f = f_lo + blockIdx.x, tid = threadIdx.x;
  const FragDesc D = desc[f];
  const int n = D.norb;
  const long long P = (long long)D.E[0] * D.E[1] * D.E[2];
  const long long ncore = (long long)D.c[0] * D.c[1] * D.c[2];

  // element offset of this fragment's rows: sum over the fragments before it of n |core|
  long long part = 0;
  for (int g = tid; g < f; g += SNT) part += (long long)desc[g].norb * desc[g].c[0] * desc[g].c[1] * desc[g].c[2];
  const long long off = block_sum_t<long long>(part, redl);
  double *out = basis + off;

  if (tid == 0) {
    int k = 0;
    for (int i = 0; i < n; ++i)
      if (eps[D.st_off + i] < eps_cut) sel[k++] = i;
    nsel_s = k;
  }
  __syncthreads();
  const int nsel = nsel_s;
  const int np = nsel + (nsel & 1);  // even size for the round-robin pairing (index nsel is a dummy)
  const int ntri = nsel * (nsel + 1) / 2;

  // 1. S = dV sum over core points of phibar_i phibar_j (upper triangle)
  double acc[LTRI];
#pragma unroll
  for (int r = 0; r < LTRI; ++r) acc[r] = 0.0;
  for (long long cp0 = 0; cp0 < ncore && nsel > 0; cp0 += LCH) {
    lcfo_tile<T>(D, psi, P, sel, nsel, ncore, cp0, tile);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < LTRI; ++r) {
      const int t = tid + r * SNT;
      if (t < ntri) {
        int i, j;
        tri_ij(t, nsel, i, j);
        const double *a = tile + i * LTS, *b = tile + j * LTS;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;  // four independent FP64 chains
#pragma unroll 4
        for (int p = 0; p < LCH; p += 4) {
          s0 = fma(a[p], b[p], s0);
          s1 = fma(a[p + 1], b[p + 1], s1);
          s2 = fma(a[p + 2], b[p + 2], s2);
          s3 = fma(a[p + 3], b[p + 3], s3);
        }
        acc[r] += (s0 + s1) + (s2 + s3);
      }
    }
    __syncthreads();
  }
  for (int t = tid; t < np * np; t += SNT) {
    const int i = t / np, j = t - i * np;
    S[i * LD + j] = 0.0;
    V[i * LD + j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < LTRI; ++r) {
    const int t = tid + r * SNT;
    if (t < ntri) {
      int i, j;
      tri_ij(t, nsel, i, j);
      S[i * LD + j] = dV * acc[r];
      S[j * LD + i] = dV * acc[r];
    }
  }
  __syncthreads();

  // 2. S = U diag(s) U^T.  As in the subspace solve: FP32 Jacobi on a float copy to the FP32 floor,
  // one FP64 Newton-Schulz step makes its vectors Q orthonormal to ~1e-11, and FP64 Jacobi on
  // B = Q^T S Q (off-diagonal ~1e-7) converges quadratically, accumulating U = Q J.  The tile's space
  // is idle here: it holds the float copies, then B.  Every FP64 product goes through registers
  // (at most RPT entries per thread), a barrier, and an in-place write.
  if (np > 0) {
    constexpr int RPT = (DC_MAX_NORB * DC_MAX_NORB + SNT - 1) / SNT;
    float *Sf = reinterpret_cast<float *>(tile), *Vf = Sf + DC_MAX_NORB * LD;
    double *B = tile;
    double r[RPT];
    for (int t = tid; t < np * np; t += SNT) {
      const int i = t / np, j = t - i * np;
      Sf[i * LD + j] = (float)S[i * LD + j];
      Vf[i * LD + j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    jacobi_sweeps<float>(Sf, Vf, np, LD, 30, 1e-12f, 0.f, 1e-9f, redf, rcf, rsf, rp, rq);
    for (int t = tid; t < np * np; t += SNT) {
      const int i = t / np, j = t - i * np;
      V[i * LD + j] = (double)Vf[i * LD + j];  // Q32
    }
    __syncthreads();
    // One Newton-Schulz step Q <- Q (3 I - Q^T Q) / 2 takes the FP32 vectors' drift from
    // orthonormality (up to ~1e-5 after many rotations) to ~1e-11; the eigenvalues below are then
    // Rayleigh quotients normalised by |u_i|^2, which removes that residue to first order.  F goes
    // through B's space (the float copies are dead), every product through registers.
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int t = tid + q * SNT;
      r[q] = 0.0;
      if (t < np * np) {
        const int i = t / np, j = t - i * np;
        double a = 0.0;
        for (int k = 0; k < np; ++k) a = fma(V[k * LD + i], V[k * LD + j], a);
        r[q] = 0.5 * ((i == j ? 3.0 : 0.0) - a);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int t = tid + q * SNT;
      if (t < np * np) B[(t / np) * LD + t % np] = r[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int t = tid + q * SNT;
      r[q] = 0.0;
      if (t < np * np) {
        const int i = t / np, j = t - i * np;
        double a = 0.0;
        for (int k = 0; k < np; ++k) a = fma(V[i * LD + k], B[k * LD + j], a);
        r[q] = a;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int t = tid + q * SNT;
      if (t < np * np) V[(t / np) * LD + t % np] = r[q];
    }
    __syncthreads();
    // W = S Q (into S), B = Q^T W (into B), each through registers
    for (int stage = 1; stage < 3; ++stage) {
      const double *X = stage == 1 ? S : V;
      const double *Y = stage == 1 ? V : S;
      double *Z = stage == 1 ? S : B;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int t = tid + q * SNT;
        r[q] = 0.0;
        if (t < np * np) {
          const int i = t / np, j = t - i * np;
          double a = 0.0;
          if (stage == 2)
            for (int k = 0; k < np; ++k) a = fma(X[k * LD + i], Y[k * LD + j], a);  // Q^T W
          else
            for (int k = 0; k < np; ++k) a = fma(X[i * LD + k], Y[k * LD + j], a);
          r[q] = a;
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int t = tid + q * SNT;
        if (t < np * np) Z[(t / np) * LD + t % np] = r[q];
      }
      __syncthreads();
    }
    // symmetrise B (equal to Q^T S Q up to rounding)
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int t = tid + q * SNT;
      r[q] = 0.0;
      if (t < np * np) {
        const int i = t / np, j = t - i * np;
        r[q] = 0.5 * (B[i * LD + j] + B[j * LD + i]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int t = tid + q * SNT;
      if (t < np * np) B[(t / np) * LD + t % np] = r[q];
    }
    __syncthreads();
    jacobi_sweeps<double>(B, V, np, LD, 40, 1e-30, 1e-20, 1e-18, red, rc, rs, rp, rq);
    // u_i = Q J e_i: B_ii = u_i^T S u_i, and s_i = B_ii / |u_i|^2; the columns are normalised
    for (int i = tid; i < nsel; i += SNT) {
      double nrm = 0.0;
      for (int k = 0; k < np; ++k) nrm = fma(V[k * LD + i], V[k * LD + i], nrm);
      sv[i] = B[i * LD + i] / nrm;
      vn[i] = rsqrt(nrm);
    }
  }
  __syncthreads();

  // 3. rank descending (ties by index), keep s > lambda_cut
  for (int i = tid; i < nsel; i += SNT) {
    int r = 0;
    for (int k = 0; k < nsel; ++k) r += (sv[k] > sv[i]) || (sv[k] == sv[i] && k < i);
    perm[r] = i;
  }
  __syncthreads();
  int m = 0;
  for (int k = 0; k < nsel; ++k) m += sv[k] > lambda_cut;
  if (tid == 0) nbasis[f] = m;
  for (int r = tid; r < n; r += SNT) s_out[D.st_off + r] = r < nsel ? sv[perm[r]] : 0.0;
  // W[i][k] = U[i][perm k] / sqrt(s_perm k) over the kept directions (into S's space)
  for (int t = tid; t < nsel * m; t += SNT) {
    const int i = t / m, k = t - i * m;
    S[i * LD + k] = V[i * LD + perm[k]] * vn[perm[k]] / sqrt(sv[perm[k]]);
  }
  __syncthreads();

  // 4. lambda_k on the core points; rows m <= k < n are zero
  for (long long cp0 = 0; cp0 < ncore; cp0 += LCH) {
    if (m > 0) lcfo_tile<T>(D, psi, P, sel, nsel, ncore, cp0, tile);
    __syncthreads();
    for (int t = tid; t < m * LCH; t += SNT) {  // kept rows: two independent FP64 chains per output
      const int k = t / LCH, p = t - k * LCH;
      const long long cp = cp0 + p;
      double v0 = 0.0, v1 = 0.0;
      int i = 0;
      for (; i + 1 < nsel; i += 2) {
        v0 = fma(tile[i * LTS + p], S[i * LD + k], v0);
        v1 = fma(tile[(i + 1) * LTS + p], S[(i + 1) * LD + k], v1);
      }
      if (i < nsel) v0 = fma(tile[i * LTS + p], S[i * LD + k], v0);
      if (cp < ncore) out[(long long)k * ncore + cp] = v0 + v1;
    }
    for (int t = m * LCH + tid; t < n * LCH; t += SNT) {  // rows m <= k < n
      const int k = t / LCH, p = t - k * LCH;
      const long long cp = cp0 + p;
      if (cp < ncore) out[(long long)k * ncore + cp] = 0.0;
    }
    __syncthreads();
  }
}

}  // namespace

namespace dck {

int launch_bounds(dc_ctx *c, int, cudaStream_t s) {
  const int m = c->params.cheb_degree;
  const int nf = c->f_hi - c->f_lo;
  if (nf <= 0) return DC_OK;
  k_bounds<<<(nf + 127) / 128, 128, 0, s>>>(c->d_desc, c->f_lo, c->f_hi, c->d_eps, c->d_bounds, m, 4 + 2 * m);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

template <typename T>
int launch_gram(dc_ctx *c, const T *Y, const T *HY, cudaStream_t s) {
  k_gram<T><<<c->n_gram_items, 256, 0, s>>>(c->d_desc, c->d_gram_items, c->d_gram_off, c->gram_chunk, Y, HY,
                                            c->d_gram);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

int launch_subspace(dc_ctx *c, int precision_bits, double *eps, cudaStream_t s, const float *cnl) {
  const int np = c->layout.max_norb + (c->layout.max_norb & 1);
  const size_t sm = 5 * (size_t)np * (np + 1) * sizeof(double);
  DC_CUDA(dc_set_smem((const void *)k_subspace, sm));
  const int fp64_sweeps = precision_bits == 32 ? 0 : 40;
  const int nf = c->f_hi - c->f_lo;
  if (nf <= 0) return DC_OK;
  k_subspace<<<nf, SNT, sm, s>>>(c->d_desc, c->d_gram_off, c->d_gram_nchunk, c->d_gram, c->dV, eps, c->d_C64,
                                 precision_bits == 32 ? c->d_C32 : nullptr, c->d_flags, fp64_sweeps, c->d_frag_order,
                                 cnl, c->d_slots, c->d_atom_D);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

template <typename T>
int launch_rotate(dc_ctx *c, const T *Y, T *out, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    // tensor cores where the context qualifies (at most 64 orbitals, 16-byte aligned point rows)
    if (launch_rotate_tc(c, Y, out, s) == DC_OK) return DC_OK;
    const int opt = (c->layout.max_norb + 7) / 8;
    const int nmax = c->layout.max_norb;
    const size_t sm = (size_t)nmax * R2PAD * sizeof(float) + (size_t)nmax * 8 * opt * sizeof(float2);
    auto run = [&](auto kern) -> int {
      DC_CUDA(dc_set_smem((const void *)kern, sm));
      kern<<<c->n_rot2_items, 256, sm, s>>>(c->d_desc, c->d_rot2_items, c->d_C32, Y, out, nmax);
      DC_CUDA(cudaGetLastError());
      return DC_OK;
    };
    switch (opt) {
      case 1: return run(k_rotate32<1>);
      case 2: return run(k_rotate32<2>);
      case 3: return run(k_rotate32<3>);
      case 4: return run(k_rotate32<4>);
      case 5: return run(k_rotate32<5>);
      case 6: return run(k_rotate32<6>);
      case 7: return run(k_rotate32<7>);
      default: return run(k_rotate32<8>);
    }
  }
  const size_t sm = ((size_t)DC_MAX_NORB * RPAD + (size_t)DC_MAX_NORB * DC_MAX_NORB) * sizeof(T);
  DC_CUDA(dc_set_smem((const void *)k_rotate<T>, sm));
  const T *C = nullptr;
  if (sizeof(T) == 8) C = reinterpret_cast<const T *>(c->d_C64);
  else C = reinterpret_cast<const T *>(c->d_C32);
  k_rotate<T><<<c->n_rot_items, 256, sm, s>>>(c->d_desc, c->d_rot_items, C, Y, out);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

template <typename T>
int launch_rotate_proj(dc_ctx *c, const T *cin, T *cout, cudaStream_t s) {
  const T *C = nullptr;
  if (sizeof(T) == 8) C = reinterpret_cast<const T *>(c->d_C64);
  else C = reinterpret_cast<const T *>(c->d_C32);
  const int nf = c->f_hi - c->f_lo;
  if (nf <= 0) return DC_OK;
  k_rotate_proj<T><<<nf, 256, 0, s>>>(c->d_desc + c->f_lo, C, cin, cout);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

template int launch_rotate_proj<double>(dc_ctx *, const double *, double *, cudaStream_t);
template int launch_rotate_proj<float>(dc_ctx *, const float *, float *, cudaStream_t);
template int launch_gram<double>(dc_ctx *, const double *, const double *, cudaStream_t);
template int launch_gram<float>(dc_ctx *, const float *, const float *, cudaStream_t);
template int launch_rotate<double>(dc_ctx *, const double *, double *, cudaStream_t);
template int launch_rotate<float>(dc_ctx *, const float *, float *, cudaStream_t);

template <typename T>
int launch_lcfo(dc_ctx *c, const T *psi, const double *eps, double eps_cut, double lambda_cut, double *basis,
                int *nbasis, double *s_out, cudaStream_t s) {
  const size_t sm = (2 * (size_t)DC_MAX_NORB * (DC_MAX_NORB + 1) + (size_t)DC_MAX_NORB * LTS) * sizeof(double);
  DC_CUDA(dc_set_smem((const void *)k_lcfo<T>, sm));
  const int nf = c->f_hi - c->f_lo;
  if (nf <= 0) return DC_OK;
  k_lcfo<T><<<nf, SNT, sm, s>>>(c->d_desc, psi, eps, eps_cut, lambda_cut, c->dV, basis, nbasis, s_out, c->f_lo);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}
template int launch_lcfo<double>(dc_ctx *, const double *, const double *, double, double, double *, int *, double *,
                                 cudaStream_t);
template int launch_lcfo<float>(dc_ctx *, const float *, const double *, double, double, double *, int *, double *,
                                cudaStream_t);

}  // namespace dck
