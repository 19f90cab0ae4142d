// Band-energy adjoint: the gradients of E_b = sum_f sum_i occ_i <psi_i|H_f|psi_i> with respect to
// the global potential and the projector strengths (dE/dpsi comes from the H-apply kernel in its
// adjoint mode, which recomputes H psi instead of storing it).
//
//   dE/dV(g) = dV sum over every fragment point j with idx_map[f][j] = g of sum_i occ_i psi_i(j)^2
//   dE/dD_a  = sum over the fragments that hold atom a of sum_i occ_i <p_a|psi_i>^2
//
// Both sums run in a fixed order (no atomics), so results are bitwise reproducible.
#include "dc_internal.h"

namespace {

template <typename T>
__global__ void k_frag_density(const FragDesc *desc, int nfrag, const T *psi, const double *occ, double *fd,
                               long long t0, long long total) {
  // one thread per fragment point in [t0, total); the fragment of a point is found by bisection on pt_off
  const long long t = t0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int lo = 0, hi = nfrag - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (desc[mid].pt_off <= t) lo = mid;
    else hi = mid - 1;
  }
  const FragDesc D = desc[lo];
  const long long P = (long long)D.E[0] * D.E[1] * D.E[2];
  const long long j = t - D.pt_off;
  const T *y = psi + D.psi_off + j;
  double s = 0.0;
  for (int i = 0; i < D.norb; ++i) {
    const double v = (double)y[(long long)i * P];
    s += occ[D.st_off + i] * v * v;
  }
  fd[t] = s;
}

__global__ void k_gather_dV(const FragDesc *desc, const int *Fn, const int *cbx, const int2 *cx, const int *cby,
                            const int2 *cy, const int *cbz, const int2 *cz, int nx, int ny, long long npts,
                            const double *fd, double dV, double *dVout) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npts) return;
  const int x = (int)(g % nx), y = (int)((g / nx) % ny), z = (int)(g / ((long long)nx * ny));
  double s = 0.0;
  for (int a = cbz[z]; a < cbz[z + 1]; ++a)
    for (int b = cby[y]; b < cby[y + 1]; ++b)
      for (int c = cbx[x]; c < cbx[x + 1]; ++c) {
        const int f = cx[c].x + Fn[0] * (cy[b].x + Fn[1] * cz[a].x);
        const FragDesc D = desc[f];
        const long long j = cx[c].y + (long long)D.E[0] * (cy[b].y + (long long)D.E[1] * cz[a].y);
        s += fd[D.pt_off + j];
      }
  dVout[g] = dV * s;
}

// per (fragment, atom slot): w = sum_i occ_i c_{i,k}^2
template <typename T>
__global__ void k_slot_weights(const FragDesc *desc, int nfrag, const T *cproj, const double *occ, double *w) {
  const int f = blockIdx.x;
  if (f >= nfrag) return;
  const FragDesc D = desc[f];
  for (int k = threadIdx.x; k < D.natom; k += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < D.norb; ++i) {
      const double c = (double)cproj[D.c_off + (long long)i * D.natom + k];
      s += occ[D.st_off + i] * c * c;
    }
    w[D.at_off + k] = s;
  }
}

__global__ void k_atom_sum(int natom, const int *beg, const int *slots, const double *w, double *dD) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= natom) return;
  double s = 0.0;
  for (int e = beg[a]; e < beg[a + 1]; ++e) s += w[slots[e]];
  dD[a] = s;
}

}  // namespace

namespace dck {

template <typename T>
int launch_frag_density(dc_ctx *c, const T *psi, const double *occ, double *fd, cudaStream_t s, bool shard_only) {
  long long t0 = 0, total = c->layout.frag_points;
  if (shard_only) {
    t0 = c->h_desc[c->f_lo].pt_off;
    total = c->f_hi < c->nfrag ? c->h_desc[c->f_hi].pt_off : c->layout.frag_points;
  }
  if (total <= t0) return DC_OK;
  k_frag_density<T><<<(unsigned)((total - t0 + 255) / 256), 256, 0, s>>>(c->d_desc, c->nfrag, psi, occ, fd, t0, total);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

int launch_gather_dV(dc_ctx *c, const double *fd, double *dV, cudaStream_t s) {
  k_gather_dV<<<(unsigned)((c->npts + 255) / 256), 256, 0, s>>>(
      c->d_desc, c->d_Fn, c->d_cover_beg[0], c->d_cover[0], c->d_cover_beg[1], c->d_cover[1],
      c->d_cover_beg[2], c->d_cover[2], c->grid.n[0], c->grid.n[1], c->npts, fd, c->dV, dV);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

int launch_dD(dc_ctx *c, const double *cproj64, const float *cproj32, const double *occ, double *dD, cudaStream_t s) {
  double *w = c->d_slot_w;
  if (cproj64) k_slot_weights<double><<<c->nfrag, 128, 0, s>>>(c->d_desc, c->nfrag, cproj64, occ, w);
  else k_slot_weights<float><<<c->nfrag, 128, 0, s>>>(c->d_desc, c->nfrag, cproj32, occ, w);
  if (c->natom > 0)
    k_atom_sum<<<(c->natom + 127) / 128, 128, 0, s>>>(c->natom, c->d_atom_slot_beg, c->d_atom_slots, w, dD);
  DC_CUDA(cudaGetLastError());
  return DC_OK;
}

template int launch_frag_density<double>(dc_ctx *, const double *, const double *, double *, cudaStream_t, bool);
template int launch_frag_density<float>(dc_ctx *, const float *, const double *, double *, cudaStream_t, bool);

}  // namespace dck
