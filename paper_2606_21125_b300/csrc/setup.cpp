// Host-side construction of the fragment decomposition and per-fragment projector data.
//
// Sec. 2.2 / Table 1: the cell is divided by a regular grid of num_fragment(1:3) into
// non-overlapping cores; each fragment adds num_rgrid_buffer(1:3) points on every side.  Cores on
// an axis of N points split F ways are [floor(kN/F), floor((k+1)N/F)).  Everything here is integer
// work or FP64 decisions taken in the same expression order as the FP64 oracle, so maps, atom
// lists and supports agree bit for bit.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <stdexcept>

#include "dc_internal.h"

namespace {

inline long long wrap(long long v, long long n) { return ((v % n) + n) % n; }

struct Factor {
  std::vector<double> val;
  std::vector<char> sup;
  bool any = false;
};

// 1-D projector factor on local axis d of a fragment: sum over images of
// exp(-(x - X - nL)^2/(2 sigma^2)) for |x - X - nL| < cut, x = (wrapped global index) * h.
Factor axis_factor(int org, int E, int N, double h, double L, double X, double sigma, double cut) {
  Factor F;
  F.val.assign(E, 0.0);
  F.sup.assign(E, 0);
  int K = (int)ceil(cut / L) + 1;
  for (int j = 0; j < E; ++j) {
    double x = (double)wrap((long long)org + j, N) * h;
    double t = x - X;
    double v = 0.0;
    for (int n = -K; n <= K; ++n) {
      double d = t - (double)n * L;
      if (fabs(d) < cut) {
        v += exp(-(d * d) / (2.0 * sigma * sigma));
        F.sup[j] = 1;
        F.any = true;
      }
    }
    F.val[j] = v;
  }
  return F;
}

}  // namespace

// Build every host-side table of the context.  Returns DC_OK or DC_ERR_ARG (message set).
int dc_build_host(dc_ctx *c, const dc_atoms_t *atoms, HostTables &out) {
  const int *n = c->grid.n;
  const int *F = c->frag_cfg.num_fragment;
  const int *b = c->buf_cfg.num_rgrid_buffer;
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 1 || F[d] < 1 || F[d] > n[d] || b[d] < 0 || !(c->grid.L[d] > 0.0)) {
      dc_set_error("dc_init: need n >= 1, 1 <= num_fragment <= n, num_rgrid_buffer >= 0, L > 0");
      return DC_ERR_ARG;
    }
    c->h[d] = c->grid.L[d] / n[d];
  }
  c->dV = c->h[0] * c->h[1] * c->h[2];
  c->volume = c->grid.L[0] * c->grid.L[1] * c->grid.L[2];
  c->npts = (long long)n[0] * n[1] * n[2];
  c->nfrag = F[0] * F[1] * F[2];
  if (c->nfrag > 4096) {
    dc_set_error("dc_init: at most 4096 fragments (the initial-orbital counter holds fragment indices below 4096)");
    return DC_ERR_ARG;
  }
  c->natom = atoms->natom;
  c->nspecies = atoms->nspecies;
  if (c->natom < 0 || c->nspecies < 1) {
    dc_set_error("dc_init: natom >= 0 and nspecies >= 1 required");
    return DC_ERR_ARG;
  }
  c->h_pos.assign(atoms->pos, atoms->pos + 3 * (size_t)c->natom);
  c->h_species.assign(atoms->species, atoms->species + c->natom);
  c->h_Zs.assign(atoms->Z, atoms->Z + c->nspecies);
  c->h_sigloc.assign(atoms->sigma_loc, atoms->sigma_loc + c->nspecies);
  c->h_sigproj.assign(atoms->sigma_proj, atoms->sigma_proj + c->nspecies);
  c->h_Ds.assign(atoms->D, atoms->D + c->nspecies);
  c->ne = 0.0;
  for (int a = 0; a < c->natom; ++a) {
    int s = c->h_species[a];
    if (s < 0 || s >= c->nspecies) {
      dc_set_error("dc_init: species index out of range");
      return DC_ERR_ARG;
    }
    c->ne += c->h_Zs[s];
  }
  for (int s = 0; s < c->nspecies; ++s) {
    if (!(c->h_sigloc[s] > 0.0) || !(c->h_sigproj[s] > 0.0)) {
      dc_set_error("dc_init: sigma_loc and sigma_proj must be > 0");
      return DC_ERR_ARG;
    }
  }

  // core boundaries per axis
  std::vector<int> starts[3];
  for (int d = 0; d < 3; ++d) {
    starts[d].resize(F[d] + 1);
    for (int k = 0; k <= F[d]; ++k) starts[d][k] = (int)(((long long)k * n[d]) / F[d]);
  }

  c->h_desc.assign(c->nfrag, FragDesc{});
  for (int kz = 0; kz < F[2]; ++kz)
    for (int ky = 0; ky < F[1]; ++ky)
      for (int kx = 0; kx < F[0]; ++kx) {
        int f = kx + F[0] * (ky + F[1] * kz);
        FragDesc &D = c->h_desc[f];
        int kk[3] = {kx, ky, kz};
        for (int d = 0; d < 3; ++d) {
          int s0 = starts[d][kk[d]], s1 = starts[d][kk[d] + 1];
          D.org[d] = s0 - b[d];
          D.c[d] = s1 - s0;
          D.b[d] = b[d];
          D.E[d] = (s1 - s0) + 2 * b[d];
          if (D.E[d] > DC_MAX_EXTENT) {
            dc_set_error("dc_init: fragment extent above 64 points on an axis");
            return DC_ERR_ARG;
          }
          if (c->frag_cfg.bc == DC_BC_PERIODIC && D.E[d] < 4) {
            dc_set_error("dc_init: periodic fragment boundary needs every extent >= 4");
            return DC_ERR_ARG;
          }
        }
      }
  if (c->frag_cfg.bc != DC_BC_ZERO && c->frag_cfg.bc != DC_BC_PERIODIC) {
    dc_set_error("dc_init: bc must be DC_BC_ZERO or DC_BC_PERIODIC");
    return DC_ERR_ARG;
  }

  // orbital counts
  for (int f = 0; f < c->nfrag; ++f) {
    FragDesc &D = c->h_desc[f];
    if (c->frag_cfg.nstate_frag > 0) {
      D.norb = c->frag_cfg.nstate_frag;
    } else {
      double ne_f = 0.0;
      for (int a = 0; a < c->natom; ++a) {
        bool inside = true;
        for (int d = 0; d < 3 && inside; ++d) {
          double lo = (double)D.org[d] * c->h[d];
          double hi = (double)(D.org[d] + D.E[d]) * c->h[d];
          int kmax = (int)ceil(((double)D.E[d] * c->h[d]) / c->grid.L[d]) + 2;
          bool hit = false;
          for (int k = -kmax; k <= kmax; ++k) {
            double x = c->h_pos[3 * a + d] + (double)k * c->grid.L[d];
            if (x >= lo && x < hi) hit = true;
          }
          inside = hit;
        }
        if (inside) ne_f += c->h_Zs[c->h_species[a]];
      }
      long long occ = (long long)ceil(ne_f / 2.0);
      long long extra = std::max(4LL, (long long)ceil(0.2 * (double)occ));
      D.norb = (int)(occ + extra);
    }
    if (D.norb < 1 || D.norb > DC_MAX_NORB) {
      dc_set_error("dc_init: orbitals per fragment must be in [1, 64]");
      return DC_ERR_ARG;
    }
    long long P = (long long)D.E[0] * D.E[1] * D.E[2];
    if (D.norb > P) {
      dc_set_error("dc_init: more orbitals than points in a fragment");
      return DC_ERR_ARG;
    }
  }

  // offsets, maps
  long long psi_off = 0, pt_off = 0, c_off = 0, sub_off = 0, tab_off = 0;
  int st_off = 0, at_off = 0, zl_off = 0;
  c->h_idx_map.clear();
  c->h_atoms.clear();
  std::vector<ProjSlot> slots;
  std::vector<double> tab;
  std::vector<int> zl_beg, zl_items;
  std::vector<int> row_beg;
  std::vector<int2> row_ent;
  std::vector<int> row_split;
  c->max_atoms = 0;
  c->max_zlist = 0;
  c->max_plane_ent = 0;
  c->max_frag_ent = 0;
  c->core_pairs = true;
  for (int d = 0; d < 3; ++d) c->max_E[d] = 0;
  int max_norb = 0;
  for (int f = 0; f < c->nfrag; ++f) {
    FragDesc &D = c->h_desc[f];
    long long P = (long long)D.E[0] * D.E[1] * D.E[2];
    for (int d = 0; d < 3; ++d) c->max_E[d] = std::max(c->max_E[d], D.E[d]);
    if ((D.b[0] & 1) || (D.c[0] & 1) || (D.E[0] & 1)) c->core_pairs = false;
    max_norb = std::max(max_norb, D.norb);
    D.psi_off = psi_off;
    D.pt_off = pt_off;
    D.st_off = st_off;
    D.at_off = at_off;
    D.tab_off = tab_off;
    D.sub_off = sub_off;
    D.zl_off = zl_off;
    // idx_map (x fastest)
    for (int jz = 0; jz < D.E[2]; ++jz)
      for (int jy = 0; jy < D.E[1]; ++jy)
        for (int jx = 0; jx < D.E[0]; ++jx) {
          long long gx = wrap((long long)D.org[0] + jx, n[0]);
          long long gy = wrap((long long)D.org[1] + jy, n[1]);
          long long gz = wrap((long long)D.org[2] + jz, n[2]);
          c->h_idx_map.push_back((int32_t)(gx + (long long)n[0] * (gy + (long long)n[1] * gz)));
        }
    // atoms whose projector support box meets the fragment, ascending
    int A = 0;
    std::vector<std::vector<char>> zsup;
    for (int a = 0; a < c->natom; ++a) {
      int s = c->h_species[a];
      double sig = c->h_sigproj[s];
      double cut = 5.0 * sig;
      Factor fx[3];
      bool ok = true;
      for (int d = 0; d < 3 && ok; ++d) {
        fx[d] = axis_factor(D.org[d], D.E[d], n[d], c->h[d], c->grid.L[d], c->h_pos[3 * a + d], sig, cut);
        ok = fx[d].any;
      }
      if (!ok) continue;
      ProjSlot S;
      S.atom = a;
      S.coef = pow(M_PI * sig * sig, -0.75);
      for (int d = 0; d < 3; ++d) {
        int lo = -1, hi = -1;
        for (int j = 0; j < D.E[d]; ++j)
          if (fx[d].sup[j]) {
            if (lo < 0) lo = j;
            hi = j + 1;
          }
        S.lo[d] = lo;
        S.hi[d] = hi;
        for (int j = 0; j < D.E[d]; ++j) tab.push_back(fx[d].val[j]);
      }
      for (int p = D.E[0] + D.E[1] + D.E[2]; p < tab_width(D); ++p) tab.push_back(0.0);
      slots.push_back(S);
      c->h_atoms.push_back(a);
      zsup.push_back(fx[2].sup);
      ++A;
    }
    D.natom = A;
    c->max_atoms = std::max(c->max_atoms, A);
    // per-plane atom lists (slots whose z factor has support on the plane)
    int total = 0;
    for (int z = 0; z < D.E[2]; ++z) {
      zl_beg.push_back((int)zl_items.size());
      for (int k = 0; k < A; ++k)
        if (zsup[k][z]) {
          zl_items.push_back(k);
          ++total;
        }
    }
    zl_beg.push_back((int)zl_items.size());
    c->max_zlist = std::max(c->max_zlist, total);
    // Row lists of the orbital-pair stencil kernel: for every row (z, y), the slots whose FP32 product
    // gz(z) gy(y) is non-zero, as (k | y << 16, bits of that product).  Each row lists first the slots
    // whose x-support lies in the left half of the row's point pairs, then those reaching both halves,
    // then those only in the right half (z-list order within each group), and row_split records the two
    // boundaries, so that a point walks only the entries that can reach its half.
    {
      const int Ex = D.E[0], Ey = D.E[1], Ez = D.E[2], tw = tab_width(D);
      const int zl0 = (int)zl_beg.size() - (Ez + 1);
      const int xb = 2 * ((((Ex + 1) / 2) + 1) / 2);  // first point of the right half (point pairs)
      const ProjSlot *fs = slots.data() + (slots.size() - A);
      D.row_off = (int)row_beg.size();
      std::vector<int2> grp[3];
      for (int z = 0; z < Ez; ++z) {
        const size_t plane_start = row_ent.size();
        for (int y = 0; y < Ey; ++y) {
          row_beg.push_back((int)row_ent.size());
          for (auto &v : grp) v.clear();
          for (int e = zl_beg[zl0 + z]; e < zl_beg[zl0 + z + 1]; ++e) {
            const int k = zl_items[e];
            const double *g = &tab[tab_off + (long long)k * tw];
            const float w = (float)g[Ex + Ey + z] * (float)g[Ex + y];
            if (w != 0.f) {
              int wb;
              std::memcpy(&wb, &w, sizeof(int));
              const int side = fs[k].hi[0] <= xb ? 0 : (fs[k].lo[0] >= xb ? 2 : 1);
              grp[side].push_back(make_int2(k | (y << 16), wb));
            }
          }
          for (const auto &v : grp) row_ent.insert(row_ent.end(), v.begin(), v.end());
          const int nl = (int)grp[0].size(), nlb = nl + (int)grp[1].size();
          row_split.push_back(nl | (nlb << 16));
        }
        c->max_plane_ent = std::max(c->max_plane_ent, (int)(row_ent.size() - plane_start));
      }
      row_beg.push_back((int)row_ent.size());
      row_split.push_back(0);  // parallel to row_beg (one sentinel per fragment)
      c->max_frag_ent = std::max(c->max_frag_ent, (int)(row_ent.size() - (size_t)row_beg[D.row_off]));
      if (row_ent.size() > (size_t)INT32_MAX / 2) {
        dc_set_error("dc_init: projector row lists too long");
        return DC_ERR_ARG;
      }
    }
    zl_off += D.E[2] + 1;
    D.c_off = c_off;
    psi_off += (long long)D.norb * P;
    pt_off += P;
    st_off += D.norb;
    at_off += A;
    tab_off += (long long)A * tab_width(D);
    c_off += (long long)A * D.norb;
    sub_off += (long long)D.norb * D.norb;
  }
  c->layout.nfrag = c->nfrag;
  c->layout.natom = c->natom;
  c->layout.npts = c->npts;
  c->layout.psi_elems = psi_off;
  c->layout.frag_points = pt_off;
  c->layout.nstates = st_off;
  c->layout.natom_frag = at_off;
  c->layout.max_norb = max_norb;
  c->layout.element_bytes = c->params.precision == DC_FP64 ? 8 : 4;

  // owner / core_local
  c->h_owner.assign(c->npts, -1);
  c->h_core_local.assign(c->npts, -1);
  for (int f = 0; f < c->nfrag; ++f) {
    const FragDesc &D = c->h_desc[f];
    for (int jz = D.b[2]; jz < D.b[2] + D.c[2]; ++jz)
      for (int jy = D.b[1]; jy < D.b[1] + D.c[1]; ++jy)
        for (int jx = D.b[0]; jx < D.b[0] + D.c[0]; ++jx) {
          long long j = jx + (long long)D.E[0] * (jy + (long long)D.E[1] * jz);
          int32_t g = c->h_idx_map[D.pt_off + j];
          if (c->h_owner[g] >= 0) {
            dc_set_error("dc_init: internal error, overlapping cores");
            return DC_ERR_ARG;
          }
          c->h_owner[g] = f;
          c->h_core_local[g] = (int32_t)j;
        }
  }
  for (long long g = 0; g < c->npts; ++g)
    if (c->h_owner[g] < 0) {
      dc_set_error("dc_init: internal error, a grid point has no owner");
      return DC_ERR_ARG;
    }

  // work items (f, i)
  c->h_items.clear();
  for (int f = 0; f < c->nfrag; ++f)
    for (int i = 0; i < c->h_desc[f].norb; ++i) c->h_items.push_back(make_int2(f, i));

  out.slots.swap(slots);
  out.tab.swap(tab);
  out.zl_beg.swap(zl_beg);
  out.zl_items.swap(zl_items);
  out.row_beg.swap(row_beg);
  out.row_ent.swap(row_ent);
  out.row_split.swap(row_split);
  return DC_OK;
}

// Per-axis cover lists: for global coordinate g on axis d, every (k_d, local j_d) with
// (org(k_d) + j_d) mod N_d == g, ordered by k_d then j_d.
void dc_build_cover(const dc_ctx *c, int d, std::vector<int> &beg, std::vector<int2> &items) {
  const int N = c->grid.n[d];
  const int F = c->frag_cfg.num_fragment[d];
  std::vector<std::vector<int2>> lists(N);
  for (int k = 0; k < F; ++k) {
    // descriptor of any fragment with index k on this axis
    int f = (d == 0) ? k : (d == 1) ? k * c->frag_cfg.num_fragment[0]
                                     : k * c->frag_cfg.num_fragment[0] * c->frag_cfg.num_fragment[1];
    const FragDesc &D = c->h_desc[f];
    for (int j = 0; j < D.E[d]; ++j) lists[wrap((long long)D.org[d] + j, N)].push_back(make_int2(k, j));
  }
  beg.assign(N + 1, 0);
  items.clear();
  for (int g = 0; g < N; ++g) {
    beg[g] = (int)items.size();
    for (auto &p : lists[g]) items.push_back(p);
  }
  beg[N] = (int)items.size();
}

void dc_shard_range(const long long *cost, int nfrag, int rank, int nranks, int *lo, int *hi) {
  long long total = 0;
  for (int f = 0; f < nfrag; ++f) total += cost[f];
  // boundaries b_0 = 0 < b_1 < ... < b_nranks = nfrag
  int prev = 0, f = 0;
  long long prefix = 0;
  int b_lo = 0, b_hi = nfrag;
  for (int r = 1; r <= nranks; ++r) {
    int b = nfrag;
    if (r < nranks) {
      // first f with prefix(f) * nranks >= r * total (prefix(f) = cost of fragments before f)
      while (f < nfrag && prefix * nranks < (long long)r * total) prefix += cost[f++];
      b = f;
      if (b < prev + 1) b = prev + 1;
      if (b > nfrag - (nranks - r)) b = nfrag - (nranks - r);
    }
    if (r == rank) b_lo = b;
    if (r == rank + 1) b_hi = b;
    prev = b;
  }
  if (rank == 0) b_lo = 0;
  *lo = b_lo;
  *hi = b_hi;
}
