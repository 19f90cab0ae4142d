// C ABI of the DC-DFT fragment solver: context lifecycle and the per-step pipeline.
//
// One SCF iteration (Sec. 2.2): V_eff[rho_in] -> per-fragment potential and spectral bounds ->
// n_pass CheFSI passes on all fragments at once -> core weights, mu, rho_out (Eqs. 2-4) ->
// energies -> linear mixing.  Every stage is a kernel on the caller's stream; the only host round
// trip is the final copy of the step statistics.
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>

#include "dc_internal.h"

namespace {
thread_local std::string g_last_error = "";
}

void dc_set_error(const std::string &msg) { g_last_error = msg; }

cudaError_t dc_set_smem(const void *func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(dev, func);
  auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done[key] = bytes;
  return e;
}

int dc_cuda_status(cudaError_t e, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return DC_ERR_OOM;
  }
  return DC_ERR_CUDA;
}

namespace {

template <typename T>
int dmalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  const cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
  if (e != cudaSuccess) {
    *p = nullptr;
    return dc_cuda_status(e, "cudaMalloc");
  }
  return DC_OK;
}

template <typename T>
int upload(T **p, const std::vector<T> &v) {
  DC_TRY(dmalloc(p, v.size()));
  if (!v.empty()) DC_CUDA(cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return DC_OK;
}

void free_ctx(dc_ctx *c) {
  if (!c) return;
  void *ptrs[] = {c->d_desc, c->d_items, c->d_idx_map, c->d_owner, c->d_core_local, c->d_slots, c->d_tab64,
                  c->d_tab32, c->d_zl_beg, c->d_zl_items, c->d_atom_D, c->d_atom_pos, c->d_atom_species,
                  c->d_species, c->d_cover_beg[0], c->d_cover_beg[1], c->d_cover_beg[2], c->d_cover[0],
                  c->d_cover[1], c->d_cover[2], c->d_vion, c->d_rho0, c->d_veff, c->d_rho_out, c->d_work,
                  c->d_rhoiG, c->d_cplx, c->d_vf64, c->d_vf32, c->blk[0], c->blk[1], c->blk[2], c->blk64[0],
                  c->blk64[1], c->blk64[2], c->d_hy64, c->d_c64[0], c->d_c64[1], c->d_c32[0], c->d_c32[1],
                  c->d_eps, c->d_q, c->d_occ, c->d_bounds, c->d_gram, c->d_gram_off, c->d_gram_nchunk, c->d_C64,
                  c->d_C32, c->d_flags, c->d_scalar, c->d_partials, c->d_gram_items, c->d_rot_items, c->d_Fn,
                  c->d_items2, c->d_row_beg, c->d_row_ent, c->d_row_split, c->d_nl_bound, c->d_rot2_items,
                  c->d_atom_slot_beg, c->d_atom_slots, c->d_slot_w, c->d_adj_vf64, c->d_adj_vf32, c->d_adj_fd,
                  c->d_dots, c->d_ig2, c->d_kerkw, c->d_rhoinG, c->d_cplxh, c->d_fftr, c->d_q_x, c->d_occ_x, c->d_aux, c->d_frag_order, c->d_rhof, c->d_vcore};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c->h_scalar_pinned) cudaFreeHost(c->h_scalar_pinned);
  for (auto &g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto &r : g.recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
  }
  for (auto &r : c->prof_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : c->prof_free) cudaEventDestroy(e);
  if (c->have_plan) {
    cufftDestroy(c->plan_z2z);
    cufftDestroy(c->plan_d2z);
    cufftDestroy(c->plan_z2d);
  }
  cudaGetLastError();
  delete c;
}

int check_flags(dc_ctx *c, cudaStream_t s) {
  unsigned fl = 0;
  DC_CUDA(cudaMemcpyAsync(&fl, c->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  DC_CUDA(cudaStreamSynchronize(s));
  if (fl) {
    DC_CUDA(cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), s));
    DC_CUDA(cudaStreamSynchronize(s));
    if (fl & DC_FLAG_TIMEOUT) {
      dc_set_error("a bounded device wait ran out (grid barrier)");
      return DC_ERR_TIMEOUT;
    }
    if (fl & DC_FLAG_NOTSPD) {
      dc_set_error("Gram matrix not positive definite in at least one fragment");
      return DC_ERR_NOCONV;
    }
    if (fl & DC_FLAG_NONFINITE) {
      dc_set_error("non-finite eigenvalue or chemical potential");
      return DC_ERR_NONFINITE;
    }
  }
  return DC_OK;
}

cudaEvent_t take_event(dc_ctx *c) {
  cudaEvent_t e = nullptr;
  if (!c->prof_free.empty()) {
    e = c->prof_free.back();
    c->prof_free.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    e = nullptr;
  }
  return e;
}

// Records a CUDA event pair around one stage launch on its stream when the profiler is on.  The
// record goes to c->prof_sink: the pending list, or the list of a graph being captured.
struct StageScope {
  dc_ctx *c;
  cudaStream_t s;
  ProfRec r{nullptr, nullptr, 0, 0.0, 0};
  bool on = false;
  StageScope(dc_ctx *c_, int stage_, cudaStream_t s_, double bytes_, int nk_) : c(c_), s(s_) {
    if (c->prof_on && c->prof_sink) {
      r.a = take_event(c);
      r.b = take_event(c);
      r.stage = stage_;
      r.bytes = bytes_;
      r.nk = nk_;
      on = r.a && r.b;
      if (on) cudaEventRecord(r.a, s);
    }
  }
  ~StageScope() {
    if (on) {
      cudaEventRecord(r.b, s);
      c->prof_sink->push_back(r);
    }
  }
};

// Add the elapsed times of completed records to the profiler sums (the device must be idle).
void prof_collect(dc_ctx *c, std::vector<ProfRec> &recs, bool recycle) {
  for (auto &r : recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.stage] += t;
      c->prof_by[r.stage] += r.bytes;
      c->prof_nl[r.stage] += r.nk;
    } else {
      cudaGetLastError();
    }
    if (recycle) {
      c->prof_free.push_back(r.a);
      c->prof_free.push_back(r.b);
    }
  }
  if (recycle) recs.clear();
}

void destroy_graphs(dc_ctx *c) {
  for (auto &g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto &r : g.recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
  }
  c->graphs.clear();
}

// Algorithmic bytes and launches of this library's kernels in the global stages (cuFFT's own launches
// are not counted; each transform is counted as one read and one write of the complex grid).
// N = grid points; a complex grid is 16N bytes, a real one 8N.
struct StageModel {
  double bytes;
  int launches;
};
StageModel potential_model(const dc_ctx *c, bool save_spectrum) {
  const double N = (double)c->npts, NH = (double)c->nh;
  (void)save_spectrum;
  if (c->params.hxc != DC_HXC_HARTREE_X) return {16.0 * N, 1};  // k_veff: V_loc in, V_eff out
  // real-to-complex FFT 8N + 16NH, k_poisson_scale 40NH, complex-to-real FFT 16NH + 8N, k_veff (V_loc,
  // V_H, rho in; V_eff out) 32N
  return {48.0 * N + 72.0 * NH, 2};
}
StageModel energy_model(const dc_ctx *c, bool spectrum_difference) {
  const double N = (double)c->npts, NH = (double)c->nh, ns = (double)c->layout.nstates;
  // band sum (occ, eps, q) and entropy (occ, q) over the states; <V, rho_out>, E_x, |rho_out - rho_in|
  // and int rho_out over the grid; every reduction is two launches (block partials, final sum)
  double b = 40.0 * ns + 48.0 * N;
  int nk = 12 + 1;  // + k_energy_combine
  if (c->params.hxc == DC_HXC_HARTREE_X) {
    // real-to-complex FFT; E_es reduction (half spectrum, 1/G^2, the ion spectrum at G and at -G)
    b += 8.0 * N + 16.0 * NH + 56.0 * NH;
    nk += 2;
  }
  // mixing
  if (!(c->params.kerker_q0 > 0.0)) {
    b += 24.0 * N;  // k_mix
    nk += 1;
  } else {
    // residual spectrum: k_sub_cplx 48NH, or k_residual 24N + real-to-complex FFT 8N + 16NH; then
    // k_kerker 40NH, complex-to-real FFT 16NH + 8N, k_add_real 24N
    b += (spectrum_difference ? 48.0 * NH : 32.0 * N + 16.0 * NH) + 56.0 * NH + 32.0 * N;
    nk += 3;
  }
  return {b, nk};
}

// Longest-first order of a work list whose items name their fragment in .x (stable, so a cell whose
// fragments all cost the same keeps its order): the block scheduler hands out CTAs roughly in index
// order, so the costliest items of uneven cells (fragments with more orbitals or points) start first
// and the short ones fill in at the end instead of one long item finishing alone.
void longest_first(const dc_ctx *c, std::vector<int2> &items, int power) {
  auto cost = [&](int f) {
    const FragDesc &D = c->h_desc[f];
    double w = (double)D.E[0] * D.E[1] * D.E[2];
    for (int k = 0; k < power; ++k) w *= D.norb;
    return w;
  };
  std::stable_sort(items.begin(), items.end(), [&](const int2 &a, const int2 &b) { return cost(a.x) > cost(b.x); });
}

double core_elems(const dc_ctx *c) {
  double s = 0.0;
  for (const auto &D : c->h_desc) s += (double)D.norb * D.c[0] * D.c[1] * D.c[2];
  return s;
}
double proj_elems(const dc_ctx *c) {
  double s = 0.0;
  for (const auto &D : c->h_desc) s += (double)D.norb * D.natom;
  return s;
}

template <typename T>
T *cproj(dc_ctx *c, int k);
template <>
double *cproj<double>(dc_ctx *c, int k) { return c->d_c64[k]; }
template <>
float *cproj<float>(dc_ctx *c, int k) { return c->d_c32[k]; }

// One CheFSI pass on the rotating blocks B (state in B[ib]); filter = false gives the plain
// Rayleigh-Ritz of the current block.  Leaves the new state index in ib.
template <typename T>
int chefsi_pass(dc_ctx *c, T *B[3], int &ib, bool filter, cudaStream_t s) {
  const int m = c->params.cheb_degree;
  const double es = sizeof(T), blk = es * (double)c->layout.psi_elems, vfb = es * (double)c->layout.frag_points;
  const double pj = es * proj_elems(c);
  int cur = ib;
  int cbuf = 0;
  if (c->proj_ok == (int)sizeof(T)) {
    cbuf = c->proj_buf;  // <p|Psi> of the state block, rotated at the end of the previous pass
  } else {
    StageScope sc(c, DC_STAGE_PROJECT, s, blk + pj, 1);
    DC_TRY(dck::launch_project<T>(c, B[cur], cproj<T>(c, 0), s));
  }
  if (filter) {
    {
      StageScope sc(c, DC_STAGE_SUBSPACE, s, 8.0 * c->layout.nstates, 1);
      DC_TRY(dck::launch_bounds(c, 0, s));
    }
    int prev = -1;
    for (int k = 0; k < m; ++k) {
      int nxt = 0;
      while (nxt == cur || nxt == prev) ++nxt;
      StageScope sc(c, DC_STAGE_HPSI, s, (k > 0 ? 3.0 : 2.0) * blk + vfb + 2.0 * pj, 1);
      DC_TRY(dck::launch_hstep<T>(c, HSTEP_CHEB, k, B[cur], prev >= 0 ? B[prev] : nullptr, B[nxt],
                                  cproj<T>(c, cbuf), cproj<T>(c, cbuf ^ 1), nullptr, nullptr, nullptr, nullptr, s));
      cbuf ^= 1;
      prev = cur;
      cur = nxt;
    }
  }
  const int hy = (cur + 1) % 3;
  // H Y feeds only the Gram.  Where the specialised kernel applies H, it applies the local part alone and
  // the subspace stage adds the nonlocal part of A = Y^T H Y from the block's projections <p|Y> (Eq. 5:
  // Y^T D P P^T Y = sum_a D_a <p_a|Y>^T <p_a|Y>), which the last filter step has already formed.
  const bool hloc = sizeof(T) == 4 && dck::hstep_specialised(c);
  {
    StageScope sc(c, DC_STAGE_HPSI, s, 2.0 * blk + vfb + (hloc ? 0.0 : pj), 1);
    DC_TRY(dck::launch_hstep<T>(c, hloc ? HSTEP_HLOC : HSTEP_HPSI, 0, B[cur], nullptr, B[hy], cproj<T>(c, cbuf),
                                nullptr, nullptr, nullptr, nullptr, nullptr, s));
  }
  {
    StageScope sc(c, DC_STAGE_GRAM, s, 2.0 * blk + 8.0 * c->gram_elems, 1);
    if (sizeof(T) == 4 && c->params.precision == DC_MIXED)
      DC_TRY(dck::launch_gram_tc(c, (const float *)B[cur], (const float *)B[hy], s));
    else
      DC_TRY(dck::launch_gram<T>(c, B[cur], B[hy], s));
  }
  {
    StageScope sc(c, DC_STAGE_SUBSPACE, s, 8.0 * c->gram_elems + (hloc ? pj : 0.0), 1);
    DC_TRY(dck::launch_subspace(c, sizeof(T) == 4 ? 32 : 64, c->d_eps, s,
                                hloc ? reinterpret_cast<const float *>(cproj<T>(c, cbuf)) : nullptr));
  }
  {
    StageScope sc(c, DC_STAGE_ROTATE, s, 2.0 * blk, 1);
    DC_TRY(dck::launch_rotate<T>(c, B[cur], B[hy], s));
  }
  {
    // <p|Y C> = <p|Y> C: the next pass starts from rotated projections instead of a pass over Psi
    StageScope sc(c, DC_STAGE_PROJECT, s, 2.0 * pj, 1);
    DC_TRY(dck::launch_rotate_proj<T>(c, cproj<T>(c, cbuf), cproj<T>(c, cbuf ^ 1), s));
  }
  c->proj_ok = (int)sizeof(T);
  c->proj_buf = cbuf ^ 1;
  ib = hy;
  return DC_OK;
}

int pass_ctx(dc_ctx *c, bool filter, int npass, cudaStream_t s) {
  for (int p = 0; p < npass; ++p) {
    if (c->params.precision == DC_FP64) {
      double *B[3] = {(double *)c->blk[0], (double *)c->blk[1], (double *)c->blk[2]};
      DC_TRY(chefsi_pass<double>(c, B, c->ib_psi, filter, s));
    } else {
      float *B[3] = {(float *)c->blk[0], (float *)c->blk[1], (float *)c->blk[2]};
      DC_TRY(chefsi_pass<float>(c, B, c->ib_psi, filter, s));
    }
  }
  return DC_OK;
}

int density_stage(dc_ctx *c, double *rho, cudaStream_t s) {
  const double es = c->params.precision == DC_FP64 ? 8.0 : 4.0;
  StageScope sc(c, DC_STAGE_DENSITY, s, 2.0 * es * core_elems(c) + 8.0 * c->npts + 32.0 * c->layout.nstates, 3);
  if (c->params.precision == DC_FP64) {
    DC_TRY(dck::launch_core_weights<double>(c, (const double *)c->blk[c->ib_psi], c->d_q, s));
    DC_TRY(dck::launch_fermi(c, c->d_eps, c->d_q, c->d_scalar, c->d_occ, s));
    DC_TRY(dck::launch_density<double>(c, (const double *)c->blk[c->ib_psi], c->d_occ, rho, s));
  } else {
    DC_TRY(dck::launch_core_weights<float>(c, (const float *)c->blk[c->ib_psi], c->d_q, s));
    DC_TRY(dck::launch_fermi(c, c->d_eps, c->d_q, c->d_scalar, c->d_occ, s));
    DC_TRY(dck::launch_density<float>(c, (const float *)c->blk[c->ib_psi], c->d_occ, rho, s));
  }
  return DC_OK;
}

// Per-fragment exchange: the fragment densities of the current state and occupations (Eq. 3 before the
// core projection), the input of the next step's fragment potentials.
int fragment_density(dc_ctx *c, cudaStream_t s) {
  if (!c->params.xc_fragment) return DC_OK;
  const double es = c->params.precision == DC_FP64 ? 8.0 : 4.0;
  StageScope sc(c, DC_STAGE_DENSITY, s, es * (double)c->layout.psi_elems + 8.0 * c->layout.frag_points, 1);
  if (c->params.precision == DC_FP64)
    return dck::launch_frag_density<double>(c, (const double *)c->blk[c->ib_psi], c->d_occ, c->d_rhof, s, true);
  return dck::launch_frag_density<float>(c, (const float *)c->blk[c->ib_psi], c->d_occ, c->d_rhof, s, true);
}

inline cudaStream_t S(void *p) { return reinterpret_cast<cudaStream_t>(p); }

// Autotune the stencil launch shape for element type T on block y (scratch block `out`).  With
// DC_TUNE_CACHE=<file>, shapes are looked up by fragment shape and atom/orbital counts and new
// results are appended to the file.
template <typename T>
int tune(dc_ctx *c, const T *y, T *out, cudaStream_t s) {
  const int ti = sizeof(T) == 8 ? 1 : 0;
  char key[160];
  snprintf(key, sizeof(key), "hstep %dx%dx%d A%d n%d %s", c->max_E[0], c->max_E[1], c->max_E[2], c->max_atoms,
           c->layout.max_norb, ti ? "f64" : "f32");
  const char *path = getenv("DC_TUNE_CACHE");
  if (path && path[0]) {
    FILE *fp = fopen(path, "r");
    if (fp) {
      char line[256];
      while (fgets(line, sizeof(line), fp)) {
        const size_t kl = strlen(key);
        if (strncmp(line, key, kl) == 0 && line[kl] == ' ') {
          c->hstep_shape[ti] = atoi(line + kl + 1);
        }
      }
      fclose(fp);
      if (c->hstep_shape[ti] >= 0) return DC_OK;
    }
  }
  c->proj_ok = 0;  // the projection buffers serve as scratch here
  DC_TRY(dck::launch_project<T>(c, y, cproj<T>(c, 0), s));
  DC_TRY(dck::tune_hstep<T>(c, y, out, cproj<T>(c, 0), s));
  if (path && path[0]) {
    FILE *fp = fopen(path, "a");
    if (fp) {
      fprintf(fp, "%s %d\n", key, c->hstep_shape[ti]);
      fclose(fp);
    }
  }
  return DC_OK;
}

// Device part of one SCF step; no host synchronisation, so it can be captured into a graph.  The
// step's scalars and device flags land in pinned host memory (flags at slot 20) and the flags are
// cleared for the next call.
int step_body(dc_ctx *c, double *rin, cudaStream_t s) {
  const bool keep_spectrum = c->params.hxc == DC_HXC_HARTREE_X;
  {
    const StageModel pm = potential_model(c, keep_spectrum);
    StageScope sc(c, DC_STAGE_POTENTIAL, s, pm.bytes, pm.launches);
    // with the Hartree term the input density's spectrum is kept for the Kerker residual below
    DC_TRY(dck::launch_potential(c, rin, s, keep_spectrum ? c->d_rhoinG : nullptr, true));
  }
  {
    const bool fx = c->params.xc_fragment != 0;
    StageScope sc(c, DC_STAGE_GATHER, s, (fx ? 40.0 : 24.0) * (double)c->layout.frag_points + (fx ? 28.0 : 0.0) * c->npts,
                  fx ? 2 : 1);
    DC_TRY(dck::launch_gather(c, s, fx ? rin : nullptr));
  }
  DC_TRY(pass_ctx(c, true, c->params.n_pass, s));
  DC_TRY(density_stage(c, c->d_rho_out, s));
  DC_TRY(fragment_density(c, s));
  {
    const StageModel em = energy_model(c, keep_spectrum);
    StageScope sc(c, DC_STAGE_ENERGY, s, em.bytes, em.launches);
    DC_TRY(dck::launch_energy(c, rin, s));
    DC_TRY(dck::launch_mix(c, rin, s, keep_spectrum ? c->d_rhoinG : nullptr));
  }
  DC_CUDA(cudaMemcpyAsync(c->h_scalar_pinned, c->d_scalar, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
  DC_CUDA(cudaMemcpyAsync(c->h_scalar_pinned + 20, c->d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  DC_CUDA(cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), s));
  return DC_OK;
}

// Capture step_body into a new graph; returns its index, or -1 (graphs then stay off for this
// context and the step runs eagerly) if capture or instantiation is not possible.
int capture_step(dc_ctx *c, double *rin, cudaStream_t s) {
  StepGraph g;
  g.ib_before = c->ib_psi;
  g.proj_before = c->proj_ok;
  g.pbuf_before = c->proj_buf;
  g.rho = rin;
  g.prof = c->prof_on;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    c->graphs_enabled = false;
    return -1;
  }
  std::vector<ProfRec> *sink = c->prof_sink;
  c->prof_sink = &g.recs;
  const int ib = c->ib_psi;
  const int st = step_body(c, rin, s);
  c->prof_sink = sink;
  g.ib_after = c->ib_psi;
  g.proj_after = c->proj_ok;
  g.pbuf_after = c->proj_buf;
  c->ib_psi = ib;
  c->proj_ok = g.proj_before;
  c->proj_buf = g.pbuf_before;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (st == DC_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (st != DC_OK || e != cudaSuccess) {
    cudaGetLastError();
    for (auto &r : g.recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    c->graphs_enabled = false;
    return -1;
  }
  c->graphs.push_back(std::move(g));
  return (int)c->graphs.size() - 1;
}

// Rayleigh-Ritz of a caller block Y in place (Y <- Y C), Ritz values into eps.  The context's two work
// blocks hold H Y and Y C; its own state block, eps, q and mu are left alone.
template <typename T>
int subspace_block(dc_ctx *c, T *Y, double *eps, cudaStream_t s) {
  T *W1 = static_cast<T *>(c->blk[(c->ib_psi + 1) % 3]);
  T *W2 = static_cast<T *>(c->blk[(c->ib_psi + 2) % 3]);
  c->proj_ok = 0;  // projection buffer 0 holds the caller block's projections below
  DC_TRY(dck::launch_project<T>(c, Y, cproj<T>(c, 0), s));
  DC_TRY(dck::launch_hstep<T>(c, HSTEP_HPSI, 0, Y, nullptr, W1, cproj<T>(c, 0), nullptr, nullptr, nullptr, nullptr,
                              nullptr, s));
  if (sizeof(T) == 4 && c->params.precision == DC_MIXED)
    DC_TRY(dck::launch_gram_tc(c, (const float *)Y, (const float *)W1, s));
  else
    DC_TRY(dck::launch_gram<T>(c, Y, W1, s));
  DC_TRY(dck::launch_subspace(c, sizeof(T) == 4 ? 32 : 64, eps, s));
  DC_TRY(dck::launch_rotate<T>(c, Y, W2, s));
  const size_t bytes = sizeof(T) * (size_t)c->layout.psi_elems;
  DC_CUDA(cudaMemcpyAsync(Y, W2, bytes, cudaMemcpyDeviceToDevice, s));
  return DC_OK;
}

}  // namespace

extern "C" {

const char *dc_error_string(int status) {
  switch (status) {
    case DC_OK: return "DC_OK";
    case DC_ERR_ARG: return "DC_ERR_ARG";
    case DC_ERR_CUDA: return "DC_ERR_CUDA";
    case DC_ERR_OOM: return "DC_ERR_OOM";
    case DC_ERR_NOCONV: return "DC_ERR_NOCONV";
    case DC_ERR_TIMEOUT: return "DC_ERR_TIMEOUT";
    case DC_ERR_NONFINITE: return "DC_ERR_NONFINITE";
    case DC_ERR_STATE: return "DC_ERR_STATE";
    default: return "DC_ERR_UNKNOWN";
  }
}

const char *dc_last_error(void) { return g_last_error.c_str(); }

static int dc_init_impl(const dc_grid_t *grid, const dc_fragments_t *fragments, const dc_buffers_t *buffers,
                        const dc_atoms_t *atoms, const dc_params_t *params, dc_ctx *c) {
  c->grid = *grid;
  c->frag_cfg = *fragments;
  c->buf_cfg = *buffers;
  c->params = *params;
  const dc_params_t &P = c->params;
  if (P.precision < DC_FP64 || P.precision > DC_MIXED || P.cheb_degree < 1 || P.cheb_degree > 64 || P.n_pass < 1 ||
      P.n_warmup < 0 || !(P.kT > 0.0) || !(P.mix_alpha >= 0.0) || P.mix_alpha > 1.0 || !(P.kerker_q0 >= 0.0) ||
      (P.hxc != DC_HXC_NONE && P.hxc != DC_HXC_HARTREE_X) || (P.xc_fragment != 0 && P.xc_fragment != 1) ||
      !(P.xi >= 0.0)) {
    dc_set_error("dc_init: invalid parameters");
    return DC_ERR_ARG;
  }
  if (P.xc_fragment && (P.hxc != DC_HXC_HARTREE_X || P.nranks > 1)) {
    dc_set_error("dc_init: per-fragment exchange needs hxc = DC_HXC_HARTREE_X and every fragment (nranks <= 1)");
    return DC_ERR_ARG;
  }
  if (atoms->natom > 0 && (!atoms->pos || !atoms->species)) {
    dc_set_error("dc_init: atoms->pos and atoms->species required");
    return DC_ERR_ARG;
  }
  if (!atoms->Z || !atoms->sigma_loc || !atoms->sigma_proj || !atoms->D) {
    dc_set_error("dc_init: species tables required");
    return DC_ERR_ARG;
  }
  HostTables ht;
  DC_TRY(dc_build_host(c, atoms, ht));
  // fragment shard (Sec. 2.5: fragments are distributed over processes): contiguous fragment ids,
  // balanced by the stencil work P_f n_f of each fragment
  c->nranks = P.nranks > 0 ? P.nranks : 1;
  c->rank = P.rank;
  if (c->rank < 0 || c->rank >= c->nranks || c->nranks > c->nfrag) {
    dc_set_error("dc_init: need 0 <= rank < nranks <= number of fragments");
    return DC_ERR_ARG;
  }
  {
    std::vector<long long> cost(c->nfrag);
    for (int f = 0; f < c->nfrag; ++f) {
      const FragDesc &D = c->h_desc[f];
      cost[f] = (long long)D.E[0] * D.E[1] * D.E[2] * D.norb;
    }
    int lo = 0, hi = c->nfrag;
    dc_shard_range(cost.data(), c->nfrag, c->rank, c->nranks, &lo, &hi);
    c->f_lo = lo;
    c->f_hi = hi;
    c->st_lo = c->h_desc[lo].st_off;
    c->st_hi = hi < c->nfrag ? (long long)c->h_desc[hi].st_off : c->layout.nstates;
    c->layout.frag_lo = lo;
    c->layout.frag_hi = hi;
    c->layout.state_lo = c->st_lo;
    c->layout.state_hi = c->st_hi;
  }
  int dev = 0;
  DC_CUDA(cudaGetDevice(&dev));
  DC_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev));

  const dc_layout_t &Lo = c->layout;
  // maps and tables
  DC_TRY(upload(&c->d_desc, c->h_desc));
  DC_TRY(upload(&c->d_items, c->h_items));
  {
    std::vector<int2> it2;
    for (int f = c->f_lo; f < c->f_hi; ++f)
      for (int i = 0; i < c->h_desc[f].norb; i += 2) it2.push_back(make_int2(f, i));
    longest_first(c, it2, 0);  // one orbital pair of a fragment: cost ~ its points
    c->n_items2 = (int)it2.size();
    DC_TRY(upload(&c->d_items2, it2));
  }
  DC_TRY(upload(&c->d_idx_map, c->h_idx_map));
  DC_TRY(upload(&c->d_owner, c->h_owner));
  DC_TRY(upload(&c->d_core_local, c->h_core_local));
  DC_TRY(upload(&c->d_slots, ht.slots));
  DC_TRY(upload(&c->d_tab64, ht.tab));
  std::vector<float> tab32(ht.tab.begin(), ht.tab.end());
  DC_TRY(upload(&c->d_tab32, tab32));
  DC_TRY(upload(&c->d_zl_beg, ht.zl_beg));
  DC_TRY(upload(&c->d_zl_items, ht.zl_items));
  DC_TRY(upload(&c->d_row_beg, ht.row_beg));
  DC_TRY(upload(&c->d_row_ent, ht.row_ent));
  DC_TRY(upload(&c->d_row_split, ht.row_split));
  std::vector<double> Datom(c->natom), posv(c->h_pos);
  for (int a = 0; a < c->natom; ++a) Datom[a] = c->h_Ds[c->h_species[a]];
  DC_TRY(upload(&c->d_atom_D, Datom));
  {
    // Upper bound of the nonlocal term per fragment (Sec. 2.2 filter bounds): sum over its slots of
    // max(D, 0) dV C^2 |gx|^2 |gy|^2 |gz|^2, fixed for the context.
    std::vector<double> nlb(c->nfrag, 0.0);
    for (int f = 0; f < c->nfrag; ++f) {
      const FragDesc &D = c->h_desc[f];
      const int tw = tab_width(D);
      for (int k = 0; k < D.natom; ++k) {
        const ProjSlot &S = ht.slots[D.at_off + k];
        const double *g = &ht.tab[D.tab_off + (long long)k * tw];
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int j = 0; j < D.E[0]; ++j) sx += g[j] * g[j];
        for (int j = 0; j < D.E[1]; ++j) sy += g[D.E[0] + j] * g[D.E[0] + j];
        for (int j = 0; j < D.E[2]; ++j) sz += g[D.E[0] + D.E[1] + j] * g[D.E[0] + D.E[1] + j];
        nlb[f] += std::max(Datom[S.atom], 0.0) * c->dV * S.coef * S.coef * sx * sy * sz;
      }
    }
    DC_TRY(upload(&c->d_nl_bound, nlb));
  }
  DC_TRY(upload(&c->d_atom_pos, posv));
  DC_TRY(upload(&c->d_atom_species, c->h_species));
  std::vector<double> spec;
  for (auto *v : {&c->h_Zs, &c->h_sigloc, &c->h_sigproj, &c->h_Ds}) spec.insert(spec.end(), v->begin(), v->end());
  DC_TRY(upload(&c->d_species, spec));
  std::vector<int> Fn(c->frag_cfg.num_fragment, c->frag_cfg.num_fragment + 3);
  DC_TRY(upload(&c->d_Fn, Fn));
  for (int d = 0; d < 3; ++d) {
    std::vector<int> beg;
    std::vector<int2> items;
    dc_build_cover(c, d, beg, items);
    DC_TRY(upload(&c->d_cover_beg[d], beg));
    DC_TRY(upload(&c->d_cover[d], items));
  }
  // per-atom slot lists (for dE/dD), fixed order by fragment
  {
    std::vector<std::vector<int>> per(c->natom);
    for (int f = 0; f < c->nfrag; ++f)
      for (int k = 0; k < c->h_desc[f].natom; ++k) per[c->h_atoms[c->h_desc[f].at_off + k]].push_back(c->h_desc[f].at_off + k);
    std::vector<int> beg(c->natom + 1, 0), sl;
    for (int a = 0; a < c->natom; ++a) {
      beg[a] = (int)sl.size();
      sl.insert(sl.end(), per[a].begin(), per[a].end());
    }
    beg[c->natom] = (int)sl.size();
    DC_TRY(upload(&c->d_atom_slot_beg, beg));
    DC_TRY(upload(&c->d_atom_slots, sl));
  }
  // work lists for the Gram and rotation kernels
  {
    // points per Gram partial: each chunk's sums are FP32 (tensor memory drained every 256 points
    // into FP32 registers, or SIMT pairs) and the chunks are added in FP64; DC_GRAM_CHUNK overrides
    // (multiple of 64, 64..65536).  Tensor-memory FP32 accumulation carries an error that grows with
    // the accumulated length, hence the 256-point drains; 4096-point chunks left the Si512 mixed-vs-FP64
    // energy difference where 2048 had it (4.5e-7 Ha/atom) and halve the Gram's item boundaries.
    // Fewer than two items per SM leave the persistent Gram CTAs unbalanced, so small cells halve it.
    c->gram_chunk = 4096;
    {
      auto items = [&](long long chunk) {
        long long k = 0;
        // counted over the whole system, not the shard: the chunking fixes the Gram's rounding, and a
      // shard must reproduce the single-context result bit for bit
      for (const auto &D : c->h_desc) k += ((long long)D.E[0] * D.E[1] * D.E[2] + chunk - 1) / chunk;
        return k;
      };
      while (c->gram_chunk > 512 && items(c->gram_chunk) < 2LL * c->sm_count) c->gram_chunk /= 2;
    }
    if (const char *gc = getenv("DC_GRAM_CHUNK")) {
      const int v = atoi(gc);
      if (v >= 64 && v <= 65536 && v % 64 == 0) c->gram_chunk = v;
    }
    std::vector<int2> gi, ri, ri2;
    std::vector<long long> goff(c->nfrag);
    std::vector<int> gn(c->nfrag);
    long long off = 0;
    for (int f = 0; f < c->nfrag; ++f) {
      const FragDesc &D = c->h_desc[f];
      const long long Pf = (long long)D.E[0] * D.E[1] * D.E[2];
      const int nch = (int)((Pf + c->gram_chunk - 1) / c->gram_chunk);
      gn[f] = nch;
      goff[f] = off;
      off += (long long)nch * 2 * D.norb * D.norb;
      if (f < c->f_lo || f >= c->f_hi) continue;  // work items of the context's shard only
      for (int ch = 0; ch < nch; ++ch) gi.push_back(make_int2(f, ch));
      const int nr = (int)((Pf + 127) / 128);
      for (int ch = 0; ch < nr; ++ch) ri.push_back(make_int2(f, ch));
      const int nr2 = (int)((Pf + 255) / 256);
      for (int ch = 0; ch < nr2; ++ch) ri2.push_back(make_int2(f, ch));
    }
    longest_first(c, gi, 2);   // Gram item: points x n^2
    longest_first(c, ri, 1);   // rotation items: points x n
    longest_first(c, ri2, 1);
    c->gram_elems = off;
    c->n_gram_items = (int)gi.size();
    c->n_rot_items = (int)ri.size();
    c->n_rot2_items = (int)ri2.size();
    DC_TRY(upload(&c->d_gram_items, gi));
    DC_TRY(upload(&c->d_rot_items, ri));
    DC_TRY(upload(&c->d_rot2_items, ri2));
    DC_TRY(upload(&c->d_gram_off, goff));
    DC_TRY(upload(&c->d_gram_nchunk, gn));
    {
      // the subspace solve (one CTA per fragment, ~n^3 FP64 work) runs its fragments longest first
      std::vector<int2> fo;
      for (int f = c->f_lo; f < c->f_hi; ++f) fo.push_back(make_int2(f, 0));
      longest_first(c, fo, 3);
      std::vector<int> order(fo.size());
      for (size_t k = 0; k < fo.size(); ++k) order[k] = fo[k].x;
      DC_TRY(upload(&c->d_frag_order, order));
    }
    DC_TRY(dmalloc(&c->d_gram, (size_t)off));
  }
  // global grid arrays
  const size_t N = (size_t)c->npts;
  DC_TRY(dmalloc(&c->d_vion, N));
  DC_TRY(dmalloc(&c->d_rho0, N));
  DC_TRY(dmalloc(&c->d_veff, N));
  DC_TRY(dmalloc(&c->d_rho_out, N));
  DC_TRY(dmalloc(&c->d_work, N));
  c->nh = (long long)c->grid.n[2] * c->grid.n[1] * (c->grid.n[0] / 2 + 1);
  const size_t NH = (size_t)c->nh;
  DC_TRY(dmalloc(&c->d_rhoiG, N));
  DC_TRY(dmalloc(&c->d_ig2, NH));
  DC_TRY(dmalloc(&c->d_kerkw, NH));
  DC_TRY(dmalloc(&c->d_rhoinG, NH));
  DC_TRY(dmalloc(&c->d_cplx, N));
  DC_TRY(dmalloc(&c->d_cplxh, NH));
  DC_TRY(dmalloc(&c->d_fftr, N));
  const int *gn = c->grid.n;
  if (cufftPlan3d(&c->plan_z2z, gn[2], gn[1], gn[0], CUFFT_Z2Z) != CUFFT_SUCCESS) {
    dc_set_error("cufftPlan3d failed");
    return DC_ERR_CUDA;
  }
  if (cufftPlan3d(&c->plan_d2z, gn[2], gn[1], gn[0], CUFFT_D2Z) != CUFFT_SUCCESS ||
      cufftPlan3d(&c->plan_z2d, gn[2], gn[1], gn[0], CUFFT_Z2D) != CUFFT_SUCCESS) {
    cufftDestroy(c->plan_z2z);
    dc_set_error("cufftPlan3d failed");
    return DC_ERR_CUDA;
  }
  c->have_plan = true;
  // fragment-point and per-state arrays
  DC_TRY(dmalloc(&c->d_vf64, (size_t)Lo.frag_points));
  DC_TRY(dmalloc(&c->d_vf32, (size_t)Lo.frag_points));
  long long cn = 0;
  for (auto &D : c->h_desc) cn += (long long)D.natom * D.norb;
  for (int k = 0; k < 2; ++k) {
    DC_TRY(dmalloc(&c->d_c64[k], (size_t)cn));
    DC_TRY(dmalloc(&c->d_c32[k], (size_t)cn));
  }
  long long sub = 0;
  for (auto &D : c->h_desc) sub += (long long)D.norb * D.norb;
  DC_TRY(dmalloc(&c->d_C64, (size_t)sub));
  DC_TRY(dmalloc(&c->d_C32, (size_t)sub));
  DC_TRY(dmalloc(&c->d_eps, (size_t)Lo.nstates));
  DC_TRY(dmalloc(&c->d_q, (size_t)Lo.nstates));
  DC_TRY(dmalloc(&c->d_occ, (size_t)Lo.nstates));
  DC_TRY(dmalloc(&c->d_dots, (size_t)Lo.nstates));
  DC_TRY(dmalloc(&c->d_q_x, (size_t)Lo.nstates));
  DC_TRY(dmalloc(&c->d_occ_x, (size_t)Lo.nstates));
  // the per-state arrays start at zero (they are readable through dc_get_state / dc_query before the
  // first solve fills them)
  for (double *d : {c->d_eps, c->d_q, c->d_occ, c->d_dots, c->d_q_x, c->d_occ_x})
    DC_CUDA(cudaMemset(d, 0, sizeof(double) * (size_t)std::max<long long>(1, Lo.nstates)));
  DC_TRY(dmalloc(&c->d_aux, 4));
  if (P.xc_fragment) {
    DC_TRY(dmalloc(&c->d_rhof, (size_t)Lo.frag_points));
    DC_TRY(dmalloc(&c->d_vcore, (size_t)c->npts));
  }
  DC_TRY(dmalloc(&c->d_bounds, (size_t)c->nfrag * (4 + 2 * P.cheb_degree)));
  DC_CUDA(cudaMemset(c->d_bounds, 0, sizeof(double) * (size_t)c->nfrag * (4 + 2 * P.cheb_degree)));
  DC_TRY(dmalloc(&c->d_flags, 8));
  DC_CUDA(cudaMemset(c->d_flags, 0, 8 * sizeof(unsigned)));
  DC_TRY(dmalloc(&c->d_scalar, 16));
  DC_CUDA(cudaMemset(c->d_scalar, 0, 16 * sizeof(double)));
  c->n_partials = 4096;
  DC_TRY(dmalloc(&c->d_partials, (size_t)c->n_partials));
  DC_TRY(dmalloc(&c->d_slot_w, (size_t)std::max<long long>(1, Lo.natom_frag)));
  DC_CUDA(cudaMallocHost((void **)&c->h_scalar_pinned, 32 * sizeof(double)));
  memset(c->h_scalar_pinned, 0, 32 * sizeof(double));
  c->prof_sink = &c->prof_pending;
  const char *graphs_env = getenv("DC_GRAPHS");
  c->graphs_enabled = !(graphs_env && graphs_env[0] == '0');
  // orbital blocks
  const size_t eb = (size_t)Lo.element_bytes;
  for (int k = 0; k < 3; ++k) {
    const cudaError_t e = cudaMalloc(&c->blk[k], eb * (size_t)Lo.psi_elems);
    if (e != cudaSuccess) {
      c->blk[k] = nullptr;
      return dc_cuda_status(e, "cudaMalloc(orbital block)");
    }
  }
  // ionic potential, starting density, starting orbitals
  cudaStream_t s = 0;
  DC_TRY(dck::launch_vion(c, s));
  if (P.precision == DC_FP64) {
    DC_TRY(dck::launch_init_psi(c, (double *)c->blk[0], s));
  } else {
    double *tmp = nullptr;
    DC_TRY(dmalloc(&tmp, (size_t)Lo.psi_elems));
    int st = dck::launch_init_psi(c, tmp, s);
    if (st == DC_OK) st = dck::launch_convert(tmp, (float *)c->blk[0], Lo.psi_elems, s);
    cudaStreamSynchronize(s);
    cudaFree(tmp);
    DC_TRY(st);
  }
  c->ib_psi = 0;
  DC_CUDA(cudaMemcpy(c->d_veff, c->d_vion, sizeof(double) * N, cudaMemcpyDeviceToDevice));
  DC_TRY(dck::launch_gather(c, s));
  DC_CUDA(cudaDeviceSynchronize());
  return check_flags(c, s);
}

int dc_init(const dc_grid_t *grid, const dc_fragments_t *fragments, const dc_buffers_t *buffers,
            const dc_atoms_t *atoms, const dc_params_t *params, dc_ctx **out) {
  if (!out) {
    dc_set_error("dc_init: out is NULL");
    return DC_ERR_ARG;
  }
  *out = nullptr;
  if (!grid || !fragments || !buffers || !atoms || !params) {
    dc_set_error("dc_init: NULL argument");
    return DC_ERR_ARG;
  }
  dc_ctx *c = new (std::nothrow) dc_ctx();
  if (!c) {
    dc_set_error("dc_init: host allocation failed");
    return DC_ERR_OOM;
  }
  int st;
  try {
    st = dc_init_impl(grid, fragments, buffers, atoms, params, c);
  } catch (...) {
    dc_set_error("dc_init: host exception (out of memory?)");
    st = DC_ERR_OOM;
  }
  if (st != DC_OK) {
    free_ctx(c);
    return st;
  }
  *out = c;
  return DC_OK;
}

void dc_finalize(dc_ctx *ctx) { free_ctx(ctx); }

int dc_query(const dc_ctx *ctx, dc_layout_t *out) {
  if (!ctx || !out) {
    dc_set_error("dc_query: NULL argument");
    return DC_ERR_ARG;
  }
  *out = ctx->layout;
  return DC_OK;
}

int dc_get_maps(const dc_ctx *c, int32_t *h_frag, int32_t *h_idx_map, int32_t *h_owner, int32_t *h_core_local,
                int32_t *h_atoms) {
  if (!c) {
    dc_set_error("dc_get_maps: NULL context");
    return DC_ERR_ARG;
  }
  if (h_frag)
    for (int f = 0; f < c->nfrag; ++f) {
      const FragDesc &D = c->h_desc[f];
      int32_t *o = h_frag + 12 * f;
      for (int d = 0; d < 3; ++d) {
        o[d] = D.org[d];
        o[3 + d] = D.E[d];
        o[6 + d] = D.c[d];
      }
      o[9] = D.norb;
      o[10] = D.natom;
      o[11] = 0;
    }
  if (h_idx_map) memcpy(h_idx_map, c->h_idx_map.data(), sizeof(int32_t) * c->h_idx_map.size());
  if (h_owner) memcpy(h_owner, c->h_owner.data(), sizeof(int32_t) * c->h_owner.size());
  if (h_core_local) memcpy(h_core_local, c->h_core_local.data(), sizeof(int32_t) * c->h_core_local.size());
  if (h_atoms) memcpy(h_atoms, c->h_atoms.data(), sizeof(int32_t) * c->h_atoms.size());
  return DC_OK;
}

int dc_get_initial(dc_ctx *c, double *d_vion, double *d_rho0, void *stream) {
  if (!c) return DC_ERR_ARG;
  const size_t N = (size_t)c->npts;
  if (d_vion) DC_CUDA(cudaMemcpyAsync(d_vion, c->d_vion, N * 8, cudaMemcpyDeviceToDevice, S(stream)));
  if (d_rho0) DC_CUDA(cudaMemcpyAsync(d_rho0, c->d_rho0, N * 8, cudaMemcpyDeviceToDevice, S(stream)));
  return DC_OK;
}

int dc_potential(dc_ctx *c, const double *d_rho, double *d_veff, void *stream) {
  if (!c || !d_rho) {
    dc_set_error("dc_potential: NULL argument");
    return DC_ERR_ARG;
  }
  DC_TRY(dck::launch_potential(c, d_rho, S(stream)));
  DC_TRY(dck::launch_gather(c, S(stream)));
  if (d_veff) DC_CUDA(cudaMemcpyAsync(d_veff, c->d_veff, 8 * (size_t)c->npts, cudaMemcpyDeviceToDevice, S(stream)));
  return DC_OK;
}

int dc_set_potential(dc_ctx *c, const double *d_veff, void *stream) {
  if (!c || !d_veff) {
    dc_set_error("dc_set_potential: NULL argument");
    return DC_ERR_ARG;
  }
  DC_CUDA(cudaMemcpyAsync(c->d_veff, d_veff, 8 * (size_t)c->npts, cudaMemcpyDeviceToDevice, S(stream)));
  DC_TRY(dck::launch_gather(c, S(stream)));
  return DC_OK;
}

int dc_hpsi(dc_ctx *c, const void *d_psi, void *d_hpsi, int dtype, void *stream) {
  if (!c || !d_psi || !d_hpsi || (dtype != DC_FP64 && dtype != DC_FP32)) {
    dc_set_error("dc_hpsi: invalid argument");
    return DC_ERR_ARG;
  }
  c->proj_ok = 0;  // projection buffer 0 holds the caller block's projections below
  const double es = dtype == DC_FP64 ? 8.0 : 4.0, blk = es * (double)c->layout.psi_elems;
  const double vfb = es * (double)c->layout.frag_points, pj = es * proj_elems(c);
  if (dtype == DC_FP64) {
    {
      StageScope sc(c, DC_STAGE_PROJECT, S(stream), blk + pj, 1);
      DC_TRY(dck::launch_project<double>(c, (const double *)d_psi, c->d_c64[0], S(stream)));
    }
    StageScope sc(c, DC_STAGE_HPSI, S(stream), 2.0 * blk + vfb + pj, 1);
    DC_TRY(dck::launch_hstep<double>(c, HSTEP_HPSI, 0, (const double *)d_psi, nullptr, (double *)d_hpsi, c->d_c64[0],
                                     nullptr, nullptr, nullptr, nullptr, nullptr, S(stream)));
  } else {
    {
      StageScope sc(c, DC_STAGE_PROJECT, S(stream), blk + pj, 1);
      DC_TRY(dck::launch_project<float>(c, (const float *)d_psi, c->d_c32[0], S(stream)));
    }
    StageScope sc(c, DC_STAGE_HPSI, S(stream), 2.0 * blk + vfb + pj, 1);
    DC_TRY(dck::launch_hstep<float>(c, HSTEP_HPSI, 0, (const float *)d_psi, nullptr, (float *)d_hpsi, c->d_c32[0],
                                    nullptr, nullptr, nullptr, nullptr, nullptr, S(stream)));
  }
  return DC_OK;
}

int dc_subspace(dc_ctx *c, void *d_psi, int dtype, double *d_eps, void *stream) {
  if (!c) {
    dc_set_error("dc_subspace: NULL context");
    return DC_ERR_ARG;
  }
  cudaStream_t s = S(stream);
  if (!d_psi) {
    DC_TRY(pass_ctx(c, false, 1, s));
    DC_TRY(check_flags(c, s));
    if (d_eps)
      DC_CUDA(cudaMemcpyAsync(d_eps, c->d_eps, 8 * (size_t)c->layout.nstates, cudaMemcpyDeviceToDevice, s));
    return DC_OK;
  }
  const int ctype = c->params.precision == DC_FP64 ? DC_FP64 : DC_FP32;
  if (dtype != ctype || !d_eps) {
    dc_set_error("dc_subspace: a caller block needs the context's element type (DC_FP64 for an FP64 context, "
                 "DC_FP32 otherwise) and an eps output");
    return DC_ERR_ARG;
  }
  if (ctype == DC_FP64) DC_TRY(subspace_block<double>(c, static_cast<double *>(d_psi), d_eps, s));
  else DC_TRY(subspace_block<float>(c, static_cast<float *>(d_psi), d_eps, s));
  return check_flags(c, s);
}

int dc_chefsi(dc_ctx *c, int n_pass, void *stream) {
  if (!c || n_pass < 0) {
    dc_set_error("dc_chefsi: invalid argument");
    return DC_ERR_ARG;
  }
  DC_TRY(pass_ctx(c, true, n_pass, S(stream)));
  return check_flags(c, S(stream));
}

int dc_warmup(dc_ctx *c, void *stream) {
  if (!c) return DC_ERR_ARG;
  cudaStream_t s = S(stream);
  DC_TRY(dck::launch_potential(c, c->d_rho0, s));
  DC_TRY(dck::launch_gather(c, s));
  c->proj_ok = 0;
  if (c->params.precision == DC_FP64) {
    DC_TRY(dck::launch_init_psi(c, (double *)c->blk[0], s));
    c->ib_psi = 0;
    if (c->hstep_shape[1] < 0) DC_TRY(tune<double>(c, (double *)c->blk[0], (double *)c->blk[1], s));
    DC_TRY(pass_ctx(c, false, 1, s));
    DC_TRY(check_flags(c, s));
    DC_TRY(pass_ctx(c, true, c->params.n_warmup, s));
  } else {
    // FP64 blocks for the warm-up, then convert the state to FP32
    const size_t ne = (size_t)c->layout.psi_elems;
    for (int k = 0; k < 3; ++k) DC_TRY(dmalloc(&c->blk64[k], ne));
    int ib = 0;
    int st = dck::launch_init_psi(c, c->blk64[0], s);
    if (st == DC_OK && c->hstep_shape[1] < 0) st = tune<double>(c, c->blk64[0], c->blk64[1], s);
    if (st == DC_OK) st = chefsi_pass<double>(c, c->blk64, ib, false, s);
    if (st == DC_OK) st = check_flags(c, s);
    for (int p = 0; st == DC_OK && p < c->params.n_warmup; ++p) st = chefsi_pass<double>(c, c->blk64, ib, true, s);
    if (st == DC_OK) st = dck::launch_convert(c->blk64[ib], (float *)c->blk[0], (long long)ne, s);
    c->proj_ok = 0;  // the FP32 state has no projections yet
    cudaStreamSynchronize(s);
    for (int k = 0; k < 3; ++k) {
      cudaFree(c->blk64[k]);
      c->blk64[k] = nullptr;
    }
    DC_TRY(st);
    c->ib_psi = 0;
    if (c->hstep_shape[0] < 0) DC_TRY(tune<float>(c, (float *)c->blk[0], (float *)c->blk[1], s));
  }
  if (c->params.xc_fragment) {
    // the first step's fragment densities: the warm state with its own Fermi level
    DC_TRY(density_stage(c, c->d_rho_out, s));
    DC_TRY(fragment_density(c, s));
  }
  DC_TRY(check_flags(c, s));
  c->warmed = true;
  c->steps_done = 0;
  return DC_OK;
}

int dc_get_state(dc_ctx *c, void *d_psi, double *d_eps, void *stream) {
  if (!c) return DC_ERR_ARG;
  if (d_psi)
    DC_CUDA(cudaMemcpyAsync(d_psi, c->blk[c->ib_psi], (size_t)c->layout.element_bytes * c->layout.psi_elems,
                            cudaMemcpyDeviceToDevice, S(stream)));
  if (d_eps) DC_CUDA(cudaMemcpyAsync(d_eps, c->d_eps, 8 * (size_t)c->layout.nstates, cudaMemcpyDeviceToDevice, S(stream)));
  return DC_OK;
}

int dc_set_state(dc_ctx *c, const void *d_psi, const double *d_eps, void *stream) {
  if (!c) return DC_ERR_ARG;
  if (d_psi)
    DC_CUDA(cudaMemcpyAsync(c->blk[c->ib_psi], d_psi, (size_t)c->layout.element_bytes * c->layout.psi_elems,
                            cudaMemcpyDeviceToDevice, S(stream)));
  if (d_eps) DC_CUDA(cudaMemcpyAsync(c->d_eps, d_eps, 8 * (size_t)c->layout.nstates, cudaMemcpyDeviceToDevice, S(stream)));
  if (d_psi) c->proj_ok = 0;
  if (c->params.xc_fragment && d_psi && d_eps) {
    // the next step's fragment densities: this state with its own Fermi level
    DC_TRY(density_stage(c, c->d_rho_out, S(stream)));
    DC_TRY(fragment_density(c, S(stream)));
    DC_TRY(check_flags(c, S(stream)));
  }
  c->warmed = true;
  return DC_OK;
}

int dc_density(dc_ctx *c, const void *d_psi, int dtype, const double *d_eps, double *d_rho, double *d_q,
               double *d_mu, void *stream) {
  if (!c || !d_rho) {
    dc_set_error("dc_density: NULL argument");
    return DC_ERR_ARG;
  }
  cudaStream_t s = S(stream);
  if (!d_psi) {
    DC_TRY(density_stage(c, d_rho, s));
    if (d_q) DC_CUDA(cudaMemcpyAsync(d_q, c->d_q, 8 * (size_t)c->layout.nstates, cudaMemcpyDeviceToDevice, s));
    if (d_mu) DC_CUDA(cudaMemcpyAsync(d_mu, c->d_scalar, 8, cudaMemcpyDeviceToDevice, s));
    return check_flags(c, s);
  }
  const int ctype = c->params.precision == DC_FP64 ? DC_FP64 : DC_FP32;
  if (dtype != ctype || !d_eps) {
    dc_set_error("dc_density: a caller block needs the context's element type and its eigenvalues d_eps");
    return DC_ERR_ARG;
  }
  if (c->nranks > 1) {
    dc_set_error("dc_density: the caller-block form needs every fragment (nranks = 1)");
    return DC_ERR_ARG;
  }
  // the caller block's weights, occupations and mu go to scratch, never to the context's own arrays
  double *q = d_q ? d_q : c->d_q_x;
  double *mu = c->d_aux;
  DC_CUDA(cudaMemsetAsync(mu, 0xff, sizeof(double), s));  // NaN: the solve starts from its bracket
  StageScope sc(c, DC_STAGE_DENSITY, s, 0.0, 3);
  if (ctype == DC_FP64) {
    DC_TRY(dck::launch_core_weights<double>(c, static_cast<const double *>(d_psi), q, s));
    DC_TRY(dck::launch_fermi(c, d_eps, q, mu, c->d_occ_x, s));
    DC_TRY(dck::launch_density<double>(c, static_cast<const double *>(d_psi), c->d_occ_x, d_rho, s));
  } else {
    DC_TRY(dck::launch_core_weights<float>(c, static_cast<const float *>(d_psi), q, s));
    DC_TRY(dck::launch_fermi(c, d_eps, q, mu, c->d_occ_x, s));
    DC_TRY(dck::launch_density<float>(c, static_cast<const float *>(d_psi), c->d_occ_x, d_rho, s));
  }
  if (d_mu) DC_CUDA(cudaMemcpyAsync(d_mu, mu, 8, cudaMemcpyDeviceToDevice, s));
  return check_flags(c, s);
}

int dc_selftest_wait(dc_ctx *c, void *stream) {
  if (!c) {
    dc_set_error("dc_selftest_wait: NULL context");
    return DC_ERR_ARG;
  }
  cudaStream_t s = S(stream);
  DC_TRY(dck::launch_wait_selftest(c, s));
  return check_flags(c, s);
}

int dc_lcfo_query(const dc_ctx *c, int64_t *basis_elems, int64_t *h_off) {
  if (!c || !basis_elems) {
    dc_set_error("dc_lcfo_query: NULL argument");
    return DC_ERR_ARG;
  }
  int64_t off = 0;
  for (size_t f = 0; f < c->h_desc.size(); ++f) {
    const FragDesc &D = c->h_desc[f];
    if (h_off) h_off[f] = off;
    off += (int64_t)D.norb * D.c[0] * D.c[1] * D.c[2];
  }
  *basis_elems = off;
  return DC_OK;
}

int dc_lcfo_basis(dc_ctx *c, const void *d_psi, int dtype, const double *d_eps, double eps_cut, double lambda_cut,
                  double *d_basis, int32_t *d_nbasis, double *d_s, void *stream) {
  if (!c || !d_psi || !d_eps || !d_basis || !d_nbasis) {
    dc_set_error("dc_lcfo_basis: NULL argument");
    return DC_ERR_ARG;
  }
  if (dtype != DC_FP64 && dtype != DC_FP32) {
    dc_set_error("dc_lcfo_basis: dtype must be DC_FP64 or DC_FP32");
    return DC_ERR_ARG;
  }
  if (!(lambda_cut >= 0.0) || eps_cut != eps_cut) {
    dc_set_error("dc_lcfo_basis: lambda_cut must be >= 0 and eps_cut a number");
    return DC_ERR_ARG;
  }
  cudaStream_t s = S(stream);
  double *sv = d_s ? d_s : c->d_work;
  if (!d_s && c->layout.nstates > c->npts) {
    dc_set_error("dc_lcfo_basis: workspace too small for the eigenvalues");
    return DC_ERR_ARG;
  }
  if (dtype == DC_FP64)
    DC_TRY(dck::launch_lcfo<double>(c, static_cast<const double *>(d_psi), d_eps, eps_cut, lambda_cut, d_basis,
                                    reinterpret_cast<int *>(d_nbasis), sv, s));
  else
    DC_TRY(dck::launch_lcfo<float>(c, static_cast<const float *>(d_psi), d_eps, eps_cut, lambda_cut, d_basis,
                                   reinterpret_cast<int *>(d_nbasis), sv, s));
  return DC_OK;
}

int dc_scf_step(dc_ctx *c, double *rho, int rho_on_host, dc_stats_t *h_stats, void *stream) {
  if (!c || !rho) {
    dc_set_error("dc_scf_step: NULL argument");
    return DC_ERR_ARG;
  }
  if (!c->warmed) {
    dc_set_error("dc_scf_step: call dc_warmup (or dc_set_state) first");
    return DC_ERR_STATE;
  }
  if (c->nranks > 1) {
    dc_set_error("dc_scf_step: a fragment shard steps with dc_step_local / dc_step_density / dc_step_finish");
    return DC_ERR_ARG;
  }
  cudaStream_t s = S(stream);
  const size_t nb = 8 * (size_t)c->npts;
  double *rin = rho;
  if (rho_on_host) {
    DC_CUDA(cudaMemcpyAsync(c->d_work, rho, nb, cudaMemcpyHostToDevice, s));
    rin = c->d_work;
  }
  // After one eager step (which also sets every kernel attribute), the device part of the step is
  // captured once per (state block, rho pointer, profiler on) and replayed as a CUDA graph.
  int gi = -1;
  if (c->graphs_enabled && c->steps_done >= 1) {
    for (size_t k = 0; k < c->graphs.size(); ++k)
      if (c->graphs[k].ib_before == c->ib_psi && c->graphs[k].rho == rin && c->graphs[k].prof == c->prof_on &&
          c->graphs[k].proj_before == c->proj_ok && c->graphs[k].pbuf_before == c->proj_buf)
        gi = (int)k;
    if (gi < 0) {
      if (c->graphs.size() >= 12) destroy_graphs(c);
      gi = capture_step(c, rin, s);
    }
  }
  if (gi >= 0) {
    DC_CUDA(cudaGraphLaunch(c->graphs[gi].exec, s));
    c->ib_psi = c->graphs[gi].ib_after;
    c->proj_ok = c->graphs[gi].proj_after;
    c->proj_buf = c->graphs[gi].pbuf_after;
  } else {
    DC_TRY(step_body(c, rin, s));
  }
  if (rho_on_host) DC_CUDA(cudaMemcpyAsync(rho, c->d_work, nb, cudaMemcpyDeviceToHost, s));
  DC_CUDA(cudaStreamSynchronize(s));
  if (gi >= 0 && c->graphs[gi].prof) prof_collect(c, c->graphs[gi].recs, false);
  int st = DC_OK;
  const unsigned fl = *reinterpret_cast<const unsigned *>(c->h_scalar_pinned + 20);
  if (fl & DC_FLAG_TIMEOUT) {
    dc_set_error("a bounded device wait ran out (grid barrier)");
    st = DC_ERR_TIMEOUT;
  } else if (fl & DC_FLAG_NOTSPD) {
    dc_set_error("Gram matrix not positive definite in at least one fragment");
    st = DC_ERR_NOCONV;
  } else if (fl & DC_FLAG_NONFINITE) {
    dc_set_error("non-finite eigenvalue or chemical potential");
    st = DC_ERR_NONFINITE;
  }
  c->steps_done++;
  if (h_stats) {
    const double *v = c->h_scalar_pinned;
    h_stats->mu = v[0];
    h_stats->eband = v[1];
    h_stats->drho = v[5];
    h_stats->ne = v[6];
    h_stats->E = v[8];
    h_stats->F = v[9];
    h_stats->step = c->steps_done;
    h_stats->status = st;
  }
  if (st != DC_OK) return st;
  const double *v = c->h_scalar_pinned;
  if (!(v[8] == v[8]) || !(v[0] == v[0]) || v[8] - v[8] != 0.0) {
    dc_set_error("dc_scf_step: non-finite energy or mu");
    return DC_ERR_NONFINITE;
  }
  return DC_OK;
}

// ---- fragment-sharded SCF step (Sec. 2.2 and 2.5) ---------------------------------------------------
int dc_step_local(dc_ctx *c, const double *d_rho_in, double *d_eps, double *d_q, void *stream) {
  if (!c || !d_rho_in || !d_eps || !d_q) {
    dc_set_error("dc_step_local: NULL argument");
    return DC_ERR_ARG;
  }
  if (!c->warmed) {
    dc_set_error("dc_step_local: call dc_warmup (or dc_set_state) first");
    return DC_ERR_STATE;
  }
  cudaStream_t s = S(stream);
  const bool keep_spectrum = c->params.hxc == DC_HXC_HARTREE_X;
  DC_TRY(dck::launch_potential(c, d_rho_in, s, keep_spectrum ? c->d_rhoinG : nullptr, true));
  DC_TRY(dck::launch_gather(c, s, c->params.xc_fragment ? d_rho_in : nullptr));
  DC_TRY(pass_ctx(c, true, c->params.n_pass, s));
  if (c->params.precision == DC_FP64)
    DC_TRY(dck::launch_core_weights<double>(c, (const double *)c->blk[c->ib_psi], c->d_q, s));
  else
    DC_TRY(dck::launch_core_weights<float>(c, (const float *)c->blk[c->ib_psi], c->d_q, s));
  const size_t ns = (size_t)c->layout.nstates, lo = (size_t)c->st_lo, cnt = (size_t)(c->st_hi - c->st_lo);
  DC_CUDA(cudaMemsetAsync(d_eps, 0, 8 * ns, s));
  DC_CUDA(cudaMemsetAsync(d_q, 0, 8 * ns, s));
  DC_CUDA(cudaMemcpyAsync(d_eps + lo, c->d_eps + lo, 8 * cnt, cudaMemcpyDeviceToDevice, s));
  DC_CUDA(cudaMemcpyAsync(d_q + lo, c->d_q + lo, 8 * cnt, cudaMemcpyDeviceToDevice, s));
  return check_flags(c, s);
}

int dc_step_density(dc_ctx *c, const double *d_eps, const double *d_q, double *d_rho_part, double *d_mu,
                    void *stream) {
  if (!c || !d_eps || !d_q || !d_rho_part) {
    dc_set_error("dc_step_density: NULL argument");
    return DC_ERR_ARG;
  }
  cudaStream_t s = S(stream);
  const size_t ns = (size_t)c->layout.nstates;
  if (d_eps != c->d_eps) DC_CUDA(cudaMemcpyAsync(c->d_eps, d_eps, 8 * ns, cudaMemcpyDeviceToDevice, s));
  if (d_q != c->d_q) DC_CUDA(cudaMemcpyAsync(c->d_q, d_q, 8 * ns, cudaMemcpyDeviceToDevice, s));
  // mu from every state (the same solve, from the same previous mu, on every rank)
  DC_TRY(dck::launch_fermi(c, c->d_eps, c->d_q, c->d_scalar, c->d_occ, s));
  if (c->params.precision == DC_FP64)
    DC_TRY(dck::launch_density<double>(c, (const double *)c->blk[c->ib_psi], c->d_occ, d_rho_part, s));
  else
    DC_TRY(dck::launch_density<float>(c, (const float *)c->blk[c->ib_psi], c->d_occ, d_rho_part, s));
  DC_TRY(fragment_density(c, s));
  if (d_mu) DC_CUDA(cudaMemcpyAsync(d_mu, c->d_scalar, 8, cudaMemcpyDeviceToDevice, s));
  return check_flags(c, s);
}

int dc_step_finish(dc_ctx *c, double *d_rho_in_out, const double *d_rho_out, dc_stats_t *h_stats, void *stream) {
  if (!c || !d_rho_in_out || !d_rho_out) {
    dc_set_error("dc_step_finish: NULL argument");
    return DC_ERR_ARG;
  }
  cudaStream_t s = S(stream);
  if (d_rho_out != c->d_rho_out)
    DC_CUDA(cudaMemcpyAsync(c->d_rho_out, d_rho_out, 8 * (size_t)c->npts, cudaMemcpyDeviceToDevice, s));
  const bool keep_spectrum = c->params.hxc == DC_HXC_HARTREE_X;
  DC_TRY(dck::launch_energy(c, d_rho_in_out, s));
  DC_TRY(dck::launch_mix(c, d_rho_in_out, s, keep_spectrum ? c->d_rhoinG : nullptr));
  DC_CUDA(cudaMemcpyAsync(c->h_scalar_pinned, c->d_scalar, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
  DC_TRY(check_flags(c, s));
  c->steps_done++;
  const double *v = c->h_scalar_pinned;
  if (h_stats) {
    h_stats->mu = v[0];
    h_stats->eband = v[1];
    h_stats->drho = v[5];
    h_stats->ne = v[6];
    h_stats->E = v[8];
    h_stats->F = v[9];
    h_stats->step = c->steps_done;
    h_stats->status = DC_OK;
  }
  if (!(v[8] == v[8]) || !(v[0] == v[0]) || v[8] - v[8] != 0.0) {
    dc_set_error("dc_step_finish: non-finite energy or mu");
    return DC_ERR_NONFINITE;
  }
  return DC_OK;
}

int dc_get_rho_out(dc_ctx *c, double *d_rho, void *stream) {
  if (!c || !d_rho) return DC_ERR_ARG;
  DC_CUDA(cudaMemcpyAsync(d_rho, c->d_rho_out, 8 * (size_t)c->npts, cudaMemcpyDeviceToDevice, S(stream)));
  return DC_OK;
}

int dc_eb_adjoint(dc_ctx *c, const void *d_psi, int dtype, const double *d_occ, const double *d_V, const double *d_D,
                  double *h_Eb, void *d_dpsi, double *d_dV, double *d_dD, void *stream) {
  if (c) c->proj_ok = 0;  // projection buffer 0 holds the caller block's projections
  if (!c || !d_psi || !d_occ || !d_V || !d_D || (dtype != DC_FP64 && dtype != DC_FP32)) {
    dc_set_error("dc_eb_adjoint: invalid argument");
    return DC_ERR_ARG;
  }
  if (c->nranks > 1) {
    dc_set_error("dc_eb_adjoint: needs every fragment (nranks = 1)");
    return DC_ERR_ARG;
  }
  cudaStream_t s = S(stream);
  if (!c->d_adj_vf64) {
    DC_TRY(dmalloc(&c->d_adj_vf64, (size_t)c->layout.frag_points));
    DC_TRY(dmalloc(&c->d_adj_vf32, (size_t)c->layout.frag_points));
    DC_TRY(dmalloc(&c->d_adj_fd, (size_t)c->layout.frag_points));
  }
  DC_TRY(dck::launch_gather_plain(c, d_V, c->d_adj_vf64, c->d_adj_vf32, s));
  if (dtype == DC_FP64) {
    const double *psi = (const double *)d_psi;
    DC_TRY(dck::launch_project<double>(c, psi, c->d_c64[0], s));
    DC_TRY(dck::launch_hstep<double>(c, HSTEP_ADJ, 0, psi, nullptr, (double *)d_dpsi, c->d_c64[0], nullptr, d_D, d_occ,
                                     c->d_dots, c->d_adj_vf64, s));
    if (d_dV) {
      DC_TRY(dck::launch_frag_density<double>(c, psi, d_occ, c->d_adj_fd, s));
      DC_TRY(dck::launch_gather_dV(c, c->d_adj_fd, d_dV, s));
    }
    if (d_dD) DC_TRY(dck::launch_dD(c, c->d_c64[0], nullptr, d_occ, d_dD, s));
  } else {
    const float *psi = (const float *)d_psi;
    DC_TRY(dck::launch_project<float>(c, psi, c->d_c32[0], s));
    DC_TRY(dck::launch_hstep<float>(c, HSTEP_ADJ, 0, psi, nullptr, (float *)d_dpsi, c->d_c32[0], nullptr, d_D, d_occ,
                                    c->d_dots, c->d_adj_vf32, s));
    if (d_dV) {
      DC_TRY(dck::launch_frag_density<float>(c, psi, d_occ, c->d_adj_fd, s));
      DC_TRY(dck::launch_gather_dV(c, c->d_adj_fd, d_dV, s));
    }
    if (d_dD) DC_TRY(dck::launch_dD(c, nullptr, c->d_c32[0], d_occ, d_dD, s));
  }
  if (h_Eb) {
    DC_TRY(dck::launch_sum(c->d_dots, c->layout.nstates, c->d_scalar + 14, c->d_partials, 0, s));
    DC_CUDA(cudaMemcpyAsync(c->h_scalar_pinned + 14, c->d_scalar + 14, 8, cudaMemcpyDeviceToHost, s));
    DC_CUDA(cudaStreamSynchronize(s));
    *h_Eb = c->h_scalar_pinned[14];
  }
  return DC_OK;
}

int dc_tuning(const dc_ctx *c, int *h_shape, float *h_ms) {
  if (!c || !h_shape) {
    dc_set_error("dc_tuning: NULL argument");
    return DC_ERR_ARG;
  }
  for (int t = 0; t < 2; ++t) {
    int *sh = h_shape + 3 * t;
    sh[0] = sh[1] = sh[2] = 0;
    if (c->hstep_shape[t] >= 0) dck::hstep_shape_info(c->hstep_shape[t], &sh[0], &sh[1], &sh[2]);
    if (h_ms)
      for (int k = 0; k < DC_TUNE_SLOTS; ++k) h_ms[DC_TUNE_SLOTS * t + k] = c->tune_ms[t][k];
  }
  return DC_OK;
}

int dc_set_tuning(dc_ctx *c, int dtype, int kind, int threads, int pairs) {
  if (!c || (dtype != DC_FP64 && dtype != DC_FP32)) {
    dc_set_error("dc_set_tuning: invalid argument");
    return DC_ERR_ARG;
  }
  const size_t esz = dtype == DC_FP64 ? sizeof(double) : sizeof(float);
  const int k = dck::hstep_shape_find(c, esz, kind, threads, pairs);
  if (k < 0) {
    dc_set_error("dc_set_tuning: no such launch shape, or it does not fit this context's fragments");
    return DC_ERR_ARG;
  }
  c->hstep_shape[dtype == DC_FP64 ? 1 : 0] = k;
  return DC_OK;
}

int dc_profile(dc_ctx *c, int enable) {
  if (!c) return DC_ERR_ARG;
  DC_CUDA(cudaDeviceSynchronize());
  prof_collect(c, c->prof_pending, true);
  if (enable) {
    for (int i = 0; i < DC_NSTAGES; ++i) {
      c->prof_ms[i] = c->prof_by[i] = 0.0;
      c->prof_nl[i] = 0;
    }
  }
  c->prof_on = enable != 0;
  c->prof_sink = &c->prof_pending;
  return DC_OK;
}

int dc_profile_read(dc_ctx *c, double *h_ms, int64_t *h_launches, double *h_bytes) {
  if (!c) return DC_ERR_ARG;
  DC_CUDA(cudaDeviceSynchronize());
  prof_collect(c, c->prof_pending, true);
  for (int i = 0; i < DC_NSTAGES; ++i) {
    if (h_ms) h_ms[i] = c->prof_ms[i];
    if (h_bytes) h_bytes[i] = c->prof_by[i];
    if (h_launches) h_launches[i] = c->prof_nl[i];
  }
  return DC_OK;
}

}  // extern "C"
