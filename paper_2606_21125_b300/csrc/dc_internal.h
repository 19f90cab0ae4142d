// Internal declarations of the DC-DFT fragment solver (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dcdft.h"

// ---------------------------------------------------------------------------------------------
// Fragment descriptor, one per fragment, resident on the device.
// ---------------------------------------------------------------------------------------------
struct FragDesc {
  int E[3];      // extent (core + 2b) per axis
  int b[3];      // buffer thickness = first core index in local coordinates
  int c[3];      // core length per axis
  int org[3];    // global index of local 0 (s_k - b, may be negative)
  int norb;      // n_f
  int natom;     // |A_f|
  int st_off;    // offset of the fragment's states in per-state arrays
  int at_off;    // offset of the fragment's atoms in per-(f,k) arrays
  long long psi_off;  // element offset of the fragment's orbital block
  long long pt_off;   // offset of the fragment's points in per-point arrays
  long long tab_off;  // offset of the fragment's projector factors (A_f * (Ex+Ey+Ez) values)
  long long c_off;    // offset of the fragment's projections (n_f * A_f values, orbital-major)
  long long sub_off;  // offset of the fragment's n_f x n_f matrices
  int zl_off;         // offset into the per-plane atom list starts (Ez + 1 entries)
  int row_off;        // offset into the per-row projector list starts (Ez * Ey + 1 entries)
};

// Row stride of one atom slot's projector factors [gx (Ex) | gy (Ey) | gz (Ez) | pad], kept even so
// that pairs of x-adjacent factors can be read as one vector.
__host__ __device__ inline int tab_width(const FragDesc &D) { return (D.E[0] + D.E[1] + D.E[2] + 1) & ~1; }

// Per-(fragment, atom slot) projector data.
struct ProjSlot {
  int atom;       // global atom index
  int lo[3];      // support [lo, hi) of the 1-D factor on each local axis
  int hi[3];
  double coef;    // (pi sigma^2)^(-3/4)
};

#define DC_TUNE_SLOTS 20   // candidate launch shapes of the stencil kernels (per element type)
#define DC_MAX_NORB 64     // subspace kernels hold n x n FP64 matrices in shared memory
#define DC_MAX_EXTENT 64   // stencil kernels hold padded planes of (E+8)^2 points

// Bounded device waits: number of polls before a wait gives up and sets the error flag.
#define DC_SPIN_LIMIT (1u << 22)

// Device-side error flags (bit set in ctx->d_flags[0]).
#define DC_FLAG_NOTSPD 1u
#define DC_FLAG_TIMEOUT 2u
#define DC_FLAG_NONFINITE 4u

struct ProfRec {
  cudaEvent_t a, b;
  int stage;
  double bytes;
  int nk;
};

struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  int ib_before = 0, ib_after = 0;
  int proj_before = 0, pbuf_before = 0, proj_after = 0, pbuf_after = 0;
  const double *rho = nullptr;
  bool prof = false;
  std::vector<ProfRec> recs;
};

struct dc_ctx {
  // configuration
  dc_grid_t grid;
  dc_fragments_t frag_cfg;
  dc_buffers_t buf_cfg;
  dc_params_t params;
  double h[3], dV, volume, ne;
  int natom, nspecies, nfrag;
  long long npts;
  dc_layout_t layout;
  int max_E[3];
  int max_atoms;      // max |A_f|
  int max_zlist;      // max over f of total per-plane list length
  int max_plane_ent;  // max over f and z of the row-list entries of one plane
  int max_frag_ent;   // max over f of the row-list entries of the whole fragment
  bool core_pairs;    // every fragment's core rows start at an even x with an even length, E_x even

  // host copies of maps (for dc_get_maps and launch planning)
  std::vector<FragDesc> h_desc;
  std::vector<int32_t> h_idx_map, h_owner, h_core_local, h_atoms;
  std::vector<double> h_pos, h_Zs, h_sigloc, h_sigproj, h_Ds;
  std::vector<int> h_species;
  std::vector<int2> h_items;  // (f, i) per state

  // device maps and tables
  FragDesc *d_desc = nullptr;
  int2 *d_items = nullptr;
  int32_t *d_idx_map = nullptr, *d_owner = nullptr, *d_core_local = nullptr;
  ProjSlot *d_slots = nullptr;
  double *d_tab64 = nullptr;   // projector 1-D factors (FP64)
  float *d_tab32 = nullptr;    // same in FP32
  int *d_zl_beg = nullptr;     // per-plane atom list starts
  int *d_zl_items = nullptr;   // per-plane atom slots
  int *d_row_beg = nullptr;    // per-row (z, y) list starts into d_row_ent
  int2 *d_row_ent = nullptr;   // (slot | y << 16, FP32 bits of gz(z) gy(y))
  int *d_row_split = nullptr;  // per row: entries reaching only the left half | (those plus both halves) << 16
  double *d_atom_D = nullptr;  // D per atom (global index)
  double *d_nl_bound = nullptr;  // per fragment: upper bound of the nonlocal operator (filter bounds)
  double *d_atom_pos = nullptr;
  int *d_atom_species = nullptr;
  double *d_species = nullptr;  // [4][nspecies]: Z, sigma_loc, sigma_proj, D
  // cover lists for the deterministic gather of dE/dV: per axis and global coordinate the
  // (fragment index along the axis, local index) pairs that cover it
  int *d_cover_beg[3] = {nullptr, nullptr, nullptr};
  int2 *d_cover[3] = {nullptr, nullptr, nullptr};

  // global grid arrays (FP64)
  double *d_vion = nullptr, *d_rho0 = nullptr, *d_veff = nullptr, *d_rho_out = nullptr, *d_work = nullptr;
  // Spectra: the per-step transforms are real-to-complex, on the half grid [nz][ny][nx/2 + 1] ("h");
  // the starting potential and density (once per context) use the full complex grid.
  long long nh = 0;            // half-grid points
  double2 *d_rhoiG = nullptr;  // rho_ion(G), full complex grid
  double *d_ig2 = nullptr;     // 1/G^2 per half-grid index (0 at G = 0), set once
  double *d_kerkw = nullptr;   // Kerker weight alpha G^2/(G^2 + q0^2)/N per half-grid index, set once
  double2 *d_rhoinG = nullptr; // the step's input density on the half grid (unnormalised forward FFT)
  double2 *d_cplx = nullptr;   // FFT work (full complex grid)
  double2 *d_cplxh = nullptr;  // FFT work (half grid)
  double *d_fftr = nullptr;    // real FFT output (N)
  cufftHandle plan_z2z = 0, plan_d2z = 0, plan_z2d = 0;
  bool have_plan = false;

  // per-fragment-point potential
  double *d_vf64 = nullptr;
  float *d_vf32 = nullptr;

  // orbital blocks: 3 rotating blocks of the context precision (index of the state in ib_psi)
  void *blk[3] = {nullptr, nullptr, nullptr};
  int ib_psi = 0;
  // FP64 blocks used by the warm-up of FP32/mixed contexts (freed after warm-up)
  double *blk64[3] = {nullptr, nullptr, nullptr};
  double *d_hy64 = nullptr;  // scratch for mixed (unused in FP64)

  // projections (n_f * A_f per fragment), two buffers (input / output of a step)
  double *d_c64[2] = {nullptr, nullptr};
  float *d_c32[2] = {nullptr, nullptr};
  // <p|Psi> of the state block is valid in buffer proj_buf when proj_ok equals the element size
  // (8 or 4); 0 = not valid (the next pass projects the block itself)
  int proj_ok = 0;
  int proj_buf = 0;

  // subspace arrays
  double *d_eps = nullptr;      // Ritz values [nstates]
  double *d_q = nullptr;        // core weights [nstates]
  double *d_occ = nullptr;      // occupations f [nstates]
  double *d_bounds = nullptr;   // per fragment: a, b_up, aL, shift, then 2*m step coefficients
  double *d_gram = nullptr;     // Gram partials [nchunk][2 n^2] per fragment
  long long gram_elems = 0;
  int gram_chunk = 0;           // points per Gram chunk
  long long *d_gram_off = nullptr;   // per fragment offset into d_gram
  int *d_gram_nchunk = nullptr;      // per fragment chunk count
  double *d_C64 = nullptr;      // rotation matrices [sub] (FP64)
  float *d_C32 = nullptr;       // same in FP32
  unsigned *d_flags = nullptr;  // device error flags
  double *d_scalar = nullptr;   // [16] mu, energies, reductions
  double *d_partials = nullptr; // reduction partials
  int n_partials = 0;
  double *h_scalar_pinned = nullptr;

  // work lists
  int2 *d_items2 = nullptr;      // (fragment, first orbital) of orbital pairs (two-orbital stencil)
  int n_items2 = 0;
  int2 *d_gram_items = nullptr;  // (fragment, chunk) of the Gram kernel
  int n_gram_items = 0;
  int2 *d_rot_items = nullptr;   // (fragment, 128-point chunk) of the FP64 rotation kernel
  int n_rot_items = 0;
  int2 *d_rot2_items = nullptr;  // (fragment, 256-point chunk) of the FP32 rotation kernel
  int n_rot2_items = 0;
  int *d_Fn = nullptr;           // num_fragment on the device
  // adjoint data: per-atom lists of (fragment, slot) entries, scratch
  int *d_atom_slot_beg = nullptr, *d_atom_slots = nullptr;
  double *d_slot_w = nullptr;
  double *d_adj_vf64 = nullptr;
  float *d_adj_vf32 = nullptr;
  double *d_adj_fd = nullptr;
  double *d_dots = nullptr;

  // stage profiler: event pairs recorded around each stage; eager records wait in prof_pending,
  // records captured into a CUDA graph belong to that graph and are read after each replay
  bool prof_on = false;
  std::vector<ProfRec> prof_pending;
  std::vector<ProfRec> *prof_sink = nullptr;  // where new records go (pending or a graph's list)
  std::vector<cudaEvent_t> prof_free;
  double prof_ms[DC_NSTAGES] = {0}, prof_by[DC_NSTAGES] = {0};
  long long prof_nl[DC_NSTAGES] = {0};

  // CUDA graphs of the SCF step, keyed by (state block, rho pointer, profiler on)
  std::vector<StepGraph> graphs;
  bool graphs_enabled = true;

  // autotuned launch shape of the stencil kernel per element type ([0] FP32, [1] FP64; -1 = default)
  int hstep_shape[2] = {-1, -1};
  float tune_ms[2][DC_TUNE_SLOTS] = {{0}};

  int steps_done = 0;
  bool warmed = false;
  int sm_count = 0;

  // fragment shard of this context (rank of nranks, Sec. 2.5): fragments [f_lo, f_hi) and their states
  // [st_lo, st_hi) are solved here; everything else (maps, potentials, the Fermi level, energies) is global
  int rank = 0, nranks = 1;
  int f_lo = 0, f_hi = 0;
  long long st_lo = 0, st_hi = 0;
  // scratch of the caller-block forms of dc_subspace/dc_density (so the context's own state is kept)
  double *d_q_x = nullptr, *d_occ_x = nullptr, *d_aux = nullptr;
  int *d_frag_order = nullptr;  // the shard's fragments, longest (most orbitals) first
  // per-fragment exchange (params.xc_fragment): sum_i f_i psi_i^2 on every fragment point (the fragment
  // density is twice this) and the potential each core point felt
  double *d_rhof = nullptr, *d_vcore = nullptr;
};

// Host-built projector tables, uploaded by dc_init.
struct HostTables {
  std::vector<ProjSlot> slots;
  std::vector<double> tab;
  std::vector<int> zl_beg, zl_items;
  std::vector<int> row_beg;
  std::vector<int2> row_ent;
  std::vector<int> row_split;
};
int dc_build_host(dc_ctx *c, const dc_atoms_t *atoms, HostTables &out);
// Fragment range [*lo, *hi) of rank `rank` of `nranks` (1 <= nranks <= nfrag): contiguous ids, each
// boundary the first fragment whose cost prefix reaches rank/nranks of the total (integer comparison),
// kept at least one fragment past the previous boundary and room for the ranks after it.
void dc_shard_range(const long long *cost, int nfrag, int rank, int nranks, int *lo, int *hi);
void dc_build_cover(const dc_ctx *c, int d, std::vector<int> &beg, std::vector<int2> &items);

// ---------------------------------------------------------------------------------------------
// Error plumbing
// ---------------------------------------------------------------------------------------------
void dc_set_error(const std::string &msg);
int dc_cuda_status(cudaError_t e, const char *what);

// Raise a kernel's dynamic shared-memory limit on the current device, once per (device, kernel, size):
// later calls (including those made while a stream is being captured) do no CUDA API work.
cudaError_t dc_set_smem(const void *func, size_t bytes);

#define DC_CUDA(call)                                          \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return dc_cuda_status(_e, #call);   \
  } while (0)

#define DC_TRY(call)              \
  do {                            \
    int _s = (call);              \
    if (_s != DC_OK) return _s;   \
  } while (0)

// ---------------------------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files)
// ---------------------------------------------------------------------------------------------
namespace dck {
// global stages
int launch_vion(dc_ctx *c, cudaStream_t s);
// with_fragment_xc: a context with per-fragment exchange leaves v_x to the gather (the SCF step); the
// warm-up and dc_potential keep the global exchange
int launch_potential(dc_ctx *c, const double *rho, cudaStream_t s, double2 *save_rhoG = nullptr,
                     bool with_fragment_xc = false);
// rho_in != nullptr: per-fragment exchange and density-template terms from d_rhof (and rho_in), and the
// core-point potential d_vcore for the energy
int launch_gather(dc_ctx *c, cudaStream_t s, const double *rho_in = nullptr);
int launch_gather_plain(dc_ctx *c, const double *V, double *vf64, float *vf32, cudaStream_t s);
int launch_energy(dc_ctx *c, const double *rho_in, cudaStream_t s);
int launch_mix(dc_ctx *c, double *rho_in, cudaStream_t s, const double2 *rho_in_G = nullptr);
int launch_init_psi(dc_ctx *c, double *psi64, cudaStream_t s);
int launch_convert(const double *src, float *dst, long long n, cudaStream_t s);
int launch_convert(const float *src, double *dst, long long n, cudaStream_t s);

// fragment Hamiltonian
template <typename T>
int launch_project(dc_ctx *c, const T *psi, T *cout, cudaStream_t s);
template <typename T>
int tune_hstep(dc_ctx *c, const T *y, T *out, T *cbuf, cudaStream_t s);
int hstep_shape_info(int shape, int *kind, int *threads, int *pairs);
int hstep_shape_find(const dc_ctx *c, size_t esz, int kind, int threads, int pairs);
template <typename T>
int launch_hstep(dc_ctx *c, int mode, int step, const T *yin, const T *yprev, T *yout, const T *cin, T *cout,
                 const double *Datom, const double *occ, double *dots, const T *vf, cudaStream_t s);
// true when FP32 H-applies of this context run the specialised kernel (the only one with HSTEP_HLOC)
bool hstep_specialised(const dc_ctx *c);
// specialised FP32 kernel (uniform cubic fragments, zero boundary, isotropic spacing): the compiled extent
// it runs for this context, or 0; and its launch (HSTEP_CHEB / HSTEP_HPSI / HSTEP_HLOC, input projections
// required)
int cheb_extent(const dc_ctx *c);
int launch_cheb(dc_ctx *c, int mode, int step, const float *yin, const float *yprev, float *yout, const float *cin,
                float *cout, cudaStream_t s);

// subspace
int launch_bounds(dc_ctx *c, int first, cudaStream_t s);
template <typename T>
int launch_gram(dc_ctx *c, const T *Y, const T *HY, cudaStream_t s);
int launch_gram_tc(dc_ctx *c, const float *Y, const float *HY, cudaStream_t s);
int launch_rotate_tc(dc_ctx *c, const float *Y, float *out, cudaStream_t s);
// 2-D tensor map over an FP32 block viewed as `rows` rows of `inner` elements (inner a multiple of 4,
// base 16-byte aligned), box (box_inner, box_rows), zero fill out of range, optional 128-byte swizzle;
// false when the driver's encoder is unavailable or the shape does not qualify.
bool tensor_map_rows(CUtensorMap *map, const float *base, long long inner, long long rows, int box_inner,
                     int box_rows, bool swizzle128);
// cnl: when not null, the FP32 projections <p|Y> (per fragment at c_off, orbital-major) of a block whose
// H Y holds only the local part of H; their nonlocal term sum_a D_a <p_a|y_i><p_a|y_j> is added to A
int launch_subspace(dc_ctx *c, int precision_bits, double *eps, cudaStream_t s, const float *cnl = nullptr);
template <typename T>
int launch_lcfo(dc_ctx *c, const T *psi, const double *eps, double eps_cut, double lambda_cut, double *basis,
                int *nbasis, double *s_out, cudaStream_t s);
template <typename T>
int launch_rotate(dc_ctx *c, const T *Y, T *out, cudaStream_t s);
template <typename T>
int launch_rotate_proj(dc_ctx *c, const T *cin, T *cout, cudaStream_t s);

// density
// core weights of the owned fragments' states into q[nstates] (other entries untouched)
template <typename T>
int launch_core_weights(dc_ctx *c, const T *psi, double *q, cudaStream_t s);
// mu (in: starting guess, out: root) and occupations of all nstates states
int launch_fermi(dc_ctx *c, const double *eps, const double *q, double *mu, double *occ, cudaStream_t s);
int launch_wait_selftest(dc_ctx *c, cudaStream_t s);
// rho[npts] on the owned fragments' cores; zero elsewhere when the context owns a shard
template <typename T>
int launch_density(dc_ctx *c, const T *psi, const double *occ, double *rho, cudaStream_t s);

// adjoint
template <typename T>
int launch_frag_density(dc_ctx *c, const T *psi, const double *occ, double *fd, cudaStream_t s,
                        bool shard_only = false);
int launch_gather_dV(dc_ctx *c, const double *fd, double *dV, cudaStream_t s);
int launch_dD(dc_ctx *c, const double *cproj64, const float *cproj32, const double *occ, double *dD, cudaStream_t s);
int launch_sum(const double *x, long long n, double *out, double *partials, int npart, cudaStream_t s);
}  // namespace dck

// modes of launch_hstep
#define HSTEP_HPSI 0  // out = H y
#define HSTEP_CHEB 1  // out = alpha (H y - shift y) + beta yprev
#define HSTEP_ADJ 2   // out = 2 occ dV H y ; dots[item] = occ dV <y|H y>
#define HSTEP_HLOC 3  // out = (-1/2 L8 + V) y, the local part of H (the specialised FP32 kernel only)
