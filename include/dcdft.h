/*
 * dcdft.h -- C ABI of the B300-native divide-and-conquer DFT fragment solver.
 *
 * The library implements the data-parallel inner part of one DC-DFT SCF
 * iteration (Sec. 2.2 of "SALMON 2.3: Implementation of divide-and-conquer
 * ground-state initialization for large-scale real-time TDDFT"): the periodic
 * cell is split into overlapping fragments (core plus buffer, Sec. 2.2 and
 * Table 1), each fragment Kohn-Sham problem (Eq. 1, Hamiltonian Eq. 5) is
 * solved for its lowest states, the global chemical potential fixes N_e, and
 * the fragment densities are projected onto their cores and summed (Eqs. 2-4).
 *
 * Conventions used by every call:
 *  - Units: Hartree atomic units (Ha, bohr).
 *  - Status: every int-returning call gives 0 (DC_OK) or a negative DC_ERR_*
 *    code; no call aborts, throws, or leaves a CUDA error pending on return.
 *    dc_error_string() names a code; dc_last_error() returns a one-line
 *    description of the last failure in this process.
 *  - Ownership: the caller owns every pointer argument; the library never
 *    keeps a pointer after a call returns.  The library owns the context
 *    (maps, projector tables, the orbital state and its work blocks, FFT
 *    plans), allocated in dc_init and freed in dc_finalize.
 *  - Memory spaces: arguments named d_* are device pointers (CUDA global
 *    memory on the current device); h_* are host pointers.
 *  - Streams: device work is issued on the given cudaStream_t (passed as
 *    void*, NULL = legacy default stream); calls that return host results
 *    synchronise that stream.  A context is not thread-safe.
 *  - Layouts:
 *      global grid arrays  [Nz][Ny][Nx], x fastest, g = x + Nx (y + Ny z);
 *      fragment id         f = kx + Fx (ky + Fy kz);
 *      orbital blocks      concatenation over f of [n_f][Ez][Ey][Ex] (x fastest),
 *                          fragment f starting at element psi_offset[f];
 *      per-state arrays    concatenation over f of [n_f] (state_offset[f]).
 *  - Element type of orbital blocks: double for DC_FP64, float for DC_FP32 and
 *    DC_MIXED (the "dtype" arguments take DC_FP64 or DC_FP32).
 */
#ifndef DCDFT_H
#define DCDFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define DC_OK 0
#define DC_ERR_ARG (-1)       /* invalid argument, size or configuration */
#define DC_ERR_CUDA (-2)      /* a CUDA runtime or cuFFT call failed */
#define DC_ERR_OOM (-3)       /* device allocation failed */
#define DC_ERR_NOCONV (-4)    /* a Gram matrix was not positive definite (Cholesky failed) */
#define DC_ERR_TIMEOUT (-5)   /* a bounded device-side wait ran out; the kernel returned early */
#define DC_ERR_NONFINITE (-6) /* NaN or Inf in an energy, mu or an eigenvalue */
#define DC_ERR_STATE (-7)     /* call out of order (e.g. dc_scf_step before dc_warmup) */

/* ---- enumerations ---------------------------------------------------------------------- */
#define DC_FP64 0  /* all fragment arithmetic in FP64 */
#define DC_FP32 1  /* FP32 stencil, Gram and rotation; FP64 subspace solves and Fermi level */
#define DC_MIXED 2 /* FP32 stencil; Gram/Rayleigh-Ritz on tensor cores from split BF16 words */

#define DC_BC_ZERO 0     /* fragment ghost points are zero (buffer edge) */
#define DC_BC_PERIODIC 1 /* ghost points wrap within the fragment extent (Sec. 2.2) */

#define DC_HXC_NONE 0      /* V_eff = V_loc only (non-interacting model) */
#define DC_HXC_HARTREE_X 1 /* V_eff = V_loc + V_H[rho] + v_x[rho] (Eq. 5, LDA exchange) */

/* ---- configuration --------------------------------------------------------------------- */
/* Periodic orthorhombic cell: n grid points and length L (bohr) per axis; h = L/n. */
typedef struct {
  int n[3];
  double L[3];
} dc_grid_t;

/* Table 1: num_fragment(1:3), nstate_frag.  nstate_frag > 0 fixes the orbital count of every
 * fragment; nstate_frag == 0 derives it from the electrons of the atoms that have an image in the
 * fragment box: n_f = ceil(Ne_f/2) + max(4, ceil(0.2 ceil(Ne_f/2))).  bc: DC_BC_*. */
typedef struct {
  int num_fragment[3];
  int bc;
  int nstate_frag;
} dc_fragments_t;

/* Table 1: num_rgrid_buffer(1:3), the buffer thickness b in grid points (Sec. 2.2). */
typedef struct {
  int num_rgrid_buffer[3];
} dc_buffers_t;

/* Atoms (host arrays, read during dc_init only).  pos[natom][3] in bohr; species[natom] in
 * [0, nspecies).  Per species: valence charge Z, Gaussian width of the local ion charge
 * sigma_loc, projector width sigma_proj and projector strength D (Ha). */
typedef struct {
  int natom;
  const double *pos;
  const int *species;
  int nspecies;
  const double *Z;
  const double *sigma_loc;
  const double *sigma_proj;
  const double *D;
} dc_atoms_t;

/* Solver parameters.  precision: DC_FP64/DC_FP32/DC_MIXED.  cheb_degree: Chebyshev filter degree
 * m (>= 1).  n_pass: CheFSI passes per SCF step.  n_warmup: passes in the starting potential before
 * the first step (run in FP64 for every precision).  hxc: DC_HXC_*.  kT: electronic temperature
 * (Ha, > 0).  mix_alpha: linear mixing weight in [0, 1]; 0 keeps rho_in fixed (the paper's fixed-density
 * DC, Sec. 2.5 use case 3).  seed: initial-orbital seed.  kerker_q0 (bohr^-1, >= 0): 0 gives plain
 * linear mixing; > 0 weights every Fourier component of the density residual by
 * mix_alpha G^2/(G^2 + q0^2) (Kerker preconditioning against long-wavelength charge sloshing).
 * rank, nranks: the context's fragment shard (Sec. 2.5: fragments are distributed over processes).
 * nranks = 0 or 1: the context solves every fragment.  nranks > 1 (at most the number of fragments):
 * the context solves only the contiguous fragment range of `rank` (dc_query: frag_lo, frag_hi), chosen
 * so that every rank's stencil work sum P_f n_f is about 1/nranks of the total; every rank still holds
 * the global grid, maps and potentials.  The sharded SCF step is dc_step_local / dc_step_density /
 * dc_step_finish with the caller's exchanges between them.
 * xc_fragment (0 or 1) and xi (>= 0): Eq. 5's per-fragment terms.  0 (default): one global V_eff with the
 * exchange of rho_in.  1 (needs DC_HXC_HARTREE_X and nranks <= 1): fragment f's potential on its point j
 * (global point g) is V_loc(g) + V_H[rho_in](g) + v_x(rho_f(j)) + (rho_f(j) - rho_in(g))/xi (the last term
 * only for xi > 0, the density-template potential), rho_f = sum_i 2 f_i |psi_i|^2 on every point of the
 * fragment (Eq. 3 before the core projection) from the orbitals and occupations the previous step ended
 * with (after dc_warmup or dc_set_state with psi and eps: of that state at its own Fermi level); the
 * energy's double counting uses the potential of the fragment owning each core point. */
typedef struct {
  int precision;
  int cheb_degree;
  int n_pass;
  int n_warmup;
  int hxc;
  double kT;
  double mix_alpha;
  uint64_t seed;
  double kerker_q0;
  int rank;
  int nranks;
  int xc_fragment;
  double xi;
} dc_params_t;

/* Sizes of everything a caller allocates for the calls below. */
typedef struct {
  int nfrag;           /* number of fragments F = Fx Fy Fz */
  int natom;           /* atoms */
  int64_t npts;        /* global grid points Nx Ny Nz */
  int64_t psi_elems;   /* elements of one orbital block: sum_f n_f P_f */
  int64_t frag_points; /* sum_f P_f (length of the fragment-point maps) */
  int64_t nstates;     /* sum_f n_f */
  int64_t natom_frag;  /* sum_f |A_f| (atoms whose projector touches fragment f) */
  int max_norb;        /* max_f n_f */
  int element_bytes;   /* 8 for DC_FP64, 4 otherwise */
  int frag_lo, frag_hi;        /* fragments [frag_lo, frag_hi) are solved by this context (all of them
                                  unless nranks > 1) */
  int64_t state_lo, state_hi;  /* their states in per-state arrays */
} dc_layout_t;

/* Per-step results (host struct filled by dc_scf_step). */
typedef struct {
  double E;     /* total energy (Ha) */
  double F;     /* free energy E - kT S (Ha) */
  double eband; /* sum_f sum_i 2 f_i eps_i q_i (Ha) */
  double mu;    /* chemical potential (Ha) */
  double drho;  /* int |rho_out - rho_in| / N_e */
  double ne;    /* int rho_out (should equal N_e) */
  int step;     /* SCF steps done so far */
  int status;   /* DC_OK or the first error seen during the step */
} dc_stats_t;

typedef struct dc_ctx dc_ctx;

/* ---- lifecycle ------------------------------------------------------------------------- */
/* Build the fragment decomposition (Sec. 2.2, Table 1), the per-fragment atom lists and
 * projector factors, the ionic potential V_loc and ion charge rho_ion(G) (on the device, via
 * cuFFT), the starting density (band-limited ion charge scaled to N_e) and the random starting
 * orbitals; allocate the orbital state and work blocks.  Synchronous.  On failure *out is NULL
 * and nothing is leaked.  Errors: DC_ERR_ARG (sizes, counts, more than 4096 fragments, n_f outside [1, 64], extents above 64),
 * DC_ERR_OOM, DC_ERR_CUDA. */
int dc_init(const dc_grid_t *grid, const dc_fragments_t *fragments, const dc_buffers_t *buffers,
            const dc_atoms_t *atoms, const dc_params_t *params, dc_ctx **out);
void dc_finalize(dc_ctx *ctx);
const char *dc_error_string(int status);
const char *dc_last_error(void);

/* Sizes of caller-allocated arrays. */
int dc_query(const dc_ctx *ctx, dc_layout_t *out);

/* Fragment maps (Sec. 2.2), host outputs, for bit-exact checks; any pointer may be NULL.
 *  h_frag[f*12 + 0..11] = origin[3] (s_k - b, may be negative), extent[3], core[3], n_f,
 *                         |A_f|, 0;
 *  h_idx_map[frag_points]  = global index of each fragment point (fragment f at
 *                            sum_{f'<f} P_f');
 *  h_owner[npts], h_core_local[npts] = fragment whose core holds g and g's local index there;
 *  h_atoms[natom_frag]     = global indices of A_f, ascending, concatenated over f. */
int dc_get_maps(const dc_ctx *ctx, int32_t *h_frag, int32_t *h_idx_map, int32_t *h_owner,
                int32_t *h_core_local, int32_t *h_atoms);

/* ---- potentials ------------------------------------------------------------------------ */
/* Copy the ionic potential V_loc[npts] and the starting density rho_0[npts] (FP64, device). */
int dc_get_initial(dc_ctx *ctx, double *d_vion, double *d_rho0, void *stream);

/* V_eff = V_loc + V_H[rho] + v_x[rho] (or V_loc for DC_HXC_NONE) from d_rho[npts] (Eq. 5);
 * stores it in the context (used by every later H application) and copies it to d_veff
 * (may be NULL).  Poisson by cuFFT, G=0 dropped. */
int dc_potential(dc_ctx *ctx, const double *d_rho, double *d_veff, void *stream);

/* Store an arbitrary V_eff[npts] (FP64, device) as the context's potential. */
int dc_set_potential(dc_ctx *ctx, const double *d_veff, void *stream);

/* ---- fragment Hamiltonian ---------------------------------------------------------------- */
/* d_hpsi = H_f d_psi for every fragment and orbital of a caller block in the layout above (Eq. 5
 * model Hamiltonian: -1/2 of the 8th-order FD Laplacian with the fragment boundary condition,
 * the context's V_eff restricted to the fragment, and sum_a D_a p_a <p_a|psi>).  dtype selects
 * double or float elements (DC_FP64 or DC_FP32).  d_psi and d_hpsi must not overlap. */
int dc_hpsi(dc_ctx *ctx, const void *d_psi, void *d_hpsi, int dtype, void *stream);

/* ---- fragment eigensolver (CheFSI) ------------------------------------------------------ */
/* Rayleigh-Ritz without filtering (Eq. 1 in the span of a block; Sec. 2.2 "orthonormalization" and
 * "diagonalization"): per fragment S = <Y|Y> (dV-weighted), S = L L^T (FP64 Cholesky), Hs = L^-1 <Y|H Y> L^-T
 * = Q diag(eps) Q^T (FP64 results, ascending eps), Y <- Y L^-T Q.  The Gram contractions run in the
 * context precision (DC_MIXED: 3xBF16 words on tensor cores, FP32 accumulation).
 *   d_psi == NULL: acts on the context's own orbital state (used once on the random start); d_eps (may
 *                  be NULL) receives a copy of the Ritz values; dtype is ignored.
 *   d_psi != NULL: a caller block in the dc_query layout (device), rotated in place, with element type
 *                  dtype equal to the context's (DC_FP64 for an FP64 context, DC_FP32 otherwise);
 *                  d_eps[nstates] (device, FP64, required) receives its Ritz values.  The context's own
 *                  state, eigenvalues, core weights and mu are not changed; its work blocks and projection
 *                  buffers are used as scratch.
 * With nranks > 1 only the context's fragment range is processed.  Errors: DC_ERR_ARG (NULL context,
 * wrong dtype, missing d_eps), DC_ERR_NOCONV (a Gram matrix not positive definite), DC_ERR_CUDA. */
int dc_subspace(dc_ctx *ctx, void *d_psi, int dtype, double *d_eps, void *stream);
/* n_pass CheFSI passes on every fragment in the current V_eff: degree-m scaled Chebyshev filter
 * with bounds from the previous Ritz values, Cholesky orthonormalisation of the Gram matrix,
 * Rayleigh-Ritz and rotation (Eq. 1).  Gram/RR in the context precision, subspace solves FP64. */
int dc_chefsi(dc_ctx *ctx, int n_pass, void *stream);
/* Starting potential from the starting density, Rayleigh-Ritz of the random block and n_warmup
 * CheFSI passes (all in FP64; the state is then converted to the context precision). */
int dc_warmup(dc_ctx *ctx, void *stream);

/* Copy the orbital state (element type of the context) and the Ritz values eps[nstates] out
 * (device); either pointer may be NULL.  dc_set_state loads them in. */
int dc_get_state(dc_ctx *ctx, void *d_psi, double *d_eps, void *stream);
int dc_set_state(dc_ctx *ctx, const void *d_psi, const double *d_eps, void *stream);

/* ---- density -------------------------------------------------------------------------- */
/* Core weights q_i^f = <psi_i|1_core|psi_i>, the chemical potential with
 * sum_f sum_i 2 f((eps_i^f - mu)/kT) q_i^f = N_e (FP64 safeguarded Newton in the bisection bracket,
 * Sec. 2.2), and the core-projected density rho_out(g) = sum_i 2 f_i^f psi_i^f(j)^2 with f = owner(g)
 * (Eqs. 2-4).
 *   d_psi == NULL: from the context's own state and eigenvalues (d_eps and dtype ignored); the
 *                  context keeps q, the occupations and mu for its energy stage.
 *   d_psi != NULL: from a caller block (dc_query layout, dtype equal to the context's element type) and
 *                  its eigenvalues d_eps[nstates] (device, FP64, required); the context's own arrays
 *                  are not changed.  Needs nranks = 1.
 * Outputs (device, FP64): d_rho[npts] (required); d_q[nstates] and d_mu[1] may be NULL.
 * Errors: DC_ERR_ARG, DC_ERR_TIMEOUT (the Fermi solve's bounded grid barrier), DC_ERR_NONFINITE,
 * DC_ERR_CUDA. */
int dc_density(dc_ctx *ctx, const void *d_psi, int dtype, const double *d_eps, double *d_rho, double *d_q,
               double *d_mu, void *stream);

/* ---- failure detection ----------------------------------------------------------------- */
/* Self-test of the library's bounded device waits; the paper has no counterpart.  It runs the grid
 * barrier of the Fermi-level kernel on a launch one block short of the arrivals the barrier expects,
 * so the wait can never complete: each block gives up after its bounded poll count (a fraction of a
 * second to about a second), records the timeout in the context's device flags and returns.  The
 * call then reads the flags, clears them and returns DC_ERR_TIMEOUT; the context stays usable.  It
 * would return DC_OK only if the barrier passed, i.e. if the bound were broken.  DC_ERR_ARG for a
 * NULL context. */
int dc_selftest_wait(dc_ctx *ctx, void *stream);

/* ---- DC-LCFO basis (Sec. 2.3, Eqs. 6-7) -------------------------------------------------- */
/* Size of the basis output of dc_lcfo_basis: *basis_elems = sum over fragments of n_f |core_f|
 * (FP64 elements); h_off (host, nfrag entries, may be NULL) receives each fragment's element offset.
 * Returns DC_ERR_ARG for a NULL context or basis_elems. */
int dc_lcfo_query(const dc_ctx *ctx, int64_t *basis_elems, int64_t *h_off);
/* The basis-construction step of DC-LCFO on every fragment.  Orbitals i of fragment f with
 * eps_i < eps_cut (strict, in orbital order) are projected onto the core (zero outside it, Eq. 3),
 * their overlap S_ij = <phibar_i|phibar_j> (dV sum over core points, Eq. 6) is diagonalised in FP64,
 * eigenvectors with eigenvalue s <= lambda_cut are dropped, and the kept ones, in descending order of
 * s, give the basis lambda_k = sum_i phibar_i U_ik / sqrt(s_k), orthonormal on the core (Eq. 7).
 *   d_psi     orbital block in the layout of dc_query (device), element type dtype (DC_FP64 or
 *             DC_FP32; FP32 values are widened to FP64 before any arithmetic).
 *   d_eps     eigenvalues of those orbitals, nstates FP64 (device), in the block's state order.
 *   eps_cut   selection energy (Ha), e.g. mu + 0.1 eV; lambda_cut >= 0 the overlap threshold.
 *   d_basis   (device, FP64, dc_lcfo_query elements) fragment f's row k (k < n_f) at element
 *             h_off[f] + k |core_f|, core points [c_z][c_y][c_x] with x fastest; rows k >= m_f are 0.
 *   d_nbasis  (device, int32, nfrag) m_f, the number of kept functions.
 *   d_s       (device, FP64, nstates, may be NULL) the eigenvalues of S per fragment in descending
 *             order, 0 past the selected count.
 * All arguments are caller-owned; the call is stream-ordered on `stream` and writes nothing else.
 * Errors: DC_ERR_ARG for NULL pointers, a bad dtype or lambda_cut < 0 (nothing is written). */
int dc_lcfo_basis(dc_ctx *ctx, const void *d_psi, int dtype, const double *d_eps, double eps_cut, double lambda_cut,
                  double *d_basis, int32_t *d_nbasis, double *d_s, void *stream);

/* Allocation-free chemical potential.  The paper has no counterpart: this is a library variant of
 * the Fermi-level solve inside dc_density (same kernel, same stopping rule), for callers that may
 * not allocate device memory where they need mu (a caller-owned pool or arena holding the device,
 * or work interleaved with other streams where cudaFree would synchronise the device).  It needs
 * no context and makes no cudaMalloc/cudaFree or other allocating call: its scratch is a fixed
 * 12,352-byte array in the library's static device memory (FP64 partials for at most 256 blocks,
 * plus barrier and error words that the call zeroes on the stream before each launch).
 * Inputs (device, FP64): d_eps[nstates] eigenvalues, d_q[nstates] core weights; n_elec >= 0
 * electrons; kT > 0 (Ha).  Solves sum_i 2 f((eps_i - mu)/kT) q_i = n_elec and writes d_mu[1]
 * and d_occ[nstates] = f_i (device).  *d_mu on entry serves as the starting guess when it lies in
 * the bracket; any value is accepted.  Synchronises the stream before returning.
 * Setup: the first call on each device looks up the scratch address (cudaGetSymbolAddress), the SM
 * count and the kernel's residency; a call with nstates = 0 does only that, so do it before any
 * stream capture begins.  The looked-up address belongs to the device's current primary context:
 * after cudaDeviceReset (or any teardown of that context) the first call that meets the stale
 * address fails with DC_ERR_CUDA and drops it, and the call after it looks the address up again, so
 * callers that reset a device should repeat the nstates = 0 setup call.  Calls on one device share the scratch: calls that overlap in time
 * (several host threads, or streams not ordered with each other) race and must be serialised by
 * the caller.  Errors: DC_ERR_ARG (nstates outside [0, 2^31 - 1], NULL pointer, bad kT or n_elec),
 * DC_ERR_TIMEOUT, DC_ERR_NONFINITE, DC_ERR_CUDA. */
int dc_fermi_level_noalloc(const double *d_eps, const double *d_q, int64_t nstates, double n_elec, double kT,
                           double *d_mu, double *d_occ, void *stream);

/* ---- SCF step ------------------------------------------------------------------------- */
/* One DC-DFT SCF iteration (Sec. 2.2): V_eff[rho_in], n_pass CheFSI passes, q, mu, rho_out,
 * energies, and linear mixing written back: rho_in <- rho_in + alpha (rho_out - rho_in).
 * rho_in_out[npts] FP64 is a device pointer if rho_on_host == 0, else a host pointer (then
 * copied in and out on the stream inside the call).  *h_stats is filled (host); the stream is
 * synchronised.  Requires dc_warmup first (DC_ERR_STATE otherwise) and nranks = 1 (a shard steps with
 * the dc_step_* calls below; DC_ERR_ARG otherwise). */
int dc_scf_step(dc_ctx *ctx, double *rho_in_out, int rho_on_host, dc_stats_t *h_stats, void *stream);

/* ---- fragment-sharded SCF step (Sec. 2.2; Sec. 2.5: fragments distributed over processes) ------ */
/* One SCF iteration of a context that owns fragments [frag_lo, frag_hi) of nranks, in three calls with
 * two exchanges that the caller makes between them (e.g. NCCL all-reduce sums; every array below is
 * zero outside the rank's own part, so a sum over ranks assembles the global array exactly):
 *   dc_step_local:   V_eff[rho_in] (every rank, identical), the rank's fragments' n_pass CheFSI passes and
 *                    core weights; writes d_eps[nstates] and d_q[nstates] (device, FP64), the rank's states
 *                    [state_lo, state_hi) filled and every other entry 0.
 *   -- caller: sum d_eps and d_q over ranks --
 *   dc_step_density: mu from all states (the same solve on every rank, from the previous mu), occupations,
 *                    and d_rho_part[npts] = rho_out on the rank's cores, 0 elsewhere; d_mu[1] may be NULL.
 *   -- caller: sum d_rho_part over ranks into rho_out --
 *   dc_step_finish:  energies, residual and mixing from rho_out (d_rho_out[npts], device) into
 *                    d_rho_in_out[npts] (device), as dc_scf_step; fills *h_stats (host, may be NULL).
 * With nranks = 1 the three calls equal dc_scf_step bit for bit.  Errors: DC_ERR_ARG (NULL pointers),
 * DC_ERR_STATE (no warm-up), DC_ERR_NOCONV, DC_ERR_TIMEOUT, DC_ERR_NONFINITE, DC_ERR_CUDA. */
int dc_step_local(dc_ctx *ctx, const double *d_rho_in, double *d_eps, double *d_q, void *stream);
int dc_step_density(dc_ctx *ctx, const double *d_eps, const double *d_q, double *d_rho_part, double *d_mu,
                    void *stream);
int dc_step_finish(dc_ctx *ctx, double *d_rho_in_out, const double *d_rho_out, dc_stats_t *h_stats, void *stream);

/* rho_out of the last dc_scf_step (device, FP64 [npts]). */
int dc_get_rho_out(dc_ctx *ctx, double *d_rho, void *stream);

/* ---- band-energy adjoint --------------------------------------------------------------- */
/* Needs nranks = 1 (DC_ERR_ARG otherwise).
 * E_b = sum_f sum_i occ_i <psi_i^f|H_f|psi_i^f> for a caller block d_psi (dtype), occupations
 * d_occ[nstates] (FP64, any values), potential d_V[npts] and per-atom strengths d_D[natom]
 * (FP64).  Writes h_Eb (host, may be NULL), d_dpsi = 2 occ_i dV H_f psi_i (dtype, may be NULL),
 * d_dV[npts] = dV sum over all fragments covering g of sum_i occ_i psi_i^2 (FP64, unweighted,
 * deterministic gather; may be NULL), d_dD[natom] = sum_f sum_i occ_i <p_a|psi_i>^2 (FP64, may
 * be NULL).  H psi is recomputed, never stored across calls.  Does not change the context's
 * potential. */
int dc_eb_adjoint(dc_ctx *ctx, const void *d_psi, int dtype, const double *d_occ, const double *d_V,
                  const double *d_D, double *h_Eb, void *d_dpsi, double *d_dV, double *d_dD, void *stream);

/* ---- autotuner ------------------------------------------------------------------------- */
/* dc_warmup times every useful launch shape of the stencil H-apply kernels on the context's own
 * fragments and keeps the fastest, separately for FP32 and FP64 elements.  A shape is (kind, threads
 * per CTA, point pairs per thread); kind 0 pairs x-adjacent points of one orbital (FP32: two
 * orbitals per CTA), kind 1 (FP32 only) interleaves two orbitals at every point, kind 2 is kind 1
 * compiled with registers capped for three 256-thread CTAs per SM, kind 3 is kind 1 with every
 * plane's projector records built once per CTA (only where they fit in shared memory), kind 4 (FP32
 * only) is the orbital-pair kernel compiled for one cubic fragment extent (18, 20, 22 or 32 points)
 * with the zero boundary and equal spacing on the three axes (256 threads up to 22 points, 512 for
 * 32); it takes Chebyshev steps and plain H-applies, and the adjoint runs the general kernel.  With the
 * environment variable DC_TUNE_CACHE=<file> results are looked up in / appended to that text file
 * (one line per fragment shape, atom and orbital count, type).
 * h_shape[6] = {fp32 kind, threads, pairs, fp64 kind, threads, pairs} (threads 0 = not tuned yet);
 * h_ms[40] (may be NULL) = best time in ms of each of the 20 candidate slots, FP32 then FP64
 * (0 = not tried). */
int dc_tuning(const dc_ctx *ctx, int *h_shape, float *h_ms);

/* Pin the stencil launch shape (kind, threads, pairs as in dc_tuning) for element type dtype
 * (DC_FP64 or DC_FP32); dc_warmup then keeps it instead of tuning.  Errors: DC_ERR_ARG when the
 * shape does not exist or cannot cover / fit this context's largest fragment. */
int dc_set_tuning(dc_ctx *ctx, int dtype, int kind, int threads, int pairs);

/* ---- stage profiler -------------------------------------------------------------------- */
/* Stages of the step, in the order they run. */
#define DC_STAGE_POTENTIAL 0 /* Poisson + exchange (cuFFT and pointwise kernels) */
#define DC_STAGE_GATHER 1    /* V_eff restricted to every fragment, spectral bounds */
#define DC_STAGE_PROJECT 2   /* projections <p_a|psi> of the first filter input */
#define DC_STAGE_HPSI 3      /* stencil H-apply kernels (Chebyshev steps and the last H Y) */
#define DC_STAGE_GRAM 4      /* Gram and Rayleigh-Ritz contractions */
#define DC_STAGE_SUBSPACE 5  /* FP64 Cholesky, eigensolve, filter coefficients */
#define DC_STAGE_ROTATE 6    /* Psi = Y C */
#define DC_STAGE_DENSITY 7   /* core weights, Fermi level, rho_out */
#define DC_STAGE_ENERGY 8    /* energies and mixing */
#define DC_NSTAGES 9

/* enable = 1 clears the counters and starts recording CUDA events around every stage launched
 * by later calls on their stream; enable = 0 stops recording.  dc_profile_read synchronises the
 * device and writes, per stage, the summed device time in ms, the number of this library's kernel
 * launches and the algorithmic bytes those launches must move (reads + writes of their operands,
 * each counted once; host arrays of DC_NSTAGES entries, any may be NULL). */
int dc_profile(dc_ctx *ctx, int enable);
int dc_profile_read(dc_ctx *ctx, double *h_ms, int64_t *h_launches, double *h_bytes);

/* ---- measurement helper ------------------------------------------------------------------ */
/* FP64 issue-rate probe (the paper has no counterpart): launches, on `stream`, one full wave of CTAs on
 * the current device in which every thread runs eight independent chains of `iters` FP64 FMAs, and
 * writes the number of FMAs launched to *h_fmas (host).  The caller times the launch (e.g. CUDA events
 * on the same stream) to get the device's measured FP64 FMA rate.  d_sink: one device double the kernel
 * may write (it does not for the inputs it uses).  Errors: DC_ERR_ARG (iters < 1, NULL pointer),
 * DC_ERR_CUDA. */
int dc_fp64_fma_probe(int64_t iters, double *d_sink, int64_t *h_fmas, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DCDFT_H */
