"""DC-DFT SCF driver (test infrastructure; FP64 oracle).

Sec. 2.2: every SCF iteration solves the independent fragment problems (Eq. 1)
in the current potential, finds the global mu, projects the fragment
densities onto their cores (Eqs. 2-4), rebuilds the Hartree and
exchange-correlation potentials from rho_tot (Eq. 5) and mixes.  Readings:

* start: random orbitals (``oracle.rng``) and a superposition of the Gaussian
  ion charges; a Rayleigh-Ritz of the random block gives the first filter
  bounds; ``n_warmup`` CheFSI passes in the starting potential precede step 1;
* each SCF step runs ``n_pass`` CheFSI passes per fragment, then the core
  weights, mu, rho_out, the energy and linear mixing.

Per-fragment exchange-correlation and the density-template potential (Eq. 5:
V_xc[rho_alpha] and V^alpha = (rho_alpha - rho_tot)/xi), switched on with
``xc_fragment`` (and ``xi`` > 0).  The paper leaves open which fragment
density enters a step; readings:

* rho_alpha is the whole-fragment density sum_i 2 f_i |phi_i^alpha|^2 (Eq. 3
  before the core projection) of the orbitals and occupations that the
  previous step ended with (after the warm-up: of the warm state and its own
  Fermi level); it is not mixed;
* the fragment potential on fragment point j (global point g) is
  V_loc(g) + V_H[rho_in](g) + v_x(rho_alpha(j)) + (rho_alpha(j) - rho_in(g))/xi,
  the last term only for xi > 0 (the paper's default is V^alpha = 0);
* the energy removes the double counting with the potential each core point
  felt, that of the fragment owning it:
  E = sum 2 f eps q - int V_core rho_out + E_es[rho_out] + E_x[rho_out].
  For one fragment spanning the cell this is the Kohn-Sham energy of the
  output orbitals, as with the global potential.
"""
from __future__ import annotations

import numpy as np

from . import chefsi, density, energy, fermi, maps, model, rng


class DCState:
    def __init__(self, cfg, fragments_subset=None):
        self.cfg = cfg
        self.grid = model.Grid(cfg["n"], cfg["L"])
        self.frags = maps.Fragments(cfg["n"], cfg["num_fragment"], cfg["num_rgrid_buffer"])
        self.pos = np.asarray(cfg["pos"], dtype=np.float64)
        self.species = np.asarray(cfg["species"], dtype=np.int64)
        self.spec = cfg["spec"]
        self.bc = cfg["bc"]
        self.hxc = cfg["hxc"]
        self.kT = float(cfg["kT"])
        self.alpha = float(cfg["mix_alpha"])
        self.m = int(cfg["cheb_degree"])
        self.ne = float(np.sum(self.spec["Z"][self.species]))
        self.owner, self.core_local = self.frags.owner()
        self.norb = maps.orbital_counts(self.frags, int(cfg["nstate_frag"]), self.grid.L, self.pos,
                                        self.species, self.spec["Z"])
        self.active = list(range(self.frags.nfrag)) if fragments_subset is None else list(fragments_subset)
        self.proj = {f: model.FragmentProjectors(self.frags, f, self.grid, self.pos, self.species, self.spec)
                     for f in self.active}
        self.vion = model.v_ion(self.grid, self.pos, self.species, self.spec)
        self.rhoiG = model.rho_ion_G(self.grid, self.pos, self.species, self.spec)
        self.rho_in = model.initial_density(self.grid, self.pos, self.species, self.spec)
        self.psi = {}
        for f in self.active:
            shp = (int(self.norb[f]),) + tuple(int(v) for v in self.frags.extent[f][::-1])
            self.psi[f] = rng.orbital_block(int(cfg["seed"]), f, shp[0], int(np.prod(shp[1:]))).reshape(shp)
        self.eps = {}
        self.step_index = 0
        self.xc_fragment = bool(cfg.get("xc_fragment", False))
        self.xi = float(cfg.get("xi", 0.0))
        if self.xc_fragment and self.hxc != "hartree_x":
            raise ValueError("per-fragment exchange needs hxc = hartree_x")
        self.rho_frag = {}

    # -- potentials -------------------------------------------------------------------------------
    def veff(self, rho_in):
        """V_eff = V_loc + V_H[rho] + v_x[rho] (hxc="hartree_x") or V_loc (hxc="none")."""
        if self.hxc == "none":
            return self.vion.copy()
        return self.vion + model.hartree(self.grid, rho_in) + model.vx(rho_in)

    def hamiltonian(self, f, V, Vf=None):
        return model.FragmentHamiltonian(self.frags, f, self.grid, V, self.proj[f], self.bc, V_frag=Vf)

    # -- per-fragment potential (xc_fragment) -------------------------------------------------------
    def fragment_density(self, f, occ_f):
        """rho_alpha on every point of fragment f: sum_i 2 f_i psi_i^2 (Eq. 3 without the core projection)."""
        return np.einsum("i,i...->...", 2.0 * occ_f, self.psi[f] ** 2)

    def fragment_potentials(self, rho_in):
        """V_alpha on every fragment point: V_loc + V_H[rho_in] restricted to the fragment, plus v_x of the
        fragment density and, for xi > 0, the density-template term (rho_alpha - rho_in)/xi (Eq. 5)."""
        Vg = (self.vion + model.hartree(self.grid, rho_in)).reshape(-1)
        rin = rho_in.reshape(-1)
        out = {}
        for f in self.active:
            idx = self.frags.idx_map(f)
            shp = self.psi[f].shape[1:]
            rf = self.rho_frag[f]
            Vf = Vg[idx].reshape(shp) + model.vx(rf)
            if self.xi > 0.0:
                Vf = Vf + (rf - rin[idx].reshape(shp)) / self.xi
            out[f] = Vf
        return out

    def update_fragment_densities(self, occ):
        for f in self.active:
            self.rho_frag[f] = self.fragment_density(f, occ[f])

    # -- fragment solves --------------------------------------------------------------------------
    def initial_rr(self, V):
        for f in self.active:
            eps, psi, _ = chefsi.rayleigh_ritz(self.hamiltonian(f, V), self.psi[f])
            self.eps[f], self.psi[f] = eps, psi

    def solve(self, V, n_pass, Vfrag=None):
        for f in self.active:
            H = self.hamiltonian(f, V, None if Vfrag is None else Vfrag[f])
            for _ in range(n_pass):
                eps, psi, _ = chefsi.chefsi_pass(H, self.psi[f], self.m, self.eps[f])
                self.eps[f], self.psi[f] = eps, psi

    def warmup(self):
        V = self.veff(self.rho_in)
        self.initial_rr(V)
        self.solve(V, int(self.cfg["n_warmup"]))
        if self.xc_fragment:
            _, _, occ, _ = self.density_stage()
            self.update_fragment_densities(occ)

    # -- density stage ----------------------------------------------------------------------------
    def density_stage(self):
        q = {f: density.core_weights(self.frags, f, self.psi[f], self.grid.dV) for f in self.active}
        eps_all = np.concatenate([self.eps[f] for f in self.active])
        q_all = np.concatenate([q[f] for f in self.active])
        mu = fermi.find_mu(eps_all, q_all, self.ne, self.kT)
        rho = np.zeros(self.grid.npts)
        occ = {}
        for f in self.active:
            occ[f] = fermi.occupation(self.eps[f], mu, self.kT)
            g, vals = density.core_density(self.frags, f, self.psi[f], occ[f])
            rho[g] = vals
        return q, mu, occ, rho.reshape(self.grid.shape())

    # -- one SCF step -----------------------------------------------------------------------------
    def scf_step(self):
        Vfrag = None
        if self.xc_fragment:
            Vfrag = self.fragment_potentials(self.rho_in)
            V = None
        else:
            V = self.veff(self.rho_in)
        self.solve(V, int(self.cfg["n_pass"]), Vfrag)
        q, mu, occ, rho_out = self.density_stage()
        eps_all = np.concatenate([self.eps[f] for f in self.active])
        q_all = np.concatenate([q[f] for f in self.active])
        occ_all = np.concatenate([occ[f] for f in self.active])
        eband = energy.band_sum(eps_all, q_all, occ_all)
        if self.xc_fragment:
            # the input potential each core point felt: that of its owner fragment
            Vcore = np.zeros(self.grid.npts)
            for f in self.active:
                cm = self.frags.core_mask(f)
                Vcore[self.frags.idx_map(f)[cm.reshape(-1)]] = Vfrag[f][cm]
            V = Vcore.reshape(self.grid.shape())
            self.update_fragment_densities(occ)
        E = energy.total_energy(self.grid, self.hxc, eband, V, rho_out, self.rhoiG)
        S = fermi.entropy(eps_all, q_all, mu, self.kT)
        drho = energy.residual(self.grid, rho_out, self.rho_in, self.ne)
        stats = dict(E=E, F=E - self.kT * S, eband=eband, mu=mu, drho=drho, natom=len(self.pos),
                     rho_out=rho_out, rho_in=self.rho_in.copy(), q=q, occ=occ,
                     eps={f: self.eps[f].copy() for f in self.active})
        self.rho_in = energy.mix(self.rho_in, rho_out, self.alpha, self.grid, float(self.cfg.get("kerker_q0", 0.0)))
        self.step_index += 1
        return stats


def run(cfg, steps=None):
    """Warm-up plus ``steps`` SCF steps; returns the per-step statistics."""
    st = DCState(cfg)
    st.warmup()
    out = []
    for _ in range(cfg["scf_steps"] if steps is None else steps):
        out.append(st.scf_step())
    return st, out
