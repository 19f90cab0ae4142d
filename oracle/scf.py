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

    # -- potentials -------------------------------------------------------------------------------
    def veff(self, rho_in):
        """V_eff = V_loc + V_H[rho] + v_x[rho] (hxc="hartree_x") or V_loc (hxc="none")."""
        if self.hxc == "none":
            return self.vion.copy()
        return self.vion + model.hartree(self.grid, rho_in) + model.vx(rho_in)

    def hamiltonian(self, f, V):
        return model.FragmentHamiltonian(self.frags, f, self.grid, V, self.proj[f], self.bc)

    # -- fragment solves --------------------------------------------------------------------------
    def initial_rr(self, V):
        for f in self.active:
            eps, psi, _ = chefsi.rayleigh_ritz(self.hamiltonian(f, V), self.psi[f])
            self.eps[f], self.psi[f] = eps, psi

    def solve(self, V, n_pass):
        for f in self.active:
            H = self.hamiltonian(f, V)
            for _ in range(n_pass):
                eps, psi, _ = chefsi.chefsi_pass(H, self.psi[f], self.m, self.eps[f])
                self.eps[f], self.psi[f] = eps, psi

    def warmup(self):
        V = self.veff(self.rho_in)
        self.initial_rr(V)
        self.solve(V, int(self.cfg["n_warmup"]))

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
        V = self.veff(self.rho_in)
        self.solve(V, int(self.cfg["n_pass"]))
        q, mu, occ, rho_out = self.density_stage()
        eps_all = np.concatenate([self.eps[f] for f in self.active])
        q_all = np.concatenate([q[f] for f in self.active])
        occ_all = np.concatenate([occ[f] for f in self.active])
        eband = energy.band_sum(eps_all, q_all, occ_all)
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
