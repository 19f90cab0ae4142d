"""Seeded synthetic workloads for the DC-DFT fragment solve.

This module only generates inputs: atomic positions, species tables and the
run parameters of each workload.  It holds none of the method's arithmetic
(no Hamiltonian, no density, no eigensolver), so both the FP64 CPU oracle and
the CUDA path may read from it.

The paper measures on a Si diamond crystal, amorphous Si (a published
structure) and liquid water (a GROMACS snapshot) (Sec. 3).  Those structures
are not available here; the workloads below are synthetic stand-ins with the
same cell sizes, atom counts, densities and grid spacings:

* ``si8``    -- Si8 diamond cell a=10.26 bohr, 20^3 grid, 2^3 fragments (10^3 core + 4), 24 orbitals.
* ``si64``   -- 2^3 supercell, 40^3 grid, 4^3 fragments (10^3 core + 5), 32 orbitals.
* ``si512``  -- 4^3 supercell, 80^3 grid, 8^3 fragments (10^3 core + 6), 48 orbitals.
* ``water``  -- 1378 rigid H2O, 65.6 bohr box, 192^3 grid, 12^3 fragments (16^3 core + 8),
  orbital count per fragment from its electron count.
* ``si_weak{64,512,4096}`` -- 2^3/4^3/8^3 supercells, 20 points per cell edge, 10^3 core + 6.

Positions come from numpy's PCG64 with the seed stated per workload.
"""
from __future__ import annotations

import copy
import math

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903

# Species: valence charge Z, local Gaussian width sigma_loc, projector width
# sigma_proj (bohr) and projector strength D (Ha).
SPECIES = {
    "Si": dict(Z=4.0, sigma_loc=0.8, sigma_proj=0.6, D=0.5),
    "O": dict(Z=6.0, sigma_loc=0.55, sigma_proj=0.45, D=0.5),
    "H": dict(Z=1.0, sigma_loc=0.40, sigma_proj=0.35, D=0.2),
}

DIAMOND_BASIS = np.array(
    [
        [0.0, 0.0, 0.0],
        [0.5, 0.5, 0.0],
        [0.5, 0.0, 0.5],
        [0.0, 0.5, 0.5],
        [0.25, 0.25, 0.25],
        [0.75, 0.75, 0.25],
        [0.75, 0.25, 0.75],
        [0.25, 0.75, 0.75],
    ]
)


def _species_table(names):
    return dict(
        names=list(names),
        Z=np.array([SPECIES[s]["Z"] for s in names], dtype=np.float64),
        sigma_loc=np.array([SPECIES[s]["sigma_loc"] for s in names], dtype=np.float64),
        sigma_proj=np.array([SPECIES[s]["sigma_proj"] for s in names], dtype=np.float64),
        D=np.array([SPECIES[s]["D"] for s in names], dtype=np.float64),
    )


def si_diamond(cells: int, a: float, disp: float, seed: int):
    """Si diamond supercell of ``cells^3`` conventional cells, displaced by N(0, disp)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = np.array([(i, j, k) for k in range(cells) for j in range(cells) for i in range(cells)], dtype=np.float64)
    frac = (idx[:, None, :] + DIAMOND_BASIS[None, :, :]).reshape(-1, 3)
    pos = frac * a
    pos = pos + rng.normal(0.0, disp, size=pos.shape)
    L = cells * a
    pos = np.mod(pos, L)
    return pos, np.zeros(len(pos), dtype=np.int32), _species_table(["Si"])


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
        ]
    )


def water_box(nmol: int, L: float, min_oo: float, seed: int):
    """Rigid H2O molecules placed by random sequential addition in a cubic box.

    O-O distances (minimum image) are at least ``min_oo``; the H positions use
    an O-H bond of 0.9572 A and an H-O-H angle of 104.52 deg, uniformly
    randomly oriented.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    oxy = np.empty((nmol, 3))
    count = 0
    tries = 0
    while count < nmol:
        tries += 1
        if tries > 200 * nmol:
            raise RuntimeError("random sequential addition did not place all molecules")
        cand = rng.uniform(0.0, L, size=3)
        if count:
            d = oxy[:count] - cand
            d -= L * np.round(d / L)
            if np.min(np.einsum("ij,ij->i", d, d)) < min_oo * min_oo:
                continue
        oxy[count] = cand
        count += 1
    r_oh = 0.9572 * BOHR_PER_ANGSTROM
    half = math.radians(104.52) / 2.0
    local_h = np.array(
        [[r_oh * math.sin(half), 0.0, r_oh * math.cos(half)], [-r_oh * math.sin(half), 0.0, r_oh * math.cos(half)]]
    )
    pos = []
    spc = []
    for m in range(nmol):
        R = _random_rotation(rng)
        pos.append(oxy[m])
        spc.append(0)
        for hvec in local_h:
            pos.append(np.mod(oxy[m] + R @ hvec, L))
            spc.append(1)
    return np.array(pos), np.array(spc, dtype=np.int32), _species_table(["O", "H"])


DEFAULT_PARAMS = dict(
    precision="fp64",  # fp64 | fp32 | mixed
    cheb_degree=10,
    n_pass=1,
    n_warmup=10,
    hxc="hartree_x",  # hartree_x | none
    kT=0.01,
    mix_alpha=0.3,
    kerker_q0=0.0,  # 0: plain linear mixing; > 0: Kerker-preconditioned (bohr^-1)
    seed=20260603,
    bc="zero",  # zero | periodic
)


def make_config(name: str, **overrides):
    """Return the workload ``name`` as a plain dict (all arrays numpy)."""
    if name == "si8":
        pos, spc, sp = si_diamond(1, 10.26, 0.05, 1001)
        cfg = dict(n=(20, 20, 20), cells=1, num_fragment=(2, 2, 2), num_rgrid_buffer=(4, 4, 4), nstate_frag=24, scf_steps=10)
    elif name == "si64":
        pos, spc, sp = si_diamond(2, 10.26, 0.1, 1002)
        cfg = dict(n=(40, 40, 40), cells=2, num_fragment=(4, 4, 4), num_rgrid_buffer=(5, 5, 5), nstate_frag=32, scf_steps=10)
    elif name == "si512":
        pos, spc, sp = si_diamond(4, 10.26, 0.3, 1003)
        cfg = dict(n=(80, 80, 80), cells=4, num_fragment=(8, 8, 8), num_rgrid_buffer=(6, 6, 6), nstate_frag=48, scf_steps=20)
    elif name == "water":
        L = 65.6
        pos, spc, sp = water_box(1378, L, 2.5 * BOHR_PER_ANGSTROM, 1004)
        cfg = dict(
            n=(192, 192, 192), L=(L, L, L), num_fragment=(12, 12, 12), num_rgrid_buffer=(8, 8, 8), nstate_frag=0, scf_steps=10
        )
    elif name.startswith("si_weak"):
        natom = int(name[len("si_weak"):])
        cells = {64: 2, 512: 4, 4096: 8}[natom]
        pos, spc, sp = si_diamond(cells, 10.26, 0.3, 1005 + cells)
        n = 20 * cells
        cfg = dict(n=(n, n, n), cells=cells, num_fragment=(2 * cells,) * 3, num_rgrid_buffer=(6, 6, 6), nstate_frag=48, scf_steps=20)
    else:
        raise KeyError(name)
    if "L" not in cfg:
        a = 10.26 * cfg["cells"]
        cfg["L"] = (a, a, a)
    cfg.pop("cells", None)
    cfg.update(copy.deepcopy(DEFAULT_PARAMS))
    # Si8 is specified with plain linear mixing; the larger cells slosh charge under it (the oracle
    # diverges on Si64 after three steps), so they use Kerker-preconditioned linear mixing.
    cfg["kerker_q0"] = 0.0 if name == "si8" else 1.0
    cfg.update(pos=pos, species=spc, spec=sp, name=name)
    cfg.update(overrides)
    return cfg


def small_config(n=(12, 12, 12), L=(7.0, 7.0, 7.0), num_fragment=(2, 2, 2), buffer=(2, 2, 2), nstate=6,
                 natom=3, seed=7, bc="zero", species=("Si",), **overrides):
    """A tiny random cell for unit tests: ``natom`` atoms placed uniformly at random."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = rng.uniform(0.0, 1.0, size=(natom, 3)) * np.asarray(L)
    spc = rng.integers(0, len(species), size=natom).astype(np.int32)
    cfg = dict(n=tuple(n), L=tuple(L), num_fragment=tuple(num_fragment), num_rgrid_buffer=tuple(buffer),
               nstate_frag=nstate, scf_steps=3)
    cfg.update(copy.deepcopy(DEFAULT_PARAMS))
    cfg.update(pos=pos, species=spc, spec=_species_table(list(species)), name="small", bc=bc)
    cfg.update(overrides)
    return cfg


CONFIG_NAMES = ["si8", "si64", "si512", "water", "si_weak64", "si_weak512", "si_weak4096"]
