"""FP64 CPU oracle for the DC-DFT fragment Kohn-Sham solve (test infrastructure).

This package is the slow, plain reference that the CUDA path is checked
against.  It is test infrastructure: only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it.  The product library
never calls into it, and it shares no code with the CUDA path; the only common
module is ``workloads`` (seeded input generators without any of the method's
arithmetic).

Every function cites the passage of the paper it follows:

* Sec. 2.2, Eqs. 1-5: fragments (cores plus buffers), fragment Hamiltonian,
  core-projected density, global chemical potential.
* The model Hamiltonian terms (8th-order finite-difference Laplacian, Gaussian
  local potential, separable Gaussian projectors) and the CheFSI inner solver
  are readings of what the paper leaves open; each is stated where it is used.

Pins (tests marked ``not gpu``) tie it to things other than itself:
finite-difference polynomial exactness, closed-form plane-wave eigenvalues,
dense brute-force diagonalisation, analytic Gaussian potentials, Fermi limits,
electron-count conservation, the single-fragment = conventional identity and
finite differences of the band energy.  One part is "parity unpinned": the
absolute physical accuracy of the model against real Si or water (there are
no real pseudopotentials here).
"""
from . import maps, model, rng, chefsi, fermi, density, energy, scf, adjoint  # noqa: F401
