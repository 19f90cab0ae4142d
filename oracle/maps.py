"""Fragment maps (test infrastructure; FP64 oracle).

Sec. 2.2: the periodic rectangular cell is divided by a regular grid of
``num_fragment(1:3)`` into non-overlapping core domains; each fragment is its
core plus a buffer of ``num_rgrid_buffer(1:3)`` grid points on every side
(Table 1).  Reading for a grid size not divisible by the fragment count: the
core of fragment k on an axis of N points split F ways is
[floor(kN/F), floor((k+1)N/F)).

Layouts: global arrays are [Nz][Ny][Nx] (x fastest, g = x + Nx(y + Ny z));
fragment arrays are [Ez][Ey][Ex]; fragment id f = kx + Fx(ky + Fy kz).
"""
from __future__ import annotations

import numpy as np


def core_starts(N: int, F: int):
    """Core boundaries s_0..s_F on one axis (Sec. 2.2, regular division)."""
    return [(k * N) // F for k in range(F + 1)]


class Fragments:
    """All fragments of a cell: origins, extents, cores and the index maps."""

    def __init__(self, n, num_fragment, buffer):
        self.n = tuple(int(v) for v in n)
        self.F = tuple(int(v) for v in num_fragment)
        self.b = tuple(int(v) for v in buffer)
        for d in range(3):
            if self.F[d] < 1 or self.F[d] > self.n[d]:
                raise ValueError("num_fragment must be in [1, N] on every axis")
            if self.b[d] < 0:
                raise ValueError("num_rgrid_buffer must be >= 0")
        self.starts = [core_starts(self.n[d], self.F[d]) for d in range(3)]
        self.nfrag = self.F[0] * self.F[1] * self.F[2]
        self.origin = np.zeros((self.nfrag, 3), dtype=np.int64)  # s_k - b (may be negative)
        self.extent = np.zeros((self.nfrag, 3), dtype=np.int64)  # E = core + 2b
        self.core = np.zeros((self.nfrag, 3), dtype=np.int64)  # core length c
        for kz in range(self.F[2]):
            for ky in range(self.F[1]):
                for kx in range(self.F[0]):
                    f = kx + self.F[0] * (ky + self.F[1] * kz)
                    for d, k in enumerate((kx, ky, kz)):
                        s0, s1 = self.starts[d][k], self.starts[d][k + 1]
                        self.origin[f, d] = s0 - self.b[d]
                        self.core[f, d] = s1 - s0
                        self.extent[f, d] = (s1 - s0) + 2 * self.b[d]
        self.npts = np.prod(self.extent, axis=1)

    def local_global_axis(self, f: int, d: int):
        """Global index on axis d of every local index j_d of fragment f (wrapped)."""
        return np.mod(self.origin[f, d] + np.arange(self.extent[f, d]), self.n[d])

    def idx_map(self, f: int):
        """idx_map[f][j] = global flat index of local flat point j (x fastest)."""
        gx = self.local_global_axis(f, 0)
        gy = self.local_global_axis(f, 1)
        gz = self.local_global_axis(f, 2)
        nx, ny = self.n[0], self.n[1]
        g = gx[None, None, :] + nx * (gy[None, :, None] + ny * gz[:, None, None])
        return g.reshape(-1).astype(np.int64)

    def core_mask(self, f: int):
        """Boolean [Ez][Ey][Ex]: True on the core Omega_0 of fragment f (Eq. 3)."""
        m = []
        for d in range(3):
            j = np.arange(self.extent[f, d])
            m.append((j >= self.b[d]) & (j < self.b[d] + self.core[f, d]))
        return m[2][:, None, None] & m[1][None, :, None] & m[0][None, None, :]

    def owner(self):
        """owner[g] = fragment whose core holds g; core_local[g] = its local index."""
        N = self.n[0] * self.n[1] * self.n[2]
        owner = np.full(N, -1, dtype=np.int64)
        core_local = np.full(N, -1, dtype=np.int64)
        for f in range(self.nfrag):
            cm = self.core_mask(f).reshape(-1)
            g = self.idx_map(f)[cm]
            if np.any(owner[g] >= 0):
                raise AssertionError("cores overlap")
            owner[g] = f
            core_local[g] = np.nonzero(cm)[0]
        return owner, core_local

    def weight_sum(self):
        """Sum over fragments of the core indicator w_f(g) at every global point."""
        N = self.n[0] * self.n[1] * self.n[2]
        w = np.zeros(N, dtype=np.int64)
        for f in range(self.nfrag):
            cm = self.core_mask(f).reshape(-1)
            np.add.at(w, self.idx_map(f)[cm], 1)
        return w


def fragment_electrons(frags: Fragments, L, pos, species, Z):
    """Electrons of the atoms with an image inside each fragment box (half-open, unwrapped).

    Reading for an orbital count "set by the electron count": the box of
    fragment f on axis d is [origin*h, (origin+E)*h).
    """
    h = [L[d] / frags.n[d] for d in range(3)]
    ne = np.zeros(frags.nfrag)
    for f in range(frags.nfrag):
        inside = np.ones(len(pos), dtype=bool)
        for d in range(3):
            lo = frags.origin[f, d] * h[d]
            hi = (frags.origin[f, d] + frags.extent[f, d]) * h[d]
            hit = np.zeros(len(pos), dtype=bool)
            kmax = int(np.ceil((frags.extent[f, d] * h[d]) / L[d])) + 2
            for k in range(-kmax, kmax + 1):
                x = pos[:, d] + k * L[d]
                hit |= (x >= lo) & (x < hi)
            inside &= hit
        ne[f] = np.sum(Z[species[inside]])
    return ne


def orbital_counts(frags: Fragments, nstate_frag: int, L, pos, species, Z):
    """Orbitals per fragment: fixed ``nstate_frag`` or, when it is 0, from the electron count.

    Auto rule: n_f = ceil(Ne_f/2) + max(4, ceil(0.2*ceil(Ne_f/2))).
    """
    if nstate_frag > 0:
        return np.full(frags.nfrag, nstate_frag, dtype=np.int64)
    ne = fragment_electrons(frags, L, pos, species, Z)
    occ = np.ceil(ne / 2.0).astype(np.int64)
    extra = np.maximum(4, np.ceil(0.2 * occ).astype(np.int64))
    return occ + extra
