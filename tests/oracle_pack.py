"""Helpers that lay oracle per-fragment arrays out in the library's packed layout (tests only)."""
import numpy as np

from oracle import scf


def pack(state, per_frag):
    """Concatenate per-fragment arrays [n_f][Ez][Ey][Ex] (or [n_f]) in fragment order."""
    return np.concatenate([np.asarray(per_frag[f]).reshape(-1) for f in range(state.frags.nfrag)])


def unpack(state, flat):
    out = {}
    off = 0
    for f in range(state.frags.nfrag):
        shp = (int(state.norb[f]),) + tuple(int(v) for v in state.frags.extent[f][::-1])
        n = int(np.prod(shp))
        out[f] = np.asarray(flat[off:off + n], dtype=np.float64).reshape(shp)
        off += n
    return out


def unpack_states(state, flat):
    out = {}
    off = 0
    for f in range(state.frags.nfrag):
        n = int(state.norb[f])
        out[f] = np.asarray(flat[off:off + n], dtype=np.float64)
        off += n
    return out


def oracle_state(cfg, subset=None):
    return scf.DCState(cfg, fragments_subset=subset)
