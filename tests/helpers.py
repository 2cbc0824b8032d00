"""Shared helpers for the GPU parity tests (no method arithmetic here)."""
import numpy as np

from oracle import oracle as O


def to_dev(host):
    import torch

    return torch.from_numpy(np.ascontiguousarray(host)).cuda()


def elem_cols(S, r, count, seed):
    """A sorted sample of element columns that always includes the first and
    last column (the ragged tail of the last column tile)."""
    E = S // (r // 8)
    if E <= count:
        return np.arange(E)
    g = np.random.default_rng(seed)
    pick = set(g.choice(E, count - 2, replace=False).tolist()) | {0, E - 1}
    return np.array(sorted(pick))


def elems(host_u8, r, cols=None):
    e = O.to_elems(host_u8, r)
    return e if cols is None else np.ascontiguousarray(e[:, cols])
