"""Helpers shared by the parity tests: run the CUDA library (through the C
ABI binding) and the FP64 oracle on the same seeded inputs and compare."""
from __future__ import annotations

import numpy as np

import oracle as O


def lib_to_oracle_perm():
    """perm[j] = oracle index of the library's direction j (matched by vector)."""
    from paper_2409_16781_gb300 import velocity_set
    cl, _ = velocity_set()
    co, _ = O.velocity_set()
    keys = {tuple(int(v) for v in co[i]): i for i in range(19)}
    return np.array([keys[tuple(int(v) for v in cl[j])] for j in range(19)])


def to_oracle_order(f_lib, perm):
    out = np.empty_like(f_lib)
    out[perm] = f_lib
    return out


def to_lib_order(f_ora, perm):
    return f_ora[perm]


def fluid_mask(flags, shape):
    if flags is None:
        return np.ones(shape, dtype=bool)
    return np.asarray(flags).reshape(shape) == 0


def pop_rel_err(f_lib, f_ora_in_lib_order, mask):
    """max over fluid cells and directions of |a - b| / |b|."""
    a = f_lib[:, mask]
    b = f_ora_in_lib_order[:, mask]
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b) / np.abs(b)))


def vel_err(u_lib, u_ora, mask):
    """max |u_lib - u_ora| / max |u_ora| over fluid cells."""
    if not mask.any():
        return 0.0
    du = np.abs(u_lib[:, mask] - u_ora[:, mask]).max()
    scale = np.abs(u_ora[:, mask]).max()
    return float(du / scale) if scale > 0 else float(du)
