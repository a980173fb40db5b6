"""Shared helpers for the tests: landscapes as torch tensors, a library fixture."""
import numpy as np

import synthetic as syn

PRM = dict(p_h=0.58, c1=0.045, c2=0.131, a=0.078, p_continue=0.3, l=30.0)


def cuda(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def set_landscape(model, land, V, th):
    import torch
    model.set_env(cuda(land.E), cuda(land.p_veg), cuda(land.p_den), cuda(V), cuda(th))


def lattice_state(H, W, rho, gam, burning=2, other=1):
    """Burning cells on the lattice (r, c) = (rho, gam) mod 3: every other cell has
    exactly one burning neighbour (or is on the lattice itself)."""
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    on = ((rr - rho) % 3 == 0) & ((cc - gam) % 3 == 0)
    return np.where(on, burning, other).astype(np.uint8), on


def lattice_direction(H, W, rho, gam):
    """Direction index d of the single burning lattice neighbour of every cell (-1 on the lattice)."""
    offs = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    dr = (rho - rr) % 3
    dc = (gam - cc) % 3
    dr = np.where(dr == 2, -1, dr)
    dc = np.where(dc == 2, -1, dc)
    d = np.full((H, W), -1, int)
    for k, (a, b) in enumerate(offs):
        d[(dr == a) & (dc == b)] = k
    return d
