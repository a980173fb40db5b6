"""Independent FP64 restatement of the differentiable form in plain PyTorch CPU ops.

TEST INFRASTRUCTURE (part of the oracle): it re-derives Eq. 1-5 and the mean-field
step (Eq. 9 with burning probabilities) with whole-array shifts instead of the C
oracle's per-cell loops, and differentiates them with autograd. It pins the C oracle's
hand-written adjoint and serves as the "FP64 autograd reference" for gradients.
"""
from __future__ import annotations

import math

import numpy as np
import torch

C_FP = 1.1486328125  # Eq. 8
# (dr, dc) from the receiving cell to the burning neighbour, fixed order
OFFSETS = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]


def _shift(x: torch.Tensor, dr: int, dc: int, fill: float = 0.0) -> torch.Tensor:
    """y[r, c] = x[r + dr, c + dc], with `fill` outside the grid."""
    H, W = x.shape
    xp = torch.nn.functional.pad(x[None, None], (1, 1, 1, 1), value=fill)[0, 0]
    return xp[1 + dr:1 + dr + H, 1 + dc:1 + dc + W]


def _inside(H: int, W: int, dr: int, dc: int) -> torch.Tensor:
    return _shift(torch.ones(H, W, dtype=torch.float64), dr, dc, 0.0)


def q_planes(E, p_veg, p_den, V, theta, p_h, c1, c2, a, l, burnable=None):
    """Stack of 8 (H, W) planes of f_p(p_propagate); all tensors FP64."""
    H, W = p_veg.shape
    out = []
    G = p_h * (1.0 + p_veg) * (1.0 + p_den)
    for (dr, dc) in OFFSETS:
        k = math.sqrt(2.0) if (dr != 0 and dc != 0) else 1.0
        E_i = _shift(E, dr, dc, 0.0)
        inside = _inside(H, W, dr, dc)
        dE = (E - E_i) * inside
        theta_s = torch.rad2deg(torch.atan(dE / (k * l)))
        phi = math.degrees(math.atan2(dr, -dc))
        cosm1 = torch.cos(torch.deg2rad(theta - phi)) - 1.0
        pw = torch.exp(c1 * V) * torch.exp(c2 * V * cosm1)
        ps = torch.exp(a * theta_s)
        q = torch.tanh(C_FP * G * pw * ps) * inside
        if burnable is not None:
            q = q * burnable
        out.append(q)
    return out


def step(a, b, qs, p_continue):
    # Eq. 9 as -expm1(sum log1p(-x)): 1 - prod(1 - x) without floating-point cancellation
    logprod = torch.zeros_like(a)
    for (dr, dc), q in zip(OFFSETS, qs):
        logprod = logprod + torch.log1p(-_shift(b, dr, dc, 0.0) * q)
    P = -torch.expm1(logprod)
    n = (1.0 - a) * P
    return a + n, n + p_continue * b


def t64(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64))


def run(land, winds, starts, params, S0, T, y=None, requires_grad=True):
    """Forward T steps with autograd on (p_h, c1, c2, a, p_veg, p_den).

    params: dict with p_h, c1, c2, a, p_continue, l (python floats).
    Returns (a_T, b_T, leaves) and, if y is given, the BCE loss as well."""
    S0 = np.asarray(S0)
    p_h = torch.tensor(params["p_h"], dtype=torch.float64, requires_grad=requires_grad)
    c1 = torch.tensor(params["c1"], dtype=torch.float64, requires_grad=requires_grad)
    c2 = torch.tensor(params["c2"], dtype=torch.float64, requires_grad=requires_grad)
    aa = torch.tensor(params["a"], dtype=torch.float64, requires_grad=requires_grad)
    pv = t64(land.p_veg).requires_grad_(requires_grad)
    pd = t64(land.p_den).requires_grad_(requires_grad)
    E = t64(land.E)
    burn = t64(S0 != 0)
    a = t64((S0 == 2) | (S0 == 3))
    b = t64(S0 == 2)
    cur, qs = None, None
    for t in range(T):
        e = max(k for k, s in enumerate(starts) if t >= s)
        if e != cur:
            V, th = winds[e]
            qs = q_planes(E, pv, pd, t64(V), t64(th), p_h, c1, c2, aa, params["l"], burn)
            cur = e
        a, b = step(a, b, qs, params["p_continue"])
    leaves = dict(p_h=p_h, c1=c1, c2=c2, a=aa, p_veg=pv, p_den=pd)
    if y is None:
        return a, b, leaves
    yh = torch.clamp(a, 1e-7, 1.0 - 1e-7)
    yt = t64(y)
    loss = -torch.mean(yt * torch.log(yh) + (1.0 - yt) * torch.log(1.0 - yh))
    return a, b, leaves, loss
