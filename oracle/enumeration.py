"""Brute-force exact outcome distributions of the discrete automaton on tiny grids.

TEST INFRASTRUCTURE (part of the oracle). Pure-Python enumeration of every joint
outcome of every step (Sec. 2.2 rules: an unburned cell ignites with probability
p_ignite of Eq. 9 when a neighbour burns; a burning cell keeps burning with probability
p_continue, else burns out; burned and non-burnable cells never change; all cells update
synchronously from the previous step's states). Exponential in the number of active
cells, so only for grids of a few cells and a few steps.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

OFFSETS = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]


def _ignite_prob(S, q, r, c):
    H, W = S.shape
    logprod = 0.0  # Eq. 9 as -expm1(sum log1p(-q)), free of cancellation
    for d, (dr, dc) in enumerate(OFFSETS):
        ri, ci = r + dr, c + dc
        if 0 <= ri < H and 0 <= ci < W and S[ri, ci] == 2:
            logprod += math.log1p(-float(q[d, r, c]))
    return -math.expm1(logprod)


def step_distribution(S, q, p_continue):
    """Exact distribution of S_next given S: list of (state bytes, probability)."""
    S = np.asarray(S, dtype=np.uint8)
    H, W = S.shape
    cells = []  # (index, prob of the "active" outcome, active value, passive value)
    for r in range(H):
        for c in range(W):
            s = S[r, c]
            if s == 1:
                p = _ignite_prob(S, q, r, c)
                if p > 0.0:
                    cells.append((r * W + c, p, 2, 1))
            elif s == 2:
                cells.append((r * W + c, p_continue, 2, 3))
    base = S.reshape(-1).copy()
    out = []
    for bits in itertools.product((0, 1), repeat=len(cells)):
        x = base.copy()
        pr = 1.0
        for (idx, p, av, pv), bit in zip(cells, bits):
            if bit:
                x[idx] = av
                pr *= p
            else:
                x[idx] = pv
                pr *= 1.0 - p
        if pr > 0.0:
            out.append((x.tobytes(), pr))
    return out


def distribution(S0, q, p_continue, T):
    """Exact distribution of S_T: dict state-bytes -> probability."""
    S0 = np.asarray(S0, dtype=np.uint8)
    shape = S0.shape
    dist = {S0.tobytes(): 1.0}
    for _ in range(T):
        nxt = {}
        for key, p in dist.items():
            S = np.frombuffer(key, dtype=np.uint8).reshape(shape)
            for k2, p2 in step_distribution(S, q, p_continue):
                nxt[k2] = nxt.get(k2, 0.0) + p * p2
        dist = nxt
    return dist


def marginals(dist, shape):
    """P(S_T[j] = s) as an array (4, H, W)."""
    m = np.zeros((4,) + tuple(shape))
    for key, p in dist.items():
        S = np.frombuffer(key, dtype=np.uint8).reshape(shape)
        for s in range(4):
            m[s] += p * (S == s)
    return m
