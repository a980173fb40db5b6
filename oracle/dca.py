"""Oracle of the paper's own differentiable-CA calibration path (Sec. 2.3): the
accumulator of p_ignite over newly ignited cells along the discrete stochastic
trajectory, its gradient with the trajectory held fixed, the step-ring selection of the
steps that carry gradient, and the loss of Eq. 10.

TEST INFRASTRUCTURE, NOT PRODUCT (as the rest of ``oracle``): plain FP64 numpy, one
whole-array operation per term of the formulas, built on the C oracle's prep, discrete
step and prep chain rule.

* ``dca_forward``: the data-flow description of Sec. 2.2 (Fig. 4): every step compares
  p_ignite (Eq. 9) with a uniform draw; the p_ignite values of the cells that ignite in
  that step are added to the accumulator. A cell ignites at most once, so its
  accumulator entry is the p_ignite of the step it ignited in (0 if it never did,
  including the initially burning cells).
* ``dca_backward``: Sec. 2.3, back-propagation. Only ignited cells have
  p_propagate contributing to p_ignite, so the gradient of a loss of the accumulator
  flows through p_ignite of the newly ignited cells, with the burning sets and the
  ignition events of the sampled trajectory held fixed. For cell j ignited at step t,
  dp_ignite_j / dq_dj = beta_i prod_{e != d} (1 - beta_e q_ej) with beta the burning
  indicators at t (Eq. 9 differentiated); q's chain rule (Eq. 1-5) is the C oracle's.
* ``step_rings``: the steps attached to the computation graph ("update by step rings"):
  the first r_first steps, the last r_last steps and r_between steps evenly between.
* ``eq10_loss``: Eq. 10, binary cross-entropy with logits on the accumulator over the
  crop to the union of non-zero predictions and targets, plus the mean squared
  difference of the 4 x 4, stride-4 average-pooled maps.
"""
from __future__ import annotations

import numpy as np

from . import Params, _epoch_of, prep, prep_adjoint, step_discrete

OFFS = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]


def _neighbour(x, dr, dc):
    """y[r, c] = x[r + dr, c + dc], 0 outside the grid."""
    H, W = x.shape
    y = np.zeros_like(x)
    rs, re = max(0, -dr), H - max(0, dr)
    cs, ce = max(0, -dc), W - max(0, dc)
    y[rs:re, cs:ce] = x[rs + dr:re + dr, cs + dc:ce + dc]
    return y


def dca_forward(land, winds, starts, prm: Params, S0, T, seed, run0=0, fire=0):
    """Discrete trajectory with the accumulator. S0: uint8 (H, W) or (R, H, W).
    Returns (S_T, acc, t_ign, states): acc / t_ign of the shape of S0 (t_ign = -1 where
    no ignition happened), states = [S_0 .. S_T]."""
    S = np.ascontiguousarray(S0, dtype=np.uint8)
    squeeze = S.ndim == 2
    S3 = S[None] if squeeze else S
    R, H, W = S3.shape
    acc = np.zeros((R, H, W))
    t_ign = np.full((R, H, W), -1, dtype=np.int64)
    states = [S3.copy()]
    qs = {}
    for t in range(T):
        e = _epoch_of(t, starts)
        if e not in qs:
            V, th = winds[e]
            qs = {e: prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm)}
        Sn, P, _ = step_discrete(S3, qs[e], prm.p_continue, seed, t, run0, fire, return_P=True)
        new = (S3 == 1) & (Sn == 2)
        acc[new] = P[new]
        t_ign[new] = t
        S3 = Sn
        states.append(S3.copy())
    if squeeze:
        return S3[0], acc[0], t_ign[0], [s[0] for s in states]
    return S3, acc, t_ign, states


def step_rings(T, r_first, r_last, r_between):
    """Boolean mask over steps 0..T-1 of the steps that carry gradient: 0..r_first-1,
    T-r_last..T-1 and r_between steps evenly spaced strictly between the two groups
    (step r_first - 1 + round((k + 1) * gap / (r_between + 1)), k < r_between, with
    gap = T - r_last - r_first + 1)."""
    m = np.zeros(T, dtype=bool)
    m[:max(0, min(T, r_first))] = True
    if r_last > 0:
        m[max(0, T - r_last):] = True
    lo, hi = r_first - 1, T - r_last
    gap = hi - lo
    for k in range(r_between):
        t = lo + int(round((k + 1) * gap / (r_between + 1)))
        if lo < t < hi:
            m[t] = True
    return m


def dca_gq(states, t_ign, q_of_step, w, mask=None):
    """dL/dq per wind epoch from dL/dacc = w (shape of t_ign): {epoch: Gq[8, H, W]}.
    q_of_step(t) -> (epoch, q[8, H, W])."""
    st = [s if s.ndim == 3 else s[None] for s in states]
    tig = t_ign if t_ign.ndim == 3 else t_ign[None]
    w3 = w if w.ndim == 3 else w[None]
    R, H, W = tig.shape
    out = {}
    for t in range(len(st) - 1):
        if mask is not None and not mask[t]:
            continue
        e, q = q_of_step(t)
        G = out.setdefault(e, np.zeros((8, H, W)))
        for r in range(R):
            sel = tig[r] == t
            if not sel.any():
                continue
            beta = (st[t][r] == 2).astype(np.float64)
            nb = [_neighbour(beta, dr, dc) for dr, dc in OFFS]
            f = [1.0 - nb[d] * q[d] for d in range(8)]
            for d in range(8):
                loo = np.ones((H, W))
                for e2 in range(8):
                    if e2 != d:
                        loo = loo * f[e2]
                G[d] += np.where(sel, w3[r] * nb[d] * loo, 0.0)
    return out


def dca_backward(land, winds, starts, prm: Params, states, t_ign, w, mask=None):
    """Gradient of sum(w * acc) w.r.t. (p_h, c1, c2, a) and per-cell p_veg, p_den, with
    the trajectory fixed. Returns (g4, g_pveg, g_pden)."""
    H, W = land.E.shape
    qs = {}

    def q_of_step(t):
        e = _epoch_of(t, starts)
        if e not in qs:
            V, th = winds[e]
            qs[e] = prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm)
        return e, qs[e]

    g4 = np.zeros(4)
    gpv = np.zeros((H, W))
    gpd = np.zeros((H, W))
    for e, G in dca_gq(states, t_ign, q_of_step, w, mask).items():
        V, th = winds[e]
        a4, pv, pd = prep_adjoint(H, W, land.E, land.p_veg, land.p_den, V, th, prm, G)
        g4 += a4
        gpv += pv
        gpd += pd
    return g4, gpv, gpd


def frozen_accumulator(land, winds, starts, prm: Params, states, t_ign):
    """The accumulator recomputed at parameters prm with the burning sets and ignition
    events of a recorded trajectory held fixed: acc_j = 1 - prod_d (1 - beta_i q_dj) at
    j's ignition step. Its derivative is what ``dca_backward`` returns."""
    st = [s if s.ndim == 3 else s[None] for s in states]
    tig = t_ign if t_ign.ndim == 3 else t_ign[None]
    R, H, W = tig.shape
    acc = np.zeros((R, H, W))
    qs = {}
    for t in range(len(st) - 1):
        e = _epoch_of(t, starts)
        if e not in qs:
            V, th = winds[e]
            qs[e] = prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm)
        q = qs[e]
        for r in range(R):
            sel = tig[r] == t
            if not sel.any():
                continue
            beta = (st[t][r] == 2).astype(np.float64)
            surv = np.ones((H, W))
            for d, (dr, dc) in enumerate(OFFS):
                surv = surv * (1.0 - _neighbour(beta, dr, dc) * q[d])
            acc[r][sel] = 1.0 - surv[sel]
    return acc if t_ign.ndim == 3 else acc[0]


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def eq10_loss(yhat, y, pool=4):
    """Eq. 10 on one map: BCE with logits of yhat against y, averaged over the crop to the
    bounding box of the union of non-zero yhat and y (0 if that union is empty), plus the
    mean of (AvgPool(y) - AvgPool(yhat))^2 over the pool x pool, stride-pool windows that
    fit in the map. Returns (loss, dL/dyhat)."""
    yhat = np.asarray(yhat, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    H, W = yhat.shape
    g = np.zeros((H, W))
    loss = 0.0
    nz = (yhat != 0) | (y != 0)
    if nz.any():
        rows = np.nonzero(nz.any(axis=1))[0]
        cols = np.nonzero(nz.any(axis=0))[0]
        r0, r1, c0, c1 = rows[0], rows[-1] + 1, cols[0], cols[-1] + 1
        x = yhat[r0:r1, c0:c1]
        t = y[r0:r1, c0:c1]
        n = x.size
        s = _sigmoid(x)
        loss += float(np.mean(-(t * np.log(s) + (1.0 - t) * np.log(1.0 - s))))
        g[r0:r1, c0:c1] += (s - t) / n
    Hp, Wp = H // pool, W // pool
    if Hp and Wp:
        yp = y[:Hp * pool, :Wp * pool].reshape(Hp, pool, Wp, pool).mean(axis=(1, 3))
        xp = yhat[:Hp * pool, :Wp * pool].reshape(Hp, pool, Wp, pool).mean(axis=(1, 3))
        diff = xp - yp
        loss += float(np.mean(diff ** 2))
        gp = 2.0 * diff / diff.size / (pool * pool)
        g[:Hp * pool, :Wp * pool] += np.repeat(np.repeat(gp, pool, axis=0), pool, axis=1)
    return loss, g
