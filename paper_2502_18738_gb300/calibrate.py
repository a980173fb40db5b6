"""Parameter calibration on the fly (Sec. 2.3, Alg. 1) over the discrete form's
accumulator: every iteration re-simulates from the initial fire with the latest
parameters and the epoch's seed, takes the loss of Eq. 10 between the accumulator and
the iteration's observed burn map, back-propagates it through p_ignite of the newly
ignited cells of the attached steps (pf_backward_dca), steps AdamW and clamps the
parameters. The simulation, the loss and the gradient run in libpfire's kernels; this
module only sequences them (PyTorch's AdamW updates the four scalars)."""
from __future__ import annotations

import numpy as np
import torch

from . import PF_DISCRETE, FireModel, pf_loss_eq10

# clamps applied after every update (Alg. 1)
BOUNDS = {"p_h": (0.2, 1.0), "c1": (0.0, 1.0), "c2": (0.0, 1.0), "a": (0.0, 1.0)}


def step_rings(T: int, r_first: int, r_last: int, r_between: int) -> np.ndarray:
    """Steps attached to the gradient ("update by step rings", Sec. 2.3): the first
    r_first and last r_last of T steps, and r_between steps evenly spaced between them
    (step r_first - 1 + round((k + 1) * gap / (r_between + 1)), gap = T - r_last - r_first + 1)."""
    m = np.zeros(T, dtype=bool)
    m[:max(0, min(T, r_first))] = True
    if r_last > 0:
        m[max(0, T - r_last):] = True
    lo, hi = r_first - 1, T - r_last
    for k in range(r_between):
        t = lo + int(round((k + 1) * (hi - lo) / (r_between + 1)))
        if lo < t < hi:
            m[t] = True
    return m


def calibrate(model: FireModel, S_init, observations, p0, p_continue=0.3, l=30.0, max_epochs=1,
              steps_update_interval=10, lr=5e-3, rings=None, seed0=0, fields=None):
    """Alg. 1. model: a discrete FireModel with one realisation and its fields set.
    S_init: CUDA uint8 [1][H][W]. observations: list over iterations of (y, wind) with y a
    CUDA FP32 [H][W] 0/1 map observed after (iteration + 1) * steps_update_interval steps
    and wind None or (V_w, theta_w) CUDA tensors applied for that iteration's simulation
    (with fields = (E, p_veg, p_den), the tensors the model's landscape was set from).
    p0: initial (p_h, c1, c2, a). rings: None (every step carries gradient) or
    (r_first, r_last, r_between). Returns (parameters, history of (epoch, iteration, loss))."""
    if model.form != PF_DISCRETE or model.R != 1:
        raise ValueError("calibrate: a discrete model with one realisation is expected")
    theta = torch.tensor([float(v) for v in p0], dtype=torch.float64, requires_grad=True)
    opt = torch.optim.AdamW([theta], lr=lr)
    acc = model.set_accumulator(torch.zeros((1, model.H, model.W), dtype=torch.float32, device="cuda"))
    g = torch.empty((model.H, model.W), dtype=torch.float32, device="cuda")
    history = []
    for epoch in range(max_epochs):
        model.reseed(seed0 + epoch)  # one seed per epoch, reused by its iterations
        for it, (y, wind) in enumerate(observations):
            steps = (it + 1) * steps_update_interval
            if wind is not None:
                if fields is None:
                    raise ValueError("calibrate: per-iteration wind needs fields=(E, p_veg, p_den)")
                model.set_env(*fields, wind[0], wind[1])
            p_h, c1, c2, a = (float(v) for v in theta.detach())
            model.set_params(p_h, c1, c2, a, p_continue, l)
            model.forward(S_init, steps)
            loss = pf_loss_eq10(acc[0], y, g)
            mask = None if rings is None else step_rings(steps, *rings)
            g4, _, _ = model.backward_dca(g[None], mask, per_cell=False)
            theta.grad = torch.tensor(g4, dtype=torch.float64)
            opt.step()
            opt.zero_grad()
            with torch.no_grad():
                for k, name in enumerate(("p_h", "c1", "c2", "a")):
                    theta[k].clamp_(*BOUNDS[name])
            history.append((epoch, it, loss))
    return [float(v) for v in theta.detach()], history
