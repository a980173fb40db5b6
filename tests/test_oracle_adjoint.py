"""Pins of the oracle's adjoint: dot-product (transpose) test of one step, full
parameter and per-cell gradients against central finite differences in FP64 and
against the independent autograd restatement."""
import numpy as np
import pytest

import synthetic as syn

PRM = dict(p_h=0.58, c1=0.045, c2=0.131, a=0.078, p_continue=0.3, l=30.0)


def test_adjoint_step_is_the_transpose(orc):
    H, W = 9, 11
    rng = np.random.default_rng(0)
    land = syn.make_landscape(H, W, 3)
    prm = orc.Params(**PRM)
    V, th = syn.smooth_wind(H, W, 3, 0, sigma=4.0)
    q = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm, burnable=land.burnable)
    a, b = syn.random_diff_state(H, W, 1, land.burnable)
    a, b = a.astype(np.float64), b.astype(np.float64)
    la1, lb1 = rng.standard_normal((H, W)), rng.standard_normal((H, W))
    Gq = np.zeros((8, H, W))
    la0, lb0 = orc.adjoint_step(a, b, q, prm.p_continue, la1, lb1, Gq)
    da, db, dq = rng.standard_normal((H, W)), rng.standard_normal((H, W)), rng.standard_normal((8, H, W))
    h = 1e-6
    ap, bp = orc.step_diff(a + h * da, b + h * db, q + h * dq, prm.p_continue)
    am, bm = orc.step_diff(a - h * da, b - h * db, q - h * dq, prm.p_continue)
    lhs = np.sum(la1 * (ap - am) + lb1 * (bp - bm)) / (2 * h)
    rhs = np.sum(la0 * da) + np.sum(lb0 * db) + np.sum(Gq * dq)
    assert lhs == pytest.approx(rhs, rel=1e-8)


def _problem(orc, H=20, W=18, T=14):
    land = syn.make_landscape(H, W, 21)
    winds = [syn.smooth_wind(H, W, 21, e, sigma=5.0) for e in range(2)]
    starts = [0, 6]
    S0 = syn.initial_state(land, [(10, 9), (3, 4)])
    y = (syn.random_state(H, W, 5) >= 2).astype(np.float64)
    return land, winds, starts, S0, y, T


def _loss(orc, land, winds, starts, S0, y, T, prm):
    a, b, _ = orc.diff_forward(land, winds, starts, prm, S0, T, keep_states=False)
    return orc.bce(a, y)[0]


def test_parameter_gradients_match_finite_differences(orc):
    land, winds, starts, S0, y, T = _problem(orc)
    prm = orc.Params(**PRM, exact=True)
    a, b, tape = orc.diff_forward(land, winds, starts, prm, S0, T)
    L, gA = orc.bce(a, y)
    g4, gpv, gpd = orc.diff_backward(land, winds, starts, prm, S0, tape, gA, np.zeros_like(gA))
    for k, name in enumerate(["p_h", "c1", "c2", "a"]):
        x = getattr(prm, name)
        h = 1e-6 * max(1.0, abs(x))
        Lp = _loss(orc, land, winds, starts, S0, y, T, Params_with(orc, prm, name, x + h))
        Lm = _loss(orc, land, winds, starts, S0, y, T, Params_with(orc, prm, name, x - h))
        fd = (Lp - Lm) / (2 * h)
        assert g4[k] == pytest.approx(fd, rel=1e-6, abs=1e-12), name
    # per-cell p_veg / p_den at a few burnable cells inside the burnt area
    rng = np.random.default_rng(1)
    cells = [tuple(c) for c in np.argwhere((a > 0.05) & (S0 == 1))]
    for idx in rng.choice(len(cells), size=4, replace=False):
        r, c = cells[idx]
        for field, g in (("p_veg", gpv), ("p_den", gpd)):
            h = 1e-6
            vals = []
            for s in (+1, -1):
                l2 = syn.Landscape(land.E, land.p_veg.copy(), land.p_den.copy(), land.burnable)
                arr = getattr(l2, field).astype(np.float64)
                arr[r, c] += s * h
                # FP64 perturbation: the oracle widens fields exactly, so pass FP64 here
                setattr(l2, field, arr)
                vals.append(_loss_f64fields(orc, l2, winds, starts, S0, y, T, prm))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert g[r, c] == pytest.approx(fd, rel=1e-5, abs=1e-11), (field, r, c)


def Params_with(orc, prm, name, value):
    d = dict(p_h=prm.p_h, c1=prm.c1, c2=prm.c2, a=prm.a, p_continue=prm.p_continue, l=prm.l)
    d[name] = value
    return orc.Params(**d, exact=True)


def _loss_f64fields(orc, land, winds, starts, S0, y, T, prm):
    # The C oracle takes FP32 fields; for a per-cell finite difference the field is
    # perturbed in FP64, so evaluate the loss with the autograd restatement instead.
    from oracle import torch_ref
    d = dict(p_h=prm.p_h, c1=prm.c1, c2=prm.c2, a=prm.a, p_continue=prm.p_continue, l=prm.l)
    _, _, _, loss = torch_ref.run(land, winds, starts, d, S0, T, y=y, requires_grad=False)
    return float(loss)


def test_gradients_match_autograd_restatement(orc):
    pytest.importorskip("torch")
    from oracle import torch_ref
    land, winds, starts, S0, y, T = _problem(orc, 16, 21, 12)
    prm = orc.Params(**PRM)
    a, b, tape = orc.diff_forward(land, winds, starts, prm, S0, T)
    L, gA = orc.bce(a, y)
    lb = np.random.default_rng(2).standard_normal(a.shape) * 1e-3   # a terminal term on b too
    g4, gpv, gpd = orc.diff_backward(land, winds, starts, prm, S0, tape, gA, lb)
    d = dict(p_h=prm.p_h, c1=prm.c1, c2=prm.c2, a=prm.a, p_continue=prm.p_continue, l=prm.l)
    at, bt, leaves, loss = torch_ref.run(land, winds, starts, d, S0, T, y=y)
    import torch
    (loss + torch.sum(bt * torch.as_tensor(lb))).backward()
    assert float(loss.detach()) == pytest.approx(L, rel=1e-12)
    for k, name in enumerate(["p_h", "c1", "c2", "a"]):
        assert g4[k] == pytest.approx(float(leaves[name].grad), rel=1e-9, abs=1e-15), name
    assert np.allclose(gpv, leaves["p_veg"].grad.numpy(), rtol=1e-9, atol=1e-15)
    assert np.allclose(gpd, leaves["p_den"].grad.numpy(), rtol=1e-9, atol=1e-15)
