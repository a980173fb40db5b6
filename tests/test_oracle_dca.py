"""Pins of the DCA oracle (accumulator of p_ignite over newly ignited cells, its
gradient with the trajectory held fixed, step rings, Eq. 10) against closed forms,
finite differences of the frozen-trajectory accumulator and PyTorch's own loss routines."""
import numpy as np
import pytest

import synthetic as syn
from oracle import Params, dca


def _case(H=26, W=22, T=14, seed=3):
    land = syn.make_landscape(H, W, seed)
    winds = [syn.smooth_wind(H, W, seed, e, sigma=6.0) for e in range(2)]
    starts = [0, T // 2]
    S0 = syn.initial_state(land, [(H // 2, W // 2), (4, 5)])
    return land, winds, starts, S0


def test_accumulator_holds_p_ignite_of_the_ignition_step(orc):
    land, winds, starts, S0 = _case()
    prm = Params(0.58, 0.045, 0.131, 0.078, 0.3)
    S_T, acc, t_ign, states = dca.dca_forward(land, winds, starts, prm, S0, 14, seed=5)
    ignited = t_ign >= 0
    assert ignited.sum() > 10
    assert np.all(acc[~ignited] == 0.0) and np.all((acc[ignited] > 0) & (acc[ignited] <= 1))
    # each ignited cell: unburned before its step, burning right after, and its entry is
    # that step's p_ignite from the plain step routine
    for r, c in np.argwhere(ignited)[:20]:
        t = t_ign[r, c]
        assert states[t][r, c] == 1 and states[t + 1][r, c] == 2
        e = 0 if t < starts[1] else 1
        q = orc.prep(*S0.shape, land.E, land.p_veg, land.p_den, *winds[e], prm)
        _, P, _ = orc.step_discrete(states[t], q, prm.p_continue, 5, t, return_P=True)
        assert acc[r, c] == P[r, c]
    q0, q1 = (orc.prep(*S0.shape, land.E, land.p_veg, land.p_den, *winds[e], prm) for e in (0, 1))
    S = orc.forward_discrete(S0, q0, prm.p_continue, seed=5, T=starts[1])
    S = orc.forward_discrete(S, q1, prm.p_continue, seed=5, T=14 - starts[1], step0=starts[1])
    assert np.array_equal(S_T, S)


def test_single_burning_neighbour_gradient_is_the_weight():
    # centre burning, cell (0, 1) ignited at step 0 by it alone: p_ignite = q, so
    # dp_ignite/dq_d = 1 for the direction pointing at the centre and 0 otherwise
    S0 = np.ones((3, 3), np.uint8)
    S0[1, 1] = 2
    t_ign = np.full((3, 3), -1)
    t_ign[0, 1] = 0
    q = np.full((8, 3, 3), 0.37)
    w = np.zeros((3, 3))
    w[0, 1] = 2.5
    G = dca.dca_gq([S0, S0], t_ign, lambda t: (0, q), w)[0]
    d_centre = dca.OFFS.index((1, 0))  # from (0, 1) the centre is one row down
    want = np.zeros((8, 3, 3))
    want[d_centre, 0, 1] = 2.5
    assert np.array_equal(G, want)
    # two burning neighbours: dP/dq_d = q_other
    S0[0, 0] = 2
    G = dca.dca_gq([S0, S0], t_ign, lambda t: (0, q), w)[0]
    d_left = dca.OFFS.index((0, -1))
    assert G[d_centre, 0, 1] == pytest.approx(2.5 * (1 - 0.37))
    assert G[d_left, 0, 1] == pytest.approx(2.5 * (1 - 0.37))


@pytest.mark.parametrize("mask_kind", ["all", "rings"])
def test_gradient_matches_finite_differences_of_the_frozen_accumulator(mask_kind):
    land, winds, starts, S0 = _case()
    T = 14
    prm = Params(0.58, 0.045, 0.131, 0.078, 0.3, exact=True)
    _, acc, t_ign, states = dca.dca_forward(land, winds, starts, prm, S0, T, seed=9)
    w = np.random.default_rng(0).standard_normal(acc.shape)
    mask = None if mask_kind == "all" else dca.step_rings(T, 2, 3, 2)
    if mask is not None:  # only the attached steps' ignitions carry gradient
        t_m = np.where((t_ign >= 0) & mask[np.maximum(t_ign, 0)], t_ign, -1)
    else:
        t_m = t_ign
    g4, gpv, gpd = dca.dca_backward(land, winds, starts, prm, states, t_ign, w, mask)

    def F(p, pv=None, pd=None):
        l2 = land if pv is None else syn.Landscape(land.E, pv, pd, land.burnable)
        return float(np.sum(w * dca.frozen_accumulator(l2, winds, starts, p, states, t_m)))

    base = dict(p_h=prm.p_h, c1=prm.c1, c2=prm.c2, a=prm.a)
    for k, name in enumerate(("p_h", "c1", "c2", "a")):
        h = 1e-6 * max(1.0, abs(base[name]))
        fd = (F(prm.with_(**{name: base[name] + h})) - F(prm.with_(**{name: base[name] - h}))) / (2 * h)
        assert g4[k] == pytest.approx(fd, rel=1e-6, abs=1e-9), name
    # per-cell p_veg / p_den at a few cells the fire reached (FP32 fields: exact steps)
    h = 2.0 ** -12
    for r, c in np.argwhere(t_m >= 0)[:4]:
        for grid, pv_or_pd in ((gpv, "pv"), (gpd, "pd")):
            f = [None, None]
            for s_i, sgn in enumerate((1, -1)):
                pv, pd = land.p_veg.copy(), land.p_den.copy()
                (pv if pv_or_pd == "pv" else pd)[r, c] += np.float32(sgn * h)
                f[s_i] = F(prm, pv, pd)
            fd = (f[0] - f[1]) / (2 * h)
            assert grid[r, c] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_step_rings():
    m = dca.step_rings(10, 2, 2, 1)
    assert list(np.nonzero(m)[0]) == [0, 1, 5, 8, 9]
    assert list(np.nonzero(dca.step_rings(10, 1, 1, 0))[0]) == [0, 9]
    assert dca.step_rings(6, 6, 0, 0).all()
    m = dca.step_rings(100, 3, 5, 4)
    assert m.sum() == 12 and m[:3].all() and m[95:].all()


def test_eq10_against_pytorch_routines():
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    rng = np.random.default_rng(2)
    H, W = 21, 18  # ragged against the 4 x 4 pool
    yhat = np.zeros((H, W))
    yhat[5:14, 3:11] = rng.uniform(0, 1, (9, 8))
    y = np.zeros((H, W))
    y[7:17, 6:13] = 1.0
    loss, g = dca.eq10_loss(yhat, y)
    x = torch.tensor(yhat, dtype=torch.float64, requires_grad=True)
    t = torch.tensor(y, dtype=torch.float64)
    r0, r1, c0, c1 = 5, 17, 3, 13  # bounding box of the union of the non-zero entries
    ref = F.binary_cross_entropy_with_logits(x[r0:r1, c0:c1], t[r0:r1, c0:c1]) + \
        F.mse_loss(F.avg_pool2d(x[None, None], 4, 4), F.avg_pool2d(t[None, None], 4, 4))
    ref.backward()
    assert loss == pytest.approx(float(ref), rel=1e-13)
    assert np.allclose(g, x.grad.numpy(), rtol=1e-12, atol=1e-15)
    # nothing predicted and nothing observed: no loss, no gradient
    l0, g0 = dca.eq10_loss(np.zeros((8, 8)), np.zeros((8, 8)))
    assert l0 == 0.0 and not g0.any()
