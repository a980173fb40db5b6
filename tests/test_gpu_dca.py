"""GPU parity of the paper's accumulator calibration path (Sec. 2.2-2.3) against the DCA
oracle: the accumulator (p_ignite of each cell at its ignition step) along the discrete
trajectory, the gradient of a loss of it with the trajectory held fixed (all steps and
step rings), and the loss of Eq. 10."""
import numpy as np
import pytest

import synthetic as syn
from oracle import Params, dca
from tests._util import PRM, cuda, set_landscape

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_2502_18738_gb300 as pf
    pf.build()
    pf.load()
    return pf


def _problem(H, W, seed, n_epochs=2, T=40):
    land = syn.make_landscape(H, W, seed)
    winds = [syn.smooth_wind(H, W, seed, e, sigma=8.0) for e in range(n_epochs)]
    starts = [int(round(e * T / n_epochs)) for e in range(n_epochs)]
    S0 = syn.initial_state(land, [(H // 2, W // 2), (H // 5, W // 4)])
    return land, winds, starts, S0


def _model(pf, land, winds, starts, H, W, R, seed):
    import torch
    m = pf.FireModel(H, W, pf.PF_DISCRETE, R, seed=seed)
    set_landscape(m, land, *winds[0])
    for (V, th), s in list(zip(winds, starts))[1:]:
        m.set_wind(cuda(V), cuda(th), s)
    m.set_params(**PRM)
    acc = m.set_accumulator(torch.zeros((R, H, W), dtype=torch.float32, device="cuda"))
    return m, acc


@pytest.mark.parametrize("kernel,k", [(1, 1), (2, 8), (2, 5)])
def test_accumulator_matches_oracle(pf, kernel, k):
    H, W, T, R = 150, 190, 40, 2
    land, winds, starts, S0 = _problem(H, W, 11, T=T)
    m, acc = _model(pf, land, winds, starts, H, W, R, seed=77)
    m.set_tuning(kernel=kernel, k=k)
    S = np.broadcast_to(S0, (R, H, W)).copy()
    out = m.forward(cuda(S), T).cpu().numpy()
    prm = Params(**PRM)
    S_T, acc_o, t_ign, _ = dca.dca_forward(land, winds, starts, prm, S, T, seed=77)
    assert np.array_equal(out, S_T)
    got = acc.cpu().numpy().astype(np.float64)
    ign = t_ign >= 0
    assert ign.sum() > 200
    assert np.all(got[~ign] == 0.0)
    assert np.all(np.abs(got[ign] - acc_o[ign]) <= 2e-6 * acc_o[ign] + 1e-7)


@pytest.mark.parametrize("rings", [None, (3, 4, 3)])
def test_dca_gradient_matches_oracle(pf, rings):
    import torch
    H, W, T, R = 120, 140, 36, 2
    land, winds, starts, S0 = _problem(H, W, 5, T=T)
    m, acc = _model(pf, land, winds, starts, H, W, R, seed=9)
    S = np.broadcast_to(S0, (R, H, W)).copy()
    m.forward(cuda(S), T)
    w = np.random.default_rng(3).standard_normal((R, H, W)).astype(np.float32)
    mask = None if rings is None else dca.step_rings(T, *rings)
    g4, gpv, gpd = m.backward_dca(cuda(w), mask)
    prm = Params(**PRM)
    _, _, t_ign, states = dca.dca_forward(land, winds, starts, prm, S, T, seed=9)
    want4, wpv, wpd = dca.dca_backward(land, winds, starts, prm, states, t_ign, w.astype(np.float64), mask)
    for k in range(4):
        assert g4[k] == pytest.approx(want4[k], rel=1e-4, abs=1e-6 * np.abs(want4).max())
    for got, want in ((gpv.cpu().numpy(), wpv), (gpd.cpu().numpy(), wpd)):
        scale = np.abs(want).max()
        assert scale > 0
        assert np.all(np.abs(got - want) <= 1e-4 * np.abs(want) + 1e-6 * scale)


def test_eq10_loss_matches_oracle(pf):
    import torch
    H, W = 203, 170  # ragged against the 4 x 4 pool
    rng = np.random.default_rng(4)
    yhat = np.zeros((H, W), np.float32)
    yhat[40:150, 30:120] = rng.uniform(0, 1, (110, 90)).astype(np.float32)
    y = np.zeros((H, W), np.float32)
    y[60:180, 50:140] = 1.0
    g = torch.empty((H, W), dtype=torch.float32, device="cuda")
    loss = pf.pf_loss_eq10(cuda(yhat), cuda(y), g)
    want, wg = dca.eq10_loss(yhat.astype(np.float64), y.astype(np.float64))
    assert loss == pytest.approx(want, rel=1e-6)
    assert np.allclose(g.cpu().numpy(), wg, rtol=1e-5, atol=1e-9)
    z = torch.zeros((16, 16), device="cuda")
    assert pf.pf_loss_eq10(z, z, g[:16, :16].contiguous()) == 0.0


def test_dca_state_errors(pf):
    import torch
    H, W = 40, 40
    land, winds, starts, S0 = _problem(H, W, 2, n_epochs=1)
    m = pf.FireModel(H, W, pf.PF_DISCRETE, 1)
    set_landscape(m, land, *winds[0])
    m.set_params(**PRM)
    w = torch.zeros((1, H, W), device="cuda")
    with pytest.raises(pf.PFireError) as e:
        m.backward_dca(w)
    assert e.value.code == pf.PF_ESTATE
    m.set_accumulator(torch.zeros((1, H, W), device="cuda"))
    m.forward(cuda(S0[None].copy()), 10)
    m.backward_dca(w)
    m.set_params(**{**PRM, "p_h": 0.5})
    with pytest.raises(pf.PFireError) as e:
        m.backward_dca(w)
    assert e.value.code == pf.PF_ESTATE
    d = pf.FireModel(H, W, pf.PF_DIFF, 1)
    with pytest.raises(pf.PFireError) as e:
        d.set_accumulator(torch.zeros((1, H, W), device="cuda"))
    assert e.value.code == pf.PF_EINVAL


def test_calibration_loop_runs(pf):
    """Alg. 1 on a 96 x 96 map: observations from the hidden parameters of the
    calibration case (p_h 0.5, c1 0.05, c2 0.12, a 0.08); starting from the workload's
    parameters, four epochs of three iterations give finite losses and keep the
    parameters inside the clamps."""
    import torch
    from paper_2502_18738_gb300.calibrate import BOUNDS, calibrate, step_rings
    H = W = 96
    land, winds, _, S0 = _problem(H, W, 7, n_epochs=1)
    m = pf.FireModel(H, W, pf.PF_DISCRETE, 1, seed=0)
    set_landscape(m, land, *winds[0])
    hidden = dict(p_h=0.5, c1=0.05, c2=0.12, a=0.08, p_continue=0.3)
    m.set_params(**hidden)
    S = cuda(S0[None].copy())
    obs = []
    for it in range(3):
        m.reseed(0)
        out = m.forward(S, (it + 1) * 10)
        obs.append(((out[0] >= 2).float().contiguous(), None))
    p, hist = calibrate(m, S, obs, (0.58, 0.045, 0.131, 0.078), max_epochs=4, steps_update_interval=10,
                        lr=2e-2, rings=(2, 3, 1), seed0=0)
    assert all(np.isfinite(p))
    for v, name in zip(p, ("p_h", "c1", "c2", "a")):
        assert BOUNDS[name][0] <= v <= BOUNDS[name][1]
    assert len(hist) == 12 and all(np.isfinite(l) and l > 0 for _, _, l in hist)
    assert p != [0.58, 0.045, 0.131, 0.078]
    assert list(np.nonzero(step_rings(10, 2, 2, 1))[0]) == [0, 1, 5, 8, 9]


def test_calibration_loop_descends_towards_the_hidden_spread_parameter(pf):
    """Alg. 1 (Eq. 10 loss, accumulator gradient, AdamW, clamps) on an easy case: flat
    terrain, no wind and uniform vegetation, so q = f_p(p_h) in every direction and only
    p_h acts (the gradients in c1, c2, a are exactly 0). Observations come from p_h = 0.5;
    from an underburning start (p_h = 0.25) two epochs raise p_h towards 0.5, and the
    Eq. 10 loss of a re-simulation with the observations' seed falls. (Eq. 10 rewards a
    larger p_ignite at every correctly ignited cell, so the loop's resting point lies
    above the observations' p_h: the test asks for the descent, not for convergence.)"""
    import torch
    from paper_2502_18738_gb300.calibrate import calibrate
    H = W = 128
    z = torch.zeros((H, W), device="cuda")
    m = pf.FireModel(H, W, pf.PF_DISCRETE, 1, seed=0)
    m.set_env(z, z, z, z, z)
    m.set_params(p_h=0.5, c1=0.045, c2=0.131, a=0.078, p_continue=0.3)
    S0 = np.ones((1, H, W), dtype=np.uint8)
    S0[0, H // 2, W // 2] = 2
    S = cuda(S0)
    obs = []
    for it in range(3):
        m.reseed(0)
        out = m.forward(S, (it + 1) * 8)
        obs.append(((out[0] >= 2).float().contiguous(), None))

    def loss_at(p_h):
        m.set_params(p_h=p_h, c1=0.045, c2=0.131, a=0.078, p_continue=0.3)
        acc = m.set_accumulator(torch.zeros((1, H, W), device="cuda"))
        m.reseed(0)
        m.forward(S, 24)
        return pf.pf_loss_eq10(acc[0], obs[2][0], torch.empty((H, W), device="cuda"))

    p0 = 0.25
    before = loss_at(p0)
    p, hist = calibrate(m, S, obs, (p0, 0.045, 0.131, 0.078), max_epochs=2, steps_update_interval=8, lr=3e-2,
                        seed0=0)
    assert 0.30 < p[0] <= 0.5 + 0.05, (p, hist)
    assert p[1:] == pytest.approx([0.045, 0.131, 0.078], abs=1e-3)  # only weight decay acts on them
    after = loss_at(p[0])
    assert after < before, (before, after, p)


def test_paper_style_model_object(pf):
    """WildfireModel (the paper's compute / reset / accumulator / state calls) runs the
    same trajectory as a FireModel, and its backward uses the attached steps."""
    import torch
    H, W, T = 80, 90, 24
    land, winds, _, S0 = _problem(H, W, 13, n_epochs=1)
    V, th = winds[0]
    fire = torch.from_numpy(S0 == 2).cuda()
    nb = torch.from_numpy(S0 == 0).cuda()
    wm = pf.WildfireModel(fire, cuda(V), cuda(th), altitude=cuda(land.E), canopy=cuda(land.p_veg),
                          density=cuda(land.p_den), non_burnable=nb, seed=3, **{k: PRM[k] for k in
                                                                               ("p_h", "c1", "c2", "a", "p_continue")})
    attach = [t < 3 or t >= T - 5 for t in range(T)]
    for t in range(T):
        wm.compute(attach=attach[t])
    m, acc = _model(pf, land, [(V, th)], [0], H, W, 1, seed=3)
    out = m.forward(cuda(S0[None].copy()), T)
    st = wm.state
    assert torch.equal(st[0], out[0] == 2) and torch.equal(st[1], out[0] == 3)
    assert torch.equal(wm.accumulator, acc)
    w = torch.from_numpy(np.random.default_rng(2).standard_normal((H, W)).astype(np.float32)).cuda()
    g_model = wm.backward(w)
    g_ref, _, _ = m.backward_dca(w[None].contiguous(), np.array(attach), per_cell=False)
    assert np.allclose(g_model, g_ref, rtol=0, atol=0)
    wm.reset(seed=3)
    assert wm.steps == 0 and int(wm.state[0].sum()) == int(fire.sum())
    out2 = pf.simulate(cuda(S0), T, E=cuda(land.E), p_veg=cuda(land.p_veg), p_den=cuda(land.p_den), V_w=cuda(V),
                       theta_w=cuda(th), seed=3, **PRM)
    assert torch.equal(out2, out)
