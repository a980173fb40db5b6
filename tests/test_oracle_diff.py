"""Pins of the oracle's differentiable (mean-field) form: exact agreement with the
discrete form's one-step expectation, invariants, light cone, and rotation/reflection
symmetry of the whole prep + step pipeline."""
import numpy as np
import pytest

import synthetic as syn

PRM = dict(p_h=0.58, c1=0.045, c2=0.131, a=0.078, p_continue=0.3, l=30.0)


def test_one_step_from_one_hot_is_the_discrete_expectation(orc):
    from oracle import enumeration as en
    H, W = 3, 4
    land = syn.make_landscape(H, W, 4, nonburnable_frac=0.0)
    prm = orc.Params(**PRM)
    V, th = syn.uniform_wind(H, W, 4.0, 200.0)
    q = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm)
    S0 = np.array([[1, 2, 1, 3], [2, 1, 1, 1], [1, 1, 2, 1]], np.uint8)
    m = en.marginals(en.distribution(S0, q, prm.p_continue, 1), (H, W))
    a, b = orc.diff_init(S0)
    a1, b1 = orc.step_diff(a, b, q, prm.p_continue)
    assert np.allclose(a1, m[2] + m[3], atol=1e-14)
    assert np.allclose(b1, m[2], atol=1e-14)


def test_invariants_and_light_cone(orc):
    H, W, T = 48, 40, 25
    land = syn.make_landscape(H, W, 2)
    prm = orc.Params(**PRM)
    winds = [syn.smooth_wind(H, W, 2, 0, sigma=6.0)]
    S0 = syn.initial_state(land, [(24, 20)])
    a, b = orc.diff_init(S0)
    q = orc.prep(H, W, land.E, land.p_veg, land.p_den, *winds[0], prm, burnable=(S0 != 0))
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    cheb = np.maximum(np.abs(rr - 24), np.abs(cc - 20))
    for t in range(1, T + 1):
        a2, b2 = orc.step_diff(a, b, q, prm.p_continue)
        assert np.all(a2 >= a - 1e-15)
        assert np.all(b2 >= -1e-15) and np.all(b2 <= a2 + 1e-15) and np.all(a2 <= 1 + 1e-15)
        assert np.all(a2[cheb > t] == 0) and np.all(b2[cheb > t] == 0)
        assert np.all(a2[S0 == 0] == 0) and np.all(b2[S0 == 0] == 0)
        a, b = a2, b2


def _run(orc, land, V, th, S0, T, prm):
    H, W = S0.shape
    a, b, _ = orc.diff_forward(land, [(V, th)], [0], prm, S0, T, keep_states=False)
    return a, b


def test_rot90_symmetry_calm_flat(orc):
    H = W = 21
    prm = orc.Params(**PRM)
    land = syn.Landscape(E=np.zeros((H, W), np.float32), p_veg=np.full((H, W), 0.4, np.float32),
                         p_den=np.zeros((H, W), np.float32), burnable=np.ones((H, W), np.uint8))
    S0 = np.ones((H, W), np.uint8)
    S0[10, 10] = 2
    S0[7, 12] = 2
    V = np.zeros((H, W), np.float32)
    a, b = _run(orc, land, V, V, S0, 8, prm)
    land_r = syn.Landscape(*(np.ascontiguousarray(np.rot90(x)) for x in
                             (land.E, land.p_veg, land.p_den, land.burnable)))
    ar, br = _run(orc, land_r, V, V, np.ascontiguousarray(np.rot90(S0)), 8, prm)
    assert np.allclose(ar, np.rot90(a), rtol=0, atol=1e-13)
    assert np.allclose(br, np.rot90(b), rtol=0, atol=1e-13)


@pytest.mark.parametrize("kind", ["rot90", "transpose"])
def test_symmetry_with_wind_and_terrain(orc, kind):
    # Rotating every field by 90 deg counter-clockwise and turning the wind by +90 deg,
    # or reflecting about the main diagonal and mapping theta -> 270 - theta, must
    # commute with the model: pins the direction tables and the wind-angle convention.
    H, W = 23, 19
    prm = orc.Params(**PRM)
    land = syn.make_landscape(H, W, 8)
    V, th = syn.smooth_wind(H, W, 8, 0, sigma=5.0)
    S0 = syn.initial_state(land, [(11, 9), (4, 15)])
    a, b = _run(orc, land, V, th, S0, 10, prm)
    if kind == "rot90":
        f = lambda x: np.ascontiguousarray(np.rot90(x))
        th2 = (th + 90.0).astype(np.float32)
    else:
        f = lambda x: np.ascontiguousarray(x.T)
        th2 = (270.0 - th).astype(np.float32)
    land2 = syn.Landscape(f(land.E), f(land.p_veg), f(land.p_den), f(land.burnable))
    a2, b2 = _run(orc, land2, f(V), f(th2), f(S0), 10, prm)
    # theta + 90 is rounded to FP32, so the cos term differs at the 1e-7 level
    assert np.allclose(a2, f(a), rtol=0, atol=5e-6)
    assert np.allclose(b2, f(b), rtol=0, atol=5e-6)
    assert np.abs(a).max() > 0.5


def test_c_oracle_matches_autograd_restatement_forward(orc):
    torch = pytest.importorskip("torch")
    from oracle import torch_ref
    H, W, T = 17, 22, 9
    land = syn.make_landscape(H, W, 12)
    prm = orc.Params(**PRM)
    winds = [syn.smooth_wind(H, W, 12, e, sigma=5.0) for e in range(2)]
    S0 = syn.initial_state(land, [(8, 11)])
    a, b, _ = orc.diff_forward(land, winds, [0, 4], prm, S0, T, keep_states=False)
    d = dict(p_h=prm.p_h, c1=prm.c1, c2=prm.c2, a=prm.a, p_continue=prm.p_continue, l=prm.l)
    at, bt, _ = torch_ref.run(land, winds, [0, 4], d, S0, T, requires_grad=False)
    assert np.allclose(a, at.numpy(), rtol=0, atol=1e-13)
    assert np.allclose(b, bt.numpy(), rtol=0, atol=1e-13)


@pytest.mark.parametrize("x", [1e-20, 1e-9, 0.3])
def test_single_source_gives_p_equal_bq_at_any_magnitude(orc, x):
    # Eq. 9 with one source: P = b q exactly, also far below FP64's 1 - x resolution
    H, W = 3, 4
    q = np.zeros((8, H, W))
    q[4, 1, 1] = 0.5          # cell (1,1) receives from its East neighbour (1,2)
    a = np.zeros((H, W))
    b = np.zeros((H, W))
    b[1, 2] = 2 * x
    a1, b1, P = orc.step_diff(a, b, q, 0.3, return_P=True)
    assert P[1, 1] == pytest.approx(x, rel=1e-14)
    assert a1[1, 1] == pytest.approx(x, rel=1e-14)
