"""Pins of the oracle's prep (Eq. 1-5): closed forms at configurations where the full
pipeline reduces to a single factor, and the direction conventions."""
import math

import numpy as np
import pytest

C = 1.1486328125
# direction index of the neighbour at offset (dr, dc) from the receiving cell
D = {(-1, -1): 0, (-1, 0): 1, (-1, 1): 2, (0, -1): 3, (0, 1): 4, (1, -1): 5, (1, 0): 6, (1, 1): 7}


def _prep3(orc, E=None, pv=0.0, pd=0.0, V=0.0, th=0.0, **kw):
    # parameters taken as exact decimals (exact=True) so that the hand-derived values
    # below apply; the fields are FP32 as everywhere else
    H = W = 3
    prm = orc.Params(**{**dict(p_h=0.58, c1=0.045, c2=0.131, a=0.078, p_continue=0.3, l=30.0), **kw},
                     exact=True)
    f = lambda v: np.full((H, W), v, dtype=np.float32)
    q = orc.prep(H, W, E, f(pv), f(pd), f(V), f(th), prm)
    return q, prm


def test_flat_calm_is_tanh_c_ph(orc):
    q, prm = _prep3(orc)
    want = math.tanh(C * prm.p_h)
    assert np.allclose(q[:, 1, 1], want, rtol=0, atol=1e-15)
    # the value derived by hand from Eq. 2-5 for p_h = 0.58: tanh(c p_h) with c of Eq. 8
    assert abs(q[0, 1, 1] - 0.5824793373) < 1e-9


def test_vegetation_density_factors(orc):
    q, prm = _prep3(orc, pv=0.4, pd=0.3)
    pv, pd = float(np.float32(0.4)), float(np.float32(0.3))
    assert abs(q[3, 1, 1] - math.tanh(C * prm.p_h * (1 + pv) * (1 + pd))) < 1e-15
    # hand-derived with decimal 0.4 and 0.3; the fields are FP32-rounded (rel. ~1e-8)
    assert abs(q[3, 1, 1] - 0.8374268840) < 1e-7
    q, prm = _prep3(orc, pv=-0.3, pd=-0.4)
    assert abs(q[3, 1, 1] - 0.2727264019) < 1e-7


def test_ph_zero_means_no_propagation(orc):
    q, _ = _prep3(orc, V=7.0, th=30.0, p_h=0.0)
    assert np.all(q == 0.0)


@pytest.mark.parametrize("theta_w, src, cos_theta", [
    (0.0, (0, -1), 1.0),     # wind toward East: spread from the West neighbour is downwind
    (0.0, (0, 1), -1.0),     # ... and from the East neighbour it is upwind
    (0.0, (-1, 0), 0.0),     # ... and from the North neighbour it is crosswind
    (90.0, (1, 0), 1.0),     # wind toward North: the South neighbour is upwind of j
    (90.0, (-1, 0), -1.0),
    (45.0, (1, -1), 1.0),    # toward North-East: the South-West neighbour
    (45.0, (-1, 1), -1.0),
    (180.0, (0, 1), 1.0),    # toward West: the East neighbour
    (45.0, (0, -1), math.cos(math.radians(45.0))),
])
def test_wind_direction_conventions(orc, theta_w, src, cos_theta):
    V = 5.0
    q, prm = _prep3(orc, V=V, th=theta_w)
    pw = math.exp(prm.c1 * V) * math.exp(prm.c2 * V * (cos_theta - 1.0))
    assert abs(q[D[src], 1, 1] - math.tanh(C * prm.p_h * pw)) < 1e-14


def test_wind_factor_hand_derived_values(orc):
    # p_w at V = 5, c1 = 0.045, c2 = 0.131 for theta = 0, 45, 90, 180 deg (hand-derived)
    q, prm = _prep3(orc, V=5.0, th=0.0, p_h=1.0)
    got = {}
    for src, ang in [((0, -1), 0), ((-1, -1), 45), ((-1, 0), 90), ((0, 1), 180)]:
        got[ang] = math.atanh(q[D[src], 1, 1]) / C
    assert abs(got[0] - 1.2523227) < 1e-6
    assert abs(got[45] - 1.0337107) < 1e-6
    assert abs(got[90] - 0.6505091) < 1e-6
    assert abs(got[180] - 0.3379018) < 1e-6


def test_slope_edge_and_diagonal(orc):
    # receiving cell 5 m above its neighbours: spread toward it is uphill (positive slope)
    E = np.zeros((3, 3), dtype=np.float32)
    E[1, 1] = 5.0
    q, prm = _prep3(orc, E=E, p_h=1.0)
    ps_edge = math.atanh(q[D[(0, -1)], 1, 1]) / C
    ps_diag = math.atanh(q[D[(-1, -1)], 1, 1]) / C
    assert abs(ps_edge - 2.0918757) < 1e-6   # atan(5/30) = 9.4623 deg
    assert abs(ps_diag - 1.6892199) < 1e-6   # atan(5/(30*sqrt 2)) = 6.7214 deg
    # the neighbour at (0, 0) receives from the centre downhill: slope negative
    ps_down = math.atanh(q[D[(1, 1)], 0, 0]) / C
    assert abs(ps_down - 1.0 / 1.6892199) < 1e-6


def test_boundary_directions_are_zero(orc):
    q, _ = _prep3(orc, V=3.0, th=10.0)
    # corner (0, 0) has neighbours only at (0,1), (1,0), (1,1)
    inside = {D[(0, 1)], D[(1, 0)], D[(1, 1)]}
    for d in range(8):
        assert (q[d, 0, 0] > 0) == (d in inside)


def test_nonburnable_mask(orc):
    H = W = 4
    prm = orc.Params(0.58, 0.045, 0.131, 0.078, 0.3)
    f = lambda v: np.full((H, W), v, dtype=np.float32)
    burn = np.ones((H, W), np.uint8)
    burn[2, 1] = 0
    q = orc.prep(H, W, None, f(0), f(0), f(1), f(0), prm, burnable=burn)
    assert np.all(q[:, 2, 1] == 0.0)
    assert np.all(q[:, 1, 1] > 0.0)


def test_constant_c_reproduces_its_design():
    # Eq. 8's c was chosen as the least-squares fit of tanh(c x) to x on [0.2, 0.8];
    # the fit lands within 0.002 of the printed value (pins the tanh form, not c).
    from scipy.optimize import minimize_scalar
    x = np.linspace(0.2, 0.8, 601)
    res = minimize_scalar(lambda c: np.sum((np.tanh(c * x) - x) ** 2), bounds=(0.5, 2), method="bounded")
    assert abs(res.x - C) < 0.002
    # the rival forms of Eq. 6/7 fit worse at their own optimum
    r6 = minimize_scalar(lambda c: np.sum((1 - c ** (-x) - x) ** 2), bounds=(1.01, 50), method="bounded")
    r7 = minimize_scalar(lambda c: np.sum((1 - (x + 1) ** (-c) - x) ** 2), bounds=(0.01, 10), method="bounded")
    assert res.fun < r6.fun and res.fun < r7.fun


def test_slope_tensor_input_reproduces_the_altitude_path(orc):
    """The H x W x 3 x 3 slope input of Sec. 2.1 ([r][c][dr+1][dc+1], degrees, Eq. 1 with E
    the cell and E-hat the neighbour) in place of E: fed the angles of an altitude map it
    gives the same q; all-zero slopes give flat ground; one angle moves only its q."""
    import numpy as np
    import synthetic as syn
    H, W = 13, 11
    land = syn.make_landscape(H, W, 2)
    V, th = syn.uniform_wind(H, W, 4.0, 30.0)
    prm = orc.Params(0.58, 0.045, 0.131, 0.078, 0.3)
    E = land.E.astype(np.float64)
    slope = np.zeros((H, W, 3, 3), np.float32)
    for dr in (-1, 0, 1):
        for dc in (-1, 0, 1):
            if dr == dc == 0:
                continue
            k = np.sqrt(2.0) if dr and dc else 1.0
            nb = np.zeros_like(E)
            rs, re_ = max(0, -dr), H - max(0, dr)
            cs, ce = max(0, -dc), W - max(0, dc)
            nb[rs:re_, cs:ce] = E[rs + dr:re_ + dr, cs + dc:ce + dc]
            slope[:, :, dr + 1, dc + 1] = np.degrees(np.arctan((E - nb) / (k * 30.0)))
    q_E = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm)
    q_s = orc.prep(H, W, None, land.p_veg, land.p_den, V, th, prm, slope=slope)
    assert np.allclose(q_s, q_E, rtol=2e-6, atol=0)  # the angles went through FP32
    flat = orc.prep(H, W, None, land.p_veg, land.p_den, V, th, prm)
    assert np.array_equal(orc.prep(H, W, None, land.p_veg, land.p_den, V, th, prm,
                                   slope=np.zeros((H, W, 3, 3), np.float32)), flat)
    one = np.zeros((H, W, 3, 3), np.float32)
    one[6, 5, 0, 2] = 20.0  # cell (6, 5), neighbour (5, 6): direction d = 2
    q1 = orc.prep(H, W, None, land.p_veg, land.p_den, V, th, prm, slope=one)
    diff = np.argwhere(q1 != flat)
    assert [tuple(x) for x in diff] == [(2, 6, 5)]
    # Eq. 4: the slope factor exp(a theta_s) multiplies p_propagate inside f_p = tanh(c x)
    x_flat = np.arctanh(flat[2, 6, 5]) / orc.C_FP
    assert np.arctanh(q1[2, 6, 5]) / orc.C_FP == pytest.approx(x_flat * np.exp(prm.a * 20.0), rel=1e-12)
