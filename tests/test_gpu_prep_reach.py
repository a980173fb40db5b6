"""q computed only within reach of the fire (the differentiable form's reach mask):
a run split into a short forward and a long pf_advance, whose fire spreads far beyond
the first call's mask, must equal the same run in one call bit for bit (the advance has
to rebuild q for its longer horizon), and p_ignite of a state set far from the previous
fire must match the oracle (pf_set_state invalidates the masked q)."""
import numpy as np
import pytest

import synthetic as syn
from tests._util import PRM, cuda, set_landscape

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_2502_18738_gb300 as pf
    pf.build()
    pf.load()
    return pf


def _model(pf, land, V, th, H, W, kernel):
    m = pf.FireModel(H, W, pf.PF_DIFF)
    set_landscape(m, land, V, th)
    m.set_params(**PRM)
    m.set_tuning(kernel=kernel)
    return m


@pytest.mark.parametrize("kernel", [1, 2])
def test_advance_beyond_the_first_horizon_equals_one_run(pf, kernel):
    H, W, T1, T2 = 512, 448, 6, 330
    land = syn.make_landscape(H, W, 12)
    V = np.full((H, W), 6.0, np.float32)
    th = np.full((H, W), 30.0, np.float32)
    S0 = syn.initial_state(land, [(H // 2, W // 2)])
    one = _model(pf, land, V, th, H, W, kernel)
    ref = one.forward(cuda(S0), T1 + T2).cpu().numpy()
    # the support of b grows by one cell per step: after T1 + T2 steps it reaches far
    # beyond T1 + 160 cells from the ignition
    rr, cc = np.nonzero(ref[1] > 0)
    assert max(np.abs(rr - H // 2).max(), np.abs(cc - W // 2).max()) > T1 + 200
    two = _model(pf, land, V, th, H, W, kernel)
    two.forward(cuda(S0), T1)
    got = two.advance(T2).cpu().numpy()
    assert np.array_equal(got, ref)


def test_ignition_map_after_set_state_far_from_the_fire(pf, orc):
    H, W = 400, 420
    land = syn.make_landscape(H, W, 13)
    V, th = syn.smooth_wind(H, W, 13, 0, sigma=8.0)
    m = _model(pf, land, V, th, H, W, 2)
    S0 = syn.initial_state(land, [(20, 20)])
    out = m.forward(cuda(S0), 5).cpu().numpy()
    # a new burning spot in the far corner, outside the reach of the first run's q
    a, b = out[0].copy(), out[1].copy()
    r, c = H - 30, W - 40
    a[r - 2:r + 3, c - 2:c + 3] = np.where(land.burnable[r - 2:r + 3, c - 2:c + 3] != 0, 0.6, 0.0)
    b[r - 2:r + 3, c - 2:c + 3] = np.where(land.burnable[r - 2:r + 3, c - 2:c + 3] != 0, 0.4, 0.0)
    a, b = a.astype(np.float32), b.astype(np.float32)
    m.set_state(5, cuda(np.stack([a, b])))
    Pg = m.ignition_map()[0].cpu().numpy()
    prm = orc.Params(**PRM)
    q = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm, burnable=land.burnable)
    _, _, P = orc.step_diff(a, b, q, prm.p_continue, return_P=True)
    near = np.zeros((H, W), bool)
    near[r - 4:r + 5, c - 4:c + 5] = True
    assert (P[near] > 0).any()
    err = np.abs(Pg - P)
    assert np.all(err <= 1e-5 * np.abs(P) + 1e-7), err.max()
