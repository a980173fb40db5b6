"""The segment recompute leaves unwritten the tiles that stay unchanged far from the fire
(their state stays in the segment's first slot, which the adjoint then reads). A state
with a large partly burned, no-longer-burning region and a fire running into it makes
tiles take every path: unwritten from the segment start, written again from slot 0 as
the fire approaches, near and live. The gradients must match the FP64 oracle's reverse
sweep over the same trajectory."""
import numpy as np
import pytest

import synthetic as syn
from tests._util import PRM, cuda, set_landscape

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-3


@pytest.fixture(scope="module")
def pf():
    import paper_2502_18738_gb300 as pf
    pf.build()
    pf.load()
    return pf


def test_gradients_with_a_long_quiescent_burned_region(pf, orc):
    H, W, T = 480, 528, 180
    land = syn.make_landscape(H, W, 21)
    V = np.full((H, W), 5.0, np.float32)
    th = np.zeros((H, W), np.float32)  # towards the east, into the burned block
    burn = land.burnable != 0
    S0 = np.where(burn, 1, 0).astype(np.uint8)
    a0 = np.zeros((H, W), np.float32)
    b0 = np.zeros((H, W), np.float32)
    a0[60:420, 200:520] = 0.65  # burned in part, nothing burning: quiescent but not void
    r, c = H // 2, 40
    a0[r - 2:r + 3, c - 2:c + 3] = 1.0
    b0[r - 2:r + 3, c - 2:c + 3] = 1.0
    a0 = np.where(burn, a0, 0).astype(np.float32)
    b0 = np.where(burn, b0, 0).astype(np.float32)

    m = pf.FireModel(H, W, pf.PF_DIFF)
    set_landscape(m, land, V, th)
    m.set_params(**PRM)
    m.set_tuning(K=30)
    m.forward(cuda(S0), 0)  # the burnable mask
    m.set_state(0, cuda(np.stack([a0, b0])))
    out = m.advance(T).cpu().numpy()
    wts = (np.random.default_rng(5).random((H, W)) * 1e-3).astype(np.float32)
    g4, gpv, gpd = m.backward(cuda(wts), cuda((0.5 * wts).astype(np.float32)))

    prm = orc.Params(**PRM)
    q = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm, burnable=burn.astype(np.uint8))
    a, b = a0.astype(np.float64), b0.astype(np.float64)
    tape = []
    for _ in range(T):
        tape.append((a, b))
        a, b = orc.step_diff(a, b, q, prm.p_continue)
    # the fire reached the block: some of it burns at the end
    assert (b[60:420, 200:520] > 1e-3).any()
    err = np.abs(out[0] - a)
    assert np.all(err <= 1e-4 * np.abs(a) + 1e-6), err.max()
    w4, wpv, wpd = orc.diff_backward(land, [(V, th)], [0], prm, S0, tape, wts.astype(np.float64),
                                     (0.5 * wts).astype(np.float64))
    for k in range(4):
        assert g4[k] == pytest.approx(w4[k], rel=GRAD_RTOL), (k, g4, w4)
    for got, want in ((gpv.cpu().numpy(), wpv), (gpd.cpu().numpy(), wpd)):
        scale = np.abs(want).max()
        assert np.all(np.abs(got - want) <= GRAD_RTOL * np.abs(want) + 1e-5 * scale)
    m.close()
