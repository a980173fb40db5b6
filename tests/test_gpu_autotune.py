"""pf_autotune: it picks one of the launch configurations, and the result of a forward
does not depend on the pick (every candidate computes the same arithmetic)."""
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


@pytest.mark.parametrize("form,R", [(0, 3), (1, 1)])
def test_autotune_picks_a_candidate_and_keeps_results(pf, form, R):
    H, W, T = 300, 260, 45
    land = syn.make_landscape(H, W, 8)
    V, th = syn.smooth_wind(H, W, 8, 0, sigma=8.0)
    S0 = syn.initial_state(land, [(150, 130), (40, 200)])
    S = np.broadcast_to(S0, (R, H, W)).copy() if form == 0 else S0
    m = pf.FireModel(H, W, form, R, seed=21)
    set_landscape(m, land, V, th)
    m.set_params(**PRM)
    ref = m.forward(cuda(S), T).cpu().numpy()
    t = m.autotune(cuda(S), 24)
    assert t["kernel"] in (1, 2)
    assert (t["k"] in (4, 8, 12)) if (form == 0 and t["kernel"] == 2) else (1 <= t["k"] <= 8)
    assert pf.pf_get_tuning(m.h)["kernel"] == t["kernel"]
    got = m.forward(cuda(S), T).cpu().numpy()
    assert np.array_equal(got, ref)
    if form == 1:  # a tape exists again after the forward
        import torch
        g = torch.full((H, W), 1e-3, device="cuda")
        g4, _, _ = m.backward(g, None)
        assert all(np.isfinite(g4))


def test_autotune_rejects_bad_arguments(pf):
    m = pf.FireModel(16, 16, 1, 1)
    S = cuda(np.ones((16, 16), np.uint8))
    with pytest.raises(pf.PFireError) as e:
        m.autotune(S, 0)
    assert e.value.code == pf.PF_EINVAL
    bad = cuda(np.full((16, 16), 9, np.uint8))
    with pytest.raises(pf.PFireError):
        m.autotune(bad, 4)
