"""Ensemble arrival probability and the evaluation metrics of Eq. 11-12 on the GPU,
against plain numpy on oracle-generated states (integer counts: exact)."""
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


def _ensemble(orc, H, W, R, T, seed):
    land = syn.make_landscape(H, W, seed)
    V, th = syn.smooth_wind(H, W, seed, 0, sigma=8.0)
    prm = orc.Params(**PRM)
    q = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm)
    S0 = np.broadcast_to(syn.initial_state(land, [(H // 2, W // 2)]), (R, H, W)).copy()
    return land, V, th, S0, orc.forward_discrete(S0, q, prm.p_continue, seed=seed, T=T)


def test_arrival_probability_counts_and_jaccard(pf, orc):
    H, W, R, T = 90, 110, 24, 25
    _, _, _, S0, S = _ensemble(orc, H, W, R, T, 3)
    aff = (S == 2) | (S == 3)
    P = pf.pf_arrival_probability(cuda(S)).cpu().numpy()
    assert np.array_equal(P, aff.sum(axis=0).astype(np.float32) / np.float32(R))
    assert pf.pf_affected_count(cuda(S)) == [int(v) for v in aff.reshape(R, -1).sum(axis=1)]
    j = pf.pf_jaccard(cuda(S[0]), cuda(S[1]))
    assert j == pytest.approx((aff[0] & aff[1]).sum() / (aff[0] | aff[1]).sum(), rel=1e-15)
    z = np.zeros((H, W), np.uint8)
    assert pf.pf_jaccard(cuda(z), cuda(z)) == 1.0


def test_manhattan_distance_over_a_run(pf, orc):
    """Eq. 12 between two realisations' affected-cell series, stepped through the ABI
    (per-step counts by pf_affected_count, the distance by pf_manhattan on the device)."""
    import torch
    H, W, T = 80, 80, 20
    land = syn.make_landscape(H, W, 5)
    V, th = syn.smooth_wind(H, W, 5, 0, sigma=8.0)
    S0 = np.broadcast_to(syn.initial_state(land, [(40, 40)]), (2, H, W)).copy()
    m = pf.FireModel(H, W, pf.PF_DISCRETE, 2, seed=4)
    set_landscape(m, land, V, th)
    m.set_params(**PRM)
    out = m.forward(cuda(S0), 0)
    series, states = [], []
    for t in range(T):
        out = m.advance(1)
        series.append(pf.pf_affected_count(out))
        states.append(out.clone())
    st = torch.stack(states)  # [T][2][H][W]
    prm = orc.Params(**PRM)
    q = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm)
    S, want = S0, []
    for t in range(T):
        S = orc.step_discrete(S, q, prm.p_continue, 4, t)
        want.append([int(((S[r] == 2) | (S[r] == 3)).sum()) for r in range(2)])
    assert series == want
    assert pf.pf_manhattan(st[:, 0].contiguous(), st[:, 1].contiguous()) == sum(abs(x - y) for x, y in want)


def test_ensemble_mean_against_the_mean_field_form(pf, orc):
    """The probability of arrival of a 512-realisation ensemble equals the oracle's (same
    draws), and the mean-field form equals the oracle's. The two forms are not equal:
    the mean-field form treats neighbours' burning as independent and, near the
    ignition, where they are strongly correlated, overestimates (a cell two rows below
    the ignition: 0.44 in the ensemble, 0.96 mean-field, after 6 steps). They stay
    strongly correlated over the map."""
    H, W, R, T = 64, 64, 512, 6
    land = syn.make_landscape(H, W, 9)
    V, th = syn.uniform_wind(H, W, 5.0, 45.0)
    S0 = syn.initial_state(land, [(32, 32)])
    m = pf.FireModel(H, W, pf.PF_DISCRETE, R, seed=1)
    set_landscape(m, land, V, th)
    m.set_params(**PRM)
    SR = np.broadcast_to(S0, (R, H, W)).copy()
    ens = pf.pf_arrival_probability(m.forward(cuda(SR), T)).cpu().numpy()
    prm = orc.Params(**PRM)
    q = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm)
    So = orc.forward_discrete(SR, q, prm.p_continue, seed=1, T=T)
    assert np.array_equal(ens, ((So == 2) | (So == 3)).sum(axis=0).astype(np.float32) / np.float32(R))
    d = pf.FireModel(H, W, pf.PF_DIFF, 1)
    set_landscape(d, land, V, th)
    d.set_params(**PRM)
    a = d.forward(cuda(S0), T)[0].cpu().numpy().astype(np.float64)
    a_o, _, _ = orc.diff_forward(land, [(V, th)], [0], prm, S0, T, keep_states=False)
    assert np.all(np.abs(a - a_o) <= 1e-4 * a_o + 1e-6)
    assert np.corrcoef(ens.ravel(), a.ravel())[0, 1] > 0.95
    assert a.sum() > ens.sum()
