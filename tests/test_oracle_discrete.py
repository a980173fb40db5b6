"""Pins of the oracle's discrete step (Sec. 2.2 rules, Eq. 9): closed forms,
invariants, and Monte-Carlo frequencies against brute-force enumeration."""
import numpy as np
import pytest

import synthetic as syn

PRM = dict(p_h=0.58, c1=0.045, c2=0.131, a=0.078, p_continue=0.3, l=30.0)


def _land_q(orc, H, W, seed=0, V=5.0, th=45.0, **kw):
    land = syn.make_landscape(H, W, seed)
    prm = orc.Params(**{**PRM, **kw})
    Vw, tw = syn.uniform_wind(H, W, V, th)
    q = orc.prep(H, W, land.E, land.p_veg, land.p_den, Vw, tw, prm)
    return land, prm, q


def test_single_burning_neighbour_gives_p_equal_q(orc):
    land, prm, q = _land_q(orc, 5, 6)
    S = np.ones((5, 6), np.uint8)
    S[2, 3] = 2
    _, P, _ = orc.step_discrete(S, q, prm.p_continue, seed=0, step=0, return_P=True)
    # receiving cell (2,2) sees the burning cell at offset (0, +1): direction 4
    assert P[2, 2] == pytest.approx(q[4, 2, 2], abs=1e-15)
    # (1, 2) sees it at offset (+1, +1): direction 7
    assert P[1, 2] == pytest.approx(q[7, 1, 2], abs=1e-15)
    assert P[0, 0] == 0.0


def test_two_neighbours_inclusion_exclusion(orc):
    land, prm, q = _land_q(orc, 4, 4)
    S = np.ones((4, 4), np.uint8)
    S[1, 1] = 2
    S[1, 3] = 2
    _, P, _ = orc.step_discrete(S, q, prm.p_continue, 0, 0, return_P=True)
    q1, q2 = q[3, 1, 2], q[4, 1, 2]   # (1,2) sees (1,1) at (0,-1) and (1,3) at (0,+1)
    assert P[1, 2] == pytest.approx(q1 + q2 - q1 * q2, abs=1e-15)


def test_draws_decide_cells(orc):
    land, prm, q = _land_q(orc, 16, 16)
    S = syn.random_state(16, 16, seed=3)
    Sn, P, u = orc.step_discrete(S, q, prm.p_continue, seed=9, step=4, run0=2, fire=1, return_P=True)
    for r in range(16):
        for c in range(16):
            u0, u1 = orc.cell_draws(9, 2, 4, 1, r * 16 + c)
            if S[r, c] == 1:
                assert u[r, c] == u0
                assert Sn[r, c] == (2 if np.float32(u0) < np.float32(P[r, c]) else 1)
            elif S[r, c] == 2:
                assert u[r, c] == u1
                assert Sn[r, c] == (2 if np.float32(u1) < np.float32(prm.p_continue) else 3)
            else:
                assert Sn[r, c] == S[r, c]


@pytest.mark.parametrize("pc", [0.0, 0.3, 1.0])
def test_invariants_over_a_run(orc, pc):
    H, W, T = 40, 36, 30
    land, prm, q = _land_q(orc, H, W, seed=1, p_continue=pc)
    S = syn.initial_state(land, [(H // 2, W // 2), (5, 7)])
    states, Ps, us = orc.trajectory_discrete(S, q, prm.p_continue, seed=5, T=T)
    burn_len = np.zeros((H, W), int)
    for t in range(T):
        a, b = states[t], states[t + 1]
        assert np.all(b[a == 0] == 0)                     # non-burnable never changes
        assert np.all(b[a == 3] == 3)                     # burned is absorbing
        assert np.all(np.isin(b[a == 2], [2, 3]))         # burning stays or burns out
        assert np.all(np.isin(b[a == 1], [1, 2]))
        # no ignition without a burning neighbour at the previous step
        burning = np.pad(a == 2, 1)
        nb = np.zeros_like(a, dtype=bool)
        for dr in (-1, 0, 1):
            for dc in (-1, 0, 1):
                if dr or dc:
                    nb |= burning[1 + dr:1 + dr + H, 1 + dc:1 + dc + W]
        assert not np.any((a == 1) & (b == 2) & ~nb)
        burn_len += (a == 2)
        if pc == 1.0:
            assert not np.any((a == 2) & (b == 3))
    if pc == 0.0:
        ever = states[-1] == 3
        assert np.all(burn_len[ever] == 1)
        assert np.all(burn_len <= 1)


@pytest.mark.parametrize("case", ["3x3_T3", "3x4_T2_pc0", "2x5_T4"])
def test_monte_carlo_matches_enumeration(orc, case):
    from oracle import enumeration as en
    if case == "3x3_T3":
        H, W, T, pc, ign = 3, 3, 3, 0.3, [(1, 1)]
    elif case == "3x4_T2_pc0":
        H, W, T, pc, ign = 3, 4, 2, 0.0, [(0, 0), (2, 3)]
    else:
        H, W, T, pc, ign = 2, 5, 4, 0.6, [(0, 2)]
    land, prm, q = _land_q(orc, H, W, seed=11, V=6.0, th=120.0, p_continue=pc)
    S0 = syn.initial_state(land, ign)
    exact = en.marginals(en.distribution(S0, q, prm.p_continue, T), (H, W))
    R = 100000
    out = orc.forward_discrete(np.broadcast_to(S0, (R, H, W)).copy(), q, prm.p_continue, seed=123, T=T)
    for s in range(4):
        f = (out == s).mean(axis=0)
        p = exact[s]
        se = np.sqrt(np.maximum(p * (1 - p), 1e-12) / R)
        z = np.abs(f - p) / se
        assert np.all((z < 5) | (np.abs(f - p) < 1e-12)), (s, f, p)
