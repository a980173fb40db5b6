"""GPU parity of the differentiable form and its adjoint against the oracle, through
the C ABI: single steps on random states (1e-5 relative), trajectories (1e-4 relative
after T), and gradients (1e-3 relative) for several checkpoint intervals."""
import numpy as np
import pytest

import synthetic as syn
from tests._util import PRM, cuda, set_landscape

pytestmark = pytest.mark.gpu

STEP_RTOL, STEP_ATOL = 1e-5, 1e-7
RUN_RTOL, RUN_ATOL = 1e-4, 1e-6
GRAD_RTOL = 1e-3


@pytest.fixture(scope="module")
def pf():
    import paper_2502_18738_gb300 as pf
    pf.build()
    pf.load()
    return pf


def _close(got, want, rtol, atol):
    err = np.abs(got - want)
    ok = err <= rtol * np.abs(want) + atol
    if not ok.all():
        bad = np.argwhere(~ok)
        ex = [(tuple(int(v) for v in i), float(got[tuple(i)]), float(want[tuple(i)])) for i in bad[:6]]
        raise AssertionError(f"{len(bad)} of {ok.size} outside tolerance; max err {err.max():.3g}; "
                             f"shape {got.shape}; first (idx, got, want): {ex}")


def _model(pf, orc, land, V, th, H, W, **kw):
    p = {**PRM, **kw}
    m = pf.FireModel(H, W, pf.PF_DIFF)
    set_landscape(m, land, V, th)
    m.set_params(**p)
    return m, orc.Params(**p)


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("H,W", [(33, 47), (64, 64), (1, 50), (50, 1), (150, 260)])
def test_single_step_random_states(pf, orc, H, W, kernel):
    land = syn.make_landscape(H, W, 2)
    V, th = syn.smooth_wind(H, W, 2, 0, sigma=6.0)
    m, prm = _model(pf, orc, land, V, th, H, W)
    m.set_tuning(kernel=kernel)
    S0 = np.where(land.burnable != 0, 1, 0).astype(np.uint8)
    m.forward(cuda(S0), 0)  # sets the burnable mask
    q = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm, burnable=land.burnable)
    a, b = syn.random_diff_state(H, W, 4, land.burnable)
    m.set_state(3, cuda(np.stack([a, b])))
    Pg = m.ignition_map()[0].cpu().numpy()   # p_ignite of the state just set
    out = m.advance(1).cpu().numpy()
    a1, b1, P = orc.step_diff(a, b, q, prm.p_continue, return_P=True)
    _close(out[0], a1, STEP_RTOL, STEP_ATOL)
    _close(out[1], b1, STEP_RTOL, STEP_ATOL)
    _close(Pg, P, STEP_RTOL, STEP_ATOL)


@pytest.mark.parametrize("kernel", [1, 2])
def test_single_step_states_below_the_first_tier_boundary(pf, orc, kernel):
    """States in 8 x 8 blocks scaled by 1e-30 (below 2^-64, so held in the first tier)
    next to ordinary ones: one step against the oracle at the per-step relative tolerance
    with no absolute floor, so the tiny values are checked as closely as the others."""
    H, W = 96, 112
    land = syn.make_landscape(H, W, 12)
    V, th = syn.smooth_wind(H, W, 12, 0, sigma=6.0)
    m, prm = _model(pf, orc, land, V, th, H, W)
    m.set_tuning(kernel=kernel)
    S0 = np.where(land.burnable != 0, 1, 0).astype(np.uint8)
    m.forward(cuda(S0), 0)
    q = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm, burnable=land.burnable)
    a, b = syn.random_diff_state(H, W, 9, land.burnable)
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    tiny = ((rr // 8 + cc // 8) % 3) == 0
    a = np.where(tiny, a * np.float32(1e-30), a).astype(np.float32)
    b = np.where(tiny, b * np.float32(1e-30), b).astype(np.float32)
    m.set_state(0, cuda(np.stack([a, b])))
    Pg = m.ignition_map()[0].cpu().numpy()
    out = m.advance(1).cpu().numpy()
    a1, b1, P = orc.step_diff(a, b, q, prm.p_continue, return_P=True)
    _close(out[0], a1, STEP_RTOL, 1e-40)
    _close(out[1], b1, STEP_RTOL, 1e-40)
    _close(Pg, P, STEP_RTOL, 1e-40)
    assert ((a1 > 0) & (a1 < 2.0 ** -64)).sum() > 100  # some cells stay in the tier


def _problem(H, W, T, seed, n_epochs=2):
    land = syn.make_landscape(H, W, seed)
    winds = [syn.smooth_wind(H, W, seed, e, sigma=8.0) for e in range(n_epochs)]
    starts = [int(round(e * T / n_epochs)) for e in range(n_epochs)]
    S0 = syn.initial_state(land, [(H // 2, W // 2), (H // 4, W // 3)])
    return land, winds, starts, S0


def _set_winds(m, winds, starts):
    for (V, th), s in list(zip(winds, starts))[1:]:
        m.set_wind(cuda(V), cuda(th), s)


@pytest.mark.parametrize("H,W,T,kernel,k", [(96, 80, 60, 1, 0), (200, 170, 120, 1, 0), (96, 80, 60, 2, 3),
                                           (200, 170, 120, 2, 8), (130, 300, 77, 2, 5), (130, 300, 77, 2, 4)])
def test_trajectory(pf, orc, H, W, T, kernel, k):
    land, winds, starts, S0 = _problem(H, W, T, 6)
    m, prm = _model(pf, orc, land, *winds[0], H, W)
    _set_winds(m, winds, starts)
    m.set_tuning(kernel=kernel, k=k)
    out = m.forward(cuda(S0), T).cpu().numpy()
    a, b, tape = orc.diff_forward(land, winds, starts, prm, S0, T)
    # every single step, fed the oracle's state, within the per-step tolerance
    for t in range(0, T, max(1, T // 12)):
        at, bt = tape[t]
        m.set_state(t, cuda(np.stack([at, bt]).astype(np.float32)))
        o1 = m.advance(1).cpu().numpy()
        a1, b1 = tape[t + 1] if t + 1 < T else (a, b)
        # the state fed in is FP32-rounded; compare with the oracle's step from it
        e = orc._epoch_of(t, starts)
        q = orc.prep(H, W, land.E, land.p_veg, land.p_den, *winds[e], prm, burnable=(S0 != 0))
        ra, rb = orc.step_diff(at.astype(np.float32), bt.astype(np.float32), q, prm.p_continue)
        _close(o1[0], ra, STEP_RTOL, STEP_ATOL)
        _close(o1[1], rb, STEP_RTOL, STEP_ATOL)
    _close(out[0], a, RUN_RTOL, RUN_ATOL)
    _close(out[1], b, RUN_RTOL, RUN_ATOL)
    assert a.max() > 0.9 and (a > 0.01).sum() > 100


@pytest.mark.parametrize("K,kernel", [(1, 1), (7, 1), (0, 1), (1, 2), (7, 2), (13, 2)])
def test_gradients_match_oracle(pf, orc, K, kernel):
    import torch
    H, W, T = 72, 64, 48
    land, winds, starts, S0 = _problem(H, W, T, 13)
    m, prm = _model(pf, orc, land, *winds[0], H, W)
    _set_winds(m, winds, starts)
    m.set_tuning(K=K, kernel=kernel)
    y = (orc.forward_discrete(S0, orc.prep(H, W, land.E, land.p_veg, land.p_den, *winds[0],
                                            orc.Params(0.5, 0.05, 0.12, 0.08, 0.3)),
                              0.3, seed=2, T=T) >= 2).astype(np.float32)
    out = m.forward(cuda(S0), T)
    a_T = out[0].contiguous()
    g_a = torch.empty_like(a_T)
    loss = pf.pf_loss_bce(a_T, cuda(y), g_a)
    g_b = cuda(np.random.default_rng(0).standard_normal((H, W)).astype(np.float32) * 1e-3)
    g4, gpv, gpd = m.backward(g_a, g_b)
    # oracle
    a, b, tape = orc.diff_forward(land, winds, starts, prm, S0, T)
    L, gA = orc.bce(a, y)
    assert loss == pytest.approx(L, rel=1e-5)
    want4, wpv, wpd = orc.diff_backward(land, winds, starts, prm, S0, tape, gA, g_b.cpu().numpy().astype(np.float64))
    for k in range(4):
        assert g4[k] == pytest.approx(want4[k], rel=GRAD_RTOL), k
    for got, want in ((gpv.cpu().numpy(), wpv), (gpd.cpu().numpy(), wpd)):
        scale = np.abs(want).max()
        assert np.all(np.abs(got - want) <= GRAD_RTOL * np.abs(want) + 1e-6 * scale)


def test_gradient_reduction_is_deterministic(pf, orc):
    import torch
    H, W, T = 60, 70, 30
    land, winds, starts, S0 = _problem(H, W, T, 17)
    m, prm = _model(pf, orc, land, *winds[0], H, W)
    _set_winds(m, winds, starts)
    m.set_tuning(K=5)
    res = []
    for _ in range(2):
        out = m.forward(cuda(S0), T)
        g = torch.ones((H, W), device="cuda") * 1e-3
        res.append(m.backward(g, None)[0])
    assert res[0] == res[1]


def test_autograd_function(pf, orc):
    import torch
    H, W, T = 40, 44, 20
    land, winds, starts, S0 = _problem(H, W, T, 19, n_epochs=1)
    m = pf.FireModel(H, W, pf.PF_DIFF)
    V, th = winds[0]
    params = torch.tensor([PRM["p_h"], PRM["c1"], PRM["c2"], PRM["a"]], dtype=torch.float64, requires_grad=True)
    pv = cuda(land.p_veg).requires_grad_(True)
    pd = cuda(land.p_den).requires_grad_(True)
    a_T, b_T = pf.DiffFire.apply(m, cuda(S0), T, params, pv, pd, PRM["p_continue"], PRM["l"],
                                 cuda(land.E), cuda(V), cuda(th))
    (a_T.sum() + 0.5 * b_T.sum()).backward()
    prm = orc.Params(**PRM)
    a, b, tape = orc.diff_forward(land, winds, starts, prm, S0, T)
    g4, gpv, gpd = orc.diff_backward(land, winds, starts, prm, S0, tape, np.ones((H, W)), 0.5 * np.ones((H, W)))
    assert np.allclose(params.grad.numpy(), g4, rtol=GRAD_RTOL)
    assert np.allclose(pv.grad.cpu().numpy(), gpv, rtol=GRAD_RTOL, atol=1e-5 * np.abs(gpv).max())


@pytest.mark.parametrize("k", [4, 8])
def test_quiescent_tiles_are_skipped_exactly(pf, orc, k):
    """A fire in one corner of a 600 x 500 grid: most blocked-kernel tiles are quiescent
    (forward: b = 0 in the whole region; adjoint: a = 0 in the whole region) for most
    steps and are skipped. The forward must equal the plain kernel's bit for bit, the
    gradients must equal the plain adjoint's within rounding, and the skipped counts
    must be positive and below the totals."""
    import torch
    H, W, T = 600, 500, 40
    land = syn.make_landscape(H, W, 21)
    V, th = syn.smooth_wind(H, W, 21, 0, sigma=8.0)
    S0 = syn.initial_state(land, [(20, 30), (35, 12)])
    runs = {}
    for kernel in (1, 2):
        m, prm = _model(pf, orc, land, V, th, H, W)
        m.set_tuning(kernel=kernel, k=k, K=9, profile=1)
        pf.pf_profile_read(m.h, reset=True)
        out = m.forward(cuda(S0), T)
        g_a = cuda(np.random.default_rng(1).standard_normal((H, W)).astype(np.float32) * 1e-3)
        g4, gpv, gpd = m.backward(g_a, None)
        runs[kernel] = (out.cpu().numpy(), g4, gpv.cpu().numpy(), pf.pf_profile_read(m.h))
        m.close()
    (o1, g1, pv1, _), (o2, g2, pv2, prof) = runs[1], runs[2]
    assert np.array_equal(o1, o2)
    for a, b in zip(g1, g2):
        assert a == pytest.approx(b, rel=1e-5)
    _close(pv2, pv1, 1e-4, 1e-6 * np.abs(pv1).max())
    for kind in ("diff_blocked", "adjoint_blocked"):
        launches, cell_steps, _, skipped = prof[kind]
        assert launches > 0 and 0 < skipped < cell_steps, (kind, prof[kind])


@pytest.mark.parametrize("K,k", [(8, 8), (11, 8), (15, 6), (22, 8)])
def test_blocked_gradients_equal_plain_with_checkpoint_segments(pf, orc, K, k):
    """Segments of K steps with wind epochs at odd steps: the blocked path (recompute in
    chunks aligned with the adjoint's launches, frozen and void tiles, recorded tile
    activity) gives the plain path's gradients; the forward states are identical."""
    import torch
    H, W, T = 420, 380, 123
    land = syn.make_landscape(H, W, 31)
    winds = [syn.smooth_wind(H, W, 31, e, sigma=8.0) for e in range(3)]
    starts = [0, 37, 90]
    S0 = syn.initial_state(land, [(60, 70), (300, 250)])
    w = cuda(np.random.default_rng(5).standard_normal((H, W)).astype(np.float32) * 1e-3)
    res = {}
    for kernel in (1, 2):
        m, prm = _model(pf, orc, land, *winds[0], H, W)
        _set_winds(m, winds, starts)
        m.set_tuning(kernel=kernel, k=k, K=K)
        out = m.forward(cuda(S0), T).cpu().numpy()
        g4, gpv, gpd = m.backward(w, None)
        res[kernel] = (out, g4, gpv.cpu().numpy())
        m.close()
    assert np.array_equal(res[1][0], res[2][0])
    for a, b in zip(res[1][1], res[2][1]):
        assert a == pytest.approx(b, rel=2e-5)
    _close(res[2][2], res[1][2], 1e-4, 1e-6 * np.abs(res[1][2]).max())


@pytest.mark.parametrize("H,W,T,kernel", [(1, 1, 3, 2), (1, 70, 9, 2), (70, 1, 9, 1), (5, 5, 0, 2), (130, 97, 1, 2)])
def test_degenerate_shapes_and_steps(pf, orc, H, W, T, kernel):
    """Single cells, single rows / columns, T = 0 and T = 1: forward and gradients equal
    the oracle's (T = 0: the gradient is zero)."""
    import torch
    land = syn.make_landscape(H, W, 17)
    V, th = syn.smooth_wind(H, W, 17, 0, sigma=4.0)
    S0 = syn.initial_state(land, [(H // 2, W // 2)])
    m, prm = _model(pf, orc, land, V, th, H, W)
    m.set_tuning(kernel=kernel)
    out = m.forward(cuda(S0), T).cpu().numpy()
    a, b, tape = orc.diff_forward(land, [(V, th)], [0], prm, S0, T)
    _close(out[0].astype(np.float64), a, RUN_RTOL, RUN_ATOL)
    _close(out[1].astype(np.float64), b, RUN_RTOL, RUN_ATOL)
    w = np.random.default_rng(1).standard_normal((H, W))
    g4, gpv, gpd = m.backward(cuda(w.astype(np.float32)), None)
    want4, wpv, wpd = orc.diff_backward(land, [(V, th)], [0], prm, S0, tape, w.astype(np.float32).astype(np.float64),
                                        np.zeros((H, W)))
    if T == 0:
        assert not any(g4) and not gpv.any()
    for k in range(4):
        assert g4[k] == pytest.approx(want4[k], rel=GRAD_RTOL, abs=1e-12)


def test_checkpoint_slots_reused_by_a_different_run(pf, orc):
    """A context keeps its checkpoint slots from run to run and writes an all-zero tile
    into a slot only where that slot may hold nonzeros: a second run whose fires lie
    elsewhere (tiles burned in the first run are zero now, and the reverse) gives the
    gradients and states of the same run on a fresh context, bit for bit."""
    import torch
    H, W, T, K = 300, 340, 70, 9
    land = syn.make_landscape(H, W, 41)
    V, th = syn.smooth_wind(H, W, 41, 0, sigma=8.0)
    S_a = syn.initial_state(land, [(60, 60), (240, 280)])
    S_b = syn.initial_state(land, [(150, 170), (60, 280)])
    w = cuda(np.random.default_rng(3).standard_normal((H, W)).astype(np.float32) * 1e-3)
    m, _ = _model(pf, orc, land, V, th, H, W)
    m.set_tuning(kernel=2, k=8, K=K)
    m.forward(cuda(S_a), T)
    m.backward(w, None)
    out = m.forward(cuda(S_b), T).cpu().numpy()
    g4, gpv, _ = m.backward(w, None)
    f, _ = _model(pf, orc, land, V, th, H, W)
    f.set_tuning(kernel=2, k=8, K=K)
    out_f = f.forward(cuda(S_b), T).cpu().numpy()
    g4_f, gpv_f, _ = f.backward(w, None)
    assert np.array_equal(out, out_f)
    assert list(g4) == list(g4_f)
    assert torch.equal(gpv, gpv_f)


@pytest.mark.parametrize("K,k", [(7, 8), (13, 8), (22, 6)])
def test_tile_tape_gives_the_recomputed_gradients(pf, orc, K, k):
    """With checkpoints, the backward copies each segment's states from the tile tape the
    forward kept (pf_tuning.tape 0) instead of recomputing them (tape 1): the states are
    the same bits, so the gradients are identical; the tape was used."""
    H, W, T = 300, 340, 90
    land = syn.make_landscape(H, W, 43)
    winds = [syn.smooth_wind(H, W, 43, e, sigma=8.0) for e in range(2)]
    starts = [0, 41]
    S0 = syn.initial_state(land, [(70, 80), (220, 250)])
    w = cuda(np.random.default_rng(7).standard_normal((H, W)).astype(np.float32) * 1e-3)
    res = {}
    for tape in (0, 1):
        m, _ = _model(pf, orc, land, *winds[0], H, W)
        _set_winds(m, winds, starts)
        m.set_tuning(kernel=2, k=k, K=K, tape=tape, profile=1)
        pf.pf_profile_read(m.h, reset=True)
        out = m.forward(cuda(S0), T).cpu().numpy()
        g4, gpv, _ = m.backward(w, None)
        prof = pf.pf_profile_read(m.h, reset=True)
        mem = pf.pf_memory_stats(m.h)
        res[tape] = (out, list(g4), gpv.cpu().numpy(), prof.get("segment_from_tape", (0,))[0], mem)
        m.close()
    assert res[0][3] > 0 and res[1][3] == 0
    # the tape held every launch of the forward (a few MB at this size); none without it
    mem0, mem1 = res[0][4], res[1][4]
    assert mem0["tape_launches"] > 0 and mem0["tape_recorded"] == mem0["tape_launches"]
    assert 0 < mem0["tape_used_bytes"] <= mem0["tape_bytes"] and mem0["tape_short"] == 0
    assert mem1["tape_bytes"] == 0 and mem1["tape_launches"] == 0
    assert mem0["K"] == mem1["K"] == K and mem0["segment_bytes"] >= (K - 1) * 2 * H * W * 4
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]
    assert np.array_equal(res[0][2], res[1][2])


def test_tile_tape_that_runs_short_gives_the_recomputed_gradients(pf, orc, monkeypatch):
    """A tile tape too small for the whole forward (capped with PF_TAPE_MAX_BLOCKS)
    records the launches that fit; the backward copies those from it and recomputes
    the others, some segments mixing both, with the same bits as a run without a tape."""
    H, W, T, K, k = 300, 340, 90, 13, 8
    land = syn.make_landscape(H, W, 43)
    winds = [syn.smooth_wind(H, W, 43, e, sigma=8.0) for e in range(2)]
    starts = [0, 41]
    S0 = syn.initial_state(land, [(70, 80), (220, 250)])
    w = cuda(np.random.default_rng(7).standard_normal((H, W)).astype(np.float32) * 1e-3)

    def run(tape, cap=None):
        if cap is None:
            monkeypatch.delenv("PF_TAPE_MAX_BLOCKS", raising=False)
        else:
            monkeypatch.setenv("PF_TAPE_MAX_BLOCKS", str(cap))
        m, _ = _model(pf, orc, land, *winds[0], H, W)
        _set_winds(m, winds, starts)
        m.set_tuning(kernel=2, k=k, K=K, tape=tape, profile=1)
        pf.pf_profile_read(m.h, reset=True)
        out = m.forward(cuda(S0), T).cpu().numpy()
        g4, gpv, _ = m.backward(w, None)
        prof = pf.pf_profile_read(m.h, reset=True)
        mem = pf.pf_memory_stats(m.h)
        m.close()
        return out, list(g4), gpv.cpu().numpy(), prof, mem

    full = run(0)
    blk = 2 * 48 * 48 * 4
    need = full[4]["tape_used_bytes"] // blk
    tiles = ((340 + 15) // 16 * 16 + 47) // 48 * ((H + 47) // 48)
    cap = max(tiles, need // 2)
    assert cap < need
    short = run(0, cap)
    ref = run(1)
    monkeypatch.delenv("PF_TAPE_MAX_BLOCKS", raising=False)
    mem = short[4]
    assert mem["tape_short"] == 1 and 0 < mem["tape_recorded"] < mem["tape_launches"]
    assert mem["tape_used_bytes"] <= cap * blk
    # both kinds of segment launch ran: copies from the tape and recomputes
    assert short[3].get("segment_from_tape", (0,))[0] > 0
    assert short[3]["diff_blocked"][0] > full[3]["diff_blocked"][0]
    for got in (short, full):
        assert np.array_equal(got[0], ref[0])
        assert got[1] == ref[1]
        assert np.array_equal(got[2], ref[2])
