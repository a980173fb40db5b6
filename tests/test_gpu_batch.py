"""Batched fires (pf_batch_submit): many independent fires of uneven size and step
count from one device work queue. Each fire must come out exactly as a context of its
own computes it (pf_forward) and as the oracle computes it (Sec. 2.2, Eq. 9, with the
fire's own Philox counter words)."""
import os

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


def _fire(H, W, seed, n_ign=2):
    land = syn.make_landscape(H, W, seed)
    V, th = syn.smooth_wind(H, W, seed, 0, sigma=6.0)
    rng = np.random.default_rng(seed)
    ign = [(int(rng.integers(H)), int(rng.integers(W))) for _ in range(n_ign)]
    return land, V, th, syn.initial_state(land, ign)


def _job(pf, land, V, th, S0, T, form, **kw):
    p = {**PRM, **{k: v for k, v in kw.items() if k in PRM}}
    extra = {k: v for k, v in kw.items() if k not in PRM}
    return pf.make_job(cuda(S0), T, form=form, E=cuda(land.E), p_veg=cuda(land.p_veg), p_den=cuda(land.p_den),
                       V_w=cuda(V), theta_w=cuda(th), **p, **extra)


# (H, W, T): several tiles with ragged edges, single rows / columns, T = 0, T not a
# multiple of the steps per work item, one fire much longer than the rest
SHAPES = [(45, 77, 37), (128, 128, 200), (1, 40, 9), (40, 1, 6), (33, 200, 0), (300, 129, 50), (64, 64, 4),
          (97, 65, 5)]


def test_discrete_batch_equals_per_fire_contexts(pf):
    seed = 0x0123456789ABCDEF
    jobs, keep, want = [], [], []
    for i, (H, W, T) in enumerate(SHAPES):
        land, V, th, S0 = _fire(H, W, 100 + i)
        m = pf.FireModel(H, W, 0, 1, seed=seed)
        set_landscape(m, land, V, th)
        m.set_params(**PRM)
        want.append(m.forward(cuda(S0), T).cpu().numpy()[0])
        m.close()
        j, out = _job(pf, land, V, th, S0, T, 0, seed=seed)
        jobs.append(j)
        keep.append((S0, out))
    pf.pf_batch_submit(jobs)
    spread = 0
    for (S0, out), w in zip(keep, want):
        got = out.cpu().numpy()
        assert np.array_equal(got, w)
        spread += int((got >= 2).sum() - (S0 >= 2).sum())
    assert spread > 100  # the fires did spread


def test_discrete_batch_matches_oracle_with_fire_and_run_words(pf, orc):
    seed = 77
    prm = orc.Params(**PRM)
    jobs, keep = [], []
    for i, (H, W, T) in enumerate(SHAPES[:6]):
        land, V, th, S0 = _fire(H, W, 200 + i)
        q = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm)
        run, fire = 3 * i + 1, 1000 + i
        ref = orc.forward_discrete(S0, q, prm.p_continue, seed=seed, T=T, run0=run, fire=fire)
        j, out = _job(pf, land, V, th, S0, T, 0, seed=seed, run=run, fire_id=fire)
        jobs.append(j)
        keep.append((out, ref))
    pf.pf_batch_submit(jobs)
    for out, ref in keep:
        assert np.array_equal(out.cpu().numpy(), ref)


def test_same_fire_different_fire_id_differs(pf):
    H, W, T = 96, 96, 60
    land, V, th, S0 = _fire(H, W, 5, n_ign=4)
    j0, o0 = _job(pf, land, V, th, S0, T, 0, seed=9, fire_id=0)
    j1, o1 = _job(pf, land, V, th, S0, T, 0, seed=9, fire_id=1)
    j2, o2 = _job(pf, land, V, th, S0, T, 0, seed=9, fire_id=0)
    pf.pf_batch_submit([j0, j1, j2])
    assert np.array_equal(o0.cpu().numpy(), o2.cpu().numpy())
    assert not np.array_equal(o0.cpu().numpy(), o1.cpu().numpy())


def test_diff_batch_equals_per_fire_contexts_and_oracle(pf, orc):
    prm = orc.Params(**PRM)
    jobs, keep = [], []
    for i, (H, W, T) in enumerate([(45, 77, 37), (1, 40, 9), (130, 70, 61), (33, 200, 0), (64, 64, 4)]):
        land, V, th, S0 = _fire(H, W, 300 + i)
        m = pf.FireModel(H, W, 1, 1)
        set_landscape(m, land, V, th)
        m.set_params(**PRM)
        m.set_tuning(kernel=1)
        plain = m.forward(cuda(S0), T).cpu().numpy()
        m.close()
        a, b, _ = orc.diff_forward(land, [(V, th)], [0], prm, S0, T, keep_states=False)
        j, out = _job(pf, land, V, th, S0, T, 1)
        jobs.append(j)
        keep.append((out, plain, a, b))
    pf.pf_batch_submit(jobs)
    for out, plain, a, b in keep:
        got = out.cpu().numpy()
        assert np.array_equal(got, plain)
        assert np.max(np.abs(got[0] - a)) < 1e-4 and np.max(np.abs(got[1] - b)) < 1e-4


def test_mixed_forms_in_one_submit(pf, orc):
    prm = orc.Params(**PRM)
    H, W, T = 70, 90, 23
    land, V, th, S0 = _fire(H, W, 11)
    q = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm)
    jd, od = _job(pf, land, V, th, S0, T, 0, seed=5, fire_id=2)
    jc, oc = _job(pf, land, V, th, S0, T + 9, 1)
    pf.pf_batch_submit([jd, jc])
    assert np.array_equal(od.cpu().numpy(), orc.forward_discrete(S0, q, prm.p_continue, seed=5, T=T, fire=2))
    a, b, _ = orc.diff_forward(land, [(V, th)], [0], prm, S0, T + 9, keep_states=False)
    got = oc.cpu().numpy()
    assert np.max(np.abs(got[0] - a)) < 1e-4 and np.max(np.abs(got[1] - b)) < 1e-4


def test_many_small_fires(pf, orc):
    """More work items than resident CTAs, fires of 1..3 tiles with 1..40 steps."""
    prm = orc.Params(**PRM)
    rng = np.random.default_rng(1)
    jobs, keep = [], []
    for i in range(300):
        H, W, T = int(rng.integers(1, 70)), int(rng.integers(1, 140)), int(rng.integers(0, 41))
        land, V, th, S0 = _fire(H, W, 1000 + i, n_ign=1)
        j, out = _job(pf, land, V, th, S0, T, 0, seed=4, fire_id=i)
        jobs.append(j)
        keep.append((out, land, V, th, S0, T, i))
    pf.pf_batch_submit(jobs)
    for out, land, V, th, S0, T, i in keep[::15]:
        q = orc.prep(*S0.shape, land.E, land.p_veg, land.p_den, V, th, prm)
        assert np.array_equal(out.cpu().numpy(), orc.forward_discrete(S0, q, prm.p_continue, seed=4, T=T, fire=i))


def test_empty_and_invalid_batches(pf):
    import torch
    pf.pf_batch_submit([])
    H, W = 8, 8
    land, V, th, S0 = _fire(H, W, 1)
    bad = S0.copy()
    bad[3, 3] = 9
    j, _ = _job(pf, land, V, th, bad, 5, 0)
    with pytest.raises(pf.PFireError) as e:
        pf.pf_batch_submit([j])
    assert e.value.code == pf.PF_EINVAL
    j, _ = _job(pf, land, V, th, S0, 5, 0, p_continue=1.5)
    with pytest.raises(pf.PFireError) as e:
        pf.pf_batch_submit([j])
    assert e.value.code == pf.PF_EINVAL
    nan = torch.full((H, W), float("nan"), device="cuda")
    j, _ = pf.make_job(cuda(S0), 5, E=nan)
    with pytest.raises(pf.PFireError) as e:
        pf.pf_batch_submit([j])
    assert e.value.code == pf.PF_EINVAL
    j, _ = _job(pf, land, V, th, S0, -1, 0)
    with pytest.raises(pf.PFireError):
        pf.pf_batch_submit([j])


def test_bounded_wait_times_out_and_library_stays_usable(pf, monkeypatch):
    """A tile that never publishes its generation (a test hook withholds it): its
    neighbours' bounded waits run out, the submit returns PF_ETIMEOUT, and the next
    submit on the same device works."""
    H, W, T = 100, 200, 20
    land, V, th, S0 = _fire(H, W, 3)
    monkeypatch.setenv("PF_BATCH_TEST_WITHHOLD", "1")
    monkeypatch.setenv("PF_BATCH_WAIT_NS", "2000000")
    j, _ = _job(pf, land, V, th, S0, T, 0)
    with pytest.raises(pf.PFireError) as e:
        pf.pf_batch_submit([j])
    assert e.value.code == pf.PF_ETIMEOUT
    monkeypatch.delenv("PF_BATCH_TEST_WITHHOLD")
    monkeypatch.delenv("PF_BATCH_WAIT_NS")
    j, out = _job(pf, land, V, th, S0, T, 0)
    pf.pf_batch_submit([j])
    m = pf.FireModel(H, W, 0, 1)
    set_landscape(m, land, V, th)
    m.set_params(**PRM)
    assert np.array_equal(out.cpu().numpy(), m.forward(cuda(S0), T).cpu().numpy()[0])


def test_batched_adjoint_matches_per_fire_backward_and_oracle(pf, orc):
    """Differentiable jobs with dL/da_T in a submit that also holds discrete fires: the
    batched adjoint (reverse-time work queue) gives the gradients a per-fire context
    computes with the plain kernels, and the oracle's."""
    import torch
    prm = orc.Params(**PRM)
    shapes = [(45, 77, 37), (100, 70, 23), (33, 40, 0), (64, 64, 4), (90, 130, 30)]
    jobs, keep = [], []
    for i, (H, W, T) in enumerate(shapes):
        land, V, th, S0 = _fire(H, W, 400 + i)
        w = torch.from_numpy(np.random.default_rng(i).standard_normal((H, W)).astype(np.float32) * 1e-2).cuda()
        gpv = torch.empty((H, W), dtype=torch.float32, device="cuda")
        gpd = torch.empty_like(gpv)
        j, out = _job(pf, land, V, th, S0, T, 1, dL_da=w, grad_pveg=gpv, grad_pden=gpd)
        jobs.append(j)
        keep.append((land, V, th, S0, T, w, j, gpv, gpd))
        jd, _ = _job(pf, land, V, th, S0, T + 3, 0, seed=2, fire_id=i)
        jobs.append(jd)
    pf.pf_batch_submit(jobs)
    for land, V, th, S0, T, w, j, gpv, gpd in keep:
        H, W = S0.shape
        g4 = j.grads.cpu().numpy()
        m = pf.FireModel(H, W, 1, 1)
        set_landscape(m, land, V, th)
        m.set_params(**PRM)
        m.set_tuning(kernel=1, K=1)
        m.forward(cuda(S0), T)
        r4, rpv, rpd = m.backward(w, None)
        m.close()
        assert np.allclose(g4, r4, rtol=1e-6, atol=1e-12), (T, g4, r4)
        assert np.allclose(gpv.cpu().numpy(), rpv.cpu().numpy(), rtol=1e-5, atol=1e-9)
        if T == 0:
            assert not g4.any()
            continue
        a, b, tape = orc.diff_forward(land, [(V, th)], [0], prm, S0, T)
        want4, wpv, _ = orc.diff_backward(land, [(V, th)], [0], prm, S0, tape, w.cpu().numpy().astype(np.float64),
                                          np.zeros((H, W)))
        for k in range(4):
            assert g4[k] == pytest.approx(want4[k], rel=1e-3, abs=1e-9)


@pytest.mark.parametrize("direct_cells", [0, 5000, 1 << 40])
def test_direct_and_queued_jobs_give_the_same_results(pf, orc, direct_cells):
    """pf_batch_submit runs jobs of at least pf_batch_set_direct_cells cells through
    contexts of their own and the rest through the persistent queue: with every job
    direct (0), a split (5000 cells) or none (2^40), the discrete fires equal the
    oracle's (their own fire_id and run words), the differentiable forwards equal the
    oracle's within the trajectory tolerance and one another bit for bit, and the
    gradients equal the oracle's (1e-3)."""
    import torch
    prm = orc.Params(**PRM)
    shapes = [(45, 77, 37), (100, 70, 23), (33, 40, 9), (90, 130, 30)]
    jobs, disc, diff = [], [], []
    for i, (H, W, T) in enumerate(shapes):
        land, V, th, S0 = _fire(H, W, 500 + i)
        q = orc.prep(H, W, land.E, land.p_veg, land.p_den, V, th, prm)
        jd, od = _job(pf, land, V, th, S0, T, 0, seed=13, run=2 + i, fire_id=40 + i)
        jobs.append(jd)
        disc.append((od, orc.forward_discrete(S0, q, prm.p_continue, seed=13, T=T, run0=2 + i, fire=40 + i)))
        w = torch.from_numpy(np.random.default_rng(i).standard_normal((H, W)).astype(np.float32) * 1e-2).cuda()
        jc, oc = _job(pf, land, V, th, S0, T, 1, dL_da=w)
        jobs.append(jc)
        diff.append((oc, jc, land, V, th, S0, T, w))
    try:
        pf.pf_batch_set_direct_cells(direct_cells)
        pf.pf_batch_submit(jobs)
        st = pf.pf_batch_last_stats()
    finally:
        pf.pf_batch_set_direct_cells(1 << 18)
    n_direct = sum(1 for H, W, _ in shapes if H * W >= direct_cells) * 2
    assert st["direct_jobs"] == n_direct
    for od, ref in disc:
        assert np.array_equal(od.cpu().numpy(), ref)
    for oc, jc, land, V, th, S0, T, w in diff:
        H, W = S0.shape
        m = pf.FireModel(H, W, 1, 1)
        set_landscape(m, land, V, th)
        m.set_params(**PRM)
        m.set_tuning(kernel=1)
        assert np.array_equal(oc.cpu().numpy(), m.forward(cuda(S0), T).cpu().numpy())
        m.close()
        a, b, tape = orc.diff_forward(land, [(V, th)], [0], prm, S0, T)
        got = oc.cpu().numpy()
        assert np.max(np.abs(got[0] - a)) < 1e-4 and np.max(np.abs(got[1] - b)) < 1e-4
        want4, _, _ = orc.diff_backward(land, [(V, th)], [0], prm, S0, tape, w.cpu().numpy().astype(np.float64),
                                        np.zeros((H, W)))
        g4 = jc.grads.cpu().numpy()
        for k in range(4):
            assert g4[k] == pytest.approx(want4[k], rel=1e-3, abs=1e-9)


def test_direct_cells_is_validated(pf):
    with pytest.raises(pf.PFireError) as e:
        pf.pf_batch_set_direct_cells(-1)
    assert e.value.code == pf.PF_EINVAL
