"""Wind epochs streamed from host memory (pf_set_wind_async) against the synchronous
pf_set_wind: the same kernels read the same values, so states and gradients must agree
bit for bit, for pinned and pageable host buffers and device buffers, across repeated
set_env cycles (buffer reuse); invalid values are reported by the next pf_wait."""
import numpy as np
import pytest

import synthetic as syn
from tests._util import PRM, cuda, set_landscape

pytestmark = pytest.mark.gpu

H, W, T, EPOCH = 150, 260, 64, 13


@pytest.fixture(scope="module")
def pf():
    import paper_2502_18738_gb300 as pf
    pf.build()
    pf.load()
    return pf


def _inputs(seed=4):
    land = syn.make_landscape(H, W, seed)
    winds = [syn.smooth_wind(H, W, seed, e, sigma=6.0) for e in range(T // EPOCH + 1)]
    S0 = syn.initial_state(land, [(H // 2, W // 3), (30, 200)])
    y = np.zeros((H, W), np.float32)
    y[40:110, 60:220] = 1.0
    return land, winds, S0, y


def _host(x, pinned):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    return t.pin_memory() if pinned else t.clone()


def _run(pf, m, S0, y, backward=True):
    import torch
    out = torch.empty((2, H, W), dtype=torch.float32, device="cuda")
    pf.pf_forward(m.h, cuda(S0), T, out)
    if not backward:
        return out.cpu().numpy(), None
    g_a = torch.empty((H, W), dtype=torch.float32, device="cuda")
    pf.pf_loss_bce(out[0], cuda(y), g_a, want_loss=False)
    g, gpv, gpd = m.backward(g_a, None)
    return out.cpu().numpy(), (np.asarray(g), gpv.cpu().numpy(), gpd.cpu().numpy())


def _sync_model(pf, land, winds):
    m = pf.FireModel(H, W, pf.PF_DIFF)
    set_landscape(m, land, *winds[0])
    for e, (V, th) in enumerate(winds[1:], start=1):
        m.set_wind(cuda(V), cuda(th), e * EPOCH)
    m.set_params(**PRM)
    return m


def _same(a, b):
    out_a, g_a = a
    out_b, g_b = b
    assert np.array_equal(out_a, out_b)
    if g_a is not None:
        for x, z in zip(g_a, g_b):
            assert np.array_equal(x, z)


@pytest.mark.parametrize("where", ["pinned", "pageable", "device"])
def test_async_epochs_equal_synchronous_ones(pf, where):
    land, winds, S0, y = _inputs()
    ref = _run(pf, _sync_model(pf, land, winds), S0, y)
    m = pf.FireModel(H, W, pf.PF_DIFF)
    m.set_params(**PRM)
    # three cycles of set_env + uploads: the later ones reuse the released epoch buffers
    for cycle in range(3):
        set_landscape(m, land, *winds[0])
        for e, (V, th) in enumerate(winds[1:], start=1):
            if where == "device":
                Vt, tht = cuda(V), cuda(th)
            else:
                Vt, tht = _host(V, where == "pinned"), _host(th, where == "pinned")
            m.set_wind_async(Vt, tht, e * EPOCH)
        _same(_run(pf, m, S0, y), ref)


def test_async_epochs_discrete_form(pf):
    import torch
    land, winds, S0, _ = _inputs(7)

    def run(async_):
        m = pf.FireModel(H, W, pf.PF_DISCRETE, realisations=3, seed=11)
        set_landscape(m, land, *winds[0])
        for e, (V, th) in enumerate(winds[1:], start=1):
            if async_:
                m.set_wind_async(_host(V, True), _host(th, True), e * EPOCH)
            else:
                m.set_wind(cuda(V), cuda(th), e * EPOCH)
        m.set_params(**PRM)
        out = torch.empty((3, H, W), dtype=torch.uint8, device="cuda")
        pf.pf_forward(m.h, cuda(np.broadcast_to(S0, (3, H, W))), T, out)
        m.wait()
        return out.cpu().numpy()

    assert np.array_equal(run(True), run(False))


def test_async_calm_epoch_and_order_check(pf):
    land, winds, S0, y = _inputs(5)
    m = pf.FireModel(H, W, pf.PF_DIFF)
    set_landscape(m, land, *winds[0])
    m.set_wind_async(None, None, EPOCH)  # calm from step EPOCH on
    with pytest.raises(pf.PFireError) as ei:
        m.set_wind_async(_host(winds[1][0], True), _host(winds[1][1], True), EPOCH)
    assert ei.value.code == -1  # PF_EINVAL, nothing queued
    m.set_params(**PRM)
    got = _run(pf, m, S0, y, backward=False)
    r = pf.FireModel(H, W, pf.PF_DIFF)
    set_landscape(r, land, *winds[0])
    r.set_wind(None, None, EPOCH)
    r.set_params(**PRM)
    _same(got, _run(pf, r, S0, y, backward=False))


def test_invalid_uploaded_values_reported_by_wait(pf):
    land, winds, S0, y = _inputs(6)
    m = pf.FireModel(H, W, pf.PF_DIFF)
    set_landscape(m, land, *winds[0])
    V = winds[1][0].copy()
    V[17, 23] = np.nan
    th = winds[1][1].copy()
    th[3, 4] = np.inf
    m.set_wind_async(_host(V, True), _host(th, True), EPOCH)
    with pytest.raises(pf.PFireError) as ei:
        m.wait()
    assert ei.value.code == -1 and "V_w and theta_w" in str(ei.value)
    m.wait()  # reported once
    # the context stays usable: replace the epochs and run
    set_landscape(m, land, *winds[0])
    for e, (Vc, thc) in enumerate(winds[1:], start=1):
        m.set_wind_async(_host(Vc, True), _host(thc, True), e * EPOCH)
    m.set_params(**PRM)
    _same(_run(pf, m, S0, y), _run(pf, _sync_model(pf, land, winds), S0, y))
