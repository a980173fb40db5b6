"""Failure handling that needs no GPU fault: an injected host-side allocation failure
(PF_FAULT_ALLOC=n fails the n-th device allocation of the process) surfaces as
PF_ENOMEM with a message, and the process keeps working afterwards."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, torch
sys.path.insert(0, {root!r})
import paper_2502_18738_gb300 as pf
pf.load()
try:
    m = pf.FireModel(64, 64, pf.PF_DIFF, 1)
    print("created")
except pf.PFireError as e:
    print("error", e.code, "cudaMalloc" in str(e) or "injected" in str(e))
m = pf.FireModel(32, 32, pf.PF_DIFF, 1)   # allocations after the injected one succeed
S = torch.ones((32, 32), dtype=torch.uint8, device="cuda"); S[16, 16] = 2
out = m.forward(S, 5)
print("after", float(out[0].sum()) > 1.0)
"""


@pytest.mark.parametrize("n", [1, 3])
def test_injected_allocation_failure(n):
    import paper_2502_18738_gb300 as pf
    pf.build()
    env = dict(os.environ, PF_FAULT_ALLOC=str(n))
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.split("\n")
    assert f"error {pf.PF_ENOMEM} True" in lines
    assert "after True" in lines


@pytest.mark.parametrize("form", [0, 1])
def test_tma_wait_timeout_reports_and_library_stays_usable(form, monkeypatch):
    """A test hook makes the temporal-blocked kernels arm their TMA barriers without
    issuing the copies (no copy is ever in flight), and bounds each wait to a few
    thousand polls: the waits run out, the kernels record the timeout and return (the
    adjoint after freeing its tensor memory), the next synchronous call reports
    PF_ETIMEOUT, and the same context then computes what a fresh one computes."""
    import numpy as np
    import torch
    import paper_2502_18738_gb300 as pf
    import synthetic as syn
    from tests._util import PRM, cuda, set_landscape
    pf.build()
    H, W, T = 160, 200, 12
    land = syn.make_landscape(H, W, 31)
    V, th = syn.smooth_wind(H, W, 31, 0, sigma=8.0)
    S0 = syn.initial_state(land, [(80, 100)])
    R = 2 if form == 0 else 1
    S_in = cuda(np.stack([S0] * R)) if form == 0 else cuda(S0)

    def model():
        m = pf.FireModel(H, W, form, R, seed=3)
        set_landscape(m, land, V, th)
        m.set_params(**PRM)
        m.set_tuning(kernel=2, k=4, K=1)
        return m

    m = model()
    monkeypatch.setenv("PF_TMA_TEST_WITHHOLD", "1")
    monkeypatch.setenv("PF_TMA_SPIN_LIMIT", "4096")
    m.forward(S_in, T)
    with pytest.raises(pf.PFireError) as e:
        m.wait()
    assert e.value.code == pf.PF_ETIMEOUT
    monkeypatch.delenv("PF_TMA_TEST_WITHHOLD")
    monkeypatch.delenv("PF_TMA_SPIN_LIMIT")
    out = m.forward(S_in, T).cpu().numpy()
    ref_m = model()
    ref = ref_m.forward(S_in, T).cpu().numpy()
    assert np.array_equal(out, ref)
    if form == 1:
        # the adjoint's waits: its kernel holds tensor memory, which it must give back
        w = torch.full((H, W), 1e-3, device="cuda")
        monkeypatch.setenv("PF_TMA_TEST_WITHHOLD", "1")
        monkeypatch.setenv("PF_TMA_SPIN_LIMIT", "4096")
        with pytest.raises(pf.PFireError) as e:
            m.backward(w, None, per_cell=False)
        assert e.value.code == pf.PF_ETIMEOUT
        monkeypatch.delenv("PF_TMA_TEST_WITHHOLD")
        monkeypatch.delenv("PF_TMA_SPIN_LIMIT")
        g, _, _ = m.backward(w, None, per_cell=False)
        g_ref, _, _ = ref_m.backward(w, None, per_cell=False)
        assert g == g_ref
    ref_m.close()
    m.close()
