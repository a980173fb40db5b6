"""The 8192 x 8192, T = 2000 differentiable workload (five fires, per-cell winds resampled
every 100 steps) in the launch configuration bench.py times, against FP64 oracle values
stored in tests/golden/diff_8192_t2000.txt (written by make_diff_8192_t2000.py, which
calls only oracle/ and synthetic/): a_T and b_T at 2000 sampled cells (1e-4 |ref| +
1e-6), the global sums, a mean-square loss against a target disc, and the adjoint's
dL/dp_h against the oracle's central finite difference of that loss (1e-3)."""
import os

import numpy as np
import pytest

import synthetic as syn
from tests._util import PRM, cuda, set_landscape

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "diff_8192_t2000.txt")
N, T = 8192, 2000
RUN_RTOL, RUN_ATOL = 1e-4, 1e-6
GRAD_RTOL = 1e-3


def _golden():
    g = {"cells": []}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            if k == "cell":
                g["cells"].append((int(v[0]), int(v[1]), float(v[2]), float(v[3])))
            elif k == "fingerprint":
                g[v[0]] = v[1:]
            else:
                g[k] = [float(x) for x in v]
    return g


@pytest.fixture(scope="module")
def pf():
    import paper_2502_18738_gb300 as pf
    pf.build()
    pf.load()
    return pf


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="golden values not generated")
def test_8192_t2000_against_stored_oracle_values(pf):
    import torch
    g = _golden()
    land = syn.make_landscape(N, N, 5)
    winds = [syn.smooth_wind(N, N, 5, e) for e in range(T // 100)]
    ign = [(N // 2, N // 2)] + syn.random_ignitions(land, 5, 4, 4)
    # the generators still produce the inputs the values were computed from (sums in
    # FP64 of FP32 fields; a relative slack for the host's libm)
    assert " ".join(f"{r},{c}" for r, c in ign) == " ".join(g["ignitions"])
    assert float(land.E.astype(np.float64).sum()) == pytest.approx(float(g["E_sum"][0]), rel=1e-6)
    assert float(winds[0][0].astype(np.float64).sum()) == pytest.approx(float(g["V0_sum"][0]), rel=1e-6)
    assert float(winds[-1][1].astype(np.float64).sum()) == pytest.approx(float(g["th19_sum"][0]), rel=1e-6)
    S0 = syn.initial_state(land, ign)
    m = pf.FireModel(N, N, pf.PF_DIFF)
    set_landscape(m, land, *winds[0])
    dev_w = [(cuda(V), cuda(th)) for V, th in winds[1:]]
    for e, (V, th) in enumerate(dev_w, start=1):
        m.set_wind(V, th, 100 * e)
    m.set_params(**PRM)
    out = m.forward(cuda(S0), T)
    a, b = out[0], out[1]
    cells = np.array(g["cells"])
    r, c = cells[:, 0].astype(np.int64), cells[:, 1].astype(np.int64)
    idx = torch.from_numpy(r * N + c).cuda()
    ga = a.reshape(-1)[idx].double().cpu().numpy()
    gb = b.reshape(-1)[idx].double().cpu().numpy()
    for got, want in ((ga, cells[:, 2]), (gb, cells[:, 3])):
        err = np.abs(got - want)
        bad = err > RUN_RTOL * np.abs(want) + RUN_ATOL
        assert not bad.any(), (int(bad.sum()), float(err.max()))
    assert float(a.double().sum()) == pytest.approx(g["sum_a"][0], rel=1e-5)
    assert float(b.double().sum()) == pytest.approx(g["sum_b"][0], rel=1e-4, abs=1e-3)
    assert abs(int((a > 0.5).sum()) - int(g["n_a_half"][0])) <= 1e-4 * g["n_a_half"][0] + 10
    # the loss of the generator and its gradient through the adjoint
    rr = torch.arange(N, device="cuda", dtype=torch.float64)
    disc = torch.hypot(rr[:, None] - N / 2, rr[None, :] - N / 2) < 0.3 * T
    y = (disc & (cuda(S0) != 0)).double()
    diff = a.double() - y
    loss = float((diff * diff).mean())
    assert loss == pytest.approx(g["loss"][0], rel=1e-5)
    seed = (2.0 * diff / (N * N)).float()
    g4, _, _ = m.backward(seed, None)
    h, lo, hi = g["fd_p_h"]
    fd = (hi - lo) / (2 * h)
    assert g4[0] == pytest.approx(fd, rel=GRAD_RTOL)
