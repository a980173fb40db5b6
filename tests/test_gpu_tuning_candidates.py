"""Every launch configuration the autotuner can pick gives the same result, bit for bit,
and that result is the oracle's: the kernel (plain / temporal-blocked), the steps per
launch k, where q comes from (materialised per wind epoch, or recomputed inside the step
kernels from the fields: Eq. 1-5 in the same arithmetic) and the discrete tile height.
The discrete form is compared exactly (the same counter-based draws, Sec. 2.2), the
differentiable one within the trajectory tolerance. Also the on-disk tuning cache and
the checkpoint-interval search."""
import os

import numpy as np
import pytest

import synthetic as syn
from tests._util import PRM, cuda, set_landscape

pytestmark = pytest.mark.gpu

RUN_RTOL, RUN_ATOL = 1e-4, 1e-6

# k = 16 is above the discrete blocked kernel's limit (12): it runs at 12
CANDS_DISCRETE = [(1, 1, p, 0) for p in (1, 2)] + [
    (2, k, p, rows) for p in (1, 2) for k in (4, 8, 12, 16) for rows in (32, 64, 128)]
CANDS_DIFF = [(1, 1, p, 0) for p in (1, 2)] + [(2, k, p, 0) for p in (1, 2) for k in (2, 4, 6, 8)]


@pytest.fixture(scope="module")
def pf():
    import paper_2502_18738_gb300 as pf
    pf.build()
    pf.load()
    return pf


def _scene(H, W, seed):
    land = syn.make_landscape(H, W, seed)
    V0, th0 = syn.smooth_wind(H, W, seed, 0, sigma=8.0)
    V1, th1 = syn.smooth_wind(H, W, seed, 1, sigma=8.0)
    return land, (V0, th0), (V1, th1)


def test_discrete_candidates_agree_with_each_other_and_the_oracle(pf, orc):
    # 150 x 300: ragged against 128-column tiles and every tile height; a wind epoch
    # that starts at step 17, inside blocked launches of every k
    H, W, R, T, t1 = 150, 300, 3, 40, 17
    land, w0, w1 = _scene(H, W, 31)
    S0 = np.stack([syn.initial_state(land, [(75, 150), (20 + 9 * r, 40)]) for r in range(R)])
    m = pf.FireModel(H, W, pf.PF_DISCRETE, R, seed=5)
    set_landscape(m, land, *w0)
    m.set_wind(cuda(w1[0]), cuda(w1[1]), t1)
    m.set_params(**PRM)
    prm = orc.Params(**PRM)
    q0 = orc.prep(H, W, land.E, land.p_veg, land.p_den, *w0, prm)
    q1 = orc.prep(H, W, land.E, land.p_veg, land.p_den, *w1, prm)
    ref = orc.forward_discrete(S0, q0, prm.p_continue, seed=5, T=t1)
    ref = orc.forward_discrete(ref, q1, prm.p_continue, seed=5, T=T - t1, step0=t1)
    assert (ref == 3).sum() + (ref == 2).sum() > 300  # the fires spread
    for kernel, k, prep, rows in CANDS_DISCRETE:
        m.set_tuning(kernel=kernel, k=k, prep=prep, tile_rows=rows)
        t = pf.pf_get_tuning(m.h)
        assert (t["kernel"], t["prep"]) == (kernel, prep)
        assert t["tile_rows"] == (rows or 64)
        out = m.forward(cuda(S0), T).cpu().numpy()
        assert np.array_equal(out, ref), (kernel, k, prep, rows, int((out != ref).sum()))


def test_diff_candidates_agree_with_each_other_and_the_oracle(pf, orc):
    H, W, T, t1 = 150, 260, 40, 17
    land, w0, w1 = _scene(H, W, 32)
    S0 = syn.initial_state(land, [(75, 130), (30, 40)])
    m = pf.FireModel(H, W, pf.PF_DIFF)
    set_landscape(m, land, *w0)
    m.set_wind(cuda(w1[0]), cuda(w1[1]), t1)
    m.set_params(**PRM)
    a, b, _ = orc.diff_forward(land, [w0, w1], [0, t1], orc.Params(**PRM), S0, T, keep_states=False)
    first = None
    for kernel, k, prep, rows in CANDS_DIFF:
        m.set_tuning(kernel=kernel, k=k, prep=prep, tile_rows=rows)
        out = m.forward(cuda(S0), T).cpu().numpy()
        if first is None:
            first = out
            for got, want in ((out[0], a), (out[1], b)):
                err = np.abs(got - want)
                assert (err <= RUN_RTOL * np.abs(want) + RUN_ATOL).all(), float(err.max())
            assert (a > 0.5).sum() > 200  # the fires spread
        else:
            assert np.array_equal(out, first), (kernel, k, prep, int((out != first).sum()))
        # the adjoint of a run whose forward recomputed q materialises its own
        if prep == 2 and kernel == 2 and k == 8:
            import torch
            g4, _, _ = m.backward(torch.full((H, W), 1e-3, device="cuda"), None)
            m.set_tuning(kernel=kernel, k=k, prep=1)
            m.forward(cuda(S0), T)
            g4m, _, _ = m.backward(torch.full((H, W), 1e-3, device="cuda"), None)
            assert np.array_equal(np.asarray(g4), np.asarray(g4m))


def test_tuning_values_are_validated(pf):
    m = pf.FireModel(16, 16, pf.PF_DISCRETE, 1)
    for kw in (dict(prep=3), dict(prep=-1), dict(tile_rows=48), dict(tile_rows=256)):
        with pytest.raises(pf.PFireError) as e:
            m.set_tuning(**kw)
        assert e.value.code == pf.PF_EINVAL


def test_autotune_cache_round_trip(pf, tmp_path):
    H, W = 120, 140
    land, w0, _ = _scene(H, W, 33)
    S0 = syn.initial_state(land, [(60, 70)])
    path = tmp_path / "tune.tsv"
    old = os.environ.get("PF_TUNE_CACHE")
    os.environ["PF_TUNE_CACHE"] = str(path)
    try:
        m = pf.FireModel(H, W, pf.PF_DISCRETE, 2, seed=3)
        set_landscape(m, land, *w0)
        m.set_params(**PRM)
        S = cuda(np.stack([S0, S0]))
        t = m.autotune(S, 12)
        lines = path.read_text().splitlines()
        assert len(lines) == 1
        key, val = lines[0].split("\t")
        assert "|launch|discrete|H=120|W=140|R=2|T=12" in key
        assert [int(v) for v in val.split()][:4] == [t["kernel"], t["k"], t["prep"], t["tile_rows"]]
        # a second search with the same key reads the file and appends nothing
        assert m.autotune(S, 12) == t
        assert len(path.read_text().splitlines()) == 1
        # the newest line of a key wins: a hand-written entry is applied as it stands
        with open(path, "a") as f:
            f.write(f"{key}\t1 1 2 0 0\n")
        t2 = m.autotune(S, 12)
        assert (t2["kernel"], t2["prep"]) == (1, 2)
        # another key (T_probe) searches again
        m.autotune(S, 13)
        assert len(path.read_text().splitlines()) == 3
        # "off" disables the file
        os.environ["PF_TUNE_CACHE"] = "off"
        m.autotune(S, 14)
        assert len(path.read_text().splitlines()) == 3
    finally:
        if old is None:
            os.environ.pop("PF_TUNE_CACHE", None)
        else:
            os.environ["PF_TUNE_CACHE"] = old


def test_checkpoint_interval_search(pf):
    import torch
    H, W, T = 96, 110, 30
    land, w0, _ = _scene(H, W, 34)
    S0 = cuda(syn.initial_state(land, [(48, 55)]))
    m = pf.FireModel(H, W, pf.PF_DIFF)
    set_landscape(m, land, *w0)
    m.set_params(**PRM)
    g = torch.full((H, W), 1e-3, device="cuda")
    m.forward(S0, T)
    ref, _, _ = m.backward(g, None)
    K = m.autotune_ckpt(S0, T)
    assert K >= 0
    assert pf.pf_get_tuning(m.h)["K"] >= 1
    with pytest.raises(pf.PFireError) as e:  # the probes left no tape
        m.backward(g, None)
    assert e.value.code == pf.PF_ESTATE
    m.forward(S0, T)
    got, _, _ = m.backward(g, None)
    assert np.array_equal(np.asarray(got), np.asarray(ref))
    d = pf.FireModel(16, 16, pf.PF_DISCRETE, 1)
    with pytest.raises(pf.PFireError) as e:
        d.autotune_ckpt(cuda(np.ones((16, 16), np.uint8)), 4)
    assert e.value.code == pf.PF_ESTATE
