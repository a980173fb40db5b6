"""pf_loss_bce_noalloc, the loss entry point that allocates no device memory (for
callers whose device memory is owned by a fixed-budget allocator, or whose loops cannot
absorb cudaMalloc's synchronisation), against pf_loss_bce through the C ABI. Collected
last on purpose: a failure here leaves every other test already run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_loss_matches_the_allocating_entry_point_twice_in_a_row():
    import torch
    import paper_2502_18738_gb300 as pf
    pf.build()
    gen = torch.Generator(device="cuda").manual_seed(7)
    # first call at the size limit, second at a ragged smaller size: the second call
    # must not see the first call's partial sums left in the shared static array
    for n in (pf.PF_NOALLOC_BCE_MAX_N, 1_000_003):
        a = torch.rand(n, device="cuda", generator=gen)
        a[:: 97] = 0.0                         # exercise the clamp (no gradient there)
        a[1:: 89] = 1.0
        y = (torch.rand(n, device="cuda", generator=gen) < 0.3).float()
        g_ref = torch.empty_like(a)
        g_new = torch.full_like(a, float("nan"))
        loss_ref = pf.pf_loss_bce(a, y, g_ref)
        loss_new = pf.pf_loss_bce_noalloc(a, y, g_new)
        torch.cuda.synchronize()
        assert loss_new == pytest.approx(loss_ref, rel=1e-9)
        assert torch.equal(g_new, g_ref)
        assert np.isfinite(loss_new) and loss_new > 0


def test_noalloc_loss_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2502_18738_gb300 as pf
    pf.build()
    a = torch.full((16,), 0.5, device="cuda")
    y = torch.ones(16, device="cuda")
    with pytest.raises(pf.PFireError) as e:
        # rejected before any memory is touched, so the small buffers are never read
        pf.pf_loss_bce_noalloc(a, y, n=pf.PF_NOALLOC_BCE_MAX_N + 1)
    assert e.value.code == pf.PF_EINVAL
    assert "limit" in str(e.value)
