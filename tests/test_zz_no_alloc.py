"""pf_loss_bce_noalloc, the loss entry point that allocates no device memory (for
callers whose device memory is owned by a fixed-budget allocator, or whose loops cannot
absorb cudaMalloc's synchronisation), against pf_loss_bce through the C ABI. Collected
last on purpose: a failure here leaves every other test already run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(n, gen):
    import torch
    a = torch.rand(n, device="cuda", generator=gen)
    a[:: 97] = 0.0                         # exercise the clamp (no gradient there)
    a[1:: 89] = 1.0
    y = (torch.rand(n, device="cuda", generator=gen) < 0.3).float()
    return a, y


def test_noalloc_loss_matches_the_allocating_entry_point_twice_in_a_row():
    import torch
    import paper_2502_18738_gb300 as pf
    pf.build()
    gen = torch.Generator(device="cuda").manual_seed(7)
    # first call at the size limit, second at a ragged smaller size: the second call
    # must not see the first call's partial sums left in the shared static array
    for n in (pf.PF_NOALLOC_BCE_MAX_N, 1_000_003):
        a, y = _inputs(n, gen)
        g_ref = torch.empty_like(a)
        g_new = torch.full_like(a, float("nan"))
        loss_ref = pf.pf_loss_bce(a, y, g_ref)
        loss_new = pf.pf_loss_bce_noalloc(a, y, g_new)
        torch.cuda.synchronize()
        assert loss_new == pytest.approx(loss_ref, rel=1e-9)
        assert torch.equal(g_new, g_ref)
        assert np.isfinite(loss_new) and loss_new > 0


def test_noalloc_loss_allocates_nothing_on_a_side_stream():
    """After one warm-up call (which loads the library's module, and with it the static
    array), further calls leave the device's free memory unchanged; run on a stream of
    the caller's, they give the same result as pf_loss_bce."""
    import torch
    import paper_2502_18738_gb300 as pf
    pf.build()
    gen = torch.Generator(device="cuda").manual_seed(11)
    n = 3_000_017
    a, y = _inputs(n, gen)
    g_ref = torch.empty_like(a)
    g_new = torch.empty_like(a)
    loss_ref = pf.pf_loss_bce(a, y, g_ref)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    pf.pf_loss_bce_noalloc(a, y, g_new, stream=side)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        g_new.fill_(float("nan"))
        side.wait_stream(torch.cuda.current_stream())
        loss_new = pf.pf_loss_bce_noalloc(a, y, g_new, stream=side)
        torch.cuda.synchronize()
        assert loss_new == pytest.approx(loss_ref, rel=1e-9)
        assert torch.equal(g_new, g_ref)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_loss_rejects_sizes_beyond_its_scratch():
    """The buffers cover all of n, so the call stays in bounds even if the size check
    were ever lost: the test would then fail on the assertion, not on the device."""
    import torch
    import paper_2502_18738_gb300 as pf
    pf.build()
    n = pf.PF_NOALLOC_BCE_MAX_N + 1
    a = torch.full((n,), 0.5, device="cuda")
    y = torch.ones(n, device="cuda")
    g = torch.empty(n, device="cuda")
    with pytest.raises(pf.PFireError) as e:
        pf.pf_loss_bce_noalloc(a, y, g)
    assert e.value.code == pf.PF_EINVAL
    assert "limit" in str(e.value)
    del a, y, g
    # mismatched lengths are rejected by the binding before the call
    a = torch.full((16,), 0.5, device="cuda")
    with pytest.raises(ValueError):
        pf.pf_loss_bce_noalloc(a, torch.ones(15, device="cuda"))
