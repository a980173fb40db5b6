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
