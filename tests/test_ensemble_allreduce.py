"""A shared-parameter ensemble split over two ranks (gloo on CPU): each rank takes the
gradient of its own fire (the FP64 oracle stands in for a rank's GPU here) and the
parameter gradients are summed with one FP64 all-reduce; every rank then holds exactly
the sum a single process computes over both fires."""
import os
import socket

import numpy as np
import pytest

import synthetic as syn
from tests._util import PRM


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fire_gradient(r):
    import oracle as orc
    H, W, T = 40, 48, 18
    land = syn.make_landscape(H, W, 60 + r)
    V, th = syn.smooth_wind(H, W, 60 + r, 0, sigma=6.0)
    S0 = syn.initial_state(land, [(10 + 7 * r, 20 + 5 * r)])
    prm = orc.Params(**PRM)
    a, b, tape = orc.diff_forward(land, [(V, th)], [0], prm, S0, T)
    g4, _, _ = orc.diff_backward(land, [(V, th)], [0], prm, S0, tape, np.ones((H, W)) / (H * W), np.zeros((H, W)))
    return [float(v) for v in g4]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    from paper_2502_18738_gb300.ensemble import allreduce_param_grads
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, allreduce_param_grads(_fire_gradient(rank))))
    finally:
        dist.destroy_process_group()


def test_parameter_gradients_summed_over_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    g0, g1 = _fire_gradient(0), _fire_gradient(1)
    want = [x + y for x, y in zip(g0, g1)]
    assert got[0] == want and got[1] == want
    assert all(abs(x) > 0 for x in g0) and all(abs(x) > 0 for x in g1)
