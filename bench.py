"""Throughput benchmark of libpfire on one GB300 (or N replicas under torchrun).

Workload (the 8192 x 8192 large-scale configuration): 67M-cell grid, l = 30 m, T = 2000
steps, differentiable (continuous-state, FP32) form, per-cell wind resampled every 100
steps (20 epochs), one ignited centre cell plus 4 random ones, BCE of the final burn
probability against a synthetic target, forward + adjoint with checkpointing, FP64
parameter-gradient reduction. One bench step = pf_forward + pf_loss_bce + pf_backward.

metric: cell-updates/s of forward + adjoint (H * W * T per step, every cell counted).
Also reported: forward-only cell-updates/s, the plain one-launch-per-step kernels as
the comparator, the roofline of the dominant kernel, the oracle on the host cores,
clocks during the timed region, and the end-to-end rate through the C ABI with host
buffers (inputs copied in and gradients copied out inside the timed region).

--impl reference times the FP64 CPU oracle (the reference arm: there is no reference
implementation to install) on a bounded crop of the same workload.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import statistics
import subprocess
import threading
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402

H = W = 8192
T = 2000
EPOCH_STEPS = 100
T_PROBE = 400   # forward steps of the autotuner's launch search
PREP_T = 500    # forward steps of the prep-variant comparison
FIELD_SEED = 5
PHILOX_SEED = 5
PARAMS = dict(p_h=0.58, c1=0.045, c2=0.131, a=0.078, p_continue=0.3, l=30.0)
HIDDEN = dict(p_h=0.5, c1=0.05, c2=0.12, a=0.08)
METRIC = "cell-updates/s fwd+adjoint (8192^2 diff form, T=2000)"
WORKLOAD = "8192x8192 differentiable fwd+adjoint, T=2000, wind resampled every 100 steps"
B_FWD, B_ADJ = 16, 24  # algorithmic bytes per cell-step: (a, b) in + out; state, lambda in, lambda out
# a frozen tile's region is constant over its adjoint launch: per cell and launch it reads
# q (32 B), the state once (8 B) and lambda (8 B), and writes lambda (8 B) and sigma (1 B)
B_FROZEN_LAUNCH = 57
B_DISC = 2  # discrete: the uint8 state in + out


# DRAM traffic of the blocked kernels measured by ncu over every launch of one timed step
# of the default workload (dram__bytes_read.sum + dram__bytes_write.sum, summed; the
# capture is summarised under profiles/), per cell-step the kernel computed.
# A figure is used only while the kernel's sources hash to the value it was taken on.
NCU_TRAFFIC = {
    # DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) per computed cell-step
    # over the timed step's launches of a 2048^2, T = 300, K = 21 run (the capture is sized
    # to end by itself), with a hash of the kernel's sources: null once they change
    "adjoint_blocked": {"files": ['kernels_adjoint_blocked.cu', 'common.cuh', 'tma.cuh', 'tmem.cuh'],
                        "sha256_16": "8984b15a96968041", "bytes_per_computed_cell_step": 23.43},
    "adjoint_frozen": {"files": ['kernels_adjoint_blocked.cu', 'common.cuh', 'tma.cuh', 'tmem.cuh'],
                       "sha256_16": "8984b15a96968041", "bytes_per_computed_cell_step": 12.68},
    "diff_blocked": {"files": ['kernels_diff_blocked.cu', 'common.cuh', 'tma.cuh', 'prep_math.cuh'],
                     "sha256_16": "6600c1b851d2f94d", "bytes_per_computed_cell_step": 12.87},
}


def ncu_traffic(kind):
    """Measured DRAM bytes per computed cell-step of a kernel kind, or None when the
    kernel has changed since the counters were taken."""
    import hashlib
    e = NCU_TRAFFIC.get(kind)
    if e is None:
        return None
    h = hashlib.sha256()
    try:
        for f in e["files"]:
            with open(os.path.join(ROOT, "paper_2502_18738_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return e["bytes_per_computed_cell_step"] if h.hexdigest()[:16] == e["sha256_16"] else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_inputs(H, W, T, seed):
    land = syn.make_landscape(H, W, seed)
    n_ep = (T + EPOCH_STEPS - 1) // EPOCH_STEPS
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        winds = list(ex.map(lambda e: syn.smooth_wind(H, W, seed, e), range(n_ep)))
    ign = [(H // 2, W // 2)] + syn.random_ignitions(land, seed, 4, 4)
    S0 = syn.initial_state(land, ign)
    # synthetic observed burn map: a disc around the ignitions, the size of the fire
    # the hidden parameters reach (stands in for the oracle-generated target of the
    # small calibration case, which is too slow to produce at 67M cells)
    rr, cc = np.ogrid[:H, :W]
    y = np.zeros((H, W), np.float32)
    for (r, c) in ign:
        y[(rr - r) ** 2 + (cc - c) ** 2 < (0.35 * T) ** 2] = 1.0
    y *= land.burnable
    return land, winds, S0, y


class Clocks:
    """nvidia-smi sampling during the timed region, kept in memory (and written to
    `path` as CSV when one is given)."""

    def __init__(self, path=None):
        self.path = path
        self.p = None
        self.lines = []

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line)

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", os.environ.get("LOCAL_RANK", "0")],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi's start-up (NVML over every GPU of the node) is kept out of the
            # timed region: the region starts once the first sample has arrived
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0 and self.p.poll() is None:
                time.sleep(0.02)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            self.p.wait()
            self.t.join(timeout=5)
        if self.path:
            with open(self.path, "w") as f:
                f.writelines(self.lines)

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(land, winds, S0, y, T_s, crop):
    """Oracle fwd + BCE + adjoint on the top-left crop x crop of the workload for T_s
    steps (bounded CPU work). Returns (cell-updates/s, seconds, threads)."""
    import oracle as orc
    orc.build()
    sl = (slice(0, crop), slice(0, crop))
    l2 = syn.Landscape(land.E[sl].copy(), land.p_veg[sl].copy(), land.p_den[sl].copy(), land.burnable[sl].copy())
    w2 = [(V[sl].copy(), th[sl].copy()) for (V, th) in winds[:1]]
    S2 = S0[sl].copy()
    S2[crop // 2, crop // 2] = 2
    prm = orc.Params(**PARAMS)
    t0 = time.perf_counter()
    a, b, tape = orc.diff_forward(l2, w2, [0], prm, S2, T_s)
    _, g = orc.bce(a, y[sl])
    orc.diff_backward(l2, w2, [0], prm, S2, tape, g, np.zeros_like(g))
    dt = time.perf_counter() - t0
    return crop * crop * T_s / dt, dt, orc.num_threads()


def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the step time a multi-replica run reports)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def prep_variants(pf, m, S0, out, timed, T):
    """Forward ms of T steps with q materialised per wind epoch (prep 1) or recomputed
    inside the step kernels (prep 2), for the plain kernel and the blocked one at k = 4, 8."""
    res = {}
    for kernel, k in ((1, 1), (2, 4), (2, 8)):
        for prep in (1, 2):
            pf.pf_set_tuning(m.h, kernel=kernel, k=k, prep=prep)
            pf.pf_forward(m.h, S0, T, out)  # warm-up
            res[f"kernel{kernel}_k{k}_prep{prep}"] = timed(lambda: pf.pf_forward(m.h, S0, T, out), 1)
    return res


def discrete_ensemble(pf, torch, timed, seed=1, N=1024, R=64, T=1000):
    """The discrete forward ensemble (N^2 grid, R realisations in one context, smooth
    per-cell wind, T steps): temporal-blocked kernel against the plain per-step kernel
    on the same GPU, cell-updates/s (N^2 R T per run)."""
    land = syn.make_landscape(N, N, seed)
    V, th = syn.smooth_wind(N, N, seed, 0)
    S0 = np.broadcast_to(syn.initial_state(land, syn.random_ignitions(land, seed)), (R, N, N)).copy()
    c = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    m = pf.FireModel(N, N, pf.PF_DISCRETE, R, seed=seed)
    m.set_env(c(land.E), c(land.p_veg), c(land.p_den), c(V), c(th))
    m.set_params(**PARAMS)
    S0d = c(S0)
    out = {}
    for name, kern in (("blocked", 2), ("plain", 1)):
        m.set_tuning(kernel=kern)
        m.forward(S0d, 20)  # warm-up
        ms = timed(lambda: m.forward(S0d, T), 1)
        out[name] = N * N * R * T / (ms / 1000.0)
        if kern == 2:
            st = m.stats()  # the near-ties of the timed run (every step, every realisation)
    # one more blocked run with per-launch events: the blocked kernel's time and the
    # cell-steps it computed (tiles with nothing burning skip their steps)
    m.set_tuning(kernel=2, profile=1)
    pf.pf_profile_read(m.h, reset=True)
    m.forward(S0d, T)
    torch.cuda.synchronize()
    n_l, cs_l, t_l, sk_l = pf.pf_profile_read(m.h, reset=True)["discrete_blocked"]
    m.close()
    hbm, how = peaks()
    achieved = B_DISC * (cs_l - sk_l) / (t_l / 1000.0) / 1e9
    return {"config": f"{N}x{N}, R={R} realisations, T={T}, discrete uint8", "unit": "cell-updates/s",
            "blocked": out["blocked"], "plain": out["plain"], "speedup": out["blocked"] / out["plain"],
            "near_ties_ignite": st["near_ties_ignite"], "near_ties_continue": st["near_ties_continue"],
            "draws_checked": "every drawn cell of the timed blocked run",
            "roofline": {"kernel": "discrete_blocked", "bound": "hbm", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "peak_source": how,
                         "alg_bytes_per_cell_step": B_DISC, "launches": n_l, "ms": t_l,
                         "computed_cell_steps": cs_l - sk_l, "skipped_frac": sk_l / max(1, cs_l)}}


def batched_fires(pf, torch, timed, n_fires=256, seed=4):
    """Uneven fires (side log-uniform in [64, 2048], T uniform in [100, 1000], 1-5
    ignitions, half discrete / half differentiable, the latter with an adjoint) through
    one pf_batch_submit, against the same fires run one after another through per-fire
    contexts with the plain per-step kernels and with the default (blocked) ones;
    cell-updates/s over sum(side^2 T), the differentiable fires counted twice (forward
    and adjoint). The submission is also timed at several routing thresholds (jobs above
    it through contexts of their own, the rest through the persistent queue)."""
    rng = np.random.default_rng(seed)
    fires = []
    for i in range(n_fires):
        side = int(round(np.exp(rng.uniform(np.log(64), np.log(2048)))))
        T = int(rng.integers(100, 1001))
        land = syn.make_landscape(side, side, 100 + i)
        V, th = syn.smooth_wind(side, side, 100 + i, 0)
        S0 = syn.initial_state(land, syn.random_ignitions(land, 100 + i))
        fires.append((side, T, i % 2, land, V, th, S0))
    c = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    dev = [(side, T, form, c(land.E), c(land.p_veg), c(land.p_den), c(V), c(th), c(S0))
           for side, T, form, land, V, th, S0 in fires]
    # forward cell-steps of every fire plus the adjoint's of the differentiable ones
    cells = sum(side * side * T * (2 if form == 1 else 1) for side, T, form, *_ in fires)
    wts = [torch.full((side, side), 1e-6, dtype=torch.float32, device="cuda") if form == 1 else None
           for side, T, form, *_ in fires]
    jobs = [pf.make_job(S0, T, form=form, seed=seed, fire_id=i, E=E, p_veg=pv, p_den=pd, V_w=V, theta_w=th,
                        dL_da=wts[i], **PARAMS)[0] for i, (side, T, form, E, pv, pd, V, th, S0) in enumerate(dev)]
    pf.pf_batch_submit(jobs)  # warm-up
    ms_batch = timed(lambda: pf.pf_batch_submit(jobs), 1)  # the library's default routing
    bst = pf.pf_batch_last_stats()
    # the routing threshold: jobs of at least `cells` cells through contexts of their own
    routing = {}
    for name, cells_min in (("queue_only", 1 << 40), ("direct_from_2^20", 1 << 20), ("direct_from_2^18", 1 << 18),
                            ("direct_from_2^16", 1 << 16), ("all_direct", 0)):
        pf.pf_batch_set_direct_cells(cells_min)
        routing[name] = {"ms": timed(lambda: pf.pf_batch_submit(jobs), 1), **pf.pf_batch_last_stats()}
    pf.pf_batch_set_direct_cells(1 << 18)
    q_only = routing["queue_only"]

    def plain_all():
        for i, (side, T, form, E, pv, pd, V, th, S0) in enumerate(dev):
            m = pf.FireModel(side, side, form, 1, seed=seed)
            m.set_env(E, pv, pd, V, th)
            m.set_params(**PARAMS)
            m.set_tuning(kernel=1)
            m.forward(S0, T)
            if form == 1:
                m.backward(wts[i], None, per_cell=False)
            m.close()
    ms_plain = timed(plain_all, 1)

    def blocked_all():  # the same with the library's default (temporal-blocked) kernels
        for i, (side, T, form, E, pv, pd, V, th, S0) in enumerate(dev):
            m = pf.FireModel(side, side, form, 1, seed=seed)
            m.set_env(E, pv, pd, V, th)
            m.set_params(**PARAMS)
            m.forward(S0, T)
            if form == 1:
                m.backward(wts[i], None, per_cell=False)
            m.close()
    ms_blocked = timed(blocked_all, 1)
    # algorithmic bytes of every cell-step (2 B discrete, 16 B differentiable forward, 24 B
    # adjoint) over the whole submission's time: an effective fraction (skipped quiescent
    # regions count too, so it may exceed 1)
    alg = sum(side * side * T * (B_DISC if form == 0 else B_FWD + B_ADJ) for side, T, form, *_ in fires)
    hbm, how = peaks()
    return {"config": f"{n_fires} fires, side log-uniform [64, 2048], T uniform [100, 1000], "
                      "half discrete / half differentiable, forward + adjoint of the differentiable ones",
            "unit": "cell-updates/s",
            "cell_steps": cells, "batched": cells / (ms_batch / 1000.0), "plain_per_fire": cells / (ms_plain / 1000.0),
            "speedup": ms_plain / ms_batch, "ms_batched": ms_batch, "ms_plain_per_fire": ms_plain,
            "blocked_per_fire": cells / (ms_blocked / 1000.0), "ms_blocked_per_fire": ms_blocked,
            "frac_hbm_alg_effective": alg / (ms_batch / 1000.0) / 1e9 / hbm,
            "default_stats": bst, "routing_ms": {k: v["ms"] for k, v in routing.items()},
            # the persistent kernels' roofline from the run with every job in the queue
            "kernels_queue_only": q_only, "roofline": batch_roofline(q_only, hbm, how)}


def batch_roofline(bst, hbm, how):
    """Roofline of the batch's two persistent kernels on the cell-steps they computed
    (items with nothing to do are skipped and not counted): 2 B per discrete and 16 B per
    differentiable forward cell-step over the forward kernel's time, 24 B per adjoint
    cell-step over the adjoint kernel's; the dominant one (more device time) first."""
    out = []
    for kernel, b, ms in (("k_batch", B_DISC * bst["disc_cell_steps"] + B_FWD * bst["diff_cell_steps"],
                           bst["ms_forward"]),
                          ("k_batch_adj", B_ADJ * bst["adj_cell_steps"], bst["ms_adjoint"])):
        ach = b / (ms / 1000.0) / 1e9 if ms > 0 else 0.0
        out.append({"kernel": kernel, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "peak_source": how, "ms": ms, "alg_bytes": b})
    out.sort(key=lambda r: -r["ms"])
    return out


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on a bounded sample, rank 0 only."""
    if rank != 0:
        return
    crop, T_s = 1024, 60
    land, winds, S0, y = make_inputs(crop, crop, EPOCH_STEPS, FIELD_SEED)
    vals = []
    for i in range(args.warmup + args.steps):
        v, dt, thr = oracle_sample(land, winds, S0, y, T_s, crop)
        if i >= args.warmup:
            vals.append((v, dt))
    value = statistics.median(v for v, _ in vals)
    ms = 1000 * statistics.median(dt for _, dt in vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{crop}x{crop} crop, {T_s} steps, one wind epoch"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": thr, "kind": "oracle",
                             "sample": f"{crop}x{crop} crop of the workload, T={T_s} fwd+adjoint, FP64 C oracle"},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def adjoint_probe(kind, N=2048, T=14):
    """Cost of the blocked adjoint per computed cell-step on one kind of tile: "frozen"
    (a = 0.65, b = 0 on every burnable cell: nothing burns, every listed tile is frozen)
    or "live" (b > 0 everywhere: every cell takes the full path). T steps taped in one
    segment, so the recompute's flags mark the frozen tiles; the second backward is
    profiled. Returns a dict for the JSON line."""
    import torch
    import paper_2502_18738_gb300 as pf
    pf.build()
    land = syn.make_landscape(N, N, 3)
    burn = land.burnable != 0
    c = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    rng = np.random.default_rng(1)
    if kind == "frozen":
        a, b = np.full((N, N), 0.65, np.float32), np.zeros((N, N), np.float32)
    else:
        a = (0.3 + 0.2 * rng.random((N, N))).astype(np.float32)
        b = (0.05 + 0.1 * rng.random((N, N))).astype(np.float32)
    ab = c(np.stack([np.where(burn, a, 0), np.where(burn, b, 0)]).astype(np.float32))
    m = pf.FireModel(N, N, pf.PF_DIFF)
    m.set_env(c(land.E), c(land.p_veg), c(land.p_den), c(np.full((N, N), 3.0, np.float32)),
              c(np.zeros((N, N), np.float32)))
    m.set_params(**PARAMS)
    m.forward(c(np.where(burn, 1, 0).astype(np.uint8)), 0)  # the burnable mask
    w = torch.full((N, N), 1e-3, device="cuda")
    for prof in (0, 1):
        pf.pf_set_tuning(m.h, K=T, profile=prof)
        pf.pf_profile_read(m.h, reset=True)
        m.set_state(0, ab)
        m.advance(T)
        m.backward(w, None, per_cell=False)
        torch.cuda.synchronize()
    p = pf.pf_profile_read(m.h, reset=True)
    # a launch of the blocked adjoint: the live-tile kernel and the frozen-tile kernel
    n, cs, ms, sk = p["adjoint_blocked"]
    ms_f = p.get("adjoint_frozen", (0, 0, 0.0, 0))[2]
    return {"probe": "adjoint_" + kind, "grid": N, "steps": T, "launches": n, "computed_cell_steps": cs - sk,
            "frozen_cell_steps": p["adjoint_tiles"][3], "ms_live_kernel": ms, "ms_frozen_kernel": ms_f,
            "ps_per_computed_cell_step": (ms + ms_f) * 1e9 / max(1, cs - sk)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=H, help="grid side (default 8192, the workload)")
    ap.add_argument("--T", type=int, default=T)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the discrete-ensemble and batched-fires comparisons against the plain kernels")
    ap.add_argument("--K", type=int, default=0, help="checkpoint interval (0 = chosen by the library)")
    ap.add_argument("--clocks-csv", default=None,
                    help="also write the clock samples of the timed region to this CSV ({rank} is replaced)")
    ap.add_argument("--k", type=int, default=0, help="steps per blocked forward launch (0 = library default)")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (launch search and checkpoint-interval search)")
    ap.add_argument("--only", choices=["discrete", "batch"],
                    help="instead of the benchmark: only the discrete ensemble or the batched fires")
    ap.add_argument("--fires", type=int, default=256, help="fires of the batched workload (with --only batch)")
    ap.add_argument("--probe", choices=["frozen", "live"],
                    help="instead of the benchmark: the blocked adjoint's cost on one kind of tile")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.probe:
        print(json.dumps(adjoint_probe(args.probe)), flush=True)
        return 0
    if args.only:
        # one secondary workload alone (for profiling it): no workload line is printed
        import torch
        import paper_2502_18738_gb300 as pf
        pf.build()

        def timed1(fn, n):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(n):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / n
        res = (discrete_ensemble(pf, torch, timed1, T=args.T if args.T != T else 1000) if args.only == "discrete"
               else batched_fires(pf, torch, timed1, n_fires=args.fires))
        print(json.dumps({"only": args.only, **res}), flush=True)
        return 0

    import torch
    import paper_2502_18738_gb300 as pf
    from paper_2502_18738_gb300.ensemble import allreduce_param_grads

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    pf.build()
    Hs = Ws = args.size
    Ts = args.T
    land, winds, S0, y = make_inputs(Hs, Ws, Ts, FIELD_SEED + rank)
    c = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    dev = dict(E=c(land.E), pv=c(land.p_veg), pd=c(land.p_den), S0=c(S0), y=c(y),
               winds=[(c(V), c(th)) for V, th in winds])
    stream = torch.cuda.current_stream()

    def setup(model):
        model.set_env(dev["E"], dev["pv"], dev["pd"], *dev["winds"][0])
        for e, (V, th) in enumerate(dev["winds"][1:], start=1):
            model.set_wind(V, th, e * EPOCH_STEPS)
        model.set_params(**PARAMS)

    m = pf.FireModel(Hs, Ws, pf.PF_DIFF, seed=PHILOX_SEED + rank)
    setup(m)
    # the autotuner picks the launch configuration (kernel, k, materialised or recomputed
    # q) on a forward probe and then the checkpoint interval on forward + adjoint of the
    # workload itself; its answers are cached on disk, keyed by GPU, grid and T
    base = dict(K=args.K, k=args.k)
    tuning = {"source": "fixed by --k / --K" if (args.k or args.K) else "library defaults (--no-tune)"}
    if not args.no_tune and args.k == 0 and args.K == 0:
        t0 = time.time()
        chosen = m.autotune(dev["S0"], T_PROBE)
        t1 = time.time()
        Kc = m.autotune_ckpt(dev["S0"], Ts)
        t2 = time.time()
        base = dict(kernel=chosen["kernel"], k=chosen["k"], prep=chosen["prep"], tile_rows=chosen["tile_rows"], K=Kc)
        tuning = {"source": "pf_autotune + pf_autotune_ckpt", "T_probe": T_PROBE, "launch_search_s": t1 - t0,
                  "ckpt_search_s": t2 - t1, "chosen": dict(base)}
    pf.pf_set_tuning(m.h, **base)
    g_a = torch.empty((Hs, Ws), dtype=torch.float32, device="cuda")
    gpv = torch.empty_like(g_a)
    gpd = torch.empty_like(g_a)
    out = torch.empty((2, Hs, Ws), dtype=torch.float32, device="cuda")

    def step():
        pf.pf_forward(m.h, dev["S0"], Ts, out)
        pf.pf_loss_bce(out[0], dev["y"], g_a, want_loss=False)
        g4 = pf.pf_backward(m.h, g_a, None, gpv, gpd)
        if dist is not None:
            # the replicas form a shared-parameter ensemble: its gradient is the sum over
            # ranks (one FP64 all-reduce of 32 bytes, the path's only exchange)
            g4 = allreduce_param_grads(g4)
        return g4

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, n):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / n, dist, "cuda")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the timed steps run without the library's per-launch CUDA events (launches are
    # counted on the host either way); one more step with them gives the per-kernel times
    pf.pf_profile_read(m.h, reset=True)
    mem0 = pf.pf_memory_stats(m.h)
    with Clocks(args.clocks_csv.replace("{rank}", str(rank)) if args.clocks_csv else None) as clk:
        ms = timed(step, args.steps)
    counts = pf.pf_profile_read(m.h, reset=True)
    mem1 = pf.pf_memory_stats(m.h)
    gpu_launches = sum(v[0] for v in counts.values())
    pf.pf_set_tuning(m.h, **base, profile=1)
    step()
    torch.cuda.synchronize()
    prof = pf.pf_profile_read(m.h, reset=True)  # one profiled step
    memst = pf.pf_memory_stats(m.h)  # the gradient path's memory and the tape's use, after it
    # device allocations and frees the library made during the timed steps (0 when steady)
    memst["allocations_in_timed_steps"] = mem1["allocations"] - mem0["allocations"]
    memst["frees_in_timed_steps"] = mem1["frees"] - mem0["frees"]
    pf.pf_set_tuning(m.h, **base)
    tun = pf.pf_get_tuning(m.h)
    cells = Hs * Ws * Ts
    value = cells * world / (ms / 1000.0)
    # forward only
    ms_fwd = timed(lambda: pf.pf_forward(m.h, dev["S0"], Ts, out), max(1, args.steps))
    # plain one-launch-per-step comparator (forward)
    ms_fwd_plain = None
    if not args.no_plain:
        pf.pf_set_tuning(m.h, **{**base, "kernel": 1, "prep": 1, "K": tun["K"]})
        ms_fwd_plain = timed(lambda: pf.pf_forward(m.h, dev["S0"], Ts, out), 1)
        pf.pf_set_tuning(m.h, **base)

    # roofline of the dominant kernel (largest share of device time in the timed region):
    # algorithmic bytes = per-cell-step bytes x the cell-steps its launches computed.
    # Cell-steps of quiescent tiles, which the kernels skip, are not counted (no state
    # bytes move for them). The blocked adjoint runs its frozen tiles in a kernel of its
    # own: those cell-steps (counted by its pre-pass) are the frozen kernel's, the rest of
    # its computed ones the live kernel's.
    hbm, how = peaks()
    total_ms = sum(v[2] for v in prof.values())
    frozen_cs = prof.get("adjoint_tiles", (0, 0, 0.0, 0))[3]
    computed = {}
    for kname, (n_l, cs_l, t_l, sk_l) in prof.items():
        if n_l == 0 or t_l <= 0.0:
            continue
        if kname == "adjoint_frozen":
            # its own bytes: B_FROZEN_LAUNCH per cell over the launch's steps (T / launches)
            computed[kname] = (frozen_cs, B_FROZEN_LAUNCH * n_l / Ts)
        elif kname == "adjoint_blocked":
            computed[kname] = (cs_l - sk_l - (frozen_cs if prof.get("adjoint_frozen", (0,))[0] else 0), B_ADJ)
        elif kname in ("adjoint_step",):
            computed[kname] = (cs_l - sk_l, B_ADJ)
        elif kname in ("diff_step", "diff_blocked"):
            computed[kname] = (cs_l - sk_l, B_FWD)

    def roofline_of(kname):
        n_l, cs_l, t_l, sk_l = prof[kname]
        comp, alg = computed[kname]
        achieved = alg * comp / (t_l / 1000.0) / 1e9
        tb = ncu_traffic(kname)
        return {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": how,
                # measured DRAM bytes per launch (ncu on a small case, per computed cell-step,
                # x this run's computed cell-steps per launch); null if the kernel changed since
                "traffic": None if tb is None else tb * comp / n_l,
                "traffic_bytes_per_computed_cell_step": tb,
                # DRAM utilisation: the measured bytes per launch over the launch's time
                "dram_frac": None if tb is None else tb * comp / (t_l / 1000.0) / 1e9 / hbm,
                "launches": n_l, "ms_per_launch": t_l / n_l, "cell_steps_per_launch": comp / n_l,
                "skipped_frac": None if kname == "adjoint_frozen" else sk_l / max(1, cs_l),
                "alg_bytes_per_cell_step": alg, "share": t_l / max(1e-9, total_ms)}

    kind = max(computed, key=lambda k: prof[k][2])
    roof = roofline_of(kind)
    roof["others"] = [roofline_of(k) for k in sorted(computed, key=lambda k: -prof[k][2]) if k != kind]
    if "adjoint_frozen" in computed and "adjoint_blocked" in computed:
        # the blocked adjoint as a whole (both kernels of each launch)
        comp_adj = computed["adjoint_blocked"][0] + frozen_cs
        t_adj = prof["adjoint_blocked"][2] + prof["adjoint_frozen"][2]
        # frac: the adjoint's 24 B per computed cell-step; frac_own_bytes: each kernel's
        # own bytes (a frozen tile reads its state once a launch, not once a step)
        own = computed["adjoint_blocked"][0] * B_ADJ + frozen_cs * computed["adjoint_frozen"][1]
        roof["adjoint_both_kernels"] = {"achieved": B_ADJ * comp_adj / (t_adj / 1000.0) / 1e9,
                                        "frac": B_ADJ * comp_adj / (t_adj / 1000.0) / 1e9 / hbm, "ms": t_adj,
                                        "frac_own_bytes": own / (t_adj / 1000.0) / 1e9 / hbm}

    # end to end through the C ABI with host buffers: inputs H2D, gradients D2H each step
    e2e = None
    if not args.no_e2e:
        hp = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        host = dict(E=hp(land.E), pv=hp(land.p_veg), pd=hp(land.p_den), S0=hp(S0), y=hp(y),
                    winds=[(hp(V), hp(th)) for V, th in winds])
        hgpv = torch.empty((Hs, Ws), dtype=torch.float32).pin_memory()
        hgpd = torch.empty_like(hgpv)
        hout = torch.empty((2, Hs, Ws), dtype=torch.float32).pin_memory()
        keys = ["E", "pv", "pd", "S0", "y"]
        h2d = sum(host[k].numel() * host[k].element_size() for k in keys)
        h2d += sum(V.numel() * 4 + th.numel() * 4 for V, th in host["winds"])
        d2h = hgpv.numel() * 4 * 2 + hout.numel() * 4 + 4 * 8
        # every input of a step lands in one of two device staging sets: a step's inputs
        # are copied in on a side stream while the previous step's adjoint runs (the
        # first step's before its forward, with its later wind epochs streamed by the
        # library from the pinned host buffers: pf_set_wind_async). Every copy of every
        # step is inside the timed region.
        stage = [dict({k: torch.empty_like(host[k], device="cuda") for k in keys},
                      winds=[(torch.empty_like(V, device="cuda"), torch.empty_like(th, device="cuda"))
                             for V, th in host["winds"]]) for _ in range(2)]
        side = torch.cuda.Stream()
        ev_in = [torch.cuda.Event(), torch.cuda.Event()]
        ev_out = torch.cuda.Event()

        def upload(st, winds_from=0):
            for k in keys:
                st[k].copy_(host[k], non_blocking=True)
            for (dV, dth), (V, th) in list(zip(st["winds"], host["winds"]))[winds_from:]:
                dV.copy_(V, non_blocking=True)
                dth.copy_(th, non_blocking=True)

        def e2e_run(n):
            for i in range(n):
                st = stage[i % 2]
                if i == 0:
                    upload(st, winds_from=len(host["winds"]))
                    st["winds"][0][0].copy_(host["winds"][0][0], non_blocking=True)
                    st["winds"][0][1].copy_(host["winds"][0][1], non_blocking=True)
                    m.set_env(st["E"], st["pv"], st["pd"], *st["winds"][0])
                    for e, (V, th) in enumerate(host["winds"][1:], start=1):
                        pf.pf_set_wind_async(m.h, Hs, Ws, V, th, e * EPOCH_STEPS)  # pinned host buffers
                else:
                    stream.wait_event(ev_in[i % 2])
                    m.set_env(st["E"], st["pv"], st["pd"], *st["winds"][0])
                    for e, (V, th) in enumerate(st["winds"][1:], start=1):
                        pf.pf_set_wind_async(m.h, Hs, Ws, V, th, e * EPOCH_STEPS)
                m.set_params(**PARAMS)
                pf.pf_forward(m.h, st["S0"], Ts, out)
                side.wait_stream(stream)  # out is final; the other staging set is free
                with torch.cuda.stream(side):
                    hout.copy_(out, non_blocking=True)
                    ev_out.record(side)
                    if i + 1 < n:
                        upload(stage[(i + 1) % 2])
                        ev_in[(i + 1) % 2].record(side)
                pf.pf_loss_bce(out[0], st["y"], g_a, want_loss=False)
                pf.pf_backward(m.h, g_a, None, gpv, gpd)
                hgpv.copy_(gpv, non_blocking=True)
                hgpd.copy_(gpd, non_blocking=True)
                stream.wait_event(ev_out)

        n_e2e = max(1, args.steps)
        e2e_run(1)  # warm-up: the staging buffers are new, the library adapts its memory to them
        ms_e2e = timed(lambda: e2e_run(n_e2e), 1) / n_e2e
        e2e = {"value": cells * world / (ms_e2e / 1000.0), "unit": "cell-updates/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e}
        del stage, host

    extras = {}
    if not args.no_extras:
        extras["prep_variants"] = {f"{Hs}x{Ws}": prep_variants(pf, m, dev["S0"], out, timed, PREP_T)}
        pf.pf_set_tuning(m.h, **base)

    # the comparisons below need their own memory (the batch's adjoint keeps every state
    # of its differentiable fires): release the workload's model and buffers first
    m.close()
    del dev, out, g_a, gpv, gpd
    torch.cuda.empty_cache()

    if not args.no_extras:
        land_s, winds_s, S0_s, _ = make_inputs(1024, 1024, PREP_T, FIELD_SEED + 7 + rank)
        ms_ = pf.FireModel(1024, 1024, pf.PF_DIFF, seed=PHILOX_SEED + rank)
        ms_.set_env(c(land_s.E), c(land_s.p_veg), c(land_s.p_den), *[c(x) for x in winds_s[0]])
        keep = [(c(V), c(th)) for V, th in winds_s[1:]]
        for e, (V, th) in enumerate(keep, start=1):
            ms_.set_wind(V, th, e * EPOCH_STEPS)
        ms_.set_params(**PARAMS)
        out_s = torch.empty((2, 1024, 1024), dtype=torch.float32, device="cuda")
        extras["prep_variants"]["1024x1024"] = prep_variants(pf, ms_, c(S0_s), out_s, timed, PREP_T)
        ms_.close()
        del keep, out_s
        extras["prep_variants"]["note"] = (f"forward only, T={PREP_T} from the workload's ignition, ms per "
                                           "forward; prep 1 = q materialised per wind epoch (its prep "
                                           "launches included), 2 = q recomputed inside the step kernels")
        extras["discrete_ensemble"] = discrete_ensemble(pf, torch, timed)
        extras["batched_fires"] = batched_fires(pf, torch, timed)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, dt, thr = oracle_sample(land, winds, S0, y, 60, 1024)
        cpu = {"value": v, "unit": "cell-updates/s", "cores": thr, "kind": "oracle", "seconds": dt,
               "sample": "1024x1024 top-left crop of the workload, T=60 fwd+adjoint, FP64 C oracle"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if (Hs == H and Ts == T) else f"{Hs}x{Ws} diff fwd+adjoint T={Ts}",
                           "H": Hs, "W": Ws, "T": Ts, "wind_epochs": len(winds),
                           "checkpoint_K": tun["K"], "kernel": tun["kernel"], "k": tun["k"], "prep": tun["prep"],
                           "tuning": tuning,
                           "gradient_memory_gb": {k: (v / 1e9 if k.endswith("_bytes") else v) for k, v in memst.items()},
                           "l2": "inputs larger than L2 (state 0.5 GB, q 2.1 GB per epoch)"},
                "fwd": {"value": cells * world / (ms_fwd / 1000.0), "unit": "cell-updates/s", "ms": ms_fwd,
                        "frac_hbm_alg_effective": B_FWD * cells / (ms_fwd / 1000.0) / 1e9 / hbm},
                "fwd_plain": None if ms_fwd_plain is None else
                {"value": cells / (ms_fwd_plain / 1000.0), "unit": "cell-updates/s", "ms": ms_fwd_plain},
                # effective fraction: every cell counted, quiescent tiles included
                "fwd_adj_frac_hbm_alg_effective": (B_FWD + B_ADJ) * cells / (ms / 1000.0) / 1e9 / hbm,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": gpu_launches,
                # one profiled step (library CUDA events around every launch)
                "kernels": {k: {"launches": n, "cell_steps": cs, "skipped_cell_steps": sk, "ms": t}
                            for k, (n, cs, t, sk) in prof.items() if n},
                "clocks": clk.summary(), **extras}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
