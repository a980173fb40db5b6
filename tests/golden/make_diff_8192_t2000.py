"""Writes diff_8192_t2000.txt: FP64 oracle values of the 8192 x 8192, T = 2000 workload
(five fires, per-cell winds resampled every 100 steps, differentiable form) for the
full-size parity test. Calls only oracle/ and synthetic/; takes about 1.5 h on 8 cores:

    python tests/golden/make_diff_8192_t2000.py

Stored: input fingerprints (sums of the fields, to detect a change of the generators),
a_T and b_T at 2000 sampled cells (1500 where a_T > 1e-12, 500 anywhere), global sums,
a mean-square loss against a target disc and that loss at p_h -/+ h (a central finite
difference of the forward).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
import synthetic as syn  # noqa: E402

N, T, SEED = 8192, 2000, 5
PRM = dict(p_h=0.58, c1=0.045, c2=0.131, a=0.078, p_continue=0.3, l=30.0)


def problem():
    land = syn.make_landscape(N, N, SEED)
    winds = [syn.smooth_wind(N, N, SEED, e) for e in range(T // 100)]
    ign = [(N // 2, N // 2)] + syn.random_ignitions(land, SEED, 4, 4)
    return land, winds, [100 * e for e in range(T // 100)], syn.initial_state(land, ign), ign


def target(S0):
    rr, cc = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    return ((np.hypot(rr - N / 2, cc - N / 2) < 0.3 * T) * (S0 != 0)).astype(np.float64)


def main():
    land, winds, starts, S0, ign = problem()
    base = orc.Params(**PRM)
    a, b, _ = orc.diff_forward(land, winds, starts, base, S0, T, keep_states=False)
    y = target(S0)
    loss = float(((a - y) ** 2).mean())
    h = 1e-3 * base.p_h
    fd = []
    for s in (-1, +1):
        prm = orc.Params(p_h=base.p_h + s * h, c1=base.c1, c2=base.c2, a=base.a, p_continue=base.p_continue,
                         l=base.l, exact=True)
        a2, _, _ = orc.diff_forward(land, winds, starts, prm, S0, T, keep_states=False)
        fd.append(float(((a2 - y) ** 2).mean()))
    rng = np.random.Generator(np.random.PCG64(2025))
    live = np.flatnonzero(a.reshape(-1) > 1e-12)
    pick = np.concatenate([rng.choice(live, 1500, replace=False), rng.choice(N * N, 500, replace=False)])
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "diff_8192_t2000.txt")
    with open(out, "w") as f:
        f.write("# FP64 oracle, 8192 x 8192, T = 2000, five fires, per-cell winds every 100 steps,\n")
        f.write("# parameters p_h=0.58 c1=0.045 c2=0.131 a=0.078 p_continue=0.3 l=30 (FP32 values);\n")
        f.write("# written by tests/golden/make_diff_8192_t2000.py (oracle/ and synthetic/ only)\n")
        f.write(f"fingerprint E_sum {float(land.E.astype(np.float64).sum())!r}\n")
        f.write(f"fingerprint V0_sum {float(winds[0][0].astype(np.float64).sum())!r}\n")
        f.write(f"fingerprint th19_sum {float(winds[-1][1].astype(np.float64).sum())!r}\n")
        f.write(f"fingerprint ignitions {' '.join(f'{r},{c}' for r, c in ign)}\n")
        f.write(f"sum_a {float(a.sum())!r}\n")
        f.write(f"sum_b {float(b.sum())!r}\n")
        f.write(f"n_a_half {int((a > 0.5).sum())}\n")
        f.write(f"loss {loss!r}\n")
        f.write(f"fd_p_h {h!r} {fd[0]!r} {fd[1]!r}\n")
        for i in pick:
            r, c = divmod(int(i), N)
            f.write(f"cell {r} {c} {float(a[r, c])!r} {float(b[r, c])!r}\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
